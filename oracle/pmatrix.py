"""Parametric H- and H^2-matrices: offline stage, online stage and MVM (§4, App. A.1, A.4).

Test infrastructure only (see ``oracle/__init__.py``).

Everything is float64 and explicit.  For every far-field block the oracle forms
L_b, H_b(theta), R_b and C_b(theta) = L_b H_b(theta) R_b^T as dense matrices
from their definitions (App. A.4, §4.2), the cluster basis U_sigma by
face-splitting (§3.3), the transfer matrices E_sigma' by Kronecker products
(§3.6.1), and for the H format S_b = U_sigma L_b and T_b = U_tau R_b directly
from their definitions (App. A.4).  It never uses a tensor-train chain to apply
C_b and it compresses every far block separately (no reuse across
translation-equivalent blocks, §5.2), which makes it slow and independent of
how the GPU path organises the same arithmetic.

Readings (where the paper is ambiguous or garbled):

* Transfer factor index order.  §3.6.1 prints [E_{s',k}]_{i,j} = ell_i^{s}(eta_j^{s'}),
  but the nestedness identity Gamma U_s = U_{s'} E_{s'} proved in App. A.3
  requires the row to be the child node and the column the parent polynomial:
  [E_{s',k}]_{j,i} = ell_i^{(B_s,k)}(eta_j^{(B_s',k)}).  That is used here.
* L_b is p_s^d x r_{b,d} (§4.2), not n_s x r (App. A.4 misprint).
* C_b = L_b H_b R_b^T (§4.2); the displayed "L_b H_b R_b" omits the transpose.
* App. A.4 Phase 3's undefined right face-splitting symbol is not needed:
  S_b and T_b are formed from their definitions.
* TT-SVD (Oseledets 2011, Alg. 1) replaces TT-cross; tolerance rule in
  ``oracle.tensor``.  Near field: delta = eps ||A_b||_F / sqrt(d_theta); far
  field: delta = eps ||M_b||_F / sqrt(Delta - 1) with the rank cap on every
  far-field TT rank.
* The "degree" of a workload is the polynomial degree, so p_theta = degree + 1.

Pins (tests/test_oracle_pmatrix.py): nestedness identity to 1e-13; with TT
tolerance 0 and theta at a Chebyshev node, D_b equals the kernel block and
C_b equals the non-parametric coupling matrix W_b of §3.6.2; with the
polynomial test kernel and tolerance 0, both formats reproduce the dense
K(theta) X to rounding for arbitrary theta; near part symmetric; interpolation
error decreasing with p_theta.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import cheb, kernels, tensor, tree


@dataclass
class NearBlock:
    s: tree.Cluster
    t: tree.Cluster
    cores: list = None  # TT of A_b: [G_1 (1, n_s n_t, r_1), G_2, ..., G_{d_theta+1}]


@dataclass
class FarBlock:
    s: tree.Cluster
    t: tree.Cluster
    cores: list = None  # TT of M_b: Delta cores in mode order (i..., k..., j...)
    L: np.ndarray = None  # p_s^d x r_{b,d}
    R: np.ndarray = None  # p_s^d x r_{b,d+d_theta}
    S: np.ndarray = None  # n_s x r_{b,d}          (H format only)
    T: np.ndarray = None  # n_t x r_{b,d+d_theta}  (H format only)


def theta_grid(lo, hi, degree):
    """Per-dimension Chebyshev nodes of B_theta (p_theta = degree + 1 per dimension)."""
    return [cheb.cheb_nodes(lo[i], hi[i], int(degree[i]) + 1) for i in range(len(lo))]


def grid_points(axes):
    """All tensor-grid points, shape (m_1, ..., m_q, q) with axis order = argument order."""
    mesh = np.meshgrid(*axes, indexing="ij")
    return np.stack(mesh, axis=-1)


def near_tensor(kernel, P, s, t, taxes):
    """A_b of §4.3: [A_b]_{(i,j), k_1..k_dtheta} = kappa(x_{s,i}, x_{t,j}; eta_k), i fastest."""
    xs = P[s.idx]
    xt = P[t.idx]
    tg = grid_points(taxes)  # (p_1, ..., p_dt, dt)
    ns, nt = xs.shape[0], xt.shape[0]
    # rows: (i, j) little-endian, i fastest -> row = i + ns * j
    X = np.repeat(xs[None, :, :], nt, axis=0).reshape(ns * nt, -1)  # row i + ns*j -> xs[i]
    Y = np.repeat(xt[:, None, :], ns, axis=1).reshape(ns * nt, -1)  # row i + ns*j -> xt[j]
    shp = (ns * nt,) + tuple(len(a) for a in taxes)
    ex = (slice(None),) + (None,) * len(taxes)
    A = kernels.kappa(kernel, X[ex], Y[ex], tg[None])
    return A.reshape(shp)


def far_tensor(kernel, s, t, taxes, p_s):
    """M_b of App. A.4: modes (i_1..i_d, k_1..k_dtheta, j_1..j_d) on the Chebyshev grids."""
    d = s.lo.size
    sx = [cheb.cheb_nodes(s.lo[k], s.hi[k], p_s) for k in range(d)]
    tx = [cheb.cheb_nodes(t.lo[k], t.hi[k], p_s) for k in range(d)]
    gs = grid_points(sx)  # (p,)*d + (d,)
    gt = grid_points(tx)
    gth = grid_points(taxes)
    dt = len(taxes)
    xs = gs.reshape(gs.shape[:-1] + (1,) * dt + (1,) * d + (d,))
    th = gth.reshape((1,) * d + gth.shape[:-1] + (1,) * d + (dt,))
    yt = gt.reshape((1,) * d + (1,) * dt + gt.shape[:-1] + (d,))
    return kernels.kappa(kernel, xs, yt, th)


def compress_far_block(args):
    """Worker: TT of M_b for one far block (boxes passed explicitly so it can run in a pool)."""
    kernel, slo, shi, tlo, thi, taxes, p_s, tol, cap = args
    s = tree.Cluster([], slo, shi, 0)
    t = tree.Cluster([], tlo, thi, 0)
    M = far_tensor(kernel, s, t, taxes, p_s)
    cores, _ = tensor.tt_svd(M, tol, cap)
    return cores


def L_matrix(cores, d, p_s):
    """L_b = prod_{i=1}^{d-1} (I_{p^{d-i}} (x) G_{b,i}^{2}) G_{b,d}^{2} (App. A.4)."""
    L = tensor.unfold2(cores[d - 1])
    for i in range(d - 1, 0, -1):  # multiply on the left: i = d-1, ..., 1
        L = np.kron(np.eye(p_s ** (d - i)), tensor.unfold2(cores[i - 1])) @ L
    return L


def RT_matrix(cores, d, dt, p_s):
    """R_b^T = G_{b,d+dt+1}^{1} prod_{i=1}^{d-1} (G_{b,d+dt+1+i}^{1} (x) I_{p^i}) (App. A.4)."""
    base = d + dt  # 0-based index of G_{b,d+dt+1}
    RT = tensor.unfold1(cores[base])
    for i in range(1, d):
        RT = RT @ np.kron(tensor.unfold1(cores[base + i]), np.eye(p_s ** i))
    return RT


def H_matrix(cores, d, vs):
    """H_b(theta) = prod_{i=1}^{d_theta} G_{b,d+i} x_2 v_i(theta_i) (App. A.4, Alg. PTTK online)."""
    H = None
    for i, v in enumerate(vs):
        Hi = tensor.mode2_vec(cores[d + i], v)
        H = Hi if H is None else H @ Hi
    return H


def basis_factors(P, c, p_s):
    """Factor matrices U_{s,k} (n_s x p_s) with [U_{s,k}]_{i,j} = ell_j^{(B_s,k)}([x_{s,i}]_k) (§3.3)."""
    x = P[c.idx]
    return [cheb.lagrange(cheb.cheb_nodes(c.lo[k], c.hi[k], p_s), x[:, k]) for k in range(c.lo.size)]


def cluster_basis(factors):
    """U_s = U_{s,d} |x U_{s,d-1} |x ... |x U_{s,1} (face-splitting, §3.3)."""
    U = factors[0]
    for F in factors[1:]:
        U = tensor.face_split(F, U)
    return U


def transfer_factors(child, p_s):
    """E_{s',k} with [E_{s',k}]_{j,i} = ell_i^{(B_s,k)}(eta_j^{(B_s',k)}) (§3.6.1, reading above)."""
    par = child.parent
    out = []
    for k in range(child.lo.size):
        pn = cheb.cheb_nodes(par.lo[k], par.hi[k], p_s)
        cn = cheb.cheb_nodes(child.lo[k], child.hi[k], p_s)
        out.append(cheb.lagrange(pn, cn))  # rows: child nodes j, columns: parent polynomials i
    return out


def transfer_matrix(factors):
    """E_{s'} = E_{s',d} (x) ... (x) E_{s',1} (§3.6.1)."""
    return tensor.kron_chain(factors[::-1])


class ParametricMatrix:
    """Parametric H or H^2 matrix over a point set, built literally from the paper.

    kernel      kernel name (oracle.kernels)
    theta_lo/hi parameter box B_theta (length d_theta)
    degree      Chebyshev degree per parameter dimension (p_theta = degree + 1)
    p_s         spatial Chebyshev nodes per dimension
    l_max       depth of the uniform cluster tree (ignored when leaf_size is set)
    eta         admissibility parameter
    tol         TT tolerance eps (0 means no truncation)
    rank_cap    cap on far-field TT ranks (None: no cap)
    fmt         "h2" or "h"
    """

    def __init__(self, points, kernel, theta_lo, theta_hi, degree, p_s, l_max, eta, tol,
                 rank_cap=None, fmt="h2", leaf_size=None, near_tol=None, near_degree=None):
        self.P = np.asarray(points, float)
        self.n, self.d = self.P.shape
        self.kernel = kernel
        self.theta_lo = np.atleast_1d(np.asarray(theta_lo, float))
        self.theta_hi = np.atleast_1d(np.asarray(theta_hi, float))
        self.dt = self.theta_lo.size
        self.degree = np.atleast_1d(np.asarray(degree, int))
        self.taxes = theta_grid(self.theta_lo, self.theta_hi, self.degree)
        # the near field's own theta grid (§4.3 compresses A_b on a grid of its own choosing)
        self.near_degree = self.degree if near_degree is None else np.atleast_1d(np.asarray(near_degree, int))
        self.taxes_near = theta_grid(self.theta_lo, self.theta_hi, self.near_degree)
        self.p_s = int(p_s)
        self.eta = float(eta)
        self.tol = float(tol)
        self.near_tol = self.tol if near_tol is None else float(near_tol)
        self.rank_cap = rank_cap
        self.fmt = fmt
        # Offline, step 1 (Algs. "Offline Stage", §4.4): cluster tree and block cluster tree.
        self.root = tree.build_cluster_tree(self.P, l_max, leaf_size=leaf_size)
        self.nodes = tree.all_nodes(self.root)
        self.leaves = [c for c in self.nodes if c.is_leaf()]
        near, far = tree.build_block_tree(self.root, self.eta)
        self.near = [NearBlock(s, t) for s, t in near]
        self.far = [FarBlock(s, t) for s, t in far]
        self._U = {}
        self._E = {}

    # ------------------------------------------------------------------ offline
    def compress_near(self, b: NearBlock):
        """TT of A_b (§4.3), delta = eps ||A_b||_F / sqrt(d_theta)."""
        if b.cores is None:
            A = near_tensor(self.kernel, self.P, b.s, b.t, self.taxes_near)
            b.cores, _ = tensor.tt_svd(A, self.near_tol, None)
        return b

    def far_args(self, b: FarBlock):
        return (self.kernel, b.s.lo, b.s.hi, b.t.lo, b.t.hi, self.taxes, self.p_s, self.tol,
                self.rank_cap)

    def finish_far(self, b: FarBlock, cores):
        """Store the TT of M_b and form L_b, R_b (and S_b, T_b for the H format)."""
        b.cores = cores
        b.L = L_matrix(cores, self.d, self.p_s)
        b.R = RT_matrix(cores, self.d, self.dt, self.p_s).T
        if self.fmt == "h":
            b.S = self.basis(b.s) @ b.L
            b.T = self.basis(b.t) @ b.R
        return b

    def compress_far(self, b: FarBlock):
        if b.cores is None:
            self.finish_far(b, compress_far_block(self.far_args(b)))
        return b

    def offline(self, targets=None, pool=None):
        """Compress the near and far blocks whose rows meet the given target leaves (all by default)."""
        near, far = self.blocks_for(targets)
        for b in near:
            self.compress_near(b)
        todo = [b for b in far if b.cores is None]
        if pool is not None and todo:
            for b, cores in zip(todo, pool.map(compress_far_block, [self.far_args(b) for b in todo])):
                self.finish_far(b, cores)
        else:
            for b in todo:
                self.compress_far(b)
        return self

    def blocks_for(self, targets=None):
        if targets is None:
            return self.near, self.far
        tset = {id(c) for c in targets}
        anc = set()
        for c in targets:
            a = c
            while a is not None:
                anc.add(id(a))
                a = a.parent
        return ([b for b in self.near if id(b.s) in tset], [b for b in self.far if id(b.s) in anc])

    def basis(self, c):
        """Explicit U_s (face-splitting of the factor matrices, §3.3)."""
        if c.id not in self._U:
            self._U[c.id] = cluster_basis(basis_factors(self.P, c, self.p_s))
        return self._U[c.id]

    def transfer(self, c):
        """Explicit E_{s'} for a non-root node (§3.6.1)."""
        if c.id not in self._E:
            self._E[c.id] = transfer_matrix(transfer_factors(c, self.p_s))
        return self._E[c.id]

    # ------------------------------------------------------------------- online
    def parametric_vectors(self, theta, deriv=None):
        return cheb.parametric_vectors(theta, self.theta_lo, self.theta_hi, self.degree, deriv)

    def check_theta(self, theta):
        th = np.atleast_1d(np.asarray(theta, float))
        if th.size != self.dt or np.any(th < self.theta_lo) or np.any(th > self.theta_hi):
            raise ValueError("theta outside the parameter box")
        return th

    @staticmethod
    def near_instance(b: NearBlock, vs):
        """D_b(theta) = reshape(G_{b,1} prod_i (G_{b,i+1} x_2 v_i), [n_s, n_t]) (§4.3)."""
        w = None
        for i, v in enumerate(vs):
            Wi = tensor.mode2_vec(b.cores[i + 1], v)
            w = Wi if w is None else w @ Wi
        G1 = tensor.freshape(b.cores[0], (b.s.n * b.t.n, b.cores[0].shape[2]))
        a = G1 @ w[:, 0]
        return tensor.freshape(a, (b.s.n, b.t.n))

    def instantiate(self, theta, targets=None, deriv=None):
        """Online stage (Alg. "Online Stage", §4.4): D_b(theta) for near blocks, H_b(theta) for far blocks.

        ``deriv = i``: instantiate dK_hat/dtheta_i instead (v_i replaced by its derivative; every
        stored quantity enters linearly in v_i).
        """
        th = self.check_theta(theta)
        if deriv is not None and not 0 <= int(deriv) < self.dt:
            raise ValueError("deriv is not a parameter dimension")
        vs = self.parametric_vectors(th, deriv)
        vs_near = cheb.parametric_vectors(th, self.theta_lo, self.theta_hi, self.near_degree, deriv)
        near, far = self.blocks_for(targets)
        inst = {"theta": th, "vs": vs, "D": {}, "H": {}}
        for b in near:
            inst["D"][id(b)] = self.near_instance(b, vs_near)
        for b in far:
            inst["H"][id(b)] = H_matrix(b.cores, self.d, vs)
        return inst

    def projected_cores(self, theta, targets=None):
        """The exact coupling core of every far block at theta in the gauge of its stored spatial
        factors: H*_b(theta) = L_b^+ W_b(theta) (R_b^T)^+, the least-squares solution of
        L_b H R_b^T = W_b(theta), where W_b(theta)[i, j] = kappa(eta^s_i, eta^t_j; theta) is the
        non-parametric coupling matrix of §3.6.2 (little-endian multi-indices) evaluated at this
        theta.  It is the target the learned surrogate of the far-field cores is trained on:
        H_b(theta) is the only theta-dependent far-field quantity (App. A.4), and this is the best
        one the fixed L_b, R_b admit.  With the interpolation exact (polynomial kernel, theta
        nodes, no truncation) it equals H_b(theta)."""
        th = self.check_theta(theta)
        _, far = self.blocks_for(targets)
        single = [[float(x)] for x in th]
        out = {}
        for b in far:
            Wt = far_tensor(self.kernel, b.s, b.t, single, self.p_s)
            W = tensor.freshape(Wt, (self.p_s ** self.d, self.p_s ** self.d))
            out[id(b)] = np.linalg.pinv(b.L) @ W @ np.linalg.pinv(b.R.T)
        return out

    def instantiate_projected(self, theta, targets=None):
        """The online stage with the far-field cores replaced by projected_cores(theta); the near
        field as instantiate()."""
        inst = self.instantiate(theta, targets)
        inst["H"] = self.projected_cores(theta, targets)
        return inst

    def coupling(self, b: FarBlock, inst):
        """C_b(theta) = L_b H_b(theta) R_b^T formed explicitly (§4.2)."""
        return b.L @ inst["H"][id(b)] @ b.R.T

    # ---------------------------------------------------------------------- MVM
    def matvec(self, inst, X, targets=None):
        """Y = K_hat(theta) X for the instantiated matrix (§4.5).

        ``targets``: restrict the output to the rows of these leaves (other rows
        are returned as NaN); the needed blocks must have been compressed.
        """
        X = np.asarray(X, float)
        if X.ndim == 1:
            return self.matvec(inst, X[:, None], targets)[:, 0]
        if self.fmt == "h":
            return self._matvec_h(inst, X, targets)
        return self._matvec_h2(inst, X, targets)

    def _matvec_h(self, inst, X, targets):
        """Parametric H MVM: Alg. "H-matrix MVM" (App. A.1) with the far line replaced (§4.5)."""
        Y = np.zeros_like(X)
        near, far = self.blocks_for(targets)
        for b in far:
            Y[b.s.idx] += b.S @ (inst["H"][id(b)] @ (b.T.T @ X[b.t.idx]))
        for b in near:
            Y[b.s.idx] += inst["D"][id(b)] @ X[b.t.idx]
        return self._mask(Y, targets)

    def _matvec_h2(self, inst, X, targets):
        """Parametric H^2 MVM: Alg. "Modified H^2-Matrix MVM" (§4.5) with explicit C_b."""
        m = X.shape[1]
        Y = np.zeros_like(X)
        xhat = {}

        def forward(c):  # Alg. FastForward (App. A.1)
            if c.is_leaf():
                xhat[c.id] = self.basis(c).T @ X[c.idx]
            else:
                acc = np.zeros((self.p_s ** self.d, m))
                for ch in c.children:
                    forward(ch)
                    acc += self.transfer(ch).T @ xhat[ch.id]
                xhat[c.id] = acc

        forward(self.root)
        near, far = self.blocks_for(targets)
        yhat = {c.id: np.zeros((self.p_s ** self.d, m)) for c in self.nodes}
        for b in far:  # multiplication stage, far part
            yhat[b.s.id] += self.coupling(b, inst) @ xhat[b.t.id]
        for b in near:  # multiplication stage, near part
            Y[b.s.idx] += inst["D"][id(b)] @ X[b.t.idx]

        def backward(c):  # Alg. FastBackward (App. A.1)
            if c.is_leaf():
                Y[c.idx] += self.basis(c) @ yhat[c.id]
            else:
                for ch in c.children:
                    yhat[ch.id] += self.transfer(ch) @ yhat[c.id]
                    backward(ch)

        backward(self.root)
        return self._mask(Y, targets)

    # ------------------------------------------------------------------ adjoint
    def matvec_transpose(self, inst, Ybar):
        """Xbar = K_hat(theta)^T Ybar, the adjoint of ``matvec`` (not in the paper; the gradient of
        a scalar function of Y with respect to X).  Every block contributes its transpose:
        D_b^T Ybar_s into the rows of t; for H, T_b H_b^T S_b^T Ybar_s; for H^2, Alg. FastForward
        on Ybar with the same nested bases, x_t += C_b^T yhat_s, then Alg. FastBackward into
        Xbar.  Needs every block compressed (``offline()`` without targets) and instantiated
        (``instantiate(theta)`` without targets); an instance of the derivative gives
        (dK_hat/dtheta)^T Ybar.
        """
        Ybar = np.asarray(Ybar, float)
        if Ybar.ndim == 1:
            return self.matvec_transpose(inst, Ybar[:, None])[:, 0]
        for b in self.near:
            if id(b) not in inst["D"]:
                raise ValueError("matvec_transpose needs an instance of every block")
        Xb = np.zeros_like(Ybar)
        for b in self.near:
            Xb[b.t.idx] += inst["D"][id(b)].T @ Ybar[b.s.idx]
        if self.fmt == "h":
            for b in self.far:
                Xb[b.t.idx] += b.T @ (inst["H"][id(b)].T @ (b.S.T @ Ybar[b.s.idx]))
            return Xb
        m = Ybar.shape[1]
        yhat = {}

        def forward(c):  # Alg. FastForward on Ybar
            if c.is_leaf():
                yhat[c.id] = self.basis(c).T @ Ybar[c.idx]
            else:
                acc = np.zeros((self.p_s ** self.d, m))
                for ch in c.children:
                    forward(ch)
                    acc += self.transfer(ch).T @ yhat[ch.id]
                yhat[c.id] = acc

        forward(self.root)
        xhat = {c.id: np.zeros((self.p_s ** self.d, m)) for c in self.nodes}
        for b in self.far:
            xhat[b.t.id] += self.coupling(b, inst).T @ yhat[b.s.id]

        def backward(c):  # Alg. FastBackward into Xbar
            if c.is_leaf():
                Xb[c.idx] += self.basis(c) @ xhat[c.id]
            else:
                for ch in c.children:
                    xhat[ch.id] += self.transfer(ch) @ xhat[c.id]
                    backward(ch)

        backward(self.root)
        return Xb

    def _mask(self, Y, targets):
        if targets is None:
            return Y
        keep = np.zeros(self.n, dtype=bool)
        for c in targets:
            keep[c.idx] = True
        Y[~keep] = np.nan
        return Y

    # ------------------------------------------------------------------ reports
    def near_ratio(self) -> float:
        """NF ratio of §6: entries of the near-field blocks over n^2."""
        return sum(b.s.n * b.t.n for b in self.near) / float(self.n) ** 2

    def dense_theta(self, theta):
        """The exact kernel matrix K(X, X; theta) (§1) for small n."""
        return kernels.dense_matrix(self.kernel, self.P, theta)


def relative_error(ref, approx, axis=0):
    """Relative 2-norm error per column, ||ref - approx|| / ||ref|| (the Error of §6)."""
    ref = np.asarray(ref, float)
    approx = np.asarray(approx, float)
    return np.linalg.norm(ref - approx, axis=axis) / np.linalg.norm(ref, axis=axis)

