"""TT-cross with greedy pivots, and TT-rounding: the compressor the paper uses (§2.1).

Test infrastructure only (see ``oracle/__init__.py``).

§2.1 approximates a tensor given entry-wise (the kernel on a tensor grid) by a variant of the
greedy cross of Savostyanov (2014, Alg. 2): starting from a single index, each sweep visits the
bonds k = 1 .. q-1 and adds one pivot to the bond's nested index sets, found by partially
pivoted cross search on the residual of the bond's two-mode unfolding (the "super core");
sweeps stop when the largest pivot residual is below eps times the largest entry seen (a
Chebyshev-norm heuristic). The interpolant is then recompressed by TT-rounding (Oseledets 2011,
Alg. 2) with the TT-SVD truncation rule of ``oracle.tensor``. Written here from those
descriptions; the paper gives no listing.

Notation. Left index sets I_k are tuples over modes 1..k, right sets J_k tuples over modes
k+1..q, |I_k| = |J_k| = r_k (bond k sits between modes k and k+1). The cross interpolant is
  T~(i_1..i_q) = C_1(i_1) P_1^{-1} C_2(i_2) P_2^{-1} ... C_q(i_q),
  C_k(i_k)[a, b] = T(I_{k-1}[a], i_k, J_k[b]),   P_k[a, b] = T(I_k[a], J_k[b]),
so the TT cores are G_k = C_k P_k^{-1} (k < q) and G_q = C_q. It interpolates T on the crosses:
T~(I_k[a], J_k[b]) = T(I_k[a], J_k[b]) for every bond (pinned in tests/test_oracle_cross.py).

Pins (tests/test_oracle_cross.py): exact recovery of tensors of known low TT rank; the
interpolation property; the error after rounding within a small multiple of eps on kernel
tensors, with ranks close to TT-SVD's; far fewer entries evaluated than the tensor has.
"""
from __future__ import annotations

import numpy as np

from .tensor import freshape, truncation_rank


class Entries:
    """Entry access to a q-way tensor given by f(idx) -> value for an (m, q) integer array of
    multi-indices; every distinct entry is evaluated once and counted."""

    def __init__(self, f, dims):
        self.f = f
        self.dims = tuple(int(n) for n in dims)
        self.cache = {}

    @property
    def count(self):
        return len(self.cache)

    def __call__(self, idx):
        idx = np.asarray(idx, dtype=np.int64).reshape(-1, len(self.dims))
        keys = [tuple(r) for r in idx.tolist()]
        missing = [i for i, k in enumerate(keys) if k not in self.cache]
        if missing:
            vals = np.asarray(self.f(idx[missing]), float).reshape(-1)
            for i, v in zip(missing, vals):
                self.cache[keys[i]] = float(v)
        return np.array([self.cache[k] for k in keys])


def _psolve(P, B):
    """P^{-1} B, by least squares (a pivot matrix may be singular after an enrichment)."""
    return np.linalg.lstsq(P, B, rcond=1e-13)[0]


def _idx(*parts):
    """Multi-indices from lists of index tuples / ints, the first list varying fastest."""
    lists = [p if isinstance(p, list) else [p] for p in parts]
    grids = np.meshgrid(*[np.arange(len(l)) for l in lists], indexing="ij")
    flat = [g.ravel(order="F") for g in grids]
    rows = []
    for t in range(flat[0].size if flat else 1):
        tup = ()
        for l, g in zip(lists, flat):
            x = l[g[t]]
            tup += tuple(x) if isinstance(x, tuple) else (int(x),)
        rows.append(tup)
    return np.array(rows, dtype=np.int64)


def _fiber_block(T, Ik, k, Jk1):
    """C_k = T(I_k[a], i_k, J_{k+1}[b]) as an array (r_k, n_k, r_{k+1}) (a fastest)."""
    vals = T(_idx(Ik, list(range(T.dims[k])), Jk1))
    return freshape(vals, (len(Ik), T.dims[k], len(Jk1)))


def _pivots(T, I, J, k):
    """P = T(I_{k+1}[a], J_{k+1}[b]) of bond k (between modes k and k+1)."""
    vals = T(_idx(I[k + 1], J[k + 1]))
    return freshape(vals, (len(I[k + 1]), len(J[k + 1])))


def _cross_cores(T, I, J):
    """Cores G_k = C_k P_k^{-1} (k < q), G_q = C_q of the cross interpolant."""
    q = len(T.dims)
    cores = []
    for k in range(q):
        C = _fiber_block(T, I[k], k, J[k + 1])
        if k < q - 1:
            P = _pivots(T, I, J, k)
            r0, n, r1 = C.shape
            G = _psolve(P.T, freshape(C, (r0 * n, r1)).T).T  # C P^{-1}
            cores.append(freshape(G, (r0, n, r1)))
        else:
            cores.append(C)
    return cores


def _residual_col(T, I, J, k, col):
    """Residual of the bond-k super core (rows (a, i_k), a fastest; columns (i_{k+1}, b)) on one
    column: exact entries minus A(:, J_{k+1}) P^{-1} A(I_{k+1}, col)."""
    j, b = col
    rows = list(range(T.dims[k]))
    exact = T(_idx(I[k], rows, j, [J[k + 2][b]]))
    left = freshape(T(_idx(I[k], rows, J[k + 1])), (len(I[k]) * T.dims[k], len(J[k + 1])))
    right = T(_idx(I[k + 1], j, [J[k + 2][b]]))
    return exact - left @ _psolve(_pivots(T, I, J, k), right)


def _residual_row(T, I, J, k, row):
    a, ik = row
    cols = list(range(T.dims[k + 1]))
    exact = T(_idx([I[k][a]], ik, cols, J[k + 2]))
    left = T(_idx([I[k][a]], ik, J[k + 1]))
    right = freshape(T(_idx(I[k + 1], cols, J[k + 2])), (len(I[k + 1]), T.dims[k + 1] * len(J[k + 2])))
    return exact - _psolve(_pivots(T, I, J, k).T, left) @ right


def _tt_eval(cores, idx):
    """Entries of a TT at the multi-indices idx (m x q)."""
    out = np.ones((idx.shape[0], 1))
    for k, G in enumerate(cores):
        out = np.einsum("ma,mab->mb", out, G[:, idx[:, k], :].transpose(1, 0, 2))
    return out[:, 0]


def tt_cross(f, dims, eps, rank_cap=None, max_sweeps=200, rook_steps=3, samples=64, seed=0):
    """Greedy TT-cross of the tensor with entries f (see Entries).  Returns (cores, ranks, T)
    with T the entry counter.  Starts from the largest of a few random entries as the single
    index; each sweep adds at most one pivot per bond (bond ranks capped at rank_cap and at the
    unfolding sizes).  A sweep whose pivot residuals are all <= eps * max |entry seen| is checked
    on `samples` random entries; if the interpolant misses one of them by more, its prefixes and
    suffixes join the index sets of the bonds wherever the sets stay nested (the restricted super
    cores can look exact while the tensor is not, e.g. for separable kernels) and the sweeps go
    on."""
    T = Entries(f, dims)
    q = len(T.dims)
    rng = np.random.default_rng(seed)
    probe = np.stack([rng.integers(0, n, 64) for n in T.dims], axis=1)
    vals = T(probe)
    start = tuple(int(x) for x in probe[int(np.argmax(np.abs(vals)))])
    vmax = float(np.max(np.abs(vals)))
    # I[k]: left sets over modes 0..k-1 (I[0] = [()]); J[k]: right sets over modes k..q-1 (J[q] = [()])
    I = [[start[:k]] for k in range(q + 1)]
    J = [[start[k:]] for k in range(q + 1)]
    for _ in range(max_sweeps):
        worst = 0.0
        for k in range(q - 1):
            rows_max = len(I[k]) * T.dims[k]
            cols_max = T.dims[k + 1] * len(J[k + 2])
            cap = min(rows_max, cols_max, rank_cap or rows_max)
            if len(I[k + 1]) >= cap:
                continue
            # partially pivoted (rook) search on the residual of the super core
            col = (int(rng.integers(T.dims[k + 1])), int(rng.integers(len(J[k + 2]))))
            best = (0.0, None, None)
            for _ in range(rook_steps):
                e = _residual_col(T, I, J, k, col)
                ir = int(np.argmax(np.abs(e)))
                row = (ir % len(I[k]), ir // len(I[k]))
                er = _residual_row(T, I, J, k, row)
                jc = int(np.argmax(np.abs(er)))
                col = (jc % T.dims[k + 1], jc // T.dims[k + 1])
                if abs(er[jc]) > best[0]:
                    best = (abs(er[jc]), row, col)
            res, row, col = best
            worst = max(worst, res)
            if row is None or res <= 1e-14 * vmax:
                continue  # the super core is reproduced
            new_i = tuple(I[k][row[0]]) + (row[1],)
            new_j = (col[0],) + tuple(J[k + 2][col[1]])
            if new_i in I[k + 1] or new_j in J[k + 1]:
                continue
            I[k + 1].append(new_i)
            J[k + 1].append(new_j)
        if worst <= eps * vmax:
            # the random check of the Chebyshev-norm heuristic
            cores = _cross_cores(T, I, J)
            probe = np.stack([rng.integers(0, n, samples) for n in T.dims], axis=1)
            exact = T(probe)
            vmax = max(vmax, float(np.max(np.abs(exact))))
            err = np.abs(_tt_eval(cores, probe) - exact)
            w = int(np.argmax(err))
            if err[w] <= eps * vmax:
                break
            x = tuple(int(v) for v in probe[w])
            # bonds that take the pair (prefix, suffix) of the missed entry: both new, room left, and
            # the sets stay nested (the cross interpolation needs I_{k+1} in I_k x n_k and
            # J_{k+1} in n_{k+1} x J_{k+2}): the pair's shorter prefix / suffix present or added too
            take = []
            for k in range(q - 1):
                rows_max = len(I[k]) * T.dims[k]
                cols_max = T.dims[k + 1] * len(J[k + 2])
                take.append(len(I[k + 1]) < min(rows_max, cols_max, rank_cap or rows_max)
                            and x[:k + 1] not in I[k + 1] and x[k + 1:] not in J[k + 1])
            changed = True
            while changed:
                changed = False
                for k in range(q - 1):
                    if not take[k]:
                        continue
                    left_ok = k == 0 or take[k - 1] or x[:k] in I[k]
                    right_ok = k + 2 >= q or take[k + 1] or x[k + 2:] in J[k + 2]
                    if not (left_ok and right_ok):
                        take[k] = False
                        changed = True
            if not any(take):
                break
            for k in range(q - 1):
                if take[k]:
                    I[k + 1].append(x[:k + 1])
                    J[k + 1].append(x[k + 1:])
    cores = _cross_cores(T, I, J)
    ranks = [1] + [len(I[k]) for k in range(1, q)] + [1]
    T.I, T.J = I, J  # the index sets, for inspection
    return cores, ranks, T


def tt_round(cores, eps, rank_cap=None):
    """TT-rounding (Oseledets 2011, Alg. 2): right-to-left orthogonalisation by QR, then
    left-to-right truncated SVDs with delta = eps ||T||_F / sqrt(q - 1) and the TT-SVD rule."""
    cores = [G.copy() for G in cores]
    q = len(cores)
    for k in range(q - 1, 0, -1):
        r0, n, r1 = cores[k].shape
        Q, R = np.linalg.qr(freshape(cores[k], (r0, n * r1)).T)
        cores[k] = freshape(Q.T, (Q.shape[1], n, r1))
        cores[k - 1] = np.einsum("anb,cb->anc", cores[k - 1], R)
    norm = float(np.linalg.norm(cores[0]))
    delta = eps * norm / np.sqrt(max(1, q - 1))
    ranks = [1]
    for k in range(q - 1):
        r0, n, r1 = cores[k].shape
        U, s, Vt = np.linalg.svd(freshape(cores[k], (r0 * n, r1)), full_matrices=False)
        r = truncation_rank(s, delta, rank_cap)
        cores[k] = freshape(U[:, :r], (r0, n, r))
        cores[k + 1] = np.einsum("ab,bnc->anc", s[:r, None] * Vt[:r], cores[k + 1])
        ranks.append(r)
    ranks.append(1)
    return cores, ranks
