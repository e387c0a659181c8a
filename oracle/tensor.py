"""Tensor primitives of §2.1 and App. A.2, and the TT-SVD compressor.

Test infrastructure only (see ``oracle/__init__.py``).

Conventions (§2.1): multi-indices flatten little-endian (the first index runs
fastest) and ``reshape`` is MATLAB's, i.e. NumPy's ``order='F'``.

TT-SVD follows Oseledets (2011), Algorithm 1, which §2.1 names as an
alternative to TT-cross.  The paper's own compressor (a TT-cross variant with
Chebyshev-norm heuristics) depends on pivoting choices; TT-SVD's truncated
result is unique, which is what lets an independent implementation agree with
this one.  Truncation rule (stated once, used for every core):

* delta = eps * ||A||_F / sqrt(q - 1) for a q-way tensor A;
* at each cut keep the smallest rank r >= 1 whose discarded tail satisfies
  sum_{i > r} s_i^2 <= delta^2;
* ties: while r < len(s) and s_r - s_{r+1} <= 1e-9 * s_1, keep one more value, so
  that a numerically tied group is kept whole;
* then the cap: if r > rank_cap, r = rank_cap, and if that splits a tied group
  (s_r - s_{r+1} <= 1e-9 * s_1) the whole group is dropped (r decreases while the
  cut still separates tied values).  A truncation that split a group of equal
  singular values would keep an arbitrary subspace of it, and no two
  implementations would agree; this keeps the truncated TT unique.

Pins (tests/test_oracle_basics.py): reconstruction error <= eps ||A||_F;
exactness on tensors of known low TT rank; the 2-way case equals the
Eckart-Young truncated SVD; the vec-kron identity; face-splitting row rule.
"""
from __future__ import annotations

import numpy as np

TIE_REL = 1e-9


def freshape(a: np.ndarray, shape) -> np.ndarray:
    """MATLAB reshape (first index fastest), §2.1."""
    return np.reshape(a, shape, order="F")


def unfold1(G: np.ndarray) -> np.ndarray:
    """G^{1} = reshape(G, [r_{i-1}, m_i r_i]) for a core G of shape (r_{i-1}, m_i, r_i) (§2.1)."""
    r0, m, r1 = G.shape
    return freshape(G, (r0, m * r1))


def unfold2(G: np.ndarray) -> np.ndarray:
    """G^{2} = reshape(G, [r_{i-1} m_i, r_i]) for a core G of shape (r_{i-1}, m_i, r_i) (§2.1)."""
    r0, m, r1 = G.shape
    return freshape(G, (r0 * m, r1))


def mode2_vec(G: np.ndarray, v: np.ndarray) -> np.ndarray:
    """G x_2 v for a 3-way core G (r0, m, r1) and a vector v of length m (§2.1): an r0 x r1 matrix."""
    return np.einsum("amb,m->ab", G, v)


def kron_chain(mats) -> np.ndarray:
    """mats[0] (x) mats[1] (x) ... (Kronecker product of App. A.2, left to right)."""
    out = np.ones((1, 1))
    for M in mats:
        out = np.kron(out, M)
    return out


def face_split(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Face-splitting product A |x B of App. A.2: row i is a_i (x) b_i."""
    assert A.shape[0] == B.shape[0]
    return np.einsum("ia,ib->iab", A, B).reshape(A.shape[0], A.shape[1] * B.shape[1])


def truncation_rank(s: np.ndarray, delta: float, rank_cap=None) -> int:
    """Rank kept at one TT-SVD cut (rule in the module docstring)."""
    s = np.asarray(s, float)
    n = s.size
    cap = n if rank_cap is None else min(n, int(rank_cap))
    tail = np.concatenate([np.cumsum((s * s)[::-1])[::-1], [0.0]])  # tail[r] = sum_{i>=r} s_i^2 (0-based)
    r = n
    for k in range(1, n + 1):
        if tail[k] <= delta * delta:
            r = k
            break
    r = max(1, r)
    tied = lambda k: n and s[0] > 0 and k < n and s[k - 1] - s[k] <= TIE_REL * s[0]
    while tied(r):
        r += 1
    if r > cap:
        r = cap
        while r > 1 and tied(r):
            r -= 1
    return r


def tt_svd(A: np.ndarray, eps: float, rank_cap=None):
    """TT decomposition of the q-way tensor A by TT-SVD (Oseledets 2011, Alg. 1).

    Returns (cores, ranks): cores[j] has shape (r_j, m_{j+1}, r_{j+1}) with
    r_0 = r_q = 1, so that A[i_1..i_q] = G_1[:, i_1, :] ... G_q[:, i_q, :] (§2.1).
    """
    dims = A.shape
    q = len(dims)
    if q == 1:
        return [A.reshape(1, dims[0], 1).copy()], [1, 1]
    norm = float(np.linalg.norm(A))
    delta = eps * norm / np.sqrt(q - 1)
    C = freshape(A, (dims[0], -1))
    r_prev = 1
    cores, ranks = [], [1]
    for k in range(q - 1):
        C = freshape(C, (r_prev * dims[k], -1))
        U, s, Vt = np.linalg.svd(C, full_matrices=False)
        r = truncation_rank(s, delta, rank_cap)
        cores.append(freshape(U[:, :r], (r_prev, dims[k], r)))
        C = s[:r, None] * Vt[:r, :]
        r_prev = r
        ranks.append(r)
    cores.append(freshape(C, (r_prev, dims[-1], 1)))
    ranks.append(1)
    return cores, ranks


def tt_full(cores) -> np.ndarray:
    """Dense tensor of a TT (the entry formula of §2.1), contracted core by core."""
    out = cores[0]  # (1, m1, r1)
    dims = [cores[0].shape[1]]
    for G in cores[1:]:
        out = np.tensordot(out, G, axes=([out.ndim - 1], [0]))
        dims.append(G.shape[1])
    return out.reshape([1] + dims + [1])[0, ..., 0]
