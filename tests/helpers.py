"""Shared helpers for the GPU parity tests: build the same workload on both sides.

The oracle and the CUDA library are built independently from the same seeded
inputs; nothing flows from the library into the oracle.
"""
import numpy as np

from oracle import pmatrix

TOL = {"fp64": 1e-10, "fp32": 1e-5}


def build_pair(P, kernel, lo, hi, degree, p_s, l_max, eta, tol, cap, fmt, prec, dedup=True,
               targets_every=None, pool=None, check_finite=False, coupling="explicit", near_shared=True):
    """Returns (product handle, oracle model, oracle target leaves or None)."""
    from paper_2511_03109_gb300 import ph

    opts = ph.make_opts(P.shape[1], lo, hi, degree, p_s, l_max, eta, tol, rank_cap=cap or 0,
                        fmt=fmt, prec=prec, dedup=dedup, check_finite=check_finite, coupling=coupling,
                        near_shared=near_shared)
    A = ph.ParametricMatrix(P, kernel, opts)
    M = pmatrix.ParametricMatrix(P, kernel, lo, hi, degree, p_s, l_max, eta, tol,
                                 rank_cap=cap or None, fmt=fmt)
    targets = None
    if targets_every:
        targets = M.leaves[::targets_every]
    M.offline(targets, pool=pool)
    return A, M, targets


def device_apply(A, theta, X, prec, ldx_pad=0, deriv=None):
    """Instantiate (or, with deriv = i, instantiate dK_hat/dtheta_i) and apply on cuda:0
    through the C ABI (raw device pointers)."""
    import torch

    dt = torch.float64 if prec == "fp64" else torch.float32
    n, m = X.shape
    ld = n + ldx_pad
    Xd = torch.zeros((m, ld), dtype=dt, device="cuda:0")
    Xd[:, :n] = torch.tensor(X.T, dtype=dt)
    Yd = torch.full((m, ld), float("nan"), dtype=dt, device="cuda:0")
    if deriv is None:
        A.instantiate(theta)
    else:
        A.instantiate_derivative(theta, deriv)
    A.matvec_ptr(Xd.data_ptr(), ld, m, Yd.data_ptr(), ld)
    torch.cuda.synchronize()
    return Yd[:, :n].double().cpu().numpy().T


def rel_err_rows(ref, got, rows=None):
    """Relative 2-norm error per column over the given rows (all rows by default)."""
    if rows is not None:
        ref, got = ref[rows], got[rows]
    return np.linalg.norm(ref - got, axis=0) / np.linalg.norm(ref, axis=0)


def target_rows(targets):
    return np.sort(np.concatenate([c.idx for c in targets]))
