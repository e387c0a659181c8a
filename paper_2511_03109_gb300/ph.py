"""ctypes binding of libph (include/ph.h): the same entry points, argument marshalling only.

Every computation runs in the CUDA library.  Importing this module loads
``lib/libph.so`` and raises ImportError when it has not been built (run
``__graft_entry__.build()``); there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libph.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libph is not built ({LIB_PATH} missing); run __graft_entry__.build()")
_lib = C.CDLL(LIB_PATH)

# ph_status
PH_OK = 0
PH_ERR_INVALID_ARG = 1
PH_ERR_THETA_OUT_OF_BOX = 2
PH_ERR_NOT_INSTANTIATED = 3
PH_ERR_OOM = 4
PH_ERR_CUDA = 5
PH_ERR_NONFINITE = 6
PH_ERR_TIMEOUT = 7
PH_ERR_IO = 8
PH_ERR_UNSUPPORTED = 9

KERNELS = {"gauss": 0, "matern32": 1, "matern52": 2, "aniso_gauss": 3, "se": 4, "exponential": 5,
           "mc": 6, "poly": 7, "polyxy": 8, "poly2": 9}
FORMATS = {"h2": 0, "h": 1}
PRECISIONS = {"fp64": 0, "fp32": 1}


class BuildOpts(C.Structure):
    _fields_ = [("d", C.c_int), ("dtheta", C.c_int), ("theta_lo", C.c_double * 3),
                ("theta_hi", C.c_double * 3), ("degree", C.c_int * 3), ("p_s", C.c_int),
                ("l_max", C.c_int), ("eta", C.c_double), ("tol", C.c_double),
                ("near_tol", C.c_double), ("rank_cap", C.c_int), ("fmt", C.c_int),
                ("prec", C.c_int), ("dedup", C.c_int), ("check_finite", C.c_int),
                ("device", C.c_int), ("coupling", C.c_int), ("near_unshared", C.c_int),
                ("near_degree", C.c_int * 3), ("compressor", C.c_int)]


class Info(C.Structure):
    _fields_ = [("n", C.c_long), ("d", C.c_int), ("dtheta", C.c_int), ("p_s", C.c_int),
                ("p_theta", C.c_int * 3), ("prec", C.c_int), ("fmt", C.c_int),
                ("n_nodes", C.c_int), ("n_leaves", C.c_int), ("tree_depth", C.c_int),
                ("n_near", C.c_long), ("n_far", C.c_long), ("n_far_keys", C.c_long),
                ("near_entries", C.c_long), ("near_rank_sum", C.c_long),
                ("near_rank_max", C.c_int), ("far_rank_max", C.c_int),
                ("far_rank_mean", C.c_double), ("near_bytes", C.c_long),
                ("near_theta_bytes", C.c_long), ("far_bytes", C.c_long),
                ("basis_bytes", C.c_long), ("alg_bytes_per_call", C.c_double),
                ("flops_per_rhs", C.c_double), ("offline_seconds", C.c_double),
                ("coupling_a_flops_per_rhs", C.c_double), ("coupling_b_flops_per_rhs", C.c_double),
                ("tensor_core_phase1", C.c_int), ("kernel_variants", C.c_int),
                ("far_core_elems", C.c_long), ("p_theta_near", C.c_int * 3)]

    def as_dict(self):
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = list(v) if isinstance(v, C.Array) else v
        return out


class SurrogateOpts(C.Structure):
    _fields_ = [("hidden", C.c_int), ("steps", C.c_int), ("batch", C.c_int), ("lr", C.c_double),
                ("accept_tol", C.c_double), ("seed", C.c_ulonglong)]


class SurrogateReport(C.Structure):
    _fields_ = [("params", C.c_long), ("out_dim", C.c_long), ("loss_first", C.c_double),
                ("loss_last", C.c_double), ("val_err_net_rms", C.c_double), ("val_err_net_max", C.c_double),
                ("val_err_poly_rms", C.c_double), ("val_err_poly_max", C.c_double),
                ("targets_seconds", C.c_double), ("train_seconds", C.c_double), ("accepted", C.c_int)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


_H = C.c_void_p
_P = C.c_void_p
_F = C.POINTER(C.c_float)

_SIGS = {
    "ph_offline_build": (C.c_int, [C.POINTER(C.c_double), C.c_long, C.c_int, C.POINTER(BuildOpts),
                                   C.POINTER(_H)]),
    "ph_instantiate": (C.c_int, [_H, C.POINTER(C.c_double), _P]),
    "ph_instantiate_derivative": (C.c_int, [_H, C.POINTER(C.c_double), C.c_int, _P]),
    "ph_matvec": (C.c_int, [_H, _P, C.c_long, C.c_int, _P, C.c_long, _P]),
    "ph_matvec_host": (C.c_int, [_H, _P, C.c_long, C.c_int, _P, C.c_long, _P]),
    "ph_matvec_transpose": (C.c_int, [_H, _P, C.c_long, C.c_int, _P, C.c_long, _P]),
    "ph_matvec_batched": (C.c_int, [_H, C.POINTER(C.c_double), C.c_int, _P, C.c_long, C.c_int, _P, C.c_long,
                                    C.c_long, C.c_int, _P]),
    "ph_matvec_noalloc": (C.c_int, [_H, _P, C.c_long, C.c_int, _P, C.c_long, _P]),
    "ph_get_info": (C.c_int, [_H, C.POINTER(Info)]),
    "ph_save": (C.c_int, [_H, C.c_char_p]),
    "ph_load": (C.c_int, [C.c_char_p, C.c_int, C.POINTER(_H)]),
    "ph_destroy": (None, [_H]),
    "ph_last_error": (C.c_char_p, [_H]),
    "ph_far_cross_check": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int)]
                           + [C.POINTER(C.c_double)] * 6 + [C.c_double, C.c_int, C.POINTER(C.c_int),
                                                            C.POINTER(C.c_double)]),
    "ph_plan_adaptive": (C.c_int, [C.POINTER(C.c_double), C.c_long, C.c_int, C.c_int, C.c_double,
                                   C.POINTER(C.c_long), C.POINTER(C.c_int)]),
    "ph_plan": (C.c_int, [C.POINTER(C.c_double), C.c_long, C.c_int, C.c_int, C.c_double,
                          C.POINTER(C.c_long), C.POINTER(C.c_int)]),
    "ph_version": (C.c_char_p, []),
    "ph_profile_enable": (C.c_int, [_H, C.c_int]),
    "ph_set_overlap": (C.c_int, [_H, C.c_int]),
    "ph_set_tensor_cores": (C.c_int, [_H, C.c_int]),
    "ph_profile_read": (C.c_int, [_H, C.POINTER(C.c_double), C.POINTER(C.c_long)]),
    "ph_selftest_wait_bound": (C.c_int, [C.c_int, C.POINTER(C.c_double)]),
    "ph_check": (C.c_int, [_H, _P]),
    "ph_inject_alloc_failure": (C.c_int, [C.c_long]),
    "ph_selftest_timeout": (C.c_int, [_H, _P]),
    "ph_far_project": (C.c_int, [_H, C.POINTER(C.c_double), C.c_int, _P, _P]),
    "ph_instantiate_cores": (C.c_int, [_H, C.POINTER(C.c_double), _P, _P]),
    "ph_surrogate_train": (C.c_int, [_H, C.POINTER(C.c_double), C.c_int, C.POINTER(C.c_double), C.c_int,
                                     C.POINTER(SurrogateOpts), C.POINTER(SurrogateReport), _P]),
    "ph_surrogate_use": (C.c_int, [_H, C.c_int]),
    "ph_mlp_check": (C.c_int, [C.c_int, C.c_int, C.c_int, _F, C.c_int, _F, _F, _F, _F, C.POINTER(C.c_double)]),
    "ph_tt_cross_check": (C.c_int, [C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_double), C.c_double, C.c_int,
                                    C.POINTER(C.c_int), C.POINTER(C.c_double), C.POINTER(C.c_long)]),
}

for _name, (_res, _args) in _SIGS.items():
    _fn = getattr(_lib, _name)
    _fn.restype = _res
    _fn.argtypes = _args
    globals()[_name] = _fn

EXPORTED = tuple(_SIGS)

PROF_KINDS = ("instantiate", "gather", "near", "upsweep_leaf", "transfer_up", "coupling",
              "transfer_down", "far_h", "combine", "coupling_b")


class PHError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"libph status {status}: {msg}")
        self.status = status


def check(status, handle=None):
    if status != PH_OK:
        raise PHError(status, ph_last_error(handle).decode(errors="replace"))
    return status


def make_opts(d, theta_lo, theta_hi, degree, p_s, l_max, eta, tol, rank_cap=0, fmt="h2",
              prec="fp32", dedup=True, check_finite=False, near_tol=-1.0, device=0,
              coupling="explicit", near_shared=True, near_degree=None, compressor="svd") -> BuildOpts:
    o = BuildOpts()
    o.d = d
    o.dtheta = len(theta_lo)
    for k in range(len(theta_lo)):
        o.theta_lo[k] = float(theta_lo[k])
        o.theta_hi[k] = float(theta_hi[k])
        o.degree[k] = int(degree[k])
    o.p_s, o.l_max, o.eta, o.tol = int(p_s), int(l_max), float(eta), float(tol)
    o.near_tol = float(near_tol)
    o.rank_cap = int(rank_cap or 0)
    o.fmt = FORMATS[fmt]
    o.prec = PRECISIONS[prec]
    o.dedup = 1 if dedup else 0
    o.check_finite = 1 if check_finite else 0
    o.device = int(device)
    o.coupling = {"explicit": 0, "chain": 1}[coupling]
    o.near_unshared = 0 if near_shared else 1
    for k in range(len(theta_lo)):
        o.near_degree[k] = 0 if near_degree is None else int(near_degree[k])
    o.compressor = {"svd": 0, "cross": 1}[compressor]
    return o


def selftest_wait_bound(device=0):
    """ph_selftest_wait_bound: returns (status, seconds the device-side wait took)."""
    waited = C.c_double(0.0)
    st = ph_selftest_wait_bound(int(device), C.byref(waited))
    return st, waited.value


def plan(points, l_max, eta, leaf_size=None):
    """Host-only tree / block tree sizes (ph_plan, or ph_plan_adaptive with leaf_size); returns
    (counts dict, perm)."""
    P = np.ascontiguousarray(points, dtype=np.float64)
    n, d = P.shape
    counts = (C.c_long * 8)()
    perm = np.empty(n, dtype=np.int32)
    if leaf_size is None:
        check(ph_plan(P.ctypes.data_as(C.POINTER(C.c_double)), n, d, int(l_max), float(eta), counts,
                      perm.ctypes.data_as(C.POINTER(C.c_int))))
    else:
        check(ph_plan_adaptive(P.ctypes.data_as(C.POINTER(C.c_double)), n, d, int(leaf_size), float(eta), counts,
                               perm.ctypes.data_as(C.POINTER(C.c_int))))
    keys = ["nodes", "leaves", "near", "far", "far_keys", "near_entries", "max_near_per_leaf", "depth"]
    return dict(zip(keys, list(counts))), perm


class ParametricMatrix:
    """Owns one libph handle.  Device buffers are passed as raw pointers (torch's data_ptr())."""

    def __init__(self, points, kernel, opts: BuildOpts):
        import numpy as np
        P = np.ascontiguousarray(points, dtype=np.float64)
        self.n, self.d = P.shape
        self.prec = "fp32" if opts.prec == 1 else "fp64"
        self.dtheta = opts.dtheta
        h = _H()
        check(ph_offline_build(P.ctypes.data_as(C.POINTER(C.c_double)), self.n, KERNELS[kernel],
                               C.byref(opts), C.byref(h)))
        self.h = h

    @classmethod
    def load(cls, path, device=0):
        self = cls.__new__(cls)
        h = _H()
        check(ph_load(path.encode(), device, C.byref(h)))
        self.h = h
        inf = self.info()
        self.n, self.d, self.dtheta = inf["n"], inf["d"], inf["dtheta"]
        self.prec = "fp32" if inf["prec"] == 1 else "fp64"
        return self

    def info(self) -> dict:
        i = Info()
        check(ph_get_info(self.h, C.byref(i)), self.h)
        return i.as_dict()

    def instantiate(self, theta, stream=0):
        th = (C.c_double * 3)(*[float(t) for t in list(theta)[:3]])
        return check(ph_instantiate(self.h, th, C.c_void_p(stream)), self.h)

    def instantiate_derivative(self, theta, dim, stream=0):
        """ph_instantiate_derivative: the handle then applies dK_hat(theta)/dtheta_dim."""
        th = (C.c_double * 3)(*[float(t) for t in list(theta)[:3]])
        return check(ph_instantiate_derivative(self.h, th, int(dim), C.c_void_p(stream)), self.h)

    def matvec_ptr(self, x_ptr, ldx, m, y_ptr, ldy, stream=0):
        return check(ph_matvec(self.h, C.c_void_p(x_ptr), ldx, m, C.c_void_p(y_ptr), ldy,
                               C.c_void_p(stream)), self.h)

    def matvec_transpose_ptr(self, y_ptr, ldy, m, x_ptr, ldx, stream=0):
        """ph_matvec_transpose: X = K_hat(theta)^T Y (device pointers, column-major)."""
        return check(ph_matvec_transpose(self.h, C.c_void_p(y_ptr), ldy, m, C.c_void_p(x_ptr), ldx,
                                         C.c_void_p(stream)), self.h)

    def matvec_batched_ptr(self, thetas, x_ptr, ldx, m, y_ptr, ldy, stride_y, deriv=-1, stream=0):
        """ph_matvec_batched: Y_t = K_hat(theta_t) X (or its theta-derivative with deriv = 0)."""
        import numpy as np
        vals = np.ascontiguousarray(np.asarray(thetas, dtype=np.float64).ravel())  # d_theta = 1
        th = (C.c_double * vals.size)(*vals.tolist())
        return check(ph_matvec_batched(self.h, th, vals.size, C.c_void_p(x_ptr), ldx, m, C.c_void_p(y_ptr), ldy,
                                       stride_y, int(deriv), C.c_void_p(stream)), self.h)

    def matvec_noalloc_ptr(self, x_ptr, ldx, m, y_ptr, ldy, stream=0):
        """ph_matvec_noalloc: same result as matvec_ptr, workspace in the library's static array."""
        return check(ph_matvec_noalloc(self.h, C.c_void_p(x_ptr), ldx, m, C.c_void_p(y_ptr), ldy,
                                       C.c_void_p(stream)), self.h)

    def matvec_host_ptr(self, x_ptr, ldx, m, y_ptr, ldy, stream=0):
        return check(ph_matvec_host(self.h, C.c_void_p(x_ptr), ldx, m, C.c_void_p(y_ptr), ldy,
                                    C.c_void_p(stream)), self.h)

    def matvec(self, X, Y=None, stream=None):
        """Y = K_hat(theta) X for torch CUDA tensors X (n x m, column-major: X.t() contiguous)."""
        import torch
        if X.dim() == 1:
            X = X[:, None]
        n, m = X.shape
        Xc = X.t().contiguous() if not _colmajor(X) else X
        if Y is None:
            Y = torch.empty((m, n), dtype=X.dtype, device=X.device).t()
        s = torch.cuda.current_stream(X.device).cuda_stream if stream is None else stream
        self.matvec_ptr(Xc.data_ptr(), n, m, Y.data_ptr(), n, s)
        return Y

    def check(self, stream=0):
        """ph_check: synchronise and report a device wait that ran out in an earlier call."""
        return check(ph_check(self.h, C.c_void_p(stream)), self.h)

    def set_overlap(self, enable=True):
        return check(ph_set_overlap(self.h, 1 if enable else 0), self.h)

    def set_tensor_cores(self, enable=True):
        return check(ph_set_tensor_cores(self.h, 1 if enable else 0), self.h)

    def profile(self, enable=True):
        return check(ph_profile_enable(self.h, 1 if enable else 0), self.h)

    def profile_read(self) -> dict:
        """{kind: (milliseconds, launches)} since the last read (synchronises)."""
        ms = (C.c_double * len(PROF_KINDS))()
        la = (C.c_long * len(PROF_KINDS))()
        check(ph_profile_read(self.h, ms, la), self.h)
        return {k: (ms[i], la[i]) for i, k in enumerate(PROF_KINDS)}

    def far_project_ptr(self, thetas, out_ptr, stream=0):
        """Projected far cores H*_k(theta) of every class for each theta into the device buffer
        out_ptr (n_theta x info()["far_core_elems"] scalars of the handle's precision)."""
        th = np.ascontiguousarray(np.atleast_2d(np.asarray(thetas, float)))
        check(ph_far_project(self.h, th.ctypes.data_as(C.POINTER(C.c_double)), th.shape[0], out_ptr, stream),
              self.h)

    def instantiate_cores_ptr(self, theta, cores_ptr, stream=0):
        th = np.ascontiguousarray(np.atleast_1d(np.asarray(theta, float)))
        check(ph_instantiate_cores(self.h, th.ctypes.data_as(C.POINTER(C.c_double)), cores_ptr, stream), self.h)

    def surrogate_train(self, thetas_train, thetas_val, hidden=0, steps=0, batch=0, lr=0.0, accept_tol=0.0,
                        seed=1, stream=0) -> dict:
        """Train the far-field surrogate on the GPU (ph_surrogate_train); returns its report."""
        tt = np.ascontiguousarray(np.atleast_2d(np.asarray(thetas_train, float)))
        tv = np.ascontiguousarray(np.atleast_2d(np.asarray(thetas_val, float)))
        o = SurrogateOpts(int(hidden), int(steps), int(batch), float(lr), float(accept_tol), int(seed))
        r = SurrogateReport()
        check(ph_surrogate_train(self.h, tt.ctypes.data_as(C.POINTER(C.c_double)), tt.shape[0],
                                 tv.ctypes.data_as(C.POINTER(C.c_double)), tv.shape[0], C.byref(o), C.byref(r),
                                 stream), self.h)
        return r.as_dict()

    def surrogate_use(self, enable=True):
        check(ph_surrogate_use(self.h, 1 if enable else 0), self.h)

    def save(self, path):
        return check(ph_save(self.h, path.encode()), self.h)

    def close(self):
        if getattr(self, "h", None):
            ph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mlp_check(n_in, hidden, n_out, params, U, T):
    """One forward pass, loss and backward pass of the library's perceptron kernels on the current
    device (ph_mlp_check): returns (Y, grads, loss)."""
    p = np.ascontiguousarray(params, np.float32)
    U = np.ascontiguousarray(U, np.float32)
    T = np.ascontiguousarray(T, np.float32)
    B = U.shape[0]
    Y = np.empty((B, n_out), np.float32)
    g = np.empty_like(p)
    loss = C.c_double()
    fp = lambda a: a.ctypes.data_as(_F)
    check(ph_mlp_check(n_in, hidden, n_out, fp(p), B, fp(U), fp(T), fp(Y), fp(g), C.byref(loss)))
    return Y, g, loss.value


def tt_cross_check(tensor, eps, cap=0):
    """The library's TT-cross + TT-rounding of a dense tensor (ph_tt_cross_check, host only):
    returns (ranks, reconstructed tensor, entries evaluated)."""
    A = np.asfortranarray(tensor, dtype=np.float64)
    dims = np.array(A.shape, dtype=np.int32)
    ranks = np.zeros(A.ndim + 1, dtype=np.int32)
    out = np.zeros(A.size, dtype=np.float64)
    ev = C.c_long()
    flat = np.ascontiguousarray(A.ravel(order="F"))
    check(ph_tt_cross_check(A.ndim, dims.ctypes.data_as(C.POINTER(C.c_int)), flat.ctypes.data_as(C.POINTER(C.c_double)),
                            float(eps), int(cap), ranks.ctypes.data_as(C.POINTER(C.c_int)),
                            out.ctypes.data_as(C.POINTER(C.c_double)), C.byref(ev)))
    return ranks.tolist(), out.reshape(A.shape, order="F"), ev.value


def far_cross_check(kernel, s_box, t_box, theta_lo, theta_hi, degree, p_s, eps, cap=0):
    """The offline build's TT-cross of one far-field tensor (ph_far_cross_check, host only):
    returns (ranks, reconstructed tensor with modes (i_1..i_d, theta.., j_1..j_d))."""
    d = len(s_box[0])
    dt = len(theta_lo)
    arr = lambda v: np.ascontiguousarray(v, dtype=np.float64)
    s_lo, s_hi, t_lo, t_hi, lo, hi = (arr(s_box[0]), arr(s_box[1]), arr(t_box[0]), arr(t_box[1]), arr(theta_lo),
                                      arr(theta_hi))
    deg = np.ascontiguousarray(degree, dtype=np.int32)
    shape = [p_s] * d + [int(g) + 1 for g in degree] + [p_s] * d
    out = np.zeros(int(np.prod(shape)), dtype=np.float64)
    ranks = np.zeros(2 * d + dt + 1, dtype=np.int32)
    dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
    check(ph_far_cross_check(KERNELS[kernel], d, dt, int(p_s), deg.ctypes.data_as(C.POINTER(C.c_int)), dp(s_lo),
                             dp(s_hi), dp(t_lo), dp(t_hi), dp(lo), dp(hi), float(eps), int(cap),
                             ranks.ctypes.data_as(C.POINTER(C.c_int)), dp(out)))
    return ranks.tolist(), out.reshape(shape, order="F")


def _colmajor(X) -> bool:
    return X.dim() == 2 and X.stride(0) == 1 and X.stride(1) == X.shape[0]


def _autograd_function():
    """torch.autograd.Function for Y = K_hat(theta) X over one handle (built lazily so that importing
    this module does not import torch).  Every product runs in libph: forward ph_instantiate +
    ph_matvec; backward dX = ph_matvec_transpose(dY), and d theta_i = <dY, dK_hat/dtheta_i X> from
    ph_instantiate_derivative + ph_matvec (the derivative of the Lagrange weights, FP64 on the
    device), after which the handle is instantiated at theta again."""
    import torch

    class KhatApply(torch.autograd.Function):
        @staticmethod
        def forward(ctx, X, theta, A):
            th = [float(t) for t in theta.detach().cpu().reshape(-1)]
            stream = torch.cuda.current_stream(X.device).cuda_stream
            Xc = X.t().contiguous()  # column-major n x m
            n, m = X.shape
            Y = torch.empty((m, n), dtype=X.dtype, device=X.device)
            A.instantiate(th, stream)
            A.matvec_ptr(Xc.data_ptr(), n, m, Y.data_ptr(), n, stream)
            ctx.A, ctx.theta, ctx.dtype, ctx.tdev = A, th, theta.dtype, theta.device
            ctx.save_for_backward(Xc)
            return Y.t()

        @staticmethod
        def backward(ctx, dY):
            (Xc,) = ctx.saved_tensors
            A, th = ctx.A, ctx.theta
            m, n = Xc.shape
            stream = torch.cuda.current_stream(Xc.device).cuda_stream
            dYc = dY.t().contiguous()
            dX = dth = None
            if ctx.needs_input_grad[0]:
                out = torch.empty_like(dYc)
                A.instantiate(th, stream)
                A.matvec_transpose_ptr(dYc.data_ptr(), n, m, out.data_ptr(), n, stream)
                dX = out.t()
            if ctx.needs_input_grad[1]:
                g = []
                tmp = torch.empty_like(dYc)
                for i in range(len(th)):
                    A.instantiate_derivative(th, i, stream)
                    A.matvec_ptr(Xc.data_ptr(), n, m, tmp.data_ptr(), n, stream)
                    g.append(torch.sum(tmp.double() * dYc.double()))
                A.instantiate(th, stream)
                dth = torch.stack(g).to(device=ctx.tdev, dtype=ctx.dtype)
            return dX, dth, None

    return KhatApply


_KHAT = None


def khat_apply(A, X, theta):
    """Y = K_hat(theta) X (X: n x m CUDA tensor, theta: tensor of d_theta values), differentiable in X
    and theta through libph's adjoint and theta-derivative products."""
    global _KHAT
    if _KHAT is None:
        _KHAT = _autograd_function()
    return _KHAT.apply(X, theta, A)
