"""The learned surrogate of the far-field cores: a two-hidden-layer perceptron in FP64.

Test infrastructure only (see ``oracle/__init__.py``).

The paper lists other parametric approximations as future work (§7); the network here is the
one the library trains on the GPU, written out plainly so that its forward values and its
gradients can be checked.  For a parameter theta in the box prod [lo_i, hi_i]:

    u   = 2 (theta - lo) / (hi - lo) - 1                (the box mapped to [-1, 1]^d_theta)
    h_1 = gelu(W_1 u + b_1)                              (hidden width n_h)
    h_2 = gelu(W_2 h_1 + b_2)
    y   = W_3 h_2 + b_3                                  (one output per stored core entry)

with gelu(x) = x Phi(x), Phi the standard normal distribution function (the exact GELU, written
with erfc, which keeps Phi accurate in the left tail).  Weights are row-major (out x in): y = W x.  The loss over a batch of B samples with
targets T (B x n_out) is L = sum (Y - T)^2 / (2 B n_out).

Pins (tests/test_oracle_mlp.py): gelu against SciPy's normal distribution function and a few
printed values of Phi; the network's gradients against central differences of the loss; a
network whose second layer is zero returns b_3; the Adam step against its closed form after one
step (Kingma & Ba 2015, Alg. 1: the first step moves every weight by lr * sign(g)).
"""
from __future__ import annotations

import math

import numpy as np

_ERFC = np.vectorize(math.erfc, otypes=[float])


def _Phi(x):
    """Standard normal distribution function, Phi(x) = erfc(-x / sqrt 2) / 2."""
    return 0.5 * _ERFC(-x / math.sqrt(2.0))


def gelu(x):
    """x Phi(x)."""
    x = np.asarray(x, float)
    return x * _Phi(x)


def gelu_grad(x):
    """d/dx [x Phi(x)] = Phi(x) + x phi(x), phi the standard normal density."""
    x = np.asarray(x, float)
    Phi = _Phi(x)
    phi = np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)
    return Phi + x * phi


def normalise(theta, lo, hi):
    """The parameter box mapped to [-1, 1]^d_theta (rows of theta are samples)."""
    theta = np.atleast_2d(np.asarray(theta, float))
    lo = np.asarray(lo, float)
    hi = np.asarray(hi, float)
    return 2.0 * (theta - lo) / (hi - lo) - 1.0


def init_params(n_in, n_h, n_out, seed):
    """Weights ~ N(0, 1 / fan_in) (a GELU network keeps unit-scale activations), zero biases."""
    rng = np.random.default_rng(seed)
    return {
        "W1": rng.standard_normal((n_h, n_in)) / math.sqrt(n_in), "b1": np.zeros(n_h),
        "W2": rng.standard_normal((n_h, n_h)) / math.sqrt(n_h), "b2": np.zeros(n_h),
        "W3": rng.standard_normal((n_out, n_h)) / math.sqrt(n_h), "b3": np.zeros(n_out),
    }


def forward(params, U):
    """Y (B x n_out) for inputs U (B x n_in, already normalised) and the intermediate values."""
    U = np.atleast_2d(np.asarray(U, float))
    a1 = U @ params["W1"].T + params["b1"]
    h1 = gelu(a1)
    a2 = h1 @ params["W2"].T + params["b2"]
    h2 = gelu(a2)
    Y = h2 @ params["W3"].T + params["b3"]
    return Y, {"U": U, "a1": a1, "h1": h1, "a2": a2, "h2": h2}


def loss(params, U, T):
    Y, _ = forward(params, U)
    B, n_out = Y.shape
    return float(np.sum((Y - T) ** 2) / (2.0 * B * n_out))


def backward(params, cache, dY):
    """Gradients of a scalar whose derivative with respect to Y is dY (backpropagation through
    the three affine maps and the two GELUs)."""
    g = {}
    g["W3"] = dY.T @ cache["h2"]
    g["b3"] = dY.sum(axis=0)
    dh2 = dY @ params["W3"]
    da2 = dh2 * gelu_grad(cache["a2"])
    g["W2"] = da2.T @ cache["h1"]
    g["b2"] = da2.sum(axis=0)
    dh1 = da2 @ params["W2"]
    da1 = dh1 * gelu_grad(cache["a1"])
    g["W1"] = da1.T @ cache["U"]
    g["b1"] = da1.sum(axis=0)
    return g


def loss_and_grad(params, U, T):
    Y, cache = forward(params, U)
    B, n_out = Y.shape
    L = float(np.sum((Y - T) ** 2) / (2.0 * B * n_out))
    return L, backward(params, cache, (Y - T) / (B * n_out))


def adam_step(params, grads, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One step of Adam (Kingma & Ba 2015, Alg. 1) on every array of params, in place; state holds
    the step count and the two moment estimates."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in params:
        m = state.setdefault("m_" + k, np.zeros_like(params[k]))
        v = state.setdefault("v_" + k, np.zeros_like(params[k]))
        m *= beta1
        m += (1.0 - beta1) * grads[k]
        v *= beta2
        v += (1.0 - beta2) * grads[k] ** 2
        mhat = m / (1.0 - beta1 ** t)
        vhat = v / (1.0 - beta2 ** t)
        params[k] -= lr * mhat / (np.sqrt(vhat) + eps)
    return params
