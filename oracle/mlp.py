"""FP64 reference of the density-compensation network (test infrastructure).

w = softplus(z), z = W3 . gelu(W2 gelu(W1 x + b1) + b2) + b3, gelu(x) =
x (1 + erf(x / sqrt 2)) / 2; loss = mean_i (log w_i - t_i)^2.  Parameters in
the library's layout W1[64][8] b1[64] W2[64][64] b2[64] W3[64] b3.  The
gradient is the chain rule written out; it is pinned by central finite
differences, the forward pass by weights with closed-form outputs (tabulated
normal distribution function), and the density fixed point by a dense
Frobenius least-squares solve and the equispaced closed form w = 1, all in
tests/test_oracle_pins.py.
"""
import numpy as np
from scipy.special import erf

SIZES = [("W1", (64, 8)), ("b1", (64,)), ("W2", (64, 64)), ("b2", (64,)), ("W3", (64,)), ("b3", ())]
NPARAM = 4801


def unpack(p):
    p = np.asarray(p, np.float64)
    out, o = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape)) if shape else 1
        out[name] = p[o:o + n].reshape(shape) if shape else p[o]
        o += n
    return out


def _gelu(x):
    return 0.5 * x * (1.0 + erf(x / np.sqrt(2.0)))


def _gelu_d(x):
    return 0.5 * (1.0 + erf(x / np.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / np.sqrt(2 * np.pi)


def _softplus(z):
    return np.where(z > 30, z, np.log1p(np.exp(np.minimum(z, 30))))


def forward(p, X):
    q = unpack(p)
    a1 = X @ q["W1"].T + q["b1"]
    h1 = _gelu(a1)
    a2 = h1 @ q["W2"].T + q["b2"]
    h2 = _gelu(a2)
    z = h2 @ q["W3"] + q["b3"]
    return _softplus(z)


def loss(p, X, t):
    return float(np.mean((np.log(forward(p, X)) - t) ** 2))


def grad(p, X, t):
    q = unpack(p)
    n = X.shape[0]
    a1 = X @ q["W1"].T + q["b1"]
    h1 = _gelu(a1)
    a2 = h1 @ q["W2"].T + q["b2"]
    h2 = _gelu(a2)
    z = h2 @ q["W3"] + q["b3"]
    w = _softplus(z)
    e = np.log(w) - t
    dz = 2.0 * e / n / w / (1.0 + np.exp(-z))
    d2 = (dz[:, None] * q["W3"][None, :]) * _gelu_d(a2)
    d1 = (d2 @ q["W2"]) * _gelu_d(a1)
    g = [d1.T @ X, d1.sum(0), d2.T @ h1, d2.sum(0), h2.T @ dz, dz.sum()]
    return np.concatenate([np.ravel(x) for x in g]), float(np.mean(e * e))


def dcf_fixed_point(y, N: int, iters: int = 300):
    """Reference of the density-compensation targets: w_i <- w_i N / sum_j
    |D_N(y_i - y_j)|^2 w_j from w = 1 (FP64, dense), |D_N(t)|^2 =
    sin^2(N t/2) / sin^2(t/2) with value N^2 at t = 0; returns
    log(max(w / mean w, 1e-4))."""
    y = np.asarray(y, np.float64)
    t = y[:, None] - y[None, :]
    s = np.sin(0.5 * t)
    small = np.abs(s) < 1e-12
    K = (np.sin(0.5 * N * t) / np.where(small, 1.0, s)) ** 2
    K[small] = float(N) * N
    w = np.ones(y.size)
    for _ in range(iters):
        w = w * N / (K @ w)
    return np.log(np.maximum(w / w.mean(), 1e-4))
