"""FP64 CPU oracle for the 1D periodic NUFFT / INUFFT (Gumerov & Duraiswami).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path never does, and this package shares no code with
the CUDA library (it does not import ``paper_1611_09379_gb300``).

What it computes (each a definition evaluated directly, see oracle.c):

* ``nudft_fwd``   g_j = sum_n c_n e^{i n y_j}                     (Eq. p1)
* ``kernel_fwd``  g_j = sum_k F_j G(y_j - x_k) f_k                 (Eq. p2, p4, p5)
* ``kernel_fwd_plain``  the same sum with Eq. p4 in plain binary64, the
                  paper's straightforward method, whose error for f = 1 is
                  the threshold error eps_th(N)            (Sec. 3.1)
* ``nudft_adj``   c'_n = sum_j e^{-i n y_j} g_j                    (adjoint of Eq. p1)
* ``kernel_adj``  u_k = sum_j conj(F_j) G(x_k - y_j) g_j           (adjoint of Eq. p4)
* ``logsin_C/D``  log-sums behind C_k and D_j                      (Eq. p8, reading c4)
* ``inverse_f``   f_k = sum_j C_k G(x_k - y_j) D_j g_j              (Eq. p6)
* ``inverse_absf`` a_k = sum_j |L_kj| |g_j|, the modulus sum of inverse_f
                  (normaliser of reading c16)
* ``inufft``      c = (1/N) DFT(inverse_f(g))                       (Eq. p1, p6)
* ``fft`` / ``dft``  radix-2 FFT and direct DFT                     (Eq. p1)
* ``exact_grid``  leaf index, nearest grid index k0 and offset delta of
                  y_j * N / (2 pi), in exact rational arithmetic   (Sec. 2.1)
* ``bernoulli``   exact Bernoulli numbers B_0..B_n                 (Eq. 10-12)
* ``lsq_dense``   c = argmin ||A c - g||, A_jn = e^{i n y_j}, by a dense
                  least-squares solve (LAPACK through numpy) for small N

Parity unpinned: none of the routines above; the paper's plotted values
(Figs. comp1, comp4-comp6) are absent from the text and nothing here
reproduces them.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
from fractions import Fraction

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into a shared library (gcc, -O2, OpenMP, no FMA contraction)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    flags = ["-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-std=gnu11"]
    if platform.machine() in ("x86_64", "AMD64"):
        flags.append("-mfma")  # hardware fma(); results identical to the libm call
    tmp = _LIB + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", *flags, _SRC, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        I = ctypes.c_int64
        sig = {
            "orc_nudft_fwd": [P, I, P, I, P, I, P],
            "orc_kernel_fwd": [P, I, P, I, P, I, P],
            "orc_kernel_fwd_plain": [P, I, P, I, P, I, P],
            "orc_cot_sum": [P, I, P, I, P],
            "orc_nudft_adj": [P, P, I, I, P, I, P],
            "orc_kernel_adj": [P, P, I, I, P, I, P],
            "orc_logsin_C": [P, I, I, P, I, P, P],
            "orc_logsin_D": [P, I, P, I, P, P],
            "orc_inverse_f": [P, P, I, I, P, P, P, P, P, I, P],
            "orc_inverse_absf": [P, P, I, I, P, P, P, I, P],
            "orc_dft": [P, I, ctypes.c_int, P],
            "orc_fft": [P, I, ctypes.c_int, P],
        }
        for name, argt in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = argt
            fn.restype = None
        lib.orc_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def num_threads() -> int:
    return int(_load().orc_num_threads())


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _idx(idx, n):
    if idx is None:
        return None, n
    a = np.ascontiguousarray(idx, dtype=np.int64)
    return a, a.size


# ---------------------------------------------------------------- forward

def nudft_fwd(c, y, idx=None) -> np.ndarray:
    """g_j = sum_{n=0}^{N-1} c_n e^{i n y_j} for j in idx (all if None)."""
    c, y = _c128(c), _f64(y)
    ia, n = _idx(idx, y.size)
    g = np.empty(n, np.complex128)
    _load().orc_nudft_fwd(_ptr(c), c.size, _ptr(y), y.size,
                          _ptr(ia) if ia is not None else None, n, _ptr(g))
    return g


def kernel_fwd(f, y, idx=None) -> np.ndarray:
    """g_j = sum_k F_j G(y_j - x_k) f_k, f on the uniform grid (Eq. p4)."""
    f, y = _c128(f), _f64(y)
    ia, n = _idx(idx, y.size)
    g = np.empty(n, np.complex128)
    _load().orc_kernel_fwd(_ptr(f), f.size, _ptr(y), y.size,
                           _ptr(ia) if ia is not None else None, n, _ptr(g))
    return g


def kernel_fwd_plain(f, y, idx=None) -> np.ndarray:
    """The paper's straightforward method (Sec. 3.1): g_j = sum_k K_jk f_k with
    K_jk of Eq. p4 evaluated literally in plain binary64 (no compensation);
    its error for f = 1 is the threshold error eps_th(N)."""
    f, y = _c128(f), _f64(y)
    ia, n = _idx(idx, y.size)
    g = np.empty(n, np.complex128)
    _load().orc_kernel_fwd_plain(_ptr(f), f.size, _ptr(y), y.size,
                                 _ptr(ia) if ia is not None else None, n, _ptr(g))
    return g


def cot_sum(f, y) -> np.ndarray:
    """h(y_j) = sum_k f_k cot((y_j - x_k)/2) for real f (Eq. p9 before splitting)."""
    f, y = _f64(f), _f64(y)
    h = np.empty(y.size, np.float64)
    _load().orc_cot_sum(_ptr(f), f.size, _ptr(y), y.size, _ptr(h))
    return h


def _dft_any(x, sign: int) -> np.ndarray:
    """fft() for power-of-two lengths, the direct dft() otherwise."""
    n = np.asarray(x).size
    return fft(x, sign) if n & (n - 1) == 0 else dft(x, sign)


def nufft_fwd(c, y, idx=None, route: str = "nudft") -> np.ndarray:
    """Forward NUFFT c_n -> g_j by either independent route."""
    if route == "nudft":
        return nudft_fwd(c, y, idx)
    f = _dft_any(c, +1)  # f_k = sum_n c_n e^{+i n x_k}
    return kernel_fwd(f, y, idx)


# ---------------------------------------------------------------- adjoint

def nudft_adj(g, y, N: int, idx=None) -> np.ndarray:
    """c'_n = sum_j e^{-i n y_j} g_j for n in idx (all N if None)."""
    g, y = _c128(g), _f64(y)
    ia, n = _idx(idx, N)
    c = np.empty(n, np.complex128)
    _load().orc_nudft_adj(_ptr(g), _ptr(y), y.size, N,
                          _ptr(ia) if ia is not None else None, n, _ptr(c))
    return c


def kernel_adj(g, y, N: int, idx=None) -> np.ndarray:
    """u_k = sum_j conj(F_j) G(x_k - y_j) g_j on the uniform grid."""
    g, y = _c128(g), _f64(y)
    ia, n = _idx(idx, N)
    u = np.empty(n, np.complex128)
    _load().orc_kernel_adj(_ptr(g), _ptr(y), y.size, N,
                           _ptr(ia) if ia is not None else None, n, _ptr(u))
    return u


def nufft_adj(g, y, N: int, route: str = "nudft") -> np.ndarray:
    if route == "nudft":
        return nudft_adj(g, y, N)
    return _dft_any(kernel_adj(g, y, N), -1)


# ---------------------------------------------------------------- inverse

def logsin_C(y, N: int, idx=None):
    """(lamC_k, nC_k): lamC_k = sum_l log|2 sin((x_k - y_l)/2)|, nC_k = #{y_l > x_k}."""
    y = _f64(y)
    ia, n = _idx(idx, N)
    lam = np.empty(n, np.float64)
    cnt = np.empty(n, np.int64)
    _load().orc_logsin_C(_ptr(y), y.size, N, _ptr(ia) if ia is not None else None,
                         n, _ptr(lam), _ptr(cnt))
    return lam, cnt


def logsin_D(y, idx=None):
    """(lamD_j, nD_j): lamD_j = -sum_{l!=j} log|2 sin((y_j - y_l)/2)|, nD_j = #{y_l > y_j}."""
    y = _f64(y)
    ia, n = _idx(idx, y.size)
    lam = np.empty(n, np.float64)
    cnt = np.empty(n, np.int64)
    _load().orc_logsin_D(_ptr(y), y.size, _ptr(ia) if ia is not None else None,
                         n, _ptr(lam), _ptr(cnt))
    return lam, cnt


def inverse_f(g, y, N: int, idx=None, lamD=None) -> np.ndarray:
    """f_k = sum_j C_k G(x_k - y_j) D_j g_j (Eq. p6, p8), M = N."""
    g, y = _c128(g), _f64(y)
    if y.size != N:
        raise ValueError("the Lagrange form needs M == N")
    ia, n = _idx(idx, N)
    lamC, nC = logsin_C(y, N, ia)
    if lamD is None:
        lamD = logsin_D(y)
    lD, nD = _f64(lamD[0]), np.ascontiguousarray(lamD[1], dtype=np.int64)
    f = np.empty(n, np.complex128)
    _load().orc_inverse_f(_ptr(g), _ptr(y), y.size, N, _ptr(lamC), _ptr(nC),
                          _ptr(lD), _ptr(nD), _ptr(ia) if ia is not None else None,
                          n, _ptr(f))
    return f


def inverse_absf(g, y, N: int, idx=None, lamD=None) -> np.ndarray:
    """a_k = sum_j |C_k G(x_k - y_j) D_j| |g_j| (the modulus of every term of
    inverse_f): the scale against which the inverse's matrix-vector product
    is compared on ill-conditioned point sets (reading c16)."""
    g, y = _c128(g), _f64(y)
    if y.size != N:
        raise ValueError("the Lagrange form needs M == N")
    ia, n = _idx(idx, N)
    lamC, _ = logsin_C(y, N, ia)
    if lamD is None:
        lamD = logsin_D(y)
    lD = _f64(lamD[0])
    a = np.empty(n, np.float64)
    _load().orc_inverse_absf(_ptr(g), _ptr(y), y.size, N, _ptr(lamC), _ptr(lD),
                             _ptr(ia) if ia is not None else None, n, _ptr(a))
    return a


def inufft(g, y, N: int) -> np.ndarray:
    """Square INUFFT g_j -> c_n: c = (1/N) sum_k f_k e^{-i n x_k} (Eq. p1) with f from Eq. p6."""
    f = inverse_f(g, y, N)
    return _dft_any(f, -1) / N


# ---------------------------------------------------------------- DFT / FFT

def dft(x, sign: int) -> np.ndarray:
    """out_n = sum_k x_k e^{sign 2 pi i n k / N} (direct, unscaled)."""
    x = _c128(x)
    out = np.empty_like(x)
    _load().orc_dft(_ptr(x), x.size, int(sign), _ptr(out))
    return out


def fft(x, sign: int) -> np.ndarray:
    """Radix-2 FFT, same convention as dft()."""
    x = _c128(x)
    n = x.size
    if n & (n - 1):
        raise ValueError("power-of-two length required")
    out = np.empty_like(x)
    _load().orc_fft(_ptr(x), n, int(sign), _ptr(out))
    return out


# ---------------------------------------------------------------- exact arithmetic

_PI_BITS = 480


def _pi_fixed(bits: int) -> int:
    """floor(pi * 2^bits) from Machin's formula pi = 16 atan(1/5) - 4 atan(1/239),
    evaluated in integer fixed point with guard bits."""
    guard = 32
    one = 1 << (bits + guard)

    def atan_inv(x: int) -> int:
        total, term, k, x2 = 0, one // x, 0, x * x
        while term:
            total += term // (2 * k + 1) if k % 2 == 0 else -(term // (2 * k + 1))
            term //= x2
            k += 1
        return total

    return (16 * atan_inv(5) - 4 * atan_inv(239)) >> guard


PI_FIXED = _pi_fixed(_PI_BITS)  # pi ~ PI_FIXED / 2^_PI_BITS, error < 2^-470


def exact_grid(y, N: int, B: int):
    """Exact grid coordinates of each y_j (Sec. 2.1, reading c3):

    Y_j = y_j N / (2 pi) evaluated with exact rationals (pi to 480 bits);
    leaf_j = floor(Y_j / (N/B)) mod B, k0_j = round(Y_j) mod N,
    delta_j = Y_j - round(Y_j) correctly rounded to binary64.
    Returns (leaf int64[M], k0 int64[M], delta float64[M]).
    """
    y = np.asarray(y, dtype=np.float64)
    s = N // B
    leaf = np.empty(y.size, np.int64)
    k0 = np.empty(y.size, np.int64)
    delta = np.empty(y.size, np.float64)
    R = 200  # fractional bits kept for Y
    for j, v in enumerate(y.tolist()):
        num, den = Fraction(v).as_integer_ratio()
        # Y * 2^R = num * N * 2^(PI_BITS + R) / (den * 2 * PI_FIXED)
        Yr = (num * N << (_PI_BITS + R)) // (den * 2 * PI_FIXED)
        Yint = Yr >> R
        leaf[j] = (Yint // s) % B
        kr = (Yr + (1 << (R - 1))) >> R  # round half up; ties cannot occur
        k0[j] = kr % N
        delta[j] = float(Fraction(Yr - (kr << R), 1 << R))
    return leaf, k0, delta


def binning(y, N: int, B: int):
    """Binning reference (Sec. 2.1, the "data structure" of Sec. 3.3, reading
    c3): (perm, leaf_start, leaf) with the points grouped by their exact leaf
    floor(y B / (2 pi)) and, inside a leaf, kept in their original order (a
    stable counting sort by leaf)."""
    leaf, _, _ = exact_grid(y, N, B)
    perm = np.argsort(leaf, kind="stable").astype(np.int64)
    leaf_start = np.searchsorted(leaf[perm], np.arange(B + 1), side="left").astype(np.int64)
    return perm, leaf_start, leaf


def bernoulli(nmax: int):
    """Exact Bernoulli numbers B_0..B_nmax (B_1 = -1/2) by the Akiyama-Tanigawa
    algorithm, as Fractions."""
    out = []
    a = [Fraction(0)] * (nmax + 1)
    for m in range(nmax + 1):
        a[m] = Fraction(1, m + 1)
        for j in range(m, 0, -1):
            a[j - 1] = j * (a[j - 1] - a[j])
        out.append(a[0])
    # Akiyama-Tanigawa yields B_1 = +1/2; use the B_1 = -1/2 convention
    if nmax >= 1:
        out[1] = -out[1]
    return out


# ---------------------------------------------------------------- least squares

def nudft_matrix(y, N: int) -> np.ndarray:
    """A_jn = e^{i n y_j} (M x N) with the phase n*y_j rounded once in FP64
    (error below N * 2^-50, i.e. under 1e-12 for N <= 1024)."""
    y = np.asarray(y, dtype=np.float64)
    n = np.arange(N, dtype=np.float64)
    return np.exp(1j * np.multiply.outer(y, n))


def lsq_dense(g, y, N: int, w=None) -> np.ndarray:
    """Weighted least squares argmin sum_j w_j |(A c)_j - g_j|^2 by a dense solve
    (problem (ii) of Sec. 2 for M > N); N <= 1024."""
    if N > 1024:
        raise ValueError("dense least squares is for N <= 1024")
    A = nudft_matrix(y, N)
    g = np.asarray(g, dtype=np.complex128)
    if w is not None:
        sw = np.sqrt(np.asarray(w, dtype=np.float64))
        A = A * sw[:, None]
        g = g * sw
    c, *_ = np.linalg.lstsq(A, g, rcond=None)
    return c


# ---------------------------------------------------------------- error norms

def rel_l2(x, ref) -> float:
    x = np.asarray(x)
    ref = np.asarray(ref)
    den = np.linalg.norm(ref)
    return float(np.linalg.norm(x - ref) / (den if den > 0 else 1.0))
