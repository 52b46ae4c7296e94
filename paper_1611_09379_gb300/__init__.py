"""Python binding of the GB300 FMM-based NUFFT / INUFFT library (libnufft_gb300.so).

Argument marshalling only: every step of every transform runs in the CUDA
kernels behind the C ABI of ``include/nufft.h``.  PyTorch supplies device
memory and streams.  There is no CPU fallback: if the shared library has not
been built (``paper_1611_09379_gb300.build.build()``), importing raises.

    import torch, paper_1611_09379_gb300 as nf
    y = torch.rand(M, dtype=torch.float64, device="cuda") * 2 * math.pi
    plan = nf.Plan(N, y, eps=1e-12, prec=nf.FP64)
    g = plan.forward(c)            # g_j = sum_n c_n e^{i n y_j}
    c2 = plan.adjoint(g)           # c2_n = sum_j e^{-i n y_j} g_j
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnufft_gb300.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        "libnufft_gb300.so is missing: build it with "
        "`python -m paper_1611_09379_gb300.build` (nvcc, sm_103a)")

_lib = ctypes.CDLL(LIB_PATH)

OK, EINVAL, ENOMEM, ECUDA, EILLCOND, ENOTCONV, ETIMEOUT, ENOTSUP = range(8)
STAGES = ("fft", "p2m", "m2m", "level2", "m2l", "targets", "other")
FP64, MIXED = 0, 1
IO_C64 = 0x1
WANT_INVERSE = 0x2
NO_GRAPH = 0x4
ADAPTIVE = 0x8

# every symbol declared in include/nufft.h
SYMBOLS = [
    "nufft_strerror", "nufft_version", "nufft_choose_params", "nufft_plan_create",
    "nufft_plan_destroy", "nufft_plan_info", "nufft_plan_params", "nufft_plan_sync",
    "nufft_plan_points", "nufft_plan_inverse_coeffs",
    "nufft_plan_set_stream", "nufft_plan_profile", "nufft_plan_stats",
    "nufft_plan_exec_fwd",
    "nufft_plan_exec_adj", "nufft_plan_exec_inv", "nufft_fwd", "nufft_adj", "inufft",
    "nufft_fwd_noalloc", "nufft_plan_solve_lsq", "nufft_plan_dcf_features",
    "nufft_dcf_features_sorted", "nufft_dcf_targets", "nufft_mlp_create", "nufft_mlp_destroy",
    "nufft_mlp_num_params", "nufft_mlp_set_params", "nufft_mlp_get_params", "nufft_mlp_infer",
    "nufft_mlp_grad", "nufft_mlp_train_step", "nufft_multi_create", "nufft_multi_exec_fwd",
    "nufft_multi_destroy", "nufft_autotune", "nufft_plan_dcf_weights", "nufft_diag_rcp",
    "nufft_diag_pipe_rates", "nufft_eps_threshold", "nufft_adaptive_depths",
    "nufft_plan_adaptive",
]


class Params(ctypes.Structure):
    _fields_ = [("lmax", ctypes.c_int), ("p", ctypes.c_int), ("q", ctypes.c_int),
                ("batch", ctypes.c_int), ("tc_level", ctypes.c_int), ("tc_near", ctypes.c_int)]


class TuneTrial(ctypes.Structure):
    _fields_ = [("params", Params), ("ms", ctypes.c_double), ("err", ctypes.c_double),
                ("accepted", ctypes.c_int)]


class LsqInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("checks", ctypes.c_int), ("resid", ctypes.c_double),
                ("resid_w", ctypes.c_double), ("data_resid", ctypes.c_double),
                ("hist", ctypes.POINTER(ctypes.c_double)), ("hist_cap", ctypes.c_int)]


OP_FWD, OP_ADJ, OP_INV = 0x1, 0x2, 0x4

_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_lib.nufft_strerror.restype = ctypes.c_char_p
_lib.nufft_strerror.argtypes = [ctypes.c_int]
_lib.nufft_version.restype = ctypes.c_int
_lib.nufft_choose_params.argtypes = [_I64, _I64, ctypes.c_double, ctypes.c_int, ctypes.POINTER(Params)]
_lib.nufft_plan_create.argtypes = [ctypes.POINTER(_P), _I64, _I64, _P, ctypes.c_double, ctypes.c_int,
                                   ctypes.POINTER(Params), ctypes.c_uint, _P]
_lib.nufft_plan_destroy.argtypes = [_P]
_lib.nufft_plan_info.argtypes = [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                 ctypes.POINTER(ctypes.c_int)]
_lib.nufft_plan_params.argtypes = [_P, ctypes.POINTER(Params)]
_lib.nufft_plan_sync.argtypes = [_P]
_lib.nufft_plan_set_stream.argtypes = [_P, _P]
_lib.nufft_plan_points.argtypes = [_P, _P, _P, _P, _P]
_lib.nufft_plan_profile.argtypes = [_P, ctypes.c_int]
_lib.nufft_multi_create.argtypes = [ctypes.POINTER(_P), ctypes.c_int, _P, _P, _P, ctypes.c_double,
                                    ctypes.c_int, _P, ctypes.c_uint, _P]
_lib.nufft_multi_exec_fwd.argtypes = [_P, _P, _P]
_lib.nufft_multi_destroy.argtypes = [_P]
_lib.nufft_plan_dcf_features.argtypes = [_P, _P]
_lib.nufft_dcf_features_sorted.argtypes = [_P, _I64, _I64, _P, _P]
_lib.nufft_dcf_targets.argtypes = [_P, _I64, _I64, _I64, ctypes.c_int, _P, _P]
_lib.nufft_mlp_create.argtypes = [ctypes.POINTER(_P)]
_lib.nufft_mlp_destroy.argtypes = [_P]
_lib.nufft_mlp_set_params.argtypes = [_P, _P, ctypes.c_int]
_lib.nufft_mlp_get_params.argtypes = [_P, _P]
_lib.nufft_mlp_infer.argtypes = [_P, _P, _I64, _P, _P]
_lib.nufft_mlp_grad.argtypes = [_P, _P, _P, _I64, _P, _P, _P]
_lib.nufft_mlp_train_step.argtypes = [_P, _P, _P, _I64, ctypes.c_float, _P, _P]
_lib.nufft_plan_solve_lsq.argtypes = [_P, _P, _P, ctypes.c_uint, ctypes.c_double, ctypes.c_int,
                                      ctypes.c_int, _P, ctypes.POINTER(LsqInfo)]
LSQ_WEIGHTED = 0x1
_lib.nufft_plan_dcf_weights.argtypes = [_P, _P, _P]
_lib.nufft_eps_threshold.argtypes = [_I64]
_lib.nufft_eps_threshold.restype = ctypes.c_double
_lib.nufft_diag_rcp.argtypes = [_P, _I64, _P, _P, _P]
_lib.nufft_diag_pipe_rates.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), _P]
_lib.nufft_plan_stats.argtypes = [_P, _P, _P]
_lib.nufft_autotune.argtypes = [_I64, _I64, _P, ctypes.c_double, ctypes.c_int, ctypes.c_uint,
                                ctypes.c_int, ctypes.c_uint, ctypes.c_int, ctypes.POINTER(Params),
                                ctypes.POINTER(TuneTrial), ctypes.c_int,
                                ctypes.POINTER(ctypes.c_int), _P]
_lib.nufft_plan_inverse_coeffs.argtypes = [_P, _P, _P, ctypes.POINTER(ctypes.c_double)]
_lib.nufft_adaptive_depths.argtypes = [_P, _I64, _I64, ctypes.c_int, _P]
_lib.nufft_plan_adaptive.argtypes = [_P, ctypes.POINTER(ctypes.c_int), _P]
for _n in ("nufft_plan_exec_fwd", "nufft_plan_exec_adj", "nufft_plan_exec_inv"):
    getattr(_lib, _n).argtypes = [_P, _P, _P]
for _n in ("nufft_fwd", "nufft_fwd_noalloc"):
    getattr(_lib, _n).argtypes = [_P, _I64, _P, _I64, ctypes.c_double, ctypes.c_int, ctypes.c_uint, _P, _P]
for _n in ("nufft_adj", "inufft"):
    getattr(_lib, _n).argtypes = [_P, _P, _I64, _I64, ctypes.c_double, ctypes.c_int, ctypes.c_uint, _P, _P]
for _n in SYMBOLS:
    if _n not in ("nufft_strerror", "nufft_version", "nufft_eps_threshold"):
        getattr(_lib, _n).restype = ctypes.c_int


class NufftError(RuntimeError):
    def __init__(self, code: int, where: str = ""):
        self.code = code
        msg = _lib.nufft_strerror(code).decode()
        super().__init__(f"{where}: {msg} (status {code})" if where else msg)


def _check(rc: int, where: str):
    if rc != OK:
        raise NufftError(rc, where)


def strerror(code: int) -> str:
    return _lib.nufft_strerror(code).decode()


def version() -> int:
    return _lib.nufft_version()


MACHINE_EPS = 0.0  # eps value of the machine-precision mode (FP64)


def eps_threshold(N: int) -> float:
    """Threshold ("machine precision") error of the FP64 path for N coefficients
    (Sec. 3.1), the accuracy eps = 0 prescribes."""
    v = _lib.nufft_eps_threshold(int(N))
    if v < 0:
        raise NufftError(EINVAL, "nufft_eps_threshold")
    return v


def adaptive_depths(leaf_start, s: int):
    """Extra tree levels of each leaf under the adaptive rule (host only):
    (max depth, int32 array of B depths) from the B + 1 leaf starts (numpy)
    and the grid points per leaf s."""
    import numpy as np
    st = np.ascontiguousarray(leaf_start, dtype=np.int32)
    B = st.size - 1
    dep = np.empty(max(B, 1), dtype=np.int32)
    D = _lib.nufft_adaptive_depths(st.ctypes.data, B, int(st[-1]), int(s), dep.ctypes.data)
    if D < 0:
        raise NufftError(EINVAL, "nufft_adaptive_depths")
    return D, dep[:B]


def choose_params(N: int, M: int, eps: float, prec: int = FP64, lmax: int = 0, p: int = 0, q: int = 0):
    """(lmax, p, q) the library would use (host only, no GPU needed)."""
    prm = Params(lmax, p, q, 1, 0, 0)
    _check(_lib.nufft_choose_params(N, M, eps, prec, ctypes.byref(prm)), "nufft_choose_params")
    return prm.lmax, prm.p, prm.q


def choose_params_full(N: int, M: int, eps: float, prec: int = FP64, lmax: int = 0, p: int = 0,
                       q: int = 0, batch: int = 1, tc_level: int = 0, tc_near: int = 0) -> dict:
    """Every resolved parameter (host only), as a dict."""
    prm = Params(lmax, p, q, batch, tc_level, tc_near)
    _check(_lib.nufft_choose_params(N, M, eps, prec, ctypes.byref(prm)), "nufft_choose_params")
    return {"lmax": prm.lmax, "p": prm.p, "q": prm.q, "batch": prm.batch, "tc_level": prm.tc_level,
            "tc_near": prm.tc_near}


def _torch():
    import torch
    return torch


def _stream_handle(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return _P(s.cuda_stream)


def _dev_ptr(t, dtype, n, what):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{what} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{what} must have dtype {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    if t.numel() != n:
        raise ValueError(f"{what} must have {n} elements, got {t.numel()}")
    return _P(t.data_ptr())


class Plan:
    """A transform plan: the binned point set and FMM workspace (Sec. 3.3).

    N: grid size (power of two); y: CUDA float64 tensor of M points in [0, 2 pi).
    prec: FP64 or MIXED; io: 'c128' or 'c64' element type of c and g;
    inverse=True precomputes C_k, D_j for :meth:`inverse` (needs M == N).
    lmax / p / q override the automatic parameters (0 = automatic).
    batch: signals sharing the points; exec calls take [batch, N] / [batch, M].
    tc_level: first tree level whose M2L runs on the tensor cores (MIXED only;
    0 = automatic, -1 = never).
    tc_near: batched forward near field on the tensor cores (MIXED, batch a
    multiple of 64; 0 = automatic, -1 = never).
    graphs: replay exec sequences as CUDA graphs (captured per buffer set).
    adaptive: refine the leaves that hold more targets than the mean for the
    forward transform (one signal; see :meth:`adaptive`).
    """

    def __init__(self, N: int, y, eps: float = 1e-12, prec: int = FP64, io: str = "c128",
                 inverse: bool = False, lmax: int = 0, p: int = 0, q: int = 0, batch: int = 1,
                 tc_level: int = 0, tc_near: int = 0, graphs: bool = True, stream=None,
                 adaptive: bool = False):
        torch = _torch()
        self.N = int(N)
        self.M = int(y.numel())
        self.prec = prec
        self.io = io
        self.cdtype = torch.complex64 if io == "c64" else torch.complex128
        self.batch = int(batch)
        flags = ((IO_C64 if io == "c64" else 0) | (WANT_INVERSE if inverse else 0) |
                 (0 if graphs else NO_GRAPH) | (ADAPTIVE if adaptive else 0))
        self._stream = stream
        h = _P()
        prm = Params(lmax, p, q, self.batch, tc_level, tc_near)
        yp = _dev_ptr(y, torch.float64, self.M, "y")
        _check(_lib.nufft_plan_create(ctypes.byref(h), self.N, self.M, yp, eps, prec,
                                      ctypes.byref(prm), flags, _stream_handle(stream)),
               "nufft_plan_create")
        self._h = h
        self.device = y.device

    def info(self):
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(_lib.nufft_plan_info(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
               "nufft_plan_info")
        return {"lmax": a.value, "p": b.value, "q": c.value}

    def params(self):
        """Every resolved parameter of the plan (lmax, p, q, batch, tc_level)."""
        prm = Params()
        _check(_lib.nufft_plan_params(self._h, ctypes.byref(prm)), "nufft_plan_params")
        return {"lmax": prm.lmax, "p": prm.p, "q": prm.q, "batch": prm.batch,
                "tc_level": prm.tc_level, "tc_near": prm.tc_near}

    def adaptive(self):
        """(levels, counts): the largest extra depth of the adaptive tree (0:
        uniform) and the number of targets refined by 0..3 levels."""
        lv = ctypes.c_int()
        cnt = (ctypes.c_int64 * 4)()
        _check(_lib.nufft_plan_adaptive(self._h, ctypes.byref(lv), ctypes.cast(cnt, _P)),
               "nufft_plan_adaptive")
        return lv.value, [int(v) for v in cnt]

    def sync(self):
        """Wait for the plan's stream; raises NufftError(ETIMEOUT) if a bounded
        device wait gave up since the last call (outputs then invalid)."""
        _check(_lib.nufft_plan_sync(self._h), "nufft_plan_sync")

    def points(self):
        """The binned point set: (perm, leaf_start, k0, delta) as CUDA tensors."""
        torch = _torch()
        B = 1 << self.info()["lmax"]
        perm = torch.empty(self.M, dtype=torch.int32, device=self.device)
        start = torch.empty(B + 1, dtype=torch.int32, device=self.device)
        k0 = torch.empty(self.M, dtype=torch.int32, device=self.device)
        delta = torch.empty(self.M, dtype=torch.float64, device=self.device)
        _check(_lib.nufft_plan_points(self._h, _P(perm.data_ptr()), _P(start.data_ptr()),
                                      _P(k0.data_ptr()), _P(delta.data_ptr())), "nufft_plan_points")
        return perm, start, k0, delta

    def inverse_coeffs(self):
        """(Ct, Dt, Lambda): C_k e^Lambda / N and D_j e^-Lambda / 2 (sorted points)."""
        torch = _torch()
        Ct = torch.empty(self.N, dtype=torch.float64, device=self.device)
        Dt = torch.empty(self.M, dtype=torch.complex128, device=self.device)
        lam = ctypes.c_double()
        _check(_lib.nufft_plan_inverse_coeffs(self._h, _P(Ct.data_ptr()), _P(Dt.data_ptr()),
                                              ctypes.byref(lam)), "nufft_plan_inverse_coeffs")
        return Ct, Dt, lam.value

    def profile(self, enable: bool = True):
        """Enable per-stage CUDA-event timing (resets the accumulated stats)."""
        _check(_lib.nufft_plan_profile(self._h, 1 if enable else 0), "nufft_plan_profile")

    def stats(self):
        """{stage: (ms, launches)} accumulated since profile() (synchronises)."""
        ms = (ctypes.c_double * len(STAGES))()
        nl = (ctypes.c_int64 * len(STAGES))()
        _check(_lib.nufft_plan_stats(self._h, ctypes.cast(ms, _P), ctypes.cast(nl, _P)),
               "nufft_plan_stats")
        return {name: (ms[i], nl[i]) for i, name in enumerate(STAGES)}

    def set_stream(self, stream):
        self._stream = stream
        _check(_lib.nufft_plan_set_stream(self._h, _stream_handle(stream)), "nufft_plan_set_stream")

    def _out(self, n, out):
        torch = _torch()
        if out is None:
            shape = (n,) if self.batch == 1 else (self.batch, n)
            out = torch.empty(shape, dtype=self.cdtype, device=self.device)
        return out

    def forward(self, c, out=None):
        """g_j = sum_n c_n e^{i n y_j} (asynchronous on the plan's stream)."""
        g = self._out(self.M, out)
        B = self.batch
        _check(_lib.nufft_plan_exec_fwd(self._h, _dev_ptr(c, self.cdtype, B * self.N, "c"),
                                        _dev_ptr(g, self.cdtype, B * self.M, "g")), "nufft_plan_exec_fwd")
        return g

    def adjoint(self, g, out=None):
        """c_n = sum_j e^{-i n y_j} g_j."""
        c = self._out(self.N, out)
        B = self.batch
        _check(_lib.nufft_plan_exec_adj(self._h, _dev_ptr(g, self.cdtype, B * self.M, "g"),
                                        _dev_ptr(c, self.cdtype, B * self.N, "c")), "nufft_plan_exec_adj")
        return c

    def inverse(self, g, out=None):
        """Band-limited c with sum_n c_n e^{i n y_j} = g_j (M == N, Eq. p6/p8)."""
        c = self._out(self.N, out)
        B = self.batch
        _check(_lib.nufft_plan_exec_inv(self._h, _dev_ptr(g, self.cdtype, B * self.M, "g"),
                                        _dev_ptr(c, self.cdtype, B * self.N, "c")), "nufft_plan_exec_inv")
        return c

    def solve_lsq(self, g, w=None, tol: float = 1e-8, maxit: int = 500, out=None, check=True,
                  check_every: int = 0, weighted: bool = False):
        """Least-squares coefficients c = argmin sum_j |(A c)_j - g_j|^2 by CG on
        the normal equations; weights w (density compensation) precondition
        them, or with weighted=True define the weighted equations A^H W A c =
        A^H W g instead.  Stopped when the unweighted normal-equation residual
        ||A^H (g - A c)|| / ||A^H g||, recomputed from c, is <= tol.  Returns
        (c, iterations, that residual); the full report (iters, checks, resid,
        resid_w, data_resid, history of the stopping test at every check) is
        kept in ``self.lsq_info``.  Raises on non-convergence unless
        check=False."""
        torch = _torch()
        c = self._out(self.N, out)
        wp = None
        if w is not None:
            wp = _dev_ptr(w, torch.float32, self.M, "w")
        info = LsqInfo()
        every = int(check_every) if check_every > 0 else 16
        cap = maxit // every + 2
        hist = (ctypes.c_double * cap)()
        info.hist = ctypes.cast(hist, ctypes.POINTER(ctypes.c_double))
        info.hist_cap = cap
        rc = _lib.nufft_plan_solve_lsq(self._h, _dev_ptr(g, self.cdtype, self.M, "g"), wp,
                                       LSQ_WEIGHTED if weighted else 0, tol, maxit,
                                       int(check_every), _dev_ptr(c, self.cdtype, self.N, "c"),
                                       ctypes.byref(info))
        self.lsq_info = {k: getattr(info, k) for k in ("iters", "checks", "resid", "resid_w",
                                                       "data_resid")}
        self.lsq_info["check_every"] = every
        self.lsq_info["history"] = [hist[i] for i in range(min(info.checks, cap))]
        if rc != OK and (check or rc != ENOTCONV):
            raise NufftError(rc, "nufft_plan_solve_lsq")
        return c, info.iters, info.resid

    def dcf_weights(self, mlp, out=None):
        """Learned density-compensation weights of the points (mean 1), float32
        CUDA tensor [M] in the original point order."""
        torch = _torch()
        w = out if out is not None else torch.empty(self.M, dtype=torch.float32, device=self.device)
        _check(_lib.nufft_plan_dcf_weights(self._h, mlp._h, _dev_ptr(w, torch.float32, self.M, "w")),
               "nufft_plan_dcf_weights")
        return w

    def dcf_features(self):
        """Density-compensation features of the points: float32 [M, 8] (original order)."""
        torch = _torch()
        feat = torch.empty(self.M, 8, dtype=torch.float32, device=self.device)
        _check(_lib.nufft_plan_dcf_features(self._h, _P(feat.data_ptr())), "nufft_plan_dcf_features")
        return feat

    def close(self):
        if getattr(self, "_h", None):
            _lib.nufft_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _oneshot(fn, a, b, c, d, eps, prec, io, out, stream, name):
    flags = IO_C64 if io == "c64" else 0
    _check(fn(a, b, c, d, eps, prec, flags, out, _stream_handle(stream)), name)


def nufft_fwd(c, N: int, y, M: int, eps: float, prec: int = FP64, io: str = "c128", stream=None):
    """One-shot forward transform in the paper's argument order: nufft_fwd(c_n, N, y_j, M, eps)."""
    torch = _torch()
    cd = torch.complex64 if io == "c64" else torch.complex128
    g = torch.empty(M, dtype=cd, device=y.device)
    _oneshot(_lib.nufft_fwd, _dev_ptr(c, cd, N, "c"), N, _dev_ptr(y, torch.float64, M, "y"), M, eps,
             prec, io, _P(g.data_ptr()), stream, "nufft_fwd")
    return g


def nufft_adj(g, y, M: int, N: int, eps: float, prec: int = FP64, io: str = "c128", stream=None):
    torch = _torch()
    cd = torch.complex64 if io == "c64" else torch.complex128
    c = torch.empty(N, dtype=cd, device=y.device)
    _oneshot(_lib.nufft_adj, _dev_ptr(g, cd, M, "g"), _dev_ptr(y, torch.float64, M, "y"), M, N, eps,
             prec, io, _P(c.data_ptr()), stream, "nufft_adj")
    return c


def inufft(g, y, M: int, N: int, eps: float, prec: int = FP64, io: str = "c128", stream=None):
    """One-shot inverse: inufft(g_j, y_j, M, N, eps) -> c_n; M == N by the Lagrange
    form (Eq. p6 / p8), M > N the least-squares solution by plain CG."""
    torch = _torch()
    cd = torch.complex64 if io == "c64" else torch.complex128
    c = torch.empty(N, dtype=cd, device=y.device)
    _oneshot(_lib.inufft, _dev_ptr(g, cd, M, "g"), _dev_ptr(y, torch.float64, M, "y"), M, N, eps,
             prec, io, _P(c.data_ptr()), stream, "inufft")
    return c


def nufft_fwd_noalloc(c, N: int, y, M: int, eps: float, prec: int = FP64, io: str = "c128",
                      out=None, stream=None):
    """nufft_fwd without memory allocation inside the library (N, M <= 2^16):
    all work buffers live in a fixed device array of the library.  The output
    tensor is the caller's (``out``), so callers that must not allocate pass
    one they own."""
    torch = _torch()
    cd = torch.complex64 if io == "c64" else torch.complex128
    g = out if out is not None else torch.empty(M, dtype=cd, device=y.device)
    _oneshot(_lib.nufft_fwd_noalloc, _dev_ptr(c, cd, N, "c"), N, _dev_ptr(y, torch.float64, M, "y"),
             M, eps, prec, io, _dev_ptr(g, cd, M, "g"), stream, "nufft_fwd_noalloc")
    return g


def diag_rcp(t):
    """The near-field pair reciprocal as the kernels compute it: (FP64 path,
    mixed path) for a float64 CUDA tensor t."""
    torch = _torch()
    n = t.numel()
    r64 = torch.empty(n, dtype=torch.float64, device=t.device)
    r32 = torch.empty(n, dtype=torch.float32, device=t.device)
    _check(_lib.nufft_diag_rcp(_dev_ptr(t, torch.float64, n, "t"), n, _P(r64.data_ptr()),
                               _P(r32.data_ptr()), _stream_handle(None)), "nufft_diag_rcp")
    return r64, r32


def pipe_rates(stream=None):
    """(FP32 reciprocals, FP32 FMAs) completed per SM per clock on this GPU."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(_lib.nufft_diag_pipe_rates(ctypes.byref(a), ctypes.byref(b), _stream_handle(stream)),
           "nufft_diag_pipe_rates")
    return a.value, b.value


def dcf_features_sorted(y_sorted, stream=None):
    """Features of S sorted point sets (float64 CUDA tensor [S, M]): float32 [S*M, 8]."""
    torch = _torch()
    S, M = y_sorted.shape
    feat = torch.empty(S * M, 8, dtype=torch.float32, device=y_sorted.device)
    _check(_lib.nufft_dcf_features_sorted(_dev_ptr(y_sorted, torch.float64, S * M, "y"), S, M,
                                          _P(feat.data_ptr()), _stream_handle(stream)),
           "nufft_dcf_features_sorted")
    return feat


def dcf_targets(y_sorted, N: int, iters: int = 300, stream=None):
    """log(w / mean w) of the fixed-point density-compensation weights, float32 [S*M]."""
    torch = _torch()
    S, M = y_sorted.shape
    out = torch.empty(S * M, dtype=torch.float32, device=y_sorted.device)
    _check(_lib.nufft_dcf_targets(_dev_ptr(y_sorted, torch.float64, S * M, "y"), S, M, N, iters,
                                  _P(out.data_ptr()), _stream_handle(stream)), "nufft_dcf_targets")
    return out


class MLP:
    """The density-compensation network (8 -> 64 -> 64 -> 1, GELU, softplus) of the library."""

    NPARAM = None

    def __init__(self, params=None):
        h = _P()
        _check(_lib.nufft_mlp_create(ctypes.byref(h)), "nufft_mlp_create")
        self._h = h
        MLP.NPARAM = _lib.nufft_mlp_num_params()
        if params is not None:
            self.set_params(params)

    def set_params(self, params, reset_optimizer=True):
        import numpy as np
        a = np.ascontiguousarray(params, dtype=np.float32)
        if a.size != MLP.NPARAM:
            raise ValueError(f"expected {MLP.NPARAM} parameters")
        _check(_lib.nufft_mlp_set_params(self._h, a.ctypes.data_as(_P), 1 if reset_optimizer else 0),
               "nufft_mlp_set_params")

    def get_params(self):
        import numpy as np
        a = np.empty(MLP.NPARAM, np.float32)
        _check(_lib.nufft_mlp_get_params(self._h, a.ctypes.data_as(_P)), "nufft_mlp_get_params")
        return a

    def infer(self, feat, out=None, stream=None):
        torch = _torch()
        n = feat.shape[0]
        w = out if out is not None else torch.empty(n, dtype=torch.float32, device=feat.device)
        _check(_lib.nufft_mlp_infer(self._h, _dev_ptr(feat, torch.float32, n * 8, "feat"), n,
                                    _dev_ptr(w, torch.float32, n, "w"), _stream_handle(stream)),
               "nufft_mlp_infer")
        return w

    def grad(self, feat, target, stream=None):
        import numpy as np
        torch = _torch()
        n = feat.shape[0]
        g = np.empty(MLP.NPARAM, np.float32)
        loss = ctypes.c_float()
        _check(_lib.nufft_mlp_grad(self._h, _dev_ptr(feat, torch.float32, n * 8, "feat"),
                                   _dev_ptr(target, torch.float32, n, "target"), n, g.ctypes.data_as(_P),
                                   ctypes.cast(ctypes.byref(loss), _P), _stream_handle(stream)),
               "nufft_mlp_grad")
        return g, loss.value

    def train_step(self, feat, target, lr, want_loss=False, stream=None):
        torch = _torch()
        n = feat.shape[0]
        loss = ctypes.c_float()
        _check(_lib.nufft_mlp_train_step(self._h, _dev_ptr(feat, torch.float32, n * 8, "feat"),
                                         _dev_ptr(target, torch.float32, n, "target"), n, lr,
                                         ctypes.cast(ctypes.byref(loss), _P) if want_loss else None,
                                         _stream_handle(stream)), "nufft_mlp_train_step")
        return loss.value if want_loss else None

    def close(self):
        if getattr(self, "_h", None):
            _lib.nufft_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Multi:
    """Independent forward transforms of uneven sizes run as one CUDA graph launch.

    ys: list of CUDA float64 point tensors; Ns: grid sizes; params: None or
    one dict per transform (lmax, p, q, tc_level, tc_near: a plan's
    parameters, 0 / missing = the formulas).  forward(cs, gs) takes lists of
    coefficient / output tensors (captures a graph the first time and
    whenever the tensors change, then replays it)."""

    def __init__(self, Ns, ys, eps: float = 1e-6, prec: int = MIXED, io: str = "c64", stream=None,
                 params=None):
        import numpy as np
        torch = _torch()
        self.Ns = [int(n) for n in Ns]
        self.Ms = [int(y.numel()) for y in ys]
        self._ys = list(ys)  # kept alive for the call
        self.cdtype = torch.complex64 if io == "c64" else torch.complex128
        n = len(self.Ns)
        Na = np.array(self.Ns, dtype=np.int64)
        Ma = np.array(self.Ms, dtype=np.int64)
        yp = (ctypes.c_void_p * n)(*[_dev_ptr(y, torch.float64, m, "y").value for y, m in zip(ys, self.Ms)])
        prm = None
        if params is not None:
            if len(params) != n:
                raise ValueError("params: one entry per transform")
            prm = (Params * n)()
            for i, d in enumerate(params):
                d = d or {}
                prm[i] = Params(int(d.get("lmax", 0)), int(d.get("p", 0)), int(d.get("q", 0)), 1,
                                int(d.get("tc_level", 0)), int(d.get("tc_near", 0)))
        h = _P()
        _check(_lib.nufft_multi_create(ctypes.byref(h), n, Na.ctypes.data_as(_P), Ma.ctypes.data_as(_P),
                                       ctypes.cast(yp, _P), eps, prec,
                                       ctypes.cast(prm, _P) if prm is not None else None,
                                       IO_C64 if io == "c64" else 0,
                                       _stream_handle(stream)), "nufft_multi_create")
        self._h = h

    def forward(self, cs, gs):
        n = len(self.Ns)
        cp = (ctypes.c_void_p * n)(*[_dev_ptr(c, self.cdtype, N, "c").value for c, N in zip(cs, self.Ns)])
        gp = (ctypes.c_void_p * n)(*[_dev_ptr(g, self.cdtype, M, "g").value for g, M in zip(gs, self.Ms)])
        _check(_lib.nufft_multi_exec_fwd(self._h, ctypes.cast(cp, _P), ctypes.cast(gp, _P)),
               "nufft_multi_exec_fwd")
        return gs

    def close(self):
        if getattr(self, "_h", None):
            _lib.nufft_multi_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
