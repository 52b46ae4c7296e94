"""Host-side checks of the C ABI (no GPU): the library loads and exports every
symbol include/nufft.h declares; parameter choice (Eq. 18.2 with reading c5,
Eq. 25 with l* = 5) and argument validation; the double-double constants."""
import os
import re
from fractions import Fraction

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def nf():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1611_09379_gb300 as nf
    return nf


def _declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", fn)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([A-Za-z_]\w*)\s*\(", txt, flags=re.M):
            if m.group(1) not in ("if", "defined"):
                names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol(nf):
    import ctypes
    lib = ctypes.CDLL(nf.LIB_PATH)
    declared = _declared_symbols()
    assert len(declared) >= 14
    for name in declared:
        assert hasattr(lib, name), name
    assert declared == set(nf.SYMBOLS)


def test_choose_params_matches_eq18_2_reading(nf):
    # reading c5: q = ceil(1/2 log2(10/(3 pi eps))), p = ceil(1 + log3(...) + lmax/log2 3)
    assert nf.choose_params(1 << 20, 1 << 20, 1e-12) == (15, 36, 20)
    assert nf.choose_params(1 << 20, 1 << 20, 1e-6, nf.MIXED) == (15, 24, 11)
    assert nf.choose_params(1 << 12, 1 << 12, 1e-12) == (7, 31, 20)
    assert nf.choose_params(1 << 24, 1 << 24, 1e-6, nf.MIXED) == (19, 26, 11)
    assert nf.choose_params(1 << 16, 1 << 16, 1e-8) == (11, 25, 14)
    # small N clamps lmax to 2
    assert nf.choose_params(8, 8, 1e-6)[0] == 2
    # explicit overrides are kept
    assert nf.choose_params(1 << 12, 1 << 12, 1e-6, nf.FP64, lmax=4, p=10, q=5) == (4, 10, 5)


@pytest.mark.parametrize("args", [
    (4, 4, 1e-6, 0),            # N < 8
    ((1 << 26) + 1, 10, 1e-6, 0),  # N above 2^26
    (1 << 10, 0, 1e-6, 0),      # M < 1
    (1 << 10, 10, 1e-16, 0),    # eps below 1e-15
    (1 << 10, 10, 0.5, 0),      # eps above 1e-1
    (1 << 10, 10, 1e-6, 7),     # unknown precision
    (1 << 10, 10, 1e-9, 1),     # mixed precision cannot reach 1e-9
])
def test_choose_params_rejects(nf, args):
    with pytest.raises(nf.NufftError) as e:
        nf.choose_params(*args)
    assert e.value.code == nf.EINVAL


@pytest.mark.parametrize("N", [1000, 12345, 3 << 10, (1 << 20) - 3])
def test_choose_params_general_n_uses_the_padded_grid(nf, N):
    """N not a power of two: the tree is chosen for the grid N' = 2^ceil(log2 N)
    (the same parameters as for N' itself)."""
    Np = 1 << (N - 1).bit_length()
    for prec, eps in ((nf.FP64, 1e-12), (nf.MIXED, 1e-6)):
        assert nf.choose_params(N, N, eps, prec) == nf.choose_params(Np, N, eps, prec)


def test_machine_precision_mode_parameters(nf):
    """eps = 0 (FP64) prescribes the threshold error eps_th(N) = log2(N') 2^-53
    (at least 1e-15) and takes p, q from Eq. 18.2 at it (Sec. 3.2); the mixed
    path has no such mode."""
    for N in (8, 1 << 10, 1 << 16, 1 << 20, 12345, 1 << 26):
        Np = 1 << (N - 1).bit_length()
        e = nf.eps_threshold(N)
        assert e == max(1e-15, (Np.bit_length() - 1) * 2.0 ** -53)
        assert nf.choose_params(N, N, 0.0, nf.FP64) == nf.choose_params(N, N, e, nf.FP64)
    p20 = nf.choose_params(1 << 20, 1 << 20, 0.0, nf.FP64)
    assert p20 == (15, 42, 25)  # eps_th(2^20) = 2.2e-15
    with pytest.raises(nf.NufftError):
        nf.choose_params(1 << 10, 1 << 10, 0.0, nf.MIXED)
    with pytest.raises(nf.NufftError):
        nf.eps_threshold(4)


def test_lmax_override_bounds(nf):
    with pytest.raises(nf.NufftError):
        nf.choose_params(1 << 10, 1 << 10, 1e-6, nf.FP64, lmax=11)
    with pytest.raises(nf.NufftError):
        nf.choose_params(1 << 10, 1 << 10, 1e-6, nf.FP64, p=65)


def test_strerror_and_version(nf):
    assert nf.strerror(0) == "success"
    assert "invalid" in nf.strerror(nf.EINVAL)
    assert nf.version() >= 100


def test_double_double_constants_are_exact(orc):
    """fl(1/(2pi)) + lo and fl(2pi) + lo in the CUDA sources equal the exact
    values to 2^-106 relative (checked against the oracle's 480-bit pi)."""
    src = open(os.path.join(ROOT, "paper_1611_09379_gb300", "csrc", "common.cuh")).read()
    val = dict(re.findall(r"constexpr double (k\w+) = ([-\d.e+]+);", src))
    pi = Fraction(orc.PI_FIXED, 1 << orc._PI_BITS)
    for hi, lo, exact in (("kInvTwoPiHi", "kInvTwoPiLo", 1 / (2 * pi)), ("kTwoPiHi", "kTwoPiLo", 2 * pi)):
        s = Fraction(float(val[hi])) + Fraction(float(val[lo]))
        assert abs(s - exact) / exact < Fraction(1, 2 ** 104)
        assert float(val[hi]) == float(exact)


def test_tc_level_choice(nf):
    """Automatic first tensor-core level: the finest levels with >= 2048
    parent boxes over all signals; FP64 plans and large p never use it."""
    d = nf.choose_params_full(1 << 20, 1 << 20, 1e-6, nf.MIXED)
    assert d["lmax"] == 15 and d["tc_level"] == 12
    assert nf.choose_params_full(1 << 20, 1 << 20, 1e-12, nf.FP64)["tc_level"] == -1
    b = nf.choose_params_full(1 << 18, 1 << 18, 1e-6, nf.MIXED, batch=64)
    assert b["lmax"] == 13 and b["tc_level"] == 6
    assert nf.choose_params_full(1 << 12, 1 << 12, 1e-6, nf.MIXED)["tc_level"] == -1  # lmax 7
    assert nf.choose_params_full(1 << 20, 1 << 20, 1e-6, nf.MIXED, tc_level=-1)["tc_level"] == -1
    assert nf.choose_params_full(1 << 20, 1 << 20, 1e-6, nf.MIXED, tc_level=9)["tc_level"] == 9
    assert nf.choose_params_full(1 << 20, 1 << 20, 1e-6, nf.MIXED, tc_level=20)["tc_level"] == -1
    # p above the kernel's limit (24): no tensor-core levels
    assert nf.choose_params_full(1 << 20, 1 << 20, 1e-6, nf.MIXED, p=30)["tc_level"] == -1
    for bad in (1, 2, 3, 31, -2):
        with pytest.raises(nf.NufftError):
            nf.choose_params_full(1 << 20, 1 << 20, 1e-6, nf.MIXED, tc_level=bad)


def test_autotune_rejects_bad_arguments(nf):
    """Argument checks come before any device work."""
    import ctypes
    best = nf.Params()
    n = ctypes.c_int(0)
    lib = nf._lib
    # null points, empty op mask, unknown op bit, reps < 1, inverse with M != N, N < 8
    assert lib.nufft_autotune(1024, 1024, None, 1e-6, 1, 0, 1, 1, 3, ctypes.byref(best), None, 0,
                              ctypes.byref(n), None) == nf.EINVAL
    fake = ctypes.c_void_p(16)  # never dereferenced: the checks fail first
    assert lib.nufft_autotune(1024, 1024, fake, 1e-6, 1, 0, 1, 0, 3, ctypes.byref(best), None, 0,
                              None, None) == nf.EINVAL
    assert lib.nufft_autotune(1024, 1024, fake, 1e-6, 1, 0, 1, 8, 3, ctypes.byref(best), None, 0,
                              None, None) == nf.EINVAL
    assert lib.nufft_autotune(1024, 1024, fake, 1e-6, 1, 0, 1, 1, 0, ctypes.byref(best), None, 0,
                              None, None) == nf.EINVAL
    assert lib.nufft_autotune(1024, 2048, fake, 1e-6, 1, 0, 1, 4, 3, ctypes.byref(best), None, 0,
                              None, None) == nf.EINVAL
    assert lib.nufft_autotune(4, 1024, fake, 1e-6, 1, 0, 1, 1, 3, ctypes.byref(best), None, 0,
                              None, None) == nf.EINVAL


def test_tune_table_roundtrip(tmp_path):
    from paper_1611_09379_gb300 import tune
    assert tune.ops_mask("fwd+inv") == 5 and tune.ops_mask(("adj",)) == 2 and tune.ops_mask(3) == 3
    k1 = tune.key(1 << 20, 1 << 20, 1e-6, 1, "c128", 1, "fwd+inv", "jitter")
    k2 = tune.key(1 << 20, 1 << 20, 1e-6, 1, "c128", 1, "fwd", "jitter")
    assert k1 != k2
    path = str(tmp_path / "table.json")
    assert tune.load_table(path) == {}
    tune.save_table({k1: {"params": {"lmax": 15}}}, path)
    assert tune.load_table(path)[k1]["params"]["lmax"] == 15


def test_tc_near_choice(nf):
    """Tensor-core near field: mixed precision with batches of 64 signals."""
    assert nf.choose_params_full(1 << 18, 1 << 18, 1e-6, nf.MIXED, batch=64)["tc_near"] == 1
    assert nf.choose_params_full(1 << 18, 1 << 18, 1e-6, nf.MIXED, batch=128)["tc_near"] == 1
    assert nf.choose_params_full(1 << 18, 1 << 18, 1e-6, nf.MIXED, batch=32)["tc_near"] == -1
    assert nf.choose_params_full(1 << 18, 1 << 18, 1e-12, nf.FP64, batch=64)["tc_near"] == -1
    assert nf.choose_params_full(1 << 18, 1 << 18, 1e-6, nf.MIXED, batch=64, tc_near=-1)["tc_near"] == -1
    with pytest.raises(nf.NufftError):
        nf.choose_params_full(1 << 18, 1 << 18, 1e-6, nf.MIXED, batch=64, tc_near=2)


def test_adaptive_depths_rule(nf):
    """The adaptive tree's depth rule (nufft_adaptive_depths): d_b is the
    largest d <= min(3, log2 s - 3) with n_b >= 2^d * mean count; equal counts
    refine nothing, the cap follows s, and bad arguments are rejected."""
    import numpy as np

    def starts(counts):
        return np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)

    D, dep = nf.adaptive_depths(starts([64] * 16), 64)
    assert D == 0 and not dep.any()
    # mean 100 over 64 leaves: counts 199 / 200 / 399 / 400 / 799 / 800 / 1600
    # straddle 2x, 4x and 8x the mean; the other 57 leaves share the rest
    c = np.array([199, 200, 399, 400, 799, 800, 1600] + [0] * 57)
    rest = 6400 - c.sum()
    c[7:] = rest // 57
    c[7] += rest - 57 * (rest // 57)
    assert c.sum() == 6400 and c[7:].max() < 200
    D, dep = nf.adaptive_depths(starts(c), 1024)
    assert list(dep[:7]) == [0, 1, 1, 2, 2, 3, 3] and D == 3
    # the cap: s = 32 allows 2 levels, s = 16 one, s = 8 none
    assert nf.adaptive_depths(starts(c), 32)[1][5] == 2
    assert nf.adaptive_depths(starts(c), 16)[0] == 1
    assert nf.adaptive_depths(starts(c), 8)[0] == 0
    # no targets: nothing refined
    assert nf.adaptive_depths(starts([0] * 8), 64)[0] == 0
    # invalid: B not a power of two, s not a power of two, decreasing starts
    with pytest.raises(nf.NufftError):
        nf.adaptive_depths(starts([1, 2, 3]), 64)
    with pytest.raises(nf.NufftError):
        nf.adaptive_depths(starts([1, 2, 3, 4]), 48)
    with pytest.raises(nf.NufftError):
        nf.adaptive_depths(np.array([0, 5, 3, 6, 10], dtype=np.int32), 64)
