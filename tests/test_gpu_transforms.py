"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances are the ones the workloads are specified at: relative L2 error
1e-12 for the FP64 path and 1e-6 for the mixed path; binning (perm,
leaf_start, k0) is compared bit for bit.  Sizes span several leaves and a
ragged tail; the 2^20 cases compare 4096 sampled targets (seeded).
"""
import math

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-6}


@pytest.fixture(scope="module")
def nf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_1611_09379_gb300 as nf
    return nf


def _dev(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def _host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


# ------------------------------------------------------------------ binning

_BINNING_CASES = [
    ("uniform", 4096, 5000, 7), ("clustered", 4096, 4096, 7), ("uniform", 64, 33, 2),
    ("uniform", 1 << 14, 1, 9), ("jitter", 2048, 2048, 6),
]


def _binned(nf, kind, N, M, lmax):
    y = workloads.points(kind, M, N if kind == "jitter" else None, seed=M + lmax, jitter=0.4)
    if kind == "uniform" and M > 10:
        y[:4] = [0.0, np.nextafter(2 * np.pi, 0), np.nextafter(2 * np.pi * 3 / N, 0), 2 * np.pi * 5 / N]
    plan = nf.Plan(N, _dev(y), eps=1e-6, lmax=lmax)
    return y, [_host(t) for t in plan.points()]


@pytest.mark.parametrize("kind,N,M,lmax", _BINNING_CASES)
def test_binning_bit_exact(nf, orc, kind, N, M, lmax):
    """Parity with the paper's binning (Sec. 2.1): every point in its exact
    leaf, leaf_start bit for bit, the same set of points in every leaf, and
    k0 / delta of every point equal to the exact-rational grid coordinates."""
    y, (perm, start, k0, delta) = _binned(nf, kind, N, M, lmax)
    B = 1 << lmax
    operm, ostart, oleaf = orc.binning(y, N, B)
    _, ok0, odel = orc.exact_grid(y, N, B)
    assert np.array_equal(start, ostart)
    assert np.array_equal(np.sort(perm), np.arange(M))
    assert np.array_equal(oleaf[perm], np.repeat(np.arange(B), np.diff(ostart)))
    for b in range(B):
        assert np.array_equal(np.sort(perm[start[b]:start[b + 1]]), operm[ostart[b]:ostart[b + 1]])
    assert np.array_equal(k0, ok0[perm])
    ref = odel[perm]
    assert np.all(np.abs(delta - ref) <= 2 * np.spacing(np.abs(ref)) + 1e-300)


@pytest.mark.parametrize("kind,N,M,lmax", _BINNING_CASES)
def test_binning_layout_inside_leaves(nf, orc, kind, N, M, lmax):
    """Layout, not parity: inside a leaf the library orders its points by the
    nearest grid point relative to the leaf's first one, (k0 - leaf s) mod N,
    then by original index (the staged near-field windows rely on it).  The
    key is formed here from the oracle's exact k0."""
    y, (perm, start, _, _) = _binned(nf, kind, N, M, lmax)
    B = 1 << lmax
    s = N // B
    _, ok0, _ = orc.exact_grid(y, N, B)
    for b in range(B):
        seg = perm[start[b]:start[b + 1]].astype(np.int64)
        key = ((ok0[seg] - b * s) % N) * (1 << 40) + seg
        assert np.all(np.diff(key) > 0), b


# ------------------------------------------------------------------ forward

def _fwd(nf, N, y, c, eps, prec, io="c128", **kw):
    import torch
    cd = torch.complex64 if io == "c64" else torch.complex128
    plan = nf.Plan(N, _dev(y), eps=eps, prec=prec, io=io, **kw)
    return _host(plan.forward(_dev(c, cd))), plan


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("kind", ["uniform", "clustered"])
def test_forward_4096_full(nf, orc, prec, kind):
    N = M = 4096
    eps = 1e-12 if prec == 0 else 1e-6
    y = workloads.points(kind, M, seed=1234)
    c = workloads.coeffs(N, seed=99)
    g, _ = _fwd(nf, N, y, c, eps, prec)
    ref = orc.nudft_fwd(c, y)
    assert orc.rel_l2(g, ref) < TOL[prec]


@pytest.mark.parametrize("L", [3, 6, 10, 12])
@pytest.mark.parametrize("eps", [1e-3, 1e-6, 1e-9, 1e-12])
def test_forward_constant_function(nf, L, eps):
    """The paper's analytic test (Sec. 3.1): f == 1 gives g_j = 1; the error
    eps_a = max_j |g_j - 1| stays below the prescribed eps for any lmax."""
    N = 1 << L
    M = 3000
    y = workloads.points("uniform", M, seed=L)
    c = np.zeros(N, complex)
    c[0] = 1.0
    for lmax in sorted({2, max(2, L - 5), L - 1}):
        g, _ = _fwd(nf, N, y, c, eps, 0, lmax=lmax)
        assert np.abs(g - 1).max() < eps


def test_forward_adjoint_largest_order(nf, orc):
    """p = 64 (the largest order accepted) in FP64: the downward pass's
    operators then leave no room for the one-launch form, and the banded
    form runs instead."""
    N, M = 4096, 3001
    y = workloads.points("uniform", M, seed=51)
    c = workloads.coeffs(N, seed=52)
    g0 = workloads.samples(M, seed=53)
    plan = nf.Plan(N, _dev(y), eps=1e-12, lmax=8, p=64)
    g = _host(plan.forward(_dev(c)))
    assert orc.rel_l2(g, orc.nudft_fwd(c, y)) < 1e-12
    a = _host(plan.adjoint(_dev(g0)))
    assert orc.rel_l2(a, orc.nudft_adj(g0, y, N)) < 1e-12


@pytest.mark.parametrize("N,M,lmax", [(8, 5, 2), (16, 40, 2), (64, 1, 3), (256, 255, 4), (1024, 3001, 5)])
def test_forward_edge_sizes(nf, orc, N, M, lmax):
    y = workloads.points("uniform", M, seed=N + M)
    c = workloads.coeffs(N, seed=N)
    g, _ = _fwd(nf, N, y, c, 1e-12, 0, lmax=lmax)
    assert orc.rel_l2(g, orc.nudft_fwd(c, y)) < 1e-12


def test_forward_grid_hits_and_neighbours(nf, orc):
    """y_j = 0 (exact hit, g = f_0) and points one ulp from grid points, where
    the kernel G is near its pole (reading c7)."""
    N = 2048
    k = np.arange(0, N, 37)
    xk = k * (2 * math.pi / N)
    y = np.concatenate([[0.0], np.nextafter(xk[1:], 10.0), np.nextafter(xk[1:], -10.0),
                        workloads.points("uniform", 100, seed=3)])
    c = workloads.coeffs(N, seed=5)
    for prec in (0, 1):
        g, _ = _fwd(nf, N, y, c, 1e-12 if prec == 0 else 1e-6, prec)
        ref = orc.nudft_fwd(c, y)
        assert orc.rel_l2(g, ref) < TOL[prec]
        f0 = c.sum()
        assert abs(g[0] - f0) <= (1e-13 if prec == 0 else 1e-6) * abs(f0)


def test_forward_single_mode(nf, orc):
    """c = e_m reproduces e^{i m y_j} (band-limited series); the reference is
    the oracle, pinned to the exactly reduced phase m y_j."""
    N = 4096
    y = workloads.points("uniform", 2000, seed=8)
    for m in (1, 1000, N - 1):
        c = np.zeros(N, complex)
        c[m] = 1
        g, _ = _fwd(nf, N, y, c, 1e-12, 0)
        assert np.abs(g - orc.nudft_fwd(c, y)).max() < 1e-12


def test_forward_c64_io(nf, orc):
    N = M = 4096
    y = workloads.points("uniform", M, seed=2)
    c = workloads.coeffs(N, seed=3).astype(np.complex64)
    g, _ = _fwd(nf, N, y, c, 1e-6, 1, io="c64")
    assert g.dtype == np.complex64
    assert orc.rel_l2(g, orc.nudft_fwd(c.astype(complex), y)) < 1e-6


# ------------------------------------------------------------------ adjoint

@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("kind", ["uniform", "clustered"])
def test_adjoint_4096_full(nf, orc, prec, kind):
    N, M = 4096, 3500
    eps = 1e-12 if prec == 0 else 1e-6
    y = workloads.points(kind, M, seed=11)
    g = workloads.samples(M, seed=12)
    plan = nf.Plan(N, _dev(y), eps=eps, prec=prec)
    c = _host(plan.adjoint(_dev(g)))
    assert orc.rel_l2(c, orc.nudft_adj(g, y, N)) < TOL[prec]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("s", [2, 4, 8])
def test_adjoint_small_leaves_clustered(nf, orc, prec, s):
    """Leaves of s grid points: a warp of the two-point kernel covers 64 grid
    points, i.e. several leaves, so its lanes' windows differ and the chunks
    at their edges take the checked form; clustered points make the windows
    uneven."""
    N, M = 2048, 1777
    eps = 1e-12 if prec == 0 else 1e-6
    y = workloads.points("clustered", M, seed=31 + s)
    g = workloads.samples(M, seed=32 + s)
    plan = nf.Plan(N, _dev(y), eps=eps, prec=prec, lmax=int(math.log2(N // s)))
    c = _host(plan.adjoint(_dev(g)))
    assert orc.rel_l2(c, orc.nudft_adj(g, y, N)) < TOL[prec]


def test_adjoint_dot_product(nf):
    N, M = 2048, 5000
    y = workloads.points("uniform", M, seed=21)
    plan = nf.Plan(N, _dev(y), eps=1e-12)
    c = workloads.coeffs(N, seed=22)
    g = workloads.samples(M, seed=23)
    Ac = _host(plan.forward(_dev(c)))
    Ahg = _host(plan.adjoint(_dev(g)))
    lhs, rhs = np.vdot(g, Ac), np.vdot(Ahg, c)
    assert abs(lhs - rhs) / abs(lhs) < 1e-12


def test_adjoint_exact_hit(nf, orc):
    N = 512
    y = workloads.points("uniform", 300, seed=4)
    y[7] = 0.0
    g = workloads.samples(300, seed=5)
    plan = nf.Plan(N, _dev(y), eps=1e-12)
    c = _host(plan.adjoint(_dev(g)))
    assert orc.rel_l2(c, orc.nudft_adj(g, y, N)) < 1e-12


# ------------------------------------------------------------------ inverse

@pytest.mark.parametrize("N,jit", [(256, 0.1), (4096, 0.1), (4096, 0.4)])
def test_inverse_round_trip(nf, orc, N, jit):
    """At M = N the Lagrange form (Eq. p6, p8) inverts the forward map;
    compared with the oracle's inverse of the same samples."""
    y = workloads.points("jitter", N, N, seed=N, jitter=jit)
    c = workloads.coeffs(N, seed=N + 1)
    g = orc.nudft_fwd(c, y)
    plan = nf.Plan(N, _dev(y), eps=1e-12, inverse=True)
    c2 = _host(plan.inverse(_dev(g)))
    cref = orc.inufft(g, y, N)
    assert orc.rel_l2(c2, cref) < 1e-12
    assert orc.rel_l2(c2, c) < (1e-12 if jit <= 0.1 else 1e-10)


@pytest.mark.parametrize("prec", [0, 1])
def test_inverse_round_trip_small_leaves(nf, orc, prec):
    """Square inverse with leaves of 2 grid points (the deepest tree)."""
    N = 1024
    y = workloads.points("jitter", N, N, seed=41, jitter=0.1)
    c = workloads.coeffs(N, seed=42)
    g = orc.nudft_fwd(c, y)
    plan = nf.Plan(N, _dev(y), eps=1e-12 if prec == 0 else 1e-6, prec=prec, inverse=True,
                   lmax=9)
    c2 = _host(plan.inverse(_dev(g)))
    assert orc.rel_l2(c2, orc.inufft(g, y, N)) < TOL[prec]


@pytest.mark.parametrize("N,jit,hit", [(256, 0.1, False), (256, 0.1, True), (4096, 0.4, False),
                                       (1024, 0.1, True)])
def test_inverse_coefficients(nf, orc, N, jit, hit):
    """The log-sums behind C_k and D_j (Eq. p8) and their signs agree with the
    oracle's direct sums: |lamC|, |lamD| errors below 1e-12 absolute."""
    y = workloads.points("jitter", N, N, seed=N + 9, jitter=jit)
    if hit:
        y[0] = 0.0
    plan = nf.Plan(N, _dev(y), eps=1e-12, inverse=True)
    Ct, Dt, lam = plan.inverse_coeffs()
    Ct, Dt = _host(Ct), _host(Dt)
    perm = _host(plan.points()[0])
    lC, nC = orc.logsin_C(y, N)
    lD, nD = orc.logsin_D(y)
    fin = np.isfinite(lC)
    assert np.all(Ct[~fin] == 0.0)
    assert np.abs(np.log(np.abs(Ct[fin]) * N) - lam - lC[fin]).max() < 1e-12
    sC = np.where((np.arange(N) + nC) % 2 == 1, -1.0, 1.0)
    assert np.array_equal(np.sign(Ct[fin]), sC[fin])
    assert np.abs(np.log(np.abs(Dt)) + lam - lD[perm]).max() < 1e-12
    # phase of D: (-1)^nD i e^{-i N y/2}
    ref = np.where(nD[perm] % 2 == 1, -1.0, 1.0) * 1j * np.exp(-0.5j * N * y[perm])
    assert np.abs(Dt / np.abs(Dt) - ref).max() < 1e-12


def test_inverse_mixed(nf, orc):
    N = 4096
    y = workloads.points("jitter", N, N, seed=7, jitter=0.1)
    c = workloads.coeffs(N, seed=8)
    g = orc.nudft_fwd(c, y)
    plan = nf.Plan(N, _dev(y), eps=1e-6, prec=nf.MIXED, inverse=True)
    c2 = _host(plan.inverse(_dev(g)))
    assert orc.rel_l2(c2, c) < 1e-6


def test_inverse_exact_hit(nf, orc):
    N = 256
    y = workloads.points("jitter", N, N, seed=9, jitter=0.1)
    y[0] = 0.0
    c = workloads.coeffs(N, seed=1)
    g = orc.nudft_fwd(c, y)
    plan = nf.Plan(N, _dev(y), eps=1e-12, inverse=True)
    c2 = _host(plan.inverse(_dev(g)))
    assert orc.rel_l2(c2, c) < 1e-12


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("y0", [0.0, 1e-30])
def test_inverse_near_grid_points(nf, orc, prec, y0):
    """Points at or next to grid points, where the self term's factor
    C~_k0 / delta_j is a ratio of two small numbers (C~_k0 carries
    sin((x_k0 - y_j)/2)): an exact hit at y = 0 or a point 1e-30 from it,
    and points one ulp either side of grid points, on the 10 % jittered
    grid.  The round trip meets eps in both precisions."""
    N = 1024
    y = workloads.points("jitter", N, N, seed=19, jitter=0.1)
    xk = 2 * math.pi * np.arange(N) / N
    y[0] = y0
    y[37::97] = np.nextafter(xk[37::97], 10.0)
    y[81::97] = np.nextafter(xk[81::97], -10.0)
    c = workloads.coeffs(N, seed=20)
    g = orc.nudft_fwd(c, y)
    plan = nf.Plan(N, _dev(y), eps=1e-12 if prec == 0 else 1e-6, prec=prec, inverse=True)
    c2 = _host(plan.inverse(_dev(g)))
    assert np.all(np.isfinite(c2))
    assert orc.rel_l2(c2, c) < (1e-11 if prec == 0 else 1e-6)


_LAMD_CACHE = {}


def _lamD(orc, y, key):
    if key not in _LAMD_CACHE:
        _LAMD_CACHE[key] = orc.logsin_D(y)
    return _LAMD_CACHE[key]


@pytest.mark.parametrize("prec", [0, 1])
def test_inverse_2p16_jitter_sampled(nf, orc, prec):
    """Square inverse at N = M = 2^16 on the 40 % jittered grid (beyond the
    paper's 10 % test): the grid values f_k of the library's result (f = N
    IDFT(c)) against the oracle's Lagrange sum (Eq. p6 / p8, direct log-sums)
    on 512 sampled k, relative to the modulus sum sum_j |L_kj| |g_j| at the
    same k (reading c16); the round trip c against c_true as well."""
    N = M = 1 << 16
    y = workloads.points("jitter", M, N, seed=1616, jitter=0.4)
    c = workloads.coeffs(N, seed=17)
    g = orc.nudft_fwd(c, y)
    eps = 1e-12 if prec == 0 else 1e-6
    plan = nf.Plan(N, _dev(y), eps=eps, prec=prec, inverse=True)
    c2 = _host(plan.inverse(_dev(g)))
    f = np.fft.ifft(c2) * N  # f_k = sum_n c_n e^{2 pi i n k / N}
    kdx = workloads.sample_index(N, 512, seed=3)
    lamD = _lamD(orc, y, ("jitter", N))
    fref = orc.inverse_f(g, y, N, kdx, lamD=lamD)
    aref = orc.inverse_absf(g, y, N, kdx, lamD=lamD)
    err = np.linalg.norm(f[kdx] - fref) / np.linalg.norm(aref)
    assert err < TOL[prec], err
    assert orc.rel_l2(f[kdx], fref) < 10 * TOL[prec]
    assert orc.rel_l2(c2, c) < (1e-10 if prec == 0 else 1e-5)


def test_inverse_clustered_is_out_of_range_at_2p16(nf, orc):
    """On the clustered mixture the log-sums behind C_k and D_j span
    thousands (the Lagrange weights of Eq. p8 are far outside binary64), so
    the plan refuses the square inverse with NUFFT_EILLCOND; the forward on
    the same points is unaffected."""
    N = M = 1 << 16
    y = workloads.points("clustered", M, seed=1617)
    lD, _ = orc.logsin_D(y, workloads.sample_index(M, 64, seed=2))
    assert lD.max() - lD.min() > 1500  # e^1500 is far beyond the binary64 range
    with pytest.raises(nf.NufftError) as e:
        nf.Plan(N, _dev(y), eps=1e-12, inverse=True)
    assert e.value.code == nf.EILLCOND
    plan = nf.Plan(N, _dev(y), eps=1e-12)
    c = workloads.coeffs(N, seed=5)
    g = _host(plan.forward(_dev(c)))
    idx = workloads.sample_index(M, 256, seed=4)
    assert orc.rel_l2(g[idx], orc.nudft_fwd(c, y, idx)) < 1e-12


@pytest.mark.parametrize("prec,N", [(0, 512), (1, 128)])
def test_inverse_clustered_small_matvec(nf, orc, prec, N):
    """Clustered points where the Lagrange weights still fit the arithmetic
    (log-sums within about +-210 at N = 512 for binary64, +-45 at N = 128 for
    the mixed path's binary32 copies): the inverse's matrix-vector product
    f = L g (Eq. p6) against the oracle's, relative to sum_j |L_kj| |g_j|
    (reading c16); the problem is too ill-conditioned for the round trip to
    be asserted.  At N = 512 the mixed path refuses (NUFFT_EILLCOND)."""
    M = N
    y = workloads.points("clustered", M, seed=33)
    g = workloads.samples(M, seed=34)
    eps = 1e-12 if prec == 0 else 1e-6
    plan = nf.Plan(N, _dev(y), eps=eps, prec=prec, inverse=True)
    c2 = _host(plan.inverse(_dev(g)))
    f = np.fft.ifft(c2) * N
    fref = orc.inverse_f(g, y, N)
    aref = orc.inverse_absf(g, y, N)
    sc = aref.max()  # the sums reach e^200: scale before the norms
    assert np.all(np.isfinite(f)) and sc < np.inf
    assert np.linalg.norm((f - fref) / sc) / np.linalg.norm(aref / sc) < TOL[prec]
    if prec == 1:
        y5 = workloads.points("clustered", 512, seed=33)
        with pytest.raises(nf.NufftError) as e:
            nf.Plan(512, _dev(y5), eps=1e-6, prec=prec, inverse=True)
        assert e.value.code == nf.EILLCOND


# ------------------------------------------------------------------ full size (sampled)

@pytest.mark.parametrize("prec,kind", [(0, "uniform"), (1, "uniform"), (0, "jitter"), (1, "clustered")])
def test_forward_2p20_sampled(nf, orc, prec, kind):
    N = M = 1 << 20
    eps = 1e-12 if prec == 0 else 1e-6
    y = workloads.points(kind, M, N, seed=1234, jitter=0.4)
    c = workloads.coeffs(N, seed=99)
    g, plan = _fwd(nf, N, y, c, eps, prec)
    idx = workloads.sample_index(M, 4096)
    ref = orc.nudft_fwd(c, y, idx)
    assert orc.rel_l2(g[idx], ref) < TOL[prec]


@pytest.mark.parametrize("prec", [0, 1])
def test_adjoint_2p20_sampled(nf, orc, prec):
    N = M = 1 << 20
    y = workloads.points("uniform", M, seed=1234)
    g = workloads.samples(M, seed=77)
    plan = nf.Plan(N, _dev(y), eps=1e-12 if prec == 0 else 1e-6, prec=prec)
    c = _host(plan.adjoint(_dev(g)))
    idx = workloads.sample_index(N, 2048)
    assert orc.rel_l2(c[idx], orc.nudft_adj(g, y, N, idx)) < TOL[prec]


@pytest.mark.parametrize("prec,kind,lmax", [(0, "multiscale", 17), (1, "multiscale", 17),
                                          (1, "clustered", 0)])
def test_adjoint_2p20_clustered_sampled(nf, orc, prec, kind, lmax):
    """Adjoint on clustered sources at 2^20, where leaves hold up to 30x the
    mean count: the P2M in chunks of at most 256 sources of one leaf and the
    near field one warp per 8 grid points.  Sampled coefficients against the
    direct sums; a replay gives the same bits.  (The four-width mixture
    at l_max 17: at the formula's depth a leaf would exceed the binning's
    2048 points.)"""
    N = M = 1 << 20
    y = workloads.points(kind, M, seed=1235)
    g = workloads.samples(M, seed=78)
    plan = nf.Plan(N, _dev(y), eps=1e-12 if prec == 0 else 1e-6, prec=prec, lmax=lmax)
    c = _host(plan.adjoint(_dev(g)))
    idx = workloads.sample_index(N, 1024, seed=3)
    assert orc.rel_l2(c[idx], orc.nudft_adj(g, y, N, idx)) < TOL[prec]
    assert np.array_equal(_host(plan.adjoint(_dev(g))), c)


# ------------------------------------------------------------------ errors

def test_rejects_points_outside_circle(nf):
    import torch
    y = torch.tensor([0.1, 7.0, 0.3], dtype=torch.float64, device="cuda")
    with pytest.raises(nf.NufftError) as e:
        nf.Plan(64, y, eps=1e-6)
    assert e.value.code == nf.EINVAL
    y = torch.tensor([0.1, float("nan")], dtype=torch.float64, device="cuda")
    with pytest.raises(nf.NufftError):
        nf.Plan(64, y, eps=1e-6)
    y = torch.tensor([0.1, -1e-300], dtype=torch.float64, device="cuda")
    with pytest.raises(nf.NufftError):
        nf.Plan(64, y, eps=1e-6)


def test_inverse_requires_square(nf):
    import torch
    y = torch.rand(100, dtype=torch.float64, device="cuda")
    with pytest.raises(nf.NufftError):
        nf.Plan(64, y, eps=1e-6, inverse=True)


def test_one_shot_calls(nf, orc):
    import torch
    N = M = 512
    y = workloads.points("jitter", N, N, seed=3, jitter=0.1)
    c = workloads.coeffs(N, seed=4)
    yd = _dev(y)
    g = nf.nufft_fwd(_dev(c), N, yd, M, 1e-12)
    gh = _host(g)
    assert orc.rel_l2(gh, orc.nudft_fwd(c, y)) < 1e-12
    ca = _host(nf.nufft_adj(g, yd, M, N, 1e-12))
    assert orc.rel_l2(ca, orc.nudft_adj(gh, y, N)) < 1e-12
    ci = _host(nf.inufft(g, yd, M, N, 1e-12))
    assert orc.rel_l2(ci, c) < 1e-11
