"""Transforms on the adaptive tree (plan flag NUFFT_ADAPTIVE): leaves holding
more points than the mean are refined by up to three levels.  Forward: their
targets evaluated at the deeper level (local expansions from the downward
pass continued with grid multipoles, near field over the 3 deeper boxes).
Adjoint / inverse: their sources as a deeper uniform tree for the near field,
the pairs that leaves through the deep boxes' multipoles and M2L into the
grid boxes.  Compared with the oracle's direct sums (Eq. p1, its adjoint,
Eq. p6) element by element, and with the uniform tree's results."""
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


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _fwd(nf, N, y, c, prec, adaptive, io="c128", **kw):
    import torch
    eps = 1e-12 if prec == 0 else 1e-6
    plan = nf.Plan(N, _dev(y), eps=eps, prec=prec, io=io, adaptive=adaptive, **kw)
    cc = c.astype(np.complex64) if io == "c64" else c
    g = plan.forward(_dev(cc))
    torch.cuda.synchronize()
    return g.cpu().numpy(), plan


@pytest.mark.parametrize("prec", [0, 1])
def test_adaptive_clustered_full(nf, orc, prec):
    """N = M = 4096, eight Gaussian clusters (6x the mean density at their
    centres): two extra levels, every target against the direct sums, and a
    graph replay gives the same bits."""
    N = M = 4096
    y = workloads.points("clustered", M, seed=41)
    c = workloads.coeffs(N, seed=42)
    g, plan = _fwd(nf, N, y, c, prec, True)
    lv, cnt = plan.adaptive()
    assert lv == 2 and sum(cnt) == M and cnt[1] > 0 and cnt[2] > 0
    assert orc.rel_l2(g, orc.nudft_fwd(c, y)) < TOL[prec]
    import torch
    g2 = plan.forward(_dev(c))
    torch.cuda.synchronize()
    assert np.array_equal(g2.cpu().numpy(), g)


@pytest.mark.parametrize("prec", [0, 1])
def test_adaptive_matches_uniform_tree(nf, orc, prec):
    """The same clustered points on both trees: the two results agree to the
    requested accuracy (both are within eps of the direct sums)."""
    N = M = 1 << 14
    y = workloads.points("clustered", M, seed=43)
    c = workloads.coeffs(N, seed=44)
    ga, pa = _fwd(nf, N, y, c, prec, True)
    gu, pu = _fwd(nf, N, y, c, prec, False)
    assert pa.adaptive()[0] >= 1 and pu.adaptive()[0] == 0
    assert orc.rel_l2(ga, gu) < 2 * TOL[prec]
    idx = workloads.sample_index(M, 256, seed=5)
    assert orc.rel_l2(ga[idx], orc.nudft_fwd(c, y, idx)) < TOL[prec]


@pytest.mark.parametrize("prec", [0, 1])
def test_adaptive_three_levels_sampled(nf, orc, prec):
    """N = 2^16, M = 2^14 (64 grid points per leaf, so up to three extra
    levels) on clusters of four widths over a uniform background: every
    depth class present, sampled targets and the densest class's targets
    against the direct sums."""
    N, M = 1 << 16, 1 << 14
    y = workloads.points("multiscale", M, seed=45)
    c = workloads.coeffs(N, seed=46)
    g, plan = _fwd(nf, N, y, c, prec, True)
    lv, cnt = plan.adaptive()
    assert lv == 3 and all(v > 0 for v in cnt), cnt
    idx = workloads.sample_index(M, 512, seed=6)
    assert orc.rel_l2(g[idx], orc.nudft_fwd(c, y, idx)) < TOL[prec]
    # the densest targets (refined three levels) on their own
    perm, start, _, _ = plan.points()
    from paper_1611_09379_gb300 import adaptive_depths
    st = start.cpu().numpy()
    _, dep = adaptive_depths(st, N >> plan.info()["lmax"])
    b3 = np.flatnonzero(dep == 3)[:4]
    pm = perm.cpu().numpy()
    j3 = np.concatenate([pm[st[b]:st[b + 1]] for b in b3])[:256]
    assert orc.rel_l2(g[j3], orc.nudft_fwd(c, y, j3)) < TOL[prec]


def test_adaptive_uniform_points_stay_uniform(nf):
    """Uniform points refine nothing: the adaptive plan runs the uniform
    tree and returns the same bits."""
    N = M = 1 << 14
    y = workloads.points("uniform", M, seed=47)
    c = workloads.coeffs(N, seed=48)
    ga, pa = _fwd(nf, N, y, c, 1, True)
    gu, _ = _fwd(nf, N, y, c, 1, False)
    assert pa.adaptive() == (0, [M, 0, 0, 0])
    assert np.array_equal(ga, gu)


@pytest.mark.parametrize("prec", [0, 1])
def test_adaptive_few_points_in_one_cluster(nf, orc, prec):
    """N = 2^16 with 60 points in one narrow cluster: the leaves are wide
    (1024 grid points), the occupied ones refined three levels (128 grid
    points per box)."""
    N, M = 1 << 16, 60
    g0 = workloads.rng(49)
    y = np.mod(1.0 + 2e-3 * g0.standard_normal(M), 2 * np.pi)
    c = workloads.coeffs(N, seed=50)
    g, plan = _fwd(nf, N, y, c, prec, True)
    lv, cnt = plan.adaptive()
    assert lv == 3 and cnt[3] > 0
    assert orc.rel_l2(g, orc.nudft_fwd(c, y)) < TOL[prec]


def test_adaptive_general_n_c64(nf, orc):
    """A coefficient count that is not a power of two (N = 3000 on the grid
    2^12) with complex64 input and output."""
    N, M = 3000, 3000
    y = workloads.points("clustered", M, seed=51)
    c = workloads.coeffs(N, seed=52)
    g, plan = _fwd(nf, N, y, c, 1, True, io="c64")
    assert plan.adaptive()[0] >= 1
    assert g.dtype == np.complex64
    assert orc.rel_l2(g, orc.nudft_fwd(c.astype(np.complex64).astype(complex), y)) < 1e-6


def test_adaptive_rejects_batches(nf):
    y = workloads.points("clustered", 1024, seed=53)
    with pytest.raises(nf.NufftError) as e:
        nf.Plan(1024, _dev(y), eps=1e-6, prec=1, batch=2, adaptive=True)
    assert e.value.code == nf.ENOTSUP


def _adj(nf, N, y, gs, prec, adaptive):
    import torch
    eps = 1e-12 if prec == 0 else 1e-6
    plan = nf.Plan(N, _dev(y), eps=eps, prec=prec, adaptive=adaptive)
    c = plan.adjoint(_dev(gs))
    torch.cuda.synchronize()
    return c.cpu().numpy(), plan


@pytest.mark.parametrize("prec", [0, 1])
def test_adaptive_adjoint_clustered_full(nf, orc, prec):
    """Adjoint, N = M = 4096 on the eight-cluster mixture (two extra levels):
    every coefficient against the direct sums; a replay gives the same bits."""
    N = M = 4096
    y = workloads.points("clustered", M, seed=41)
    gs = workloads.samples(M, seed=55)
    c, plan = _adj(nf, N, y, gs, prec, True)
    assert plan.adaptive()[0] == 2
    assert orc.rel_l2(c, orc.nudft_adj(gs, y, N)) < TOL[prec]
    import torch
    c2 = plan.adjoint(_dev(gs))
    torch.cuda.synchronize()
    assert np.array_equal(c2.cpu().numpy(), c)


@pytest.mark.parametrize("prec", [0, 1])
def test_adaptive_adjoint_three_levels_sampled(nf, orc, prec):
    """Adjoint, N = 2^16, M = 2^14 on clusters of four widths (every depth
    class present): sampled coefficients against the direct sums, and the
    uniform tree's result on the same points."""
    N, M = 1 << 16, 1 << 14
    y = workloads.points("multiscale", M, seed=45)
    gs = workloads.samples(M, seed=56)
    c, plan = _adj(nf, N, y, gs, prec, True)
    lv, cnt = plan.adaptive()
    assert lv == 3 and all(v > 0 for v in cnt), cnt
    kdx = workloads.sample_index(N, 512, seed=8)
    assert orc.rel_l2(c[kdx], orc.nudft_adj(gs, y, N, kdx)) < TOL[prec]
    cu, _ = _adj(nf, N, y, gs, prec, False)
    assert orc.rel_l2(c, cu) < 2 * TOL[prec]


def _two_density(N):
    """N points equispaced at two densities: 48 % of them on [0, 0.4 pi)."""
    n1 = int(N * 0.48)
    a = 0.4 * np.pi
    return np.concatenate([(np.arange(n1) + 0.5) * a / n1,
                           a + (np.arange(N - n1) + 0.5) * (2 * np.pi - a) / (N - n1)])


@pytest.mark.parametrize("prec,N,kind", [(0, 128, "two"), (1, 128, "two"), (0, 512, "clustered")])
def test_adaptive_inverse_matvec(nf, orc, prec, N, kind):
    """Square inverse on point sets whose density varies enough to refine a
    leaf while the Lagrange weights (Eq. p8) still fit the arithmetic: the
    matrix-vector product f = L g (Eq. p6) against the oracle's, relative to
    sum_j |L_kj| |g_j| (reading c16), as on the uniform tree."""
    y = _two_density(N) if kind == "two" else workloads.points("clustered", N, seed=33)
    g = workloads.samples(N, seed=34)
    eps = 1e-12 if prec == 0 else 1e-6
    plan = nf.Plan(N, _dev(y), eps=eps, prec=prec, inverse=True, adaptive=True)
    assert plan.adaptive()[0] >= 1
    import torch
    c2 = plan.inverse(_dev(g))
    torch.cuda.synchronize()
    f = np.fft.ifft(c2.cpu().numpy()) * N
    fref = orc.inverse_f(g, y, N)
    aref = orc.inverse_absf(g, y, N)
    sc = aref.max()
    assert np.all(np.isfinite(f)) and sc < np.inf
    assert np.linalg.norm((f - fref) / sc) / np.linalg.norm(aref / sc) < TOL[prec]
