"""Least-squares INUFFT (M > N) by CG on the normal equations through the
C ABI, against a dense least-squares solve (small N) and against the known
band-limited solution c_true of consistent data g = A c_true (any size)."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


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


def _host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.mark.parametrize("weighted", [False, True])
def test_lsq_small_matches_dense_solve(nf, orc, weighted):
    """Uniform points with M = 4N (a well-posed least-squares problem)."""
    N, M = 256, 1024
    y = workloads.points("uniform", M, seed=5)
    c_true = workloads.coeffs(N, seed=6)
    g = orc.nudft_fwd(c_true, y)
    w = (np.random.default_rng(2).random(M) + 0.5).astype(np.float32) if weighted else None
    plan = nf.Plan(N, _dev(y), eps=1e-13)
    c, it, res = plan.solve_lsq(_dev(g), None if w is None else _dev(w), tol=1e-12, maxit=3000)
    c = _host(c)
    assert res <= 1e-12
    cref = orc.lsq_dense(g, y, N, w)
    assert orc.rel_l2(c, cref) < 1e-8
    assert orc.rel_l2(c, c_true) < 1e-8


def test_lsq_uniform_recovers_band_limited_solution(nf, orc):
    """M = 4N uniform points at N = 2^12: CG reaches 1e-10 and returns c_true
    of the consistent samples."""
    N, M = 1 << 12, 1 << 14
    y = workloads.points("uniform", M, seed=7)
    c_true = workloads.coeffs(N, seed=8)
    g = orc.nudft_fwd(c_true, y)
    plan = nf.Plan(N, _dev(y), eps=1e-12)
    c, it, res = plan.solve_lsq(_dev(g), tol=1e-10, maxit=5000)
    c = _host(c)
    assert res <= 1e-10
    assert orc.rel_l2(c, c_true) < 1e-8


def test_lsq_contrast_residual(nf, orc):
    """1:100 density contrast (the learned-weights workload): the sparse arcs
    are below Nyquist, so c is not determined there, but CG still drives the
    normal-equation residual to 1e-8 and the solution reproduces the samples."""
    N, M = 1 << 11, 1 << 13
    y = workloads.points("contrast", M, seed=7)
    c_true = workloads.coeffs(N, seed=8)
    g = orc.nudft_fwd(c_true, y)
    plan = nf.Plan(N, _dev(y), eps=1e-12)
    c, it, res = plan.solve_lsq(_dev(g), tol=1e-8, maxit=20000)
    assert res <= 1e-8
    idx = workloads.sample_index(M, 512)
    assert orc.rel_l2(orc.nudft_fwd(_host(c), y, idx), g[idx]) < 1e-4


def test_lsq_zero_data_and_nonconvergence(nf):
    import torch
    N, M = 64, 256
    y = _dev(workloads.points("uniform", M, seed=1))
    plan = nf.Plan(N, y, eps=1e-12)
    g = torch.zeros(M, dtype=torch.complex128, device="cuda")
    c, it, res = plan.solve_lsq(g)
    assert it == 0 and float(_host(c.abs()).max()) == 0.0
    g = _dev(workloads.samples(M, seed=3))  # inconsistent data still converges (normal equations)
    c, it, res = plan.solve_lsq(g, tol=1e-30, maxit=3, check=False)
    assert it == 3
    with pytest.raises(nf.NufftError) as e:
        plan.solve_lsq(g, tol=1e-30, maxit=3)
    assert e.value.code == nf.ENOTCONV
