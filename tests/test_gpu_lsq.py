"""Least-squares INUFFT (M > N) by CG on the normal equations through the
C ABI, against a dense least-squares solve (small N), against the known
band-limited solution c_true of consistent data g = A c_true (any size), and
with the solver's reported residuals (the unweighted normal-equation
residual it stops on, the data residual) recomputed by the oracle, up to the
full least-squares workload (N = 2^16, M = 2^18)."""
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


def test_lsq_reported_residuals_match_oracle(nf, orc):
    """A solve stopped early (not converged): the reported data residual
    ||g - A c|| / ||g|| and normal-equation residual ||A^H (g - A c)|| /
    ||A^H g|| equal the oracle's direct sums (all targets, all frequencies)
    for the returned c."""
    N, M = 1 << 11, 1 << 13
    y = workloads.points("contrast", M, seed=11)
    c_true = workloads.coeffs(N, seed=12)
    g = orc.nudft_fwd(c_true, y)
    plan = nf.Plan(N, _dev(y), eps=1e-12)
    c, it, res = plan.solve_lsq(_dev(g), tol=1e-14, maxit=150, check=False, check_every=50)
    info = plan.lsq_info
    assert it == 150 and info["checks"] == 3 and len(info["history"]) == 3
    ch = _host(c)
    e = g - orc.nudft_fwd(ch, y)
    d_ref = np.linalg.norm(e) / np.linalg.norm(g)
    r_ref = np.linalg.norm(orc.nudft_adj(e, y, N)) / np.linalg.norm(orc.nudft_adj(g, y, N))
    assert abs(info["data_resid"] - d_ref) <= 1e-6 * d_ref
    assert abs(res - r_ref) <= 1e-6 * r_ref
    assert res == info["history"][-1]
    assert info["history"][0] > info["history"][-1]


def test_lsq_learned_weights_same_stopping_test(nf, orc):
    """Weighted (learned density compensation) and plain solves stop on the
    same unweighted residual, and both return c_true of consistent samples
    on a well-sampled set."""
    from paper_1611_09379_gb300 import dcf
    N, M = 1 << 10, 1 << 12
    y = workloads.points("uniform", M, seed=13)
    c_true = workloads.coeffs(N, seed=14)
    g = orc.nudft_fwd(c_true, y)
    plan = nf.Plan(N, _dev(y), eps=1e-12)
    w = plan.dcf_weights(dcf.load())
    assert abs(float(w.double().mean()) - 1.0) < 1e-6
    for ww in (None, w):
        c, it, res = plan.solve_lsq(_dev(g), ww, tol=1e-10, maxit=3000)
        assert res <= 1e-10
        assert orc.rel_l2(_host(c), c_true) < 1e-8


def test_inufft_one_shot_least_squares(nf, orc):
    """inufft(g, y, M, N, eps) with M > N returns the least-squares solution
    (plain CG through the library), equal to a dense solve; M < N is
    rejected."""
    import torch
    N, M = 256, 1024
    y = workloads.points("uniform", M, seed=15)
    c_true = workloads.coeffs(N, seed=16)
    g = orc.nudft_fwd(c_true, y) + 1e-3 * workloads.samples(M, seed=17)  # inconsistent data
    c = _host(nf.inufft(_dev(g), _dev(y), M, N, 1e-12))
    assert orc.rel_l2(c, orc.lsq_dense(g, y, N)) < 1e-9
    with pytest.raises(nf.NufftError) as e:
        nf.inufft(_dev(g[:100]), _dev(y[:100]), 100, N, 1e-12)
    assert e.value.code == nf.EINVAL
    del torch


def test_lsq_workload_size_against_oracle(nf, orc):
    """The least-squares workload at full size (N = 2^16, M = 2^18, 1:100
    density contrast, consistent samples of a random band-limited c_true):
    plain and learned-weight CG, each capped at 1200 iterations.  For both,
    the reported data residual equals the oracle's ||g - A c|| / ||g|| over
    all 2^18 points, A^H (g - A c) from the library's transforms equals the
    oracle's on 512 sampled frequencies, and the reported normal-equation
    residual agrees with the one estimated from those samples."""
    import torch
    from paper_1611_09379_gb300 import dcf
    N, M = 1 << 16, 1 << 18
    y = workloads.points("contrast", M, seed=1234)
    c_true = workloads.coeffs(N, seed=99)
    g = orc.nudft_fwd(c_true, y)
    gd = _dev(g)
    plan = nf.Plan(N, _dev(y), eps=1e-10)
    w = plan.dcf_weights(dcf.load())
    kdx = workloads.sample_index(N, 512, seed=8)
    ahg_ref = orc.nudft_adj(g, y, N, kdx)
    ahg = plan.adjoint(gd)
    ahg_norm = float(torch.linalg.vector_norm(ahg))
    assert orc.rel_l2(_host(ahg)[kdx], ahg_ref) < 1e-9
    out = {}
    for name, ww in (("plain", None), ("learned", w)):
        c, it, res = plan.solve_lsq(gd, ww, tol=1e-8, maxit=1200, check=False, check_every=300)
        info = dict(plan.lsq_info)
        ch = _host(c)
        e = g - orc.nudft_fwd(ch, y)
        d_ref = np.linalg.norm(e) / np.linalg.norm(g)
        assert abs(info["data_resid"] - d_ref) <= 1e-4 * d_ref, (name, info, d_ref)
        u = _host(plan.adjoint(gd - plan.forward(c)))
        u_ref = orc.nudft_adj(e, y, N, kdx)
        assert np.linalg.norm(u[kdx] - u_ref) <= 1e-6 * np.linalg.norm(u_ref), name
        assert abs(np.linalg.norm(u) / ahg_norm - res) <= 1e-4 * res, name
        est = np.sqrt(N / kdx.size) * np.linalg.norm(u_ref) / ahg_norm
        assert 0.5 * res <= est <= 2.0 * res, (name, est, res)
        out[name] = (it, res, d_ref)
    print("lsq at the workload size, 1200 iterations:", out)
