"""M2L + L2L on the tensor cores (three TF32 passes, FP32 accumulation)
through the C ABI: the tensor-core levels give the oracle's result at the
mixed tolerance, and agree with the FP32 SIMT kernels, for forward, adjoint
and inverse, partial tiles (levels with fewer than 64 parents), batches and
the range of expansion orders p the mixed path uses."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu
TOL = 1e-6  # mixed path, relative L2 against the FP64 oracle


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


@pytest.mark.parametrize("eps", [1e-3, 1e-6, 1e-7])
def test_tc_forward_adjoint_all_levels(nf, orc, eps):
    """Every level from 4 to l_max on the tensor cores (levels 4..6 hold 8..32
    parents: partial tiles), against the oracle and the SIMT path."""
    N, M = 1 << 14, 20000
    y = workloads.points("uniform", M, seed=41)
    c = workloads.coeffs(N, seed=42)
    gs = workloads.samples(M, seed=43)
    tc = nf.Plan(N, _dev(y), eps=eps, prec=nf.MIXED, tc_level=4)
    simt = nf.Plan(N, _dev(y), eps=eps, prec=nf.MIXED, tc_level=-1)
    prm = tc.params()
    assert prm["tc_level"] == 4 and simt.params()["tc_level"] == -1
    g_tc = tc.forward(_dev(c)).cpu().numpy()
    a_tc = tc.adjoint(_dev(gs)).cpu().numpy()
    tc.sync()
    g_s = simt.forward(_dev(c)).cpu().numpy()
    a_s = simt.adjoint(_dev(gs)).cpu().numpy()
    tol = max(TOL, 10 * eps)
    idx = workloads.sample_index(M, 2048)
    assert orc.rel_l2(g_tc[idx], orc.nudft_fwd(c, y, idx)) < tol
    assert orc.rel_l2(a_tc, orc.nudft_adj(gs, y, N)) < tol
    # the two engines differ by FP32 rounding only
    assert orc.rel_l2(g_tc, g_s) < 1e-6
    assert orc.rel_l2(a_tc, a_s) < 1e-6


def test_tc_automatic_level_2p20(nf, orc):
    """The bench workload's plan (N = M = 2^20, jittered points): the
    automatic choice puts the finest levels on the tensor cores."""
    N = M = 1 << 20
    y = workloads.points("jitter", M, N, seed=1234, jitter=0.4)
    c = workloads.coeffs(N, seed=99)
    plan = nf.Plan(N, _dev(y), eps=1e-6, prec=nf.MIXED)
    prm = plan.params()
    assert 4 <= prm["tc_level"] <= prm["lmax"]
    g = plan.forward(_dev(c)).cpu().numpy()
    plan.sync()
    idx = workloads.sample_index(M, 1024)
    assert orc.rel_l2(g[idx], orc.nudft_fwd(c, y, idx)) < TOL


def test_tc_inverse_roundtrip(nf, orc):
    N = 1 << 12
    y = workloads.points("jitter", N, N, seed=7, jitter=0.1)
    c = workloads.coeffs(N, seed=8)
    g = orc.nudft_fwd(c, y)
    plan = nf.Plan(N, _dev(y), eps=1e-6, prec=nf.MIXED, inverse=True, tc_level=4)
    c2 = plan.inverse(_dev(g)).cpu().numpy()
    plan.sync()
    assert orc.rel_l2(c2, c) < 1e-5


@pytest.mark.parametrize("batch", [3, 16])
def test_tc_batched(nf, orc, batch):
    """Signals as extra GEMM rows: every signal of a batch matches the oracle."""
    N = M = 1 << 13
    y = workloads.points("uniform", M, seed=batch)
    C = np.stack([workloads.coeffs(N, seed=50 + b) for b in range(batch)]).astype(np.complex64)
    plan = nf.Plan(N, _dev(y), eps=1e-6, prec=nf.MIXED, io="c64", batch=batch, tc_level=5)
    g = plan.forward(_dev(C)).cpu().numpy()
    plan.sync()
    idx = workloads.sample_index(M, 512)
    for b in range(batch):
        ref = orc.nudft_fwd(C[b].astype(complex), y, idx)
        assert orc.rel_l2(g[b][idx], ref) < TOL


def test_tc_clustered_points(nf, orc):
    N = M = 1 << 15
    y = workloads.points("clustered", M, seed=9)
    c = workloads.coeffs(N, seed=10)
    plan = nf.Plan(N, _dev(y), eps=1e-6, prec=nf.MIXED, tc_level=6)
    g = plan.forward(_dev(c)).cpu().numpy()
    plan.sync()
    idx = workloads.sample_index(M, 1024)
    assert orc.rel_l2(g[idx], orc.nudft_fwd(c, y, idx)) < TOL


@pytest.mark.parametrize("kind,N,M", [("uniform", 1 << 14, 1 << 14), ("clustered", 1 << 13, 1 << 13),
                                      ("uniform", 1 << 12, 3001)])
def test_tc_near_field_batched_forward(nf, orc, kind, N, M):
    """64 signals: the near field as a tensor-core GEMM matches the oracle and
    the SIMT kernels (clustered points: sparse windows, many chunks; M not a
    multiple of the tile: a ragged last tile)."""
    batch = 64
    y = workloads.points(kind, M, seed=71)
    C = (workloads.rng(72).standard_normal((batch, N)) +
         1j * workloads.rng(73).standard_normal((batch, N))).astype(np.complex64)
    tc = nf.Plan(N, _dev(y), eps=1e-6, prec=nf.MIXED, io="c64", batch=batch, tc_near=1)
    simt = nf.Plan(N, _dev(y), eps=1e-6, prec=nf.MIXED, io="c64", batch=batch, tc_near=-1)
    assert tc.params()["tc_near"] == 1 and simt.params()["tc_near"] == -1
    g = tc.forward(_dev(C)).cpu().numpy()
    tc.sync()
    gs = simt.forward(_dev(C)).cpu().numpy()
    assert orc.rel_l2(g, gs) < 1e-6
    idx = workloads.sample_index(M, 256)
    for b in (0, 33, 63):
        ref = orc.nudft_fwd(C[b].astype(complex), y, idx)
        assert orc.rel_l2(g[b][idx], ref) < 1e-6
