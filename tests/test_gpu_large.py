"""Large transforms through the C ABI, checked on sampled outputs the oracle
computes one by one: N = 2^21 (the FFT in three passes) in both precisions,
and the large workload N = M = 2^24, complex64 data, uniform points,
forward and adjoint at eps = 1e-6 (mixed precision)."""
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


@pytest.mark.parametrize("prec,eps,tol", [(0, 1e-12, 1e-12), (1, 1e-6, 1e-6)])
def test_three_pass_fft_2p21(nf, orc, prec, eps, tol):
    N = M = 1 << 21
    y = workloads.points("uniform", M, seed=31)
    c = workloads.coeffs(N, seed=32)
    g_in = workloads.samples(M, seed=33)
    plan = nf.Plan(N, _dev(y), eps=eps, prec=prec)
    g = plan.forward(_dev(c)).cpu().numpy()
    a = plan.adjoint(_dev(g_in)).cpu().numpy()
    idx = workloads.sample_index(M, 256)
    assert orc.rel_l2(g[idx], orc.nudft_fwd(c, y, idx)) < tol
    kdx = workloads.sample_index(N, 256, seed=5)
    assert orc.rel_l2(a[kdx], orc.nudft_adj(g_in, y, N, kdx)) < tol


def test_large_2p24_c64_forward_adjoint(nf, orc):
    N = M = 1 << 24
    y = workloads.points("uniform", M, seed=1238)
    c = workloads.coeffs(N, seed=34).astype(np.complex64)
    g_in = workloads.samples(M, seed=35).astype(np.complex64)
    plan = nf.Plan(N, _dev(y), eps=1e-6, prec=nf.MIXED, io="c64")
    g = plan.forward(_dev(c)).cpu().numpy()
    a = plan.adjoint(_dev(g_in)).cpu().numpy()
    plan.sync()
    idx = workloads.sample_index(M, 128)
    assert orc.rel_l2(g[idx], orc.nudft_fwd(c.astype(complex), y, idx)) < 1e-6
    kdx = workloads.sample_index(N, 128, seed=6)
    assert orc.rel_l2(a[kdx], orc.nudft_adj(g_in.astype(complex), y, N, kdx)) < 1e-6
