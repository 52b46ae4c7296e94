"""Batched transforms (many signals sharing one point set) through the C ABI:
every signal of a batch equals the single-signal transform of that signal
and the oracle, for forward, adjoint and inverse, both precisions."""
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


@pytest.mark.parametrize("batch", [4, 3, 8])
@pytest.mark.parametrize("prec", [0, 1])
def test_batched_forward_adjoint(nf, orc, batch, prec):
    import torch
    N, M = 2048, 3000
    eps = 1e-12 if prec == 0 else 1e-6
    y = workloads.points("uniform", M, seed=batch)
    C = np.stack([workloads.coeffs(N, seed=10 + b) for b in range(batch)])
    Gs = np.stack([workloads.samples(M, seed=20 + b) for b in range(batch)])
    plan = nf.Plan(N, _dev(y), eps=eps, prec=prec, batch=batch)
    g = plan.forward(_dev(C)).cpu().numpy()
    c = plan.adjoint(_dev(Gs)).cpu().numpy()
    single = nf.Plan(N, _dev(y), eps=eps, prec=prec)
    for b in range(batch):
        assert orc.rel_l2(g[b], orc.nudft_fwd(C[b], y)) < TOL[prec]
        assert orc.rel_l2(c[b], orc.nudft_adj(Gs[b], y, N)) < TOL[prec]
        gs = single.forward(_dev(C[b])).cpu().numpy()
        assert np.abs(g[b] - gs).max() <= 1e-6 * np.abs(gs).max()


def test_batched_inverse_c64(nf, orc):
    N = 1024
    batch = 8
    y = workloads.points("jitter", N, N, seed=3, jitter=0.1)
    C = np.stack([workloads.coeffs(N, seed=30 + b) for b in range(batch)])
    G = np.stack([orc.nudft_fwd(C[b], y) for b in range(batch)]).astype(np.complex64)
    plan = nf.Plan(N, _dev(y), eps=1e-6, prec=nf.MIXED, io="c64", inverse=True, batch=batch)
    c = plan.inverse(_dev(G)).cpu().numpy()
    for b in range(batch):
        assert orc.rel_l2(c[b], C[b]) < 1e-5  # complex64 input samples


def test_batched_64_signals_2p18_sampled(nf, orc):
    """The batched workload's shape: 64 complex64 signals, N = M = 2^18,
    uniform points, eps = 1e-6 (sampled targets per signal)."""
    N = M = 1 << 18
    batch = 64
    y = workloads.points("uniform", M, seed=1234)
    rng = workloads.rng(5)
    C = (rng.standard_normal((batch, N)) + 1j * rng.standard_normal((batch, N))).astype(np.complex64)
    plan = nf.Plan(N, _dev(y), eps=1e-6, prec=nf.MIXED, io="c64", batch=batch)
    g = plan.forward(_dev(C)).cpu().numpy()
    idx = workloads.sample_index(M, 256)
    for b in (0, 17, 63):
        ref = orc.nudft_fwd(C[b].astype(complex), y, idx)
        assert orc.rel_l2(g[b][idx], ref) < 1e-6
