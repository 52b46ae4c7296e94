"""Machine-precision mode (Sec. 3.1-3.2): eps = 0 prescribes the FP64 path's
threshold error eps_th(N) (nufft_eps_threshold) and takes p, q from Eq. 18.2
at it.  Checked with the paper's analytic test (f = 1, exact answer g = 1:
eps_a = max_j |g_j - 1| over all points) and against the oracle's direct
sum: the error is at the threshold (no smaller eps helps) and within it."""
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


@pytest.mark.parametrize("N", [1 << 8, 1 << 12, 1 << 16, 1 << 20, 50000])
def test_machine_precision_mode(nf, orc, N):
    import torch
    M = N
    y = workloads.points("uniform", M, seed=900 + N % 97)
    yd = torch.from_numpy(y).cuda()
    e0 = torch.zeros(N, dtype=torch.complex128, device="cuda")
    e0[0] = 1.0
    eth = nf.eps_threshold(N)
    plan = nf.Plan(N, yd, eps=0.0, prec=nf.FP64)
    ea = float((plan.forward(e0) - 1.0).abs().max())
    assert ea <= 1.5 * eth, (ea, eth)
    # at the floor: prescribing the smallest eps accepted does not do better
    deep = nf.Plan(N, yd, eps=1e-15, prec=nf.FP64)
    ea_deep = float((deep.forward(e0) - 1.0).abs().max())
    assert ea <= 1.5 * ea_deep + 1e-16
    c = workloads.coeffs(N, seed=5)
    g = plan.forward(torch.from_numpy(c).cuda()).cpu().numpy()
    idx = workloads.sample_index(M, 512, seed=6)
    assert orc.rel_l2(g[idx], orc.nudft_fwd(c, y, idx)) < eth
    info = plan.params()
    assert info["p"] <= 64 and info["q"] <= 32
