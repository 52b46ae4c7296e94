"""Exec calls replay CUDA graphs of their kernel sequences: results equal,
bit for bit, those of kernels launched one by one, for repeated calls on the
same buffers (replay, with the inputs changed in place), for new buffers (a
new capture) and for every operation, and the graph path steps aside while
profiling."""
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


@pytest.mark.parametrize("prec,eps", [(0, 1e-12), (1, 1e-6)])
def test_graph_replay_matches_direct_launches(nf, prec, eps):
    import torch
    N = M = 1 << 14
    y = workloads.points("jitter", M, N, seed=61, jitter=0.1)
    c1, c2 = workloads.coeffs(N, seed=62), workloads.coeffs(N, seed=63)
    gp = nf.Plan(N, _dev(y), eps=eps, prec=prec, inverse=True)
    dp = nf.Plan(N, _dev(y), eps=eps, prec=prec, inverse=True, graphs=False)
    cin = _dev(c1)
    g = torch.empty(M, dtype=torch.complex128, device="cuda")
    for rep in range(3):
        if rep == 2:
            cin.copy_(_dev(c2))  # same buffer, new contents: the replay reads them
        gp.forward(cin, out=g)
        ref = dp.forward(cin)
        assert torch.equal(g, ref)
    # other buffers and the other operations
    g2 = gp.forward(_dev(c1))
    assert torch.equal(g2, dp.forward(_dev(c1)))
    for _ in range(2):
        a = gp.adjoint(g)
        assert torch.equal(a, dp.adjoint(g))
        ci = gp.inverse(g)
        assert torch.equal(ci, dp.inverse(g))
    gp.profile(True)  # profiled calls launch directly; same results
    assert torch.equal(gp.forward(cin), ref)
    gp.profile(False)
    gp.sync()
