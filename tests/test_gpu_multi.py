"""Uneven batches: independent forward transforms of different N, M and
points, executed as one CUDA graph launch, against the oracle (sampled) and
the single-plan path; replays give identical results."""
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


def test_uneven_batch_graph(nf, orc):
    import torch
    rng = workloads.rng(12)
    U = rng.integers(10, 17, size=24)  # N = M = 2^U, U in 10..16 (the batched workload's range)
    U[:2] = [10, 16]                   # both ends present
    Ns = [1 << int(u) for u in U]
    ys = [torch.from_numpy(workloads.points("uniform", n, seed=100 + i)).cuda() for i, n in enumerate(Ns)]
    cs_h = [workloads.coeffs(n, seed=200 + i).astype(np.complex64) for i, n in enumerate(Ns)]
    cs = [torch.from_numpy(c).cuda() for c in cs_h]
    gs = [torch.empty(n, dtype=torch.complex64, device="cuda") for n in Ns]
    multi = nf.Multi(Ns, ys, eps=1e-6, prec=nf.MIXED, io="c64")
    multi.forward(cs, gs)
    first = [g.cpu().numpy().copy() for g in gs]
    for g in gs:
        g.zero_()
    multi.forward(cs, gs)  # replay of the captured graph
    for i, n in enumerate(Ns):
        g = gs[i].cpu().numpy()
        assert np.array_equal(g, first[i])
        yh = ys[i].cpu().numpy()
        idx = workloads.sample_index(n, 128, seed=i)
        ref = orc.nudft_fwd(cs_h[i].astype(complex), yh, idx)
        assert orc.rel_l2(g[idx], ref) < 1e-6, (i, n)
    single = nf.Plan(Ns[0], ys[0], eps=1e-6, prec=nf.MIXED, io="c64")
    gs0 = single.forward(cs[0]).cpu().numpy()
    assert np.abs(gs0 - first[0]).max() <= 1e-6 * np.abs(gs0).max()


def test_uneven_batch_with_parameters(nf, orc):
    """Per-transform parameters (as the autotuner gives per size class: lower
    p and q than the formulas' at the formulas' depth): each transform agrees
    with a single plan of the same parameters and meets 1e-6 against the
    oracle; a wrong-length parameter list is rejected."""
    import torch
    Ns = [1 << 10, 1 << 13, 1 << 16, 1 << 12]
    ys = [torch.from_numpy(workloads.points("uniform", n, seed=300 + i)).cuda() for i, n in enumerate(Ns)]
    cs_h = [workloads.coeffs(n, seed=400 + i).astype(np.complex64) for i, n in enumerate(Ns)]
    cs = [torch.from_numpy(c).cuda() for c in cs_h]
    gs = [torch.empty(n, dtype=torch.complex64, device="cuda") for n in Ns]
    prm = []
    for n in Ns:
        d = nf.choose_params_full(n, n, 1e-6, nf.MIXED)
        prm.append({"lmax": d["lmax"], "p": 11, "q": 5, "tc_level": -1, "tc_near": -1})
    multi = nf.Multi(Ns, ys, eps=1e-6, prec=nf.MIXED, io="c64", params=prm)
    multi.forward(cs, gs)
    for i, n in enumerate(Ns):
        g = gs[i].cpu().numpy()
        single = nf.Plan(n, ys[i], eps=1e-6, prec=nf.MIXED, io="c64", lmax=prm[i]["lmax"], p=11, q=5,
                         tc_level=-1)
        assert single.params()["p"] == 11 and single.params()["q"] == 5
        gsng = single.forward(cs[i]).cpu().numpy()
        assert np.abs(gsng - g).max() <= 1e-6 * np.abs(gsng).max(), i
        idx = workloads.sample_index(n, 128, seed=i)
        assert orc.rel_l2(g[idx], orc.nudft_fwd(cs_h[i].astype(complex), ys[i].cpu().numpy(), idx)) < 1e-6
    with pytest.raises(ValueError):
        nf.Multi(Ns, ys, eps=1e-6, prec=nf.MIXED, io="c64", params=prm[:2])
