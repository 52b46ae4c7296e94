"""Autotuner through the C ABI: the chosen parameters are among the
candidates tried, the plan made with them matches the FP64 oracle at the
requested tolerance, and the persistent table returns the same choice
without searching again."""
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


@pytest.mark.parametrize("prec,eps,ops", [(1, 1e-6, "fwd"), (1, 1e-6, "fwd+inv"), (0, 1e-12, "fwd+adj")])
def test_autotune_choice_is_accurate(nf, orc, tmp_path, prec, eps, ops):
    from paper_1611_09379_gb300 import tune
    N = M = 1 << 14
    y = workloads.points("jitter", M, N, seed=21, jitter=0.4)
    c = workloads.coeffs(N, seed=22)
    path = str(tmp_path / "tune.json")
    ent = tune.autotune(N, _dev(y), eps, prec=prec, ops=ops, reps=3, tag="jitter", path=path)
    assert not ent["from_table"]
    trials = ent["trials"]
    assert len(trials) >= 4
    chosen = [t for t in trials if t["accepted"]]
    assert chosen and all(t["params"] == ent["params"] for t in chosen)
    # the choice is at least as fast as the formula's parameters (trial 0)
    assert min(t["ms"] for t in chosen) <= trials[0]["ms"] * 1.0001
    # and within the accuracy rule
    assert all(t["err"] <= max(0.25 * eps, min(1.5 * trials[0]["err"], 0.5 * eps))
               or t["params"] == trials[0]["params"] for t in chosen)
    plan = tune.tuned_plan(N, _dev(y), eps, prec=prec, ops=ops, tag="jitter", path=path)
    assert plan.params()["lmax"] == ent["params"]["lmax"]
    g = plan.forward(_dev(c)).cpu().numpy()
    idx = workloads.sample_index(M, 1024)
    assert orc.rel_l2(g[idx], orc.nudft_fwd(c, y, idx)) < eps
    # second call: from the table, same parameters
    again = tune.autotune(N, _dev(y), eps, prec=prec, ops=ops, tag="jitter", path=path)
    assert again["from_table"] and again["params"] == ent["params"]


def test_autotune_batched_c64(nf, orc, tmp_path):
    from paper_1611_09379_gb300 import tune
    N = M = 1 << 13
    batch = 8
    y = workloads.points("uniform", M, seed=23)
    ent = tune.autotune(N, _dev(y), 1e-6, prec=nf.MIXED, io="c64", batch=batch, ops="fwd",
                        reps=2, path=str(tmp_path / "t.json"))
    p = ent["params"]
    assert p["batch"] == batch
    C = np.stack([workloads.coeffs(N, seed=60 + b) for b in range(batch)]).astype(np.complex64)
    plan = nf.Plan(N, _dev(y), eps=1e-6, prec=nf.MIXED, io="c64", batch=batch, lmax=p["lmax"],
                   p=p["p"], q=p["q"], tc_level=p["tc_level"])
    g = plan.forward(_dev(C)).cpu().numpy()
    idx = workloads.sample_index(M, 256)
    for b in (0, 7):
        assert orc.rel_l2(g[b][idx], orc.nudft_fwd(C[b].astype(complex), y, idx)) < 1e-6
