"""Learned density compensation: the network's GPU gradients against the FP64
oracle, features of a plan against the batched training features, and what
the trained network gains over plain CG in the least-squares INUFFT."""
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


def test_mlp_gradient_matches_oracle(nf):
    import torch
    from oracle import mlp as omlp
    from paper_1611_09379_gb300 import dcf
    rng = np.random.default_rng(1)
    p = dcf.init_params(3)
    X = rng.standard_normal((3000, 8)).astype(np.float32)
    t = (0.5 * rng.standard_normal(3000)).astype(np.float32)
    m = nf.MLP(p)
    g, loss = m.grad(torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda())
    gref, lref = omlp.grad(p.astype(np.float64), X.astype(np.float64), t.astype(np.float64))
    assert abs(loss - lref) <= 1e-4 * lref
    assert np.abs(g - gref).max() <= 1e-4 * np.abs(gref).max()


def test_mlp_inference_bf16_weights(nf):
    """Inference with BF16-rounded weights and FP32 accumulation stays within
    the BF16 rounding of the FP64 network."""
    import torch
    from oracle import mlp as omlp
    from paper_1611_09379_gb300 import dcf
    p = dcf.init_params(5)
    X = np.random.default_rng(2).standard_normal((5000, 8)).astype(np.float32)
    w = nf.MLP(p).infer(torch.from_numpy(X).cuda()).cpu().numpy()
    wref = omlp.forward(p.astype(np.float64), X.astype(np.float64))
    assert np.abs(np.log(w) - np.log(wref)).max() < 0.05


def test_dcf_targets_match_reference_iteration(nf):
    """The GPU fixed-point density-compensation targets equal the FP64
    reference iteration (oracle) up to FP32 rounding."""
    import torch
    from oracle import mlp as omlp
    sets = np.stack([np.sort(workloads.points("contrast", 512, seed=300 + i)) for i in range(3)])
    got = nf.dcf_targets(torch.from_numpy(sets).cuda(), 128, iters=100).cpu().numpy().reshape(3, 512)
    for i in range(3):
        ref = omlp.dcf_fixed_point(sets[i], 128, iters=100)
        assert np.abs(np.exp(got[i]) - np.exp(ref)).max() < 2e-2  # weights have mean 1
        assert np.std(ref) > 0.3  # the weights do vary over the contrast family


def test_plan_features_equal_batched_features(nf):
    import torch
    N, M = 1 << 10, 1 << 12
    y = workloads.points("contrast", M, seed=4)
    plan = nf.Plan(N, torch.from_numpy(y).cuda(), eps=1e-6)
    f_plan = plan.dcf_features().cpu().numpy()
    order = np.argsort(y, kind="stable")
    f_sorted = nf.dcf_features_sorted(torch.from_numpy(y[order][None, :].copy()).cuda()).cpu().numpy()
    assert np.abs(f_plan[order] - f_sorted).max() < 1e-4


def test_training_reduces_loss(nf):
    """The library's forward/backward/Adam kernels train the network: the loss
    on 3000 generated point sets (N = 256, M = 1024) falls by 40 % or more in
    10 epochs."""
    from paper_1611_09379_gb300 import dcf
    sets = np.stack([workloads.points("contrast", 1024, seed=1000 + i) for i in range(3000)])
    feat, target = dcf.training_data(sets, 256)
    mlp, losses = dcf.train(feat, target, epochs=10)
    assert losses[-1] < 0.6 * losses[0]


def test_learned_weights_reduce_cg_iterations(nf, orc):
    """The shipped network (trained on the GPU by the library's kernels on 10k
    generated point sets at N = 256, M = 1024) against plain CG on a 4x
    oversampled 1:100 contrast problem at N = 2^12: both solves stop on the
    same test, the unweighted normal-equation residual recomputed from the
    iterate (<= 1e-8), the learned weights in fewer iterations; the reported
    data residual equals the oracle's."""
    import torch
    from paper_1611_09379_gb300 import dcf
    mlp = dcf.load()
    N, M = 1 << 12, 1 << 14
    y = workloads.points("contrast", M, seed=77)
    c_true = workloads.coeffs(N, seed=78)
    g = orc.nudft_fwd(c_true, y)
    plan = nf.Plan(N, torch.from_numpy(y).cuda(), eps=1e-12)
    gd = torch.from_numpy(g).cuda()
    _, it_plain, r_plain = plan.solve_lsq(gd, tol=1e-8, maxit=40000)
    w = dcf.weights(plan, mlp)
    c, it_learn, r_learn = plan.solve_lsq(gd, w, tol=1e-8, maxit=40000)
    assert r_plain <= 1e-8 and r_learn <= 1e-8
    print("iterations plain", it_plain, "learned", it_learn)
    assert it_learn < 0.8 * it_plain, (it_learn, it_plain)
    d_ref = orc.rel_l2(orc.nudft_fwd(c.cpu().numpy(), y), g)
    assert abs(plan.lsq_info["data_resid"] - d_ref) <= 1e-4 * d_ref
