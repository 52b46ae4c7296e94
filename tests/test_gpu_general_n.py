"""Grid sizes N that are not powers of two, through the C ABI.

The series of Eq. p1 with N coefficients is the series with N' =
2^ceil(log2 N) coefficients whose top N' - N are zero, so the library runs
the FMM and its FFT on the N' grid (zero padding on input, truncation on
output inside the FFT passes).  The oracle evaluates the definitions
directly at N: the direct NUDFT with exact phases (forward, adjoint) and a
dense least-squares solve; its grid routes are pinned at non-power-of-two N
by the closed forms in test_oracle_pins.py (the square inverse by its round
trip and a dense solve)."""
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


def _host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("N,M,kind", [(1000, 1000, "uniform"), (3 << 10, 2500, "clustered"),
                                      (12345, 12345, "uniform"), ((1 << 16) - 1, 4096, "uniform"),
                                      (100000, 100000, "clustered"), (9, 20, "uniform")])
def test_forward_adjoint_general_n(nf, orc, prec, N, M, kind):
    """Forward and adjoint at N not a power of two against the direct sums
    (all targets / frequencies up to 2^14, else 1024 sampled)."""
    eps = 1e-12 if prec == 0 else 1e-6
    y = workloads.points(kind, M, seed=N % 1000 + M)
    c = workloads.coeffs(N, seed=3)
    gin = workloads.samples(M, seed=4)
    plan = nf.Plan(N, _dev(y), eps=eps, prec=prec)
    g = _host(plan.forward(_dev(c)))
    a = _host(plan.adjoint(_dev(gin)))
    assert g.shape == (M,) and a.shape == (N,)
    idx = workloads.sample_index(M, 1024 if M > 16384 else M, seed=5)
    kdx = workloads.sample_index(N, 1024 if N > 16384 else N, seed=6)
    assert orc.rel_l2(g[idx], orc.nudft_fwd(c, y, idx)) < TOL[prec]
    assert orc.rel_l2(a[kdx], orc.nudft_adj(gin, y, N, kdx)) < TOL[prec]


def test_one_shot_and_c64_general_n(nf, orc):
    import torch
    N, M = 5000, 7000
    y = workloads.points("uniform", M, seed=8)
    c = workloads.coeffs(N, seed=9)
    g = _host(nf.nufft_fwd(_dev(c), N, _dev(y), M, 1e-12))
    idx = workloads.sample_index(M, 512, seed=1)
    ref = orc.nudft_fwd(c, y, idx)
    assert orc.rel_l2(g[idx], ref) < 1e-12
    g32 = _host(nf.nufft_fwd(_dev(c.astype(np.complex64)), N, _dev(y), M, 1e-6, nf.MIXED, io="c64"))
    assert orc.rel_l2(g32[idx].astype(complex), orc.nudft_fwd(c.astype(np.complex64), y, idx)) < 1e-6
    a = _host(nf.nufft_adj(_dev(g.astype(complex)), _dev(y), M, N, 1e-12))
    kdx = workloads.sample_index(N, 512, seed=2)
    assert orc.rel_l2(a[kdx], orc.nudft_adj(g, y, N, kdx)) < 1e-12
    del torch


def test_batched_general_n(nf, orc):
    """Several signals sharing points, N not a power of two: each signal
    against the direct sum (the batch stride of the caller's data is N)."""
    N, M, B = 3000, 4000, 4
    y = workloads.points("uniform", M, seed=10)
    C = np.stack([workloads.coeffs(N, seed=20 + b) for b in range(B)])
    plan = nf.Plan(N, _dev(y), eps=1e-12, batch=B)
    G = _host(plan.forward(_dev(C)))
    idx = workloads.sample_index(M, 256, seed=3)
    for b in range(B):
        assert orc.rel_l2(G[b][idx], orc.nudft_fwd(C[b], y, idx)) < 1e-12
    A = _host(plan.adjoint(_dev(G)))
    kdx = workloads.sample_index(N, 256, seed=4)
    for b in range(B):
        assert orc.rel_l2(A[b][kdx], orc.nudft_adj(G[b], y, N, kdx)) < 1e-12


def test_lsq_general_n(nf, orc):
    """Least squares at N not a power of two (M = 4N, uniform): CG reaches the
    dense solve, plain and with the learned preconditioner; inufft's one-shot
    M > N form too."""
    from paper_1611_09379_gb300 import dcf
    N, M = 300, 1200
    y = workloads.points("uniform", M, seed=11)
    c_true = workloads.coeffs(N, seed=12)
    g = orc.nudft_fwd(c_true, y) + 1e-4 * workloads.samples(M, seed=13)
    cref = orc.lsq_dense(g, y, N)
    plan = nf.Plan(N, _dev(y), eps=1e-13)
    w = plan.dcf_weights(dcf.load())
    for ww in (None, w):
        c, it, res = plan.solve_lsq(_dev(g), ww, tol=1e-12, maxit=5000)
        assert orc.rel_l2(_host(c), cref) < 1e-9
    c1 = _host(nf.inufft(_dev(g), _dev(y), M, N, 1e-12))
    assert orc.rel_l2(c1, cref) < 1e-9


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("N,jit", [(1000, 0.1), (3000, 0.4), (12345, 0.1)])
def test_square_inverse_general_n(nf, orc, prec, N, jit):
    """Square inverse (M = N points, Eq. p6 / p8) for N not a power of two: the
    library evaluates the Lagrange form at the N' grid points, C(x) =
    e^{i N x / 2} prod sin((x - y_l)/2) being complex there; against the
    oracle's inverse on the N grid itself and the round trip."""
    y = workloads.points("jitter", N, N, seed=N + 7, jitter=jit)
    c = workloads.coeffs(N, seed=N + 8)
    g = orc.nudft_fwd(c, y)
    eps = 1e-12 if prec == 0 else 1e-6
    plan = nf.Plan(N, _dev(y), eps=eps, prec=prec, inverse=True)
    c2 = _host(plan.inverse(_dev(g)))
    assert c2.shape == (N,)
    cref = orc.inufft(g, y, N)
    assert orc.rel_l2(c2, cref) < TOL[prec] * (1 if jit <= 0.1 else 10)
    assert orc.rel_l2(c2, c) < (1e-11 if prec == 0 else 1e-5)
    ci = _host(nf.inufft(_dev(g), _dev(y), N, N, eps, prec))
    assert orc.rel_l2(ci, cref) < TOL[prec] * (1 if jit <= 0.1 else 10)


def test_uneven_batch_log_uniform_n(nf, orc):
    """The uneven batch with N = M drawn log-uniform in [2^10, 2^16] as real
    numbers (rounded to integers), one graph launch."""
    import torch
    rng = workloads.rng(21)
    Ns = [int(round(2.0 ** u)) for u in rng.uniform(10, 16, size=12)]
    Ns[:2] = [1024, 65536]
    ys = [_dev(workloads.points("uniform", n, seed=300 + i)) for i, n in enumerate(Ns)]
    cs_h = [workloads.coeffs(n, seed=400 + i).astype(np.complex64) for i, n in enumerate(Ns)]
    cs = [_dev(c) for c in cs_h]
    gs = [torch.empty(n, dtype=torch.complex64, device="cuda") for n in Ns]
    multi = nf.Multi(Ns, ys, eps=1e-6, prec=nf.MIXED, io="c64")
    multi.forward(cs, gs)
    for i, n in enumerate(Ns):
        idx = workloads.sample_index(n, 128, seed=i)
        ref = orc.nudft_fwd(cs_h[i].astype(complex), ys[i].cpu().numpy(), idx)
        assert orc.rel_l2(gs[i].cpu().numpy()[idx], ref) < 1e-6, (i, n)
