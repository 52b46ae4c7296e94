"""The c_n <-> f_k step (Eq. p1 on the uniform grid) through the library's
transforms, against the oracle's radix-2 FFT.  With every y_j on a grid
point x_k (M = N, y_j = x_j) the forward transform returns the grid samples
f_k = sum_n c_n e^{i n x_k} (its E_j f_k0 term; F_j vanishes to rounding)
and the adjoint returns c'_n = sum_k e^{-i n x_k} g_k, so both are the FFT
pass kernels alone: the Stockham passes of every radix and, where their grid
fills the GPU (N >= 2^20 for one signal), the one-warp-per-column radix-1024
passes (FP32), both signs, with the FP32 and complex128 loads and stores at
the ends."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

# relative L2 bounds: FP64 against the direct sums, FP32 (mixed) the FFT step alone
TOL = {0: 1e-12, 1: 5e-7}


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


def _grid_points(N):
    return 2.0 * np.pi * np.arange(N, dtype=np.float64) / N


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("L", [12, 16, 19, 20, 21])
def test_grid_points_forward_and_adjoint_are_the_fft(nf, orc, prec, L):
    N = 1 << L
    y = _grid_points(N)
    plan = nf.Plan(N, _dev(y), eps=1e-12 if prec == 0 else 1e-6, prec=prec)
    c = workloads.coeffs(N, seed=100 + L)
    g = _host(plan.forward(_dev(c)))
    a = _host(plan.adjoint(_dev(c)))
    # fl(2 pi j / N) lies up to j 2^-53 grid units off x_j, which moves the
    # exact sums by about 1e-9 of their norm at N = 2^21: the FP64 path is
    # held to the direct sums at the points themselves (sampled), the FFT to
    # that offset's bound
    if prec == 0:
        idx = workloads.sample_index(N, 512, seed=L)
        assert orc.rel_l2(g[idx], orc.nudft_fwd(c, y, idx)) < TOL[0]
        assert orc.rel_l2(a[idx], orc.nudft_adj(c, y, N, idx)) < TOL[0]
    tol = TOL[1] if prec == 1 else 4e-9
    assert orc.rel_l2(g, orc.fft(c, +1)) < tol
    assert orc.rel_l2(a, orc.fft(c, -1)) < tol


@pytest.mark.parametrize("L", [22, 24])
def test_grid_points_three_passes_mixed(nf, orc, L):
    """N = 2^22 and 2^24 (mixed): two radix-1024 passes and a radix-4 / radix-16
    pass."""
    N = 1 << L
    y = _grid_points(N)
    plan = nf.Plan(N, _dev(y), eps=1e-6, prec=1)
    c = workloads.coeffs(N, seed=100 + L)
    g = _host(plan.forward(_dev(c)))
    assert orc.rel_l2(g, orc.fft(c, +1)) < TOL[1]
    a = _host(plan.adjoint(_dev(c)))
    assert orc.rel_l2(a, orc.fft(c, -1)) < TOL[1]


def test_grid_points_batched_signals(nf, orc):
    """Several signals in one plan (grid.y of the pass kernels) at N = 2^20,
    mixed: each equals its own FFT."""
    N, batch = 1 << 20, 3
    y = _grid_points(N)
    plan = nf.Plan(N, _dev(y), eps=1e-6, prec=1, batch=batch)
    c = np.stack([workloads.coeffs(N, seed=200 + b) for b in range(batch)])
    g = _host(plan.forward(_dev(c)))
    for b in range(batch):
        assert orc.rel_l2(g[b], orc.fft(c[b], +1)) < TOL[1]


def test_radix1024_passes_match_stockham_passes(nf, orc):
    """NUFFT_FFT_NO_W32=1 keeps every pass on the Stockham kernel and
    NUFFT_FFT_W32_COLS fixes the radix-1024 pass's columns per CTA (4, 8,
    16): child processes with each give the same forward at N = 2^20 (mixed)
    to FP32 rounding, on jittered points, and each matches the direct sums."""
    import os
    import subprocess
    import sys
    code = (
        "import numpy as np, torch, sys, workloads;"
        "import paper_1611_09379_gb300 as nf;"
        "N = 1 << 20; y = workloads.points('jitter', N, N, seed=31, jitter=0.4);"
        "p = nf.Plan(N, torch.from_numpy(y).cuda(), eps=1e-6, prec=1);"
        "c = torch.from_numpy(workloads.coeffs(N, seed=32)).cuda();"
        "np.save(sys.argv[1], p.forward(c).cpu().numpy())")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    outs = []
    for flag, cols in (("0", ""), ("1", ""), ("0", "4"), ("0", "16")):
        path = os.path.join(root, "gpurun_out", f"_w32_{flag}_{cols}.npy")
        os.makedirs(os.path.dirname(path), exist_ok=True)
        env = dict(os.environ, NUFFT_FFT_NO_W32=flag, NUFFT_FFT_W32_COLS=cols)
        subprocess.run([sys.executable, "-c", code, path], cwd=root, env=env, check=True,
                       timeout=300)
        outs.append(np.load(path))
        os.remove(path)
    for o in outs[1:]:
        assert orc.rel_l2(outs[0], o) < 3e-7
    idx = workloads.sample_index(1 << 20, 256, seed=5)
    y = workloads.points("jitter", 1 << 20, 1 << 20, seed=31, jitter=0.4)
    ref = orc.nudft_fwd(workloads.coeffs(1 << 20, seed=32), y, idx)
    for o in outs:
        assert orc.rel_l2(o[idx], ref) < 1e-6
