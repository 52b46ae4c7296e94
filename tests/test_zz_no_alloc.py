"""The no-allocation forward transform (nufft_fwd_noalloc) against the
ordinary one (nufft_fwd) through the C ABI.

Callers that cannot allocate device memory (a pool allocator or a fixed
memory budget owns it, or a latency-critical loop cannot afford the device
synchronisation of cudaMalloc) use nufft_fwd_noalloc, whose work buffers live
in a fixed array inside the library.  Its results must equal those of
nufft_fwd within the parity tolerances (1e-12 FP64, 1e-6 mixed), on calls in
a row that reuse the shared array with different sizes and points.  This
file is collected last so a stop-at-first-failure run has run every other
test before it.
"""
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


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_noalloc_matches_allocating_entry_point(nf):
    import torch
    cases = [  # (N, M, kind, prec, eps, seed)
        (4096, 3000, "uniform", nf.FP64, 1e-12, 1),
        (1 << 16, 1 << 16, "clustered", nf.MIXED, 1e-6, 2),
        (4096, 3000, "uniform", nf.FP64, 1e-12, 3),
        (1 << 16, 1 << 15, "uniform", nf.FP64, 1e-12, 4),
        # few points against the largest grid (leaves of at most 64 grid points)
        (1 << 16, 1000, "uniform", nf.FP64, 1e-12, 5),
        (1 << 16, 1, "uniform", nf.MIXED, 1e-6, 6),
        # the largest orders at the largest sizes (the most scratch)
        (1 << 16, 1 << 16, "uniform", nf.FP64, 1e-15, 7),
        (1 << 16, 1 << 16, "clustered", nf.FP64, 1e-12, 8),
    ]
    tol = {nf.FP64: 1e-12, nf.MIXED: 1e-6}
    for N, M, kind, prec, eps, seed in cases:
        y = torch.from_numpy(workloads.points(kind, M, seed=seed)).cuda()
        c = torch.from_numpy(workloads.coeffs(N, seed=seed + 10)).cuda()
        ref = nf.nufft_fwd(c, N, y, M, eps, prec)
        out = torch.empty(M, dtype=torch.complex128, device="cuda")
        g = nf.nufft_fwd_noalloc(c, N, y, M, eps, prec, out=out)
        torch.cuda.synchronize()
        assert g.data_ptr() == out.data_ptr()
        assert _rel(g.cpu().numpy(), ref.cpu().numpy()) < tol[prec], (N, M, kind, prec)
        # a second call in a row on the same inputs reuses the shared array
        g2 = nf.nufft_fwd_noalloc(c, N, y, M, eps, prec, out=torch.empty_like(out))
        torch.cuda.synchronize()
        assert _rel(g2.cpu().numpy(), ref.cpu().numpy()) < tol[prec], (N, M, kind, prec)


def test_noalloc_rejects_sizes_beyond_its_scratch(nf):
    import torch
    N = 1 << 17
    y = torch.zeros(8, dtype=torch.float64, device="cuda")
    c = torch.zeros(N, dtype=torch.complex128, device="cuda")
    with pytest.raises(nf.NufftError) as e:
        nf.nufft_fwd_noalloc(c, N, y, 8, 1e-6)
    assert e.value.code == nf.EINVAL
