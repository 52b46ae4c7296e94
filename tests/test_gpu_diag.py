"""The near-field pair reciprocal and the pipe rates behind the target
kernels' roofline, through the C ABI.

The pair loops (the singular part 2/t of Eq. p20 over a leaf and its two
neighbours) take one reciprocal per pair, |t| >= 1/2 in grid units (a
point's nearest grid point is handled in closed form).  The FP64 path uses
the hardware estimate refined by two Newton-Raphson steps r <- r + r (1 - t r)
(the textbook iteration for 1/t, quadratic convergence), the mixed path the
FP32 special-function reciprocal; both are checked against correctly rounded
IEEE division over the whole range the kernels meet and beyond."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_1611_09379_gb300 as nf
    return nf


def _ulps(x, ref):
    return np.abs(x - ref) / np.spacing(np.abs(ref))


def test_pair_reciprocal_error_bounds(nf):
    import torch
    rng = np.random.default_rng(0)
    mag = np.concatenate([
        np.exp(rng.uniform(np.log(0.5), np.log(2.0 ** 27), 200000)),  # log-uniform range
        0.5 + np.arange(64) * np.spacing(0.5),                         # the smallest |t|
        np.nextafter(2.0 ** np.arange(-1, 27), 0), 2.0 ** np.arange(-1, 27),
        np.arange(1, 4097) + 0.5, np.arange(1, 4097) - 0.5 + 1e-9,    # half-integer offsets
    ])
    t = np.concatenate([mag, -mag])
    r64, r32 = nf.diag_rcp(torch.from_numpy(t).cuda())
    torch.cuda.synchronize()
    r64, r32 = r64.cpu().numpy(), r32.cpu().numpy()
    ref64 = 1.0 / t
    assert _ulps(r64, ref64).max() <= 1.0  # measured: the refined estimate is within 1 ulp
    t32 = t.astype(np.float32)
    ref32 = (np.float32(1.0) / t32).astype(np.float32)
    # in units of the FP32 spacing of the correctly rounded quotient
    err32 = np.abs(r32.astype(np.float64) - ref32.astype(np.float64))
    assert (err32 / np.spacing(np.abs(ref32)).astype(np.float64)).max() <= 1.0
    assert np.all(np.isfinite(r64)) and np.all(np.isfinite(r32))


def test_pipe_rates_are_plausible(nf):
    """Reciprocals and FMAs per SM per clock: the special-function unit's FP32
    reciprocal is a fraction of the FMA rate (16 vs 128 lanes on this
    architecture); the measurement lands near those counts."""
    rcp, ffma = nf.pipe_rates()
    assert 8.0 <= rcp <= 40.0, rcp
    assert 64.0 <= ffma <= 260.0, ffma
    assert ffma > 3 * rcp
