"""The kernels of a transform are launched with programmatic dependent launch
(each waits for its predecessor with griddepcontrol.wait before it touches
data the predecessor wrote).  Results equal, bit for bit, those of a process
that launches every kernel with full stream serialization (NUFFT_NO_PDL set),
for the forward, adjoint and inverse, both precisions, one signal and a batch
of four, with and without graph replay.  Likewise the upward pass in one
launch (the last CTA of each group carries on, counted by atomics) against
one launch per band of levels (NUFFT_NO_FUSED_UP set): same sums in the same
order, so the same bits; a lost count or an unpublished write would show."""
import os
import subprocess
import sys

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# Computes every case and saves the outputs to the .npz named on the command line.
_SCRIPT = r"""
import sys
import numpy as np
import torch
sys.path.insert(0, ROOT)
sys.path.insert(0, ROOT + "/tests")
import paper_1611_09379_gb300 as nf
import workloads
out = {}
for prec, eps, N in ((nf.FP64, 1e-12, 1 << 15), (nf.MIXED, 1e-6, 1 << 15), (nf.MIXED, 1e-6, 1 << 19)):
    M = N
    y = workloads.points("jitter", M, N, seed=81, jitter=0.3)
    for batch in (1, 4):
        C = np.stack([workloads.coeffs(N, seed=82 + b) for b in range(batch)])
        cin = torch.from_numpy(C if batch > 1 else C[0]).cuda()
        for graphs in (True, False):
            with nf.Plan(N, torch.from_numpy(y).cuda(), eps=eps, prec=prec, inverse=True,
                         batch=batch, graphs=graphs) as plan:
                g = plan.forward(cin)
                a = plan.adjoint(g)
                ci = plan.inverse(g)
                torch.cuda.synchronize()
                key = f"{prec}_{N}_{batch}_{int(graphs)}"
                out[key + "_g"] = g.cpu().numpy()
                out[key + "_a"] = a.cpu().numpy()
                out[key + "_i"] = ci.cpu().numpy()
np.savez(sys.argv[1], **out)
""".replace("ROOT", repr(ROOT))


def _run(path, no_pdl=False, no_fused_up=False):
    env = dict(os.environ)
    env.pop("NUFFT_NO_PDL", None)
    env.pop("NUFFT_NO_FUSED_UP", None)
    if no_pdl:
        env["NUFFT_NO_PDL"] = "1"
    if no_fused_up:
        env["NUFFT_NO_FUSED_UP"] = "1"
    r = subprocess.run([sys.executable, "-c", _SCRIPT, str(path)], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return np.load(path)


@pytest.fixture(scope="module")
def default_run(tmp_path_factory):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    return _run(tmp_path_factory.mktemp("pdl") / "default.npz")


def _same(a, b):
    assert sorted(a.files) == sorted(b.files) and len(a.files) == 36
    for k in a.files:
        assert np.array_equal(a[k], b[k]), k
        assert np.all(np.isfinite(a[k])), k


def test_pdl_matches_serialized_launches(default_run, tmp_path):
    _same(default_run, _run(tmp_path / "serial.npz", no_pdl=True))


def test_one_launch_upward_pass_matches_banded_launches(default_run, tmp_path):
    _same(default_run, _run(tmp_path / "banded.npz", no_fused_up=True))
