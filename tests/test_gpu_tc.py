"""The tcgen05 implicit-GEMM convolutions against the CUDA-core kernels of the same BF16 network.

Both paths take BF16 activations and weights and accumulate in FP32; only the summation order
differs, which can flip the BF16 rounding of an activation by one ulp (2^-8 relative) and then
propagate, so outputs agree to about 1e-2 normwise.  The CUDA-core path is selected in a child
process with HELM_DISABLE_TC=1 (the library reads it once when a network is created).
"""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

CHILD = r"""
import sys, numpy as np, torch
sys.path.insert(0, {root!r})
from paper_2607_16906_b300 import helm, synth
rng = synth.rng_for(91)
sizes = ((40, 28, 12), (150, 150, 13))          # ragged tiles at every level, one grid not a multiple of 16
out = []
for nx, ny, p in sizes:
    c = synth.skull_velocity(nx, ny, p, rng)
    spec = helm.SystemSpec(nx, ny, synth.grid_spacing(10.0), p, synth.angular_frequency())
    ctx = helm.Context([spec], torch.tensor(c.ravel(), device="cuda"))
    net = helm.UNet(synth.kaiming_uniform_params(helm.weight_segments(), 42))
    v = (rng.standard_normal(3 * spec.n) + 1j * rng.standard_normal(3 * spec.n)).astype(np.complex64)
    vd = torch.tensor(v, device="cuda"); zd = torch.empty_like(vd)
    helm.helm_precond_apply(ctx, net, vd, zd, 3)
    out.append(zd.cpu().numpy())
np.save({path!r}, np.concatenate(out))
"""


def _run(path, disable, disable_row=False):
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, HELM_DISABLE_TC="1" if disable else "0", HELM_DISABLE_ROW="1" if disable_row else "0")
    r = subprocess.run([sys.executable, "-c", CHILD.format(root=root, path=path)], env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return np.load(path)


def test_tcgen05_convs_match_cuda_core_convs(tmp_path):
    """Default tcgen05 path (row-tile kernels for the narrow layers, 9-box kernels for the rest), the
    9-box kernels alone, and the CUDA-core kernels agree pairwise."""
    tc = _run(str(tmp_path / "tc.npy"), disable=False)
    box = _run(str(tmp_path / "box.npy"), disable=False, disable_row=True)
    cc = _run(str(tmp_path / "cc.npy"), disable=True)
    assert np.isfinite(tc).all() and np.isfinite(box).all()
    n1 = 3 * (40 + 24) * (28 + 24)
    for seg in (slice(0, n1), slice(n1, None)):
        for a, b in ((tc, cc), (box, cc), (tc, box)):
            e = np.linalg.norm(a[seg] - b[seg]) / np.linalg.norm(b[seg])
            assert e <= 1.5e-2, e
