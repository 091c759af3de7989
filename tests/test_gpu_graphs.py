"""The BF16 network application replayed from captured CUDA graphs gives the eager result bit for
bit, for every system of an uneven batch, and reports the same kernel count; the row-conv tile
heights the autotuner picks do not change a bit of it either."""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

from paper_2607_16906_b300 import synth

from .gpu_util import make_ctx, random_batch, small_problems, to_dev

pytestmark = pytest.mark.gpu

CHILD = r"""
import sys, numpy as np, torch
sys.path.insert(0, {root!r})
from paper_2607_16906_b300 import helm, synth
from tests.gpu_util import make_ctx, random_batch, small_problems, to_dev
probs = small_problems(((40, 28, 12), (150, 150, 13), (64, 64, 8)), seed=5)
ctx = make_ctx(probs)
net = helm.UNet(synth.kaiming_uniform_params(helm.weight_segments(), 42))
_, flat = random_batch(probs, 2, 9, np.complex64)
v = to_dev(flat, torch.complex64)
z = torch.empty_like(v)
for _ in range(3):
    helm.helm_precond_apply(ctx, net, v, z, 2)
np.save({path!r}, z.cpu().numpy())
"""


@pytest.fixture(scope="module")
def helm():
    from paper_2607_16906_b300 import helm as h
    return h


def test_graph_replay_matches_eager_bitwise(helm, tmp_path):
    probs = small_problems(((40, 28, 12), (150, 150, 13), (64, 64, 8)), seed=5)
    ctx = make_ctx(probs)
    net = helm.UNet(synth.kaiming_uniform_params(helm.weight_segments(), 42))
    _, flat = random_batch(probs, 2, 9, np.complex64)
    v = to_dev(flat, torch.complex64)
    outs, counts = [], []
    for _ in range(4):  # eager, capture + replay, replay, replay
        z = torch.zeros_like(v)
        l0 = helm.helm_launch_count()
        helm.helm_precond_apply(ctx, net, v, z, 2)
        torch.cuda.synchronize()
        counts.append(helm.helm_launch_count() - l0)
        outs.append(z.cpu().numpy())
    assert np.isfinite(outs[0]).all() and np.abs(outs[0]).max() > 0
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
    # the first call also times the row-conv tile candidates of each new layer shape
    assert counts[0] >= counts[1] == counts[2] == counts[3], counts
    # the same inputs in processes with graphs switched off, and with graphs and the tile autotuner
    # both off (every row-conv layer at its first tile height): the same bits
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    for name, extra in (("eager", {"HELM_DISABLE_GRAPHS": "1"}),
                        ("untuned", {"HELM_DISABLE_GRAPHS": "1", "HELM_AUTOTUNE": "0"})):
        path = str(tmp_path / f"{name}.npy")
        env = dict(os.environ, **extra)
        r = subprocess.run([sys.executable, "-c", CHILD.format(root=root, path=path)], env=env, capture_output=True,
                           text=True, timeout=600, cwd=root)
        assert r.returncode == 0, r.stderr[-2000:]
        assert np.array_equal(np.load(path), outs[0]), name
    assert len(helm.helm_tuned_tiles()) > 0


def test_graph_follows_moving_slots(helm):
    """Replays read the input and output pointers of each call: applying the network to two
    different vectors in alternation gives each its own eager result."""
    probs = small_problems(((48, 40, 8),), seed=6)
    ctx = make_ctx(probs)
    net = helm.UNet(synth.kaiming_uniform_params(helm.weight_segments(), 42))
    _, fa = random_batch(probs, 1, 10, np.complex64)
    _, fb = random_batch(probs, 1, 11, np.complex64)
    va, vb = to_dev(fa, torch.complex64), to_dev(fb, torch.complex64)
    za, zb = torch.empty_like(va), torch.empty_like(vb)
    helm.helm_precond_apply(ctx, net, va, za, 1)  # eager
    ref_a = za.cpu().numpy()
    helm.helm_precond_apply(ctx, net, vb, zb, 1)  # capture + replay
    ref_b = zb.cpu().numpy()
    for _ in range(2):
        za2, zb2 = torch.zeros_like(va), torch.zeros_like(vb)
        helm.helm_precond_apply(ctx, net, va, za2, 1)
        helm.helm_precond_apply(ctx, net, vb, zb2, 1)
        assert np.array_equal(za2.cpu().numpy(), ref_a)
        assert np.array_equal(zb2.cpu().numpy(), ref_b)
    assert not np.array_equal(ref_a, ref_b)
