"""The paper's U-Net variant (network kind 1; Sec. 3.1, Tab. 2) on the GPU against the oracle's
plain strided / transposed convolutions (oracle/unet_paper.py).

The CUDA path computes every 8x8 stride-2 layer as a 5x5 convolution of space-to-depth rearranged
data (tcgen05 in BF16, CUDA cores in FP64) and every transposed layer as a 5x5 convolution written
depth-to-space; the oracle uses the definitions.  FP64: 1e-12 of the column maximum.  BF16 against
the oracle's BF16 emulation: 2e-2 normwise per column (FP32 summation order flips BF16 roundings,
which the nonlinear network propagates)."""
import numpy as np
import pytest
import torch

from oracle import fgmres as fg
from oracle import helmholtz as hz
from oracle import unet_paper as up
from paper_2607_16906_b300 import synth

from .gpu_util import make_ctx, random_batch, small_problems, split, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def helm():
    from paper_2607_16906_b300 import helm as h
    return h


@pytest.fixture(scope="module")
def theta(helm):
    return synth.kaiming_uniform_params(helm.paper_weight_segments(), 42)


def _oracle(theta, probs, vs, bf16):
    out = []
    for p, v in zip(probs, vs):
        out.append(up.precondition(theta, v, p.c, p.p, p.h, p.omega, bf16=bf16))
    return out


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_paper_network_matches_oracle(helm, theta, dtype):
    probs = small_problems(((20, 14, 5), (40, 40, 12), (50, 30, 7)), seed=91)
    ctx = make_ctx(probs)
    net = helm.UNet(theta, kind=1)
    nrhs = 2
    per, flat = random_batch(probs, nrhs, 92, np.complex64 if dtype == torch.complex64 else np.complex128)
    v = to_dev(flat, dtype)
    z = torch.empty_like(v)
    helm.helm_precond_apply(ctx, net, v, z, nrhs)
    got = split(z.cpu().numpy().astype(np.complex128), probs, nrhs)
    vin = [a.astype(np.complex128) for a in per]
    if dtype == torch.complex128:
        ref = _oracle(theta, probs, vin, bf16=False)
        for g, r in zip(got, ref):
            assert np.abs(g - r).max() <= 1e-12 * np.abs(r).max()
    else:
        ref = _oracle(theta, probs, vin, bf16=True)
        for g, r in zip(got, ref):
            for k in range(nrhs):
                e = np.linalg.norm(g[k] - r[k]) / np.linalg.norm(r[k])
                assert e <= 2e-2, e


def test_paper_network_in_fgmres_matches_oracle_cycle(helm, theta):
    """One FP64 FGMRES(8) cycle preconditioned by the paper's variant equals the oracle's cycle."""
    probs = small_problems(((20, 14, 5),), seed=93)
    p = probs[0]
    ctx = make_ctx(probs)
    net = helm.UNet(theta, kind=1)
    b = to_dev(p.b.ravel(), torch.complex128)
    x = torch.zeros_like(b)
    helm.helm_fgmres_solve(ctx, net, b, x, 1, m=8, tol=1e-300, mixed=False, max_restarts=1, orth="dcgs2")
    A = hz.assemble(p.c, p.p, p.h, p.omega)
    pre = lambda v: up.precondition(theta, v.reshape(1, p.Ny, p.Nx), p.c, p.p, p.h, p.omega)[0].ravel()
    res = fg.cycle(lambda u: A @ u, pre, p.b[0].ravel(), 8, 0.0, orth="dcgs2")
    assert np.linalg.norm(x.cpu().numpy() - res.x) <= 1e-9 * np.linalg.norm(res.x)


def test_paper_network_mixed_solve_reaches_the_direct_solution(helm, theta):
    probs = small_problems(((40, 40, 12), (33, 27, 6)), seed=94, nrhs=2)
    ctx = make_ctx(probs)
    net = helm.UNet(theta, kind=1)
    b = to_dev(np.concatenate([p.b.ravel() for p in probs]), torch.complex128)
    x = torch.zeros_like(b)
    rc, info = helm.helm_fgmres_solve(ctx, net, b, x, 2, m=60, tol=1e-6, mixed=True, max_outer=40, inner_tol=1e-5,
                                      orth="dcgs2")
    assert rc == helm.HELM_OK, info
    for p, xs in zip(probs, split(x.cpu().numpy(), probs, 2)):
        A = hz.assemble(p.c, p.p, p.h, p.omega)
        for r in range(2):
            xd = hz.solve_direct(A, p.b[r].ravel())
            assert hz.relres(A, xs[r].ravel(), p.b[r].ravel()) <= 1e-6
            assert np.linalg.norm(xs[r].ravel() - xd) <= 1e-5 * np.linalg.norm(xd)


def test_paper_network_training_is_refused(helm, theta):
    probs = small_problems(((20, 14, 5),), seed=95)
    ctx = make_ctx(probs)
    net = helm.UNet(theta, kind=1)
    b = to_dev(probs[0].b.ravel(), torch.complex64)
    with pytest.raises(helm.HelmError, match="not built"):
        helm.helm_train_step(ctx, net, b)
