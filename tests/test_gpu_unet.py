"""Parity of the CUDA U-Net preconditioner z = N(alpha v)/alpha (eq. 6) against the oracle (a3).

FP64 path: within 1e-12 of the oracle's FP64 network (max-normalised, per column).
BF16 path: against the oracle's BF16 emulation (conv inputs and weights rounded to bfloat16, wide
accumulation); FP32 accumulation order can flip the rounding of an activation by one bf16 ulp
(2^-8 relative), which then propagates, so the bound is normwise 1e-2 per column.
"""
import numpy as np
import pytest
import torch

from oracle import unet
from paper_2607_16906_b300 import synth

from .gpu_util import make_ctx, random_batch, small_problems, split, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def helm():
    from paper_2607_16906_b300 import helm as h
    return h


@pytest.fixture(scope="module")
def theta():
    return synth.kaiming_uniform_params(unet.param_segments(), 42)


def _oracle_pre(problems, per, theta, bf16):
    return [unet.precondition(theta, a, p.c, p.h, bf16=bf16) for p, a in zip(problems, per)]


def test_fp64_network_matches_oracle(helm, theta):
    probs = small_problems(((20, 14, 5), (13, 9, 3)))     # padded grids 32x24 and 16x24
    nrhs = 2
    ctx = make_ctx(probs)
    net = helm.UNet(theta)
    per, flat = random_batch(probs, nrhs, 21)
    v = to_dev(flat, torch.complex128)
    z = torch.empty_like(v)
    helm.helm_precond_apply(ctx, net, v, z, nrhs)
    got = split(z.cpu().numpy(), probs, nrhs)
    ref = _oracle_pre(probs, per, theta, bf16=False)
    for g, r in zip(got, ref):
        for k in range(nrhs):
            assert np.abs(g[k] - r[k]).max() <= 1e-12 * np.abs(r[k]).max()


def test_bf16_network_matches_oracle_emulation(helm, theta):
    probs = small_problems(((40, 40, 12), (20, 14, 5)))
    nrhs = 3
    ctx = make_ctx(probs)
    net = helm.UNet(theta)
    per, flat = random_batch(probs, nrhs, 22, np.complex64)
    v = to_dev(flat, torch.complex64)
    z = torch.empty_like(v)
    helm.helm_precond_apply(ctx, net, v, z, nrhs)
    got = split(z.cpu().numpy().astype(np.complex128), probs, nrhs)
    ref = _oracle_pre(probs, [a.astype(np.complex128) for a in per], theta, bf16=True)
    ref64 = _oracle_pre(probs, [a.astype(np.complex128) for a in per], theta, bf16=False)
    for g, r, r64 in zip(got, ref, ref64):
        for k in range(nrhs):
            e = np.linalg.norm(g[k] - r[k]) / np.linalg.norm(r[k])
            assert e <= 1e-2, e
            # and the BF16 network stays close to the FP64 network
            assert np.linalg.norm(g[k] - r64[k]) / np.linalg.norm(r64[k]) <= 5e-2


def test_bf16_network_full_size_sampled_column(helm, theta):
    """Fine-grid workload (576^2, 32 RHS) in one launch; column 5 checked against the oracle in full."""
    prob = synth.fine_multi_rhs_problem()
    ctx = make_ctx([prob])
    nrhs = 32
    rng = synth.rng_for(23)
    vs = (rng.standard_normal((nrhs, prob.Ny, prob.Nx)) + 1j * rng.standard_normal((nrhs, prob.Ny, prob.Nx)))
    vs = vs.astype(np.complex64)
    v = to_dev(vs.ravel(), torch.complex64)
    z = torch.empty_like(v)
    helm.helm_precond_apply(ctx, net := helm.UNet(theta), v, z, nrhs)
    g = z.cpu().numpy().reshape(nrhs, prob.Ny, prob.Nx)
    assert np.isfinite(g).all()
    k = 5
    r = unet.precondition(theta, vs[k:k + 1].astype(np.complex128), prob.c, prob.h, bf16=True)[0]
    assert np.linalg.norm(g[k] - r) / np.linalg.norm(r) <= 1e-2
    del net


def test_zero_input_column_gives_zero(helm, theta):
    probs = small_problems(((20, 14, 5),))
    ctx = make_ctx(probs)
    net = helm.UNet(theta)
    v = ctx.new_vector(2, torch.complex64)
    v[: probs[0].n] = 1.0 + 0.5j
    z = torch.empty_like(v)
    helm.helm_precond_apply(ctx, net, v, z, 2)
    zz = z.cpu().numpy()
    assert np.all(zz[probs[0].n:] == 0)
    assert np.isfinite(zz).all()


def test_weights_round_trip(helm, theta):
    net = helm.UNet(theta)
    assert np.array_equal(net.weights(), theta)
    with pytest.raises(helm.HelmError):
        helm.UNet(theta[:-1])
