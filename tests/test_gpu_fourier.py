"""The Fourier-differentiation operator (helm_apply_fourier; Sec. 2.1, Tab. 1) against the oracle's
numpy-FFT operator on an uneven batch of power-of-two grids, in FP64 (1e-12 of the column maximum)
and FP32 (1e-5: a few units of FP32 rounding times the log2(N) depth of four transforms)."""
import numpy as np
import pytest
import torch

from oracle import fourier as fo
from paper_2607_16906_b300 import synth

from .gpu_util import make_ctx, random_batch, split, to_dev

pytestmark = pytest.mark.gpu

# (nx, ny, p): Nx, Ny powers of two with the PML; the paper's own grid is 64 x 64 (Tab. 1)
SIZES = ((56, 56, 4), (112, 48, 8), (16, 240, 8), (1008, 496, 8))


@pytest.fixture(scope="module")
def helm():
    from paper_2607_16906_b300 import helm as h
    return h


def _probs():
    rng = synth.rng_for(81)
    out = []
    for nx, ny, p in SIZES:
        c = synth.skull_velocity(nx, ny, p, rng, thickness=(2, 4))
        out.append(synth.Problem(nx, ny, p, synth.grid_spacing(10.0), synth.angular_frequency(), c,
                                 np.zeros((1, ny + 2 * p, nx + 2 * p), complex)))
    return out


@pytest.mark.parametrize("dtype,tol", [(torch.complex128, 1e-12), (torch.complex64, 1e-5)])
def test_fourier_operator_matches_oracle(helm, dtype, tol):
    probs = _probs()
    ctx = make_ctx(probs)
    nrhs = 2
    per, flat = random_batch(probs, nrhs, 82)
    x = to_dev(flat, dtype)
    y = torch.full_like(x, float("nan"))
    helm.helm_apply_fourier(ctx, x, y, nrhs)
    got = split(y.cpu().numpy().astype(np.complex128), probs, nrhs)
    xin = split(x.cpu().numpy().astype(np.complex128), probs, nrhs)
    for p, g, u in zip(probs, got, xin):
        for r in range(nrhs):
            ref = fo.apply(u[r], p.c, p.p, p.h, p.omega)
            assert np.abs(g[r] - ref).max() <= tol * np.abs(ref).max(), (p.Nx, p.Ny, r)


def test_fourier_operator_rejects_other_sizes(helm):
    probs = [synth.Problem(20, 20, 4, synth.grid_spacing(10.0), synth.angular_frequency(),
                           np.full((28, 28), 1500.0), np.zeros((1, 28, 28), complex))]
    ctx = make_ctx(probs)
    x = torch.zeros(ctx.npts, dtype=torch.complex128, device="cuda")
    with pytest.raises(helm.HelmError, match="powers of two"):
        helm.helm_apply_fourier(ctx, x, torch.zeros_like(x))
