"""Parity of the CUDA stencil, its adjoint and the FP64 residual against the oracle (a2, a8)."""
import numpy as np
import pytest
import torch

from oracle import helmholtz as hz
from paper_2607_16906_b300 import synth

from .gpu_util import make_ctx, random_batch, small_problems, split, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def helm():
    from paper_2607_16906_b300 import helm as h
    return h


def _oracle_apply(problems, per, adjoint=False):
    f = hz.apply_adjoint if adjoint else hz.apply
    return [np.stack([f(a[r], p.c, p.p, p.h, p.omega) for r in range(a.shape[0])]) for p, a in zip(problems, per)]


@pytest.mark.parametrize("adjoint", [False, True])
def test_fp64_stencil_matches_oracle(helm, adjoint):
    """FP64 stencil within 1e-12 (relative to the column's max) of the oracle, uneven batch, 3 RHS."""
    probs = small_problems(((20, 14, 5), (13, 9, 3), (1, 1, 0), (8, 1, 2)))
    nrhs = 3
    ctx = make_ctx(probs)
    per, flat = random_batch(probs, nrhs, 5)
    x = to_dev(flat, torch.complex128)
    y = torch.empty_like(x)
    helm.helm_apply(ctx, x, y, nrhs, adjoint=adjoint)
    got = split(y.cpu().numpy(), probs, nrhs)
    ref = _oracle_apply(probs, per, adjoint)
    for g, r in zip(got, ref):
        for k in range(nrhs):
            assert np.abs(g[k] - r[k]).max() <= 1e-12 * np.abs(r[k]).max()


def test_fp32_stencil_matches_oracle(helm):
    probs = small_problems()
    nrhs = 2
    ctx = make_ctx(probs)
    per, flat = random_batch(probs, nrhs, 6, np.complex64)
    x = to_dev(flat, torch.complex64)
    y = torch.empty_like(x)
    helm.helm_apply(ctx, x, y, nrhs)
    got = split(y.cpu().numpy().astype(np.complex128), probs, nrhs)
    ref = _oracle_apply(probs, [a.astype(np.complex128) for a in per])
    for g, r in zip(got, ref):
        for k in range(nrhs):
            # FP32 arithmetic on O(1/h^2) coefficients: a few ulps of the largest term
            assert np.abs(g[k] - r[k]).max() <= 2e-6 * np.abs(r[k]).max()


@pytest.mark.parametrize("variant", [1, 2, 3, 4])
@pytest.mark.parametrize("adjoint", [False, True])
def test_fp32_stencil_segments_and_fallback(helm, adjoint, variant):
    """FP32 stencil and adjoint: even-width systems take the TMA-tiled kernel (ragged last tile in x
    and y, a width of exactly one tile, zero-filled halo at every edge), with the k^2 tile staged by
    TMA (widths 64 and 100 at 16-byte aligned offsets) or read from global memory (width 114, 30);
    the odd-width system takes the one-point-per-thread kernel.  Every tile candidate of the
    autotuner (16, 32 or 64 rows, 2-4 stages) is run."""
    probs = small_problems(((60, 5, 2), (80, 30, 10), (100, 37, 7), (20, 14, 5), (13, 9, 3)), seed=23)
    nrhs = 3
    ctx = make_ctx(probs)
    per, flat = random_batch(probs, nrhs, 31, np.complex64)
    x = to_dev(flat, torch.complex64)
    y = torch.empty_like(x)
    helm.helm_set_stencil_variant(variant)
    try:
        helm.helm_apply(ctx, x, y, nrhs, adjoint=adjoint)
    finally:
        helm.helm_set_stencil_variant(0)
    got = split(y.cpu().numpy().astype(np.complex128), probs, nrhs)
    ref = _oracle_apply(probs, [a.astype(np.complex128) for a in per], adjoint)
    for g, r in zip(got, ref):
        for k in range(nrhs):
            assert np.abs(g[k] - r[k]).max() <= 2e-6 * np.abs(r[k]).max()


def test_adjoint_dot_product_on_gpu(helm):
    probs = small_problems()
    ctx = make_ctx(probs)
    _, fx = random_batch(probs, 1, 7)
    _, fy = random_batch(probs, 1, 8)
    x, y = to_dev(fx, torch.complex128), to_dev(fy, torch.complex128)
    Ax, AHy = torch.empty_like(x), torch.empty_like(y)
    helm.helm_apply(ctx, x, Ax)
    helm.helm_apply_adjoint(ctx, y, AHy)
    o = 0
    for p in probs:
        sl = slice(o, o + p.n)
        lhs = torch.vdot(y[sl], Ax[sl]).item()
        rhs = torch.vdot(AHy[sl], x[sl]).item()
        assert abs(lhs - rhs) <= 1e-13 * torch.linalg.norm(Ax[sl]).item() * torch.linalg.norm(y[sl]).item()
        o += p.n


def test_relres_matches_oracle(helm):
    probs = small_problems()
    nrhs = 2
    ctx = make_ctx(probs)
    per_x, fx = random_batch(probs, nrhs, 9)
    per_b, fb = random_batch(probs, nrhs, 10)
    got = helm.helm_relres(ctx, to_dev(fx, torch.complex128), to_dev(fb, torch.complex128), nrhs)
    k = 0
    for p, xs, bs in zip(probs, per_x, per_b):
        A = hz.assemble(p.c, p.p, p.h, p.omega)
        for r in range(nrhs):
            ref = hz.relres(A, xs[r].ravel(), bs[r].ravel())
            assert abs(got[k] - ref) <= 1e-12 * ref
            k += 1


def test_full_size_fine_grid_32_rhs(helm):
    """512^2 interior + 32 PML, 32 RHS (the fine-grid multi-RHS workload): FP32 and FP64 stencils
    against the oracle's matrix-free stencil on every point."""
    prob = synth.fine_multi_rhs_problem()
    ctx = make_ctx([prob])
    nrhs = 32
    rng = synth.rng_for(12)
    xs = (rng.standard_normal((nrhs, prob.Ny, prob.Nx)) + 1j * rng.standard_normal((nrhs, prob.Ny, prob.Nx)))
    ref = hz.apply(xs, prob.c, prob.p, prob.h, prob.omega)
    x64 = to_dev(xs.ravel(), torch.complex128)
    y64 = torch.empty_like(x64)
    helm.helm_apply(ctx, x64, y64, nrhs)
    g = y64.cpu().numpy().reshape(ref.shape)
    assert np.abs(g - ref).max() <= 1e-12 * np.abs(ref).max()
    xs32 = xs.astype(np.complex64)
    ref32 = hz.apply(xs32.astype(np.complex128), prob.c, prob.p, prob.h, prob.omega)
    x32 = to_dev(xs32.ravel(), torch.complex64)
    y32 = torch.empty_like(x32)
    helm.helm_apply(ctx, x32, y32, nrhs)
    g32 = y32.cpu().numpy().reshape(ref.shape).astype(np.complex128)
    assert np.abs(g32 - ref32).max() <= 2e-6 * np.abs(ref32).max()


def test_invalid_arguments_are_reported(helm):
    probs = small_problems()
    ctx = make_ctx(probs)
    x = ctx.new_vector(1)
    with pytest.raises(helm.HelmError):
        helm.helm_apply(ctx, x, x)          # aliasing
    with pytest.raises(ValueError):
        helm.helm_apply(ctx, x, torch.empty(3, dtype=torch.complex128, device="cuda"))
    bad_c = torch.full((probs[0].n,), -1.0, dtype=torch.float64, device="cuda")
    with pytest.raises(helm.HelmError):
        helm.Context([helm.SystemSpec(probs[0].nx, probs[0].ny, probs[0].h, probs[0].p, probs[0].omega)], bad_c)
