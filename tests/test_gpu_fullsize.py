"""Full-size checks of the solver workloads in the launch configurations the solver uses.

At these sizes the oracle cannot run FGMRES itself; it checks what holds at any size or what it can
compute one output at a time: the FP64 true residual the solver reports for every column (eq. 10)
against the oracle's CSR matrix and the returned x, the stencil on every point (eq. 3), and the
preconditioner (eqs. 5-7) on a window whose centre lies farther than the network's receptive field
(44 cells, plus the 8-cell pooling alignment) from the window edge.
"""
import os

import numpy as np
import pytest
import torch

from oracle import helmholtz as hz
from oracle import unet
from paper_2607_16906_b300 import synth

from .gpu_util import make_ctx, to_dev

pytestmark = pytest.mark.gpu

WEIGHTS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2607_16906_b300",
                       "weights", "unet_trained.npy")


@pytest.fixture(scope="module")
def helm():
    from paper_2607_16906_b300 import helm as h
    return h


@pytest.fixture(scope="module")
def trained():
    return np.load(WEIGHTS)


def _check_reported_residuals(probs, nrhs, x, info):
    """Per column: the solver's FP64 true residual equals the oracle's CSR residual of x."""
    flat = x.cpu().numpy()
    k = o = 0
    for p in probs:
        A = hz.assemble(p.c, p.p, p.h, p.omega)
        for r in range(nrhs):
            xr = flat[o + r * p.n: o + (r + 1) * p.n]
            ref = hz.relres(A, xr, p.b[r].ravel())
            assert abs(info[k]["relres_true"] - ref) <= 1e-9 * ref, (k, info[k]["relres_true"], ref)
            assert ref < 1.0, (k, ref)  # the preconditioned cycle reduced the residual
            k += 1
        o += nrhs * p.n
        del A


def test_fine_grid_32_rhs_mixed_cycle(helm, trained):
    """576^2, 32 RHS in one call, DCGS2, trained BF16 network: one 20-vector FP32 cycle + FP64 residual."""
    prob = synth.fine_multi_rhs_problem()
    ctx = make_ctx([prob])
    net = helm.UNet(trained)
    b = to_dev(prob.b.ravel(), torch.complex128)
    x = torch.zeros_like(b)
    rc, info = helm.helm_fgmres_solve(ctx, net, b, x, 32, m=20, tol=1e-6, mixed=True, max_outer=1, inner_tol=1e-5,
                                      orth="dcgs2")
    assert rc == helm.HELM_NOT_CONVERGED
    assert all(c["iters"] == 20 and c["status"] == "NOT_CONVERGED" for c in info)
    _check_reported_residuals([prob], 32, x, info)


def test_large_grid_stencil_every_point(helm):
    """2176^2 (2048^2 + 64 PML), 8 RHS: FP32 and FP64 stencil on every point against the oracle."""
    prob = synth.large_problem()
    ctx = make_ctx([prob])
    rng = synth.rng_for(41)
    xs = rng.standard_normal((8, prob.Ny, prob.Nx)) + 1j * rng.standard_normal((8, prob.Ny, prob.Nx))
    x64 = to_dev(xs.ravel(), torch.complex128)
    y64 = torch.empty_like(x64)
    helm.helm_apply(ctx, x64, y64, 8)
    ref = hz.apply(xs, prob.c, prob.p, prob.h, prob.omega)
    g = y64.cpu().numpy().reshape(ref.shape)
    assert np.abs(g - ref).max() <= 1e-12 * np.abs(ref).max()
    del x64, y64, g
    xs32 = xs.astype(np.complex64)
    ref32 = hz.apply(xs32.astype(np.complex128), prob.c, prob.p, prob.h, prob.omega)
    x32 = to_dev(xs32.ravel(), torch.complex64)
    y32 = torch.empty_like(x32)
    helm.helm_apply(ctx, x32, y32, 8)
    g32 = y32.cpu().numpy().reshape(ref.shape).astype(np.complex128)
    assert np.abs(g32 - ref32).max() <= 2e-6 * np.abs(ref32).max()


def test_large_grid_network_window_and_cycle(helm, trained):
    """2176^2, 8 line-array RHS: the BF16 network on the full grid agrees with the oracle's BF16
    emulation on a 256^2 window (centre 128^2 compared), and one 10-vector mixed cycle reports the
    true residual the oracle computes."""
    prob = synth.large_problem()
    ctx = make_ctx([prob])
    net = helm.UNet(trained)
    rng = synth.rng_for(43)
    vs = (rng.standard_normal((8, prob.Ny, prob.Nx)) + 1j * rng.standard_normal((8, prob.Ny, prob.Nx)))
    vs = vs.astype(np.complex64)
    v = to_dev(vs.ravel(), torch.complex64)
    z = torch.empty_like(v)
    helm.helm_precond_apply(ctx, net, v, z, 8)
    g = z.cpu().numpy().reshape(8, prob.Ny, prob.Nx)
    assert np.isfinite(g).all()
    del v, z
    y0, x0, win, margin = 1000, 504, 256, 64  # window origin a multiple of 8 (pooling alignment)
    for k in (0, 5):
        vk = vs[k].astype(np.complex128)
        alpha = np.sqrt(vk.size) / np.linalg.norm(vk)
        xin = unet.network_input((vk * alpha)[None, y0:y0 + win, x0:x0 + win], prob.c[y0:y0 + win, x0:x0 + win])
        y = unet.forward(trained, xin, bf16=True)
        ref = (y[0, 0] + 1j * y[0, 1]) * (prob.h * prob.h / alpha)
        c = slice(margin, win - margin)
        got = g[k, y0:y0 + win, x0:x0 + win][c, c]
        assert np.linalg.norm(got - ref[c, c]) / np.linalg.norm(ref[c, c]) <= 1e-2
    b = to_dev(prob.b.ravel(), torch.complex128)
    x = torch.zeros_like(b)
    rc, info = helm.helm_fgmres_solve(ctx, net, b, x, 8, m=10, tol=1e-8, mixed=True, max_outer=1, inner_tol=1e-5,
                                      orth="dcgs2")
    assert all(c["iters"] == 10 for c in info)
    _check_reported_residuals([prob], 8, x, info)


def test_uneven_batch_64_systems_mixed_cycle(helm, trained):
    """64 systems with sides {256..1024} + PML 16-32 in one context: one 10-vector mixed cycle; each
    system's reported FP64 true residual equals the oracle's."""
    probs = synth.uneven_problems()
    ctx = make_ctx(probs)
    net = helm.UNet(trained)
    b = to_dev(np.concatenate([p.b.ravel() for p in probs]), torch.complex128)
    x = torch.zeros_like(b)
    rc, info = helm.helm_fgmres_solve(ctx, net, b, x, 1, m=10, tol=1e-6, mixed=True, max_outer=1, inner_tol=1e-5,
                                      orth="dcgs2")
    assert len(info) == 64 and all(c["iters"] == 10 for c in info)
    _check_reported_residuals(probs, 1, x, info)
