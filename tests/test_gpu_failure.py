"""Failure detection without a GPU fault: a pipeline wait that runs out, an allocation that fails,
and batches beyond the launch limits.

The waits are made to run out by a host-set flag (helm_inject_fault) that stops the TMA producer of
one kernel launch from requesting its first tile, with a short wait budget (helm_set_wait_budget).
The kernel then records its error code, lets its own copies land, releases its tensor memory and
returns; helm_fgmres_solve reports HELM_TIMEOUT without applying that cycle's update, and the next
call on the same context and network runs normally.  Nothing here traps, faults or hangs.
"""
import numpy as np
import pytest
import torch

from oracle import unet as ou
from paper_2607_16906_b300 import synth

from .gpu_util import make_ctx, small_problems, to_dev

pytestmark = pytest.mark.gpu

SHORT_BUDGET = 4_000_000   # clock64 cycles, about 2 ms


@pytest.fixture(scope="module")
def helm():
    from paper_2607_16906_b300 import helm as h
    return h


@pytest.fixture(autouse=True)
def _restore(helm):
    yield
    helm.helm_inject_fault(helm.HELM_FAULT_NONE, 0)
    helm.helm_set_wait_budget(0)


def _problem(seed):
    probs = small_problems(((40, 40, 12),), seed=seed)      # Nx = 64: the FP32 TMA stencil runs
    return probs, make_ctx(probs), to_dev(np.concatenate([p.b.ravel() for p in probs]), torch.complex128)


def _solve(helm, ctx, net, b, orth, m=12):
    x = torch.zeros_like(b)
    rc, info = helm.helm_fgmres_solve(ctx, net, b, x, 1, m=m, tol=1e-300, mixed=True, max_outer=2, orth=orth)
    return x, info


def test_stencil_wait_timeout_is_reported_and_the_context_recovers(helm):
    _, ctx, b = _problem(61)
    x_ref, info_ref = _solve(helm, ctx, None, b, "cgs2")
    x = torch.zeros_like(b)
    helm.helm_set_wait_budget(SHORT_BUDGET)
    helm.helm_inject_fault(helm.HELM_FAULT_STENCIL_TILE, 1)
    rc, info = helm.helm_fgmres_solve(ctx, None, b, x, 1, m=6, tol=1e-6, mixed=True, max_outer=3)
    assert rc == helm.HELM_TIMEOUT and info[0]["status"] == "TIMEOUT"
    assert torch.count_nonzero(x).item() == 0           # the cycle's update was not applied
    helm.helm_set_wait_budget(0)
    x2, info2 = _solve(helm, ctx, None, b, "cgs2")       # the same solve as before the fault
    assert torch.equal(x2, x_ref) and info2 == info_ref


@pytest.mark.parametrize("orth", ["dcgs2", "cgs2"])
def test_convolution_wait_timeout_is_reported_and_the_network_recovers(helm, orth):
    probs, ctx, b = _problem(62)
    p = probs[0]
    theta = synth.kaiming_uniform_params(ou.param_segments(), 42)
    net = helm.UNet(theta)
    _solve(helm, ctx, net, b, orth)                      # tile tuning and one-time set-up
    x_ref, info_ref = _solve(helm, ctx, net, b, orth)
    x = torch.zeros_like(b)
    helm.helm_set_wait_budget(SHORT_BUDGET)
    helm.helm_inject_fault(helm.HELM_FAULT_CONV_TILE, 1)
    rc, info = helm.helm_fgmres_solve(ctx, net, b, x, 1, m=4, tol=1e-6, mixed=True, max_outer=2, orth=orth)
    assert rc == helm.HELM_TIMEOUT and info[0]["status"] == "TIMEOUT"
    assert torch.count_nonzero(x).item() == 0
    helm.helm_set_wait_budget(0)
    x2, info2 = _solve(helm, ctx, net, b, orth)
    assert torch.equal(x2, x_ref) and info2 == info_ref
    # and the network still computes what the oracle computes
    rng = synth.rng_for(63)
    v = (rng.standard_normal(p.n) + 1j * rng.standard_normal(p.n)).astype(np.complex64)
    vd = torch.tensor(v, device="cuda")
    zd = torch.empty_like(vd)
    helm.helm_precond_apply(ctx, net, vd, zd)
    zr = ou.precondition(theta, v.reshape(1, p.Ny, p.Nx).astype(complex), p.c, p.h, bf16=True)[0].ravel()
    assert np.linalg.norm(zd.cpu().numpy() - zr) <= 1e-2 * np.linalg.norm(zr)


def test_injected_allocation_failure_reports_oom(helm):
    _, ctx, b = _problem(64)
    x = torch.zeros_like(b)
    helm.helm_inject_fault(helm.HELM_FAULT_ALLOC, 1)
    with pytest.raises(helm.HelmError) as e:
        helm.helm_fgmres_solve(ctx, None, b, x, 1, m=8, tol=1e-6, mixed=True, max_outer=4)
    assert e.value.status == helm.HELM_ERR_OOM and "injected" in str(e.value)
    x2, info2 = _solve(helm, ctx, None, b, "cgs2")
    _, ctx_fresh, _ = _problem(64)
    x3, info3 = _solve(helm, ctx_fresh, None, b, "cgs2")
    assert torch.equal(x2, x3) and info2 == info3


def test_batches_beyond_the_launch_limit_are_rejected_before_any_launch(helm):
    """nsys * nrhs is one grid dimension of the column kernels: 65,536 columns are refused with
    HELM_ERR_INVALID_ARG by every entry point (tensors are sized correctly, so nothing could read
    out of bounds even if a launch happened)."""
    probs = small_problems(((4, 4, 1),), seed=65)
    ctx = make_ctx(probs)
    nrhs = helm.HELM_MAX_COLUMNS + 1
    v = torch.zeros(ctx.npts * nrhs, dtype=torch.complex128, device="cuda")
    w = torch.zeros_like(v)
    for call in (lambda: helm.helm_apply(ctx, v, w, nrhs),
                 lambda: helm.helm_relres(ctx, v, w, nrhs),
                 lambda: helm.helm_relres_noalloc(ctx, v, w, torch.zeros(nrhs, dtype=torch.float64, device="cuda"),
                                                  nrhs),
                 lambda: helm.helm_fgmres_solve(ctx, None, v, w, nrhs, m=2)):
        with pytest.raises(helm.HelmError) as e:
            call()
        assert e.value.status == helm.HELM_ERR_INVALID_ARG and "HELM_MAX_COLUMNS" in str(e.value)
    # the limit itself is accepted
    ok = helm.HELM_MAX_COLUMNS
    helm.helm_apply(ctx, v[:ctx.npts * ok], w[:ctx.npts * ok], ok)
    torch.cuda.synchronize()
