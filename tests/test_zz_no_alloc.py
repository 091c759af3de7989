"""The allocation-free relative residual, called through the C ABI.

helm_relres_noalloc exists for callers that may not allocate device memory while they run (for
example when another framework's caching allocator has reserved the device memory up front, or in
a loop where a cudaMalloc would stall the device).  It must give the same per-column relative
residual as helm_relres, call after call, although its scratch is a fixed array that every call
reuses.  This file is collected last so that a failure here cannot hide any other test.
"""
import numpy as np
import pytest
import torch

from .gpu_util import make_ctx, random_batch, small_problems, to_dev

pytestmark = pytest.mark.gpu


def test_noalloc_relres_matches_allocating_entry_point_twice():
    from paper_2607_16906_b300 import helm
    probs = small_problems(((20, 14, 5), (13, 9, 3), (40, 33, 12)), seed=41)
    nrhs = 3
    ctx = make_ctx(probs)
    ncol = len(probs) * nrhs
    for call, seed in enumerate((51, 52)):
        _, fx = random_batch(probs, nrhs, seed)
        _, fb = random_batch(probs, nrhs, seed + 100)
        x, b = to_dev(fx, torch.complex128), to_dev(fb, torch.complex128)
        ref = helm.helm_relres(ctx, x, b, nrhs)
        out = torch.full((ncol,), -1.0, dtype=torch.float64, device="cuda")
        helm.helm_relres_noalloc(ctx, x, b, out, nrhs)
        got = out.cpu().numpy()
        assert np.all(np.abs(got - ref) <= 1e-12 * ref), (call, got, ref)


def test_noalloc_rejects_batches_beyond_the_fixed_scratch():
    from paper_2607_16906_b300 import helm
    # Nx = 30, Ny = 80: 1 x 10 stencil blocks -> 20 scratch doubles per column; 2^20 doubles hold
    # 52,428 columns, so 60,000 columns (within the launch limit of 65,535) exceed the fixed array
    probs = small_problems(((20, 70, 5),), seed=42)
    ctx = make_ctx(probs)
    nrhs = 60000
    x = torch.zeros(ctx.npts * nrhs, dtype=torch.complex128, device="cuda")
    out = torch.zeros(nrhs, dtype=torch.float64, device="cuda")
    with pytest.raises(helm.HelmError, match="fixed maximum"):
        helm.helm_relres_noalloc(ctx, x, x, out, nrhs)
