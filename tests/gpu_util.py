"""Helpers for the GPU tests: build contexts from the seeded synthetic problems."""
import numpy as np
import torch

from paper_2607_16906_b300 import synth


def specs_of(problems):
    from paper_2607_16906_b300 import helm
    return [helm.SystemSpec(p.nx, p.ny, p.h, p.p, p.omega) for p in problems]


def make_ctx(problems):
    from paper_2607_16906_b300 import helm
    c = torch.tensor(np.concatenate([p.c.ravel() for p in problems]), dtype=torch.float64, device="cuda")
    return helm.Context(specs_of(problems), c)


def small_problems(sizes=((20, 14, 5), (13, 9, 3)), seed=17, nrhs=1, ppw=10.0):
    """Uneven systems (nx, ny, p) with skull rings and random point sources."""
    rng = synth.rng_for(seed)
    out = []
    for nx, ny, p in sizes:
        c = synth.skull_velocity(nx, ny, p, rng, thickness=(1, 2))
        b = np.stack([synth.point_sources(nx, ny, p, rng, 2) for _ in range(nrhs)])
        out.append(synth.Problem(nx, ny, p, synth.grid_spacing(ppw), synth.angular_frequency(), c, b))
    return out


def random_batch(problems, nrhs, seed, dtype=np.complex128):
    """List (per system) of [nrhs][Ny][Nx] random complex arrays, and their flat concatenation."""
    rng = synth.rng_for(seed)
    per = [(rng.standard_normal((nrhs, p.Ny, p.Nx)) + 1j * rng.standard_normal((nrhs, p.Ny, p.Nx))).astype(dtype)
           for p in problems]
    flat = np.concatenate([a.ravel() for a in per])
    return per, flat


def to_dev(flat, dtype):
    return torch.tensor(flat, device="cuda").to(dtype).contiguous()


def split(flat, problems, nrhs):
    out, o = [], 0
    for p in problems:
        k = nrhs * p.n
        out.append(flat[o:o + k].reshape(nrhs, p.Ny, p.Nx))
        o += k
    return out
