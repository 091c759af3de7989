"""Seeded synthetic inputs: velocity fields, sources, network parameters.

This module only draws numbers. It holds none of the solver's arithmetic
(no PML profile, no wavenumber, no stencil, no network layer). Both the CPU
oracle and the CUDA path take their inputs from here, so that they see the
same bytes.

Stand-ins for the paper's data (Sec. 3.2, Sec. 4.2, Sec. 4.3), which are not
available here:
  * skull ring + filtered noise   stands in for the idealised skulls and the
                                  head-CT slices of Sec. 4.2-4.3;
  * log-normal Gaussian random field (smooth heterogeneous media);
  * unit-modulus point sources and a 32-element line array with random phases
    stand in for the dirac-type sources and the arc transducer of Sec. 4.3.

Units are physical: c in m/s, h in metres, omega in rad/s.  The paper's
normalised setting (omega = 1, c in [1, 2]) maps onto this by c / 1500 m/s.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
from scipy import ndimage

C_WATER = 1500.0          # m/s
F_SOURCE = 5.0e5          # Hz; 500 kHz transcranial-ultrasound band (Sec. 4.3 uses 490 kHz)


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


@dataclass
class Problem:
    """One velocity field on a grid with PML, plus its right-hand sides.

    Grid: interior nx x ny cells plus p PML cells per side; arrays are
    row-major [Ny][Nx] with Nx = nx + 2p, Ny = ny + 2p.
    """
    nx: int
    ny: int
    p: int
    h: float
    omega: float
    c: np.ndarray                      # float64 [Ny][Nx], m/s
    b: np.ndarray                      # complex128 [nrhs][Ny][Nx]
    meta: dict = field(default_factory=dict)

    @property
    def Nx(self) -> int:
        return self.nx + 2 * self.p

    @property
    def Ny(self) -> int:
        return self.ny + 2 * self.p

    @property
    def n(self) -> int:
        return self.Nx * self.Ny

    @property
    def nrhs(self) -> int:
        return self.b.shape[0]


def grid_spacing(ppw: float) -> float:
    """Cell size h such that the water wavelength spans `ppw` cells."""
    return (C_WATER / F_SOURCE) / ppw


def angular_frequency() -> float:
    return 2.0 * np.pi * F_SOURCE


def _filtered_noise(rng, shape, sigma_cells, std):
    w = rng.standard_normal(shape)
    f = ndimage.gaussian_filter(w, sigma_cells, mode="wrap")
    s = f.std()
    return f * (std / s) if s > 0 else f


def skull_velocity(nx: int, ny: int, p: int, rng: np.random.Generator, *,
                   thickness=(6, 8), ring_speed=(2600.0, 3000.0),
                   noise_std=50.0, noise_sigma=2.0) -> np.ndarray:
    """Water background + elliptical skull-like ring + Gaussian-filtered noise.

    Ring: centre offset U(+-0.05 n), semi-axes U[0.30, 0.42] n, thickness an
    integer in [thickness[0], thickness[1]] cells, constant speed drawn from
    U(ring_speed).  Noise: white N(0,1), Gaussian filter of `noise_sigma` cells,
    rescaled to `noise_std` m/s, added everywhere; result clipped at 1400 m/s.
    """
    Nx, Ny = nx + 2 * p, ny + 2 * p
    c = np.full((Ny, Nx), C_WATER)
    cx = (Nx - 1) / 2.0 + rng.uniform(-0.05, 0.05) * nx
    cy = (Ny - 1) / 2.0 + rng.uniform(-0.05, 0.05) * ny
    ax = rng.uniform(0.30, 0.42) * nx
    ay = rng.uniform(0.30, 0.42) * ny
    t = int(rng.integers(thickness[0], thickness[1] + 1))
    speed = rng.uniform(*ring_speed)
    yy, xx = np.mgrid[0:Ny, 0:Nx].astype(np.float64)
    outer = ((xx - cx) / ax) ** 2 + ((yy - cy) / ay) ** 2 <= 1.0
    inner = ((xx - cx) / (ax - t)) ** 2 + ((yy - cy) / (ay - t)) ** 2 <= 1.0
    c[outer & ~inner] = speed
    c = c + _filtered_noise(rng, c.shape, noise_sigma, noise_std)
    return np.maximum(c, 1400.0)


def grf_velocity(nx: int, ny: int, p: int, rng: np.random.Generator, *,
                 corr_cells=16.0, log_std=0.2, mean=2000.0) -> np.ndarray:
    """Log-normal Gaussian random field: log c = log(mean) + GRF, clipped to [1400, 3000] m/s."""
    Nx, Ny = nx + 2 * p, ny + 2 * p
    g = _filtered_noise(rng, (Ny, Nx), corr_cells / np.sqrt(2.0), log_std)
    return np.clip(mean * np.exp(g), 1400.0, 3000.0)


def point_sources(nx: int, ny: int, p: int, rng: np.random.Generator, count=1) -> np.ndarray:
    """`count` unit-modulus point sources with random phases at random interior nodes."""
    Nx, Ny = nx + 2 * p, ny + 2 * p
    b = np.zeros((Ny, Nx), np.complex128)
    for _ in range(count):
        i = int(rng.integers(p, p + nx))
        j = int(rng.integers(p, p + ny))
        b[j, i] += np.exp(1j * rng.uniform(0.0, 2.0 * np.pi))
    return b


def line_array(nx: int, ny: int, p: int, rng: np.random.Generator, elements=32) -> np.ndarray:
    """`elements` consecutive nodes along one interior row, each e^{i phi}, phi ~ U[0, 2pi)."""
    Nx, Ny = nx + 2 * p, ny + 2 * p
    b = np.zeros((Ny, Nx), np.complex128)
    elements = min(elements, nx)
    j = int(rng.integers(p, p + ny))
    i0 = int(rng.integers(p, p + nx - elements + 1))
    b[j, i0:i0 + elements] = np.exp(1j * rng.uniform(0.0, 2.0 * np.pi, elements))
    return b


def gaussian_sources(nx, ny, p, rng) -> np.ndarray:
    """Complex N(0,1) i.i.d. entries over the whole grid (the paper's N(0,1) sources)."""
    Nx, Ny = nx + 2 * p, ny + 2 * p
    return rng.standard_normal((Ny, Nx)) + 1j * rng.standard_normal((Ny, Nx))


# ---------------------------------------------------------------- workloads

def small_problem(seed=1000, nx=128, p=16, ppw=10.0) -> Problem:
    """128^2 interior + 16 PML, one skull ring, one random unit point source."""
    rng = rng_for(seed)
    c = skull_velocity(nx, nx, p, rng)
    b = point_sources(nx, nx, p, rng, 1)[None]
    return Problem(nx, nx, p, grid_spacing(ppw), angular_frequency(), c, b,
                   {"workload": f"skull {nx}^2+{p} PML, 1 point source", "seed": seed, "ppw": ppw})


def fine_multi_rhs_problem(seed=3000, nx=512, p=32, nrhs=32, ppw=10.0) -> Problem:
    """512^2 interior + 32 PML, one skull velocity, `nrhs` random point sources."""
    rng = rng_for(seed)
    c = skull_velocity(nx, nx, p, rng)
    b = np.stack([point_sources(nx, nx, p, rng, 1) for _ in range(nrhs)])
    return Problem(nx, nx, p, grid_spacing(ppw), angular_frequency(), c, b,
                   {"workload": f"skull {nx}^2+{p} PML, {nrhs} point-source RHS", "seed": seed, "ppw": ppw})


def large_problem(seed=5000, nx=2048, p=64, nrhs=8, ppw=12.0) -> Problem:
    """2048^2 interior + 64 PML, thin skull ring, `nrhs` line-array RHS."""
    rng = rng_for(seed)
    c = skull_velocity(nx, nx, p, rng, thickness=(10, 14), ring_speed=(2600.0, 3200.0))
    b = np.stack([line_array(nx, nx, p, rng) for _ in range(nrhs)])
    return Problem(nx, nx, p, grid_spacing(ppw), angular_frequency(), c, b,
                   {"workload": f"skull {nx}^2+{p} PML, {nrhs} line-array RHS", "seed": seed, "ppw": ppw})


def training_batch(seed=2000, batch=64, nx=128, p=16, ppw=10.0):
    """Mixed training batch at one grid: half skull, half log-normal GRF velocities;
    half 1-5 random point sources, half a 32-element line array.

    Returns (c [B][Ny][Nx] float64, b [B][Ny][Nx] complex128, h, omega).
    """
    rng = rng_for(seed)
    cs, bs = [], []
    for k in range(batch):
        cs.append(skull_velocity(nx, nx, p, rng) if k < batch // 2 else grf_velocity(nx, nx, p, rng))
        if rng.uniform() < 0.5:
            bs.append(point_sources(nx, nx, p, rng, int(rng.integers(1, 6))))
        else:
            bs.append(line_array(nx, nx, p, rng))
    return np.stack(cs), np.stack(bs), grid_spacing(ppw), angular_frequency()


def uneven_problems(seed=4000, count=64, sides=(256, 384, 512, 768, 1024)):
    """`count` systems with interior sides drawn from `sides`, PML 16-32, PPW U[8,12]."""
    rng = rng_for(seed)
    out = []
    for k in range(count):
        nx = int(sides[int(rng.integers(0, len(sides)))])
        p = int(rng.integers(16, 33))
        ppw = float(rng.uniform(8.0, 12.0))
        c = skull_velocity(nx, nx, p, rng)
        b = point_sources(nx, nx, p, rng, 1)[None]
        out.append(Problem(nx, nx, p, grid_spacing(ppw), angular_frequency(), c, b,
                           {"seed": seed, "index": k, "ppw": ppw}))
    return out


def kaiming_uniform_params(segments, seed=42) -> np.ndarray:
    """Flat float64 parameter vector drawn from a seeded PCG64 stream.

    `segments` is a list of (count, fan_in, kind) with kind "w" (weights,
    U(+-sqrt(6/fan_in)), i.e. Kaiming-uniform for ReLU) or "b" (bias,
    U(+-1/sqrt(fan_in))).  The caller supplies the layout; seed 42 is the
    paper's random seed (Tab. 3).
    """
    rng = rng_for(seed)
    parts = []
    for count, fan_in, kind in segments:
        bound = np.sqrt(6.0 / fan_in) if kind == "w" else 1.0 / np.sqrt(fan_in)
        parts.append(rng.uniform(-bound, bound, int(count)))
    return np.concatenate(parts) if parts else np.zeros(0)
