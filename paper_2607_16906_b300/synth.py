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


# ---------------------------------------------------------------- the paper's training distributions
#
# Sec. 3.2 draws velocities and sources independently from small menus and mixes them with fixed
# probabilities (Tab. 4, datasets D0-D5).  The paper's c is normalised to [1, 2]; here c = 1500 m/s
# times that value.  TruncIdealSkulls (cropped idealised skull images) is not available: the
# skull ring above stands in for it.

def uniform_velocity(nx: int, ny: int, p: int, rng: np.random.Generator) -> np.ndarray:
    """U([1, 2]): every entry of c drawn independently, c = 1500 m/s x U[1, 2]."""
    Nx, Ny = nx + 2 * p, ny + 2 * p
    return C_WATER * rng.uniform(1.0, 2.0, (Ny, Nx))


def constant_velocity(nx: int, ny: int, p: int, rng: np.random.Generator) -> np.ndarray:
    """randConstant (Sec. 3.2) and gamma-constant (App. B): one value gamma ~ U[1, 2] everywhere."""
    Nx, Ny = nx + 2 * p, ny + 2 * p
    return np.full((Ny, Nx), C_WATER * rng.uniform(1.0, 2.0))


def square_velocity(nx: int, ny: int, p: int, rng: np.random.Generator = None, frac=0.5) -> np.ndarray:
    """square (Sec. 3.2): c = 2 (3000 m/s) on a centred square, 1 (1500 m/s) elsewhere; the square's
    side is `frac` of the interior's smaller side (the paper does not give it)."""
    Nx, Ny = nx + 2 * p, ny + 2 * p
    c = np.full((Ny, Nx), C_WATER)
    side = max(1, int(round(frac * min(nx, ny))))
    y0, x0 = (Ny - side) // 2, (Nx - side) // 2
    c[y0:y0 + side, x0:x0 + side] = 2.0 * C_WATER
    return c


def layered_velocity(nx: int, ny: int, p: int, rng: np.random.Generator, layers=4, faulted=False,
                     alpha=1.0, beta=2.0) -> np.ndarray:
    """4layered / 4faulted (App. B): `layers` horizontal layers, each of one speed 1500 m/s x
    U[alpha, beta]; interfaces at sorted random interior rows.  Faulted: right of a random
    vertical fault line every interface is shifted by one common random offset (a throw of 5-20 %
    of the interior height, up or down), so the layers stay aligned but are discontinuous."""
    Nx, Ny = nx + 2 * p, ny + 2 * p
    speeds = C_WATER * rng.uniform(alpha, beta, layers)
    cuts = np.sort(rng.choice(np.arange(p + 1, p + ny), layers - 1, replace=False))
    rows = np.arange(Ny)[:, None] * np.ones((1, Nx))
    shift = np.zeros((Ny, Nx))
    if faulted:
        xf = int(rng.integers(p + nx // 4, p + 3 * nx // 4))
        throw = int(round(rng.uniform(0.05, 0.20) * ny)) * (1 if rng.uniform() < 0.5 else -1)
        shift[:, xf:] = throw
    layer = np.searchsorted(cuts, rows - shift, side="right")
    return speeds[layer]


def dirac_sources(nx: int, ny: int, p: int, rng: np.random.Generator, m=1, amplitude=None) -> np.ndarray:
    """m dirac (App. B): m entries of b set to +-1 (random signs) at random interior nodes; with
    `amplitude` (Sec. 3.2's dirac: 60) every entry gets that value instead."""
    Nx, Ny = nx + 2 * p, ny + 2 * p
    b = np.zeros((Ny, Nx), np.complex128)
    for _ in range(m):
        i = int(rng.integers(p, p + nx))
        j = int(rng.integers(p, p + ny))
        b[j, i] = amplitude if amplitude is not None else (1.0 if rng.uniform() < 0.5 else -1.0)
    return b


def dirac1_source(nx: int, ny: int, p: int, amplitude=60.0, at=None) -> np.ndarray:
    """dirac1: one entry `amplitude` at `at` = (row, column), by default the grid centre (Sec. 3.2;
    the tests of Sec. 4.2 put amplitude 1 at a fixed off-centre node)."""
    Nx, Ny = nx + 2 * p, ny + 2 * p
    b = np.zeros((Ny, Nx), np.complex128)
    j, i = at if at is not None else (Ny // 2, Nx // 2)
    b[j, i] = amplitude
    return b


def dirac4_source(nx: int, ny: int, p: int, amplitude=30.0) -> np.ndarray:
    """dirac4 (Sec. 3.2): four entries `amplitude` at fixed nodes, here the interior's quarter points."""
    Nx, Ny = nx + 2 * p, ny + 2 * p
    b = np.zeros((Ny, Nx), np.complex128)
    for fy in (0.25, 0.75):
        for fx in (0.25, 0.75):
            b[p + int(fy * ny), p + int(fx * nx)] = amplitude
    return b


def dirac1_smooth_source(nx: int, ny: int, p: int, at=None, sigma=2.0) -> np.ndarray:
    """dirac1_smooth (Sec. 4.2): a Gaussian bump exp(-((x - c_x)^2 + (y - c_y)^2) / (2 sigma^2)) in
    grid units, sigma = 2, centred at `at` = (c_y, c_x) (default: the node the paper's (60, 32) on a
    64 x 64 grid maps to).  The printed formula repeats x in its second term; read as y."""
    Nx, Ny = nx + 2 * p, ny + 2 * p
    cy, cx = at if at is not None else (int(round(32 / 64 * (Ny - 1))), int(round(60 / 64 * (Nx - 1))))
    yy, xx = np.mgrid[0:Ny, 0:Nx].astype(np.float64)
    return np.exp(-((xx - cx) ** 2 + (yy - cy) ** 2) / (2.0 * sigma * sigma)).astype(np.complex128)


# Tab. 4: source and velocity menus with their probabilities per dataset
SOURCE_MENU = ("normal", "dirac", "dirac1", "dirac4")
VELOCITY_MENU = ("uniform", "skull", "constant", "square")
DATASETS = {
    "D0": ((0.6, 0.3, 0.05, 0.05), (0.5, 0.5, 0.0, 0.0)),
    "D1": ((1.0, 0.0, 0.0, 0.0), (0.5, 0.5, 0.0, 0.0)),
    "D2": ((0.6, 0.3, 0.05, 0.05), (0.4, 0.4, 0.1, 0.1)),
    "D3": ((1.0, 0.0, 0.0, 0.0), (0.4, 0.4, 0.1, 0.1)),
    "D4": ((1.0, 0.0, 0.0, 0.0), (0.0, 1.0, 0.0, 0.0)),
    "D5": ((1.0, 0.0, 0.0, 0.0), (1.0, 0.0, 0.0, 0.0)),
}


def dataset_sample(name: str, nx: int, p: int, rng: np.random.Generator):
    """One (c, b, source kind, velocity kind) pair of dataset `name` (Tab. 4) on an nx^2 + p PML grid."""
    sp, vp = DATASETS[name]
    sk = SOURCE_MENU[int(rng.choice(4, p=sp))]
    vk = VELOCITY_MENU[int(rng.choice(4, p=vp))]
    c = {"uniform": uniform_velocity, "skull": skull_velocity, "constant": constant_velocity,
         "square": square_velocity}[vk](nx, nx, p, rng)
    if sk == "normal":
        b = gaussian_sources(nx, nx, p, rng)
    elif sk == "dirac":
        b = dirac_sources(nx, nx, p, rng, 1, amplitude=60.0)
    elif sk == "dirac1":
        b = dirac1_source(nx, nx, p)
    else:
        b = dirac4_source(nx, nx, p)
    return c, b, sk, vk


def appendix_b_problem(kind: str, seed=6000, nx=128, p=16, ppw=10.0, nrhs=4, m=2) -> Problem:
    """App. B test cases: velocity `kind` in {"gamma-constant", "4layered", "4faulted"}; sources
    alternate between m dirac (+-1 at m random nodes) and dirac1_smooth."""
    rng = rng_for(seed)
    vel = {"gamma-constant": constant_velocity,
           "4layered": lambda *a: layered_velocity(*a, layers=4),
           "4faulted": lambda *a: layered_velocity(*a, layers=4, faulted=True)}[kind]
    c = vel(nx, nx, p, rng)
    b = np.stack([dirac_sources(nx, nx, p, rng, m) if k % 2 == 0 else dirac1_smooth_source(nx, nx, p)
                  for k in range(nrhs)])
    return Problem(nx, nx, p, grid_spacing(ppw), angular_frequency(), c, b,
                   {"workload": f"App. B {kind}, {m} dirac / dirac1_smooth, {nx}^2+{p} PML", "seed": seed, "ppw": ppw})


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
    U(+-sqrt(6/fan_in)), i.e. Kaiming-uniform for ReLU), "b" (bias,
    U(+-1/sqrt(fan_in))) or "s" (PReLU slopes: the usual initial value 0.25,
    nothing drawn).  The caller supplies the layout; seed 42 is the paper's
    random seed (Tab. 3).
    """
    rng = rng_for(seed)
    parts = []
    for count, fan_in, kind in segments:
        if kind == "s":
            parts.append(np.full(int(count), 0.25))
            continue
        bound = np.sqrt(6.0 / fan_in) if kind == "w" else 1.0 / np.sqrt(fan_in)
        parts.append(rng.uniform(-bound, bound, int(count)))
    return np.concatenate(parts) if parts else np.zeros(0)
