"""The seeded generators produce the inputs the workloads are described with: grid shapes, value
ranges, source structure, determinism by seed and the Kaiming-uniform bounds of the network
parameters."""
import numpy as np
import pytest

from oracle import unet
from paper_2607_16906_b300 import synth


def test_wavelength_and_frequency():
    assert synth.grid_spacing(10.0) == pytest.approx(3e-4)  # 3 mm water wavelength / 10
    assert synth.angular_frequency() == pytest.approx(2 * np.pi * 5e5)


def test_skull_velocity_recipe():
    rng = synth.rng_for(1)
    nx, p = 128, 16
    c = synth.skull_velocity(nx, nx, p, rng)
    assert c.shape == (nx + 2 * p, nx + 2 * p)
    assert c.min() >= 1400.0
    # water background with ~50 m/s noise, a ring near 2600-3000 m/s
    assert abs(np.median(c) - 1500.0) < 20.0
    ring = c > 2200.0
    assert 0.02 < ring.mean() < 0.3
    assert 2400.0 < np.median(c[ring]) < 3200.0
    # the noise is 50 m/s std away from the ring
    water = np.abs(c - 1500.0) < 400.0
    assert 35.0 < c[water].std() < 65.0


def test_skull_velocity_large_case_ring():
    c = synth.skull_velocity(512, 512, 32, synth.rng_for(2), thickness=(10, 14), ring_speed=(2600.0, 3200.0))
    ring = c > 2200.0
    assert 2450.0 < np.median(c[ring]) < 3350.0


def test_grf_velocity_range_and_log_normality():
    c = synth.grf_velocity(128, 128, 16, synth.rng_for(3))
    assert c.min() >= 1400.0 and c.max() <= 3000.0
    lg = np.log(c / 2000.0)
    assert abs(lg.mean()) < 0.1 and 0.1 < lg.std() < 0.3


def test_sources_structure():
    rng = synth.rng_for(4)
    nx, p = 64, 8
    b = synth.point_sources(nx, nx, p, rng, 3)
    nz = np.flatnonzero(b)
    assert 1 <= nz.size <= 3
    j, i = np.unravel_index(nz, b.shape)
    assert (i >= p).all() and (i < p + nx).all() and (j >= p).all() and (j < p + nx).all()
    la = synth.line_array(nx, nx, p, rng)
    rows = np.flatnonzero(np.abs(la).sum(axis=1))
    assert rows.size == 1
    cols = np.flatnonzero(la[rows[0]])
    assert cols.size == 32 and np.all(np.diff(cols) == 1)
    assert np.allclose(np.abs(la[rows[0], cols]), 1.0)
    g = synth.gaussian_sources(nx, nx, p, rng)
    assert g.shape == (nx + 2 * p,) * 2 and abs(g.real.std() - 1.0) < 0.05 and abs(g.imag.std() - 1.0) < 0.05


def test_workloads_are_deterministic_and_sized():
    a, b = synth.small_problem(), synth.small_problem()
    assert np.array_equal(a.c, b.c) and np.array_equal(a.b, b.b)
    assert (a.Nx, a.Ny, a.nrhs) == (160, 160, 1)
    f = synth.fine_multi_rhs_problem(nrhs=4)
    assert (f.Nx, f.nrhs) == (576, 4)
    cs, bs, h, om = synth.training_batch(batch=8, nx=32, p=8)
    assert cs.shape == (8, 48, 48) and bs.shape == (8, 48, 48)
    probs = synth.uneven_problems(count=8)
    assert all(pr.nx in (256, 384, 512, 768, 1024) and 16 <= pr.p <= 32 for pr in probs)


def test_kaiming_uniform_bounds():
    segs = unet.param_segments()
    theta = synth.kaiming_uniform_params(segs, 42)
    assert theta.size == unet.param_count() == 482050
    o = 0
    for n, fan_in, kind in segs:
        bound = np.sqrt(6.0 / fan_in) if kind == "w" else 1.0 / np.sqrt(fan_in)  # Kaiming-uniform for ReLU
        part = theta[o:o + n]
        assert np.abs(part).max() <= bound
        if n >= 1000:  # the draws fill the interval
            assert np.abs(part).max() > 0.99 * bound and abs(part.mean()) < 0.05 * bound
        o += n
    assert np.array_equal(theta, synth.kaiming_uniform_params(segs, 42))
    assert not np.array_equal(theta, synth.kaiming_uniform_params(segs, 43))
