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


# ---------------------------------------------------------------- Tab. 4 menus and App. B cases

def test_paper_velocity_menus():
    rng = synth.rng_for(11)
    u = synth.uniform_velocity(30, 20, 4, rng)
    assert u.shape == (28, 38) and u.min() >= 1500 and u.max() <= 3000 and np.unique(u).size == u.size
    c = synth.constant_velocity(30, 20, 4, rng)
    assert np.unique(c).size == 1 and 1500 <= c[0, 0] <= 3000
    sq = synth.square_velocity(40, 40, 4)
    assert set(np.unique(sq)) == {1500.0, 3000.0} and (sq == 3000).sum() == 20 * 20
    assert sq[24, 24] == 3000 and sq[4, 4] == 1500


def test_layered_and_faulted_velocities():
    rng = synth.rng_for(12)
    lay = synth.layered_velocity(64, 64, 8, rng, layers=4)
    assert np.unique(lay).size == 4 and (lay >= 1500).all() and (lay <= 3000).all()
    assert (lay == lay[:, :1]).all()                 # aligned horizontal layers: constant along rows
    rows = [lay[j, 0] for j in range(lay.shape[0])]
    changes = sum(1 for a, b in zip(rows, rows[1:]) if a != b)
    assert changes == 3                              # four layers, three interfaces
    rng = synth.rng_for(12)
    fau = synth.layered_velocity(64, 64, 8, rng, layers=4, faulted=True)
    assert np.unique(fau).size == 4
    cols_differ = [x for x in range(1, fau.shape[1]) if (fau[:, x] != fau[:, x - 1]).any()]
    assert len(cols_differ) == 1                     # one vertical fault line
    xf = cols_differ[0]
    left, right = fau[:, xf - 1], fau[:, xf]
    # right of the fault the same layer sequence appears shifted by one throw
    shifts = [s for s in range(-20, 21) if s != 0 and (np.roll(left, s)[25:55] == right[25:55]).all()]
    assert shifts


def test_dirac_type_sources():
    rng = synth.rng_for(13)
    b = synth.dirac_sources(50, 40, 5, rng, m=3)
    nz = b[b != 0]
    assert nz.size == 3 and set(np.abs(nz.real)) == {1.0} and (nz.imag == 0).all()
    b60 = synth.dirac_sources(50, 40, 5, rng, m=1, amplitude=60.0)
    assert b60[b60 != 0].tolist() == [60.0]
    d1 = synth.dirac1_source(50, 40, 5)
    assert d1[25, 30] == 60.0 and np.count_nonzero(d1) == 1
    d4 = synth.dirac4_source(40, 40, 4)
    assert np.count_nonzero(d4) == 4 and set(d4[d4 != 0].real) == {30.0}
    g = synth.dirac1_smooth_source(64, 64, 0, at=(32, 60), sigma=2.0)
    assert g[32, 60] == 1.0
    assert np.isclose(g[32, 62], np.exp(-0.5)) and np.isclose(g[34, 60], np.exp(-0.5))   # sigma = 2 in x and y
    assert np.isclose(g[30, 58], np.exp(-1.0))


def test_dataset_mixtures_follow_their_probabilities():
    rng = synth.rng_for(14)
    for name, (sp, vp) in synth.DATASETS.items():
        assert abs(sum(sp) - 1) < 1e-12 and abs(sum(vp) - 1) < 1e-12
    n = 1500
    ks = [synth.dataset_sample("D2", 8, 2, rng)[2:] for _ in range(n)]
    sk = np.array([synth.SOURCE_MENU.index(a) for a, _ in ks])
    vk = np.array([synth.VELOCITY_MENU.index(b) for _, b in ks])
    sp, vp = synth.DATASETS["D2"]
    for k in range(4):
        assert abs((sk == k).mean() - sp[k]) < 4 * np.sqrt(sp[k] * (1 - sp[k]) / n) + 1e-9
        assert abs((vk == k).mean() - vp[k]) < 4 * np.sqrt(vp[k] * (1 - vp[k]) / n) + 1e-9
    assert all(synth.dataset_sample("D4", 8, 2, rng)[3] == "skull" for _ in range(20))
    assert all(synth.dataset_sample("D5", 8, 2, rng)[2:] == ("normal", "uniform") for _ in range(20))


def test_appendix_b_problems():
    for kind in ("gamma-constant", "4layered", "4faulted"):
        pr = synth.appendix_b_problem(kind, nx=32, p=4, nrhs=4, m=2)
        assert pr.c.shape == (40, 40) and pr.b.shape == (4, 40, 40)
        assert np.count_nonzero(pr.b[0]) == 2 and np.abs(pr.b[1]).max() == 1.0
        assert np.unique(pr.c).size == (1 if kind == "gamma-constant" else 4)
