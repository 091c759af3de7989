"""Pins of the oracle's Helmholtz operator against closed forms, library routines and invariants.

Each test would fail on a plausible slip in oracle/helmholtz.py: a wrong sign
of the PML damping (Green's-function and reflection tests), a wrong
half-node index (symmetry, Green's function, manufactured solution), a
dropped k^2 or 1/h^2 (manufactured solution), a conjugation error in the
adjoint (dot-product test).
"""
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import helmholtz as hz
from paper_2607_16906_b300 import synth

OMEGA = synth.angular_frequency()


def _small(seed=7, nx=20, ny=14, p=5, ppw=10.0):
    rng = synth.rng_for(seed)
    c = synth.skull_velocity(nx, ny, p, rng, thickness=(2, 3))
    return c, p, synth.grid_spacing(ppw)


def test_complex_symmetric_exactly():
    c, p, h = _small()
    A = hz.assemble(c, p, h, OMEGA)
    D = (A - A.T).tocoo()
    assert D.nnz == 0 or np.max(np.abs(D.data)) == 0.0
    assert np.abs(A.imag).max() > 0          # the PML makes A complex


def test_matrix_free_equals_csr():
    c, p, h = _small()
    A = hz.assemble(c, p, h, OMEGA)
    rng = synth.rng_for(3)
    u = rng.standard_normal((3,) + c.shape) + 1j * rng.standard_normal((3,) + c.shape)
    for k in range(3):
        ref = A @ u[k].ravel()
        got = hz.apply(u[k], c, p, h, OMEGA).ravel()
        assert np.linalg.norm(got - ref) <= 1e-14 * np.linalg.norm(ref)


def test_no_pml_is_real_symmetric_and_textbook_laplacian():
    """sigma_max = 0: A is the real 5-point -Lap_h - k^2 with Dirichlet walls."""
    c, p, h = _small()
    A = hz.assemble(c, p, h, OMEGA, sigma_max=0.0)
    assert np.abs(A.imag).max() == 0.0
    Ny, Nx = c.shape
    L1x = sp.diags([-np.ones(Nx - 1), 2 * np.ones(Nx), -np.ones(Nx - 1)], [-1, 0, 1])
    L1y = sp.diags([-np.ones(Ny - 1), 2 * np.ones(Ny), -np.ones(Ny - 1)], [-1, 0, 1])
    lap = (sp.kron(sp.eye(Ny), L1x) + sp.kron(L1y, sp.eye(Nx))) / h ** 2
    ref = lap - sp.diags(((OMEGA / c) ** 2).ravel())
    assert abs(A - ref).max() <= 1e-12 * abs(ref).max()


def test_pml_profile_values_at_layer_edges():
    """eq. 2: sigma vanishes on the interior nodes and reaches sigma_max at the outermost node."""
    c, p, h = _small()
    _, sx, sxh, sy, syh = hz.coefficients(c, p, h, OMEGA)
    Ny, Nx = c.shape
    assert np.all(sx[p:Nx - p] == 1.0) and np.all(sy[p:Ny - p] == 1.0)
    assert sx[0] == pytest.approx(1 + 2j) and sx[-1] == pytest.approx(1 + 2j)
    assert sy[0] == pytest.approx(1 + 2j)
    # half nodes inside the interior are undamped; the ones in the layer are damped and increase outward
    assert np.all(sxh[p + 1:Nx - p] == 1.0)
    assert np.all(np.diff(sxh[:p + 1].imag) < 0)


def test_pml_profile_matches_table1_configuration():
    """tests/golden/pml_tab1_profile.txt: eq. 2 with the Tab. 1 PML (l = 4, sigma_max = 2, omega = 1),
    written out by hand at the nodes and half nodes of a 4-cell layer with unit spacing."""
    path = os.path.join(os.path.dirname(__file__), "golden", "pml_tab1_profile.txt")
    rows = np.loadtxt(path, comments="#")
    t, d = rows[:, 0], rows[:, 1]
    s = hz.stretch(t, 8, 4, 1.0, 1.0, 2.0)  # 8 interior cells, 4-cell layer
    assert np.array_equal(s.real, rows[:, 2]) and np.array_equal(s.imag, rows[:, 3])
    # the mirrored positions on the right edge (first node past the interior is t = 4 + 8)
    s_r = hz.stretch(4 + 8 - 1 + d, 8, 4, 1.0, 1.0, 2.0)
    assert np.array_equal(s_r.imag, rows[:, 3])


def test_adjoint_dot_product_and_conjugate_transpose():
    c, p, h = _small()
    A = hz.assemble(c, p, h, OMEGA)
    rng = synth.rng_for(11)
    x = rng.standard_normal(c.shape) + 1j * rng.standard_normal(c.shape)
    y = rng.standard_normal(c.shape) + 1j * rng.standard_normal(c.shape)
    Ax = hz.apply(x, c, p, h, OMEGA)
    AHy = hz.apply_adjoint(y, c, p, h, OMEGA)
    lhs = np.vdot(y, Ax)          # <Ax, y> = y^H A x
    rhs = np.vdot(AHy, x)         # <x, A^H y> = (A^H y)^H x
    assert abs(lhs - rhs) <= 1e-14 * np.linalg.norm(Ax) * np.linalg.norm(y)
    ref = A.conj().T @ y.ravel()
    assert np.linalg.norm(AHy.ravel() - ref) <= 1e-14 * np.linalg.norm(ref)


def test_direct_solve_matches_dense_bruteforce():
    """16x16 interior + 4 PML: sparse LU == dense numpy.linalg.solve."""
    rng = synth.rng_for(5)
    c = synth.skull_velocity(16, 16, 4, rng, thickness=(2, 3))
    h = synth.grid_spacing(10.0)
    A = hz.assemble(c, 4, h, OMEGA)
    b = synth.point_sources(16, 16, 4, rng, 3).ravel()
    x = hz.solve_direct(A, b)
    xd = np.linalg.solve(A.toarray(), b)
    assert np.linalg.norm(x - xd) <= 1e-12 * np.linalg.norm(xd)
    assert hz.relres(A, x, b) <= 1e-13


def _greens_error(ppw, lam_interior=6.0, lam_pml=1.0):
    h = synth.grid_spacing(ppw)
    lam = synth.C_WATER / synth.F_SOURCE
    nx = int(round(lam_interior * ppw))
    nx += nx % 2 == 0          # odd: the source sits on the centre node
    p = int(round(lam_pml * ppw))
    N = nx + 2 * p
    c = np.full((N, N), synth.C_WATER)
    A = hz.assemble(c, p, h, OMEGA)
    b = np.zeros((N, N), complex)
    mid = N // 2
    b[mid, mid] = 1.0 / h ** 2             # discrete delta
    u = hz.solve_direct(A, b.ravel()).reshape(N, N)
    yy, xx = np.mgrid[0:N, 0:N]
    r = np.hypot(xx - mid, yy - mid) * h
    ring = (r >= 1.0 * lam) & (r <= 2.0 * lam)
    G = hz.greens_function(OMEGA / synth.C_WATER, r[ring])
    return np.abs(u[ring] - G).max() / np.abs(G).max()


@pytest.mark.slow
def test_greens_function_second_order_convergence():
    """(i/4) H0^(1)(k r) is the outgoing solution of -Lap u - k^2 u = delta (eq. 1 with the
    Sommerfeld condition).  On a fixed annulus 1-2 wavelengths from the source the
    error of the discrete solution must fall at second order in h."""
    e = [_greens_error(ppw) for ppw in (10.0, 20.0, 40.0)]
    orders = [np.log2(e[i] / e[i + 1]) for i in range(2)]
    assert all(1.7 <= o <= 2.4 for o in orders), (e, orders)
    assert e[-1] < 0.05, e


def _manufactured_error(cells_per_unit):
    """u* = (1+0.5i) q^6, q = 1 - r^2/R^2 on r < R, in a smooth heterogeneous medium."""
    lam = synth.C_WATER / synth.F_SOURCE
    L = 3.0 * lam                        # interior side length
    nx = int(round(3.0 * cells_per_unit))
    h = L / nx
    p = cells_per_unit                   # one wavelength of PML at every resolution
    N = nx + 2 * p
    yy, xx = np.mgrid[0:N, 0:N].astype(float)
    X = (xx - (N - 1) / 2.0) * h
    Y = (yy - (N - 1) / 2.0) * h
    R = 1.2 * lam
    c = 1500.0 + 600.0 * np.exp(-((X - 0.3 * lam) ** 2 + Y ** 2) / (0.8 * lam) ** 2)
    rr2 = X ** 2 + Y ** 2
    q = np.clip(1.0 - rr2 / R ** 2, 0.0, None)
    amp = 1.0 + 0.5j
    u_star = amp * q ** 6
    lap = amp * (-24.0 * q ** 5 / R ** 2 + 120.0 * rr2 * q ** 4 / R ** 4)
    f = -lap - (OMEGA / c) ** 2 * u_star
    A = hz.assemble(c, p, h, OMEGA)
    u = hz.solve_direct(A, f.ravel()).reshape(N, N)
    return np.abs(u - u_star).max() / np.abs(u_star).max()


@pytest.mark.slow
def test_manufactured_solution_second_order():
    e = [_manufactured_error(k) for k in (20, 40, 80)]
    orders = [np.log2(e[i] / e[i + 1]) for i in range(2)]
    assert all(1.8 <= o <= 2.2 for o in orders), (e, orders)


def test_pml_absorbs_outgoing_waves():
    """Enlarging the interior (same PML) barely changes the solution on the common region.

    A PML with the wrong sign of sigma, or none, reflects O(1) energy back."""
    ppw = 10.0
    h = synth.grid_spacing(ppw)
    sols = []
    for extra in (0, 20):
        nx, p = 41 + 2 * extra, 16
        N = nx + 2 * p
        c = np.full((N, N), synth.C_WATER)
        b = np.zeros((N, N), complex)
        b[N // 2, N // 2] = 1.0
        u = hz.solve_direct(hz.assemble(c, p, h, OMEGA), b.ravel()).reshape(N, N)
        m = N // 2
        sols.append(u[m - 20:m + 21, m - 20:m + 21])
    d = np.abs(sols[0] - sols[1]).max() / np.abs(sols[1]).max()
    assert d < 2e-3, d
    # with sigma = 0 the Dirichlet walls reflect everything: the same comparison changes at O(1)
    sols0 = []
    for extra in (0, 20):
        nx, p = 41 + 2 * extra, 16
        N = nx + 2 * p
        c = np.full((N, N), synth.C_WATER)
        b = np.zeros((N, N), complex)
        b[N // 2, N // 2] = 1.0
        u = hz.solve_direct(hz.assemble(c, p, h, OMEGA, sigma_max=0.0), b.ravel()).reshape(N, N)
        m = N // 2
        sols0.append(u[m - 20:m + 21, m - 20:m + 21])
    d0 = np.abs(sols0[0] - sols0[1]).max() / np.abs(sols0[1]).max()
    assert d0 > 100 * d
