"""Pins of the Fourier-differentiation operator oracle (Sec. 2.1, Tab. 1; reading in oracle/fourier.py)."""
import numpy as np

from oracle import fourier as fo
from oracle import helmholtz as hz
from paper_2607_16906_b300 import synth

OMEGA = synth.angular_frequency()


def test_fourier_mode_is_an_eigenvector_without_pml():
    """sigma = 0 (no PML), constant c: u = exp(i (kx x + ky y)) with grid wavenumbers gives
    A_F u = (kx^2 + ky^2 - k^2) u exactly."""
    Nx, Ny, h = 32, 24, synth.grid_spacing(10.0)
    c = np.full((Ny, Nx), 1700.0)
    k2 = (OMEGA / 1700.0) ** 2
    for a, b in ((1, 0), (3, -2), (-7, 5), (15, 11)):
        kx, ky = 2 * np.pi * a / (Nx * h), 2 * np.pi * b / (Ny * h)
        jj, ii = np.mgrid[0:Ny, 0:Nx]
        u = np.exp(1j * (kx * ii * h + ky * jj * h))
        got = fo.apply(u, c, 0, h, OMEGA)
        assert np.abs(got - (kx * kx + ky * ky - k2) * u).max() <= 1e-12 * (kx * kx + ky * ky + k2)


def _dft_derivative_matrix(N, h):
    """D = F^-1 diag(i kappa) F from the DFT's definition F_jq = exp(-2 pi i j q / N) (no FFT),
    with the Nyquist multiplier 0 for even N."""
    j = np.arange(N)
    F = np.exp(-2j * np.pi * np.outer(j, j) / N)
    Finv = np.conj(F) / N
    q = np.where(j < (N + 1) // 2, j, j - N).astype(float)
    kap = 2 * np.pi * q / (N * h)
    if N % 2 == 0:
        kap[N // 2] = 0.0
    return Finv @ np.diag(1j * kap) @ F


def test_operator_equals_dense_assembly_from_the_dft_definition():
    rng = synth.rng_for(3)
    for nx, ny, p in ((6, 4, 2), (7, 6, 1)):               # even and odd grid sizes
        c = synth.skull_velocity(nx, ny, p, rng, thickness=(1, 1))
        h = synth.grid_spacing(6.0)
        Ny, Nx = c.shape
        k2, sx, _, sy, _ = hz.coefficients(c, p, h, OMEGA)
        Dx, Dy = _dft_derivative_matrix(Nx, h), _dft_derivative_matrix(Ny, h)
        Ix, Iy = np.eye(Nx), np.eye(Ny)
        Sx, Sy = np.diag(1 / sx), np.diag(1 / sy)
        # row-major [Ny][Nx] flattening: x acts on the fast index
        Ax = np.kron(Iy, Sx @ Dx @ Sx @ Dx)
        Ay = np.kron(Sy @ Dy @ Sy @ Dy, Ix)
        A = -(Ax + Ay) - np.diag(k2.ravel())
        u = rng.standard_normal((Ny, Nx)) + 1j * rng.standard_normal((Ny, Nx))
        got = fo.apply(u, c, p, h, OMEGA).ravel()
        ref = A @ u.ravel()
        assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max()


def test_agrees_with_the_five_point_operator_to_second_order():
    """On a smooth field compactly supported in the interior (where s = 1), the 5-point operator
    differs from the spectral one by its O(h^2) truncation error: halving h divides the gap by 4."""
    errs = []
    for n in (32, 64, 128):
        p = n // 8
        L = 1.0e-2
        h = L / n
        N = n + 2 * p
        c = np.full((N, N), 1500.0)
        x = (np.arange(N) - (N - 1) / 2) * h
        X, Y = np.meshgrid(x, x)
        r2 = (X ** 2 + Y ** 2) / (0.3 * L) ** 2
        u = np.where(r2 < 1, (1 - r2) ** 6, 0.0) * np.exp(1j * 300 * X)
        a5 = hz.apply(u, c, p, h, OMEGA)
        af = fo.apply(u, c, p, h, OMEGA)
        errs.append(np.abs(a5 - af).max() / np.abs(af).max())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert (np.abs(rates - 2.0) < 0.3).all(), (errs, rates)
