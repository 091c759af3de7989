"""Oracle: the Fourier-differentiation Helmholtz operator with a PML (test infrastructure only).

The paper discretises the derivatives of eq. 1 by Fourier differentiation on the N x N grid that
includes the PML (Sec. 2.1; Tab. 1: FFT on the last two axes), with the damping sigma of eq. 2.
Reading used here (the paper gives no formula for the stretched operator):

    A_F u = -[ (1/s_x) D_x((1/s_x) D_x u) + (1/s_y) D_y((1/s_y) D_y u) ] - k^2 u,
    s_x(i) = 1 + i sigma_x(i) / omega  (sigma of eq. 2 at node i, as in oracle.helmholtz),
    D_x u = IDFT_x( i kappa DFT_x(u) ),  kappa_q = 2 pi q / (N_x h), q in [-N_x/2, N_x/2),

with the Nyquist mode (q = -N_x/2 for even N_x) of each first derivative set to zero, so that D_x
maps real grids to real grids.  The sign follows the rest of the repository (A = -(Lap + k^2)).  The
grid is periodic, as Fourier differentiation makes it; the PML absorbs what reaches it.

Each step is numpy.fft (a library primitive) applied along one axis.

Pins (tests/test_oracle_fourier.py): without a PML, a Fourier mode is an eigenvector with eigenvalue
kappa_x^2 + kappa_y^2 - k^2 exactly; the operator equals a dense matrix assembled from the DFT's
definition (F_jq = exp(-2 pi i j q / N), no FFT) at small N; on smooth fields it agrees with the
5-point operator of oracle.helmholtz to the latter's O(h^2).
"""
from __future__ import annotations

import numpy as np

from . import helmholtz as hz


def wavenumbers(N: int, h: float) -> np.ndarray:
    """kappa_q = 2 pi q / (N h) in numpy's FFT order, with the Nyquist entry set to 0."""
    q = np.fft.fftfreq(N, d=1.0) * N                 # integers in FFT order
    kap = 2.0 * np.pi * q / (N * h)
    if N % 2 == 0:
        kap[N // 2] = 0.0
    return kap


def derivative(u: np.ndarray, axis: int, h: float) -> np.ndarray:
    """Spectral first derivative of the grid u along `axis` (periodic)."""
    N = u.shape[axis]
    shape = [1] * u.ndim
    shape[axis] = N
    kap = wavenumbers(N, h).reshape(shape)
    return np.fft.ifft(1j * kap * np.fft.fft(u, axis=axis), axis=axis)


def apply(u: np.ndarray, c: np.ndarray, p: int, h: float, omega: float, sigma_max=None) -> np.ndarray:
    """A_F u for u complex [Ny][Nx] (or [..., Ny, Nx]), c [Ny][Nx] in m/s (same units as h, omega).
    The node stretch factors s(i) and k^2 are those of oracle.helmholtz (eq. 2, sigma_max = 2 omega
    by default)."""
    k2, sx, _, sy, _ = hz.coefficients(c, p, h, omega, sigma_max)
    sx = sx[None, :]
    sy = sy[:, None]
    u = np.asarray(u, np.complex128)
    tx = derivative(derivative(u, -1, h) / sx, -1, h) / sx
    ty = derivative(derivative(u, -2, h) / sy, -2, h) / sy
    return -(tx + ty) - k2 * u
