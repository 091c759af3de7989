"""Oracle: the discrete Helmholtz operator with PML (test infrastructure only).

Problem (eq. 1, with the sign flipped to -Lap u - k^2 u = f, k = omega / c):
the unbounded domain is truncated to the grid and surrounded by a PML whose
damping follows eq. 2 (quadratic in the depth into the layer).

Reading of the PML (the paper gives sigma only): complex coordinate
stretching d/dx -> (1/s_x) d/dx with s_x = 1 + i sigma_x / omega.  Multiplying
the stretched equation by s_x s_y gives the complex-symmetric form

  (A u)_{j,i} = -[ a_{i+1/2}(u_{i+1} - u_i) - a_{i-1/2}(u_i - u_{i-1})
                 + b_{j+1/2}(u_{j+1} - u_j) - b_{j-1/2}(u_j - u_{j-1}) ] / h^2
                - s_x(i) s_y(j) k^2_{j,i} u_{j,i},
  a_{i+1/2} = s_y(j) / s_x(i+1/2),   b_{j+1/2} = s_x(i) / s_y(j+1/2),

with homogeneous Dirichlet ghost values outside the grid (i = x index,
j = y index, arrays row-major [Ny][Nx]).  sigma_max defaults to 2 omega, the
paper's value at omega = 1 (Tab. 1).  sigma is sampled at the node or
half-node position; depth d is measured from the interior edge; ell = p h.

Pins (tests/test_oracle_helmholtz.py):
  assemble        A == A^T exactly; matrix-free stencil == CSR matvec; sigma = 0
                  gives a real symmetric matrix; Green's function (i/4) H0(kr)
                  converges at second order in h; manufactured solution with
                  observed order 2; PML reflection bound by domain enlargement.
  apply_adjoint   dot-product test <Ax, y> == <x, A^H y>; equals conj-transpose CSR.
  solve_direct    dense numpy.linalg.solve on a 16x16 (+4 PML) grid.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla
from scipy import special


def _depth(t, nx_int, p, h):
    """Distance (m) of grid position t (in cells, may be half-integer) into the PML."""
    t = np.asarray(t, dtype=np.float64)
    d = np.maximum(0.0, np.maximum(p - t, t - (p + nx_int - 1)))
    return d * h


def sigma_profile(t, nx_int, p, h, sigma_max):
    """Eq. 2: sigma = sigma_max (d / ell)^2 inside the PML, 0 in the interior."""
    if p == 0:
        return np.zeros_like(np.asarray(t, dtype=np.float64))
    ell = p * h
    d = _depth(t, nx_int, p, h)
    return sigma_max * (d / ell) ** 2


def stretch(t, nx_int, p, h, omega, sigma_max):
    """s = 1 + i sigma / omega at positions t."""
    return 1.0 + 1j * sigma_profile(t, nx_int, p, h, sigma_max) / omega


def coefficients(c, p, h, omega, sigma_max=None):
    """Return (k2 [Ny][Nx], sx node [Nx], sx half [Nx+1], sy node [Ny], sy half [Ny+1]).

    Half arrays hold the values at positions -1/2, 1/2, ..., N - 1/2.
    """
    if sigma_max is None:
        sigma_max = 2.0 * omega
    Ny, Nx = c.shape
    nx, ny = Nx - 2 * p, Ny - 2 * p
    k2 = (omega / np.asarray(c, np.float64)) ** 2
    sx = stretch(np.arange(Nx), nx, p, h, omega, sigma_max)
    sxh = stretch(np.arange(Nx + 1) - 0.5, nx, p, h, omega, sigma_max)
    sy = stretch(np.arange(Ny), ny, p, h, omega, sigma_max)
    syh = stretch(np.arange(Ny + 1) - 0.5, ny, p, h, omega, sigma_max)
    return k2, sx, sxh, sy, syh


def assemble(c, p, h, omega, sigma_max=None) -> sp.csr_matrix:
    """The n x n complex matrix A (n = Nx Ny, row index j*Nx + i) as CSR."""
    k2, sx, sxh, sy, syh = coefficients(c, p, h, omega, sigma_max)
    Ny, Nx = c.shape
    jj, ii = np.meshgrid(np.arange(Ny), np.arange(Nx), indexing="ij")
    row = (jj * Nx + ii).ravel()
    sxi = sx[ii].ravel()
    syj = sy[jj].ravel()
    aE = (syj / sxh[ii.ravel() + 1]) / h ** 2        # a_{i+1/2} / h^2
    aW = (syj / sxh[ii.ravel()]) / h ** 2            # a_{i-1/2} / h^2
    bN = (sxi / syh[jj.ravel() + 1]) / h ** 2        # b_{j+1/2} / h^2
    bS = (sxi / syh[jj.ravel()]) / h ** 2            # b_{j-1/2} / h^2
    diag = aE + aW + bN + bS - sxi * syj * k2.ravel()
    rows, cols, vals = [row], [row], [diag]
    iv, jv = ii.ravel(), jj.ravel()
    for mask, off, coef in ((iv + 1 < Nx, 1, aE), (iv - 1 >= 0, -1, aW),
                            (jv + 1 < Ny, Nx, bN), (jv - 1 >= 0, -Nx, bS)):
        rows.append(row[mask])
        cols.append(row[mask] + off)
        vals.append(-coef[mask])
    n = Nx * Ny
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n)).tocsr()
    return A


def apply(u, c, p, h, omega, sigma_max=None):
    """Matrix-free A u for u of shape [..., Ny, Nx] (plain numpy slicing)."""
    k2, sx, sxh, sy, syh = coefficients(c, p, h, omega, sigma_max)
    u = np.asarray(u, np.complex128)
    Ny, Nx = c.shape
    up = np.zeros(u.shape[:-2] + (Ny + 2, Nx + 2), np.complex128)
    up[..., 1:-1, 1:-1] = u
    uc = up[..., 1:-1, 1:-1]
    ue, uw = up[..., 1:-1, 2:], up[..., 1:-1, :-2]
    un, us = up[..., 2:, 1:-1], up[..., :-2, 1:-1]
    SX = sx[None, :]
    SY = sy[:, None]
    flux_x = SY * ((ue - uc) / sxh[None, 1:] - (uc - uw) / sxh[None, :-1])
    flux_y = SX * ((un - uc) / syh[1:, None] - (uc - us) / syh[:-1, None])
    return -(flux_x + flux_y) / h ** 2 - SX * SY * k2 * uc


def apply_adjoint(u, c, p, h, omega, sigma_max=None):
    """A^H u.  Since A = A^T, A^H u = conj(A conj(u))."""
    return np.conj(apply(np.conj(u), c, p, h, omega, sigma_max))


def solve_direct(A: sp.spmatrix, b: np.ndarray) -> np.ndarray:
    """Sparse direct LU (scipy SuperLU) solve of A x = b for b of shape [n] or [n, k]."""
    lu = spla.splu(A.tocsc())
    return lu.solve(np.asarray(b, np.complex128))


def relres(A, x, b):
    """Backward error eta_b = ||A x - b|| / ||b|| (eq. 10)."""
    return np.linalg.norm(A @ x - b) / np.linalg.norm(b)


def greens_function(k, r):
    """Outgoing free-space Green's function of -Lap - k^2 in 2D: (i/4) H0^(1)(k r)."""
    return 0.25j * special.hankel1(0, k * r)
