"""Oracle: physics-informed loss, its gradient, and the AdamW update (test infrastructure only).

Loss (eq. 9): L(b, c) = ||b - A(c) u_hat||^2 / ||b||^2 with u_hat = N_theta(b, c),
i.e. the squared backward error eta_b(u_hat)^2.  Cost (eq. 8): the batch mean.
The network sees b scaled to unit RMS (alpha = sqrt(n) / ||b||) and its output is
scaled back by h^2 / alpha (the network approximates the inverse of the
dimensionless h^2 A, as oracle.unet.precondition does); the loss is invariant to alpha.

Gradient w.r.t. the network output channels (Re u, Im u):
  dL/d(Re u) + i dL/d(Im u) = -2 A^H r / ||b||^2,  r = b - A u_hat,
then back through the network (oracle.unet.backward).

Optimiser (Tab. 3 gives Adam, lr 1e-3 -> 1e-5, clip 1): the reading is AdamW
(decoupled weight decay, Loshchilov & Hutter) with beta = (0.9, 0.999),
eps = 1e-8, gradient clipped by its global L2 norm before the update.

Pins (tests/test_oracle_train.py): the gradient matches a central finite
difference of the loss in random parameter directions; it matches torch
autograd through torch.nn.functional ops and a sparse-matrix product in FP64;
the AdamW step matches torch.optim.AdamW on the same gradient.
"""
from __future__ import annotations

import numpy as np

from . import helmholtz as hz
from . import unet
from . import unet_paper


def loss_and_grad(theta, b, c, p, h, omega, bf16=False, want_grad=True, kind=0):
    """Mean over the batch of eq. 9, and its gradient w.r.t. theta.

    b: complex [B][Ny][Nx]; c: [B][Ny][Nx] velocity per sample.  kind 0: oracle.unet; kind 1: the
    paper's variant (oracle.unet_paper), whose input also carries the PML field.
    Returns (loss, grad or None, per-sample losses).
    """
    b = np.asarray(b, np.complex128)
    B, Ny, Nx = b.shape
    n = Ny * Nx
    nb = np.sqrt((np.abs(b) ** 2).reshape(B, -1).sum(1))
    alpha = np.sqrt(n) / nb
    bt = b * alpha[:, None, None]                       # unit-RMS source, ||bt||^2 = n
    if kind == 0:
        x = unet.network_input(bt, c)
        y, act = unet.forward(theta, x, bf16=bf16, keep=True)
    else:
        x = np.concatenate([unet_paper.network_input(bt[s:s + 1], c[s], p, h, omega) for s in range(B)])
        y, act = unet_paper.forward(theta, x, bf16=bf16, keep=True)
    u = (y[:, 0, :Ny, :Nx] + 1j * y[:, 1, :Ny, :Nx]) * h * h
    losses = np.zeros(B)
    gy = np.zeros_like(y)
    for s in range(B):
        r = bt[s] - hz.apply(u[s], c[s], p, h, omega)
        losses[s] = np.sum(np.abs(r) ** 2) / n
        if want_grad:
            g = -2.0 * h * h * hz.apply_adjoint(r, c[s], p, h, omega) / n / B
            gy[s, 0, :Ny, :Nx] = g.real
            gy[s, 1, :Ny, :Nx] = g.imag
    if not want_grad:
        return losses.mean(), None, losses
    gtheta = unet.backward(theta, act, gy)[0] if kind == 0 else unet_paper.backward(theta, act, gy)
    return losses.mean(), gtheta, losses


def clip_by_global_norm(g, max_norm):
    nrm = np.linalg.norm(g)
    if max_norm > 0 and nrm > max_norm:
        return g * (max_norm / (nrm + 1e-6)), nrm
    return g, nrm


def adamw_step(theta, g, m, v, t, lr, wd=0.01, beta1=0.9, beta2=0.999, eps=1e-8):
    """One AdamW step (t counts from 1).  Returns new (theta, m, v)."""
    theta = theta * (1.0 - lr * wd)
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v
