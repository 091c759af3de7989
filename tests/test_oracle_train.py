"""Pins of the oracle's physics-informed loss (eqs. 8-9), its gradient and AdamW."""
import numpy as np
import torch
import torch.nn.functional as F

from oracle import helmholtz as hz
from oracle import train, unet
from paper_2607_16906_b300 import synth

OMEGA = synth.angular_frequency()


def _batch(B=2, nx=8, p=4, seed=21):
    rng = synth.rng_for(seed)
    c = np.stack([synth.skull_velocity(nx, nx, p, rng, thickness=(1, 2)) for _ in range(B)])
    b = np.stack([synth.point_sources(nx, nx, p, rng, 2) for _ in range(B)])
    return c, b, p, synth.grid_spacing(10.0)


def test_loss_is_squared_backward_error():
    """eq. 9: L = eta_b(u_hat)^2, computed independently from the CSR matrix."""
    theta = synth.kaiming_uniform_params(unet.param_segments(), 42)
    c, b, p, h = _batch()
    L, _, per = train.loss_and_grad(theta, b, c, p, h, OMEGA, want_grad=False)
    for s in range(b.shape[0]):
        u = unet.precondition(theta, b[s:s + 1], c[s], h)[0]
        A = hz.assemble(c[s], p, h, OMEGA)
        eta = hz.relres(A, u.ravel(), b[s].ravel())
        assert abs(per[s] - eta ** 2) <= 1e-12 * eta ** 2
    assert abs(L - per.mean()) <= 1e-15 * L


def test_gradient_central_difference():
    theta = synth.kaiming_uniform_params(unet.param_segments(), 42)
    c, b, p, h = _batch()
    L, g, _ = train.loss_and_grad(theta, b, c, p, h, OMEGA)
    rng = synth.rng_for(8)
    for _ in range(3):
        d = rng.standard_normal(theta.size)
        eps = 1e-8           # small enough that no ReLU kink is crossed in 482k directions
        Lp = train.loss_and_grad(theta + eps * d, b, c, p, h, OMEGA, want_grad=False)[0]
        Lm = train.loss_and_grad(theta - eps * d, b, c, p, h, OMEGA, want_grad=False)[0]
        fd = (Lp - Lm) / (2 * eps)
        assert abs(fd - g @ d) <= 1e-6 * abs(fd), (fd, g @ d)


def test_gradient_matches_torch_autograd_dense():
    theta = synth.kaiming_uniform_params(unet.param_segments(), 42)
    c, b, p, h = _batch()
    L, g, _ = train.loss_and_grad(theta, b, c, p, h, OMEGA)
    B, Ny, Nx = b.shape
    tt = torch.tensor(theta, requires_grad=True)
    parts, off = {}, 0
    for name, kind, ci, co in unet.LAYERS:
        shp = unet._wshape(kind, ci, co)
        nw = int(np.prod(shp))
        parts[name] = (tt[off:off + nw].reshape(shp), tt[off + nw:off + nw + co])
        off += nw + co

    def cv(name, t, act=True, pad=1):
        y = F.conv2d(t, *parts[name], padding=pad)
        return F.relu(y) if act else y

    def up(name, t):
        return F.conv_transpose2d(t, *parts[name], stride=2)

    total = 0
    for s in range(B):
        A = torch.tensor(hz.assemble(c[s], p, h, OMEGA).toarray())
        bs = torch.tensor(b[s].ravel())
        a = np.sqrt(Ny * Nx) / np.linalg.norm(b[s])
        x = np.zeros((1, 3, 16, 16))
        x[0, 0, :Ny, :Nx] = (a * b[s]).real
        x[0, 1, :Ny, :Nx] = (a * b[s]).imag
        x[0, 2, :Ny, :Nx] = c[s] / 1500.0
        xt = torch.tensor(x)
        s1 = cv("enc1b", cv("enc1a", xt))
        s2 = cv("enc2b", cv("enc2a", F.max_pool2d(s1, 2)))
        s3 = cv("enc3b", cv("enc3a", F.max_pool2d(s2, 2)))
        hh = cv("botb", cv("bota", F.max_pool2d(s3, 2)))
        hh = cv("dec3b", cv("dec3a", torch.cat([s3, up("up3", hh)], 1)))
        hh = cv("dec2b", cv("dec2a", torch.cat([s2, up("up2", hh)], 1)))
        hh = cv("dec1b", cv("dec1a", torch.cat([s1, up("up1", hh)], 1)))
        y = cv("final", hh, act=False, pad=0)[0, :, :Ny, :Nx]
        u = torch.complex(y[0], y[1]).reshape(-1) * (h * h / a)
        r = bs - A @ u
        total = total + (r.abs() ** 2).sum() / (bs.abs() ** 2).sum()
    (total / B).backward()
    assert abs(L - (total / B).item()) <= 1e-12 * L
    assert np.abs(g - tt.grad.numpy()).max() <= 1e-9 * np.abs(g).max()


def test_adamw_matches_torch():
    rng = synth.rng_for(4)
    theta = rng.standard_normal(50)
    m = np.zeros(50)
    v = np.zeros(50)
    p = torch.nn.Parameter(torch.tensor(theta.copy()))
    opt = torch.optim.AdamW([p], lr=1e-3, betas=(0.9, 0.999), eps=1e-8, weight_decay=0.01)
    for t in range(1, 6):
        g = rng.standard_normal(50)
        theta, m, v = train.adamw_step(theta, g, m, v, t, 1e-3, 0.01)
        p.grad = torch.tensor(g)
        opt.step()
        assert np.abs(theta - p.detach().numpy()).max() <= 1e-14


def test_clip_matches_torch():
    g = np.arange(10.0)
    gc, n = train.clip_by_global_norm(g, 1.0)
    p = torch.nn.Parameter(torch.zeros(10))
    p.grad = torch.tensor(g, dtype=torch.float64).float()
    tn = torch.nn.utils.clip_grad_norm_([p], 1.0)
    assert abs(n - tn.item()) <= 1e-5 * n
    assert np.abs(gc - p.grad.double().numpy()).max() <= 1e-6


def test_loss_gradient_of_the_paper_network_matches_central_differences():
    """Eq. 9 through network kind 1 (oracle.unet_paper): the gradient matches a central difference."""
    from oracle import unet_paper as upn
    rng = synth.rng_for(21)
    nx, p = 20, 6
    h, om = synth.grid_spacing(10.0), synth.angular_frequency()
    c = np.stack([synth.skull_velocity(nx, nx, p, rng, thickness=(2, 3)) for _ in range(2)])
    b = np.stack([synth.point_sources(nx, nx, p, rng, 2) for _ in range(2)])
    theta = upn.init_params(synth.kaiming_uniform_params(upn.param_segments(), 3))
    L, g, _ = train.loss_and_grad(theta, b, c, p, h, om, kind=1)
    d = rng.standard_normal(theta.size)
    d /= np.linalg.norm(d)
    eps = 1e-7
    Lp, _, _ = train.loss_and_grad(theta + eps * d, b, c, p, h, om, want_grad=False, kind=1)
    Lm, _, _ = train.loss_and_grad(theta - eps * d, b, c, p, h, om, want_grad=False, kind=1)
    assert abs((Lp - Lm) / (2 * eps) - g @ d) <= 1e-5 * abs(g @ d) + 1e-12
