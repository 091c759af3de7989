"""Pins of the oracle for the paper's U-Net variant (Sec. 3.1, Tab. 2): each op and the whole
forward against torch.nn.functional in FP64 on the CPU (a library cross-check of the oracle's own
loops), shapes and the parameter count."""
import numpy as np
import torch
import torch.nn.functional as F

from oracle import helmholtz as hz
from oracle import unet_paper as up
from paper_2607_16906_b300 import synth


def _theta(seed=5):
    return up.init_params(synth.kaiming_uniform_params(up.param_segments(), seed))


def test_parameter_count_and_layout():
    assert up.param_count() == 665930
    P = up.unpack(_theta())
    assert P["enc1"][0].shape == (32, 5, 8, 8) and P["dec2"][0].shape == (64, 32, 8, 8)
    assert P["out"][0].shape == (2, 32, 1, 1) and P["out"][2] is None
    assert all(P[n][2] == 0.25 for n in ("enc1", "enc4", "dec0"))


def test_strided_conv_and_transposed_conv_equal_torch():
    rng = synth.rng_for(2)
    x = rng.standard_normal((2, 6, 16, 24))
    W = rng.standard_normal((7, 6, 8, 8))
    b = rng.standard_normal(7)
    ref = F.conv2d(torch.tensor(x), torch.tensor(W), torch.tensor(b), stride=2, padding=3).numpy()
    got = up.conv_down(x, W, b)
    assert got.shape == (2, 7, 8, 12) and np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    Wt = rng.standard_normal((6, 5, 8, 8))
    bt = rng.standard_normal(5)
    ref = F.conv_transpose2d(torch.tensor(x), torch.tensor(Wt), torch.tensor(bt), stride=2, padding=3).numpy()
    got = up.conv_up(x, Wt, bt)
    assert got.shape == (2, 5, 32, 48) and np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    a = 0.3
    assert np.allclose(up.prelu(x, a), F.prelu(torch.tensor(x), torch.tensor([a], dtype=torch.float64)).numpy())


def test_forward_equals_a_torch_composition():
    theta = _theta(7)
    rng = synth.rng_for(3)
    x = rng.standard_normal((2, 5, 32, 48))
    P = {k: tuple(torch.tensor(np.asarray(v)) if v is not None else None for v in t)
         for k, t in up.unpack(theta).items()}
    t = torch.tensor(x)

    def act(y, a):
        return F.prelu(y, a.reshape(1))

    e = []
    h = t
    for n in ("enc1", "enc2", "enc3", "enc4"):
        W, b, a = P[n]
        h = act(F.conv2d(h, W, b, stride=2, padding=3), a)
        e.append(h)
    W, b, a = P["dec3"]
    h = act(F.conv_transpose2d(e[3], W, b, stride=2, padding=3), a)
    for n, skip in (("dec2", e[2]), ("dec1", e[1]), ("dec0", e[0])):
        W, b, a = P[n]
        h = act(F.conv_transpose2d(torch.cat([h, skip], 1), W, b, stride=2, padding=3), a)
    W, b, _ = P["out"]
    ref = F.conv2d(h, W, b).numpy()
    got = up.forward(theta, x)
    assert got.shape == (2, 2, 32, 48)
    assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max()


def test_network_input_channels():
    rng = synth.rng_for(4)
    nx, p = 20, 6
    c = synth.skull_velocity(nx, nx, p, rng, thickness=(2, 3))
    h, om = synth.grid_spacing(10.0), synth.angular_frequency()
    v = rng.standard_normal((1, 32, 32)) + 1j * rng.standard_normal((1, 32, 32))
    x = up.network_input(v, c, p, h, om)
    assert x.shape == (1, 5, 32, 32)
    _, sx, _, sy, _ = hz.coefficients(c, p, h, om)
    assert np.allclose(x[0, 3] + 1j * x[0, 4], np.outer(sy, sx) - 1)
    assert (x[0, 3:, p:p + nx, p:p + nx] == 0).all()          # no PML field in the interior
    assert np.allclose(x[0, 2], c / 1500.0)


def test_backward_equals_torch_autograd_and_central_differences():
    theta = _theta(9)
    rng = synth.rng_for(10)
    x = rng.standard_normal((2, 5, 32, 32))
    gy = rng.standard_normal((2, 2, 32, 32))
    y, act = up.forward(theta, x, keep=True)
    g = up.backward(theta, act, gy)
    # torch autograd on the same composition
    th = torch.tensor(theta, requires_grad=True)
    off, P = 0, {}
    for name, kind, ci, co in up.LAYERS:
        shp = up._wshape(kind, ci, co)
        nw = int(np.prod(shp))
        W = th[off:off + nw].reshape(shp)
        off += nw
        b = th[off:off + co]
        off += co
        a = None
        if kind != "conv1":
            a = th[off:off + 1]
            off += 1
        P[name] = (W, b, a)
    t = torch.tensor(x)
    e = []
    h = t
    for n in ("enc1", "enc2", "enc3", "enc4"):
        W, b, a = P[n]
        h = F.prelu(F.conv2d(h, W, b, stride=2, padding=3), a)
        e.append(h)
    W, b, a = P["dec3"]
    h = F.prelu(F.conv_transpose2d(e[3], W, b, stride=2, padding=3), a)
    for n, skip in (("dec2", e[2]), ("dec1", e[1]), ("dec0", e[0])):
        W, b, a = P[n]
        h = F.prelu(F.conv_transpose2d(torch.cat([h, skip], 1), W, b, stride=2, padding=3), a)
    W, b, _ = P["out"]
    out = F.conv2d(h, W, b)
    (out * torch.tensor(gy)).sum().backward()
    ref = th.grad.numpy()
    assert np.abs(g - ref).max() <= 1e-10 * np.abs(ref).max()
    # central differences along a random unit direction (a short step, so that no pre-activation
    # crosses the PReLU kink between the two evaluations)
    d = rng.standard_normal(theta.size)
    d /= np.linalg.norm(d)
    eps = 1e-7
    fp = (up.forward(theta + eps * d, x) * gy).sum()
    fm = (up.forward(theta - eps * d, x) * gy).sum()
    assert abs((fp - fm) / (2 * eps) - g @ d) <= 1e-5 * abs(g @ d)
