"""Pins of the oracle's U-Net against torch.nn.functional (a library cross-check in FP64 on the CPU)
and against finite differences.  A transposed weight index, a wrong concat order, a wrong
pooling window or a missed ReLU mask fails one of these."""
import numpy as np
import pytest
import torch
import torch.nn.functional as F

from oracle import unet
from paper_2607_16906_b300 import synth


def _theta(seed=42):
    return synth.kaiming_uniform_params(unet.param_segments(), seed)


def test_parameter_count_closed_form():
    # 16/32/64/128 channels, two 3x3 convs per level, 2x2 up-convs, 1x1 head:
    # 482,050 parameters (3x3: 9 ci co + co each; up: 4 ci co + co; head 16*2 + 2).
    assert unet.param_count() == 482050
    assert _theta().size == 482050


def test_bf16_round_matches_torch():
    rng = synth.rng_for(1)
    x = np.concatenate([rng.standard_normal(10000) * 10 ** rng.uniform(-5, 5, 10000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.01171875, 3.0e38, 1e-40]])
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(unet.bf16_round(x), ref)


def test_primitive_ops_match_torch():
    rng = synth.rng_for(2)
    x = rng.standard_normal((2, 5, 8, 12))
    W = rng.standard_normal((7, 5, 3, 3))
    b = rng.standard_normal(7)
    ref = F.conv2d(torch.tensor(x), torch.tensor(W), torch.tensor(b), padding=1).numpy()
    assert np.abs(unet.conv2d(x, W, b, 1) - ref).max() <= 1e-13
    Wt = rng.standard_normal((5, 3, 2, 2))
    bt = rng.standard_normal(3)
    ref = F.conv_transpose2d(torch.tensor(x), torch.tensor(Wt), torch.tensor(bt), stride=2).numpy()
    assert np.abs(unet.conv_transpose2x2(x, Wt, bt) - ref).max() <= 1e-13
    ref = F.max_pool2d(torch.tensor(x), 2).numpy()
    assert np.array_equal(unet.maxpool2(x)[0], ref)


def _torch_unet(theta, x):
    P = {k: (torch.tensor(np.ascontiguousarray(W)), torch.tensor(np.ascontiguousarray(b)))
         for k, (W, b) in unet.unpack(theta).items()}

    def c(name, t, act=True, pad=1):
        y = F.conv2d(t, *P[name], padding=pad)
        return F.relu(y) if act else y

    def up(name, t):
        return F.conv_transpose2d(t, *P[name], stride=2)

    s1 = c("enc1b", c("enc1a", x))
    s2 = c("enc2b", c("enc2a", F.max_pool2d(s1, 2)))
    s3 = c("enc3b", c("enc3a", F.max_pool2d(s2, 2)))
    h = c("botb", c("bota", F.max_pool2d(s3, 2)))
    h = c("dec3b", c("dec3a", torch.cat([s3, up("up3", h)], 1)))
    h = c("dec2b", c("dec2a", torch.cat([s2, up("up2", h)], 1)))
    h = c("dec1b", c("dec1a", torch.cat([s1, up("up1", h)], 1)))
    return c("final", h, act=False, pad=0)


def test_forward_matches_torch_composition():
    theta = _theta()
    rng = synth.rng_for(3)
    x = rng.standard_normal((2, 3, 24, 16))
    ref = _torch_unet(theta, torch.tensor(x)).numpy()
    got = unet.forward(theta, x)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_backward_matches_torch_autograd():
    theta = _theta()
    rng = synth.rng_for(4)
    x = rng.standard_normal((2, 3, 16, 16))
    gy = rng.standard_normal((2, 2, 16, 16))
    tt = torch.tensor(theta, requires_grad=True)
    xt = torch.tensor(x, requires_grad=True)
    # rebuild the torch net from the differentiable flat vector
    parts, off = {}, 0
    for name, kind, ci, co in unet.LAYERS:
        shp = unet._wshape(kind, ci, co)
        nw = int(np.prod(shp))
        parts[name] = (tt[off:off + nw].reshape(shp), tt[off + nw:off + nw + co])
        off += nw + co

    def c(name, t, act=True, pad=1):
        y = F.conv2d(t, *parts[name], padding=pad)
        return F.relu(y) if act else y

    def up(name, t):
        return F.conv_transpose2d(t, *parts[name], stride=2)

    s1 = c("enc1b", c("enc1a", xt))
    s2 = c("enc2b", c("enc2a", F.max_pool2d(s1, 2)))
    s3 = c("enc3b", c("enc3a", F.max_pool2d(s2, 2)))
    h = c("botb", c("bota", F.max_pool2d(s3, 2)))
    h = c("dec3b", c("dec3a", torch.cat([s3, up("up3", h)], 1)))
    h = c("dec2b", c("dec2a", torch.cat([s2, up("up2", h)], 1)))
    h = c("dec1b", c("dec1a", torch.cat([s1, up("up1", h)], 1)))
    y = c("final", h, act=False, pad=0)
    (y * torch.tensor(gy)).sum().backward()
    _, act = unet.forward(theta, x, keep=True)
    gtheta, gx = unet.backward(theta, act, gy)
    assert np.abs(gtheta - tt.grad.numpy()).max() <= 1e-11 * np.abs(tt.grad.numpy()).max()
    assert np.abs(gx - xt.grad.numpy()).max() <= 1e-11 * np.abs(xt.grad.numpy()).max()


def test_backward_matches_central_difference():
    theta = _theta()
    rng = synth.rng_for(5)
    x = rng.standard_normal((1, 3, 16, 16))
    gy = rng.standard_normal((1, 2, 16, 16))
    _, act = unet.forward(theta, x, keep=True)
    gtheta, _ = unet.backward(theta, act, gy)
    for k in range(3):
        d = rng.standard_normal(theta.size)
        eps = 1e-8           # small enough that no ReLU kink or pooling switch is crossed
        fp = np.sum(unet.forward(theta + eps * d, x) * gy)
        fm = np.sum(unet.forward(theta - eps * d, x) * gy)
        fd = (fp - fm) / (2 * eps)
        assert abs(fd - gtheta @ d) <= 1e-6 * abs(fd), (fd, gtheta @ d)


def test_precondition_pads_to_multiple_of_8_and_is_scale_invariant():
    theta = _theta()
    rng = synth.rng_for(6)
    v = rng.standard_normal((2, 13, 21)) + 1j * rng.standard_normal((2, 13, 21))
    c = 1500.0 + 100 * rng.standard_normal((13, 21))
    z = unet.precondition(theta, v, c, 0.5)
    assert z.shape == v.shape
    z2 = unet.precondition(theta, 3.7 * v, c, 0.5)
    assert np.abs(z2 - 3.7 * z).max() <= 1e-12 * np.abs(z2).max()
    # manual padding reference: zero-pad to 16 x 24, run the network, crop
    a = np.sqrt(13 * 21) / np.linalg.norm(v[0])
    x = np.zeros((1, 3, 16, 24))
    x[0, 0, :13, :21] = (a * v[0]).real
    x[0, 1, :13, :21] = (a * v[0]).imag
    x[0, 2, :13, :21] = c / 1500.0
    y = unet.forward(theta, x)[0, :, :13, :21]
    assert np.abs(0.25 * (y[0] + 1j * y[1]) / a - z[0]).max() <= 1e-12 * np.abs(z[0]).max()
