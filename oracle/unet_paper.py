"""Oracle: the paper's own U-Net variant (Sec. 3.1, Tab. 2), forward pass (test infrastructure only).

Tab. 2 fixes: 5 input channels, 2 output channels, PReLU, depth 4, 32 channels per layer and per
state, convolution kernel 8 / stride 2 / padding 3, batch normalisation, biases.  Fig. 2 (the
diagram) is missing, so the wiring below is this project's reading:

  inputs (Sec. 3.1): Re v, Im v, c / 1500 m/s, Re sigma_c, Im sigma_c with the complex PML field
      sigma_c = s_x(i) s_y(j) - 1 (zero in the interior; s = 1 + i sigma / omega, eq. 2);
  encoder: e_l = PReLU_l(conv_{8,2,3}(e_{l-1})), l = 1..4, channels 5 -> 32 -> 32 -> 32 -> 32
      (each halves the grid);
  decoder: d_3 = PReLU(convT_{8,2,3}(e_4)); d_2 = PReLU(convT(cat[d_3, e_3]));
      d_1 = PReLU(convT(cat[d_2, e_2])); d_0 = PReLU(convT(cat[d_1, e_1])) (each doubles the grid);
  output: 1x1 conv 32 -> 2 (Re z, Im z).
  Batch normalisation at inference is a per-channel affine map, folded here into the preceding
  convolution's weights and bias (no separate parameters).  PReLU has one slope per layer.
  The grid is zero-padded at the bottom/right to a multiple of 16 and cropped back.
  665,930 parameters (the paper quotes about 832 K for its wiring).

Parameter vector (flat float64): per layer weight, bias, PReLU slope (no slope for the output
layer); conv weights [C_out][C_in][8][8], transposed-conv weights [C_in][C_out][8][8]; layers
enc1 enc2 enc3 enc4 dec3 dec2 dec1 dec0 out.

Every convolution is the plain definition (sums over taps of a matmul); the forward is pinned
against torch.nn.functional and the backward (gradients of every weight, bias and PReLU slope)
against torch autograd and central differences in tests/test_oracle_unet_paper.py.
"""
from __future__ import annotations

import numpy as np

from . import helmholtz as hz
from .unet import bf16_round

K, S, P = 8, 2, 3
WIDTH = 32
C_REF = 1500.0
# (name, kind, c_in, c_out)
LAYERS = (
    ("enc1", "down", 5, WIDTH), ("enc2", "down", WIDTH, WIDTH), ("enc3", "down", WIDTH, WIDTH),
    ("enc4", "down", WIDTH, WIDTH),
    ("dec3", "up", WIDTH, WIDTH), ("dec2", "up", 2 * WIDTH, WIDTH), ("dec1", "up", 2 * WIDTH, WIDTH),
    ("dec0", "up", 2 * WIDTH, WIDTH),
    ("out", "conv1", WIDTH, 2),
)


def _wshape(kind, ci, co):
    return {"down": (co, ci, K, K), "up": (ci, co, K, K), "conv1": (co, ci, 1, 1)}[kind]


def param_segments():
    """(count, fan_in, kind) per tensor for the seeded generator; slopes use kind 's'."""
    seg = []
    for _, kind, ci, co in LAYERS:
        fan = ci * (K * K if kind != "conv1" else 1)
        seg.append((int(np.prod(_wshape(kind, ci, co))), fan, "w"))
        seg.append((co, fan, "b"))
        if kind != "conv1":
            seg.append((1, fan, "s"))
    return seg


def param_count():
    return sum(s[0] for s in param_segments())


def init_params(rng_params):
    """Kaiming-uniform weights and biases from the flat draw, PReLU slopes set to 0.25 (the usual
    initial slope)."""
    theta = np.array(rng_params, np.float64)
    off = 0
    for count, _, kind in param_segments():
        if kind == "s":
            theta[off:off + count] = 0.25
        off += count
    return theta


def unpack(theta):
    theta = np.asarray(theta, np.float64)
    out, off = {}, 0
    for name, kind, ci, co in LAYERS:
        shp = _wshape(kind, ci, co)
        nw = int(np.prod(shp))
        W = theta[off:off + nw].reshape(shp)
        off += nw
        b = theta[off:off + co]
        off += co
        a = None
        if kind != "conv1":
            a = theta[off]
            off += 1
        out[name] = (W, b, a)
    assert off == theta.size, (off, theta.size)
    return out


def conv_down(x, W, b):
    """y[n,o,i,j] = b[o] + sum_{c,ky,kx} W[o,c,ky,kx] x[n,c,2i+ky-3,2j+kx-3] (zero outside)."""
    N, C, H, Wd = x.shape
    Ho, Wo = (H + 2 * P - K) // S + 1, (Wd + 2 * P - K) // S + 1
    xp = np.zeros((N, C, H + 2 * P + 1, Wd + 2 * P + 1), np.result_type(x, W))
    xp[:, :, P:P + H, P:P + Wd] = x
    y = np.zeros((N, W.shape[0], Ho, Wo), np.result_type(x, W))
    for ky in range(K):
        for kx in range(K):
            patch = xp[:, :, ky:ky + S * Ho:S, kx:kx + S * Wo:S]
            y += np.einsum("oc,nchw->nohw", W[:, :, ky, kx], patch, optimize=True)
    return y + b[None, :, None, None]


def conv_up(x, W, b):
    """Transposed conv: y[n,o,2i+ky-3,2j+kx-3] += W[c,o,ky,kx] x[n,c,i,j], output 2H x 2W."""
    N, C, H, Wd = x.shape
    O = W.shape[1]
    Ho, Wo = (H - 1) * S - 2 * P + K, (Wd - 1) * S - 2 * P + K
    yp = np.zeros((N, O, Ho + 2 * P + 1, Wo + 2 * P + 1), np.result_type(x, W))
    for ky in range(K):
        for kx in range(K):
            contrib = np.einsum("co,nchw->nohw", W[:, :, ky, kx], x, optimize=True)
            yp[:, :, ky:ky + S * H:S, kx:kx + S * Wd:S] += contrib
    return yp[:, :, P:P + Ho, P:P + Wo] + b[None, :, None, None]


def prelu(x, a):
    return np.where(x > 0, x, a * x)


def conv_down_backward(x, W, g):
    """Gradients of conv_down w.r.t. x, W, b given g = dL/dy."""
    N, C, H, Wd = x.shape
    Ho, Wo = g.shape[2], g.shape[3]
    xp = np.zeros((N, C, H + 2 * P + 1, Wd + 2 * P + 1))
    xp[:, :, P:P + H, P:P + Wd] = x
    gxp = np.zeros_like(xp)
    gW = np.zeros_like(W)
    for ky in range(K):
        for kx in range(K):
            patch = xp[:, :, ky:ky + S * Ho:S, kx:kx + S * Wo:S]
            gW[:, :, ky, kx] = np.einsum("nohw,nchw->oc", g, patch, optimize=True)
            gxp[:, :, ky:ky + S * Ho:S, kx:kx + S * Wo:S] += np.einsum("oc,nohw->nchw", W[:, :, ky, kx], g,
                                                                      optimize=True)
    return gxp[:, :, P:P + H, P:P + Wd], gW, g.sum(axis=(0, 2, 3))


def conv_up_backward(x, W, g):
    """Gradients of conv_up w.r.t. x, W, b given g = dL/dy (y of size 2H x 2W)."""
    N, C, H, Wd = x.shape
    O = W.shape[1]
    gp = np.zeros((N, O, g.shape[2] + 2 * P + 1, g.shape[3] + 2 * P + 1))
    gp[:, :, P:P + g.shape[2], P:P + g.shape[3]] = g
    gx = np.zeros_like(x)
    gW = np.zeros_like(W)
    for ky in range(K):
        for kx in range(K):
            gs = gp[:, :, ky:ky + S * H:S, kx:kx + S * Wd:S]          # dL/d contrib[n,o,i,j]
            gW[:, :, ky, kx] = np.einsum("nchw,nohw->co", x, gs, optimize=True)
            gx += np.einsum("co,nohw->nchw", W[:, :, ky, kx], gs, optimize=True)
    return gx, gW, g.sum(axis=(0, 2, 3))


def forward(theta, x, bf16=False, keep=False):
    """x [N, 5, H, W] (H, W multiples of 16) -> [N, 2, H, W].  bf16: conv inputs and weights rounded
    to bfloat16 (FP64 accumulation), as the mixed path does.  keep: also return what backward needs."""
    Pm = unpack(theta)
    q = bf16_round if bf16 else (lambda a: a)
    act = {}

    def layer(name, inp):
        W, b, a = Pm[name]
        kind = dict((n, k) for n, k, _, _ in LAYERS)[name]
        xin = q(inp)
        if kind == "down":
            pre = conv_down(xin, q(W), b)
        elif kind == "up":
            pre = conv_up(xin, q(W), b)
        else:
            y = np.einsum("oc,nchw->nohw", q(W)[:, :, 0, 0], xin) + b[None, :, None, None]
            act[name] = (xin, None)
            return y
        act[name] = (xin, pre)
        return prelu(pre, a)

    e1 = layer("enc1", x)
    e2 = layer("enc2", e1)
    e3 = layer("enc3", e2)
    e4 = layer("enc4", e3)
    d3 = layer("dec3", e4)
    d2 = layer("dec2", np.concatenate([d3, e3], axis=1))
    d1 = layer("dec1", np.concatenate([d2, e2], axis=1))
    d0 = layer("dec0", np.concatenate([d1, e1], axis=1))
    y = layer("out", d0)
    return (y, act) if keep else y


def backward(theta, act, gy):
    """Flat gradient (weights, biases, PReLU slopes in the parameter order) given gy = dL/dy and the
    activations saved by forward(keep=True)."""
    Pm = unpack(theta)
    grads = {}

    def layer_b(name, g):
        W, b, a = Pm[name]
        kind = dict((n, k) for n, k, _, _ in LAYERS)[name]
        xin, pre = act[name]
        if kind == "conv1":
            gW = np.einsum("nohw,nchw->oc", g, xin)[:, :, None, None]
            grads[name] = (gW, g.sum(axis=(0, 2, 3)), None)
            return np.einsum("oc,nohw->nchw", W[:, :, 0, 0], g)
        ga = float(np.sum(g * np.where(pre > 0, 0.0, pre)))
        g = g * np.where(pre > 0, 1.0, a)
        if kind == "down":
            gx, gW, gb = conv_down_backward(xin, W, g)
        else:
            gx, gW, gb = conv_up_backward(xin, W, g)
        grads[name] = (gW, gb, ga)
        return gx

    g = layer_b("out", gy)
    g = layer_b("dec0", g)
    gd1, ge1 = g[:, :WIDTH], g[:, WIDTH:]
    g = layer_b("dec1", gd1)
    gd2, ge2 = g[:, :WIDTH], g[:, WIDTH:]
    g = layer_b("dec2", gd2)
    gd3, ge3 = g[:, :WIDTH], g[:, WIDTH:]
    ge4 = layer_b("dec3", gd3)
    ge3 = ge3 + layer_b("enc4", ge4)
    ge2 = ge2 + layer_b("enc3", ge3)
    ge1 = ge1 + layer_b("enc2", ge2)
    layer_b("enc1", ge1)
    parts = []
    for name, kind, _, _ in LAYERS:
        gW, gb, ga = grads[name]
        parts += [gW.ravel(), gb.ravel()]
        if kind != "conv1":
            parts.append(np.array([ga]))
    return np.concatenate(parts)


def network_input(v, c, p, h, omega, sigma_max=None):
    """(Re v, Im v, c / 1500, Re sigma_c, Im sigma_c) for v complex [B][Ny][Nx], padded to multiples
    of 16 at the bottom/right."""
    v = np.asarray(v)
    B, Ny, Nx = v.shape
    _, sx, _, sy, _ = hz.coefficients(c, p, h, omega, sigma_max)
    sig = sy[:, None] * sx[None, :] - 1.0
    cc = np.broadcast_to(np.asarray(c, np.float64) / C_REF, v.shape)
    x = np.stack([v.real, v.imag, cc, np.broadcast_to(sig.real, v.shape), np.broadcast_to(sig.imag, v.shape)],
                 axis=1)
    Hp, Wp = -(-Ny // 16) * 16, -(-Nx // 16) * 16
    out = np.zeros((B, 5, Hp, Wp))
    out[:, :, :Ny, :Nx] = x
    return out


def precondition(theta, v, c, p, h, omega, bf16=False):
    """z = h^2 N(alpha v, c, sigma) / alpha per batch entry, alpha = sqrt(n) / ||v|| (as oracle.unet)."""
    v = np.asarray(v, np.complex128)
    B, Ny, Nx = v.shape
    nrm = np.sqrt((np.abs(v) ** 2).reshape(B, -1).sum(1))
    alpha = np.where(nrm > 0, np.sqrt(Ny * Nx) / np.where(nrm > 0, nrm, 1.0), 0.0)
    y = forward(theta, network_input(v * alpha[:, None, None], c, p, h, omega), bf16=bf16)[:, :, :Ny, :Nx]
    inv = np.where(alpha > 0, 1.0 / np.where(alpha > 0, alpha, 1.0), 0.0)
    return (y[:, 0] + 1j * y[:, 1]) * (h * h * inv)[:, None, None]
