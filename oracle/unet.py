"""Oracle: the U-Net neural operator N_theta, forward and backward (test infrastructure only).

The paper's network (Sec. 3.1, Fig. 2, Tab. 2) is a depth-4 U-Net: an encoder
that downsamples, a bottleneck, a decoder that upsamples, skip connections.
This oracle implements the reading used throughout the project:

  level l = 1..4 with widths 16, 32, 64, 128; per level two 3x3 convolutions
  (zero padding 1, bias) each followed by ReLU; 2x2 max-pool between encoder
  levels; 2x2 stride-2 transposed convolution (bias, no activation) going up;
  decoder input = concat[skip, up] along channels; final 1x1 convolution
  16 -> 2, no activation; no normalisation layers.

Inputs (eq. 7 recast as an image, Sec. 3.1): channels (Re v, Im v, c / 1500 m/s);
outputs (Re z, Im z).  Grids are zero-padded at the bottom/right to a
multiple of 8 and cropped back.

Parameter vector layout (flat float64, in this order, per layer weight then
bias): enc1a, enc1b, enc2a, enc2b, enc3a, enc3b, bota, botb, up3, dec3a,
dec3b, up2, dec2a, dec2b, up1, dec1a, dec1b, final.  Conv weights are
[C_out][C_in][kh][kw]; transposed-conv weights are [C_in][C_out][2][2].
482,050 parameters in total.

Every conv is a loop over taps of a matmul (a library primitive), written in
the plain definition of cross-correlation.

Pins (tests/test_oracle_unet.py): each op equals torch.nn.functional
(conv2d, conv_transpose2d, max_pool2d, relu) in FP64 on the CPU; the whole
forward equals a torch.nn composition; backward equals torch autograd and a
central finite difference; the parameter count equals the closed form.
"""
from __future__ import annotations

import numpy as np

CHANNELS = (16, 32, 64, 128)
IN_CH = 3
OUT_CH = 2
C_REF = 1500.0

# (name, kind, c_in, c_out) in parameter order
LAYERS = (
    ("enc1a", "conv3", IN_CH, 16), ("enc1b", "conv3", 16, 16),
    ("enc2a", "conv3", 16, 32), ("enc2b", "conv3", 32, 32),
    ("enc3a", "conv3", 32, 64), ("enc3b", "conv3", 64, 64),
    ("bota", "conv3", 64, 128), ("botb", "conv3", 128, 128),
    ("up3", "up2", 128, 64), ("dec3a", "conv3", 128, 64), ("dec3b", "conv3", 64, 64),
    ("up2", "up2", 64, 32), ("dec2a", "conv3", 64, 32), ("dec2b", "conv3", 32, 32),
    ("up1", "up2", 32, 16), ("dec1a", "conv3", 32, 16), ("dec1b", "conv3", 16, 16),
    ("final", "conv1", 16, OUT_CH),
)


def _wshape(kind, ci, co):
    if kind == "conv3":
        return (co, ci, 3, 3)
    if kind == "conv1":
        return (co, ci, 1, 1)
    return (ci, co, 2, 2)


def _fan_in(kind, ci, co):
    return ci * {"conv3": 9, "conv1": 1, "up2": 1}[kind]


def param_segments():
    """(count, fan_in, 'w'|'b') per tensor, in parameter order (input to the seeded generator)."""
    seg = []
    for _, kind, ci, co in LAYERS:
        seg.append((int(np.prod(_wshape(kind, ci, co))), _fan_in(kind, ci, co), "w"))
        seg.append((co, _fan_in(kind, ci, co), "b"))
    return seg


def param_count():
    return sum(s[0] for s in param_segments())


def unpack(theta):
    """Flat vector -> dict name -> (W, b) views."""
    theta = np.asarray(theta, np.float64)
    out, off = {}, 0
    for name, kind, ci, co in LAYERS:
        shp = _wshape(kind, ci, co)
        nw = int(np.prod(shp))
        W = theta[off:off + nw].reshape(shp)
        off += nw
        b = theta[off:off + co]
        off += co
        out[name] = (W, b)
    assert off == theta.size, (off, theta.size)
    return out


def pack(grads):
    parts = []
    for name, _, _, _ in LAYERS:
        gW, gb = grads[name]
        parts += [gW.ravel(), gb.ravel()]
    return np.concatenate(parts)


def bf16_round(x):
    """Round float values to the nearest bfloat16 (ties to even), returned as float64.

    Emulates the conversion the mixed path applies to every conv input.
    """
    f = np.asarray(x, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    out = r.view(np.float32).astype(np.float64)
    nan = np.isnan(f)
    if nan.any():
        out[nan] = np.nan
    return out


# ------------------------------------------------------------------ primitive ops

def conv2d(x, W, b, pad):
    """Cross-correlation: y[n,o,y,x] = b[o] + sum_{c,dy,dx} W[o,c,dy,dx] x[n,c,y+dy-pad,x+dx-pad]."""
    N, C, Hh, Ww = x.shape
    O, _, kh, kw = W.shape
    xp = np.zeros((N, C, Hh + 2 * pad, Ww + 2 * pad), x.dtype)
    xp[:, :, pad:pad + Hh, pad:pad + Ww] = x
    Ho, Wo = Hh + 2 * pad - kh + 1, Ww + 2 * pad - kw + 1
    y = np.zeros((N, O, Ho, Wo), np.result_type(x, W))
    for dy in range(kh):
        for dx in range(kw):
            patch = xp[:, :, dy:dy + Ho, dx:dx + Wo]               # [N, C, Ho, Wo]
            y += np.einsum("oc,nchw->nohw", W[:, :, dy, dx], patch, optimize=True)
    return y + b[None, :, None, None]


def conv2d_backward(x, W, g, pad):
    """Gradients of conv2d w.r.t. x, W, b given g = dL/dy."""
    N, C, Hh, Ww = x.shape
    O, _, kh, kw = W.shape
    xp = np.zeros((N, C, Hh + 2 * pad, Ww + 2 * pad), x.dtype)
    xp[:, :, pad:pad + Hh, pad:pad + Ww] = x
    Ho, Wo = g.shape[2], g.shape[3]
    gxp = np.zeros_like(xp)
    gW = np.zeros_like(W)
    for dy in range(kh):
        for dx in range(kw):
            patch = xp[:, :, dy:dy + Ho, dx:dx + Wo]
            gW[:, :, dy, dx] = np.einsum("nohw,nchw->oc", g, patch, optimize=True)
            gxp[:, :, dy:dy + Ho, dx:dx + Wo] += np.einsum("oc,nohw->nchw", W[:, :, dy, dx], g, optimize=True)
    gx = gxp[:, :, pad:pad + Hh, pad:pad + Ww]
    gb = g.sum(axis=(0, 2, 3))
    return gx, gW, gb


def conv_transpose2x2(x, W, b):
    """Stride-2 2x2 transposed conv: y[n,o,2i+dy,2j+dx] = b[o] + sum_c x[n,c,i,j] W[c,o,dy,dx]."""
    N, C, Hh, Ww = x.shape
    O = W.shape[1]
    y = np.zeros((N, O, 2 * Hh, 2 * Ww), np.result_type(x, W))
    for dy in range(2):
        for dx in range(2):
            y[:, :, dy::2, dx::2] = np.einsum("co,nchw->nohw", W[:, :, dy, dx], x, optimize=True)
    return y + b[None, :, None, None]


def conv_transpose2x2_backward(x, W, g):
    gx = np.zeros_like(x)
    gW = np.zeros_like(W)
    for dy in range(2):
        for dx in range(2):
            gs = g[:, :, dy::2, dx::2]
            gx += np.einsum("co,nohw->nchw", W[:, :, dy, dx], gs, optimize=True)
            gW[:, :, dy, dx] = np.einsum("nchw,nohw->co", x, gs, optimize=True)
    return gx, gW, g.sum(axis=(0, 2, 3))


def maxpool2(x):
    """2x2 max-pool, stride 2.  Also returns the argmax (first maximum in row-major window order)."""
    N, C, Hh, Ww = x.shape
    win = x.reshape(N, C, Hh // 2, 2, Ww // 2, 2).transpose(0, 1, 2, 4, 3, 5).reshape(N, C, Hh // 2, Ww // 2, 4)
    idx = np.argmax(win, axis=-1)
    return np.take_along_axis(win, idx[..., None], -1)[..., 0], idx


def maxpool2_backward(g, idx, shape):
    N, C, Hh, Ww = shape
    win = np.zeros((N, C, Hh // 2, Ww // 2, 4), g.dtype)
    np.put_along_axis(win, idx[..., None], g[..., None], -1)
    return win.reshape(N, C, Hh // 2, Ww // 2, 2, 2).transpose(0, 1, 2, 4, 3, 5).reshape(shape)


def relu(x):
    return np.maximum(x, 0.0)


# ------------------------------------------------------------------ network

def forward(theta, x, bf16=False, keep=False):
    """U-Net forward on an image batch x [N, 3, H, W] (H, W multiples of 8).

    With bf16=True every conv input and weight is rounded to bfloat16 first
    (FP32/FP64 accumulation), as the mixed-precision path does.
    Returns y [N, 2, H, W] (and the saved activations when keep=True).
    """
    P = unpack(theta)
    q = bf16_round if bf16 else (lambda a: a)
    act = {}

    def conv(name, inp, relu_after=True, pad=1):
        W, b = P[name]
        xin = q(inp)
        y = conv2d(xin, q(W), b, pad)
        act[name] = (xin, y)
        return relu(y) if relu_after else y

    def up(name, inp):
        W, b = P[name]
        xin = q(inp)
        y = conv_transpose2x2(xin, q(W), b)
        act[name] = (xin, y)
        return y

    h = conv("enc1a", x)
    s1 = conv("enc1b", h)
    p1, i1 = maxpool2(s1)
    h = conv("enc2a", p1)
    s2 = conv("enc2b", h)
    p2, i2 = maxpool2(s2)
    h = conv("enc3a", p2)
    s3 = conv("enc3b", h)
    p3, i3 = maxpool2(s3)
    h = conv("bota", p3)
    h = conv("botb", h)
    u = up("up3", h)
    h = conv("dec3a", np.concatenate([s3, u], axis=1))
    h = conv("dec3b", h)
    u = up("up2", h)
    h = conv("dec2a", np.concatenate([s2, u], axis=1))
    h = conv("dec2b", h)
    u = up("up1", h)
    h = conv("dec1a", np.concatenate([s1, u], axis=1))
    h = conv("dec1b", h)
    y = conv("final", h, relu_after=False, pad=0)
    act["pool"] = ((s1.shape, i1), (s2.shape, i2), (s3.shape, i3))
    return (y, act) if keep else y


def backward(theta, act, gy):
    """dL/dtheta (flat) and dL/dx given gy = dL/dy and the activations saved by forward(keep=True)."""
    P = unpack(theta)
    grads = {}
    (sh1, i1), (sh2, i2), (sh3, i3) = act["pool"]

    def conv_b(name, g, relu_after=True, pad=1):
        xin, y = act[name]
        if relu_after:
            g = g * (y > 0)
        gx, gW, gb = conv2d_backward(xin, P[name][0], g, pad)
        grads[name] = (gW, gb)
        return gx

    def up_b(name, g):
        xin, _ = act[name]
        gx, gW, gb = conv_transpose2x2_backward(xin, P[name][0], g)
        grads[name] = (gW, gb)
        return gx

    g = conv_b("final", gy, relu_after=False, pad=0)
    g = conv_b("dec1b", g)
    g = conv_b("dec1a", g)
    gs1, gu = g[:, :16], g[:, 16:]
    g = up_b("up1", gu)
    g = conv_b("dec2b", g)
    g = conv_b("dec2a", g)
    gs2, gu = g[:, :32], g[:, 32:]
    g = up_b("up2", gu)
    g = conv_b("dec3b", g)
    g = conv_b("dec3a", g)
    gs3, gu = g[:, :64], g[:, 64:]
    g = up_b("up3", gu)
    g = conv_b("botb", g)
    g = conv_b("bota", g)
    gs3 = gs3 + maxpool2_backward(g, i3, sh3)
    g = conv_b("enc3b", gs3)
    g = conv_b("enc3a", g)
    gs2 = gs2 + maxpool2_backward(g, i2, sh2)
    g = conv_b("enc2b", gs2)
    g = conv_b("enc2a", g)
    gs1 = gs1 + maxpool2_backward(g, i1, sh1)
    g = conv_b("enc1b", gs1)
    gx = conv_b("enc1a", g)
    return pack(grads), gx


# ------------------------------------------------------------------ preconditioner

def pad8(a):
    """Zero-pad the last two axes up to multiples of 8 (bottom/right)."""
    H, W = a.shape[-2:]
    Hp, Wp = -(-H // 8) * 8, -(-W // 8) * 8
    if (Hp, Wp) == (H, W):
        return a
    out = np.zeros(a.shape[:-2] + (Hp, Wp), a.dtype)
    out[..., :H, :W] = a
    return out


def network_input(v, c):
    """Image tensor (Re v, Im v, c / 1500) for v [B][Ny][Nx] complex, c [Ny][Nx] or [B][Ny][Nx]."""
    v = np.asarray(v)
    B = v.shape[0]
    cc = np.broadcast_to(np.asarray(c, np.float64), v.shape)
    x = np.stack([v.real, v.imag, cc / C_REF], axis=1)
    assert x.shape[0] == B
    return pad8(x)


def precondition(theta, v, c, h, bf16=False):
    """z = h^2 N_theta(alpha v, c) / alpha with alpha = sqrt(n) / ||v|| per batch entry (eq. 6).

    v: complex [B][Ny][Nx]; c: [Ny][Nx] (shared) or [B][Ny][Nx]; h: grid spacing.
    The scale alpha gives the network input unit RMS.  The factor h^2 makes the
    network approximate the inverse of the dimensionless operator h^2 A, whose
    entries are O(1) as in the paper's omega = 1 setting (Tab. 1); FGMRES is
    invariant to the scale of each z in exact arithmetic.
    """
    v = np.asarray(v, np.complex128)
    B, Ny, Nx = v.shape
    nrm = np.sqrt((np.abs(v) ** 2).reshape(B, -1).sum(1))
    alpha = np.where(nrm > 0, np.sqrt(Ny * Nx) / np.where(nrm > 0, nrm, 1.0), 0.0)
    x = network_input(v * alpha[:, None, None], c)
    y = forward(theta, x, bf16=bf16)[:, :, :Ny, :Nx]
    z = y[:, 0] + 1j * y[:, 1]
    inv = np.where(alpha > 0, 1.0 / np.where(alpha > 0, alpha, 1.0), 0.0)
    return z * (h * h * inv)[:, None, None]
