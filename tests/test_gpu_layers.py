"""Each tensor-core convolution of the BF16 network (Sec. 3.1; eq. 6 applies the network) checked
on its own against the oracle's plain convolutions, element by element.

Every 3x3 layer runs through helm_unet_layer_forward with each kernel the library can pick for it:
every rows-per-tile variant of the row-tile kernel (the autotuner's candidates) and the 9-box
kernel; the 2x2 up-convs through their GEMM kernel; the last 3x3 layer with the 1x1 output layer
fused into its epilogue.  Inputs are BF16 values and the weights are rounded to BF16 as the library
rounds them (FP64 -> FP32 -> BF16, nearest even); the oracle accumulates in FP64.  The images have
odd heights (no rows-per-tile value divides them) and widths that leave a ragged last 128-pixel
segment.  Bound per element: the final BF16 rounding of the output (2^-8 relative, one unit when
FP32 accumulation pushes a value across a rounding boundary) plus 2e-5 of the layer's largest
output for the FP32 accumulation itself.
"""
import numpy as np
import pytest
import torch

from oracle import unet as ou
from paper_2607_16906_b300 import synth

pytestmark = pytest.mark.gpu

FULL = (37, 200)    # row-tile layers: odd height, 200 = 128 + 72 pixels per row
SMALL = (19, 72)    # wide layers (9-box kernels only)
# layers the row-tile kernels serve (C_in <= 64 in 8-channel slices, C_out <= 64, see conv_row.cu)
ROW_LAYERS = {0, 1, 2, 3, 4, 12, 13, 15, 16}


@pytest.fixture(scope="module")
def helm():
    from paper_2607_16906_b300 import helm as h
    return h


@pytest.fixture(scope="module")
def net_theta(helm):
    theta = synth.kaiming_uniform_params(ou.param_segments(), 42)
    # larger biases than the Kaiming draw so that ReLU clips part of every layer
    rng = synth.rng_for(5)
    P = ou.unpack(theta)
    for name, (W, b) in P.items():
        b[:] = 0.2 * rng.standard_normal(b.shape)
    return helm.UNet(theta), theta


def _bf16_tensor(rng, shape):
    x = torch.tensor(rng.standard_normal(shape), dtype=torch.float32).to(torch.bfloat16)
    return x.cuda().contiguous(), x.float().numpy().astype(np.float64)


def _variants(helm, net, layer, args, in1=None):
    """Every kernel the layer has: row-tile variants 1..k (until the library says there are no
    more) and the 9-box kernel (-1); up-convs have one kernel."""
    kind = helm.helm_unet_layers()[min(layer, 16)][2]
    if kind == 1:
        return [0]
    out = [-1] if layer != helm.HELM_LAYER_DEC1B_FINAL else []
    v = 1
    while True:
        try:
            helm.helm_unet_layer_forward(net, layer, *args, in1=in1, variant=v)
        except helm.HelmError:
            break
        out.append(v)
        v += 1
    return out


def _bound(ref, zb=None):
    scale = np.abs(ref).max()
    base = np.abs(ref) if zb is None else zb
    return 2.0 ** -8 * base + 2e-5 * scale


@pytest.mark.parametrize("layer", list(range(17)))
def test_layer_matches_oracle_convolution(helm, net_theta, layer):
    net, theta = net_theta
    name, kind, ci, co = ou.LAYERS[layer]
    P = ou.unpack(theta)
    W, b = P[name]
    Wq = ou.bf16_round(W)
    rng = synth.rng_for(700 + layer)
    B = 2
    row_layer = layer in ROW_LAYERS
    H, Wd = FULL if row_layer else SMALL
    concat = name in ("dec3a", "dec2a", "dec1a")
    c0 = 16 if layer == 0 else (ci // 2 if concat else ci)
    in0, x0 = _bf16_tensor(rng, (B, H, Wd, c0))
    in1, x1 = (None, None)
    if concat:
        in1, x1 = _bf16_tensor(rng, (B, H, Wd, ci // 2))
    xin = x0 if not concat else np.concatenate([x0, x1], axis=3)
    xin = xin.transpose(0, 3, 1, 2)  # NCHW
    if layer == 0:
        xin = xin[:, :3]              # channels 3..15 carry data but have zero weights
    if kind == "up2":
        ref = ou.conv_transpose2x2(xin, Wq, b).transpose(0, 2, 3, 1)
        out = torch.empty((B, 2 * H, 2 * Wd, co), dtype=torch.bfloat16, device="cuda")
    else:
        ref = ou.relu(ou.conv2d(xin, Wq, b, 1)).transpose(0, 2, 3, 1)
        out = torch.empty((B, H, Wd, co), dtype=torch.bfloat16, device="cuda")
    args = (in0, out, B, H, Wd)
    variants = _variants(helm, net, layer, args, in1) if kind != "up2" else [0]
    if row_layer:
        assert len([v for v in variants if v > 0]) >= 2, variants   # the autotuner's candidates
    for v in variants:
        out.fill_(float("nan"))
        ry = helm.helm_unet_layer_forward(net, layer, in0, out, B, H, Wd, in1=in1, variant=v)
        torch.cuda.synchronize()
        got = out.float().cpu().numpy().astype(np.float64)
        assert np.isfinite(got).all(), (layer, v)
        err = np.abs(got - ref)
        bad = err > _bound(ref)
        assert not bad.any(), (name, v, ry, err.max(), np.argwhere(bad)[:5])
        if v > 0:
            assert ry in (1, 2, 4, 8)


def test_fused_output_layer_matches_oracle(helm, net_theta):
    """dec1b (3x3, 16 -> 16, ReLU, BF16 rounding) with the final 1x1 conv 16 -> 2 in its epilogue."""
    net, theta = net_theta
    P = ou.unpack(theta)
    W, b = P["dec1b"]
    Wf, bf = P["final"]
    rng = synth.rng_for(777)
    B, (H, Wd) = 2, FULL
    in0, x0 = _bf16_tensor(rng, (B, H, Wd, 16))
    a = ou.bf16_round(ou.relu(ou.conv2d(x0.transpose(0, 3, 1, 2), ou.bf16_round(W), b, 1)))
    Wfq = ou.bf16_round(Wf)[:, :, 0, 0]                    # [2][16]
    ref = np.einsum("oc,nchw->nhwo", Wfq, a) + bf
    zb = np.einsum("oc,nchw->nhwo", np.abs(Wfq), np.abs(a))
    out = torch.empty((B, H, Wd, 2), dtype=torch.float32, device="cuda")
    args = (in0, out, B, H, Wd)
    variants = _variants(helm, net, helm.HELM_LAYER_DEC1B_FINAL, args)
    assert len(variants) >= 2
    for v in [0] + variants:
        out.fill_(float("nan"))
        helm.helm_unet_layer_forward(net, helm.HELM_LAYER_DEC1B_FINAL, in0, out, B, H, Wd, variant=v)
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.float64)
        err = np.abs(got - ref)
        assert (err <= _bound(ref, zb)).all(), (v, err.max())


def test_layer_entry_rejects_what_it_cannot_run(helm, net_theta):
    net, _ = net_theta
    x = torch.zeros(2 * 8 * 8 * 64, dtype=torch.bfloat16, device="cuda")
    y = torch.zeros_like(x)
    with pytest.raises(helm.HelmError):      # decoder conv without its second input
        helm.helm_unet_layer_forward(net, 9, x, y, 2, 8, 8)
    with pytest.raises(helm.HelmError):      # second input given to an encoder conv
        helm.helm_unet_layer_forward(net, 4, x, y, 2, 8, 8, in1=x)
    with pytest.raises(helm.HelmError):      # bottleneck has no row-tile kernel
        helm.helm_unet_layer_forward(net, 6, x, y, 1, 8, 8, variant=1)
    with pytest.raises(helm.HelmError):
        helm.helm_unet_layer_forward(net, 18, x, y, 1, 8, 8)
    small = torch.zeros(100, dtype=torch.bfloat16, device="cuda")
    with pytest.raises(ValueError, match="out"):   # output smaller than B H W C_out (checked before the call)
        helm.helm_unet_layer_forward(net, 4, x, small, 2, 8, 8)
    with pytest.raises(ValueError, match="in0"):   # up-conv input smaller than B H W C_in
        helm.helm_unet_layer_forward(net, 8, x, y, 2, 8, 8)
