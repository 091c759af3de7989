"""Each tensor-core layer of network kind 1 (the paper's variant, Sec. 3.1, Tab. 2) checked on its own
against the oracle's plain strided and transposed 8x8 convolutions, element by element.

The library computes the first three 8x8 stride-2 layers, where their output grid has even sides, as
a 3x3 convolution over 4 x 4 blocks of their input (a strided tensor-map view; the first layer reads the space-to-depth
packed input through a stride-2 view), with the 2 x 2 output phases as 128 GEMM columns written
depth-to-space; the last encoder layer and odd grids as a 5x5 convolution of space-to-depth data.  Every transposed
layer is a 5x5 convolution written depth-to-space; the last one also with the 1x1 output layer fused
into its epilogue.  The oracle applies the definitions in FP64 to the same BF16 inputs and
BF16-rounded weights.  The GEMM grids leave ragged tiles in both directions, for each tile height the
library picks, in both encoder forms.

Bound per element: the final BF16 rounding of the output (2^-8 of the value) plus 2e-5 of the sum of
the absolute products that make the output (FP32 accumulation).  For the fused output layer the
activation it reads may sit one BF16 unit (2^-7 relative) away from the oracle's: 2^-7 of the sum of
|activation x weight| plus the propagated accumulation bound.
"""
import numpy as np
import pytest
import torch

from oracle import unet as ou
from oracle import unet_paper as up
from paper_2607_16906_b300 import synth

pytestmark = pytest.mark.gpu

# (B, H, W) of the 5x5 GEMM grid (the encoder's output grid): tiles of one 8 x 16 block (12 x 20, 9 x 33),
# and grids on which the library stacks 2 or 4 blocks per tile with a ragged last tile row (60 x 20,
# 30 x 36).  The even grids run enc1..enc3 in the phase form (GEMM grids 6 x 10: one block per tile;
# 30 x 10 and 15 x 18: two), 9 x 33 and enc4 in the 5x5 form
GRIDS = ((2, 12, 20), (1, 9, 33), (1, 60, 20), (2, 30, 36))
NAMES = ("enc1", "enc2", "enc3", "enc4", "dec3", "dec2", "dec1", "dec0")


@pytest.fixture(scope="module")
def helm():
    from paper_2607_16906_b300 import helm as h
    return h


@pytest.fixture(scope="module")
def net_theta(helm):
    theta = synth.kaiming_uniform_params(helm.paper_weight_segments(), 42)
    rng = synth.rng_for(7)
    for name, (W, b, a) in up.unpack(theta).items():
        b[:] = 0.2 * rng.standard_normal(b.shape)   # biases that move part of every layer below zero
    return helm.UNet(theta, kind=1), up.unpack(theta)


def _bf16(rng, shape):
    """A BF16 NHWC CUDA tensor and its values as float64 NCHW."""
    x = torch.tensor(rng.standard_normal(shape), dtype=torch.float32).to(torch.bfloat16)
    return x.cuda().contiguous(), np.transpose(x.float().numpy().astype(np.float64), (0, 3, 1, 2))


def _q(W):
    """Weights as the library rounds them (FP64 -> FP32 -> BF16)."""
    return ou.bf16_round(np.asarray(W, np.float32))


def _layer_ref(P, l, x):
    """Pre-activation, PReLU output and the sum of absolute products of layer l on input x (NCHW)."""
    W, b, a = P[NAMES[l]]
    conv = up.conv_down if l < 4 else up.conv_up
    pre = conv(x, _q(W), b)
    S = conv(np.abs(x), np.abs(_q(W)), np.zeros_like(b)) + np.abs(b)[None, :, None, None]
    return pre, up.prelu(pre, a), S


def _check(got, ref, S):
    bound = 2.0 ** -8 * np.maximum(np.abs(ref), np.abs(got)) + 2e-5 * S + 1e-30
    err = np.abs(got - ref)
    assert (err <= bound).all(), (float((err / bound).max()), np.unravel_index(np.argmax(err / bound), err.shape))


@pytest.mark.parametrize("grid", GRIDS)
@pytest.mark.parametrize("layer", range(8))
def test_paper_layer_matches_oracle(helm, net_theta, layer, grid):
    net, P = net_theta
    B, H, W = grid
    rng = synth.rng_for(700 + layer)
    if layer == 0:
        # network input on the 2H x 2W grid: 5 channels used of 8, packed space-to-depth
        x = np.zeros((B, 2 * H, 2 * W, 8), np.float32)
        x[..., :5] = rng.standard_normal((B, 2 * H, 2 * W, 5))
        xt = torch.tensor(x).to(torch.bfloat16)
        xin = np.transpose(xt.float().numpy().astype(np.float64), (0, 3, 1, 2))[:, :5]
        s2d = xt.reshape(B, H, 2, W, 2, 8).permute(0, 1, 3, 2, 4, 5).reshape(B, H, W, 32)
        in0, in1 = s2d.cuda().contiguous(), None
        out = torch.empty(B, H, W, 32, dtype=torch.bfloat16, device="cuda")
    elif layer <= 3:
        in0, xin = _bf16(rng, (B, 2 * H, 2 * W, 32))
        in1 = None
        out = torch.empty(B, H, W, 32, dtype=torch.bfloat16, device="cuda")
    else:
        in0, x0 = _bf16(rng, (B, H, W, 32))
        in1, xin = None, x0
        if layer >= 5:                                   # the concatenation [decoder, skip]
            in1, x1 = _bf16(rng, (B, H, W, 32))
            xin = np.concatenate([x0, x1], axis=1)
        out = torch.empty(B, 2 * H, 2 * W, 32, dtype=torch.bfloat16, device="cuda")
    helm.helm_paper_layer_forward(net, layer, in0, out, B, H, W, in1=in1)
    torch.cuda.synchronize()
    got = np.transpose(out.float().cpu().numpy().astype(np.float64), (0, 3, 1, 2))
    _, ref, S = _layer_ref(P, layer, xin)
    assert got.shape == ref.shape
    _check(got, ref, S)


@pytest.mark.parametrize("grid", GRIDS)
def test_paper_last_layer_with_fused_output(helm, net_theta, grid):
    net, P = net_theta
    B, H, W = grid
    rng = synth.rng_for(790)
    in0, x0 = _bf16(rng, (B, H, W, 32))
    in1, x1 = _bf16(rng, (B, H, W, 32))
    z = torch.empty(B, 2 * H, 2 * W, 2, dtype=torch.float32, device="cuda")
    helm.helm_paper_layer_forward(net, helm.HELM_PAPER_LAYER_DEC0_FINAL, in0, z, B, H, W, in1=in1)
    torch.cuda.synchronize()
    got = np.transpose(z.cpu().numpy().astype(np.float64), (0, 3, 1, 2))
    _, post, S = _layer_ref(P, 7, np.concatenate([x0, x1], axis=1))
    d0 = ou.bf16_round(post)
    Wo, bo, _ = P["out"]
    wq = _q(Wo)[:, :, 0, 0]
    ref = np.einsum("oc,nchw->nohw", wq, d0) + bo[None, :, None, None]
    Sd = np.einsum("oc,nchw->nohw", np.abs(wq), np.abs(d0))
    Ss = np.einsum("oc,nchw->nohw", np.abs(wq), S)
    bound = 2.0 ** -7 * Sd + 2e-5 * Ss + 1e-6 * (Sd + np.abs(bo)[None, :, None, None])
    err = np.abs(got - ref)
    assert (err <= bound).all(), float((err / bound).max())


def test_paper_layer_rejects_bad_arguments(helm, net_theta):
    net, _ = net_theta
    t = torch.zeros(1, 8, 16, 32, dtype=torch.bfloat16, device="cuda")
    big = torch.zeros(1, 16, 32, 32, dtype=torch.bfloat16, device="cuda")
    with pytest.raises(helm.HelmError, match="in1"):
        helm.helm_paper_layer_forward(net, 5, t, big, 1, 8, 16)        # decoder concat without the skip
    with pytest.raises(ValueError, match="out"):
        helm.helm_paper_layer_forward(net, 5, t, t, 1, 8, 16, in1=t)   # output smaller than 2H x 2W x 32
    with pytest.raises(ValueError, match="in0"):
        helm.helm_paper_layer_forward(net, 1, t, t, 1, 8, 16)          # encoder input smaller than 2H x 2W
    with pytest.raises(helm.HelmError, match="range"):
        helm.helm_paper_layer_forward(net, 9, t, t, 1, 8, 16)
    k0 = helm.UNet(synth.kaiming_uniform_params(helm.weight_segments(), 1))
    with pytest.raises(helm.HelmError, match="kind 1"):
        helm.helm_paper_layer_forward(k0, 0, t, t, 1, 8, 16)
