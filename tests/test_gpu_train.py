"""Parity of the CUDA training path (a9: eqs. 8-9, conv backward, AdamW) against the oracle."""
import numpy as np
import pytest
import torch

from oracle import train as ot
from oracle import unet as ou
from paper_2607_16906_b300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def helm():
    from paper_2607_16906_b300 import helm as h
    return h


def _batch(B=3, nx=20, p=6, seed=61):
    rng = synth.rng_for(seed)
    c = np.stack([synth.skull_velocity(nx, nx, p, rng, thickness=(2, 3)) if k % 2 == 0
                  else synth.grf_velocity(nx, nx, p, rng) for k in range(B)])
    b = np.stack([synth.point_sources(nx, nx, p, rng, 2) if k % 2 == 0 else synth.gaussian_sources(nx, nx, p, rng)
                  for k in range(B)])
    return c, b, nx, p, synth.grid_spacing(10.0), synth.angular_frequency()


def _ctx(helm, c, nx, p, h, om):
    specs = [helm.SystemSpec(nx, nx, h, p, om) for _ in range(c.shape[0])]
    return helm.Context(specs, torch.tensor(c.ravel(), device="cuda"))


def test_fp64_loss_and_gradient_match_oracle(helm):
    c, b, nx, p, h, om = _batch()
    theta = synth.kaiming_uniform_params(ou.param_segments(), 42)
    ctx = _ctx(helm, c, nx, p, h, om)
    net = helm.UNet(theta)
    L, g = helm.helm_loss_grad(ctx, net, torch.tensor(b.ravel(), device="cuda"))
    Lr, gr, _ = ot.loss_and_grad(theta, b, c, p, h, om)
    assert abs(L - Lr) <= 1e-11 * Lr
    g = g.cpu().numpy()
    assert np.abs(g - gr).max() <= 1e-9 * np.abs(gr).max()


def test_fp64_gradient_central_difference(helm):
    """Central difference of the GPU loss itself (FP64 path) along random parameter directions."""
    c, b, nx, p, h, om = _batch(B=2, seed=62)
    theta = synth.kaiming_uniform_params(ou.param_segments(), 43)
    ctx = _ctx(helm, c, nx, p, h, om)
    bd = torch.tensor(b.ravel(), device="cuda")
    _, g = helm.helm_loss_grad(ctx, helm.UNet(theta), bd)
    g = g.cpu().numpy()
    rng = synth.rng_for(7)
    for _ in range(2):
        d = rng.standard_normal(theta.size)
        eps = 1e-8
        Lp, _ = helm.helm_loss_grad(ctx, helm.UNet(theta + eps * d), bd)
        Lm, _ = helm.helm_loss_grad(ctx, helm.UNet(theta - eps * d), bd)
        fd = (Lp - Lm) / (2 * eps)
        assert abs(fd - g @ d) <= 1e-6 * abs(fd), (fd, g @ d)


def test_autograd_function_matches_oracle_and_central_difference(helm):
    """HelmholtzLoss (torch.autograd.Function over the library's loss and gradient, FP64 path):
    the forward equals the oracle's eq. 9, backward equals the oracle's gradient, and the central
    difference of the forward along a random direction (weights loaded by helm_unet_set_weights)
    equals the directional derivative."""
    c, b, nx, p, h, om = _batch(B=2, seed=64)
    theta = synth.kaiming_uniform_params(ou.param_segments(), 45)
    ctx = _ctx(helm, c, nx, p, h, om)
    net = helm.UNet(np.zeros_like(theta))  # weights come from theta through set_weights
    bd = torch.tensor(b.ravel(), device="cuda")
    t = torch.tensor(theta, device="cuda", requires_grad=True)
    loss = helm.HelmholtzLoss.apply(t, ctx, net, bd)
    (2.0 * loss).backward()
    Lr, gr, _ = ot.loss_and_grad(theta, b, c, p, h, om)
    assert abs(loss.item() - Lr) <= 1e-11 * Lr
    g = t.grad.cpu().numpy() / 2.0
    assert np.abs(g - gr).max() <= 1e-9 * np.abs(gr).max()
    d = synth.rng_for(8).standard_normal(theta.size)
    eps = 1e-8
    with torch.no_grad():
        td = torch.tensor(d, device="cuda")
        Lp = helm.HelmholtzLoss.apply(t + eps * td, ctx, net, bd).item()
        Lm = helm.HelmholtzLoss.apply(t - eps * td, ctx, net, bd).item()
    fd = (Lp - Lm) / (2 * eps)
    assert abs(fd - g @ d) <= 1e-6 * abs(fd), (fd, g @ d)


def test_bf16_gradient_close_to_oracle_emulation(helm):
    """BF16 activations and weights, FP32 gradients: the loss matches the oracle's BF16 emulation
    and the gradient points the same way (cosine > 0.999, normwise error <= 5e-2)."""
    c, b, nx, p, h, om = _batch(seed=63)
    theta = synth.kaiming_uniform_params(ou.param_segments(), 42)
    ctx = _ctx(helm, c, nx, p, h, om)
    b32 = b.astype(np.complex64)
    L, g = helm.helm_loss_grad(ctx, helm.UNet(theta), torch.tensor(b32.ravel(), device="cuda"))
    Lr, gr, _ = ot.loss_and_grad(theta, b32.astype(complex), c, p, h, om, bf16=True)
    assert abs(L - Lr) <= 2e-2 * Lr
    g = g.cpu().numpy()
    cos = g @ gr / (np.linalg.norm(g) * np.linalg.norm(gr))
    assert cos > 0.999, cos
    assert np.linalg.norm(g - gr) <= 5e-2 * np.linalg.norm(gr)


def test_train_step_is_clipped_adamw_on_the_gradient(helm):
    c, b, nx, p, h, om = _batch(seed=64)
    theta = synth.kaiming_uniform_params(ou.param_segments(), 42)
    ctx = _ctx(helm, c, nx, p, h, om)
    bd = torch.tensor(b.astype(np.complex64).ravel(), device="cuda")
    net = helm.UNet(theta)
    L0, g = helm.helm_loss_grad(ctx, net, bd)
    g = g.cpu().numpy()
    lr, wd, clip = 1e-3, 0.01, 1.0
    loss, gn = helm.helm_train_step(ctx, net, bd, lr=lr, wd=wd, clip=clip)
    assert abs(loss - L0) <= 1e-12 * L0
    assert abs(gn - np.linalg.norm(g)) <= 1e-12 * gn
    gc, _ = ot.clip_by_global_norm(g, clip)
    ref, _, _ = ot.adamw_step(theta, gc, np.zeros_like(theta), np.zeros_like(theta), 1, lr, wd)
    got = net.weights()
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_training_reduces_the_loss(helm):
    c, b, nx, p, h, om = _batch(B=4, nx=40, p=8, seed=65)
    theta = synth.kaiming_uniform_params(ou.param_segments(), 42)
    ctx = _ctx(helm, c, nx, p, h, om)
    bd = torch.tensor(b.astype(np.complex64).ravel(), device="cuda")
    net = helm.UNet(theta)
    losses = [helm.helm_train_step(ctx, net, bd, lr=1e-3, wd=0.0, clip=1.0)[0] for _ in range(60)]
    assert np.isfinite(losses).all()
    assert losses[-1] < 0.2 * losses[0], (losses[0], losses[-1])


def test_training_rejects_mixed_grid_sizes(helm):
    rng = synth.rng_for(66)
    c1 = synth.skull_velocity(20, 20, 6, rng)
    c2 = synth.skull_velocity(24, 24, 6, rng)
    h, om = synth.grid_spacing(10.0), synth.angular_frequency()
    specs = [helm.SystemSpec(20, 20, h, 6, om), helm.SystemSpec(24, 24, h, 6, om)]
    ctx = helm.Context(specs, torch.tensor(np.concatenate([c1.ravel(), c2.ravel()]), device="cuda"))
    b = torch.ones(ctx.npts, dtype=torch.complex64, device="cuda")
    with pytest.raises(helm.HelmError):
        helm.helm_train_step(ctx, helm.UNet(synth.kaiming_uniform_params(ou.param_segments(), 1)), b)


def test_epoch_training_loop_resumes_exactly(tmp_path):
    """Epochs over a fixed sample set (Tab. 4 dataset D0), AdamW with the cosine schedule, validation
    by solver iteration count, checkpoint with the AdamW state: stopping after one epoch and resuming
    gives the same weights, bit for bit, as running both epochs at once."""
    from paper_2607_16906_b300 import synth
    from paper_2607_16906_b300 import train_precond as tp
    prob = synth.small_problem(seed=1900, nx=32, p=8)
    val = tp.Validator(prob, m=20, max_outer=10)
    kw = dict(dataset="D0", samples=16, nx=24, p=4, batch=8, lr_max=1e-3, lr_min=1e-4, val_every=1,
              validator=val, verbose=False)
    net_a, st_a = tp.train_epochs(epochs=2, checkpoint=str(tmp_path / "a.npz"), out=str(tmp_path / "a.npy"), **kw)
    assert len(st_a["history"]) == 2 and all("val" in r for r in st_a["history"])
    assert st_a["step"] == 4 and st_a["best"] is not None
    ck = str(tmp_path / "b.npz")
    tp.train_epochs(epochs=2, stop_after=1, checkpoint=ck, **kw)   # interrupted after the first epoch
    _, (m1, v1, s1), st1 = tp.load_checkpoint(ck)
    assert s1 == 2 and st1["epoch"] == 1 and np.abs(m1).sum() > 0
    net_b, st_b = tp.train_epochs(epochs=2, checkpoint=ck, resume=True, **kw)
    assert st_b["step"] == 4
    assert np.array_equal(net_a.weights(), net_b.weights())
    best = np.load(str(tmp_path / "a.npy"))
    assert best.size == net_a.nparams


# ---------------------------------------------------------------- network kind 1 (the paper's variant)

def _theta_paper(helm, seed=42):
    return synth.kaiming_uniform_params(helm.paper_weight_segments(), seed)


def test_paper_network_fp64_loss_and_gradient_match_oracle(helm):
    """Eq. 9 through network kind 1: the FP64 loss and gradient (CUDA cores, through the 5x5
    reformulation and its gather back to the 8x8 weights) equal the oracle's plain strided
    convolutions, including the PReLU slope gradients."""
    c, b, nx, p, h, om = _batch(B=3, nx=20, p=6, seed=63)
    theta = _theta_paper(helm)
    ctx = _ctx(helm, c, nx, p, h, om)
    net = helm.UNet(theta, kind=1)
    L, g = helm.helm_loss_grad(ctx, net, torch.tensor(b.ravel(), device="cuda"))
    Lr, gr, _ = ot.loss_and_grad(theta, b, c, p, h, om, kind=1)
    assert abs(L - Lr) <= 1e-11 * Lr
    g = g.cpu().numpy()
    assert np.abs(g - gr).max() <= 1e-9 * np.abs(gr).max()


def test_paper_network_mixed_gradient_and_training(helm):
    """The mixed training path of kind 1 (the tcgen05 layers in BF16 with FP32 accumulation for the
    forward, activations and pre-activations kept in BF16, FP32 backward on CUDA cores) matches the
    oracle's BF16 emulation: loss to 2e-2, gradient cosine > 0.999 and normwise error <= 5e-2 (as for
    kind 0); a few AdamW steps lower the batch loss."""
    c, b, nx, p, h, om = _batch(B=4, nx=28, p=6, seed=64)
    theta = _theta_paper(helm, 44)
    ctx = _ctx(helm, c, nx, p, h, om)
    net = helm.UNet(theta, kind=1)
    b32 = torch.tensor(b.ravel().astype(np.complex64), device="cuda")
    L, g = helm.helm_loss_grad(ctx, net, b32)
    Lr, gr, _ = ot.loss_and_grad(theta, b.astype(np.complex64).astype(complex), c, p, h, om, kind=1, bf16=True)
    g = g.cpu().numpy()
    assert abs(L - Lr) <= 2e-2 * Lr, (L, Lr)
    cos = g @ gr / (np.linalg.norm(g) * np.linalg.norm(gr))
    assert cos > 0.999, cos
    assert np.linalg.norm(g - gr) <= 5e-2 * np.linalg.norm(gr)
    losses = [helm.helm_train_step(ctx, net, b32, lr=1e-3, wd=0.0, clip=1.0)[0] for _ in range(12)]
    assert losses[-1] < 0.9 * losses[0], losses
