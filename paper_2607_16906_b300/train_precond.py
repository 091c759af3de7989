"""Train the U-Net preconditioner with helm_train_step (eqs. 8-9) on seeded synthetic batches.

    python -m paper_2607_16906_b300.train_precond --steps 3000 --out weights.npy [--log log.json]

Data (Sec. 3.2 describes mixed datasets; the paper's skull and CT data are not available here):
velocities alternate between skull rings with noise and log-normal Gaussian random fields,
128 x 128 interior + 16 PML cells at 10 points per water wavelength; each step draws fresh sources
for a fixed batch of velocities, with the paper's D0-style mix of source types: N(0,1) fields
(60 %), 1-5 random point sources (30 %) and a 32-element line array (10 %).  Optimiser: AdamW,
learning rate cosine-decayed from lr_max to lr_min (Tab. 3: 1e-3 -> 1e-5), global-norm clip 1,
seed 42 (Tab. 3).  Every numerical step runs in libhelm; this script only draws the data.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np
import torch

from . import helm, synth


def make_batch_contexts(nctx, batch, nx, p, ppw, rng):
    """`nctx` contexts of `batch` velocities each (alternately skull ring and log-normal GRF)."""
    h, om = synth.grid_spacing(ppw), synth.angular_frequency()
    ctxs = []
    for _ in range(nctx):
        cs = [synth.skull_velocity(nx, nx, p, rng) if k % 2 == 0 else synth.grf_velocity(nx, nx, p, rng)
              for k in range(batch)]
        specs = [helm.SystemSpec(nx, nx, h, p, om) for _ in range(batch)]
        ctxs.append(helm.Context(specs, torch.tensor(np.concatenate([c.ravel() for c in cs]), device="cuda")))
    return ctxs


def draw_sources(batch, nx, p, rng, p_gauss=0.6, p_point=0.3):
    """Sources: N(0,1) fields with probability p_gauss, 1-5 point sources with p_point, else a line array."""
    out = []
    for _ in range(batch):
        u = rng.uniform()
        if u < p_gauss:
            out.append(synth.gaussian_sources(nx, nx, p, rng))
        elif u < p_gauss + p_point:
            out.append(synth.point_sources(nx, nx, p, rng, int(rng.integers(1, 6))))
        else:
            out.append(synth.line_array(nx, nx, p, rng))
    return np.concatenate([b.ravel() for b in out]).astype(np.complex64)


def train(steps=3000, grids=((128, 64),), p=16, ppw=10.0, lr_max=1e-3, lr_min=1e-5, wd=0.01, clip=1.0, seed=42,
          nctx=8, init=None, log_every=50, verbose=True, p_gauss=0.6, p_point=0.3, checkpoint=None, save_every=0):
    """AdamW on eq. 9 over batches cycling through `grids` = ((interior side, batch size), ...).
    With `checkpoint` and `save_every` > 0 the weights are also written there every `save_every` steps."""
    rng = synth.rng_for(seed)
    theta = init if init is not None else synth.kaiming_uniform_params(helm.weight_segments(), seed)
    net = helm.UNet(theta)
    pool = []  # (context, nx, batch)
    for nx, batch in grids:
        pool += [(c, nx, batch) for c in make_batch_contexts(nctx, batch, nx, p, ppw, rng)]
    order = [k for k in range(len(pool))]
    log = []
    t0 = time.time()
    for it in range(steps):
        lr = lr_min + 0.5 * (lr_max - lr_min) * (1.0 + math.cos(math.pi * it / max(1, steps)))
        ctx, nx, batch = pool[order[it % len(pool)]]
        b = torch.tensor(draw_sources(batch, nx, p, rng, p_gauss, p_point), device="cuda")
        loss, gn = helm.helm_train_step(ctx, net, b, lr=lr, wd=wd, clip=clip)
        if it % log_every == 0 or it == steps - 1:
            log.append({"step": it, "loss": loss, "grad_norm": gn, "lr": lr, "s": time.time() - t0})
            if verbose:
                print(f"step {it:5d} loss {loss:.4f} |g| {gn:.3g} lr {lr:.2e} {time.time() - t0:.1f}s", flush=True)
        if checkpoint and save_every > 0 and (it + 1) % save_every == 0:
            save_weights(checkpoint, net.weights())
    return net.weights(), log


def save_weights(path, w):
    """Write weights atomically (temporary file, then rename)."""
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = path + ".tmp.npy"
    np.save(tmp, w)
    os.replace(tmp, path)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--grids", default="128x64", help="comma list of <interior side>x<batch>")
    ap.add_argument("--pml", type=int, default=16)
    ap.add_argument("--nctx", type=int, default=8)
    ap.add_argument("--p-gauss", type=float, default=0.6)
    ap.add_argument("--p-point", type=float, default=0.3)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--out", required=True)
    ap.add_argument("--log", default=None)
    ap.add_argument("--init", default=None)
    ap.add_argument("--save-every", type=int, default=0, help="also write --out every N steps")
    a = ap.parse_args()
    init = np.load(a.init) if a.init else None
    grids = tuple(tuple(int(v) for v in g.split("x")) for g in a.grids.split(","))
    w, log = train(steps=a.steps, grids=grids, p=a.pml, lr_max=a.lr, init=init, nctx=a.nctx, p_gauss=a.p_gauss,
                   p_point=a.p_point, checkpoint=a.out, save_every=a.save_every)
    save_weights(a.out, w)
    if a.log:
        with open(a.log, "w") as f:
            json.dump(log, f)


if __name__ == "__main__":
    main()
