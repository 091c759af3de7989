"""Train the U-Net preconditioner with helm_train_step (eqs. 8-9).

Two modes, both running every numerical step in libhelm (this script only draws data and keeps
the schedule):

epochs (Sec. 3.2-3.4, Tab. 3-4):
    python -m paper_2607_16906_b300.train_precond --dataset D0 --samples 10000 --epochs 50 \
        --out best.npy --checkpoint run.npz [--resume] [--val-every 5]
  A fixed set of `samples` (c, b) pairs drawn once from dataset D0-D5 (Tab. 4, on the synthetic
  menus of synth.py), kept on the GPU; every epoch visits all of them in a seeded random order, in
  batches of `batch` systems of one grid (one context whose velocities are replaced per batch by
  helm_set_velocity).  AdamW (beta 0.9/0.999, eps 1e-8, weight decay 0.01), learning rate
  cosine-decayed from lr_max to lr_min over all steps (Tab. 3: 1e-3 -> 1e-5), global-norm clip 1
  (Tab. 3), seed 42.  The checkpoint holds the weights, the AdamW moments and step count, the epoch
  and the validation history, so a resumed run continues exactly where it stopped.  Validation is
  the solver's own figure of merit, not the loss: every `val_every` epochs the mixed FGMRES solves
  a held-out set of right-hand sides (point sources on a held-out skull at the fine-grid size by
  default) and the mean iteration count to eta_b <= 1e-6 is recorded; the weights with the fewest
  iterations (ties: more converged) are written to --out.

streaming (the mode the shipped weights were trained with):
    python -m paper_2607_16906_b300.train_precond --steps 3000 --out weights.npy [--grids 128x64,...]
  Fresh sources every step over a fixed pool of velocity batches.
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


# ---------------------------------------------------------------- schedule and data (host logic)

def cosine_lr(step: int, total: int, lr_max: float, lr_min: float) -> float:
    """Cosine decay from lr_max at step 0 to lr_min at step `total` (Tab. 3: 1e-3 -> 1e-5)."""
    t = min(max(step, 0), max(total, 1)) / max(total, 1)
    return lr_min + 0.5 * (lr_max - lr_min) * (1.0 + math.cos(math.pi * t))


def epoch_order(epoch: int, count: int, seed: int) -> np.ndarray:
    """The sample order of one epoch: a permutation seeded by (seed, epoch), so a resumed run
    visits the samples in the same order as an uninterrupted one."""
    return synth.rng_for(seed * 100003 + epoch).permutation(count)


def make_sample_set(dataset: str, count: int, nx: int, p: int, seed: int):
    """`count` (c, b) pairs of dataset D0-D5 on an nx^2 + p PML grid: c float32 [S][Ny][Nx] (m/s),
    b complex64 [S][Ny][Nx]; plus the per-sample (source kind, velocity kind) labels."""
    rng = synth.rng_for(seed)
    N = nx + 2 * p
    cs = np.empty((count, N, N), np.float32)
    bs = np.empty((count, N, N), np.complex64)
    kinds = []
    for k in range(count):
        c, b, sk, vk = synth.dataset_sample(dataset, nx, p, rng)
        cs[k], bs[k] = c, b
        kinds.append((sk, vk))
    return cs, bs, kinds


def batches(order: np.ndarray, batch: int):
    """Consecutive full batches of `order` (a trailing partial batch is dropped, as usual)."""
    for k in range(0, len(order) - batch + 1, batch):
        yield order[k:k + batch]


# ---------------------------------------------------------------- checkpoints

def save_checkpoint(path, net: "helm.UNet", state: dict):
    """Weights, AdamW moments and step, and the loop state, written atomically (.npz)."""
    m, v, step = net.adam_state()
    os.makedirs(os.path.dirname(os.path.abspath(path)) or ".", exist_ok=True)
    tmp = path + ".tmp.npz"
    np.savez(tmp, weights=net.weights(), adam_m=m, adam_v=v, adam_step=np.int64(step),
             state=np.array(json.dumps(state)))
    os.replace(tmp, path)


def load_checkpoint(path):
    """(weights, (m, v, step), state) from save_checkpoint."""
    z = np.load(path, allow_pickle=False)
    return z["weights"], (z["adam_m"], z["adam_v"], int(z["adam_step"])), json.loads(str(z["state"]))


def save_weights(path, w):
    """Write weights atomically (temporary file, then rename)."""
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = path + ".tmp.npy"
    np.save(tmp, w)
    os.replace(tmp, path)


# ---------------------------------------------------------------- validation by iteration count

class Validator:
    """Mean FGMRES iterations to eta_b <= tol on a held-out problem (mixed path, DCGS2)."""

    def __init__(self, prob, m=512, max_outer=20, tol=1e-6, inner_tol=1e-5):
        self.prob = prob
        spec = helm.SystemSpec(prob.nx, prob.ny, prob.h, prob.p, prob.omega)
        self.ctx = helm.Context([spec], torch.tensor(prob.c.ravel(), device="cuda"))
        self.b = torch.tensor(prob.b.ravel(), device="cuda")
        self.kw = dict(m=m, tol=tol, mixed=True, max_outer=max_outer, inner_tol=inner_tol, orth="dcgs2")

    def __call__(self, net):
        x = torch.zeros_like(self.b)
        _, info = helm.helm_fgmres_solve(self.ctx, net, self.b, x, self.prob.nrhs, **self.kw)
        its = [c["iters"] for c in info]
        return {"mean_iters": float(np.mean(its)), "converged": int(sum(c["status"] == "OK" for c in info)),
                "worst_relres": float(max(c["relres_true"] for c in info))}


def better(a, b):
    """Validation record a beats b: more right-hand sides converged, then fewer iterations."""
    if b is None:
        return True
    return (a["converged"], -a["mean_iters"]) > (b["converged"], -b["mean_iters"])


# ---------------------------------------------------------------- epoch mode

def train_epochs(dataset="D0", samples=10000, nx=128, p=16, ppw=10.0, batch=32, epochs=50, lr_max=1e-3,
                 lr_min=1e-5, wd=0.01, clip=1.0, seed=42, init=None, out=None, checkpoint=None, resume=False,
                 val_every=5, validator=None, verbose=True, log_every=50, stop_after=None, kind=0):
    """Epoch mode (module docstring).  `epochs` fixes the schedule; `stop_after` ends this invocation
    after that many epochs in all (a later call with resume=True continues the same schedule).
    kind: network kind (0: the 16/32/64/128 U-Net, 1: the paper's variant)."""
    h, om = synth.grid_spacing(ppw), synth.angular_frequency()
    cs, bs, _ = make_sample_set(dataset, samples, nx, p, seed)
    c_dev = torch.tensor(cs, device="cuda")
    b_dev = torch.tensor(bs, device="cuda")
    ctx = helm.Context([helm.SystemSpec(nx, nx, h, p, om) for _ in range(batch)], c_dev[:batch].reshape(-1))
    state = {"epoch": 0, "step": 0, "best": None, "history": [], "dataset": dataset, "samples": samples,
             "batch": batch, "epochs": epochs, "seed": seed, "kind": kind}
    if resume and checkpoint and os.path.exists(checkpoint):
        w, (m, v, st), state = load_checkpoint(checkpoint)
        net = helm.UNet(w, kind=kind)
        net.set_adam_state(m, v, st)
    else:
        segs = helm.weight_segments() if kind == 0 else helm.paper_weight_segments()
        theta = init if init is not None else synth.kaiming_uniform_params(segs, seed)
        net = helm.UNet(theta, kind=kind)
    steps_per_epoch = samples // batch
    total = steps_per_epoch * epochs
    t0 = time.time()
    last = epochs if stop_after is None else min(epochs, stop_after)
    while state["epoch"] < last:
        ep = state["epoch"]
        losses = []
        for idx in batches(epoch_order(ep, samples, seed), batch):
            sel = torch.as_tensor(idx, device="cuda")
            ctx.set_velocity(c_dev.index_select(0, sel).reshape(-1))
            bb = b_dev.index_select(0, sel).reshape(-1).contiguous()
            lr = cosine_lr(state["step"], total, lr_max, lr_min)
            loss, gn = helm.helm_train_step(ctx, net, bb, lr=lr, wd=wd, clip=clip)
            losses.append(loss)
            state["step"] += 1
            if verbose and state["step"] % log_every == 0:
                print(f"epoch {ep} step {state['step']} loss {loss:.4f} |g| {gn:.3g} lr {lr:.2e} "
                      f"{time.time() - t0:.0f}s", flush=True)
        rec = {"epoch": ep, "loss": float(np.mean(losses)), "s": time.time() - t0}
        state["epoch"] = ep + 1
        if validator is not None and (state["epoch"] % val_every == 0 or state["epoch"] == epochs):
            rec["val"] = validator(net)
            if better(rec["val"], state["best"]):
                state["best"] = dict(rec["val"], epoch=ep)
                if out:
                    save_weights(out, net.weights())
        state["history"].append(rec)
        if verbose:
            print(json.dumps(rec), flush=True)
        if checkpoint:
            save_checkpoint(checkpoint, net, state)
    if out and validator is None:
        save_weights(out, net.weights())
    return net, state


# ---------------------------------------------------------------- streaming mode

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
    log = []
    t0 = time.time()
    for it in range(steps):
        lr = cosine_lr(it, steps, lr_max, lr_min)
        ctx, nx, batch = pool[it % len(pool)]
        b = torch.tensor(draw_sources(batch, nx, p, rng, p_gauss, p_point), device="cuda")
        loss, gn = helm.helm_train_step(ctx, net, b, lr=lr, wd=wd, clip=clip)
        if it % log_every == 0 or it == steps - 1:
            log.append({"step": it, "loss": loss, "grad_norm": gn, "lr": lr, "s": time.time() - t0})
            if verbose:
                print(f"step {it:5d} loss {loss:.4f} |g| {gn:.3g} lr {lr:.2e} {time.time() - t0:.1f}s", flush=True)
        if checkpoint and save_every > 0 and (it + 1) % save_every == 0:
            save_weights(checkpoint, net.weights())
    return net.weights(), log


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--init", default=None)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--lr-min", type=float, default=1e-5)
    ap.add_argument("--pml", type=int, default=16)
    # epoch mode
    ap.add_argument("--dataset", default=None, choices=sorted(synth.DATASETS), help="epoch mode: Tab. 4 dataset")
    ap.add_argument("--samples", type=int, default=10000)
    ap.add_argument("--grid", type=int, default=128, help="interior side of the training grid")
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--epochs", type=int, default=50)
    ap.add_argument("--checkpoint", default=None)
    ap.add_argument("--resume", action="store_true")
    ap.add_argument("--val-every", type=int, default=5)
    ap.add_argument("--val-rhs", type=int, default=16, help="held-out right-hand sides of the fine-grid workload")
    ap.add_argument("--seed", type=int, default=42, help="epoch mode: seed of the sample set and epoch order")
    ap.add_argument("--no-val", action="store_true")
    ap.add_argument("--kind", type=int, default=0, help="network kind: 0 (16/32/64/128 U-Net) or 1 (the paper's)")
    # streaming mode
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--grids", default="128x64", help="comma list of <interior side>x<batch>")
    ap.add_argument("--nctx", type=int, default=8)
    ap.add_argument("--p-gauss", type=float, default=0.6)
    ap.add_argument("--p-point", type=float, default=0.3)
    ap.add_argument("--save-every", type=int, default=0, help="also write --out every N steps")
    ap.add_argument("--log", default=None)
    a = ap.parse_args()
    init = np.load(a.init) if a.init else None
    if a.dataset:
        val = None if a.no_val else Validator(synth.fine_multi_rhs_problem(seed=3900, nrhs=a.val_rhs))
        _, state = train_epochs(dataset=a.dataset, samples=a.samples, nx=a.grid, p=a.pml, batch=a.batch,
                                epochs=a.epochs, lr_max=a.lr, lr_min=a.lr_min, init=init, out=a.out,
                                checkpoint=a.checkpoint, resume=a.resume, val_every=a.val_every, validator=val,
                                kind=a.kind, seed=a.seed)
        if a.log:
            with open(a.log, "w") as f:
                json.dump(state, f)
        return
    grids = tuple(tuple(int(v) for v in g.split("x")) for g in a.grids.split(","))
    w, log = train(steps=a.steps, grids=grids, p=a.pml, lr_max=a.lr, lr_min=a.lr_min, init=init, nctx=a.nctx,
                   p_gauss=a.p_gauss, p_point=a.p_point, checkpoint=a.out, save_every=a.save_every)
    save_weights(a.out, w)
    if a.log:
        with open(a.log, "w") as f:
            json.dump(log, f)


if __name__ == "__main__":
    main()
