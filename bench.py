#!/usr/bin/env python
"""Benchmark: batched Helmholtz solves per second to a true relative residual of 1e-6.

Workload (the fine-grid multi-RHS configuration): 512 x 512 interior + 32 PML cells per side
(576 x 576 = 331,776 unknowns), one seeded skull-ring velocity field with noise, 32 random point
sources solved together, 10 points per water wavelength.  Mixed path: FP32 complex Krylov basis
and stencil, BF16 U-Net preconditioner with FP32 accumulation, FP64 Givens / true residual /
iterative refinement.  One step = one batched solve of all 32 right-hand sides from x0 = 0.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl cuda|reference]

Prints one JSON line (rank 0).  Under torchrun every rank solves its own replica (weak scaling,
no collective on the data path); value = converged solves of all ranks / max elapsed time.
`--impl reference` times the CPU FP64 oracle (the project's reference implementation of the same
method) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WEIGHTS = os.path.join(ROOT, "paper_2607_16906_b300", "weights", "unet_paper_trained.npy")
METRIC = "Helmholtz solves/s to rel.res 1e-6: batched mixed vs plain FP64, same B300"
STENCIL_BYTES_FP32 = 16.0           # read z (8 B) + write A z (8 B) per point; k^2 (4 B/pt) read once per 32 RHS
# FGMRES iterations per right-hand side of this workload with the trained network, as measured by
# the CUDA arm (mean over the 32 RHS, FGMRES(128), up to 80 cycles); the reference arm, which
# runs in a process of its own, scales its measured per-iteration time by it (the CUDA arm prints its
# own measured mean)
REF_ITERS_PER_SOLVE = 4964
# DRAM bytes per basis vector and point of one DCGS2 step (k_dsweepA 8.00 B + k_dsweepB 8.06 B),
# from the ncu counters of the current sweep kernels
DCGS2_DRAM_B_PER_VPT = 16.06
# DRAM bytes of one application of the kind-1 network per full-resolution pixel (input packing and
# the eight tcgen05 layers, output layer fused), from the ncu counters of the current kernels on
# 4 RHS of this workload (None until measured)
PAPER_NET_DRAM_B_PER_PX = None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="cuda", choices=["cuda", "reference"])
    ap.add_argument("--m", type=int, default=128,
                    help="Krylov vectors per cycle (Sec. 4 uses 512; 128 is the fastest of 128..1024 measured with "
                         "the trained kind-1 network)")
    ap.add_argument("--max-outer", type=int, default=80,
                    help="FP64 refinement steps = FGMRES(m) cycles (budget m x 80 = 10,240 iterations per RHS)")
    ap.add_argument("--inner-tol", type=float, default=1e-5)
    ap.add_argument("--orth", default="dcgs2", choices=["cgs2", "dcgs2"])
    ap.add_argument("--nrhs", type=int, default=32)
    ap.add_argument("--rhs-batch", type=int, default=32, help="right-hand sides per solver call within a step")
    ap.add_argument("--weights", default=WEIGHTS)
    ap.add_argument("--no-plain", action="store_true", help="skip the plain-FP64 and identity comparators")
    ap.add_argument("--plain-rhs", type=int, default=1, help="right-hand sides of the plain-FP64 comparator")
    ap.add_argument("--ident-rhs", type=int, default=4, help="right-hand sides of the unpreconditioned comparator")
    ap.add_argument("--no-small", action="store_true", help="skip the small single-RHS configuration")
    ap.add_argument("--large", action="store_true",
                    help="also solve the large configuration (2176^2, line arrays, FP64 refinement to 1e-8)")
    ap.add_argument("--large-rhs", type=int, default=2)
    ap.add_argument("--large-m", type=int, default=256)
    ap.add_argument("--large-outer", type=int, default=60, help="refinement steps (cycles) of the large solve")
    ap.add_argument("--uneven", action="store_true", help="also solve the uneven 64-system batch in one call")
    ap.add_argument("--uneven-m", type=int, default=128)
    ap.add_argument("--uneven-outer", type=int, default=80, help="refinement steps (cycles) of the uneven solve")
    ap.add_argument("--only-extra", action="store_true",
                    help="skip the timed main workload: run only the legs asked for with --large / --uneven / "
                         "--fourier / --paper-net")
    ap.add_argument("--fourier", action="store_true", help="with --only-extra: the Fourier operator leg")
    ap.add_argument("--paper-net", action="store_true", help="with --only-extra: the kind-1 network leg")
    ap.add_argument("--train-leg", action="store_true", help="with --only-extra: the training-step leg")
    ap.add_argument("--train-steps", type=int, default=10, help="timed steps of the training-step leg")
    ap.add_argument("--extra-rhs", type=int, default=8, help="right-hand sides of the --fourier / --paper-net legs")
    ap.add_argument("--reps", type=int, default=10, help="timed repetitions of the --fourier / --paper-net legs")
    ap.add_argument("--no-cpu", action="store_true", help="skip the bounded CPU-oracle baseline")
    ap.add_argument("--no-train", action="store_true", help="skip the training-step throughput measurement")
    return ap.parse_args()


def load_weights(path, segments):
    from paper_2607_16906_b300 import synth
    if path and os.path.exists(path):
        return np.load(path), "trained in-repo by helm_train_step (" + os.path.basename(path) + ")"
    return synth.kaiming_uniform_params(segments, 42), "seeded Kaiming-uniform (untrained)"


def network_name(kind):
    """The network kind, named."""
    if kind == 1:
        return "kind 1: the paper's U-Net (5 inputs incl. PML sigma, 32 channels, 8x8 stride-2 convs, PReLU)"
    return "kind 0: 3-input 16/32/64/128 U-Net (3x3 convs, ReLU)"


def oracle_precond(theta, prob):
    """The oracle's FP64 network application z = M(v) for one right-hand side of `prob`."""
    from oracle import unet as ou
    from oracle import unet_paper as oup
    if theta.size == oup.param_count():
        return lambda v: oup.precondition(theta, v.reshape(1, prob.Ny, prob.Nx), prob.c, prob.p, prob.h,
                                          prob.omega)[0].ravel()
    return lambda v: ou.precondition(theta, v.reshape(1, prob.Ny, prob.Nx), prob.c, prob.h)[0].ravel()


def workload(nrhs, seed_offset=0):
    from paper_2607_16906_b300 import synth
    return synth.fine_multi_rhs_problem(seed=3000 + seed_offset, nrhs=nrhs)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    def __init__(self, index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.seek(0)
        return parse_clock_samples(self.f.read())


def parse_clock_samples(text):
    """Median SM clock under load (samples above half the highest), the maximum clock and the
    throttle reasons seen, from nvidia-smi rows `index, sm MHz, max MHz, power, active mask,
    hw_slowdown, hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap`."""
    rows = [r.split(",") for r in text.strip().splitlines() if r.strip()]
    sm, smax, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for r in rows:
        try:
            s_, m_ = float(r[1]), float(r[2])
            act = [r[5 + k].strip().lower() == "active" for k in range(len(names))]
        except (ValueError, IndexError):
            continue
        sm.append(s_)
        smax.append(m_)
        reasons.update(nm for nm, a in zip(names, act) if a)
    load = [s for s in sm if s > 0.5 * max(sm)] if sm else []
    return {"sm_mhz": statistics.median(load) if load else None, "sm_max_mhz": max(smax) if smax else None,
            "reasons": sorted(reasons), "samples": len(sm)}


def cpu_oracle_iteration_time(prob, theta, iters=5, basis=256):
    """Seconds per FGMRES iteration of the CPU FP64 oracle on one right-hand side of the workload at
    a Krylov basis of `basis` vectors: `iters` iterations of the oracle's own cycle (network, CSR
    stencil, CGS2 at j <= iters) plus, for the basis the cycle has not yet built, `iters` times the
    oracle's CGS2 arithmetic (two passes h = V^H w, w -= V h) on `basis` unit vectors."""
    from oracle import fgmres as fg
    from oracle import helmholtz as hz
    A = hz.assemble(prob.c, prob.p, prob.h, prob.omega)
    pre = oracle_precond(theta, prob)
    t0 = time.perf_counter()
    fg.cycle(lambda u: A @ u, pre, prob.b[0].ravel(), iters, 0.0)
    t_cycle = time.perf_counter() - t0
    rng = np.random.default_rng(0)
    V = rng.standard_normal((basis, prob.n)) + 1j * rng.standard_normal((basis, prob.n))
    V /= np.linalg.norm(V, axis=1, keepdims=True)
    w = rng.standard_normal(prob.n) + 0j
    t0 = time.perf_counter()
    for _ in range(iters):
        for _ in range(2):
            hh = np.conj(V @ np.conj(w))   # V^H w
            w = w - V.T @ hh
    t_orth = time.perf_counter() - t0
    return (t_cycle + t_orth) / iters


def splu_seconds(prob):
    """Sparse direct LU factorisation + one solve (the oracle's reference solution), seconds."""
    from oracle import helmholtz as hz
    A = hz.assemble(prob.c, prob.p, prob.h, prob.omega)
    t0 = time.perf_counter()
    hz.solve_direct(A, prob.b[0].ravel())
    return time.perf_counter() - t0


def bench_config(args, wdesc, world, kind):
    """The workload description both arms print."""
    return {"workload": "fine-grid multi-RHS: 512^2+32 PML (576^2), 32 point-source RHS, skull ring",
            "nrhs": args.nrhs, "rhs_per_call": max(1, min(args.rhs_batch, args.nrhs)), "m": args.m,
            "max_outer": args.max_outer, "orth": args.orth, "tol": 1e-6, "inner_tol": args.inner_tol, "ppw": 10,
            "weights": wdesc, "network": network_name(kind),
            "l2": "inputs and Krylov basis (GBs) larger than L2",
            "parallelism": f"replicas x{world}"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import unet as ou
    from oracle import unet_paper as oup
    prob = workload(args.nrhs)
    theta, wdesc = load_weights(args.weights, ou.param_segments())
    times = []
    for _ in range(args.warmup):
        cpu_oracle_iteration_time(prob, theta, iters=1, basis=32)
    for _ in range(args.steps):
        times.append(cpu_oracle_iteration_time(prob, theta, iters=2, basis=args.m // 2))
    t_it = statistics.median(times)
    val = 1.0 / (t_it * REF_ITERS_PER_SOLVE)
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_it * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(args, wdesc, 1, 1 if theta.size == oup.param_count() else 0),
            "cpu_baseline": {"value": val, "unit": "solves/s", "cores": cores, "kind": "oracle",
                             "sample": f"2 FGMRES iterations of one RHS per step (numpy FP64 U-Net, CSR stencil, "
                                       f"CGS2 at the mean basis {args.m // 2}), extrapolated by {REF_ITERS_PER_SOLVE} "
                                       f"iterations per solve (the CUDA arm's measured mean)"},
            "e2e": {"value": val, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def measured_solve(helm, ctx, net, prob, nrhs, kw, what):
    """Solve the first `nrhs` right-hand sides of the workload from x0 = 0 and time it (CUDA events)."""
    import torch
    b = torch.tensor(prob.b[:nrhs].ravel(), device="cuda")
    x = torch.zeros_like(b)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = helm.helm_launch_count()
    e0.record()
    _, info = helm.helm_fgmres_solve(ctx, net, b, x, nrhs, **kw)
    e1.record()
    torch.cuda.synchronize()
    s = e0.elapsed_time(e1) / 1e3
    conv = sum(1 for c in info if c["status"] == "OK")
    its = [c["iters"] for c in info]
    return {"what": what, "rhs": nrhs, "converged": conv, "seconds": s, "solves_per_s": conv / s,
            "iters": its, "mean_iters": float(np.mean(its)), "relres_true_max": max(c["relres_true"] for c in info),
            "launches": helm.helm_launch_count() - l0, "opts": {k: v for k, v in kw.items()}}


def small_configuration(helm, theta_trained):
    """The small single-RHS configuration: 128^2 interior + 16 PML (160^2), one skull, one point
    source, FGMRES(30), tol 1e-6, at most 100 cycles.  Plain FP64 with the seeded (untrained) network
    as specified for this configuration and with the trained one, the mixed path with the trained
    network (median of 3 timed solves), and unpreconditioned GMRES."""
    import torch
    from paper_2607_16906_b300 import synth
    prob = synth.small_problem(seed=1000)
    spec = helm.SystemSpec(prob.nx, prob.ny, prob.h, prob.p, prob.omega)
    ctx = helm.Context([spec], torch.tensor(prob.c.ravel(), device="cuda"))
    trained = helm.UNet(theta_trained)
    segs = helm.weight_segments() if trained.kind == 0 else helm.paper_weight_segments()
    seeded = helm.UNet(synth.kaiming_uniform_params(segs, 42), kind=trained.kind)
    # (network, options, timed repetitions): the slow FP64 runs once (after a short warm-up solve)
    runs = {"plain_fp64_seeded_net": (seeded, dict(m=30, tol=1e-6, mixed=False, max_restarts=100, orth="dcgs2"), 1),
            "plain_fp64_trained_net": (trained, dict(m=30, tol=1e-6, mixed=False, max_restarts=100, orth="dcgs2"), 1),
            "mixed_trained_net": (trained, dict(m=30, tol=1e-6, mixed=True, max_outer=100, inner_tol=1e-5,
                                                orth="dcgs2"), 3),
            "gmres_identity": (None, dict(m=30, tol=1e-6, mixed=True, max_outer=100, inner_tol=1e-5,
                                          orth="dcgs2"), 1)}
    out = {"workload": "128^2+16 PML (160^2), 1 skull, 1 point source, FGMRES(30), tol 1e-6, <= 100 cycles"}
    for name, (net, kw, reps) in runs.items():
        warm = dict(kw)
        warm.update(max_restarts=1, max_outer=1)
        measured_solve(helm, ctx, net, prob, 1, warm, name)  # warm-up (graphs, tile tuning)
        rs = sorted((measured_solve(helm, ctx, net, prob, 1, kw, name) for _ in range(reps)),
                    key=lambda d: d["seconds"])
        r = rs[len(rs) // 2]
        r["launches_per_iter"] = r["launches"] / max(1, r["mean_iters"])
        out[name] = r
    return out


def timed_flushed(fn, reps=10):
    """Mean CUDA-event time (ms) of fn over `reps` launches after 3 untimed ones, each preceded by an
    L2 flush (a 256 MB write, then a 256 MB read of another buffer)."""
    import torch
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    flush_r = torch.ones(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    tot = 0.0
    for it in range(reps + 3):
        flush.fill_(it)
        flush_r.sum()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record()
        fn()
        a1.record()
        torch.cuda.synchronize()
        if it >= 3:
            tot += a0.elapsed_time(a1)
    return tot / max(1, reps)


def fourier_leg(helm, h, omega, peaks, nrhs=8, reps=10):
    """The paper's discretisation: the Fourier-differentiation operator (FP32) on a 1024^2 grid (the
    largest power-of-two side, 1008^2 + 8 PML) x `nrhs` RHS against its algorithmic 52 B per point
    (row pass 16 B, column pass 36 B)."""
    import torch
    from paper_2607_16906_b300 import synth as sy
    c = sy.skull_velocity(1008, 1008, 8, sy.rng_for(77))
    fctx = helm.Context([helm.SystemSpec(1008, 1008, h, 8, omega)], torch.tensor(c.ravel(), device="cuda"))
    fx = torch.randn(fctx.npts * nrhs, dtype=torch.complex64, device="cuda")
    fy = torch.empty_like(fx)
    f_ms = timed_flushed(lambda: helm.helm_apply_fourier(fctx, fx, fy, nrhs), reps)
    f_bytes = 52.0 * fctx.npts * nrhs
    hbm = peaks.get("hbm_gbs", 6400.0)
    return {"bound": "hbm", "achieved": f_bytes / (f_ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
            "frac": f_bytes / (f_ms / 1e3) / 1e9 / hbm, "ms": f_ms, "bytes_per_launch": f_bytes,
            "kernels": f"k_fourier_x + k_fourier_y (FP32, 1024^2 x {nrhs} RHS)", "l2": "flushed before each launch"}


# Network kind 1, MACs per full-resolution pixel.  Algorithmic: 8x8 down layers 64 C_in 32 per output
# pixel at 1/4, 1/16, 1/64, 1/256 of the pixels (C_in = 5, 32, 32, 32), up layers 64 C_in 32 per input
# pixel at 1/256, 1/64, 1/16, 1/4 (C_in = 32, 64, 64, 64), output layer 32 x 2: 51,264.  Executed on
# the tensor cores (structural zeros included): enc1..enc3 9 taps x K x 128 columns at 1/16, 1/64,
# 1/256 (K = 128, 512, 512), enc4 25 x 128 x 32 at 1/256, up layers 25 x K x 128 at 1/256, 1/64, 1/16,
# 1/4 (K = 32, 64, 64, 64), output layer: 88,800.
PAPER_NET_ALG_MACS = (64 * 32 * (5 / 4 + 32 * (1 / 16 + 1 / 64 + 1 / 256)) +
                      64 * 32 * (32 / 256 + 64 / 64 + 64 / 16 + 64 / 4) + 64)
PAPER_NET_EXE_MACS = (9 * 128 * 128 / 16 + 9 * 512 * 128 * (1 / 64 + 1 / 256) + 25 * 128 * 32 / 256 +
                      25 * 128 * (32 / 256 + 64 / 64 + 64 / 16 + 64 / 4) + 64)


def paper_net_leg(helm, ctx, nrhs, peaks, reps=5):
    """The paper's U-Net variant (network kind 1, seeded weights): one BF16 application to `nrhs`
    right-hand sides of the context, against the measured burst BF16 rate on the algorithmic flops of
    the 8x8 layers and the output layer (51,264 MAC per full-resolution pixel) and on the flops the
    tensor cores execute (88,800 MAC, structural zeros included: enc1..enc3 as 3x3 convolutions over
    4 x 4 input blocks, enc4 and the decoder as 5x5 convolutions)."""
    import torch
    from paper_2607_16906_b300 import synth as sy
    pn = helm.UNet(sy.kaiming_uniform_params(helm.paper_weight_segments(), 42), kind=1)
    pv = torch.randn(ctx.npts * nrhs, dtype=torch.complex64, device="cuda")
    pz = torch.empty_like(pv)
    helm.helm_precond_apply(ctx, pn, pv, pz, nrhs)
    p_ms = timed_flushed(lambda: helm.helm_precond_apply(ctx, pn, pv, pz, nrhs), reps)
    alg, exe = PAPER_NET_ALG_MACS, PAPER_NET_EXE_MACS
    pk = peaks.get("bf16_tflops", 1800.0)
    px = ctx.npts * nrhs
    a_tf = 2.0 * alg * px / (p_ms / 1e3) / 1e12
    e_tf = 2.0 * exe * px / (p_ms / 1e3) / 1e12
    return {"bound": "tensor", "achieved": a_tf, "peak": pk, "unit": "TFLOP/s", "frac": a_tf / pk, "ms": p_ms,
            "flop_per_pixel": 2.0 * alg, "executed_flop_per_pixel": 2.0 * exe, "executed_frac": e_tf / pk,
            "what": f"network kind 1 (the paper's variant), BF16 on tcgen05, {nrhs} RHS; frac on the 8x8 layers' "
                    "algorithmic flops, executed_frac on the GEMM flops run (structural zeros included)",
            "peak_source": "measured burst bf16 (MEASURED_PEAKS.json)"}


def train_leg(helm, theta, steps=10):
    """Training-step throughput on the training configuration (64 x (128^2 + 16 PML), mixed skull /
    GRF velocities, point-source and line-array sources): helm_train_step = network forward, adjoint
    stencil, conv backward, AdamW (eqs. 8-9) for the weights' network kind; 3 warm-up and `steps`
    timed steps on a copy of the weights."""
    import torch
    from paper_2607_16906_b300 import synth
    cs, bs, th, om = synth.training_batch()
    nb, nt = cs.shape[0], cs.shape[1] - 32
    tctx = helm.Context([helm.SystemSpec(nt, nt, th, 16, om) for _ in range(nb)],
                        torch.tensor(cs.ravel(), device="cuda"))
    tnet = helm.UNet(theta)
    tb = torch.tensor(bs.ravel().astype(np.complex64), device="cuda")
    for _ in range(3):
        helm.helm_train_step(tctx, tnet, tb, lr=1e-5)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record()
    losses = [helm.helm_train_step(tctx, tnet, tb, lr=1e-5)[0] for _ in range(steps)]
    t1.record()
    torch.cuda.synchronize()
    tms = t0.elapsed_time(t1) / steps
    return {"steps_per_s": 1e3 / tms, "ms_per_step": tms, "samples_per_s": nb * 1e3 / tms,
            "network_kind": tnet.kind,
            "batch": f"{nb} x {nt}^2 + 16 PML (skull / GRF velocities, point / line-array sources)",
            "loss_first": losses[0], "loss_last": losses[-1]}


def large_configuration(helm, theta, nrhs, m, max_outer=60):
    """The large configuration: 2048^2 interior + 64 PML (2176^2, 4.7 M unknowns), 12 points per
    wavelength, thin skull ring, line-array sources; mixed path with FP64 refinement to eta_b <= 1e-8.
    FGMRES(m) with m = `m` and up to `max_outer` cycles (the configuration names FGMRES(50); the kind-0
    network stalls with restarts of 256 or less, the kind-1 network does not on the 576^2 workload);
    `nrhs` of the 8 right-hand sides.  The plain FP64 path is timed over 3 iterations and
    extrapolated to the mixed path's count (labelled)."""
    import torch
    from paper_2607_16906_b300 import synth
    prob = synth.large_problem(seed=5000, nrhs=nrhs)
    spec = helm.SystemSpec(prob.nx, prob.ny, prob.h, prob.p, prob.omega)
    ctx = helm.Context([spec], torch.tensor(prob.c.ravel(), device="cuda"))
    net = helm.UNet(theta)
    measured_solve(helm, ctx, net, prob, nrhs, dict(m=4, tol=1e-300, mixed=True, max_outer=1), "warm-up")
    helm.helm_profile_enable(ctx, True)
    r = measured_solve(helm, ctx, net, prob, nrhs, dict(m=m, tol=1e-8, mixed=True, max_outer=max_outer, inner_tol=1e-5,
                                                        orth="dcgs2"),
                       "mixed path, FP64 refinement to 1e-8")
    prof = helm.helm_profile_read(ctx)
    work = helm.helm_profile_work(ctx)
    helm.helm_profile_enable(ctx, False)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm = peaks.get("hbm_gbs", 6400.0)
    r["phases_ms"] = {k: v[0] for k, v in prof.items()}
    if prof["orth"][0] > 0:
        gbs = work["orth"] / (prof["orth"][0] / 1e3) / 1e9
        r["orth_roofline"] = {"achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm}
    if prof["stencil"][0] > 0:
        gbs = work["stencil"] / (prof["stencil"][0] / 1e3) / 1e9
        r["stencil_roofline"] = {"achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm}
    p = measured_solve(helm, ctx, net, prob, nrhs, dict(m=3, tol=1e-300, mixed=False, max_restarts=1, orth="dcgs2"),
                       "plain FP64, 3 iterations")
    per_it = p["seconds"] / 3
    r["plain_fp64_extrapolated"] = {"s_per_iter": per_it, "solves_per_s": nrhs / (per_it * max(1.0, r["mean_iters"])),
                                    "sample": "3 FP64 iterations of all RHS (FP64 U-Net on CUDA cores) x the mixed "
                                              "path's mean iteration count (extrapolated)"}
    r["workload"] = f"2048^2+64 PML (2176^2), PPW 12, thin skull ring, {nrhs} of 8 line-array RHS, FGMRES({m})"
    return r


def uneven_configuration(helm, theta, m, max_outer=80):
    """The uneven batch: 64 systems with sides drawn from {256..1024} + PML 16..32 and 8-12 points per
    wavelength, one point source each, all in one context and one solver call (mixed path, FGMRES(m),
    up to `max_outer` cycles, tol 1e-6).  Reports converged systems, iterations and launches per
    iteration."""
    import torch
    from paper_2607_16906_b300 import synth
    probs = synth.uneven_problems()
    specs = [helm.SystemSpec(p.nx, p.ny, p.h, p.p, p.omega) for p in probs]
    ctx = helm.Context(specs, torch.tensor(np.concatenate([p.c.ravel() for p in probs]), device="cuda"))
    net = helm.UNet(theta)
    b = torch.tensor(np.concatenate([p.b.ravel() for p in probs]), device="cuda")
    x = torch.zeros_like(b)
    helm.helm_fgmres_solve(ctx, net, b, x, 1, m=4, tol=1e-300, mixed=True, max_outer=1)  # warm-up
    x.zero_()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = helm.helm_launch_count()
    e0.record()
    _, info = helm.helm_fgmres_solve(ctx, net, b, x, 1, m=m, tol=1e-6, mixed=True, max_outer=max_outer, inner_tol=1e-5,
                                     orth="dcgs2")
    e1.record()
    torch.cuda.synchronize()
    s = e0.elapsed_time(e1) / 1e3
    conv = [c["status"] == "OK" for c in info]
    its = [c["iters"] for c in info]
    by_side = {}
    for p, c, it in zip(probs, conv, its):
        d = by_side.setdefault(p.nx, {"systems": 0, "converged": 0, "iters": []})
        d["systems"] += 1
        d["converged"] += int(c)
        d["iters"].append(it)
    for d in by_side.values():
        d["mean_iters"] = float(np.mean(d.pop("iters")))
    launches = helm.helm_launch_count() - l0
    return {"workload": "64 systems, sides {256..1024} + PML 16..32, PPW 8-12, 1 point source each, one call",
            "m": m, "converged": int(sum(conv)), "systems": len(probs), "seconds": s, "solves_per_s": sum(conv) / s,
            "mean_iters": float(np.mean(its)), "max_iters": int(max(its)), "launches": launches,
            "launches_per_iter": launches / max(1, max(its)), "by_side": by_side,
            "points": int(sum(p.n for p in probs))}


def run_cuda(args):
    import torch
    from paper_2607_16906_b300 import helm, replicas, synth

    rank, world, local = replicas.env_ranks()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if args.only_extra:  # the large / uneven configurations alone (rank 0), no timed main workload
        if rank == 0:
            theta, wdesc = load_weights(args.weights, helm.weight_segments())
            out = {"metric": METRIC, "extra_legs_only": True, "weights": wdesc}
            if args.large:
                out["large_2176"] = large_configuration(helm, theta, args.large_rhs, args.large_m, args.large_outer)
            if args.uneven:
                out["uneven_64"] = uneven_configuration(helm, theta, args.uneven_m, args.uneven_outer)
            if args.train_leg:
                out["train_step"] = train_leg(helm, theta, args.train_steps)
            peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
                os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
            if args.fourier or args.paper_net:
                fp = workload(1)
                if args.fourier:
                    out["fourier_roofline"] = fourier_leg(helm, fp.h, fp.omega, peaks, args.extra_rhs, args.reps)
                if args.paper_net:
                    fspec = helm.SystemSpec(fp.nx, fp.ny, fp.h, fp.p, fp.omega)
                    fctx = helm.Context([fspec], torch.tensor(fp.c.ravel(), device="cuda"))
                    out["paper_unet"] = paper_net_leg(helm, fctx, args.extra_rhs, peaks, args.reps)
            print(json.dumps(out), flush=True)
        if dist:
            dist.destroy_process_group()
        return
    prob = workload(args.nrhs, seed_offset=rank)
    nrhs = args.nrhs
    spec = helm.SystemSpec(prob.nx, prob.ny, prob.h, prob.p, prob.omega)
    ctx = helm.Context([spec], torch.tensor(prob.c.ravel(), device="cuda"))
    theta, wdesc = load_weights(args.weights, helm.weight_segments())
    net = helm.UNet(theta)
    b = torch.tensor(prob.b.ravel(), device="cuda")
    x = torch.zeros_like(b)
    opts = dict(m=args.m, tol=1e-6, mixed=True, max_outer=args.max_outer, inner_tol=args.inner_tol, orth=args.orth)
    rb = max(1, min(args.rhs_batch, nrhs))
    nsub = (nrhs + rb - 1) // rb

    def solve_all(bb, xx):
        """All right-hand sides of the step, `rb` per solver call (the Krylov basis of rb columns fits HBM)."""
        info = []
        for k in range(nsub):
            r0, r1 = k * rb, min(nrhs, (k + 1) * rb)
            sl = slice(r0 * prob.n, r1 * prob.n)
            xs = xx[sl]
            xs.zero_()
            _, inf = helm.helm_fgmres_solve(ctx, net, bb[sl], xs, r1 - r0, **opts)
            info += inf
        return info

    def step():
        return 0, solve_all(b, x)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    replicas.barrier(dev)
    helm.helm_profile_enable(ctx, True)
    clocks = ClockSampler(local)
    l0 = helm.helm_launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record()
    converged, iters, infos = 0, [], []
    for _ in range(args.steps):
        rc, info = step()
        converged += sum(1 for c in info if c["status"] == "OK")
        iters += [c["iters"] for c in info]
        infos = info
    ev1.record()
    torch.cuda.synchronize()
    replicas.barrier(dev)
    launches = helm.helm_launch_count() - l0
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    prof = helm.helm_profile_read(ctx)
    work = helm.helm_profile_work(ctx)
    helm.helm_profile_enable(ctx, False)
    ms, converged = replicas.reduce_step(ms, converged, dev)  # max time, summed solves over ranks
    value = converged / (ms / 1e3)
    mean_iters = float(np.mean(iters)) if iters else 0.0

    # end to end through the public API: pinned host b -> device, solve, device x -> pinned host
    b_host = torch.tensor(prob.b.ravel()).pin_memory()
    x_host = torch.empty_like(b_host).pin_memory()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    conv_e2e = 0
    e2e_steps = 1  # one full step (a step is a whole batched solve: tens of seconds)
    for _ in range(e2e_steps):
        bd = b_host.to("cuda", non_blocking=True)
        xd = torch.zeros_like(bd)
        info = solve_all(bd, xd)
        x_host.copy_(xd, non_blocking=True)
        conv_e2e += sum(1 for c in info if c["status"] == "OK")
    e1.record()
    torch.cuda.synchronize()
    ms_e2e = e0.elapsed_time(e1)
    ms_e2e, conv_e2e = replicas.reduce_step(ms_e2e, conv_e2e, dev)
    nbytes = b_host.numel() * b_host.element_size()

    # dominant phase -> roofline (algorithmic work counted by the library for the timed region)
    peaks = {}
    pk_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk_path):
        peaks = json.load(open(pk_path))
    dom = max(prof, key=lambda k: prof[k][0])
    phase_rooflines = {}
    for ph in ("precond", "stencil", "orth"):
        t_s = prof[ph][0] / 1e3
        if t_s <= 0 or work[ph] <= 0:
            continue
        if ph == "precond":
            ach = work[ph] / t_s / 1e12
            pk = peaks.get("bf16_tflops_sustained", 1400.0)
            phase_rooflines[ph] = {"bound": "tensor", "achieved": ach, "peak": pk, "unit": "TFLOP/s",
                                   "frac": ach / pk, "ms": prof[ph][0]}
        else:
            ach = work[ph] / t_s / 1e9
            pk = peaks.get("hbm_gbs", 6400.0)
            phase_rooflines[ph] = {"bound": "hbm", "achieved": ach, "peak": pk, "unit": "GB/s", "frac": ach / pk,
                                   "ms": prof[ph][0]}
    names = {"precond": "U-Net preconditioner (tcgen05 BF16 convs + CUDA-core glue), all launches of the step",
             "orth": f"{args.orth.upper()} orthogonalisation sweeps (k_dsweepA/k_dsweepB or k_mdot/k_maxpy)",
             "stencil": "k_stencil_tma<float>"}
    roof = dict(phase_rooflines.get(dom, {"bound": "hbm", "achieved": None, "peak": None, "unit": "GB/s",
                                          "frac": None}))
    roof.update({"kernel": names.get(dom, dom), "traffic": None,
                 "peak_source": "measured (MEASURED_PEAKS.json)" if peaks else "fallback"})
    if dom == "precond" and net.kind == 1 and prof["precond"][1] > 0:
        # one "launch" of the preconditioner = one network application to the solver call's columns
        npx = ctx.npts * rb
        roof.update({"traffic": PAPER_NET_DRAM_B_PER_PX * npx if PAPER_NET_DRAM_B_PER_PX else None,
                     "algorithmic_per_application": work["precond"] / prof["precond"][1],
                     "applications": prof["precond"][1],
                     "traffic_source": "ncu DRAM bytes of one application's kernels per pixel x pixels"})
    if dom == "orth" and args.orth == "dcgs2" and prof["orth"][1] > 0:
        # one "launch" of the orthogonalisation = one DCGS2 step (sweep A + sweep B + 3 small
        # kernels); its algorithmic bytes are 16 nv + 48 B per point, nv the step's basis size
        npt = ctx.npts * rb  # points per solver call
        alg_step = work["orth"] / prof["orth"][1]
        nv_mean = max(0.0, (alg_step / npt - 48.0) / 16.0)
        roof.update({"traffic": DCGS2_DRAM_B_PER_VPT * nv_mean * npt, "algorithmic_per_step": alg_step,
                     "mean_basis": nv_mean, "steps": prof["orth"][1],
                     "traffic_source": "ncu DRAM bytes per basis-vector point x mean basis size"})

    # stencil alone against HBM (32 RHS of the workload).  L2 is flushed before every launch by
    # writing one 256 MB buffer and then reading another, so that the write-back of the flush's
    # dirty lines happens before the timed launch rather than inside it.
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    flush_r = torch.ones(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    z32 = torch.randn(ctx.npts * nrhs, dtype=torch.complex64, device="cuda")
    w32 = torch.empty_like(z32)
    tot = 0.0
    for it in range(13):
        flush.fill_(it)
        flush_r.sum()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record()
        helm.helm_apply(ctx, z32, w32, nrhs)
        s1.record()
        torch.cuda.synchronize()
        if it >= 3:
            tot += s0.elapsed_time(s1)
    st_ms = tot / 10
    st_bytes = STENCIL_BYTES_FP32 * ctx.npts * nrhs + 4.0 * ctx.npts
    st_gbs = st_bytes / (st_ms / 1e3) / 1e9
    hbm = peaks.get("hbm_gbs", 6400.0)
    stencil = {"bound": "hbm", "achieved": st_gbs, "peak": hbm, "unit": "GB/s", "frac": st_gbs / hbm,
               "ms": st_ms, "bytes_per_launch": st_bytes, "kernel": "k_stencil_tma<float> (FP32, 32 RHS)",
               "l2": "flushed before each launch (write 256 MB, read 256 MB)",
               "tile": [t for t in helm.helm_tuned_stencil() if t["nrhs"] == nrhs]}

    fourier = fourier_leg(helm, prob.h, prob.omega, peaks) if rank == 0 else None
    paper_net = paper_net_leg(helm, ctx, nrhs, peaks) if rank == 0 else None

    train = train_leg(helm, theta, args.train_steps) if rank == 0 and not args.no_train else None

    # comparators of the metric, measured to the same tolerance on a stated subset of the same
    # right-hand sides: the plain FP64 GPU path (FP64 basis, stencil and network) and unpreconditioned
    # GMRES (mixed path without the network), both with the same FGMRES(m) and cycle budget
    plain = ident = small = None
    if rank == 0 and not args.no_plain:
        plain = measured_solve(helm, ctx, net, prob, args.plain_rhs,
                               dict(m=args.m, tol=1e-6, mixed=False, max_restarts=args.max_outer, orth=args.orth),
                               "plain FP64 GPU path: FP64 Krylov basis and stencil, FP64 U-Net on CUDA cores, "
                               "FP64 Givens")
        ident = measured_solve(helm, ctx, None, prob, args.ident_rhs, dict(opts),
                               "unpreconditioned GMRES (z_j = v_j), mixed path, same m and cycle budget")
    if rank == 0 and not args.no_small:
        small = small_configuration(helm, theta)
    large = large_configuration(helm, theta, args.large_rhs, args.large_m, args.large_outer) if rank == 0 and args.large else None
    uneven = uneven_configuration(helm, theta, args.uneven_m, args.uneven_outer) if rank == 0 and args.uneven else None
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:  # the CPU baseline is quoted at N = 1 only
        from oracle import unet as ou  # the bounded CPU-oracle baseline leg
        th_o, _ = load_weights(args.weights, ou.param_segments())
        t_it = cpu_oracle_iteration_time(prob, th_o, iters=5, basis=args.m // 2)
        t_lu = splu_seconds(prob)
        cpu = {"value": 1.0 / (t_it * max(mean_iters, 1.0)), "unit": "solves/s", "cores": os.cpu_count(),
               "kind": "oracle", "sample": f"5 FGMRES iterations of one RHS ({t_it:.2f} s each: numpy FP64 U-Net, "
                                           f"CSR stencil, CGS2 at the mean basis {args.m // 2}), extrapolated to "
                                           f"the measured {mean_iters:.0f} iterations per solve",
               "splu_s_per_system": t_lu, "splu": "scipy SuperLU factorisation + solve of the 576^2 system (the "
                                                  "oracle's reference solution; not an iterative baseline)"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "c64/bf16 (f64 refinement)", "data": "synthetic",
                "config": bench_config(args, wdesc, world, net.kind),
                "converged": converged, "columns": args.steps * nrhs * world,
                "mean_iters_per_solve": mean_iters,
                "relres_true_max": max(c["relres_true"] for c in infos) if infos else None,
                "phases_ms": {k: v[0] for k, v in prof.items()},
                "roofline": roof, "phase_rooflines": phase_rooflines, "phase_work": work,
                "stencil_roofline": stencil, "fourier_roofline": fourier, "paper_unet": paper_net,
                "plain_fp64": plain, "gmres_identity": ident, "small_160": small, "train_step": train,
                "large_2176": large, "uneven_64": uneven,
                "launches_per_iter": launches / max(1.0, sum(iters) / max(1, nrhs)),
                "autotune": [f"{t['c_out']}<-{8 * t['slices']} {t['images']}x{t['H']}x{t['W']}: RY={t['rows_per_tile']}"
                             for t in helm.helm_tuned_tiles()],
                "cpu_baseline": cpu, "clocks": clk, "gpu_launches": launches,
                "e2e": {"value": conv_e2e / (ms_e2e / 1e3), "unit": "solves/s", "h2d_bytes_per_step": nbytes,
                        "d2h_bytes_per_step": nbytes, "steps": e2e_steps}}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_cuda(args)


if __name__ == "__main__":
    main()
