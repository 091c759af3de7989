"""Host-side parts of the benchmark that need no GPU: the clock-sample parser and the reference
arm's JSON line (the CPU oracle timed on the host cores)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_clock_samples_parse():
    text = "\n".join([
        "0, 2032, 2032, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1965, 2032, 1100.2, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 345, 2032, 150.0, 0x0, Not Active, Not Active, Not Active, Not Active",   # idle sample
        "garbage line",
        "0, 2032, 2032, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ])
    r = bench.parse_clock_samples(text)
    assert r["samples"] == 4 and r["sm_max_mhz"] == 2032.0
    assert r["sm_mhz"] == 2032.0          # median of the three samples under load
    assert r["reasons"] == ["sw_power_cap"]
    assert bench.parse_clock_samples("")["sm_mhz"] is None


def test_reference_arm_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == "solves/s"
    assert line["value"] > 0 and line["higher_is_better"] is True
    assert line["config"]["workload"].startswith("fine-grid multi-RHS")
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]


def test_network_flop_accounting_matches_the_oracle_network():
    """The algorithmic MACs per full-resolution pixel the bench reports network kind 1 against (Sec. 3.1,
    Tab. 2) equal a count over the shapes of the oracle's forward pass on a 32 x 32 input: an 8x8
    strided layer does 64 C_in C_out per output pixel, a transposed one 64 C_in C_out per input pixel,
    the 1x1 output layer C_in C_out per pixel."""
    import numpy as np
    from oracle import unet_paper as up
    from paper_2607_16906_b300 import synth
    theta = synth.kaiming_uniform_params(up.param_segments(), 42)
    x = synth.rng_for(5).standard_normal((1, 5, 32, 32))
    _, act = up.forward(theta, x, keep=True)
    macs = 0
    for name, kind, ci, co in up.LAYERS:
        xin, pre = act[name]
        assert xin.shape[1] == ci
        if kind == "down":
            macs += pre.shape[2] * pre.shape[3] * 64 * ci * co
        elif kind == "up":
            macs += xin.shape[2] * xin.shape[3] * 64 * ci * co
        else:
            macs += xin.shape[2] * xin.shape[3] * ci * co
    assert macs / (32 * 32) == bench.PAPER_NET_ALG_MACS == 51264
    # every executed product of the reformulated GEMMs is a product of the 8x8 layers or a structural zero
    assert bench.PAPER_NET_EXE_MACS >= bench.PAPER_NET_ALG_MACS
