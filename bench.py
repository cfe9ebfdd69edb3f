#!/usr/bin/env python3
"""Benchmark of the N-body/SPH step: particle-steps/s (gravity + SPH).

Workload (default, the largest single-GPU configuration): the 2^24-particle
disk model -- 90 % stars in an exponential disk (R_d = 1, z_d = 0.1), 10 % gas
(R_d = 2, u log-uniform in [1e-3, 1e-1]) in a static NFW halo (r_s = 8,
M_s = 30), G = 1, eps = 0.01, Barnes-Hut tree gravity with theta = 0.5 and
monopole + quadrupole, 64 SPH neighbours, kick-drift-kick steps of
dt = 1e-3, with the energy and momentum drift over 20 steps (the timed
steps, continued untimed to 20 when fewer were timed; --config disk: the
2^20 disk with 20 % gas, drift over 10 steps).  A step is one full KDK step
through the C ABI (tree build, gravity, halo, kernel size, density, force,
kicks, drift).  Inputs are resident in HBM when the timed region starts; L2 is
flushed (256 MiB write on the same stream) before every timed step.  Besides
the gravity kernel's FP32 roofline, the line reports the HBM fraction of the
tree build (sort + octree + moments + hydro tree) and of the two SPH passes
against their algorithmic bytes.

The same JSON line carries the supernova half of the metric under "sn"
(rank 0, one GPU): SN regions per second of the surrogate path (256 ragged
regions of 2e4 - 3e5 gas particles, log-uniform, voxelised to 64^3, BF16 U-Net
forward, Gibbs remap, one CUDA-graph replay per batch) against the plain
CFL-limited integration of 1e5-particle regions over 0.1 Myr on the same GPU
(one region alone, 32 regions in one context, and with hierarchical
individual timesteps), with the trained network's field error on held-out
seeds computed in the same run and the U-Net forward's tensor throughput
against the measured BF16 peak.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--no-sn]

With N > 1 (torchrun) every rank runs an independent replica on its own GPU
(the step has no exchange on one GPU; replicas only) and rank 0 prints the
whole-job value from the max time over ranks.  ``--impl reference`` times the
FP64 CPU checker on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2510_23330_gb300 import ics  # noqa: E402

METRIC = "particle-steps/s (grav+SPH)"
UNIT = "particle-steps/s"
# FP32 peak: 152 SMs x 128 FP32 lanes x 2 flop (FMA) x 2070 MHz maximum SM clock
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
# flops per interaction: the paper's count for the monopole pair (Table 4),
# and this library's own count for the quadrupole particle-cell term
FLOP_PP = 27
FLOP_PC = 59
# U-Net forward per 64^3 region: 3^3 convolutions, transposed convolutions
# and the head with the network's own 5 input channels (algorithmic count)
UNET_GFLOP_64 = 29.0497
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
# Algorithmic bytes per unit of the HBM-bound phases:
#  tree build, per particle: positions read 24 + key write 8 + 4 radix passes
#    of (key, index) read and written 4 x 24 + the permutation of ~48 B of
#    state read and written 96 + node build 8 + moments 28 = 260 B;
#  kNN + density, per gas particle: state read 28 + neighbour list written
#    256 + h^2 8, then state 40 + list read 256 + rho/P/c written 12 = 600 B;
#  hydro force, per gas particle: state 56 + symmetric list ~4 x 66 +
#    results 16 = ~390 B (neighbour state re-reads hit L2 in Morton order).
BYTES_TREE_PER_PARTICLE = 260
BYTES_KNN_DENSITY_PER_GAS = 600
BYTES_FORCE_PER_GAS = 390


def workload(name: str, seed: int):
    if name == "disk":
        n = 1 << 20
        p = ics.config_disk(n, gas_frac=0.2, seed=seed)
        desc = "disk-2^20: 838,861 stars + 209,715 gas, NFW halo, tree theta=0.5 quad, 64 NN, KDK dt=1e-3"
    elif name == "large":
        n = 1 << 24
        p = ics.config_disk(n, gas_frac=0.1, seed=seed)
        desc = "disk-2^24: 15,099,494 stars + 1,677,722 gas, NFW halo, tree theta=0.5 quad, 64 NN, KDK dt=1e-3"
    elif name == "tiny":
        n = 8192
        p = ics.config_tiny(seed)
        desc = "plummer-8192: 4,096 stars + 4,096 gas, direct-sum gravity, 64 NN, KDK dt=1e-3"
    else:
        raise SystemExit(f"unknown config {name}")
    return p, desc


def params(name):
    if name == "tiny":
        return dict(gravity=0, cfg={})
    return dict(gravity=1, cfg=dict(nfw_ms=ics.NFW_MS, nfw_rs=ics.NFW_RS, theta=0.5, multipole=1,
                                    n_leaf=16, n_group=64))


class ClockSampler:
    """nvidia-smi samples (every 20 ms) tagged with host time."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.samples = []
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "20"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.perf_counter(), [s.strip() for s in line.split(",")]))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, t0, t1):
        if not self.proc:
            return None
        win = [s for t, s in self.samples if t0 <= t <= t1] or [s for t, s in self.samples[-3:]]
        if not win:
            return None
        sm = [float(s[0]) for s in win if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in win if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in win for k in range(4) if len(s) > 4 + k and s[4 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(win)}


def gravity_traffic(config):
    """DRAM bytes per gravity launch of the full workload, from the committed
    ncu summary of that workload's gravity kernels, if the kernel source is
    unchanged since the capture (else None)."""
    name = {"disk": "gravity_tree_disk2p20.txt", "large": "gravity_tree_disk2p24.txt"}.get(config)
    if name is None:
        return None
    path = os.path.join(ROOT, "profiles", name)
    src = os.path.join(ROOT, "paper_2510_23330_gb300", "csrc", "gravity.cu")
    try:
        text = open(path).read()
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    vals = dict(line.split(":", 1) for line in text.splitlines() if ":" in line and not line.startswith("#"))
    if vals.get("source_sha256_16", "").strip() != sha:
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def cpu_baseline(p, name, knn_seconds=6.0, n_g=64, n_leaf=16):
    """The FP64 oracle on a bounded sample of one force evaluation (about
    15-25 s of CPU work): the full tree build plus every k-th group's walk
    (k = N / 2^18, scaled by k) and brute-force kNN of as many sampled gas
    particles as take about knn_seconds (scaled to all gas)."""
    import oracle
    oracle.build()
    n = p["x"].shape[0]
    gi = np.nonzero(p["type"] == 1)[0]
    stride = max(1, n >> 18)
    t0 = time.perf_counter()
    tb, tw, st = oracle.tree_gravity_sampled(p, stride, theta=0.5, n_leaf=n_leaf, n_g=n_g, quad=True)
    t_grav = tb + tw * stride
    g = {k: np.asarray(p[k][gi], np.float64) for k in ("x", "y", "z")}
    rng = np.random.default_rng(0)
    # calibrate on 64 particles, then time a sample sized to about knn_seconds
    ns = min(64, gi.size)
    t1 = time.perf_counter()
    oracle.knn(g, 64, sample=np.sort(rng.choice(gi.size, ns, replace=False)))
    t64 = max(time.perf_counter() - t1, 1e-4)
    ns = int(min(gi.size, max(ns, ns * knn_seconds / t64)))
    s = np.sort(rng.choice(gi.size, ns, replace=False))
    t1 = time.perf_counter()
    oracle.knn(g, 64, sample=s)
    t_knn = (time.perf_counter() - t1) * gi.size / ns
    total = t_grav + t_knn
    return {"value": n / total, "unit": UNIT, "cores": oracle.num_threads(), "cpu_model": cpu_model(),
            "kind": "oracle",
            "sample": (f"one force evaluation of {name}: tree build + 1/{stride} of the group walks "
                       f"(x{stride}), brute-force kNN of {ns} gas particles (x{gi.size / ns:.0f}); "
                       f"SPH density/force sums and kicks not included; measured {time.perf_counter() - t0:.1f} s"),
            "seconds_per_step_estimate": total}


def sn_regions(nreg, distinct, lo, hi, seed):
    """nreg supernova regions with gas counts log-uniform in [lo, hi], built
    from `distinct` generated regions, each placed nreg / distinct times on a
    lattice of centres 180 pc apart (3 region sides, so the cubes never
    overlap).  Returns (particles, centres, counts)."""
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(np.log(lo), np.log(hi), distinct)).astype(int)
    base = [ics.sn_region(int(m), seed=seed + k, grid=32) for k, m in enumerate(sizes)]
    parts, centers, counts = {}, [], []
    for r in range(nreg):
        b = base[r % distinct]
        o = (180.0 * (r % 16), 180.0 * (r // 16), 0.0)
        centers.append(o)
        counts.append(b["x"].size)
        for key, val in b.items():
            if key == "x":
                val = val + o[0]
            elif key == "y":
                val = val + o[1]
            parts.setdefault(key, []).append(val)
    p = {k: np.concatenate(v) for k, v in parts.items()}
    p["id"] = np.arange(p["x"].size, dtype=np.int64)
    return p, centers, np.asarray(counts)


def sn_bench(stream, galnb, torch, nreg=256, reps=3, plain_runs=True, global_step=None):
    """SN regions/s: batched surrogate vs plain integration (see module doc).
    nreg and plain_runs=False only serve profiling (--sn-only --sn-regions).
    global_step (a callable running one global KDK step on its own stream):
    also time the coupled step of config 5 (coupled_bench).  The supernova
    work runs on its own non-default stream, which graph capture needs."""
    from paper_2510_23330_gb300 import surrogate as S
    stream = torch.cuda.Stream(device=stream.device)
    sp = stream.cuda_stream
    net = galnb.UNet(5, 5, 16, 4, 64, stream=sp)
    trained = os.path.exists(S.WEIGHTS)
    meta = S.load_weights(net, S.WEIGHTS) if trained else {}
    if not trained:
        net.set_params(S.he_init(seed=0))
    # --- tile shapes of the tensor-core convolutions for the batch, by timing
    tune_ms = net.autotune(nreg)
    # --- surrogate: one graph replay per batch of nreg ragged regions
    p, centers, counts = sn_regions(nreg, 16, 20000, 300000, seed=7)
    ctx = galnb.Context(stream=sp)
    ctx.set_particles(p)
    ctx.compute_sph_density()
    ctx.sn_surrogate_batch(net, centers, seed=0)  # first call captures the graph
    ms = []
    for r in range(reps):
        ctx.compute_sph_density()  # the coupled step has it from the global step
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        ctx.sn_surrogate_batch(net, centers, seed=r + 1)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    coupled = coupled_bench(torch, global_step, ctx, net, centers) if global_step else None
    # stage split, eager with the phase timers
    ctx.compute_sph_density()
    ctx.set_timing(True)
    ctx.phase_times(reset=True)
    ctx.sn_surrogate_batch(net, centers, seed=99)
    ph, _, _ = ctx.phase_times(reset=True)
    ctx.set_timing(False)
    ctx.close()
    # --- U-Net forward alone, device tensors, batch 32
    xb = torch.randn(32, 64, 64, 64, 5, device=stream.device)
    yb = torch.empty_like(xb)
    for _ in range(2):
        net.forward(xb, out=yb)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(3):
        net.forward(xb, out=yb)
    e1.record(stream)
    torch.cuda.synchronize()
    fwd_ms = e0.elapsed_time(e1) / 3
    # --- one training step (forward, MSE, back-propagation, Adam) at batch 1,
    # on a separate network so the timed weights stay the trained ones
    tnet = galnb.UNet(5, 5, 16, 4, 64, stream=sp)
    tnet.set_params(S.he_init(seed=1))
    x1, y1 = xb[:1].contiguous(), yb[:1].contiguous()
    torch.cuda.synchronize()
    for _ in range(3):
        tnet.train_step(x1, y1, 1e-5)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(10):
        tnet.train_step(x1, y1, 1e-5)
    e1.record(stream)
    torch.cuda.synchronize()
    train_ms = e0.elapsed_time(e1) / 10
    tnet.close()
    del xb, yb
    # --- plain: CFL-limited integration of a 1e5-particle region over 0.1 Myr,
    # one region at a time (held-out seeds 1900, 1901; also pairs for the
    # field error), and many regions in one context (the GPU full)
    plain, pairs = [], []
    for seed in ((1900, 1901) if plain_runs else ()):
        x, y, info = S.make_pair(seed, n=100000, grid=64, stream=sp)
        plain.append(info)
        pairs.append((x, y))
    plain_s = float(np.median([i["seconds"] for i in plain])) if plain else float("nan")
    field = None
    if plain_runs:
        Xh, Yh, _ = S.make_pairs(list(range(1902, 1910)), n=100000, grid=64, workers=4)
        X = np.concatenate([np.stack([q[0] for q in pairs]).reshape((-1,) + Xh.shape[1:]), Xh.astype(np.float32)])
        Y = np.concatenate([np.stack([q[1] for q in pairs]).reshape((-1,) + Yh.shape[1:]), Yh.astype(np.float32)])
        ev = S.evaluate_arrays(net, X, Y)
        field = {"rmse_surrogate": ev["rmse_surrogate_all"], "rmse_no_feedback": ev["rmse_identity_all"],
                 "rmse_surrogate_per_channel": ev["rmse_surrogate"], "held_out_seeds": [1900, 1909],
                 "trained": trained, "weights": os.path.relpath(S.WEIGHTS, ROOT) if trained else None,
                 "train_seeds": meta.get("train_seeds"), "epochs": meta.get("epochs"),
                 "units": "standardised channels, mean over 5 channels and 10 held-out seeds, computed in this run "
                          "with the network timed above"}
    batched = plain_batched(galnb, torch, stream, steps_single=float(np.median([i["steps"] for i in plain]))
                            if plain else 175.0) if plain_runs else None
    # --- plain with hierarchical individual timesteps, same region as the first run
    hier = None
    if plain_runs:
        _, yh, hi = S.make_pair(1900, n=100000, grid=64, stream=sp, integrator="hier")
        hier = {"seconds_per_region": hi["seconds"], "regions_per_s": 1.0 / hi["seconds"],
                "block_steps": hi["steps"], "particle_updates": hi["updates"], "wakeups": hi["wakeups"],
                "updates_vs_shared": hi["updates"] / plain[0]["updates"],
                "rmse_vs_shared": float(np.mean(S.rmse(yh, pairs[0][1]))), "max_level": 20,
                "note": "all particles drifted, predicted and evaluated at every block step; the particles whose "
                        "step ends (or whose CFL level became finer) are kicked"}
    net.close()
    sur_ms = float(np.median(ms))
    try:
        peaks = json.load(open(PEAKS))
        peak, peak_note = float(peaks["bf16_tflops"]), "of measured (cuBLAS bf16 burst, MEASURED_PEAKS.json)"
    except (OSError, KeyError, ValueError):
        peak, peak_note = 1900.0, "of fallback"
    tflops = UNET_GFLOP_64 * 32 / fwd_ms  # GFLOP per ms = TFLOP/s
    sur_rate = nreg / (sur_ms * 1e-3)
    plain_rates = [r for r in (1.0 / plain_s if plain else None,
                               hier["regions_per_s"] if hier else None,
                               batched["regions_per_s_equivalent"] if batched else None) if r]
    best_plain = max(plain_rates) if plain_rates else None
    return {
        "metric": "SN regions/s: surrogate vs plain at fixed error",
        "surrogate_regions_per_s": sur_rate,
        "plain_regions_per_s": 1.0 / plain_s,
        "best_plain_regions_per_s": best_plain,
        "speedup_vs_best_plain": sur_rate / best_plain if best_plain else None,
        "surrogate": {"regions": nreg, "gas_particles": int(counts.sum()),
                      "counts_min_max": [int(counts.min()), int(counts.max())], "grid": 64, "side_pc": 60.0,
                      "ms_per_batch": sur_ms, "batch_ms": ms, "graph": True, "trained_weights": trained,
                      "stage_ms": {k: ph[k] for k in ("VOXELISE", "UNET", "REMAP")},
                      "note": "16 generated regions placed 16 times each; density from the global step not timed"},
        "plain": {"particles": 100000, "t_end_myr": 0.1, "seconds_per_region": plain_s,
                  "steps": [int(i["steps"]) for i in plain], "gravity": "none (SN region integrator)",
                  "note": "one region per context, integrated alone"},
        "plain_batched": batched,
        "coupled_step": coupled,
        "plain_hier": hier,
        "field_error": field,
        "unet_roofline": {"bound": "tensor", "achieved": tflops, "peak": peak, "unit": "TFLOP/s",
                          "frac": tflops / peak, "note": f"whole forward, {UNET_GFLOP_64} GFLOP per 64^3 region, "
                                                          f"batch 32, {peak_note}", "ms_per_region": fwd_ms / 32},
        "unet_tile_autotune_ms": {"forward_before": tune_ms[0], "forward_after": tune_ms[1], "batch": nreg},
        "unet_training_step": {"ms": train_ms, "batch": 1, "grid": 64,
                               "achieved_tflops": 3 * UNET_GFLOP_64 / train_ms,
                               "frac": 3 * UNET_GFLOP_64 / train_ms / peak,
                               "note": "forward + MSE + back-propagation (input and weight gradients on tcgen05) + "
                                       "Adam, counted as 3x the forward's flops; batch 1 as the paper trains"},
    }


def coupled_bench(torch, global_step, ctx_sn, net, centers, reps=3):
    """The batched coupled step (config 5, Sec. 3.2: the pool nodes predict
    the supernova regions while the main nodes integrate the galaxy): one
    global KDK step of the galaxy context (its own stream) and one
    graph-replayed surrogate batch of the region context (another stream),
    issued from two host threads so that they share the GPU, against the two
    run one after the other.  Wall-clock milliseconds, the median of reps;
    the regions' density before each batch is computed outside the timing."""
    import threading

    def prep():
        ctx_sn.compute_sph_density()
        torch.cuda.synchronize()

    def batch(seed):
        ctx_sn.sn_surrogate_batch(net, centers, seed=seed)

    res = {"global": [], "batch": [], "sequential": [], "concurrent": []}
    for r in range(reps):
        prep()
        t0 = time.perf_counter()
        global_step()
        res["global"].append(time.perf_counter() - t0)
        t0 = time.perf_counter()
        batch(100 + r)
        res["batch"].append(time.perf_counter() - t0)
        prep()
        t0 = time.perf_counter()
        global_step()
        batch(200 + r)
        res["sequential"].append(time.perf_counter() - t0)
        prep()
        th = threading.Thread(target=batch, args=(300 + r,))
        t0 = time.perf_counter()
        th.start()
        global_step()
        th.join()
        res["concurrent"].append(time.perf_counter() - t0)
    med = {k: 1e3 * float(np.median(v)) for k, v in res.items()}
    return {"global_step_ms": med["global"], "batch_ms": med["batch"], "sequential_ms": med["sequential"],
            "concurrent_ms": med["concurrent"], "overlap_gain": med["sequential"] / med["concurrent"],
            "regions": len(centers),
            "note": "wall clock, median of 3: one 2^24 global KDK step and one 256-region surrogate batch, one "
                    "after the other or issued together from two host threads on two streams"}


def plain_batched(galnb, torch, stream, nreg=32, n=100000, steps=8, steps_single=175.0):
    """The plain CFL-limited integrator with nreg supernova regions of n gas
    particles in one context (centres 180 pc apart, 10^51 erg injected in each;
    seeds 1900 + k): particle-steps per second of the KDK step with the GPU
    full, and the per-region time that rate gives a region taking
    steps_single steps (its own CFL step count when integrated alone)."""
    parts, centers = {}, []
    for k in range(nreg):
        r = dict(ics.sn_region(n, seed=1900 + k))
        o = (180.0 * (k % 8), 180.0 * (k // 8), 0.0)
        r["x"], r["y"] = r["x"] + o[0], r["y"] + o[1]
        centers.append(o)
        for key, val in r.items():
            parts.setdefault(key, []).append(val)
    p = {k: np.concatenate(v) for k, v in parts.items()}
    p["id"] = np.arange(p["x"].size, dtype=np.int64)
    ctx = galnb.Context(stream=stream.cuda_stream)
    ctx.set_particles(p)
    ctx.compute_sph_density()
    for o in centers:
        ctx.inject_energy(o, ics.E_SN_CODE)
    ctx.integrate_cfl(1.0, max_steps=2)  # initial forces and two steps untimed
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    _, nst = ctx.integrate_cfl(1.0, max_steps=steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ctx.close()
    ms = e0.elapsed_time(e1)
    pss = p["x"].size * nst / (ms * 1e-3)
    sec = n * steps_single / pss
    return {"regions": nreg, "particles": int(p["x"].size), "steps_timed": int(nst), "ms_per_step": ms / max(nst, 1),
            "particle_steps_per_s": pss, "seconds_per_region_equivalent": sec, "regions_per_s_equivalent": 1.0 / sec,
            "note": f"{nreg} regions in one context share the CFL step; per region: {n} particles x "
                    f"{steps_single:.0f} steps (its own step count) at the batched rate"}


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if os.environ.get("GNB_BENCH_BACKEND", "nccl") == "nccl" else "gloo")
    return world, rank, local


def reduce_max(x, world, device=None):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(units_per_rank, steps, world, tmax_ms):
    """Units processed by all ranks per second, timed by the slowest rank
    (weak scaling: every rank steps its own replica)."""
    return units_per_rank * steps * world / (tmax_ms * 1e-3)


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# steps over which each workload reports its energy and momentum drift
DRIFT_STEPS = {"large": 20, "disk": 10}


def run_ours(args, world, rank, local):
    import torch
    from paper_2510_23330_gb300 import galnb

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    p, desc = workload(args.config, seed=rank)
    pr = params(args.config)
    if args.sph == "pressure":
        pr["cfg"]["sph_variant"] = 1  # pressure-energy SPH (smoothed pressure)
    mode = pr["gravity"]
    n = int(p["x"].shape[0])
    ctx = galnb.Context(stream=stream.cuda_stream, **pr["cfg"])
    ctx.set_particles(p)
    tuning = None
    if args.n_leaf:
        pr["cfg"]["n_leaf"] = args.n_leaf
        ctx.set_params(n_leaf=args.n_leaf)
    if args.n_group:
        pr["cfg"]["n_group"] = args.n_group
        ctx.set_params(n_group=args.n_group)
    elif mode == 1 and not args.no_autotune:
        from paper_2510_23330_gb300 import autotune
        (nl, ng), table = autotune.tune_tree(ctx, mode)
        pr["cfg"]["n_leaf"], pr["cfg"]["n_group"] = nl, ng
        tuning = {k: round(v, 4) for k, v in table.items()}
    ctx.compute_forces(mode)
    for _ in range(args.warmup):
        ctx.step_kdk(args.dt, 1, mode)
    d0 = ctx.diagnostics()  # FP64 energies, momentum, angular momentum before the timed steps
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MiB > 129 MB L2
    clocks = ClockSampler(local) if not args.no_clocks else None
    ctx.set_timing(True)
    ctx.phase_times(reset=True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    npp = npc = 0
    barrier(world)
    torch.cuda.synchronize()
    h0 = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        ctx.step_kdk(args.dt, 1, mode)
        ev[k][1].record(stream)
        st = ctx.stats()
        npp += st["NPP"]
        npc += st["NPC"]
    torch.cuda.synchronize()
    h1 = time.perf_counter()
    barrier(world)
    if clocks:
        time.sleep(0.05)
        clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    d1 = ctx.diagnostics()
    e0, e1 = float(np.sum(d0[:4])), float(np.sum(d1[:4]))
    # momentum scale: sum m |v| of the initial state
    psc = float(np.sum(p["m"] * np.sqrt(p["vx"].astype(np.float64) ** 2 + p["vy"] ** 2 + p["vz"] ** 2)))
    total_ms = sum(step_ms)
    phases, calls, launches = ctx.phase_times(reset=True)
    ctx.set_timing(False)
    # the workload's drift is reported over its own step count (20 for the
    # 2^24 disk, 10 for the 2^20 disk): untimed steps continue the run to that
    # count when fewer were timed
    dsteps = max(args.steps, DRIFT_STEPS.get(args.config, args.steps))
    d2 = d1
    if dsteps > args.steps:
        ctx.step_kdk(args.dt, dsteps - args.steps, mode)
        d2 = ctx.diagnostics()
    e2 = float(np.sum(d2[:4]))
    tmax = reduce_max(total_ms, world, dev)
    value = whole_job_value(n, args.steps, world, tmax)
    # dominant kernel: the gravity walk + PP/PC kernel
    g_calls = max(calls["GRAVITY"], 1)
    g_ms = phases["GRAVITY"] / g_calls
    flops = (FLOP_PP * npp + FLOP_PC * npc) / max(args.steps, 1)
    achieved = flops / (g_ms * 1e-3) / 1e12
    traffic = gravity_traffic(args.config)
    try:
        hbm_peak, hbm_note = float(json.load(open(PEAKS))["hbm_gbs"]), "of measured (copy, MEASURED_PEAKS.json)"
    except (OSError, KeyError, ValueError):
        hbm_peak, hbm_note = 6800.0, "of fallback"
    n_gas = int(np.sum(p["type"] == 1))

    def hbm_entry(phase_names, bytes_total, what):
        ms = sum(phases[k] for k in phase_names) / max(args.steps, 1)
        gbs = bytes_total / (ms * 1e-3) / 1e9 if ms > 0 else None
        return {"bound": "hbm", "phases": list(phase_names), "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                "frac": gbs / hbm_peak if gbs else None, "ms_per_step": ms, "algorithmic_bytes": bytes_total,
                "note": f"{what}; {hbm_note}"}

    rooflines = {
        "tree_build": hbm_entry(("SORT", "TREE", "HYDRO_TREE"), BYTES_TREE_PER_PARTICLE * n,
                                f"{BYTES_TREE_PER_PARTICLE} B per particle"),
        "knn_density": hbm_entry(("KNN",), BYTES_KNN_DENSITY_PER_GAS * n_gas,
                                 f"{BYTES_KNN_DENSITY_PER_GAS} B per gas particle"),
        "hydro_force": hbm_entry(("FORCE",), BYTES_FORCE_PER_GAS * n_gas, f"{BYTES_FORCE_PER_GAS} B per gas particle"),
    }
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tmax / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": desc, "n": n, "n_gas": int(np.sum(p["type"] == 1)), "dt": args.dt,
                   "gravity": "tree" if mode == 1 else "direct", **pr["cfg"], "n_ngb": 64,
                   "l2": "flushed before every timed step (256 MiB write)",
                   "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "alu", "kernel": "k_grav_walk + k_grav_eval (walk, PP/PC)", "achieved": achieved,
                     "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS,
                     "traffic": traffic,
                     "note": (f"flops = {FLOP_PP}/PP + {FLOP_PC}/PC interaction; peak = 152 SMs x 128 lanes x 2 x "
                              f"2070 MHz (FP32 CUDA cores)"),
                     "ms_per_launch": g_ms},
        "rooflines_hbm": rooflines,
        "interactions_per_step": {"pp": npp / args.steps, "pc": npc / args.steps},
        "tree_tuning_ms": tuning,
        "phases_ms_per_step": {k: v / args.steps for k, v in phases.items()},
        "gpu_launches": int(launches),
        "step_ms": step_ms,
        "drift": {"steps": dsteps, "energy_rel": (e2 - e0) / abs(e0) if e0 else None,
                  "momentum_rel": float(np.linalg.norm(d2[4:7] - d0[4:7])) / max(psc, 1e-300),
                  "energy_before": e0, "energy_after": e2,
                  "timed_steps": {"steps": args.steps, "energy_rel": (e1 - e0) / abs(e0) if e0 else None,
                                  "momentum_rel": float(np.linalg.norm(d1[4:7] - d0[4:7])) / max(psc, 1e-300)},
                  "note": "E = E_kin + E_pot + E_ext + E_th (FP64 reductions, the static halo included); "
                          "|dP| relative to sum m|v|; the NFW halo is external, so P is not conserved exactly"},
    }
    if clocks:
        out["clocks"] = clocks.summary(h0, h1)
    if rank == 0 and world == 1 and not args.no_e2e:
        out["e2e"] = e2e(args, p, pr, stream, galnb, torch)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(p, desc, n_g=int(pr["cfg"].get("n_group", 64)),
                                           n_leaf=int(pr["cfg"].get("n_leaf", 16)))
    if rank == 0 and world == 1 and not args.no_sn:
        out["sn"] = sn_bench(stream, galnb, torch, global_step=lambda: ctx.step_kdk(args.dt, 1, mode))
    ctx.close()
    return out


def e2e(args, p, pr, stream, galnb, torch):
    """Same metric through the public API with host buffers: every step
    uploads the particles with the accelerations of their state from pinned
    host memory (gnb_set_state: the step kicks with them, as a KDK
    integration carries them from one step to the next), steps once and reads
    the new state and its accelerations back into the same pinned arrays (the
    next step's input)."""
    n = int(p["x"].shape[0])
    state = dict(p)
    state.update(ax=np.zeros(n, np.float32), ay=np.zeros(n, np.float32), az=np.zeros(n, np.float32),
                 dudt=np.zeros(n, np.float32), h2=np.zeros(n, np.float64))
    host = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for k, v in state.items()}
    outs = {"X": "x", "Y": "y", "Z": "z", "VX": "vx", "VY": "vy", "VZ": "vz", "U": "u",
            "AX": "ax", "AY": "ay", "AZ": "az", "DUDT": "dudt", "H2": "h2"}
    ctx = galnb.Context(stream=stream.cuda_stream, **pr["cfg"])
    steps = max(1, min(args.steps, 5))
    h2d = sum(t.numel() * t.element_size() for t in host.values())
    d2h = sum(host[k].numel() * host[k].element_size() for k in outs.values())
    ctx.set_particles(host)
    ctx.step_kdk(args.dt, 1, pr["gravity"])
    back = {f: host[k] for f, k in outs.items()}
    ctx.get_fields(back)
    # one untimed round of the measured path (upload with the state's
    # accelerations, step, export) before the timed ones
    ctx.set_state(host, pr["gravity"])
    ctx.step_kdk(args.dt, 1, pr["gravity"])
    ctx.get_fields(back)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        ctx.set_state(host, pr["gravity"])
        ctx.step_kdk(args.dt, 1, pr["gravity"])
        ctx.get_fields(back)
    t1 = time.perf_counter()
    ctx.close()
    return {"value": n * steps / (t1 - t0), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "steps": steps,
            "note": "per step: gnb_set_state from pinned host arrays (state, accelerations, du/dt, kernel supports), "
                    "one KDK step (one force evaluation; the caller order is re-sorted along the Morton curve), "
                    "gnb_get_fields of the new state into the same arrays (one wait)"}


def run_reference(args, world, rank, local):
    """The FP64 oracle as it stands, on a bounded sample of each step."""
    if rank != 0:
        return None
    p, desc = workload(args.config, seed=0)
    n = int(p["x"].shape[0])
    for _ in range(args.warmup):
        pass  # the sampled oracle has no warm state; warm-up steps are not needed
    secs = []
    cb = None
    for _ in range(args.steps):
        cb = cpu_baseline(p, desc, knn_seconds=2.0, n_g=128)
        secs.append(cb["seconds_per_step_estimate"])
    value = n * args.steps / sum(secs)
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(secs) / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": desc, "n": n},
            "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle", "cores": cb["cores"],
                             "cpu_model": cb["cpu_model"], "sample": cb["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="large", choices=["disk", "large", "tiny"])
    ap.add_argument("--dt", type=float, default=1e-3)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--n-group", type=int, default=0, help="fixed group size n_g (skips the autotuner)")
    ap.add_argument("--n-leaf", type=int, default=0, help="leaf size n_leaf (with --n-group: no autotuner)")
    ap.add_argument("--sph", default="density", choices=["density", "pressure"],
                    help="SPH formulation: density-energy (default) or pressure-energy")
    ap.add_argument("--no-sn", action="store_true", help="skip the supernova surrogate-vs-plain section")
    ap.add_argument("--sn-only", action="store_true",
                    help="profiling: only the supernova section, printed alone (not the bench line)")
    ap.add_argument("--sn-regions", type=int, default=256, help="regions of the --sn-only batch")
    ap.add_argument("--sn-no-plain", action="store_true", help="--sn-only without the plain integrations")
    args = ap.parse_args()
    if args.impl == "reference":
        # the CPU checker runs once, on rank 0; other ranks exit without work
        world = int(os.environ.get("WORLD_SIZE", "1"))
        rank = int(os.environ.get("RANK", "0"))
        out = run_reference(args, world, rank, 0)
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    if args.sn_only:
        import torch
        from paper_2510_23330_gb300 import galnb
        stream = torch.cuda.current_stream(torch.device("cuda", 0))
        out = sn_bench(stream, galnb, torch, nreg=args.sn_regions, plain_runs=not args.sn_no_plain)
        print(json.dumps(out), flush=True)
        return
    world, rank, local = dist_init()
    out = run_ours(args, world, rank, local)
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
