"""Supernova surrogate: training pairs from the plain integrator, training,
evaluation and the surrogate-vs-plain comparison (Sec. 3.2-3.3, 5.3).

Pairs: a turbulent region of gas (ics.sn_region) is voxelised just before the
explosion (input) and again after the plain CFL-limited integration of the
injected 10^51 erg over 0.1 Myr (target).  The network is the library's BF16
U-Net trained with MSE and Adam at batch size 1 (Sec. 3.3).  The plain
integration is both the training signal and the reference the surrogate's
error is measured against; "identity" (the input grid taken as the prediction, i.e. the region
without the supernova's feedback) is the baseline the surrogate must beat.

    python -m paper_2510_23330_gb300.surrogate --train 48 --test 8 --out report.json
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import galnb, ics


def make_pair(seed: int, n: int = 100000, grid: int = 64, side: float = 60.0, courant: float = 0.3,
              stream=None, integrator: str = "cfl", max_level: int = 20):
    """(input grid, target grid, info) of one supernova region, integrated
    with the shared CFL step ("cfl") or individual timesteps ("hier")."""
    p = ics.sn_region(n, seed=seed, side=side)
    c = galnb.Context(stream=stream)
    c.set_particles(p)
    c.compute_sph_density()
    x = c.voxelise([(0.0, 0.0, 0.0)], side, grid)[0]
    c.inject_energy((0.0, 0.0, 0.0), ics.E_SN_CODE)
    t0 = time.perf_counter()
    if integrator == "hier":
        t, steps, updates, wakes = c.integrate_hier(ics.T_SN_END, courant, max_level=max_level,
                                                    mode=galnb.GNB_GRAV_NONE)
        extra = {"updates": updates, "wakeups": wakes}
    else:
        t, steps = c.integrate_cfl(ics.T_SN_END, courant, mode=galnb.GNB_GRAV_NONE)
        extra = {"updates": int(steps) * n}
    dt_wall = time.perf_counter() - t0
    c.compute_sph_density()
    y = c.voxelise([(0.0, 0.0, 0.0)], side, grid)[0]
    c.close()
    return x, y, {"seed": seed, "steps": int(steps), "t": t, "seconds": dt_wall, "n": n, **extra}


def rmse(a, b):
    """Per-channel RMS difference of standardised grids."""
    d = (np.asarray(a, np.float64) - np.asarray(b, np.float64)).reshape(-1, 5)
    return np.sqrt(np.mean(d * d, axis=0))


def train(net: "galnb.UNet", pairs, epochs: int, lr: float, seed: int = 0):
    rng = np.random.default_rng(seed)
    hist = []
    for _ in range(epochs):
        losses = []
        for k in rng.permutation(len(pairs)):
            x, y = pairs[k][0], pairs[k][1]
            losses.append(net.train_step(x[None], y[None], lr))
        hist.append(float(np.mean(losses)))
    return hist


def evaluate(net: "galnb.UNet", pairs):
    s, i = [], []
    for x, y, _ in pairs:
        pred = net.forward(x[None])[0]
        s.append(rmse(pred, y))
        i.append(rmse(x, y))
    return {"rmse_surrogate": np.mean(s, axis=0).tolist(), "rmse_identity": np.mean(i, axis=0).tolist(),
            "rmse_surrogate_all": float(np.mean(s)), "rmse_identity_all": float(np.mean(i))}


def batch_regions(nreg: int, n: int, side: float = 60.0, seed0: int = 1000):
    """nreg regions laid out far apart in one particle set, with region
    sizes log-uniform in [n/15, n] (the ragged batch of the coupled step)."""
    rng = np.random.default_rng(seed0)
    sizes = np.exp(rng.uniform(np.log(max(n // 15, 2000)), np.log(n), nreg)).astype(int)
    parts, centers = {}, []
    for k, m in enumerate(sizes):
        r = ics.sn_region(int(m), seed=seed0 + k, side=side, grid=32)
        o = (3.0 * side * (k % 16), 3.0 * side * (k // 16), 0.0)
        r = dict(r)
        r["x"], r["y"] = r["x"] + o[0], r["y"] + o[1]
        centers.append(o)
        for key, val in r.items():
            parts.setdefault(key, []).append(val)
    p = {k: np.concatenate(v) for k, v in parts.items()}
    p["id"] = np.arange(p["x"].size, dtype=np.int64)
    return p, centers, sizes


def time_surrogate(net: "galnb.UNet", nreg: int, n: int, reps: int = 5, stream=None):
    """Regions per second of the batched, graph-replayed surrogate step."""
    import torch
    p, centers, sizes = batch_regions(nreg, n)
    c = galnb.Context(stream=stream)
    c.set_particles(p)
    c.compute_sph_density()
    c.sn_surrogate_batch(net, centers, seed=0)      # capture
    times = []
    for r in range(reps):
        c.compute_sph_density()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c.sn_surrogate_batch(net, centers, seed=r + 1)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    c.close()
    return nreg / float(np.median(times)), {"regions": nreg, "particles": int(sizes.sum()),
                                              "seconds": float(np.median(times))}


def he_init(cin=5, cout=5, base=16, levels=4, seed=0):
    """He-normal weights and zero biases in the library's flat parameter
    order (per layer W[taps][cin][cout] then b[cout])."""
    rng = np.random.default_rng(seed)
    layers = []
    c = cin
    for l in range(levels):
        layers += [(27, c, base << l), (27, base << l, base << l)]
        c = base << l
    for l in range(levels - 2, -1, -1):
        layers += [(8, base << (l + 1), base << l), (27, 2 * (base << l), base << l), (27, base << l, base << l)]
    layers.append((1, base, cout))
    out = []
    for taps, ci, co in layers:
        fan = ci if taps == 8 else taps * ci
        out.append(rng.normal(0.0, np.sqrt(2.0 / fan), taps * ci * co))
        out.append(np.zeros(co))
    return np.concatenate(out).astype(np.float32)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=48)
    ap.add_argument("--test", type=int, default=8)
    ap.add_argument("--n", type=int, default=100000)
    ap.add_argument("--grid", type=int, default=64)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--batch-regions", type=int, default=64)
    ap.add_argument("--out", default="surrogate_report.json")
    a = ap.parse_args()
    import torch
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        sp = stream.cuda_stream
        t0 = time.perf_counter()
        tr = [make_pair(s, a.n, a.grid, stream=sp) for s in range(a.train)]
        te = [make_pair(1900 + s, a.n, a.grid, stream=sp) for s in range(a.test)]
        t_data = time.perf_counter() - t0
        net = galnb.UNet(5, 5, 16, 4, a.grid, stream=sp)
        net.set_params(he_init(seed=0))
        before = evaluate(net, te)
        t1 = time.perf_counter()
        hist = train(net, tr, a.epochs, a.lr)
        t_train = time.perf_counter() - t1
        after_train = evaluate(net, tr)
        after = evaluate(net, te)
        plain_s = float(np.median([info["seconds"] for _, _, info in tr + te]))
        sur_rate, sur_info = time_surrogate(net, a.batch_regions, a.n, stream=sp)
    rep = {
        "pairs": {"train": a.train, "test": a.test, "particles": a.n, "grid": a.grid,
                  "data_seconds": t_data, "plain_steps_median": float(np.median([i["steps"] for *_, i in tr + te]))},
        "training": {"epochs": a.epochs, "lr": a.lr, "seconds": t_train, "loss_first_epoch": hist[0],
                     "loss_last_epoch": hist[-1]},
        "held_out_before_training": before, "held_out": after, "train_set": after_train,
        "plain_regions_per_s": 1.0 / plain_s, "plain_seconds_per_region": plain_s,
        "surrogate_regions_per_s": sur_rate, "surrogate_batch": sur_info,
        "speedup": sur_rate * plain_s,
        "channels": ["log10 rho + 0.33", "(log10 T - 2)/2", "vx/20", "vy/20", "vz/20"],
    }
    with open(a.out, "w") as fh:
        json.dump(rep, fh, indent=1)
    print(json.dumps({k: rep[k] for k in ("plain_regions_per_s", "surrogate_regions_per_s", "speedup")}))
    print(json.dumps(rep["held_out"]))


if __name__ == "__main__":
    main()
