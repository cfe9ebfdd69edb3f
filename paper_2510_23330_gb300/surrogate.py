"""Supernova surrogate: training pairs from the plain integrator, training,
evaluation and the surrogate-vs-plain comparison (Sec. 3.2-3.3, 5.3).

Pairs: a turbulent region of gas (ics.sn_region) is voxelised just before the
explosion (input) and again after the plain CFL-limited integration of the
injected 10^51 erg over 0.1 Myr (target).  The network is the library's BF16
U-Net trained with MSE and Adam at batch size 1 (Sec. 3.3).  The plain
integration is both the training signal and the reference the surrogate's
error is measured against; "identity" (the input grid taken as the prediction, i.e. the region
without the supernova's feedback) is the baseline the surrogate must beat.

    python -m paper_2510_23330_gb300.surrogate --train 1900 --test 100 --epochs 20 --report report.txt

trains the network on seeds 0-1899, saves it (float16) to ``weights/`` and
reports the held-out field error on seeds 1900-1999.
"""
from __future__ import annotations

import argparse
import json
import os
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


def make_pairs(seeds, n: int = 100000, grid: int = 64, workers: int = 4, integrator: str = "cfl"):
    """Pairs of many seeds as float16 arrays X, Y [len(seeds), grid, grid,
    grid, 5] plus per-seed info.  `workers` regions are integrated at once,
    each by its own host thread on its own CUDA stream: one region of 1e5
    particles does not fill the GPU, several do."""
    import threading
    import torch
    k = len(seeds)
    X = np.empty((k, grid, grid, grid, 5), np.float16)
    Y = np.empty_like(X)
    infos = [None] * k
    errors = []
    streams = [torch.cuda.Stream() for _ in range(max(1, workers))]

    def run(w):
        try:
            for i in range(w, k, len(streams)):
                x, y, info = make_pair(int(seeds[i]), n, grid, stream=streams[w].cuda_stream, integrator=integrator)
                X[i], Y[i], infos[i] = x.reshape(X.shape[1:]), y.reshape(Y.shape[1:]), info
        except Exception as e:  # reported after the join
            errors.append(e)

    threads = [threading.Thread(target=run, args=(w,)) for w in range(len(streams))]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    if errors:
        raise errors[0]
    return X, Y, infos


def rmse(a, b):
    """Per-channel RMS difference of standardised grids."""
    d = (np.asarray(a, np.float64) - np.asarray(b, np.float64)).reshape(-1, 5)
    return np.sqrt(np.mean(d * d, axis=0))


def train(net: "galnb.UNet", pairs, epochs: int, lr: float, seed: int = 0):
    """Adam at batch size 1 (Sec. 3.3) over (x, y, info) pairs in host memory."""
    rng = np.random.default_rng(seed)
    hist = []
    for _ in range(epochs):
        losses = []
        for k in rng.permutation(len(pairs)):
            x, y = pairs[k][0], pairs[k][1]
            losses.append(net.train_step(x[None], y[None], lr))
        hist.append(float(np.mean(losses)))
    return hist


def train_device(net: "galnb.UNet", X, Y, epochs: int, lr: float, seed: int = 0, lr_final: float | None = None):
    """Adam at batch size 1 over pairs held on the device (torch float16
    tensors [k, G, G, G, 5], widened to FP32 per step); the learning rate
    decays geometrically from lr to lr_final over the epochs.  Returns the
    mean loss of every epoch."""
    import torch
    rng = np.random.default_rng(seed)
    hist = []
    k = X.shape[0]
    xb = torch.empty((1,) + tuple(X.shape[1:]), dtype=torch.float32, device=X.device)
    yb = torch.empty_like(xb)
    for e in range(epochs):
        f = e / max(epochs - 1, 1)
        lr_e = lr if lr_final is None else lr * (lr_final / lr) ** f
        losses = []
        for i in rng.permutation(k):
            xb.copy_(X[i:i + 1])
            yb.copy_(Y[i:i + 1])
            torch.cuda.current_stream().synchronize()
            losses.append(net.train_step(xb, yb, lr_e))
        hist.append(float(np.mean(losses)))
    return hist


WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "unet_sn64_base16.npz")


def save_weights(net: "galnb.UNet", path: str = WEIGHTS, meta: dict | None = None):
    """The network's parameters rounded to float16 (the forward pass uses
    BF16 operands, so the stored precision is above what inference uses)."""
    os.makedirs(os.path.dirname(path), exist_ok=True)
    np.savez_compressed(path, params=net.get_params().astype(np.float16),
                        meta=json.dumps(meta or {}))


def load_weights(net: "galnb.UNet", path: str = WEIGHTS) -> dict:
    """Loads parameters saved by save_weights; returns their metadata."""
    d = np.load(path)
    net.set_params(d["params"].astype(np.float32))
    return json.loads(str(d["meta"]))


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


def evaluate_arrays(net: "galnb.UNet", X, Y):
    """Held-out field error of pairs in arrays (numpy float16 [k, G, G, G, 5]):
    per-channel RMSE of the surrogate and of the identity (no feedback)."""
    s, i = [], []
    for k in range(X.shape[0]):
        x = X[k].astype(np.float32)
        y = Y[k].astype(np.float32)
        s.append(rmse(net.forward(x[None])[0], y))
        i.append(rmse(x, y))
    return {"rmse_surrogate": np.mean(s, axis=0).tolist(), "rmse_identity": np.mean(i, axis=0).tolist(),
            "rmse_surrogate_all": float(np.mean(s)), "rmse_identity_all": float(np.mean(i))}


def main():
    """Training run: pairs of seeds [0, train) and held-out seeds
    [1900, 1900 + test), Adam at batch size 1 on the GPU, weights saved in
    float16 and the held-out error evaluated with the saved weights."""
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=1900)
    ap.add_argument("--test", type=int, default=100)
    ap.add_argument("--n", type=int, default=100000)
    ap.add_argument("--grid", type=int, default=64)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--lr-final", type=float, default=1e-4)
    ap.add_argument("--workers", type=int, default=6)
    ap.add_argument("--save", default=WEIGHTS)
    ap.add_argument("--report", default="surrogate_report.txt")
    a = ap.parse_args()
    import torch
    t0 = time.perf_counter()
    Xtr, Ytr, itr = make_pairs(list(range(a.train)), a.n, a.grid, workers=a.workers)
    Xte, Yte, ite = make_pairs(list(range(1900, 1900 + a.test)), a.n, a.grid, workers=a.workers)
    t_data = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    net = galnb.UNet(5, 5, 16, 4, a.grid, stream=stream.cuda_stream)
    net.set_params(he_init(seed=0))
    before = evaluate_arrays(net, Xte[:16], Yte[:16])
    Xd = torch.from_numpy(Xtr).cuda()
    Yd = torch.from_numpy(Ytr).cuda()
    t1 = time.perf_counter()
    hist = train_device(net, Xd, Yd, a.epochs, a.lr, lr_final=a.lr_final)
    t_train = time.perf_counter() - t1
    del Xd, Yd
    meta = {"train_seeds": [0, a.train], "test_seeds": [1900, 1900 + a.test], "particles": a.n, "grid": a.grid,
            "epochs": a.epochs, "lr": [a.lr, a.lr_final], "loss_last_epoch": hist[-1]}
    save_weights(net, a.save, meta)
    load_weights(net, a.save)  # evaluate what was saved
    after = evaluate_arrays(net, Xte, Yte)
    train_fit = evaluate_arrays(net, Xtr[:100], Ytr[:100])
    steps = [i["steps"] for i in itr + ite]
    secs = [i["seconds"] for i in itr + ite]
    lines = [
        "# Supernova surrogate: training on plain-integrator pairs and held-out field error",
        f"# command (GB300): python -m paper_2510_23330_gb300.surrogate --train {a.train} --test {a.test} "
        f"--n {a.n} --grid {a.grid} --epochs {a.epochs} --lr {a.lr} --lr-final {a.lr_final} --workers {a.workers}",
        "# pairs: 1e5-particle turbulent regions (lognormal density sigma 1, Kolmogorov velocity 10 km/s rms, 100 K),",
        "#   10^51 erg into the 64 nearest gas particles, plain CFL integration (Courant 0.3) over 0.1 Myr, voxelised 64^3;",
        f"#   train seeds 0-{a.train - 1}, held-out seeds 1900-{1900 + a.test - 1}.",
        "# network: the library's BF16 U-Net (4 levels, base 16), Adam at batch size 1 on the GPU (tcgen05 path),",
        "#   learning rate decaying geometrically over the epochs; weights saved in float16 and evaluated as saved.",
        "# rmse: root-mean-square difference of the standardised channels (log10 rho + 0.33, (log10 T - 2)/2,",
        "#   v/20 km/s), prediction vs the plain integration, mean over the held-out seeds; identity = the input",
        "#   grid taken as the prediction (the region without the supernova's feedback).",
        f"train_pairs: {a.train}",
        f"test_pairs: {a.test}",
        f"epochs: {a.epochs}",
        f"lr: {a.lr} -> {a.lr_final}",
        f"pair_generation_seconds: {t_data:.1f}  ({a.workers} regions at a time)",
        f"training_seconds: {t_train:.1f}",
        f"loss_first_epoch: {hist[0]:.4f}",
        f"loss_last_epoch: {hist[-1]:.4f}",
        f"rmse_surrogate_all: {after['rmse_surrogate_all']:.4f}",
        f"rmse_identity_all: {after['rmse_identity_all']:.4f}",
        f"rmse_untrained_all: {before['rmse_surrogate_all']:.4f}  (first 16 held-out seeds)",
        f"rmse_train_fit_all: {train_fit['rmse_surrogate_all']:.4f}  (first 100 training seeds)",
        "rmse_surrogate_per_channel: " + ", ".join(f"{v:.4f}" for v in after["rmse_surrogate"]),
        "rmse_identity_per_channel: " + ", ".join(f"{v:.4f}" for v in after["rmse_identity"]),
        f"plain_seconds_per_region_median: {float(np.median(secs)):.4f}",
        f"plain_steps_median: {float(np.median(steps)):.1f}",
        "loss_per_epoch: " + ", ".join(f"{h:.4f}" for h in hist),
    ]
    with open(a.report, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    print("\n".join(lines[-12:]))


if __name__ == "__main__":
    main()
