"""FP64 oracle of the supernova surrogate's 3D U-Net (Sec. 3.3: a U-Net of 3D
convolutions mapping the gas around a supernova on a 64^3 grid to its state
0.1 Myr later; MSE loss, Adam, batch size 1).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Readings (the paper does not give the layers): four levels with widths
16, 32, 64, 128; two 3^3 convolutions with zero "same" padding and ReLU per
level; 2^3 max-pool down; 2^3 stride-2 transposed convolution up; the skip
tensor is concatenated before the up-sampled one; a 1^3 linear head.
Tensors are (batch, z, y, x, channel).  ``bf16=True`` rounds the network
input, the weights and every stored activation to bfloat16 (round to nearest
even), at the points where the GPU path stores BF16, so that both sides take
the same rounding decisions.
"""
from __future__ import annotations

import numpy as np

TAPS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def bf16(a):
    """Round float64/float32 values to the nearest bfloat16 (ties to even)."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def layer_spec(cin=5, cout=5, base=16, levels=4):
    """Ordered list of (name, kind, in channels, out channels)."""
    w = [base << l for l in range(levels)]
    spec = []
    c = cin
    for l in range(levels):
        spec.append((f"enc{l}a", "conv3", c, w[l]))
        spec.append((f"enc{l}b", "conv3", w[l], w[l]))
        c = w[l]
    for l in range(levels - 2, -1, -1):
        spec.append((f"up{l}", "up2", w[l + 1], w[l]))
        spec.append((f"dec{l}a", "conv3", 2 * w[l], w[l]))
        spec.append((f"dec{l}b", "conv3", w[l], w[l]))
    spec.append(("head", "conv1", w[0], cout))
    return spec


def init_params(seed=0, cin=5, cout=5, base=16, levels=4):
    """He-normal weights, zero biases.  conv3: W[27, cin, cout]; up2:
    W[8, cin, cout]; conv1: W[1, cin, cout]."""
    rng = np.random.default_rng(seed)
    ntap = {"conv3": 27, "up2": 8, "conv1": 1}
    p = {}
    for name, kind, ci, co in layer_spec(cin, cout, base, levels):
        fan = ntap[kind] * ci if kind != "up2" else ci
        p[name + ".w"] = rng.normal(0.0, np.sqrt(2.0 / fan), (ntap[kind], ci, co))
        p[name + ".b"] = np.zeros(co)
    return p


def conv3(x, W, b):
    """out[v] = sum_tap x[v + tap] @ W[tap] + b (zero padding)."""
    B, D, H, Wd, C = x.shape
    xp = np.zeros((B, D + 2, H + 2, Wd + 2, C))
    xp[:, 1:-1, 1:-1, 1:-1] = x
    out = np.zeros((B, D, H, Wd, W.shape[2]))
    for t, (dz, dy, dx) in enumerate(TAPS):
        out += xp[:, 1 + dz:1 + dz + D, 1 + dy:1 + dy + H, 1 + dx:1 + dx + Wd] @ W[t]
    return out + b


def conv3_backward(x, W, dz_):
    """Gradients of conv3 with respect to x, W and b."""
    B, D, H, Wd, C = x.shape
    xp = np.zeros((B, D + 2, H + 2, Wd + 2, C))
    xp[:, 1:-1, 1:-1, 1:-1] = x
    dxp = np.zeros_like(xp)
    dW = np.zeros_like(W)
    g2 = dz_.reshape(-1, dz_.shape[-1])
    for t, (dz, dy, dx) in enumerate(TAPS):
        sl = (slice(None), slice(1 + dz, 1 + dz + D), slice(1 + dy, 1 + dy + H), slice(1 + dx, 1 + dx + Wd))
        dxp[sl] += dz_ @ W[t].T
        dW[t] = xp[sl].reshape(-1, C).T @ g2
    return dxp[:, 1:-1, 1:-1, 1:-1], dW, g2.sum(axis=0)


def maxpool2(x):
    B, D, H, Wd, C = x.shape
    r = x.reshape(B, D // 2, 2, H // 2, 2, Wd // 2, 2, C).transpose(0, 1, 3, 5, 2, 4, 6, 7)
    r = r.reshape(B, D // 2, H // 2, Wd // 2, 8, C)
    idx = np.argmax(r, axis=4)
    return np.take_along_axis(r, idx[:, :, :, :, None, :], axis=4)[:, :, :, :, 0, :], idx


def maxpool2_backward(dy, idx, shape):
    B, D, H, Wd, C = shape
    g = np.zeros((B, D // 2, H // 2, Wd // 2, 8, C))
    np.put_along_axis(g, idx[:, :, :, :, None, :], dy[:, :, :, :, None, :], axis=4)
    g = g.reshape(B, D // 2, H // 2, Wd // 2, 2, 2, 2, C).transpose(0, 1, 4, 2, 5, 3, 6, 7)
    return g.reshape(B, D, H, Wd, C)


def up2(x, W, b):
    """Transposed 2^3 stride-2 convolution: out[2v + t] = x[v] @ W[t] + b,
    t = (tz, ty, tx) in {0,1}^3 as t = 4 tz + 2 ty + tx."""
    B, D, H, Wd, C = x.shape
    out = np.zeros((B, 2 * D, 2 * H, 2 * Wd, W.shape[2]))
    for t in range(8):
        tz, ty, tx = (t >> 2) & 1, (t >> 1) & 1, t & 1
        out[:, tz::2, ty::2, tx::2] = x @ W[t]
    return out + b


def up2_backward(x, W, dy):
    B, D, H, Wd, C = x.shape
    dx = np.zeros_like(x)
    dW = np.zeros_like(W)
    for t in range(8):
        tz, ty, tx = (t >> 2) & 1, (t >> 1) & 1, t & 1
        g = dy[:, tz::2, ty::2, tx::2]
        dx += g @ W[t].T
        dW[t] = x.reshape(-1, C).T @ g.reshape(-1, g.shape[-1])
    return dx, dW, dy.reshape(-1, dy.shape[-1]).sum(axis=0)


def forward(p, x, levels=4, bf=False):
    """Returns (prediction, cache).  The prediction is the head's linear output."""
    R = bf16 if bf else (lambda a: a)
    q = {k: (R(v) if k.endswith(".w") else v) for k, v in p.items()}
    cache = {"q": q}
    h = R(x)
    cache["x"] = h
    skips = []
    for l in range(levels):
        a = R(np.maximum(conv3(h, q[f"enc{l}a.w"], q[f"enc{l}a.b"]), 0.0))
        cache[f"enc{l}a.in"], cache[f"enc{l}a.out"] = h, a
        bb = R(np.maximum(conv3(a, q[f"enc{l}b.w"], q[f"enc{l}b.b"]), 0.0))
        cache[f"enc{l}b.in"], cache[f"enc{l}b.out"] = a, bb
        if l < levels - 1:
            skips.append(bb)
            h, idx = maxpool2(bb)
            cache[f"pool{l}.idx"], cache[f"pool{l}.shape"] = idx, bb.shape
        else:
            h = bb
    for l in range(levels - 2, -1, -1):
        u = R(up2(h, q[f"up{l}.w"], q[f"up{l}.b"]))
        cache[f"up{l}.in"] = h
        cat = np.concatenate([skips[l], u], axis=-1)
        a = R(np.maximum(conv3(cat, q[f"dec{l}a.w"], q[f"dec{l}a.b"]), 0.0))
        cache[f"dec{l}a.in"], cache[f"dec{l}a.out"] = cat, a
        bb = R(np.maximum(conv3(a, q[f"dec{l}b.w"], q[f"dec{l}b.b"]), 0.0))
        cache[f"dec{l}b.in"], cache[f"dec{l}b.out"] = a, bb
        h = bb
    W = q["head.w"]
    y = h @ W[0] + q["head.b"]
    cache["head.in"] = h
    return y, cache


def stored_slots(cin=5, base=16, levels=4, grid=16):
    """(name, grid, channels) of the tensors a forward pass stores, in the
    order: input; per level enc a, enc b (and the pooled tensor below the
    coarsest level); per decoder level, coarse to fine, up, dec a, dec b."""
    out = [("x", grid, cin)]
    for l in range(levels):
        w, g = base << l, grid >> l
        out += [(f"enc{l}a.out", g, w), (f"enc{l}b.out", g, w)]
        if l < levels - 1:
            out.append((f"pool{l}.out", g // 2, w))
    for l in range(levels - 2, -1, -1):
        w, g = base << l, grid >> l
        out += [(f"up{l}.out", g, w), (f"dec{l}a.out", g, w), (f"dec{l}b.out", g, w)]
    return out


def cache_at(p, acts, levels=4, bf=True):
    """The backward pass's cache for given stored forward tensors ``acts``
    (name -> array, names as in ``stored_slots``): the same cache ``forward``
    builds, with the max-pool routing (first maximum) recomputed from the
    stored enc b outputs.  Evaluating ``backward`` on it checks
    back-propagation layer by layer at that forward state."""
    R = bf16 if bf else (lambda a: a)
    q = {k: (R(v) if k.endswith(".w") else v) for k, v in p.items()}
    cache = {"q": q, "x": acts["x"]}
    h = acts["x"]
    for l in range(levels):
        cache[f"enc{l}a.in"], cache[f"enc{l}a.out"] = h, acts[f"enc{l}a.out"]
        cache[f"enc{l}b.in"], cache[f"enc{l}b.out"] = acts[f"enc{l}a.out"], acts[f"enc{l}b.out"]
        if l < levels - 1:
            _, idx = maxpool2(acts[f"enc{l}b.out"])
            cache[f"pool{l}.idx"], cache[f"pool{l}.shape"] = idx, acts[f"enc{l}b.out"].shape
            h = acts[f"pool{l}.out"]
        else:
            h = acts[f"enc{l}b.out"]
    for l in range(levels - 2, -1, -1):
        cache[f"up{l}.in"] = h
        cat = np.concatenate([acts[f"enc{l}b.out"], acts[f"up{l}.out"]], axis=-1)
        cache[f"dec{l}a.in"], cache[f"dec{l}a.out"] = cat, acts[f"dec{l}a.out"]
        cache[f"dec{l}b.in"], cache[f"dec{l}b.out"] = acts[f"dec{l}a.out"], acts[f"dec{l}b.out"]
        h = acts[f"dec{l}b.out"]
    cache["head.in"] = h
    return cache


def mse(y, target):
    d = y - target
    return float(np.mean(d * d)), 2.0 * d / d.size


def backward(p, cache, dy, levels=4, bf=False):
    """Gradients of every parameter given dL/dy (FP64 back-propagation
    through the forward of ``cache``).  ``bf=True`` rounds every stored
    activation gradient to bfloat16 where the GPU path stores it (the loss
    gradient, each input-gradient output, the pool routing plus skip sum)."""
    R = bf16 if bf else (lambda a: a)
    q = cache["q"]
    g = {}
    dy = R(dy)
    h = cache["head.in"]
    g["head.w"] = (h.reshape(-1, h.shape[-1]).T @ dy.reshape(-1, dy.shape[-1]))[None]
    g["head.b"] = dy.reshape(-1, dy.shape[-1]).sum(axis=0)
    dh = R(dy @ q["head.w"][0].T)
    dskip = {}
    # decoder in reverse order of the forward pass (level 0 first)
    for l in range(0, levels - 1):
        dzb = dh * (cache[f"dec{l}b.out"] > 0)
        da, g[f"dec{l}b.w"], g[f"dec{l}b.b"] = conv3_backward(cache[f"dec{l}b.in"], q[f"dec{l}b.w"], dzb)
        dza = R(da) * (cache[f"dec{l}a.out"] > 0)
        dcat, g[f"dec{l}a.w"], g[f"dec{l}a.b"] = conv3_backward(cache[f"dec{l}a.in"], q[f"dec{l}a.w"], dza)
        dcat = R(dcat)
        cs = cache[f"enc{l}b.out"].shape[-1]
        dskip[l] = dcat[..., :cs]
        du = dcat[..., cs:]
        dh, g[f"up{l}.w"], g[f"up{l}.b"] = up2_backward(cache[f"up{l}.in"], q[f"up{l}.w"], du)
        dh = R(dh)
    # dh is now the gradient of the bottleneck output (enc{levels-1}b.out)
    for l in range(levels - 1, -1, -1):
        if l < levels - 1:
            dh = R(maxpool2_backward(dh, cache[f"pool{l}.idx"], cache[f"pool{l}.shape"]) + dskip[l])
        dzb = dh * (cache[f"enc{l}b.out"] > 0)
        da, g[f"enc{l}b.w"], g[f"enc{l}b.b"] = conv3_backward(cache[f"enc{l}b.in"], q[f"enc{l}b.w"], dzb)
        dza = R(da) * (cache[f"enc{l}a.out"] > 0)
        dh, g[f"enc{l}a.w"], g[f"enc{l}a.b"] = conv3_backward(cache[f"enc{l}a.in"], q[f"enc{l}a.w"], dza)
        dh = R(dh)
    return g


def adam_init(p):
    return {"t": 0, "m": {k: np.zeros_like(v) for k, v in p.items()}, "v": {k: np.zeros_like(v) for k, v in p.items()}}


def adam_step(p, g, st, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """Adam (Kingma & Ba 2014, the optimiser named in Sec. 3.3)."""
    st["t"] += 1
    t = st["t"]
    out = {}
    for k, v in p.items():
        m = st["m"][k] = b1 * st["m"][k] + (1 - b1) * g[k]
        s = st["v"][k] = b2 * st["v"][k] + (1 - b2) * g[k] * g[k]
        mh = m / (1 - b1 ** t)
        sh = s / (1 - b2 ** t)
        out[k] = v - lr * mh / (np.sqrt(sh) + eps)
    return out
