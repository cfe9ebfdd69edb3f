"""Pins of the U-Net oracle: a delta input through a 3^3 convolution returns
the mirrored kernel, a 1^3 convolution is a matrix product, a transposed
convolution places each input voxel's product in its 2^3 block, max-pool picks
block maxima, finite differences confirm the back-propagated gradients, and
one Adam step matches its closed form."""
import numpy as np
import pytest

from oracle import unet
from oracle import unet as U


def test_conv_delta_returns_mirrored_kernel():
    rng = np.random.default_rng(0)
    W = rng.normal(size=(27, 1, 1))
    x = np.zeros((1, 5, 5, 5, 1))
    x[0, 2, 2, 2, 0] = 1.0
    y = unet.conv3(x, W, np.zeros(1))
    for t, (dz, dy, dx) in enumerate(unet.TAPS):
        # out[v] = sum_t x[v + t] W[t]  ->  the impulse at c lands at c - t
        assert y[0, 2 - dz, 2 - dy, 2 - dx, 0] == W[t, 0, 0]
    assert np.count_nonzero(y) == 27


def test_conv1_is_matmul_and_bias():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 3, 4, 5, 6))
    W = rng.normal(size=(6, 7))
    b = rng.normal(size=7)
    ref = np.einsum("bzyxc,cd->bzyxd", x, W) + b
    W27 = np.zeros((27, 6, 7))
    W27[13] = W  # the centre tap (0, 0, 0)
    assert unet.TAPS[13] == (0, 0, 0)
    assert np.allclose(unet.conv3(x, W27, b), ref, rtol=1e-13)


def test_up2_blocks_and_maxpool():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(1, 2, 2, 2, 3))
    W = rng.normal(size=(8, 3, 4))
    y = unet.up2(x, W, np.zeros(4))
    assert y.shape == (1, 4, 4, 4, 4)
    assert np.allclose(y[0, 3, 2, 1], x[0, 1, 1, 0] @ W[4 + 0 + 1])
    z = rng.normal(size=(1, 4, 4, 4, 2))
    m, idx = unet.maxpool2(z)
    assert np.allclose(m[0, 1, 0, 1], z[0, 2:4, 0:2, 2:4].reshape(-1, 2).max(axis=0))


def test_bf16_rounding():
    v = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -3.14159265, 1e-30])
    r = unet.bf16(v)
    assert r[0] == 1.0 and r[1] == 1.0          # tie to even
    assert r[2] == 1.0 + 2 ** -7                 # above half: rounds up
    assert abs(r[3] + 3.140625) < 1e-12
    assert abs(r[4] / 1e-30 - 1) < 2 ** -8


def test_gradients_by_finite_differences():
    p = unet.init_params(seed=3, cin=5, cout=5, base=4, levels=3)
    rng = np.random.default_rng(4)
    x = rng.normal(size=(1, 8, 8, 8, 5))
    t = rng.normal(size=(1, 8, 8, 8, 5))
    y, cache = unet.forward(p, x, levels=3)
    loss, dy = unet.mse(y, t)
    g = unet.backward(p, cache, dy, levels=3)
    for name in ("enc0a.w", "enc2b.w", "up0.w", "dec1a.w", "head.w", "enc1a.b", "up1.b"):
        flat = p[name].reshape(-1)
        for k in rng.choice(flat.size, 3, replace=False):
            e = 1e-6 * max(1.0, abs(flat[k]))
            pp = {a: b.copy() for a, b in p.items()}
            pp[name].reshape(-1)[k] += e
            lp, _ = unet.mse(unet.forward(pp, x, levels=3)[0], t)
            pp[name].reshape(-1)[k] -= 2 * e
            lm, _ = unet.mse(unet.forward(pp, x, levels=3)[0], t)
            fd = (lp - lm) / (2 * e)
            an = g[name].reshape(-1)[k]
            assert abs(fd - an) <= 1e-6 * max(abs(fd), abs(an)) + 1e-12, (name, k, fd, an)


def test_adam_first_step_closed_form():
    p = {"w": np.array([1.0, -2.0])}
    g = {"w": np.array([0.5, -0.25])}
    st = unet.adam_init(p)
    q = unet.adam_step(p, g, st, lr=0.1)
    # after one step m_hat = g, v_hat = g^2: the update is lr * sign(g) (up to eps)
    assert np.allclose(q["w"], p["w"] - 0.1 * np.sign(g["w"]), atol=1e-7)


def test_cache_at_own_activations_reproduces_backward():
    """The cache rebuilt from a forward pass's own stored tensors gives the
    same gradients as the forward pass's cache (bit for bit)."""
    rng = np.random.default_rng(4)
    levels, grid = 3, 8
    p = U.init_params(2, 5, 5, 8, levels)
    for k in p:
        if k.endswith(".b"):
            p[k] = rng.normal(0, 0.1, p[k].shape)
    x = U.bf16(rng.normal(size=(2, grid, grid, grid, 5)))
    y, cache = U.forward(p, x, levels=levels, bf=True)
    _, dy = U.mse(y, rng.normal(size=y.shape))
    acts = {"x": cache["x"]}
    for name, g, c in U.stored_slots(5, 8, levels, grid)[1:]:
        if name.startswith("pool"):
            l = int(name[4])
            acts[name] = U.maxpool2(cache[f"enc{l}b.out"])[0]
        elif name.startswith("up"):
            l = int(name[2])
            acts[name] = cache[f"dec{l}a.in"][..., cache[f"enc{l}b.out"].shape[-1]:]
        else:
            acts[name] = cache[name]
        assert acts[name].shape[1:] == (g, g, g, c)
    g0 = U.backward(p, cache, dy, levels=levels, bf=True)
    g1 = U.backward(p, U.cache_at(p, acts, levels=levels, bf=True), dy, levels=levels, bf=True)
    for k in g0:
        assert np.array_equal(g0[k], g1[k]), k
