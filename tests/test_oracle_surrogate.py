"""Pins of the oracle's particle <-> grid mappings: the counter-based
generator against published SplitMix64 outputs, Shepard averaging as a
partition of unity, the kernel-convolved mass on the grid, and the Gibbs
remap's particle count and sampled marginals."""
import os

import numpy as np
from scipy import stats

from paper_2510_23330_gb300 import ics

HERE = os.path.dirname(os.path.abspath(__file__))


def test_splitmix64_golden(orc):
    from oracle import surrogate as S
    vals = [int(l) for l in open(os.path.join(HERE, "golden", "splitmix64_seed1234567.txt"))
            if l.strip() and not l.startswith("#")]
    x = 1234567
    for v in vals:
        # splitmix64(x) is next() applied to state x
        assert S.splitmix64(x) == v
        x = (x + 0x9E3779B97F4A7C15) & ((1 << 64) - 1)
    u = S.uniform(7, 11, 3)
    assert u == (S.splitmix64((S.splitmix64(18) + 3) & ((1 << 64) - 1)) >> 11) * 2.0 ** -53


def _lattice_region(n_side, side):
    p = ics.lattice(n_side, spacing=side / n_side, mass=1.0, u=1.0,
                    origin=(-0.5 * side + 0.5 * side / n_side,) * 3)
    return p


def test_shepard_partition_of_unity_and_mass(orc):
    from oracle import surrogate as S
    side, grid, ns = 16.0, 16, 24
    p = _lattice_region(ns, side)
    s = orc.state(p)
    s["vx"][:] = 3.0
    g = {k: s[k] for k in ("x", "y", "z", "m")}
    g["u"] = s["u"]
    nbr, h2 = orc.knn(g, 64)
    rho, _, _ = orc.density(g, nbr, h2)
    acc = S.accumulate(s["x"], s["y"], s["z"], s["m"], np.sqrt(h2), rho, s["u"] * S.T_PER_U, s["vx"], s["vy"],
                       s["vz"], (0, 0, 0), side, grid)
    z = S.standardise(acc)
    full = acc[:, 1] > 0
    assert np.allclose(z[full, 1], (np.log10(S.T_PER_U) - 2) / 2, atol=1e-12)   # T uniform
    assert np.allclose(z[full, 2], 3.0 / 20.0, atol=1e-12)                      # vx uniform
    # kernel-convolved mass on the grid: interior voxels hold the lattice density
    d3 = (side / grid) ** 3
    inner = np.zeros((grid,) * 3, bool)
    inner[4:-4, 4:-4, 4:-4] = True
    mean_rho = ns ** 3 / side ** 3
    assert abs(np.mean(acc[:, 0].reshape((grid,) * 3)[inner]) / mean_rho - 1.0) < 0.02


def test_gibbs_remap_count_and_marginals(orc):
    from oracle import surrogate as S
    grid, side = 8, 8.0
    fx = np.array([1, 2, 3, 4, 4, 3, 2, 1], float)
    fy = np.array([5, 1, 1, 1, 1, 1, 1, 5], float)
    fz = np.ones(8)
    w = (fz[:, None, None] * fy[None, :, None] * fx[None, None, :]).reshape(-1)
    pred = np.zeros((grid ** 3, 5))
    pred[:, 0] = np.log10(w) + 0.33
    n = 20000
    rng = np.random.default_rng(0)
    pos = rng.uniform(-4, 4, (n, 3))
    vox, newp, u, v = S.remap(pred, np.arange(n), pos, (0, 0, 0), side, grid, seed=5, sweeps=4)
    assert vox.shape == (n, 3) and np.all((vox >= 0) & (vox < grid))
    assert np.all(np.floor(newp + 4.0).astype(int) == vox)
    for a, f in ((0, fx), (1, fy)):
        obs = np.bincount(vox[:, a], minlength=grid)
        exp = f / f.sum() * n
        assert stats.chisquare(obs, exp).pvalue > 1e-3
    vox2, _, _, _ = S.remap(pred, np.arange(n), pos, (0, 0, 0), side, grid, seed=5, sweeps=4)
    assert np.array_equal(vox, vox2)
