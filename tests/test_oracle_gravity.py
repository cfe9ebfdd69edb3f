"""Pins of the oracle's gravity (Eq. 1) against facts fixed outside it:
a Kepler orbit, the Plummer sphere's potential energy in closed form, and
momentum conservation from pairwise antisymmetry."""
import numpy as np
import pytest

from paper_2510_23330_gb300 import ics


def test_kepler_orbit_period_and_energy(orc):
    """Two bodies, m1 = m2 = 1/2, a = 1, e = 0.5, eps = 0, G = 1: after one
    period 2 pi (Kepler's third law) the pair is back at pericentre and the
    leapfrog energy error stays bounded at O(dt^2); E = -G m1 m2 / (2a)."""
    p = ics.kepler_pair(a=1.0, e=0.5)
    s = orc.state(p)
    cfg = orc.Config(gravity="direct")
    f = orc.forces(s, cfg)
    e0 = orc.diagnostics(s, f)
    # velocities are stored in FP32, so E is exact only to ~1e-8
    assert abs((e0[0] + e0[1]) - (-0.125)) < 1e-7
    nsteps = 4000
    dt = 2 * np.pi / nsteps
    emax = 0.0
    for _ in range(nsteps):
        s, f = orc.kdk_step(s, f, dt, cfg)
        d = orc.diagnostics(s, f)
        emax = max(emax, abs((d[0] + d[1]) / -0.125 - 1.0))
    # back at pericentre: separation a(1-e) = 0.5 along +x for body 2
    sep = np.array([s["x"][1] - s["x"][0], s["y"][1] - s["y"][0], s["z"][1] - s["z"][0]])
    assert np.allclose(sep, [0.5, 0.0, 0.0], atol=2e-3)
    assert emax < 2e-3
    # momentum of the pair stays zero
    assert abs(d[4]) < 1e-13 and abs(d[5]) < 1e-13


def test_plummer_potential_energy_closed_form(orc):
    """E[W_N] = -(3 pi / 32)(1 - 1/N) for G = M = a = 1; the ensemble mean over
    seeds must agree within 3 standard errors (softening bias O(eps^2) is
    far below that)."""
    n, seeds = 2048, 24
    w = []
    for s in range(seeds):
        p = ics.plummer(n, seed=100 + s, eps=0.001)
        g = orc.direct_gravity(p)
        w.append(0.5 * np.sum(p["m"].astype(np.float64) * g["phi"]))
    w = np.array(w)
    expect = -(3 * np.pi / 32) * (1 - 1 / n)
    se = w.std(ddof=1) / np.sqrt(seeds)
    assert abs(w.mean() - expect) < 3 * se, (w.mean(), expect, se)
    assert se < 0.01 * abs(expect)


def test_momentum_conserved_pairwise(orc):
    p = ics.plummer(1024, seed=3)
    g = orc.direct_gravity(p)
    m = p["m"].astype(np.float64)
    tot = np.array([np.sum(m * g[k]) for k in ("ax", "ay", "az")])
    scale = np.sum(m * g["asum"])
    assert np.linalg.norm(tot) / scale < 1e-13


def test_point_mass_far_field(orc):
    """A test particle far from a compact cluster feels -G M r / r^3 to
    O((size/r)^2): checks sign, G and the inverse-square law."""
    rng = np.random.default_rng(0)
    k = 200
    pos = rng.uniform(-0.01, 0.01, (k, 3))
    pos = np.vstack([pos, [[10.0, 0.0, 0.0]]])
    p = {"x": pos[:, 0].copy(), "y": pos[:, 1].copy(), "z": pos[:, 2].copy(),
         "m": np.full(k + 1, 1.0 / k), "eps": np.zeros(k + 1)}
    p["m"][-1] = 1e-9
    g = orc.direct_gravity(p, G=2.0)
    com = np.mean(pos[:k], axis=0)
    d = pos[-1] - com
    expect = -2.0 * 1.0 * d / np.linalg.norm(d) ** 3
    got = np.array([g["ax"][-1], g["ay"][-1], g["az"][-1]])
    assert np.allclose(got, expect, rtol=1e-5)
    assert abs(g["phi"][-1] - (-2.0 / np.linalg.norm(d))) < 1e-6
