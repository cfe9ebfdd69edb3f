"""Pins of the oracle's gravity (Eq. 1) against facts fixed outside it:
a Kepler orbit, the Plummer sphere's potential energy in closed form, and
momentum conservation from pairwise antisymmetry."""
import numpy as np
import pytest
from scipy import integrate

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


# --------------------------------------------------------------------------
# Static NFW halo (disk model's external potential).  The oracle writes the
# enclosed mass and the potential in closed form; these pins fix them from
# the halo's density profile alone, rho(r) = rho_s / ((r/rs) (1 + r/rs)^2)
# with Ms = 4 pi rho_s rs^3, by numerical quadrature and differentiation.
# --------------------------------------------------------------------------
_MS, _RS = 30.0, 8.0


def _nfw_points():
    r = np.array([1e-3, 0.05, 0.7, 3.0, 8.0, 20.0, 150.0])
    u = np.array([[0.6, -0.48, 0.64], [0.0, 0.0, 1.0], [-1.0, 0.0, 0.0], [0.36, 0.48, 0.8],
                  [0.0, -0.6, 0.8], [0.48, 0.64, 0.6], [-0.8, 0.0, -0.6]])
    return {"x": r * u[:, 0], "y": r * u[:, 1], "z": r * u[:, 2]}, r


def _menc_quad(r, G=1.0):
    rho_s = _MS / (4.0 * np.pi * _RS ** 3)
    f = lambda s: 4.0 * np.pi * s * s * rho_s / ((s / _RS) * (1.0 + s / _RS) ** 2)
    return integrate.quad(f, 0.0, r, epsabs=0.0, epsrel=1e-13, limit=200)[0]


def test_nfw_enclosed_mass_and_circular_speed(orc):
    """G M(<r) / r^2 = |a| and v_c^2 = r |a| = G M(<r) / r, with M(<r) the
    quadrature of the density profile; a points to the centre."""
    for G in (1.0, 4.30091e-3):
        p, r = _nfw_points()
        ax, ay, az, _ = orc.nfw(p, _MS, _RS, G)
        amag = np.sqrt(ax * ax + ay * ay + az * az)
        for i, ri in enumerate(r):
            m = _menc_quad(ri)
            assert abs(amag[i] * ri * ri / (G * m) - 1.0) < 1e-10, (ri, amag[i])
            assert abs(ri * amag[i] / (G * m / ri) - 1.0) < 1e-10
        # radial and inward: a . x = -|a| r
        adotx = ax * p["x"] + ay * p["y"] + az * p["z"]
        assert np.allclose(adotx, -amag * r, rtol=1e-12)


def test_nfw_potential_is_the_integral_of_the_force(orc):
    """Phi(r) = -G int_r^inf M(<s) / s^2 ds (Phi -> 0 at infinity), and a =
    -grad Phi by central differences (relative 1e-8); Phi(0) = -G Ms / rs."""
    p, r = _nfw_points()
    _, _, _, pot = orc.nfw(p, _MS, _RS)
    for i, ri in enumerate(r):
        tail = integrate.quad(lambda s: _menc_quad(s) / (s * s), ri, np.inf, epsabs=0.0,
                              epsrel=1e-11, limit=400)[0]
        assert abs(pot[i] / -tail - 1.0) < 1e-8, (ri, pot[i], -tail)
    ax, ay, az, _ = orc.nfw(p, _MS, _RS)
    for i, ri in enumerate(r):
        if ri < 0.01:
            continue
        h = 1e-4 * ri
        g = []
        for k in ("x", "y", "z"):
            pp = {a: np.array([p[a][i]]) for a in ("x", "y", "z")}
            pm = {a: np.array([p[a][i]]) for a in ("x", "y", "z")}
            pp[k] = pp[k] + h
            pm[k] = pm[k] - h
            g.append((orc.nfw(pp, _MS, _RS)[3][0] - orc.nfw(pm, _MS, _RS)[3][0]) / (2 * h))
        a = np.array([ax[i], ay[i], az[i]])
        assert np.linalg.norm(a + np.array(g)) < 1e-8 * np.linalg.norm(a), (ri, a, g)
    z = {"x": np.zeros(1), "y": np.zeros(1), "z": np.zeros(1)}
    ex, ey, ez, p0 = orc.nfw(z, _MS, _RS)
    assert ex[0] == 0.0 and ey[0] == 0.0 and ez[0] == 0.0
    assert abs(p0[0] / (-_MS / _RS) - 1.0) < 1e-15
