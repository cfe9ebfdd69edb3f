"""Pins of the oracle's SPH part: kernel normalisation and smoothness, kNN
against scipy's k-d tree, the uniform-lattice density and force, a linear
pressure gradient, momentum and energy conservation, and the viscosity
sign."""
import numpy as np
import pytest
from scipy import integrate
from scipy.spatial import cKDTree

from paper_2510_23330_gb300 import ics


def test_kernel_normalisation_and_smoothness(orc):
    h = 0.7
    f = lambda r: 4 * np.pi * r * r * orc.kernel(np.array([r]), h)[0][0]
    val, _ = integrate.quad(f, 0, h, points=[0.5 * h], epsabs=1e-13, epsrel=1e-13)
    assert abs(val - 1.0) < 1e-10
    r = np.array([0.0, 0.5 * h - 1e-9, 0.5 * h + 1e-9, h - 1e-9, h, 1.2 * h])
    w, dw = orc.kernel(r, h)
    assert dw[0] == 0.0 and w[4] == 0.0 and w[5] == 0.0 and dw[4] == 0.0
    assert abs(w[1] - w[2]) < 1e-7 * w[1] and abs(dw[1] - dw[2]) < 1e-6 * abs(dw[1])
    rr = np.linspace(0.01, 0.99, 99) * h
    wp, _ = orc.kernel(rr + 1e-6, h)
    wm, _ = orc.kernel(rr - 1e-6, h)
    _, dwr = orc.kernel(rr, h)
    assert np.allclose((wp - wm) / 2e-6, dwr, rtol=1e-5, atol=1e-8)


def test_knn_matches_kdtree(orc):
    rng = np.random.default_rng(7)
    pos = rng.normal(size=(3000, 3)) * np.array([1.0, 1.0, 0.1])
    g = {"x": pos[:, 0].copy(), "y": pos[:, 1].copy(), "z": pos[:, 2].copy()}
    nbr, h2 = orc.knn(g, 64)
    d, j = cKDTree(pos).query(pos, k=64)
    assert np.array_equal(np.sort(nbr, axis=1), np.sort(j, axis=1))
    assert np.allclose(h2, d[:, -1] ** 2, rtol=1e-12)
    assert np.all(nbr[:, 0] == np.arange(3000))  # self first (d^2 = 0)


def test_knn_ties_broken_by_index(orc):
    """On a lattice the 64th neighbour falls inside a shell of equal
    distances; the members kept are the lowest indices of that shell."""
    p = ics.lattice(9)
    nbr, h2 = orc.knn(p, 64, sample=np.array([364]))  # centre of 9^3
    d2 = ((p["x"] - p["x"][364]) ** 2 + (p["y"] - p["y"][364]) ** 2
          + (p["z"] - p["z"][364]) ** 2)
    shell6 = np.nonzero(np.isclose(d2, 6.0))[0]
    inner = np.nonzero(d2 < 5.5)[0]
    assert h2[0] == 6.0
    assert set(nbr[0]) == set(inner) | set(shell6[:64 - inner.size])


def test_lattice_density_closed_form(orc):
    """Simple cubic lattice, spacing D: shells at d^2/D^2 = 0,1,2,3,4,5,6 hold
    1,6,12,8,6,24,24 points, so the 64th neighbour lies at d^2 = 6 D^2 and
    rho = m sum_shell n_s W(sqrt(d_s^2), sqrt(6) D); this lattice sum is
    within 0.1 % of the continuum value m / D^3."""
    D, m = 0.5, 2.0
    p = ics.lattice(11, spacing=D, mass=m, u=1.0)
    c = 11 ** 3 // 2
    nbr, h2 = orc.knn(p, 64, sample=np.array([c]))
    assert h2[0] == 6.0 * D * D
    rho, P, cs = orc.density(p, nbr, h2, sample=np.array([c]))
    shells = np.array([0, 1, 2, 3, 4, 5, 6], float)
    counts = np.array([1, 6, 12, 8, 6, 24, 7], float)
    w, _ = orc.kernel(np.sqrt(shells) * D, np.sqrt(6.0) * D)
    assert np.isclose(rho[0], m * np.sum(counts * w), rtol=1e-13)
    assert abs(rho[0] / (m / D ** 3) - 1.0) < 1e-3
    assert np.isclose(P[0], (2.0 / 3.0) * rho[0] * 1.0, rtol=1e-14)
    assert np.isclose(cs[0], np.sqrt(5.0 / 3.0 * P[0] / rho[0]), rtol=1e-14)


def _lattice_sph(orc, n_side, u):
    p = ics.lattice(n_side, spacing=1.0, mass=1.0, u=1.0)
    g = {k: np.asarray(p[k], np.float64) for k in ("x", "y", "z", "m")}
    g["u"] = u
    return p, g, orc.sph(g, 64, u=u, v=(np.zeros(n_side ** 3),) * 3)


def test_lattice_uniform_pressure_no_force(orc):
    n = 12
    p, g, h = _lattice_sph(orc, n, np.ones(n ** 3))
    x, y, z = p["x"], p["y"], p["z"]
    interior = (x > 3) & (x < n - 4) & (y > 3) & (y < n - 4) & (z > 3) & (z < n - 4)
    a = np.sqrt(h["ax"] ** 2 + h["ay"] ** 2 + h["az"] ** 2)
    assert a[interior].max() < 1e-12 * h["asum"][interior].max()
    assert np.all(h["dudt"][interior] == 0.0)


def test_linear_pressure_gradient(orc):
    """u = 1 + 0.01 x on a lattice: rho is uniform, so a_x = -grad P / rho =
    -(gamma - 1) du/dx to within the SPH discretisation error."""
    n = 14
    p = ics.lattice(n)
    u = 1.0 + 0.01 * p["x"]
    _, _, h = _lattice_sph(orc, n, u)
    x, y, z = p["x"], p["y"], p["z"]
    interior = (x > 3) & (x < n - 4) & (y > 3) & (y < n - 4) & (z > 3) & (z < n - 4)
    expect = -(2.0 / 3.0) * 0.01
    assert np.allclose(h["ax"][interior], expect, rtol=0.05)
    assert np.abs(h["ay"][interior]).max() < 1e-3 * abs(expect)


def _random_gas(n, seed):
    p = ics.uniform_random(n, seed=seed, gas_frac=1.0)
    g = {k: np.asarray(p[k], np.float64) for k in ("x", "y", "z", "m", "u", "vx", "vy", "vz")}
    return g


def test_force_conserves_momentum_and_energy(orc):
    g = _random_gas(2000, 11)
    h = orc.sph(g, 64, alpha=1.0)
    m = g["m"]
    scale = np.sum(m * h["asum"])
    for k in ("ax", "ay", "az"):
        assert abs(np.sum(m * h[k])) < 1e-13 * scale
    de = np.sum(m * (g["vx"] * h["ax"] + g["vy"] * h["ay"] + g["vz"] * h["az"] + h["dudt"]))
    de_scale = np.sum(m * (np.abs(g["vx"] * h["ax"]) + np.abs(g["vy"] * h["ay"])
                           + np.abs(g["vz"] * h["az"]) + np.abs(h["dudt"])))
    assert abs(de) < 1e-12 * de_scale


def test_viscosity_heats_converging_flow_only(orc):
    n = 10
    p = ics.lattice(n)
    g = {k: np.asarray(p[k], np.float64) for k in ("x", "y", "z", "m")}
    g["u"] = np.full(n ** 3, 1e-6)
    conv = -0.5 * (g["x"] - g["x"].mean())
    zero = np.zeros(n ** 3)
    h_in = orc.sph(g, 64, alpha=1.0, u=g["u"], v=(conv, zero, zero))
    h_out = orc.sph(g, 64, alpha=1.0, u=g["u"], v=(-conv, zero, zero))
    h_off = orc.sph(g, 64, alpha=0.0, u=g["u"], v=(conv, zero, zero))
    c = n ** 3 // 2
    assert h_in["dudt"][c] > 0
    # expanding flow: only the (tiny) pressure work, which cools
    assert h_out["dudt"][c] < 0 and abs(h_out["dudt"][c]) < 1e-3 * h_in["dudt"][c]
    assert abs(h_off["dudt"][c]) < 1e-3 * h_in["dudt"][c]


# ---- pressure-energy SPH (the smoothed-pressure "density and pressure" form)
def test_pressure_form_equals_density_form_for_uniform_u(orc):
    """With one u for all particles the smoothed pressure is (gamma-1) u rho
    and the pair coefficients (gamma-1)^2 u^2 / P equal P / rho^2: the two
    formulations give the same forces and du/dt."""
    g = _random_gas(1500, 21)
    g["u"] = np.full(1500, 0.7)
    a = orc.sph(g, 64, alpha=1.0)
    b = orc.sph(g, 64, alpha=1.0, pressure=True)
    assert np.allclose(b["P"], a["P"], rtol=1e-13, atol=0)
    for k in ("ax", "ay", "az"):
        assert np.max(np.abs(b[k] - a[k])) < 1e-12 * np.max(a["asum"])
    assert np.max(np.abs(b["dudt"] - a["dudt"])) < 1e-12 * np.max(np.abs(a["dudt"]))


def test_pressure_form_conserves_momentum_and_energy(orc):
    g = _random_gas(2000, 22)
    g["u"] = g["u"] * (1.0 + 3.0 * np.random.default_rng(1).uniform(size=2000))
    h = orc.sph(g, 64, alpha=1.0, pressure=True)
    m = g["m"]
    scale = np.sum(m * h["asum"])
    for k in ("ax", "ay", "az"):
        assert abs(np.sum(m * h[k])) < 1e-13 * scale
    de = np.sum(m * (g["vx"] * h["ax"] + g["vy"] * h["ay"] + g["vz"] * h["az"] + h["dudt"]))
    de_scale = np.sum(m * (np.abs(g["vx"] * h["ax"]) + np.abs(g["vy"] * h["ay"])
                           + np.abs(g["vz"] * h["az"]) + np.abs(h["dudt"])))
    assert abs(de) < 1e-12 * de_scale


def test_pressure_form_has_no_force_at_a_contact(orc):
    """A lattice with masses 1 | 4 and u 4 | 1 across x = 6.5 is in pressure
    equilibrium (rho u = 4 on both sides).  Density-energy SPH smooths rho
    across the contact and pushes the particles next to it (the pressure
    blip); with the smoothed pressure m u = 4 everywhere, so the interior
    force vanishes to rounding."""
    n = 14
    p = ics.lattice(n)
    left = p["x"] < 6.5
    g = {k: np.asarray(p[k], np.float64) for k in ("x", "y", "z")}
    g["m"] = np.where(left, 1.0, 4.0)
    g["u"] = np.where(left, 4.0, 1.0)
    zero = (np.zeros(n ** 3),) * 3
    a = orc.sph(g, 64, u=g["u"], v=zero)
    b = orc.sph(g, 64, u=g["u"], v=zero, pressure=True)
    x, y, z = p["x"], p["y"], p["z"]
    interior = (x > 3) & (x < n - 4) & (y > 3) & (y < n - 4) & (z > 3) & (z < n - 4)
    contact = interior & (np.abs(x - 6.5) < 1.0)
    blip = np.max(np.abs(a["ax"][contact]))
    assert blip > 1e-2 * np.max(a["asum"][contact])  # density-energy SPH: a real spurious force
    ab = np.sqrt(b["ax"] ** 2 + b["ay"] ** 2 + b["az"] ** 2)
    assert np.max(ab[interior]) < 1e-12 * np.max(b["asum"][interior])


def test_force_sum_scales_bound_the_sums(orc):
    """asum and dusum are sums of term magnitudes: they bound |a| and |du/dt|
    (triangle inequality); with all velocities zero, du/dt and its scale
    vanish."""
    p = ics.uniform_random(1500, seed=8, gas_frac=1.0)
    g = {k: np.asarray(p[k], np.float64) for k in ("x", "y", "z", "m", "u", "vx", "vy", "vz")}
    h = orc.sph(g, 64)
    a = np.sqrt(h["ax"] ** 2 + h["ay"] ** 2 + h["az"] ** 2)
    assert np.all(a <= h["asum"] * (1 + 1e-12))
    assert np.all(np.abs(h["dudt"]) <= h["dusum"] * (1 + 1e-12)) and np.all(h["dusum"] > 0)
    z = orc.sph(g, 64, v=(np.zeros(1500), np.zeros(1500), np.zeros(1500)))
    assert np.all(z["dudt"] == 0) and np.all(z["dusum"] == 0)
