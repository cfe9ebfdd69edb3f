"""GPU parity of the SPH path against the FP64 oracle.

Bit-exact: neighbour sets and the kernel support h^2 (the exact FP64 d^2 of
the 64th neighbour, ties broken by gas rank).  Floating point: density
within 1e-5 relative; hydro acceleration within 1e-5 of sum_j |a_ij|; du/dt
within 1e-5 of its summation's scale.
"""
import numpy as np
import pytest

from paper_2510_23330_gb300 import ics

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def G():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_23330_gb300 import galnb
    return galnb


def _gas(p):
    gi = np.nonzero(p["type"] == 1)[0]
    g = {k: np.asarray(p[k][gi], np.float64) for k in ("x", "y", "z", "m", "u", "vx", "vy", "vz")}
    return gi, g


def _check_knn(G, orc, p, sample=None, **kw):
    c = G.Context(**kw)
    c.set_particles(p)
    c.compute_sph_density()
    gi, g = _gas(p)
    nb = c.get("NBR")
    h2 = c.get("H2")
    if sample is None:
        sample = np.arange(gi.size)
    ref_nbr, ref_h2 = orc.knn(g, 64, sample=sample)
    ref_sets = np.sort(gi[ref_nbr], axis=1)
    assert np.array_equal(nb[sample], ref_sets)
    assert np.array_equal(h2[gi[sample]], ref_h2)
    return c, gi, g, ref_nbr, ref_h2


def test_knn_exact_plummer(G, orc):
    _check_knn(G, orc, ics.config_tiny())


def test_knn_exact_lattice_ties(G, orc):
    """Many equal distances: the 64th neighbour lies inside a shell of 24
    equidistant points and the kept members are the lowest gas ranks."""
    p = ics.lattice(12, spacing=0.5)
    c, gi, g, ref_nbr, ref_h2 = _check_knn(G, orc, p)
    interior = (p["x"] > 1.4) & (p["x"] < 4.1) & (p["y"] > 1.4) & (p["y"] < 4.1) & (p["z"] > 1.4) & (p["z"] < 4.1)
    assert np.all(ref_h2[interior] == 1.5)


@pytest.mark.parametrize("n", [64, 65, 300, 5000])
def test_knn_ragged_sizes(G, orc, n):
    p = ics.uniform_random(n, seed=n, gas_frac=1.0)
    _check_knn(G, orc, p)


def test_knn_mixed_types_and_clustered(G, orc):
    p = ics.exp_disk(20000, gas_frac=0.3, seed=5)
    _check_knn(G, orc, p)


def test_density_and_force(G, orc):
    p = ics.config_tiny()
    c = G.Context()
    c.set_particles(p)
    c.compute_sph_density()
    c.compute_sph_force()
    gi, g = _gas(p)
    h = orc.sph(g, 64)
    rho = c.get("RHO")[gi]
    assert np.max(np.abs(rho - h["rho"]) / h["rho"]) < TOL
    assert np.max(np.abs(c.get("PRES")[gi] - h["P"]) / h["P"]) < TOL
    assert np.max(np.abs(c.get("CS")[gi] - h["c"]) / h["c"]) < TOL
    ax, ay, az = (c.get(k)[gi] for k in ("AX", "AY", "AZ"))
    err = np.sqrt((ax - h["ax"]) ** 2 + (ay - h["ay"]) ** 2 + (az - h["az"]) ** 2) / h["asum"]
    assert err.max() < TOL
    du = c.get("DUDT")[gi]
    du_scale = np.max(np.abs(h["dudt"])) + 1e-30
    assert np.max(np.abs(du - h["dudt"])) / du_scale < 10 * TOL


def test_density_force_with_velocity_and_viscosity(G, orc):
    p = ics.uniform_random(3000, seed=3, gas_frac=1.0)
    c = G.Context(alpha_visc=1.0)
    c.set_particles(p)
    c.compute_sph_density()
    c.compute_sph_force()
    gi, g = _gas(p)
    h = orc.sph(g, 64, alpha=1.0)
    ax, ay, az = (c.get(k)[gi] for k in ("AX", "AY", "AZ"))
    err = np.sqrt((ax - h["ax"]) ** 2 + (ay - h["ay"]) ** 2 + (az - h["az"]) ** 2) / h["asum"]
    assert err.max() < TOL
    m = g["m"]
    # GPU momentum conservation of the hydro force
    tot = np.array([np.sum(m * a) for a in (ax, ay, az)])
    assert np.linalg.norm(tot) / np.sum(m * h["asum"]) < 1e-6


def test_disk_full_size_knn_sampled(G, orc):
    """2^20-particle disk (209,715 gas): neighbour sets and h^2 of a random
    sample of 400 gas particles are exact; density within 1e-5."""
    p = ics.config_disk(1 << 20)
    gi = np.nonzero(p["type"] == 1)[0]
    rng = np.random.default_rng(2)
    s = np.sort(rng.choice(gi.size, 400, replace=False))
    c, gi, g, ref_nbr, ref_h2 = _check_knn(G, orc, p, sample=s)
    rho, _, _ = orc.density(g, ref_nbr, ref_h2, sample=s)
    assert np.max(np.abs(c.get("RHO")[gi[s]] - rho) / rho) < TOL


def test_knn_unrankable_clump_reports_ecapacity(G, orc):
    """200 gas particles at one point: their 64 nearest neighbours are
    exact ties at d = 0, more than the buffer of entries ranked in FP64 (64)
    holds, so the search reports GNB_ECAPACITY after its bounded retries; the
    context then works on a regular set."""
    p = ics.uniform_random(3000, seed=11, gas_frac=1.0)
    for k in ("x", "y", "z"):
        p[k] = np.array(p[k], copy=True)
        p[k][:200] = p[k][0]
    c = G.Context()
    c.set_particles(p)
    with pytest.raises(G.GalnbError) as e:
        c.compute_sph_density()
    assert e.value.code == G.GNB_ECAPACITY
    q = ics.uniform_random(3000, seed=12, gas_frac=1.0)
    c.set_particles(q)
    c.compute_sph_density()
    gi, g = _gas(q)
    ref_nbr, ref_h2 = orc.knn(g, 64)
    assert np.array_equal(c.get("NBR"), np.sort(gi[ref_nbr], axis=1))


def _exploded(orc, n, seed):
    p = ics.sn_region(n, seed=seed, grid=32)
    s, _ = orc.inject_energy(orc.state(p), (0.0, 0.0, 0.0), ics.E_SN_CODE)
    return p, s


def test_pressure_energy_density_and_force(G, orc):
    """Pressure-energy SPH (sph_variant = 1) on an exploded region, where u
    spans orders of magnitude: smoothed pressure, sound speed, accelerations
    and du/dt against the oracle's pressure form."""
    p, s = _exploded(orc, 4000, 31)
    c = G.Context(sph_variant=1)
    c.set_particles(p)
    c.inject_energy((0.0, 0.0, 0.0), ics.E_SN_CODE)
    c.compute_sph_density()
    c.compute_sph_force()
    g = {k: np.asarray(s[k], np.float64) for k in ("x", "y", "z", "m", "u", "vx", "vy", "vz")}
    h = orc.sph(g, 64, alpha=1.0, pressure=True)
    u_gpu = c.get("U").astype(np.float64)
    assert np.max(np.abs(u_gpu - g["u"]) / g["u"]) < 2e-7  # same injected energies (FP32 storage)
    assert np.max(np.abs(c.get("RHO") - h["rho"]) / h["rho"]) < TOL
    assert np.max(np.abs(c.get("PRES") - h["P"]) / h["P"]) < TOL
    assert np.max(np.abs(c.get("CS") - h["c"]) / h["c"]) < TOL
    ax, ay, az = (c.get(k) for k in ("AX", "AY", "AZ"))
    err = np.sqrt((ax - h["ax"]) ** 2 + (ay - h["ay"]) ** 2 + (az - h["az"]) ** 2) / h["asum"]
    assert err.max() < TOL
    du = c.get("DUDT")
    assert np.max(np.abs(du - h["dudt"])) / np.max(np.abs(h["dudt"])) < 10 * TOL
    # the two formulations do differ here
    d = orc.sph(g, 64, alpha=1.0)
    assert np.max(np.abs(d["P"] - h["P"]) / h["P"]) > 1e-2


def test_pressure_energy_cfl_integration_matches_oracle(G, orc):
    p, s = _exploded(orc, 5000, 32)
    cfg = orc.Config(gravity="none", sph="pressure")
    f = orc.forces(s, cfg)
    span = 0.0
    for _ in range(5):
        dt = orc.cfl_dt(f, 0.3)
        s, f = orc.kdk_step(s, f, dt, cfg)
        span += dt
    c = G.Context(sph_variant=1)
    c.set_particles(p)
    c.inject_energy((0.0, 0.0, 0.0), ics.E_SN_CODE)
    t, n = c.integrate_cfl(span, 0.3, mode=G.GNB_GRAV_NONE)
    assert abs(t - span) < 1e-12 * span and n in (5, 6)
    for k in ("X", "Y", "Z"):
        assert np.max(np.abs(c.get(k) - s[k.lower()])) < 1e-5 * 60.0
    vmax = np.max(np.abs(s["vx"]))
    for k in ("VX", "VY", "VZ"):
        assert np.max(np.abs(c.get(k) - s[k.lower()])) < 2e-3 * vmax
    u = c.get("U")
    assert np.max(np.abs(u - s["u"]) / (np.abs(s["u"]) + 1e-3 * np.max(s["u"]))) < 2e-3
