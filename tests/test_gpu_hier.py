"""GPU parity of the plain integration with hierarchical individual
timesteps against the oracle (block steps, updates, wake-ups and every
particle's level identical; the state within the shared-step tolerances),
the Sedov-Taylor blast with individual steps, and the error paths."""
import numpy as np
import pytest

from paper_2510_23330_gb300 import ics

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_23330_gb300 import galnb
    return galnb


def test_hier_matches_oracle(G, orc):
    """An exploded 5000-particle region over 12 of its shortest CFL steps
    (K = 12): 27 block steps with wake-ups on four levels.  Every level
    decision of the oracle lies at least 4e-5 (relative) from a level
    boundary, far outside the FP32 error of the GPU's signal velocities, so
    the decisions must agree exactly."""
    p = ics.sn_region(5000, seed=21, grid=32)
    cfg = orc.Config(gravity="none")
    s, _ = orc.inject_energy(orc.state(p), (0.0, 0.0, 0.0), ics.E_SN_CODE)
    f = orc.forces(s, cfg)
    span = 12 * float(np.min(orc.cfl_steps(f, len(s["x"]), 0.3)))
    ref, _, info = orc.integrate_hier(s, span, 0.3, cfg, max_level=12)
    assert info["margin"] > 4e-5 and info["wakeups"] > 0 and len(set(info["level"])) >= 4
    c = G.Context()
    c.set_particles(p)
    c.inject_energy((0.0, 0.0, 0.0), ics.E_SN_CODE)
    t, steps, updates, wakes = c.integrate_hier(span, 0.3, max_level=12, mode=G.GNB_GRAV_NONE)
    assert t == info["t"] == span
    assert (steps, updates, wakes) == (info["steps"], info["updates"], info["wakeups"])
    assert np.array_equal(c.get("LEVEL"), info["level"])
    side = 60.0
    for k in ("X", "Y", "Z"):
        assert np.max(np.abs(c.get(k) - ref[k.lower()])) < 1e-5 * side
    vmax = np.max(np.abs(ref["vx"]))
    for k in ("VX", "VY", "VZ"):
        assert np.max(np.abs(c.get(k) - ref[k.lower()])) < 2e-3 * vmax
    u = c.get("U")
    assert np.max(np.abs(u - ref["u"]) / (np.abs(ref["u"]) + 1e-3 * np.max(ref["u"]))) < 2e-3


def test_hier_sedov_taylor_blast_gpu(G):
    p = ics.uniform_box(32, seed=1)
    c = G.Context()
    c.set_particles(p)
    n = len(p["m"])
    e0 = float(np.sum(p["m"].astype(np.float64) * p["u"]))
    c.inject_energy((0.0, 0.0, 0.0), 1.0)
    t_end = (0.3 / 1.15) ** 2.5
    t, steps, updates, wakes = c.integrate_hier(t_end, 0.3, max_level=20, mode=G.GNB_GRAV_NONE)
    assert t == t_end and steps > 10 and wakes > 0
    assert updates < 0.5 * steps * n  # most particles are not updated at most block steps
    lev = c.get("LEVEL")
    assert lev.min() >= 0 and len(np.unique(lev)) >= 3
    x, y, z = c.get("X"), c.get("Y"), c.get("Z")
    r = np.sqrt(x * x + y * y + z * z)
    rho = c.get("RHO")
    shell = rho >= np.percentile(rho, 99)
    R = 1.15 * t ** 0.4
    assert abs(np.median(r[shell]) / R - 1.0) < 0.07
    m = p["m"].astype(np.float64)
    vx, vy, vz, u = (c.get(k).astype(np.float64) for k in ("VX", "VY", "VZ", "U"))
    e = 0.5 * np.sum(m * (vx * vx + vy * vy + vz * vz)) + np.sum(m * u)
    assert abs(e - e0 - 1.0) < 2e-3


def test_hier_errors_leave_the_context_usable(G):
    p = ics.sn_region(4000, seed=3, grid=32)
    c = G.Context()
    c.set_particles(p)
    with pytest.raises(G.GalnbError) as e:
        c.get("LEVEL")
    assert e.value.code == G.GNB_ESTATE
    for bad in ((0.0, 0.3, 12), (0.1, 0.0, 12), (0.1, 0.3, 0), (0.1, 0.3, 41), (float("nan"), 0.3, 12)):
        with pytest.raises(G.GalnbError) as e:
            c.integrate_hier(bad[0], bad[1], max_level=bad[2])
        assert e.value.code == G.GNB_EINVAL
    c.inject_energy((0.0, 0.0, 0.0), ics.E_SN_CODE)
    # the hot centre needs steps far below 0.1 / 2^4
    with pytest.raises(G.GalnbError) as e:
        c.integrate_hier(0.1, 0.3, max_level=4)
    assert e.value.code == G.GNB_ECAPACITY
    t, n = c.integrate_cfl(1e-4, 0.3, mode=G.GNB_GRAV_NONE)
    assert t == 1e-4 and n >= 1
    t, steps, updates, wakes = c.integrate_hier(1e-4, 0.3, max_level=20)
    assert t == 1e-4 and steps >= 1 and updates >= len(p["m"])
    assert np.all(np.isfinite(c.get("X"))) and c.get("LEVEL").min() >= 0


@pytest.mark.parametrize("max_steps", [3, 1 << 20])
def test_hier_with_direct_gravity_matches_oracle(G, orc, max_steps):
    """Stars and gas under direct self-gravity (stars on level 0, gas on its
    CFL levels; the force passes sort and build the gravity tree, so the step
    state must follow the particles through every sort).  Stopping after
    max_steps block steps leaves the same unsynchronised state as the
    oracle's."""
    p = ics.plummer(3000, seed=3, n_gas=1000, u_gas=0.05)
    cfg = orc.Config(gravity="direct")
    s = orc.state(p)
    f = orc.forces(s, cfg)
    span = 7.3 * float(np.min(orc.cfl_steps(f, len(s["x"]), 0.3)))
    ref, _, info = orc.integrate_hier(s, span, 0.3, cfg, max_level=10, max_steps=max_steps)
    assert info["margin"] > 1e-4 and len(set(info["level"])) >= 3
    c = G.Context()
    c.set_particles(p)
    t, steps, updates, wakes = c.integrate_hier(span, 0.3, max_level=10, max_steps=max_steps,
                                                mode=G.GNB_GRAV_DIRECT)
    assert t == info["t"] and (steps, updates, wakes) == (info["steps"], info["updates"], info["wakeups"])
    assert (t < span) == (max_steps == 3)
    assert np.array_equal(c.get("LEVEL"), info["level"])
    r = np.sqrt(ref["x"] ** 2 + ref["y"] ** 2 + ref["z"] ** 2)
    for k in ("X", "Y", "Z"):
        assert np.max(np.abs(c.get(k) - ref[k.lower()])) < 1e-5 * np.percentile(r, 90)
    vmax = np.max(np.abs(ref["vx"]))
    for k in ("VX", "VY", "VZ"):
        assert np.max(np.abs(c.get(k) - ref[k.lower()])) < 1e-4 * vmax
    gas = p["type"] == 1
    u = c.get("U")
    assert np.max(np.abs(u[gas] - ref["u"][gas]) / np.abs(ref["u"][gas])) < 1e-3
