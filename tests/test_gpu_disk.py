"""GPU parity on the disk model in the benchmark's launch configuration
(theta = 0.5, quadrupole, n_leaf = 16, groups of n_g = 128 -- the group size
the autotuner picks for the disk -- 64 SPH neighbours, the static NFW halo),
at 2^17 particles (26,214 gas), per particle against the FP64 oracle:

  * neighbour sets and h^2 bit for bit;
  * density, pressure and sound speed within 1e-5 relative;
  * total acceleration within 1e-5 of its summation scale
    sum_j |a_ij| (gravity) + sum_j |a_ij| (hydro) + |a_NFW|;
  * du/dt within 1e-5 of its own summation scale (the magnitudes of its
    pressure and viscosity terms), particle by particle;
  * NFW acceleration and potential per particle (stars only, no
    self-gravity) within 1e-5 relative;
  * one kick-drift-kick step: positions, velocities and u per particle.
"""
import numpy as np
import pytest

from paper_2510_23330_gb300 import ics

pytestmark = pytest.mark.gpu

TOL = 1e-5
N = 1 << 17
NG = 128


@pytest.fixture(scope="module")
def G():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_23330_gb300 import galnb
    return galnb


def _cfg(orc):
    return orc.Config(gravity="tree", theta=0.5, n_leaf=16, n_g=NG, quad=True, nfw_ms=ics.NFW_MS,
                      nfw_rs=ics.NFW_RS)


def _ctx(G, p):
    c = G.Context(theta=0.5, n_leaf=16, n_group=NG, multipole=1, nfw_ms=ics.NFW_MS, nfw_rs=ics.NFW_RS)
    c.set_particles(p)
    return c


def _scales(orc, s, f):
    ex, ey, ez, _ = orc.nfw(s, ics.NFW_MS, ics.NFW_RS)
    scale = f["grav"]["asum"] + np.sqrt(ex * ex + ey * ey + ez * ez)
    scale[f["gas_index"]] += f["sph"]["asum"]
    return scale


def _check_forces(c, orc, s, f):
    gi = f["gas_index"]
    h = f["sph"]
    assert np.array_equal(c.get("NBR"), np.sort(gi[h["nbr"]], axis=1))
    assert np.array_equal(c.get("H2")[gi], h["h2"])
    for k, r in (("RHO", h["rho"]), ("PRES", h["P"]), ("CS", h["c"])):
        assert np.max(np.abs(c.get(k)[gi] - r) / r) < TOL, k
    a = [c.get(k) for k in ("AX", "AY", "AZ")]
    d = np.sqrt((a[0] - f["ax"]) ** 2 + (a[1] - f["ay"]) ** 2 + (a[2] - f["az"]) ** 2)
    err = d / _scales(orc, s, f)
    assert err.max() < TOL, err.max()
    du = c.get("DUDT")[gi]
    derr = np.abs(du - h["dudt"]) / h["dusum"]
    assert derr.max() < TOL, derr.max()


def test_disk_2p17_forces_per_particle(G, orc):
    p = ics.config_disk(N)
    c = _ctx(G, p)
    c.compute_forces(G.GNB_GRAV_TREE)
    s = orc.state(p)
    f = orc.forces(s, _cfg(orc))
    _check_forces(c, orc, s, f)
    st = c.stats()
    assert st["NPP"] == f["grav"]["n_pp"] and st["NPC"] == f["grav"]["n_pc"]
    assert st["GROUPS"] == f["grav"]["groups"]


def test_disk_2p17_one_kdk_step_per_particle(G, orc):
    p = ics.config_disk(N)
    dt = 1e-3
    c = _ctx(G, p)
    c.step_kdk(dt, 1, G.GNB_GRAV_TREE)
    cfg = _cfg(orc)
    s = orc.state(p)
    f = orc.forces(s, cfg)
    s1, f1 = orc.kdk_step(s, f, dt, cfg)
    sc0 = _scales(orc, s, f)
    sc1 = _scales(orc, s1, f1)
    vmag = np.abs(s["vx"]) + np.abs(s["vy"]) + np.abs(s["vz"])
    for k in ("X", "Y", "Z"):
        # the drift uses the half-kick velocity rounded to FP32 (2^-24) and the
        # FP32 force (error below TOL of its scale): relative to dt (|v| + dt
        # scale) that is below TOL
        err = np.abs(c.get(k) - s1[k.lower()]) / (dt * (vmag + dt * sc0) + 1e-15)
        assert err.max() < TOL, k
    vscale = vmag + dt * (sc0 + sc1)
    for k in ("VX", "VY", "VZ"):
        assert np.max(np.abs(c.get(k) - s1[k.lower()]) / vscale) < TOL, k
    gi = f["gas_index"]
    uscale = s["u"][gi] + dt * (f["sph"]["dusum"] + f1["sph"]["dusum"])
    assert np.max(np.abs(c.get("U")[gi] - s1["u"][gi]) / uscale) < TOL


def test_nfw_halo_per_particle(G, orc):
    """Stars only and no self-gravity: the acceleration is the halo's alone."""
    p = ics.exp_disk(20000, gas_frac=0.0, seed=6)
    c = G.Context(nfw_ms=ics.NFW_MS, nfw_rs=ics.NFW_RS)
    c.set_particles(p)
    c.compute_forces(G.GNB_GRAV_NONE)
    ex, ey, ez, pot = orc.nfw(orc.state(p), ics.NFW_MS, ics.NFW_RS)
    a = [c.get(k) for k in ("AX", "AY", "AZ")]
    amag = np.sqrt(ex * ex + ey * ey + ez * ez)
    d = np.sqrt((a[0] - ex) ** 2 + (a[1] - ey) ** 2 + (a[2] - ez) ** 2)
    assert np.max(d / amag) < TOL
    assert np.max(np.abs(c.get("POT_EXT") - pot) / np.abs(pot)) < TOL
