"""Pins of the oracle's supernova-region integration: exact injected energy,
the Sedov-Taylor blast radius R = xi0 (E t^2 / rho)^{1/5} (xi0 = 1.15 for
gamma = 5/3) and energy conservation of the CFL-limited leapfrog."""
import numpy as np

from paper_2510_23330_gb300 import ics


def test_injection_members_and_energy(orc):
    p = ics.sn_region(4000, seed=2, grid=32)
    s = orc.state(p)
    pos = (0.5, -1.0, 2.0)
    E = ics.E_SN_CODE
    s1, info = orc.inject_energy(s, pos, E)
    d = np.sqrt((s["x"] - pos[0]) ** 2 + (s["y"] - pos[1]) ** 2 + (s["z"] - pos[2]) ** 2)
    nearest = np.argsort(d, kind="stable")[:64]
    assert set(info["members"]) == set(nearest)
    assert np.isclose(info["h"], np.sort(d)[63], rtol=1e-12)
    assert abs(info["energy_added"] / E - 1.0) < 1e-12
    changed = np.nonzero(s1["u"] != s["u"])[0]
    assert set(changed) <= set(nearest) and len(changed) >= 60  # W(h) = 0 for the 64th
    assert abs(np.sum(s["m"] * (s1["u"] - s["u"])) / E - 1.0) < 1e-12


def test_sedov_taylor_blast(orc):
    p = ics.uniform_box(16, seed=1)
    s = orc.state(p)
    cfg = orc.Config(gravity="none")
    e0 = np.sum(s["m"] * s["u"])
    s, info = orc.inject_energy(s, (0.0, 0.0, 0.0), 1.0)
    t_end = (0.3 / 1.15) ** 2.5
    s, f, t, nst = orc.integrate_cfl(s, t_end, 0.3, cfg)
    assert abs(t - t_end) < 1e-12 and nst > 5
    r = np.sqrt(s["x"] ** 2 + s["y"] ** 2 + s["z"] ** 2)
    rho = f["sph"]["rho"]
    shell = rho >= np.percentile(rho, 97)
    R = 1.15 * (1.0 * t * t / 1.0) ** 0.2
    assert abs(np.median(r[shell]) / R - 1.0) < 0.06
    e = 0.5 * np.sum(s["m"] * (s["vx"] ** 2 + s["vy"] ** 2 + s["vz"] ** 2)) + np.sum(s["m"] * s["u"])
    assert abs(e - e0 - 1.0) < 1e-3
