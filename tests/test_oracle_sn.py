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


# --------------------------------------------------------------------------
# Signal velocity and CFL timestep on a hand-built three-particle line.
# Particles at x = 0, 1, 3 with sound speeds 1, 2, 3; particle 2 moves at
# vx = -5 toward particle 1.  Neighbour rows (self first): 0 -> {0, 1},
# 1 -> {1, 0}, 2 -> {2, 1}, so the pair (1, 2) reaches particle 1 only
# through the symmetric set S_1 = N_1 u {j : 1 in N_j}.
#   pair (0,1): w = 0            -> c0 + c1          = 3
#   pair (2,1): w = (-5)(2)/2 = -5 -> c2 + c1 - 3w    = 20
#   vsig = max(2 c_i, pairs of S_i) = {3, 20, 20}.
# With h = {2, 0.5, 3}: dt = 0.3 min(h / vsig) = 0.3 * 0.025 = 0.0075.
# --------------------------------------------------------------------------
def _line3():
    g = {"x": np.array([0.0, 1.0, 3.0]), "y": np.zeros(3), "z": np.zeros(3),
         "vx": np.array([0.0, 0.0, -5.0]), "vy": np.zeros(3), "vz": np.zeros(3)}
    c = np.array([1.0, 2.0, 3.0])
    nbr = np.array([[0, 1], [1, 0], [2, 1]], np.int64)
    return g, c, nbr


def _vsig_planted(g, c, nbr, mistake):
    """The same rule with one plausible slip, to show that the pin below
    tells it apart."""
    n, k = nbr.shape
    out = 2.0 * c if mistake != "no_floor" else np.zeros(n)
    for i in range(n):
        for j in nbr[i]:
            if j == i:
                continue
            d = np.array([g[a][i] - g[a][j] for a in ("x", "y", "z")])
            dv = np.array([g[a][i] - g[a][j] for a in ("vx", "vy", "vz")])
            r = np.linalg.norm(d)
            w = dv @ d / r
            if mistake == "no_w":
                v = c[i] + c[j]
            elif mistake == "two_ci":
                v = 2 * c[i] - 3 * min(w, 0.0)
            elif mistake == "w_sign":
                v = c[i] + c[j] - 3 * max(w, 0.0)
            else:
                v = c[i] + c[j] - 3 * min(w, 0.0)
            out[i] = max(out[i], v)
            if mistake != "one_sided":
                out[j] = max(out[j], v)
    return out


def test_signal_velocity_hand_built(orc):
    g, c, nbr = _line3()
    vs = orc.sph_vsig(g, nbr, c)
    assert np.array_equal(vs, [3.0, 20.0, 20.0])
    for mistake in ("no_w", "two_ci", "w_sign", "one_sided"):
        assert not np.array_equal(_vsig_planted(g, c, nbr, mistake), vs), mistake
    assert np.array_equal(_vsig_planted(g, c, nbr, None), vs)


def test_cfl_timestep_hand_built(orc):
    g, c, nbr = _line3()
    f = {"sph": {"h2": np.array([4.0, 0.25, 9.0]), "vsig": orc.sph_vsig(g, nbr, c)}}
    dt = orc.cfl_dt(f, 0.3)
    assert abs(dt - 0.0075) < 1e-15
    # plausible slips: h^2 for h, max for min, vsig of the 2 c_i floor only
    h2, vs = f["sph"]["h2"], f["sph"]["vsig"]
    assert abs(0.3 * np.min(h2 / vs) - dt) > 1e-4
    assert abs(0.3 * np.max(np.sqrt(h2) / vs) - dt) > 1e-4
    assert abs(0.3 * np.min(np.sqrt(h2) / (2 * c)) - dt) > 1e-4
