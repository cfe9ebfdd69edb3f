"""Pins of the oracle's hierarchical (block) individual-timestep integrator:
level rules against enumeration, closed-form trajectories under constant and
time-linear accelerations (exact for kick-drift-kick whatever the step
sequence), the block-tick sequence of a scripted wake-up, the reduction to
the shared-timestep leapfrog when every particle has the same level, and the
Sedov-Taylor blast with CFL levels."""
import numpy as np
import pytest

from paper_2510_23330_gb300 import ics


def _particles(n, x, v):
    s = {"x": np.array([p[0] for p in x], float), "y": np.array([p[1] for p in x], float),
         "z": np.array([p[2] for p in x], float), "vx": np.array([p[0] for p in v], float),
         "vy": np.array([p[1] for p in v], float), "vz": np.array([p[2] for p in v], float),
         "m": np.ones(n), "eps": np.zeros(n), "u": np.zeros(n), "type": np.zeros(n, np.uint8),
         "id": np.arange(n)}
    return s


def test_levels_match_enumeration(orc):
    rng = np.random.default_rng(3)
    K, span = 6, 0.75
    dtc = np.concatenate([span * 2.0 ** -rng.uniform(-1, 8, 400), span * 2.0 ** -np.arange(0, 8),
                          [np.inf]])
    got = orc.hier_cfl_level(dtc, K, span)
    for d, g in zip(dtc, got):
        ok = [k for k in range(K + 1) if span / 2 ** k <= d]
        assert g == (min(ok) if ok else -1)
    for T in range(0, 2 ** (K + 1) + 1, 2):
        ok = [k for k in range(K + 1) if T % 2 ** (K + 1 - k) == 0]
        assert orc.hier_align_level(T, K) == min(ok)


def test_time_linear_coupling_closed_form(orc):
    """A has the constant acceleration g on level 0; B, on level 2, feels
    c times A's predicted velocity.  Kick-drift-kick is exact for A, and
    B's kicks are trapezoid sums of a linear function of time (exact), so
    v_B(T) = v_B0 + c (v_A0 T + g T^2 / 2); each of B's four steps drifts
    c g dt^3 / 6 short of the exact path.  Wrong prediction times (A is
    predicted backwards from its mid-step at t = T/4) break the velocity."""
    g, c, T = 0.7, 1.3, 2.0
    s = _particles(2, [(0.1, 0.2, 0.3), (-0.4, 0.5, 0.0)], [(0.3, -0.2, 0.1), (0.05, 0.0, -0.1)])

    def force_fn(st, u=None, v=None):
        vax = st["vx"][0] if v is None else v[0][0]
        return {"ax": np.array([g, c * vax]), "ay": np.zeros(2), "az": np.zeros(2), "dudt": np.zeros(2)}

    def step_fn(f, n):
        return np.array([T, T / 4])

    out, _, info = orc.integrate_hier(s, T, 0.3, None, max_level=4, force_fn=force_fn, step_fn=step_fn)
    assert info["t"] == T and info["steps"] == 4 and info["updates"] == 5 and info["wakeups"] == 0
    assert list(info["level"]) == [0, 2]
    assert np.isclose(out["vx"][0], 0.3 + g * T, rtol=0, atol=1e-14)
    assert np.isclose(out["x"][0], 0.1 + 0.3 * T + 0.5 * g * T * T, rtol=0, atol=1e-14)
    vb = 0.05 + c * (0.3 * T + 0.5 * g * T * T)
    assert np.isclose(out["vx"][1], vb, rtol=0, atol=1e-13)
    dt = T / 4
    xb = -0.4 + 0.05 * T + c * (0.3 * T * T / 2 + g * T ** 3 / 6) - 4 * c * g * dt ** 3 / 6
    assert np.isclose(out["x"][1], xb, rtol=0, atol=1e-13)
    assert out["vy"][0] == -0.2 and abs(out["y"][0] - (0.2 - 0.2 * T)) < 1e-15


def test_wakeup_tick_sequence_and_exactness(orc):
    """Scripted CFL steps (K = 3, 16 ticks): A starts on level 0, is woken at
    tick 4 by a CFL step of 0.13 T (level 3, aligned: next end at tick 6),
    then asks for level 0 but alignment holds it at 3 at tick 6 and at 1 at
    tick 8.  B ticks on level 2.  Under a constant acceleration the cut
    step's corrected kick and drift keep A on the exact parabola."""
    g, T = -0.9, 1.0
    s = _particles(2, [(1.0, 0.0, 0.0), (0.0, 0.0, 0.0)], [(0.2, 0.0, 0.0), (1.0, 0.0, 0.0)])
    times = []

    def force_fn(st, u=None, v=None):
        times.append(st["x"][1])  # B drifts at unit speed with no force: x_B = t
        return {"ax": np.array([g, 0.0]), "ay": np.zeros(2), "az": np.zeros(2), "dudt": np.zeros(2)}

    def step_fn(f, n):
        t = times[-1]
        return np.array([0.13 * T if abs(t - 0.25) < 1e-12 else T, T / 4])

    out, _, info = orc.integrate_hier(s, T, 0.3, None, max_level=3, force_fn=force_fn, step_fn=step_fn)
    assert np.allclose(times, [0.0, 0.25, 0.375, 0.5, 0.75, 1.0], rtol=0, atol=1e-15)
    assert info["steps"] == 5 and info["updates"] == 8 and info["wakeups"] == 1
    assert list(info["level"]) == [1, 2]
    assert np.isclose(out["x"][0], 1.0 + 0.2 * T + 0.5 * g * T * T, rtol=0, atol=1e-14)
    assert np.isclose(out["vx"][0], 0.2 + g * T, rtol=0, atol=1e-14)


def test_single_level_reduces_to_shared_leapfrog(orc):
    """All particles on level 2 (a constant step): four block steps are the
    shared kick-drift-kick leapfrog with dt = T/4 on the real SPH forces."""
    p = ics.uniform_box(10, seed=4, u=0.5)
    rng = np.random.default_rng(5)
    s = orc.state(p)
    for k in ("vx", "vy", "vz"):
        s[k] = rng.normal(0.0, 0.3, s[k].shape)
    cfg = orc.Config(gravity="none")
    T = 0.05
    out, f, info = orc.integrate_hier(s, T, 0.3, cfg, max_level=5,
                                      step_fn=lambda ff, n: np.full(n, 0.3 * T))
    assert info["steps"] == 4 and info["updates"] == 4 * len(s["x"]) and info["wakeups"] == 0
    ref, rf = s, orc.forces(s, cfg)
    for _ in range(4):
        ref, rf = orc.kdk_step(ref, rf, T / 4, cfg)
    for k in ("x", "y", "z", "vx", "vy", "vz", "u"):
        scale = np.max(np.abs(ref[k]))
        assert np.max(np.abs(out[k] - ref[k])) <= 1e-12 * scale, k


@pytest.mark.slow
def test_sedov_blast_with_individual_steps(orc):
    """The blast radius and total energy hold with CFL levels and wake-ups,
    while far fewer particle updates are made than by shared steps."""
    p = ics.uniform_box(16, seed=1)
    s = orc.state(p)
    cfg = orc.Config(gravity="none")
    e0 = np.sum(s["m"] * s["u"])
    s, _ = orc.inject_energy(s, (0.0, 0.0, 0.0), 1.0)
    t_end = (0.3 / 1.15) ** 2.5
    out, f, info = orc.integrate_hier(s, t_end, 0.3, cfg, max_level=16)
    assert info["t"] == t_end
    assert info["wakeups"] > 0 and len(set(info["level"])) >= 3
    assert info["updates"] < 0.5 * info["steps"] * len(s["x"])
    r = np.sqrt(out["x"] ** 2 + out["y"] ** 2 + out["z"] ** 2)
    rho = f["sph"]["rho"]
    shell = rho >= np.percentile(rho, 97)
    R = 1.15 * (t_end * t_end) ** 0.2
    assert abs(np.median(r[shell]) / R - 1.0) < 0.06
    e = 0.5 * np.sum(out["m"] * (out["vx"] ** 2 + out["vy"] ** 2 + out["vz"] ** 2)) + np.sum(out["m"] * out["u"])
    assert abs(e - e0 - 1.0) < 1e-3
