"""Pins of the oracle's kick-drift-kick step (Sec. 3.2): time reversibility
and energy conservation of the coupled gravity + SPH system."""
import numpy as np

from paper_2510_23330_gb300 import ics


def _flip(s):
    s = dict(s)
    for k in ("vx", "vy", "vz"):
        s[k] = -s[k]
    return s


import pytest


@pytest.mark.parametrize("n_gas", [0, 256])
def test_kdk_time_reversible(orc, n_gas):
    """n steps forward, velocities flipped, n steps back: positions return to
    the start to round-off (viscosity off).  The gas pressure uses the
    internal energy predicted with the previous du/dt, which is not time
    symmetric, so u returns only to O(dt^3) per step."""
    p = ics.plummer(512, seed=4, n_gas=n_gas)
    cfg = orc.Config(gravity="direct", alpha=0.0)
    s0 = orc.state(p)
    s, f = s0, orc.forces(s0, cfg)
    for _ in range(8):
        s, f = orc.kdk_step(s, f, 1e-3, cfg)
    s = _flip(s)
    f = orc.forces(s, cfg)
    for _ in range(8):
        s, f = orc.kdk_step(s, f, 1e-3, cfg)
    for k in ("x", "y", "z"):
        assert np.max(np.abs(s[k] - s0[k])) < 1e-12 * (1 + np.max(np.abs(s0[k])))
    tol_u = 1e-12 if n_gas == 0 else 1e-8
    assert np.max(np.abs(s["u"] - s0["u"])) <= tol_u * (1 + np.max(np.abs(s0["u"])))


def test_kdk_energy_conserved(orc):
    p = ics.plummer(1024, seed=6, n_gas=512)
    cfg = orc.Config(gravity="direct", alpha=1.0)
    s = orc.state(p)
    f = orc.forces(s, cfg)
    d0 = orc.diagnostics(s, f)
    e0 = d0[0] + d0[1] + d0[2] + d0[3]
    for _ in range(10):
        s, f = orc.kdk_step(s, f, 1e-3, cfg)
    d = orc.diagnostics(s, f)
    e = d[0] + d[1] + d[2] + d[3]
    assert abs(e / e0 - 1.0) < 1e-5
    assert np.all(np.abs(d[4:7] - d0[4:7]) < 1e-12)
