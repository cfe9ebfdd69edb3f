"""Checkpoint and resume through the C ABI (gnb_save / gnb_load for the
particle state, gnb_unet_save / gnb_unet_load for the network with its Adam
state).

Round trip: every field a loaded context returns equals the saving
context's bit for bit.  Resume: a star-only tree-gravity run continued from
the file matches the uninterrupted run bit for bit (the tree build, walk and
evaluation are deterministic, and the sort order depends only on the keys and
caller indices).  With gas, the kernel-size search and the symmetric lists
append entries with atomics, so sums may take another order from one run to
the next; the artificial viscosity's switch between approaching and receding
pairs can turn such a last-bit difference into a small change of one pair's
term, so two runs of the same state agree to ~1e-10 of the extent after two
steps, not bit for bit.  The gas resume is compared at that scale.  A
network resumed from its checkpoint trains on as the saved one does, which a
network given only its parameters (Adam state reset) does not.
"""
import numpy as np
import pytest

from paper_2510_23330_gb300 import ics

pytestmark = pytest.mark.gpu

STATE = ["X", "Y", "Z", "VX", "VY", "VZ", "U", "ID"]
GRAV = ["AX", "AY", "AZ", "POT", "POT_EXT", "AGRAV_X", "AGRAV_Y", "AGRAV_Z"]
GAS = ["DUDT", "RHO", "PRES", "CS", "H2"]


@pytest.fixture(scope="module")
def G():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_23330_gb300 import galnb
    return galnb


def _fields(c, names):
    return {k: c.get(k) for k in names}


def _same(a, b):
    for k in a:
        assert a[k].dtype == b[k].dtype and np.array_equal(a[k].view(np.uint8), b[k].view(np.uint8)), k


def test_star_only_resume_is_bit_exact(G, tmp_path):
    p = ics.plummer(8192, seed=11, n_gas=0)
    kw = dict(theta=0.5, multipole=1, n_group=64)
    a = G.Context(**kw)
    a.set_particles(p)
    a.step_kdk(1e-3, 2)
    path = tmp_path / "stars.gnb"
    a.save(str(path))
    b = G.Context(**kw)
    b.load(str(path))
    assert b.n == a.n and b.n_gas == 0
    _same(_fields(a, STATE + GRAV), _fields(b, STATE + GRAV))
    a.step_kdk(1e-3, 3)
    b.step_kdk(1e-3, 3)
    _same(_fields(a, STATE + GRAV), _fields(b, STATE + GRAV))


def test_gas_round_trip_and_resume(G, tmp_path):
    p = ics.config_disk(1 << 15, seed=5)
    kw = dict(theta=0.5, multipole=1, n_group=64, nfw_ms=ics.NFW_MS, nfw_rs=ics.NFW_RS)
    a = G.Context(**kw)
    a.set_particles(p)
    a.step_kdk(1e-3, 2)
    path = tmp_path / "disk.gnb"
    a.save(str(path))
    b = G.Context(**kw)
    b.load(str(path))
    assert (b.n, b.n_gas) == (a.n, a.n_gas)
    _same(_fields(a, STATE + GRAV + GAS), _fields(b, STATE + GRAV + GAS))
    with pytest.raises(G.GalnbError):
        b.get("NBR")  # neighbour lists are not in the file
    a.step_kdk(1e-3, 2)
    b.step_kdk(1e-3, 2)
    fa, fb = _fields(a, STATE), _fields(b, STATE)
    assert np.array_equal(fa["ID"], fb["ID"])
    scale = max(np.ptp(fa["X"]), np.ptp(fa["Y"]), np.ptp(fa["Z"]))
    for k in ("X", "Y", "Z"):
        assert np.max(np.abs(fa[k] - fb[k])) <= 1e-9 * scale, k
    vmax = max(np.max(np.abs(fa[k])) for k in ("VX", "VY", "VZ"))
    for k in ("VX", "VY", "VZ"):
        assert np.max(np.abs(fa[k].astype(np.float64) - fb[k])) <= 1e-4 * vmax, k
    gas = p["type"] == 1
    du = np.abs(fa["U"].astype(np.float64) - fb["U"])[gas]
    assert np.max(du / fa["U"][gas]) <= 1e-4


def test_state_file_errors(G, tmp_path):
    c = G.Context()
    with pytest.raises(G.GalnbError) as e:
        c.load(str(tmp_path / "missing.gnb"))
    assert e.value.code == G.GNB_EINVAL
    with pytest.raises(G.GalnbError) as e:
        c.save(str(tmp_path / "empty.gnb"))  # no particles yet
    assert e.value.code == G.GNB_ESTATE
    c.set_particles(ics.plummer(256, seed=2, n_gas=0))
    path = tmp_path / "short.gnb"
    c.save(str(path))
    data = path.read_bytes()
    path.write_bytes(data[: len(data) // 2])
    d = G.Context()
    with pytest.raises(G.GalnbError) as e:
        d.load(str(path))
    assert e.value.code == G.GNB_EINVAL
    path.write_bytes(b"not a state file" + data[16:])
    with pytest.raises(G.GalnbError) as e:
        d.load(str(path))
    assert e.value.code == G.GNB_EINVAL


def test_unet_checkpoint_resumes_training(G, tmp_path):
    from paper_2510_23330_gb300 import surrogate as S
    shape = dict(cin=5, cout=5, base=16, levels=3, grid=16)
    rng = np.random.default_rng(3)
    x = rng.standard_normal((2, 16, 16, 16, 5)).astype(np.float32)
    y = rng.standard_normal((2, 16, 16, 16, 5)).astype(np.float32)
    a = G.UNet(**shape)
    a.set_params(S.he_init(cin=5, cout=5, base=16, levels=3, seed=4))
    for _ in range(3):
        a.train_step(x[:1], y[:1], 1e-3)
    path = tmp_path / "net.gnbu"
    a.save(str(path))
    b = G.UNet(**shape)
    b.load(str(path))
    assert np.array_equal(a.get_params(), b.get_params())
    assert np.array_equal(a.forward(x), b.forward(x))
    # one more step on both: the same update (the weight gradients add
    # split-K partial sums with atomics, so within FP32 rounding)
    c = G.UNet(**shape)
    c.set_params(a.get_params())  # parameters only: Adam restarts at step 1
    a.train_step(x[1:], y[1:], 1e-3)
    b.train_step(x[1:], y[1:], 1e-3)
    c.train_step(x[1:], y[1:], 1e-3)
    pa, pb, pc = a.get_params(), b.get_params(), c.get_params()
    step = np.abs(pa - S.he_init(cin=5, cout=5, base=16, levels=3, seed=4)).max()
    assert np.max(np.abs(pa - pb)) <= 1e-3 * step
    assert np.max(np.abs(pa - pc)) > 1e-2 * step
    other = G.UNet(cin=5, cout=5, base=8, levels=3, grid=16)
    with pytest.raises(G.GalnbError) as e:
        other.load(str(path))
    assert e.value.code == G.GNB_EMISMATCH
    for n in (a, b, c, other):
        n.close()


def _state(c, p):
    """The particles of context c with the accelerations of their state, in
    the caller's order."""
    s = {k: p[k] for k in ("id", "type", "m", "eps")}
    for k, f in (("x", "X"), ("y", "Y"), ("z", "Z"), ("vx", "VX"), ("vy", "VY"), ("vz", "VZ"), ("u", "U"),
                 ("ax", "AX"), ("ay", "AY"), ("az", "AZ"), ("dudt", "DUDT"), ("h2", "H2")):
        s[k] = c.get(f)
    return s


def test_set_state_continues_without_a_force_pass(G):
    """gnb_set_state with a context's state and accelerations: the next KDK
    step kicks with them (one force evaluation per step, not two) and, for
    stars (deterministic tree gravity), gives the context's own next step bit
    for bit."""
    p = ics.plummer(8192, seed=12, n_gas=0)
    kw = dict(theta=0.5, multipole=1, n_group=64)
    a = G.Context(**kw)
    a.set_particles(p)
    a.step_kdk(1e-3, 2)
    b = G.Context(**kw)
    b.set_state(_state(a, p))
    for f in ("AX", "AY", "AZ"):
        assert np.array_equal(a.get(f), b.get(f)), f
    b.set_timing(True)
    a.step_kdk(1e-3, 1)
    b.step_kdk(1e-3, 1)
    _, calls, _ = b.phase_times()
    assert calls["GRAVITY"] == 1
    _same(_fields(a, STATE + ["AX", "AY", "AZ"]), _fields(b, STATE + ["AX", "AY", "AZ"]))
    # a plain upload evaluates the forces first
    c = G.Context(**kw)
    c.set_particles({k: v for k, v in _state(b, p).items() if k in p})
    c.set_timing(True)
    c.step_kdk(1e-3, 1)
    assert c.phase_times()[1]["GRAVITY"] == 2
    for x in (a, b, c):
        x.close()


def test_set_state_gas(G):
    """With gas: the supports and du/dt go with the state; the continued
    step matches the context's own within the run-to-run spread of the
    kernel-size search's atomics (see the module docstring)."""
    p = ics.config_disk(1 << 15, seed=6)
    kw = dict(theta=0.5, multipole=1, n_group=64, nfw_ms=ics.NFW_MS, nfw_rs=ics.NFW_RS)
    a = G.Context(**kw)
    a.set_particles(p)
    a.step_kdk(1e-3, 2)
    b = G.Context(**kw)
    b.set_state(_state(a, p))
    assert b.n_gas == a.n_gas
    a.step_kdk(1e-3, 1)
    b.step_kdk(1e-3, 1)
    fa, fb = _fields(a, STATE), _fields(b, STATE)
    scale = max(np.ptp(fa["X"]), np.ptp(fa["Y"]), np.ptp(fa["Z"]))
    for k in ("X", "Y", "Z"):
        assert np.max(np.abs(fa[k] - fb[k])) <= 1e-9 * scale, k
    vmax = max(np.max(np.abs(fa[k])) for k in ("VX", "VY", "VZ"))
    for k in ("VX", "VY", "VZ"):
        assert np.max(np.abs(fa[k].astype(np.float64) - fb[k])) <= 1e-4 * vmax, k
    gas = p["type"] == 1
    assert np.max(np.abs(fa["U"].astype(np.float64) - fb["U"])[gas] / fa["U"][gas]) <= 1e-4
    with pytest.raises(G.GalnbError) as e:
        b.set_state(_state(a, p), mode=7)
    assert e.value.code == G.GNB_EINVAL
    for x in (a, b):
        x.close()


def test_get_fields_equals_get(G):
    """gnb_get_fields: the same values as one gnb_get per field, host and
    device destinations; a field that is not current fails before any copy."""
    torch = pytest.importorskip("torch")
    p = ics.config_disk(1 << 14, seed=8)
    c = G.Context(theta=0.5, multipole=1, n_group=64, nfw_ms=ics.NFW_MS, nfw_rs=ics.NFW_RS)
    c.set_particles(p)
    c.step_kdk(1e-3, 1)
    names = ["X", "VZ", "U", "AX", "DUDT", "H2", "ID"]
    ref = {k: c.get(k) for k in names}
    host = {k: np.zeros_like(v) for k, v in ref.items()}
    c.get_fields(host)
    dev = {k: torch.zeros(v.shape[0], dtype=getattr(torch, str(v.dtype)), device="cuda") for k, v in ref.items()}
    c.get_fields(dev)
    for k in names:
        assert np.array_equal(host[k], ref[k]), k
        assert np.array_equal(dev[k].cpu().numpy(), ref[k]), k
    d = G.Context()
    d.set_particles(p)
    out = {"X": np.zeros(p["x"].shape[0]), "AX": np.full(p["x"].shape[0], 7.0, np.float32)}
    with pytest.raises(G.GalnbError) as e:
        d.get_fields(out)  # no forces yet
    assert e.value.code == G.GNB_ESTATE
    assert np.all(out["X"] == 0.0) and np.all(out["AX"] == 7.0)
    for x in (c, d):
        x.close()
