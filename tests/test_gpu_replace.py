"""GPU tests of gnb_replace_region (Sec. 3.2, step 4: the particles of a
supernova region come back from the surrogate and overwrite the particles
with the same IDs).  The region's members are replaced by the oracle's Gibbs
remap of them, handed back in a shuffled order with IDs unrelated to the
caller indices; the state read back must be the replacement bit for bit, and
every other particle must be untouched.  Rejected calls (unknown, repeated
or ambiguous IDs, too many particles, a non-finite position) must change
nothing."""
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


def _state(c):
    return {k: c.get(k) for k in ("X", "Y", "Z", "VX", "VY", "VZ", "U", "ID")}


def _region(n, seed, grid):
    p = ics.sn_region(n, seed=seed, grid=grid)
    rng = np.random.default_rng(seed + 100)
    p["id"] = (10 ** 12 + 3 * rng.permutation(n)).astype(np.int64)   # not the caller index
    return p, rng


@pytest.mark.parametrize("device", [False, True])
def test_replace_region_by_oracle_remap(G, orc, device):
    import torch
    from oracle import surrogate as S
    p, rng = _region(15000, 4, 32)
    c = G.Context()
    c.set_particles(p)
    c.compute_sph_density()          # the particles now sit in Morton order, not caller order
    side, cen, grid = 60.0, (1.0, -2.0, 0.5), 32
    pred = c.voxelise([cen], side=side, grid=grid)
    s = orc.state(p)
    mem = np.nonzero(S.members(s, [cen], side) == 0)[0]
    pos = np.stack([s["x"], s["y"], s["z"]], axis=1)[mem]
    _, rp, ru, rv = S.remap(pred[0].reshape(-1, 5).astype(np.float64), p["id"][mem], pos, cen, side, grid,
                            seed=9, sweeps=4)
    perm = rng.permutation(mem.size)
    rep = {"id": p["id"][mem][perm], "x": rp[perm, 0].copy(), "y": rp[perm, 1].copy(), "z": rp[perm, 2].copy(),
           "vx": rv[perm, 0].astype(np.float32), "vy": rv[perm, 1].astype(np.float32),
           "vz": rv[perm, 2].astype(np.float32), "u": ru[perm].astype(np.float32)}
    before = _state(c)
    if device:
        rep = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in rep.items()}
        torch.cuda.synchronize()
    c.replace_region(rep)
    after = _state(c)
    tgt = mem[perm]
    for k, key in (("X", 0), ("Y", 1), ("Z", 2)):
        assert np.array_equal(after[k][tgt], rp[perm, key])
    for k, key in (("VX", 0), ("VY", 1), ("VZ", 2)):
        assert np.array_equal(after[k][tgt], rv[perm, key].astype(np.float32))
    assert np.array_equal(after["U"][tgt], ru[perm].astype(np.float32))
    others = np.setdiff1d(np.arange(p["x"].size), mem)
    for k in after:
        assert np.array_equal(after[k][others], before[k][others]), k
    assert np.array_equal(after["ID"], p["id"])
    # the context goes on from the new state
    c.compute_sph_density()
    assert np.all(np.isfinite(c.get("RHO")))


def test_replace_region_rejections_change_nothing(G):
    p, rng = _region(3000, 5, 16)
    p["id"][7] = p["id"][8]              # one ID held by two particles
    c = G.Context()
    c.set_particles(p)
    c.compute_sph_density()
    before = _state(c)
    sel = np.array([1, 2, 3, 4, 5, 100, 2000])
    base = {"id": p["id"][sel].copy(), "x": p["x"][sel] + 0.1, "y": p["y"][sel], "z": p["z"][sel],
            "vx": p["vx"][sel], "vy": p["vy"][sel], "vz": p["vz"][sel], "u": p["u"][sel] * 2}
    cases = []
    bad = dict(base, id=base["id"].copy())
    bad["id"][3] = -12345                # not held
    cases.append((bad, G.GNB_EMISMATCH))
    bad = dict(base, id=base["id"].copy())
    bad["id"][3] = base["id"][5]         # repeated in the input
    cases.append((bad, G.GNB_EMISMATCH))
    bad = dict(base, id=base["id"].copy())
    bad["id"][0] = p["id"][7]            # ambiguous: held twice
    cases.append((bad, G.GNB_EMISMATCH))
    big = {k: np.concatenate([p[k], p[k][:1]]) for k in base}
    cases.append((big, G.GNB_EMISMATCH))  # more particles than held
    bad = dict(base, x=base["x"].copy())
    bad["x"][2] = np.nan
    cases.append((bad, G.GNB_EINVAL))
    for q, code in cases:
        with pytest.raises(G.GalnbError) as e:
            c.replace_region(q)
        assert e.value.code == code
        after = _state(c)
        for k in after:
            assert np.array_equal(after[k], before[k]), k
    # the density of the untouched state is still current and readable
    assert np.all(np.isfinite(c.get("RHO")))
    c.replace_region(base)               # a valid call still works afterwards
    x = c.get("X")
    assert np.array_equal(x[sel], base["x"])
