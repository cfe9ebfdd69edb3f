"""Pins of the oracle's tree path: Morton order against a recursive octant
partition, octree against a set-based construction, moments against
closed forms, and tree gravity against direct summation (theta -> 0 limit,
theta = 0.5 accuracy, multipole order)."""
import numpy as np
import pytest

from paper_2510_23330_gb300 import ics


def _recursive_octant_order(cells, idx, level=0):
    """Order of particles produced by recursive subdivision into octants
    (x high bit most significant, then y, then z), ties by input index."""
    if idx.size <= 1 or level == 21:
        return list(np.sort(idx))
    b = 20 - level
    out = []
    for o in range(8):
        bx, by, bz = (o >> 2) & 1, (o >> 1) & 1, o & 1
        sel = idx[(((cells[idx, 0] >> b) & 1) == bx) & (((cells[idx, 1] >> b) & 1) == by)
                  & (((cells[idx, 2] >> b) & 1) == bz)]
        if sel.size:
            out += _recursive_octant_order(cells, sel, level + 1)
    return out


def test_morton_golden_corners(orc):
    """Points at the box corners and half-way planes have keys fixed by the
    21-bit-per-axis interleave (x at bit 3b+2, y at 3b+1, z at 3b)."""
    x = np.array([0.0, 4.0, 2.0, 0.0, 0.0, 2.0 - 1e-12])
    y = np.array([0.0, 4.0, 0.0, 2.0, 0.0, 0.0])
    z = np.array([0.0, 4.0, 0.0, 0.0, 2.0, 0.0])
    p = {"x": x, "y": y, "z": z}
    key, cells, lo, L = orc.morton(p)
    assert L == 4.0 and np.all(lo == 0.0)
    assert key[0] == 0
    assert key[1] == (1 << 63) - 1          # clamped to 2^21 - 1 on every axis
    assert key[2] == 1 << 62
    assert key[3] == 1 << 61
    assert key[4] == 1 << 60
    assert key[5] == sum(1 << (3 * b + 2) for b in range(20))
    assert cells[5, 0] == (1 << 20) - 1


def test_root_box_power_of_two(orc):
    p = {"x": np.array([-1.0, 2.5]), "y": np.array([0.0, 0.0]), "z": np.array([0.0, 1.0])}
    lo, L = orc.root_box(p)
    assert L == 4.0 and lo[0] == -1.0
    p = {"x": np.array([0.0, 2.0]), "y": np.zeros(2), "z": np.zeros(2)}
    assert orc.root_box(p)[1] == 2.0
    p = {"x": np.zeros(3), "y": np.zeros(3), "z": np.zeros(3)}
    assert orc.root_box(p)[1] == 1.0


def test_morton_order_equals_recursive_octants(orc):
    p = ics.plummer(3000, seed=5)
    # duplicate some positions to exercise the index tie-break
    for k in ("x", "y", "z"):
        p[k][100:110] = p[k][0]
    key, cells, _, _ = orc.morton(p)
    order = orc.sort_order(key)
    ref = _recursive_octant_order(cells.astype(np.int64), np.arange(3000))
    assert np.array_equal(order, np.array(ref))


def _setbased_tree(skey, n_leaf):
    """Nodes as a set of (level, prefix, first, count), built level by level
    from distinct prefixes: a level-l cell exists iff its parent holds more
    than n_leaf particles."""
    nodes = {(0, 0): (0, skey.size)}
    out = [(0, 0, 0, skey.size)]
    frontier = [(0, 0)]
    for lev in range(1, 22):
        sh = 3 * (21 - lev)
        pre = (skey >> np.uint64(sh)).astype(np.uint64)
        parents = {p for p in frontier if nodes[p][1] > n_leaf}
        uniq, first, cnt = np.unique(pre, return_index=True, return_counts=True)
        nxt = []
        for u, f, c in zip(uniq, first, cnt):
            par = (lev - 1, int(u) >> 3)
            if par in parents:
                nodes[(lev, int(u))] = (int(f), int(c))
                out.append((lev, int(u), int(f), int(c)))
                nxt.append((lev, int(u)))
        frontier = nxt
        if not frontier:
            break
    return sorted(out)


@pytest.mark.parametrize("n_leaf", [1, 8, 16])
def test_octree_matches_setbased_construction(orc, n_leaf):
    p = ics.exp_disk(4000, seed=2)
    key, _, _, _ = orc.morton(p)
    sk = key[orc.sort_order(key)]
    t = orc.octree(sk, n_leaf)
    got = sorted(zip(t["level"].tolist(), [int(v) for v in t["prefix"]],
                     t["first"].tolist(), t["count"].tolist()))
    assert got == _setbased_tree(sk, n_leaf)
    # breadth-first: levels non-decreasing, prefixes increasing within a level
    lev = t["level"]
    assert np.all(np.diff(lev) >= 0)
    for l in np.unique(lev):
        pr = t["prefix"][lev == l]
        assert np.all(pr[1:] > pr[:-1])
    leaves = t["nchild"] == 0
    assert t["count"][leaves].sum() == 4000
    assert np.all((t["count"][leaves] <= n_leaf) | (lev[leaves] == 21))


def test_octree_coincident_particles_stop_at_level_21(orc):
    p = {"x": np.r_[np.zeros(40), 1.0], "y": np.zeros(41), "z": np.zeros(41)}
    key, _, _, _ = orc.morton(p)
    sk = key[orc.sort_order(key)]
    t = orc.octree(sk, 4)
    assert t["level"].max() == 21
    big = (t["nchild"] == 0) & (t["count"] > 4)
    assert np.all(t["level"][big] == 21) and t["count"][big].sum() == 40


def test_moments_closed_form(orc):
    """Two masses 1 and 3 at x = -3 and x = +1: COM at 0; traceless
    Q = sum m (3 d d - d^2 I) gives Qxx = 2*(1*9 + 3*1) = 24, Qyy = Qzz = -12."""
    tree = {"first": np.array([0], np.int64), "count": np.array([2], np.int64),
            "level": np.array([0], np.int32)}
    sp = {"x": np.array([-3.0, 1.0]), "y": np.zeros(2), "z": np.zeros(2),
          "m": np.array([1.0, 3.0]), "eps": np.array([0.1, 0.3])}
    mo = orc.moments(tree, sp)
    assert mo["M"][0] == 4.0
    assert np.allclose(mo["com"][0], 0.0, atol=1e-15)
    assert np.allclose(mo["Q"][0], [24.0, -12.0, -12.0, 0, 0, 0])
    assert np.isclose(mo["eps2"][0], (1 * 0.01 + 3 * 0.09) / 4)


def test_moments_parallel_axis_and_traceless(orc):
    """Parent quadrupole equals the sum of children's quadrupoles shifted by
    the parallel-axis theorem; every Q is traceless."""
    p = ics.plummer(2000, seed=9)
    key, _, _, _ = orc.morton(p)
    o = orc.sort_order(key)
    sp = {k: np.asarray(p[k], np.float64)[o] for k in ("x", "y", "z", "m", "eps")}
    t = orc.octree(key[o], 8)
    mo = orc.moments(t, sp)
    Q = mo["Q"]
    assert np.allclose(Q[:, 0] + Q[:, 1] + Q[:, 2], 0, atol=1e-12)
    for k in np.nonzero(t["nchild"] > 0)[0][:50]:
        ch = range(t["child"][k], t["child"][k] + t["nchild"][k])
        q = np.zeros(6)
        for c in ch:
            s = mo["com"][c] - mo["com"][k]
            m = mo["M"][c]
            ss = s @ s
            q += Q[c] + m * np.array([3 * s[0] ** 2 - ss, 3 * s[1] ** 2 - ss, 3 * s[2] ** 2 - ss,
                                      3 * s[0] * s[1], 3 * s[0] * s[2], 3 * s[1] * s[2]])
        assert np.allclose(q, Q[k], rtol=1e-9, atol=1e-12 * np.abs(Q[k]).max())


def test_groups_partition_particles(orc):
    p = ics.exp_disk(5000, seed=4)
    key, _, _, _ = orc.morton(p)
    t = orc.octree(np.sort(key), 16)
    for n_g in (16, 64, 300):
        g = orc.groups(t, n_g)
        f, c = t["first"][g], t["count"][g]
        assert np.array_equal(f[1:], f[:-1] + c[:-1]) and f[0] == 0 and f.sum() >= 0
        assert c.sum() == 5000
        assert np.all((c <= n_g) | (t["nchild"][g] == 0))


def _parents(t):
    par = np.full(t["level"].shape[0], -1, np.int64)
    for k in range(t["level"].shape[0]):
        if t["nchild"][k]:
            par[t["child"][k]:t["child"][k] + t["nchild"][k]] = k
    return par


def test_groups_are_the_highest_cells_within_n_g(orc):
    """Groups are the highest cells with count <= n_g (or leaves): every
    group's parent holds more than n_g particles, so no group could be
    merged one level up; the root is a group iff N <= n_g.  A walk that
    stopped one level too deep, or too high, fails this."""
    p = ics.exp_disk(5000, seed=4)
    key, _, _, _ = orc.morton(p)
    t = orc.octree(np.sort(key), 16)
    par = _parents(t)
    for n_g in (16, 64, 300, 4999, 5000, 6000):
        g = orc.groups(t, n_g)
        if n_g >= 5000:
            assert list(g) == [0]
            continue
        assert 0 not in set(g)
        assert np.all(t["count"][par[g]] > n_g)
        # every cell not inside a group has count > n_g and is not a leaf
        inside = np.zeros(t["level"].shape[0], bool)
        stack = list(g)
        while stack:
            k = stack.pop()
            inside[k] = True
            stack += list(range(t["child"][k], t["child"][k] + t["nchild"][k])) if t["nchild"][k] else []
        outside = ~inside
        assert np.all(t["count"][outside] > n_g) and np.all(t["nchild"][outside] > 0)


def _tree_err(orc, p, **kw):
    d = orc.direct_gravity(p)
    t = orc.tree_gravity(p, **kw)
    ad = np.sqrt(d["ax"] ** 2 + d["ay"] ** 2 + d["az"] ** 2)
    da = np.sqrt((t["ax"] - d["ax"]) ** 2 + (t["ay"] - d["ay"]) ** 2 + (t["az"] - d["az"]) ** 2)
    return da / ad, t, d


def test_tree_theta_to_zero_is_direct_sum(orc):
    p = ics.plummer(2000, seed=1)
    e, t, d = _tree_err(orc, p, theta=1e-9, n_leaf=8, n_g=32)
    assert t["n_pc"] == 0
    assert e.max() < 1e-12
    assert np.allclose(t["phi"], d["phi"], rtol=1e-12)


def test_tree_accuracy_theta_half(orc):
    p = ics.plummer(4096, seed=0)
    e, t, _ = _tree_err(orc, p, theta=0.5, n_leaf=16, n_g=64)
    assert np.percentile(e, 99) < 1e-2
    assert t["n_pc"] > 0
    e_mono, _, _ = _tree_err(orc, p, theta=0.5, n_leaf=16, n_g=64, quad=False)
    assert np.percentile(e, 99) < np.percentile(e_mono, 99)
    e_wide, _, _ = _tree_err(orc, p, theta=0.8, n_leaf=16, n_g=64)
    assert np.median(e_wide) > np.median(e)


def test_multipole_error_order(orc):
    """Far-field error of one cell: O((s/d)^2) for a monopole and O((s/d)^3)
    with the quadrupole, seen through the tree with a single distant target."""
    rng = np.random.default_rng(1)
    k = 64
    cl = rng.uniform(0.0, 1.0, (k, 3))
    slopes = {}
    for quad in (False, True):
        errs = []
        ds = [8.0, 16.0, 32.0, 64.0]
        for dist in ds:
            pos = np.vstack([cl, [[dist, 0.3, 0.7]]])
            p = {"x": pos[:, 0].copy(), "y": pos[:, 1].copy(), "z": pos[:, 2].copy(),
                 "m": np.r_[rng.uniform(0.5, 1.5, k), 1e-12], "eps": np.zeros(k + 1)}
            e, t, _ = _tree_err(orc, p, theta=0.9, n_leaf=64, n_g=1, quad=quad)
            errs.append(e[-1])
        slopes[quad] = np.polyfit(np.log(ds), np.log(errs), 1)[0]
    assert -2.4 < slopes[False] < -1.6
    assert -3.4 < slopes[True] < -2.6


def test_single_particle_cell_equals_pp(orc):
    """A cell holding one particle has Q = 0 and eps2 = eps_j^2, so its
    particle-cell term equals the particle-particle term of Eq. 1."""
    # one particle per level-1 octant of a root box of side 128, so every
    # accepted cell holds exactly one particle
    pos = np.array([[0.0, 0.0, 0.0], [100.0, 100.0, 100.0], [100.0, 0.0, 100.0]])
    p = {"x": pos[:, 0].copy(), "y": pos[:, 1].copy(), "z": pos[:, 2].copy(),
         "m": np.array([1.0, 2.0, 3.0]), "eps": np.array([0.1, 0.2, 0.3])}
    t = orc.tree_gravity(p, theta=0.5, n_leaf=1, n_g=1)
    d = orc.direct_gravity(p)
    assert t["n_pc"] > 0
    for k in ("ax", "ay", "az", "phi"):
        assert np.allclose(t[k], d[k], rtol=1e-13, atol=0)
