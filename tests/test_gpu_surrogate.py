"""GPU parity of the surrogate's particle <-> grid mappings (voxelise, Gibbs
remap) against the oracle, and invariants of the batched, graph-captured
surrogate step."""
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


def _region_state(G, orc, n=20000, seed=3):
    p = ics.sn_region(n, seed=seed, grid=32)
    c = G.Context()
    c.set_particles(p)
    c.compute_sph_density()
    return p, c


def test_voxelise_matches_oracle(G, orc):
    from oracle import surrogate as S
    p, c = _region_state(G, orc)
    grid = 32
    z = c.voxelise([(0.0, 0.0, 0.0)], side=60.0, grid=grid)[0].reshape(-1, 5)
    s = orc.state(p)
    rho = c.get("RHO").astype(np.float64)
    h = np.sqrt(c.get("H2"))
    mask = S.members(s, [(0.0, 0.0, 0.0)], 60.0) == 0
    ref = S.voxelise(s, rho, h, (0.0, 0.0, 0.0), 60.0, grid, region_mask=mask)
    assert np.max(np.abs(z[:, 0] - ref[:, 0])) < 2e-4
    assert np.max(np.abs(z[:, 1] - ref[:, 1])) < 2e-4
    assert np.max(np.abs(z[:, 2:] - ref[:, 2:])) < 1e-4 * max(1.0, np.max(np.abs(ref[:, 2:])))


# grid 64 and 32: the two-level (coarse block, then voxel) search over the
# line sums; grid 20: the binary search
@pytest.mark.parametrize("grid", [32, 64, 20])
def test_remap_matches_oracle(G, orc, grid):
    from oracle import surrogate as S
    p, c = _region_state(G, orc, n=15000, seed=4)
    side, cen = 60.0, (1.0, -2.0, 0.5)
    pred = c.voxelise([cen], side=side, grid=grid)
    s = orc.state(p)
    mem = np.nonzero(S.members(s, [cen], side) == 0)[0]
    c.remap_regions([cen], pred, side=side, seed=9, sweeps=4)
    x, y, z = c.get("X"), c.get("Y"), c.get("Z")
    newp = np.stack([x, y, z], axis=1)
    pos = np.stack([s["x"], s["y"], s["z"]], axis=1)[mem]
    vox, rp, ru, rv = S.remap(pred[0].reshape(-1, 5).astype(np.float64), p["id"][mem], pos, cen, side, grid,
                              seed=9, sweeps=4)
    lo = np.asarray(cen) - 0.5 * side
    gv = np.floor((newp[mem] - lo) / (side / grid)).astype(np.int64)
    assert np.array_equal(gv, vox)
    assert np.max(np.abs(newp[mem] - rp)) < 1e-12 * side
    others = np.setdiff1d(np.arange(p["x"].size), mem)
    assert np.array_equal(newp[others], pos_all(s)[others])
    assert np.allclose(c.get("U")[mem], ru, rtol=1e-6)
    v = np.stack([c.get("VX"), c.get("VY"), c.get("VZ")], axis=1)[mem]
    assert np.allclose(v, rv, rtol=1e-6, atol=1e-6)


def pos_all(s):
    return np.stack([s["x"], s["y"], s["z"]], axis=1)


def test_batched_surrogate_step_invariants(G, orc):
    from oracle import unet as U
    import torch
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        regions = [ics.sn_region(8000 + 3000 * k, seed=10 + k, grid=32) for k in range(4)]
        offs = [(200.0 * k, 0.0, 0.0) for k in range(4)]
        parts = {}
        for k, (r, o) in enumerate(zip(regions, offs)):
            r = dict(r)
            r["x"] = r["x"] + o[0]
            for key, val in r.items():
                parts.setdefault(key, []).append(val)
        p = {k: np.concatenate(v) for k, v in parts.items()}
        p["id"] = np.arange(p["x"].size, dtype=np.int64)
        c = G.Context(stream=stream.cuda_stream)
        c.set_particles(p)
        c.compute_sph_density()
        net = G.UNet(5, 5, 16, 4, 32, stream=stream.cuda_stream)
        spec = U.layer_spec(5, 5, 16, 4)
        prm = U.init_params(1, 5, 5, 16, 4)
        net.set_params(np.concatenate([np.concatenate([prm[n + ".w"].ravel(), prm[n + ".b"]])
                                       for n, *_ in spec]).astype(np.float32))
        c.sn_surrogate_batch(net, offs, side=60.0, seed=1, sweeps=8, use_graph=True)
        ids = c.get("ID")
        x, y, z = c.get("X"), c.get("Y"), c.get("Z")
        for k, o in enumerate(offs):
            lo = np.asarray(o) - 30.0
            sel = (np.abs(p["x"] - o[0]) <= 30) & (np.abs(p["y"]) <= 30) & (np.abs(p["z"]) <= 30)
            q = np.stack([x[sel], y[sel], z[sel]], axis=1)
            assert np.all((q >= lo) & (q <= lo + 60.0))       # members stay in their cube
        assert np.array_equal(ids, p["id"])                    # IDs and count conserved
        assert np.all(np.isfinite(c.get("U"))) and np.all(c.get("U") > 0)
        # replay: the same shapes reuse the captured graph
        c.compute_sph_density()
        c.sn_surrogate_batch(net, offs, side=60.0, seed=2, sweeps=8, use_graph=True)
        assert np.all(np.isfinite(c.get("X")))
    stream.synchronize()


def test_batched_surrogate_step_matches_oracle_remap(G, orc):
    """Eight Gibbs sweeps inside the graph-captured batch of four regions:
    every member of region r ends where the oracle's remap of r puts it, given
    the prediction the batch itself computed (read back from the network):
    voxel choices bit for bit, positions within 1e-12 of the side, u and v
    within 1e-6 relative; particles outside the regions do not move."""
    import torch
    from oracle import surrogate as S
    stream = torch.cuda.Stream()
    side, grid, seed = 60.0, 32, 21
    with torch.cuda.stream(stream):
        regions = [ics.sn_region(7000 + 2500 * k, seed=60 + k, grid=32) for k in range(4)]
        offs = [(150.0 * k, -30.0 * k, 10.0 * k) for k in range(4)]
        parts = {}
        for r, o in zip(regions, offs):
            r = dict(r)
            for a, key in enumerate(("x", "y", "z")):
                r[key] = r[key] + o[a]
            for key, val in r.items():
                parts.setdefault(key, []).append(val)
        p = {k: np.concatenate(v) for k, v in parts.items()}
        p["id"] = np.arange(p["x"].size, dtype=np.int64) * 5 + 17
        c = G.Context(stream=stream.cuda_stream)
        c.set_particles(p)
        c.compute_sph_density()
        net = _net32(G, stream)
        c.sn_surrogate_batch(net, offs, side=side, seed=seed, sweeps=8, use_graph=True)
        pred = net.get_output(len(offs))
        got = {k: c.get(k) for k in ("X", "Y", "Z", "U", "VX", "VY", "VZ", "ID")}
    stream.synchronize()
    s = orc.state(p)
    reg = S.members(s, offs, side)
    newp = np.stack([got["X"], got["Y"], got["Z"]], axis=1)
    pos0 = np.stack([s["x"], s["y"], s["z"]], axis=1)
    assert np.array_equal(got["ID"], p["id"])
    assert np.array_equal(newp[reg < 0], pos0[reg < 0])
    for r, cen in enumerate(offs):
        mem = np.nonzero(reg == r)[0]
        assert mem.size > 1000
        vox, rp, ru, rv = S.remap(pred[r].reshape(-1, 5).astype(np.float64), p["id"][mem], pos0[mem], cen, side,
                                  grid, seed=seed, sweeps=8)
        lo = np.asarray(cen) - 0.5 * side
        gv = np.floor((newp[mem] - lo) / (side / grid)).astype(np.int64)
        assert np.array_equal(gv, vox), r
        assert np.max(np.abs(newp[mem] - rp)) < 1e-12 * side
        assert np.allclose(got["U"][mem], ru, rtol=1e-6)
        v = np.stack([got["VX"], got["VY"], got["VZ"]], axis=1)[mem]
        assert np.allclose(v, rv, rtol=1e-6, atol=1e-6)


def test_pipelined_batch_matches_sequential(G, orc):
    """The batch pipelined over region chunks (voxelise / U-Net / remap of
    different chunks on three streams, one captured graph), with eight Gibbs
    sweeps.  Every member of region r ends where the oracle's remap of r puts
    it, given the prediction the pipelined batch itself computed (voxel
    choices bit for bit, positions within 1e-12 of the side, u and v within
    1e-6 relative): each chunk's remap read its own regions' prediction and
    line sums.  And that prediction equals the sequential batch's up to the
    network's BF16 rounding of its input: the voxel sums are FP32 reductions
    in no fixed order, so a few inputs may round to the other BF16
    neighbour, which moves a region's prediction by ~1e-3 (relative L2);
    a chunk that read another chunk's grid would move it by O(1).  (The
    difference between two sequential runs is no yardstick: they often
    agree bit for bit, and sometimes by the same ~1e-3.)"""
    import torch
    from oracle import surrogate as S
    stream = torch.cuda.Stream()
    side, grid, seed = 60.0, 32, 5
    with torch.cuda.stream(stream):
        regions = [ics.sn_region(6000 + 2000 * k, seed=30 + k, grid=32) for k in range(5)]
        offs = [(150.0 * k, 40.0 * k, 0.0) for k in range(5)]
        parts = {}
        for r, o in zip(regions, offs):
            r = dict(r)
            r["x"] = r["x"] + o[0]
            r["y"] = r["y"] + o[1]
            for key, val in r.items():
                parts.setdefault(key, []).append(val)
        p = {k: np.concatenate(v) for k, v in parts.items()}
        p["id"] = np.arange(p["x"].size, dtype=np.int64) * 3 + 1
        net = _net32(G, stream)
        preds, outs = [], []
        for chunks in (1, 3):
            c = G.Context(stream=stream.cuda_stream)
            c.set_particles(p)
            c.set_sn_chunks(chunks)
            c.compute_sph_density()
            c.sn_surrogate_batch(net, offs, side=side, seed=seed, sweeps=8, use_graph=True)
            preds.append(net.get_output(len(offs)))
            outs.append({k: c.get(k) for k in ("X", "Y", "Z", "U", "VX", "VY", "VZ", "ID")})
            c.close()
    stream.synchronize()
    pred_s, pred_p = preds
    got = outs[1]
    for r in range(len(offs)):
        d = np.linalg.norm(pred_p[r] - pred_s[r]) / np.linalg.norm(pred_s[r])
        assert d < 2e-2, (r, d)
    s = orc.state(p)
    reg = S.members(s, offs, side)
    newp = np.stack([got["X"], got["Y"], got["Z"]], axis=1)
    pos0 = np.stack([s["x"], s["y"], s["z"]], axis=1)
    assert np.array_equal(got["ID"], p["id"])
    assert np.array_equal(newp[reg < 0], pos0[reg < 0])
    for r, cen in enumerate(offs):
        mem = np.nonzero(reg == r)[0]
        assert mem.size > 1000
        vox, rp, ru, rv = S.remap(pred_p[r].reshape(-1, 5).astype(np.float64), p["id"][mem], pos0[mem], cen, side,
                                  grid, seed=seed, sweeps=8)
        lo = np.asarray(cen) - 0.5 * side
        gv = np.floor((newp[mem] - lo) / (side / grid)).astype(np.int64)
        assert np.array_equal(gv, vox), r
        assert np.max(np.abs(newp[mem] - rp)) < 1e-12 * side
        assert np.allclose(got["U"][mem], ru, rtol=1e-6)
        v = np.stack([got["VX"], got["VY"], got["VZ"]], axis=1)[mem]
        assert np.allclose(v, rv, rtol=1e-6, atol=1e-6)


def _net32(G, stream):
    from oracle import unet as U
    net = G.UNet(5, 5, 16, 4, 32, stream=stream.cuda_stream)
    spec = U.layer_spec(5, 5, 16, 4)
    prm = U.init_params(5, 5, 5, 16, 4)
    net.set_params(np.concatenate([np.concatenate([prm[n + ".w"].ravel(), prm[n + ".b"]])
                                   for n, *_ in spec]).astype(np.float32))
    return net


def test_async_batch_applied_at_once_matches_the_batch(G, orc):
    """Submitted and applied with no step between, the asynchronous batch
    places every member exactly where the synchronous batch does (no Gibbs
    sweeps: the voxel of the old position and the seeded offset)."""
    import torch
    stream = torch.cuda.Stream()
    p = ics.sn_region(12000, seed=41, grid=32)
    cen = [(0.5, -1.0, 2.0)]
    with torch.cuda.stream(stream):
        net = _net32(G, stream)
        out = []
        for mode in ("sync", "async"):
            c = G.Context(stream=stream.cuda_stream)
            c.set_particles(p)
            c.compute_sph_density()
            if mode == "sync":
                c.sn_surrogate_batch(net, cen, side=60.0, seed=3, sweeps=0, use_graph=False)
            else:
                c.sn_async_submit(net, cen, side=60.0, seed=3, sweeps=0)
                assert c.sn_async_pending()
                c.sn_async_apply()
                assert not c.sn_async_pending()
            out.append({k: c.get(k) for k in ("X", "Y", "Z", "U", "ID")})
            c.close()
    stream.synchronize()
    a, b = out
    for k in ("X", "Y", "Z", "ID"):
        assert np.array_equal(a[k], b[k])
    assert np.all(np.isfinite(b["U"])) and np.all(b["U"] > 0)


def test_async_batch_deferred_over_global_steps(G, orc):
    """Submit, three KDK steps (the particle arrays are re-sorted every step),
    apply: the members are replaced from their snapshot (starting voxel of the
    snapshot position, seeded draws -- the oracle's remap, bit for bit), the
    other particles are those of the same three steps without the batch."""
    from oracle import surrogate as S
    import torch
    stream = torch.cuda.Stream()
    p = ics.sn_region(12000, seed=43, grid=32)
    cen = (0.5, -1.0, 2.0)
    side, grid, seed = 60.0, 32, 11
    s0 = orc.state(p)
    mem = np.nonzero(S.members(s0, [cen], side) == 0)[0]
    assert mem.size > 1000
    with torch.cuda.stream(stream):
        net = _net32(G, stream)
        res = {}
        for mode in ("plain", "async"):
            c = G.Context(stream=stream.cuda_stream)
            c.set_particles(p)
            c.compute_sph_density()
            if mode == "async":
                c.sn_async_submit(net, [cen], side=side, seed=seed, sweeps=0)
                with pytest.raises(G.GalnbError):
                    c.sn_async_submit(net, [cen], side=side, seed=seed, sweeps=0)  # one pending batch
                with pytest.raises(G.GalnbError):
                    c.voxelise([cen], side=side, grid=grid)
            c.compute_forces(G.GNB_GRAV_NONE)
            c.step_kdk(1e-4, 3, G.GNB_GRAV_NONE)
            if mode == "async":
                c.sn_async_apply()
                with pytest.raises(G.GalnbError):
                    c.sn_async_apply()  # nothing pending
            res[mode] = np.stack([c.get("X"), c.get("Y"), c.get("Z")], axis=1)
            assert np.array_equal(c.get("ID"), p["id"])
            c.close()
    stream.synchronize()
    # (the symmetric SPH force sums reverse-neighbour lists filled in no fixed
    # order, so two runs of the same steps differ in the last bits)
    others = np.setdiff1d(np.arange(p["x"].size), mem)
    assert np.max(np.abs(res["async"][others] - res["plain"][others])) < 1e-9 * side
    pos0 = np.stack([s0["x"], s0["y"], s0["z"]], axis=1)[mem]
    pred = np.zeros((grid ** 3, 5))  # positions do not depend on the prediction without sweeps
    vox, rp, _, _ = S.remap(pred, p["id"][mem], pos0, cen, side, grid, seed=seed, sweeps=0)
    assert np.max(np.abs(res["async"][mem] - rp)) < 1e-12 * side
    assert not np.array_equal(res["async"][mem], res["plain"][mem])
