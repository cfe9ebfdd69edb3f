"""The allocation-free entry point gnb_morton_order_noalloc, for callers that
cannot allocate device memory (their memory is owned by another allocator,
or cudaMalloc/cudaFree would stall a latency-sensitive loop).  Its keys and
order must equal those of the context path (gnb_set_particles +
gnb_build_tree + gnb_get), bit for bit, on two calls in a row that reuse its
static scratch array, and for particles that all sit at one point (zero
extent, root side 1); a call must leave the device's free memory and
PyTorch's allocation count unchanged; sizes beyond its maximum are
rejected.

This file is collected last so that a run stopping at the first failure
has already run every other test."""
import numpy as np
import pytest

from paper_2510_23330_gb300 import ics

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_23330_gb300 import galnb
    return torch, galnb


def _noalloc(torch, galnb, p):
    n = p["x"].shape[0]
    dev = {k: torch.from_numpy(np.ascontiguousarray(p[k])).cuda() for k in ("x", "y", "z")}
    keys = torch.empty(n, dtype=torch.int64, device="cuda")
    order = torch.empty(n, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    rc = galnb.gnb_morton_order_noalloc(n, dev["x"].data_ptr(), dev["y"].data_ptr(), dev["z"].data_ptr(),
                                        keys.data_ptr(), order.data_ptr(), stream.cuda_stream)
    torch.cuda.synchronize()
    return rc, keys.cpu().numpy().view(np.uint64), order.cpu().numpy()


def _context_path(galnb, p):
    c = galnb.Context()
    c.set_particles(p)
    c.build_tree()
    k, o = c.get("KEY"), c.get("ORDER")
    c.close()
    return k, o


def test_noalloc_matches_context_path_two_calls(env):
    torch, galnb = env
    inputs = [ics.config_disk(200000, seed=3),
              ics.plummer(galnb.GNB_NOALLOC_MAX_N, seed=4, n_gas=0)]
    for p in inputs:  # two calls in a row on the same scratch array
        rc, keys, order = _noalloc(torch, galnb, p)
        assert rc == galnb.GNB_OK
        kref, oref = _context_path(galnb, p)
        assert np.array_equal(keys, kref)
        assert np.array_equal(order, oref)


def test_noalloc_rejects_sizes_beyond_maximum(env):
    torch, galnb = env
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    out = torch.zeros(16, dtype=torch.int64, device="cuda")
    for n in (0, galnb.GNB_NOALLOC_MAX_N + 1):
        rc = galnb.gnb_morton_order_noalloc(n, buf.data_ptr(), buf.data_ptr(), buf.data_ptr(), out.data_ptr(),
                                            out.data_ptr(), None)
        assert rc == galnb.GNB_EINVAL


def test_noalloc_all_particles_at_one_point(env):
    """Zero extent: the root side is 1, every key is 0 and the order is the
    caller order (ties by caller index)."""
    torch, galnb = env
    n = 5000
    p = ics.plummer(n, seed=5, n_gas=0)
    for k in ("x", "y", "z"):
        p[k] = np.full(n, 0.375)
    rc, keys, order = _noalloc(torch, galnb, p)
    assert rc == galnb.GNB_OK
    assert np.all(keys == 0) and np.array_equal(order, np.arange(n))
    kref, oref = _context_path(galnb, p)
    assert np.array_equal(keys, kref) and np.array_equal(order, oref)


def test_noalloc_call_allocates_nothing(env):
    """Around one call (after a first call, which loads this entry point's
    device code and with it the static array), the device's free memory must
    not drop by an allocation (cudaMalloc hands out at least 2 MiB pages;
    the buffers of this size would be 2 MiB each) and PyTorch's allocator
    must see no new allocation."""
    torch, galnb = env
    n = galnb.GNB_NOALLOC_MAX_N
    p = ics.plummer(n, seed=6, n_gas=0)
    dev = {k: torch.from_numpy(np.ascontiguousarray(p[k])).cuda() for k in ("x", "y", "z")}
    keys = torch.empty(n, dtype=torch.int64, device="cuda")
    order = torch.empty(n, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream

    def call():
        return galnb.gnb_morton_order_noalloc(n, dev["x"].data_ptr(), dev["y"].data_ptr(), dev["z"].data_ptr(),
                                              keys.data_ptr(), order.data_ptr(), stream)

    assert call() == galnb.GNB_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    allocs0 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    assert call() == galnb.GNB_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    allocs1 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    assert free0 - free1 < (2 << 20), (free0, free1)
    assert allocs1 == allocs0
