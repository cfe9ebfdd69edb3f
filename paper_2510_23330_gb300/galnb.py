"""Thin ctypes binding of the C ABI in ``include/galnb.h``.

Every ``gnb_*`` function here has the C function's name and arguments and only
marshals them; all work runs in ``libgalnb.so``.  There is no fallback: if the
library cannot be built or loaded, ``lib()`` raises.  ``Context`` is a small
convenience wrapper that turns numpy or torch arrays into the pointers the C
calls take and raises ``GalnbError`` on a non-zero return code.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

GNB_OK = 0
GNB_EINVAL = -1
GNB_ENOMEM = -2
GNB_ECUDA = -3
GNB_ESTATE = -4
GNB_ECAPACITY = -5
GNB_ETIMEOUT = -6
GNB_EMISMATCH = -7

GNB_STAR = 0
GNB_GAS = 1
GNB_GRAV_DIRECT = 0
GNB_GRAV_TREE = 1
GNB_GRAV_NONE = 2
GNB_CONV_AUTO = 0
GNB_CONV_MMA_SYNC = 2

FIELDS = ["X", "Y", "Z", "VX", "VY", "VZ", "AX", "AY", "AZ", "POT", "U", "DUDT", "RHO", "PRES", "CS", "H2",
          "KEY", "ORDER", "NBR", "NODES", "GROUPS", "ID", "AGRAV_X", "AGRAV_Y", "AGRAV_Z", "LEVEL",
          "POT_EXT", "NODE_LINKS"]
F = {name: i for i, name in enumerate(FIELDS)}
FIELD_DTYPE = {"X": np.float64, "Y": np.float64, "Z": np.float64, "H2": np.float64, "KEY": np.uint64,
               "ORDER": np.int64, "NBR": np.int64, "NODES": np.int64, "NODE_LINKS": np.int64, "GROUPS": np.int64, "ID": np.int64,
               "LEVEL": np.int32}
STATS = ["N", "NGAS", "NODES", "GROUPS", "NPP", "NPC", "GAS_NODES", "KNN_PASSES", "NSYM", "MAXLEVEL"]


class gnb_config(C.Structure):
    _fields_ = [("G", C.c_double), ("theta", C.c_double), ("gamma", C.c_double), ("alpha_visc", C.c_double),
                ("n_leaf", C.c_int), ("n_group", C.c_int), ("n_ngb", C.c_int), ("multipole", C.c_int),
                ("nfw_ms", C.c_double), ("nfw_rs", C.c_double), ("cuda_stream", C.c_void_p),
                ("sph_variant", C.c_int)]


_lock = threading.Lock()
_lib = None
_vp = C.c_void_p


def lib():
    """Load libgalnb.so, building it first if the sources changed."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = C.CDLL(path)
            _declare(L)
            _lib = L
    return _lib


def library_path() -> str:
    return _build.LIB


def _declare(L):
    L.gnb_config_default.argtypes = [C.POINTER(gnb_config)]
    L.gnb_config_default.restype = None
    L.gnb_create.argtypes = [C.POINTER(_vp), C.POINTER(gnb_config)]
    L.gnb_destroy.argtypes = [_vp]
    L.gnb_destroy.restype = None
    L.gnb_set_particles.argtypes = [_vp, C.c_int64] + [_vp] * 11 + [C.c_int]
    L.gnb_set_state.argtypes = [_vp, C.c_int64] + [_vp] * 16 + [C.c_int, C.c_int]
    L.gnb_get_fields.argtypes = [_vp, C.c_int, _vp, _vp, _vp, C.c_int]
    L.gnb_build_tree.argtypes = [_vp]
    L.gnb_compute_gravity.argtypes = [_vp, C.c_int]
    L.gnb_compute_sph_density.argtypes = [_vp]
    L.gnb_compute_sph_force.argtypes = [_vp]
    L.gnb_compute_forces.argtypes = [_vp, C.c_int]
    L.gnb_step_kdk.argtypes = [_vp, C.c_double, C.c_int, C.c_int]
    L.gnb_get.argtypes = [_vp, C.c_int, _vp, C.c_int64, C.c_int]
    L.gnb_diagnostics.argtypes = [_vp, C.POINTER(C.c_double)]
    L.gnb_stats.argtypes = [_vp, C.POINTER(C.c_int64)]
    L.gnb_last_error.argtypes = [_vp]
    L.gnb_last_error.restype = C.c_char_p
    L.gnb_set_timing.argtypes = [_vp, C.c_int]
    L.gnb_set_timing.restype = C.c_int
    L.gnb_set_sn_chunks.argtypes = [_vp, C.c_int]
    L.gnb_set_sn_chunks.restype = C.c_int
    L.gnb_sn_async_submit.argtypes = [_vp, _vp, C.c_int, _vp, C.c_double, C.c_uint64, C.c_int]
    L.gnb_sn_async_submit.restype = C.c_int
    L.gnb_sn_async_apply.argtypes = [_vp]
    L.gnb_sn_async_apply.restype = C.c_int
    L.gnb_sn_async_pending.argtypes = [_vp]
    L.gnb_sn_async_pending.restype = C.c_int
    L.gnb_phase_times.argtypes = [_vp, C.POINTER(C.c_double), C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                  C.c_int]
    L.gnb_phase_times.restype = C.c_int
    L.gnb_replace_region.argtypes = [_vp, C.c_int64] + [_vp] * 8 + [C.c_int]
    L.gnb_replace_region.restype = C.c_int
    L.gnb_morton_order_noalloc.argtypes = [C.c_int64, _vp, _vp, _vp, _vp, _vp, _vp]
    L.gnb_morton_order_noalloc.restype = C.c_int
    L.gnb_set_config.argtypes = [_vp, C.POINTER(gnb_config)]
    L.gnb_set_config.restype = C.c_int
    L.gnb_inject_energy.argtypes = [_vp, C.POINTER(C.c_double), C.c_double, C.POINTER(C.c_double)]
    L.gnb_inject_energy.restype = C.c_int
    L.gnb_cfl_timestep.argtypes = [_vp, C.c_double, C.POINTER(C.c_double)]
    L.gnb_cfl_timestep.restype = C.c_int
    L.gnb_integrate_cfl.argtypes = [_vp, C.c_double, C.c_double, C.c_int, C.c_int, C.POINTER(C.c_double),
                                    C.POINTER(C.c_int64)]
    L.gnb_integrate_cfl.restype = C.c_int
    L.gnb_integrate_hier.argtypes = [_vp, C.c_double, C.c_double, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double),
                                     C.POINTER(C.c_int64)]
    L.gnb_integrate_hier.restype = C.c_int
    L.gnb_voxelise.argtypes = [_vp, C.c_int, C.POINTER(C.c_double), C.c_double, C.c_int, _vp, C.c_int]
    L.gnb_voxelise.restype = C.c_int
    L.gnb_remap_regions.argtypes = [_vp, C.c_int, C.POINTER(C.c_double), C.c_double, C.c_int, _vp, C.c_uint64,
                                    C.c_int, C.c_int]
    L.gnb_remap_regions.restype = C.c_int
    L.gnb_sn_surrogate_batch.argtypes = [_vp, _vp, C.c_int, C.POINTER(C.c_double), C.c_double, C.c_uint64, C.c_int,
                                         C.c_int]
    L.gnb_sn_surrogate_batch.restype = C.c_int
    L.gnb_unet_create.argtypes = [C.POINTER(_vp), C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, _vp]
    L.gnb_unet_create.restype = C.c_int
    L.gnb_unet_destroy.argtypes = [_vp]
    L.gnb_unet_destroy.restype = None
    L.gnb_unet_num_params.argtypes = [_vp]
    L.gnb_unet_num_params.restype = C.c_int64
    for name in ("gnb_unet_get_params", "gnb_unet_set_params", "gnb_unet_get_grads"):
        getattr(L, name).argtypes = [_vp, _vp, C.c_int]
        getattr(L, name).restype = C.c_int
    L.gnb_unet_get_output.argtypes = [_vp, C.c_int, _vp, C.c_int]
    L.gnb_unet_get_output.restype = C.c_int
    L.gnb_unet_get_activation.argtypes = [_vp, C.c_int, C.c_int, _vp, C.c_int]
    L.gnb_unet_get_activation.restype = C.c_int
    L.gnb_unet_autotune.argtypes = [_vp, C.c_int, C.POINTER(C.c_double)]
    L.gnb_unet_autotune.restype = C.c_int
    L.gnb_unet_set_conv_impl.argtypes = [_vp, C.c_int]
    L.gnb_unet_set_conv_impl.restype = C.c_int
    L.gnb_unet_test_wait_timeout.argtypes = [_vp]
    L.gnb_unet_test_wait_timeout.restype = C.c_int
    for name in ("gnb_save", "gnb_load", "gnb_unet_save", "gnb_unet_load"):
        getattr(L, name).argtypes = [_vp, C.c_char_p]
        getattr(L, name).restype = C.c_int
    L.gnb_unet_forward.argtypes = [_vp, C.c_int, _vp, _vp, C.c_int]
    L.gnb_unet_forward.restype = C.c_int
    L.gnb_unet_train_step.argtypes = [_vp, C.c_int, _vp, _vp, C.c_double, C.POINTER(C.c_double), C.c_int]
    L.gnb_unet_train_step.restype = C.c_int
    for name in ("gnb_create", "gnb_set_particles", "gnb_set_state", "gnb_get_fields", "gnb_build_tree",
                 "gnb_compute_gravity",
                 "gnb_compute_sph_density", "gnb_compute_sph_force", "gnb_compute_forces", "gnb_step_kdk",
                 "gnb_get", "gnb_diagnostics", "gnb_stats"):
        getattr(L, name).restype = C.c_int


# -------------------------------------------------------------- same-name calls
def gnb_config_default(cfg):
    lib().gnb_config_default(C.byref(cfg))


def gnb_create(out, cfg):
    return lib().gnb_create(out, C.byref(cfg))


def gnb_destroy(ctx):
    lib().gnb_destroy(ctx)


def gnb_set_config(ctx, cfg):
    return lib().gnb_set_config(ctx, C.byref(cfg))


def gnb_set_particles(ctx, n, id, type, x, y, z, vx, vy, vz, m, eps, u, on_device):
    return lib().gnb_set_particles(ctx, n, id, type, x, y, z, vx, vy, vz, m, eps, u, on_device)


def gnb_get_fields(ctx, nf, fields, dst, cap, on_device):
    return lib().gnb_get_fields(ctx, nf, fields, dst, cap, on_device)


def gnb_set_state(ctx, n, id, type, x, y, z, vx, vy, vz, m, eps, u, h2, ax, ay, az, dudt, grav_mode, on_device):
    return lib().gnb_set_state(ctx, n, id, type, x, y, z, vx, vy, vz, m, eps, u, h2, ax, ay, az, dudt, grav_mode,
                               on_device)


def gnb_build_tree(ctx):
    return lib().gnb_build_tree(ctx)


def gnb_compute_gravity(ctx, mode):
    return lib().gnb_compute_gravity(ctx, mode)


def gnb_compute_sph_density(ctx):
    return lib().gnb_compute_sph_density(ctx)


def gnb_compute_sph_force(ctx):
    return lib().gnb_compute_sph_force(ctx)


def gnb_compute_forces(ctx, mode):
    return lib().gnb_compute_forces(ctx, mode)


def gnb_step_kdk(ctx, dt, nsteps, mode):
    return lib().gnb_step_kdk(ctx, dt, nsteps, mode)


def gnb_replace_region(ctx, n, id, x, y, z, vx, vy, vz, u, on_device):
    return lib().gnb_replace_region(ctx, n, id, x, y, z, vx, vy, vz, u, on_device)


def gnb_get(ctx, field, dst, cap, on_device):
    return lib().gnb_get(ctx, field, dst, cap, on_device)


def gnb_diagnostics(ctx, out):
    return lib().gnb_diagnostics(ctx, out)


def gnb_stats(ctx, out):
    return lib().gnb_stats(ctx, out)


def gnb_last_error(ctx):
    r = lib().gnb_last_error(ctx)
    return r.decode() if r else ""


def gnb_inject_energy(ctx, pos, energy, info):
    return lib().gnb_inject_energy(ctx, pos, energy, info)


def gnb_cfl_timestep(ctx, courant, dt):
    return lib().gnb_cfl_timestep(ctx, courant, dt)


def gnb_integrate_cfl(ctx, t_span, courant, max_steps, gravity_mode, t_done, steps_done):
    return lib().gnb_integrate_cfl(ctx, t_span, courant, max_steps, gravity_mode, t_done, steps_done)


def gnb_integrate_hier(ctx, t_span, courant, max_level, max_steps, gravity_mode, t_done, info):
    return lib().gnb_integrate_hier(ctx, t_span, courant, max_level, max_steps, gravity_mode, t_done, info)


def gnb_voxelise(ctx, nreg, centers, side, grid, out, on_device):
    return lib().gnb_voxelise(ctx, nreg, centers, side, grid, out, on_device)


def gnb_remap_regions(ctx, nreg, centers, side, grid, pred, seed, sweeps, on_device):
    return lib().gnb_remap_regions(ctx, nreg, centers, side, grid, pred, seed, sweeps, on_device)


def gnb_sn_surrogate_batch(ctx, net, nreg, centers, side, seed, sweeps, use_graph):
    return lib().gnb_sn_surrogate_batch(ctx, net, nreg, centers, side, seed, sweeps, use_graph)


def _centers(centers):
    c = np.ascontiguousarray(np.asarray(centers, np.float64).reshape(-1))
    return c, (C.c_double * c.size)(*c)


def gnb_unet_create(out, cin, cout, base, levels, grid, stream):
    return lib().gnb_unet_create(out, cin, cout, base, levels, grid, stream)


def gnb_unet_destroy(net):
    lib().gnb_unet_destroy(net)


def gnb_unet_num_params(net):
    return lib().gnb_unet_num_params(net)


def gnb_unet_set_conv_impl(net, impl):
    return lib().gnb_unet_set_conv_impl(net, impl)


def gnb_unet_test_wait_timeout(net):
    return lib().gnb_unet_test_wait_timeout(net)


def gnb_unet_get_params(net, dst, on_device):
    return lib().gnb_unet_get_params(net, dst, on_device)


def gnb_unet_set_params(net, src, on_device):
    return lib().gnb_unet_set_params(net, src, on_device)


def gnb_unet_save(net, path):
    return lib().gnb_unet_save(net, os.fsencode(path))


def gnb_unet_load(net, path):
    return lib().gnb_unet_load(net, os.fsencode(path))


def gnb_save(ctx, path):
    return lib().gnb_save(ctx, os.fsencode(path))


def gnb_load(ctx, path):
    return lib().gnb_load(ctx, os.fsencode(path))


def gnb_unet_get_grads(net, dst, on_device):
    return lib().gnb_unet_get_grads(net, dst, on_device)


def gnb_unet_get_output(net, batch, dst, on_device):
    return lib().gnb_unet_get_output(net, batch, dst, on_device)


def gnb_unet_autotune(net, batch, out_ms):
    return lib().gnb_unet_autotune(net, batch, out_ms)


def gnb_unet_get_activation(net, slot, batch, dst, on_device):
    return lib().gnb_unet_get_activation(net, slot, batch, dst, on_device)


def gnb_unet_forward(net, batch, x, y, on_device):
    return lib().gnb_unet_forward(net, batch, x, y, on_device)


def gnb_unet_train_step(net, batch, x, target, lr, loss, on_device):
    return lib().gnb_unet_train_step(net, batch, x, target, lr, loss, on_device)


class UNet:
    """Owner of one gnb_unet (marshalling only)."""

    def __init__(self, cin=5, cout=5, base=16, levels=4, grid=64, stream=None):
        h = _vp()
        rc = gnb_unet_create(C.byref(h), cin, cout, base, levels, grid, stream)
        if rc != GNB_OK:
            raise GalnbError(rc, "gnb_unet_create failed")
        self.h, self.cin, self.cout, self.grid = h, cin, cout, grid

    def close(self):
        if getattr(self, "h", None):
            gnb_unet_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _chk(rc, what):
        if rc != GNB_OK:
            raise GalnbError(rc, what)

    def set_conv_impl(self, impl):
        """GNB_CONV_AUTO (tcgen05 where supported) or GNB_CONV_MMA_SYNC."""
        self._chk(gnb_unet_set_conv_impl(self.h, impl), "set_conv_impl")

    def num_params(self):
        return int(gnb_unet_num_params(self.h))

    def get_params(self):
        out = np.empty(self.num_params(), np.float32)
        self._chk(gnb_unet_get_params(self.h, out.ctypes.data, 0), "get_params")
        return out

    def get_grads(self):
        out = np.empty(self.num_params(), np.float32)
        self._chk(gnb_unet_get_grads(self.h, out.ctypes.data, 0), "get_grads")
        return out

    def get_output(self, batch):
        """FP32 output [batch, G, G, G, cout] of the last forward pass."""
        g = self.grid
        out = np.empty((batch, g, g, g, self.cout), np.float32)
        self._chk(gnb_unet_get_output(self.h, batch, out.ctypes.data, 0), "get_output")
        return out

    def autotune(self, batch):
        """Pick each 3^3 layer's tensor-core tile plan by timing; returns the
        forward pass's milliseconds (before, after)."""
        out = (C.c_double * 2)()
        self._chk(gnb_unet_autotune(self.h, batch, out), "autotune")
        return out[0], out[1]

    def get_activation(self, slot, batch, grid, channels):
        """Stored tensor `slot` of the last forward pass as FP32
        [batch, grid, grid, grid, channels] (see gnb_unet_get_activation)."""
        out = np.empty((batch, grid, grid, grid, channels), np.float32)
        self._chk(gnb_unet_get_activation(self.h, slot, batch, out.ctypes.data, 0), "get_activation")
        return out

    def set_params(self, flat):
        flat = np.ascontiguousarray(flat, dtype=np.float32)
        assert flat.size == self.num_params()
        self._chk(gnb_unet_set_params(self.h, flat.ctypes.data, 0), "set_params")

    def save(self, path):
        """Parameters and Adam state to a checkpoint file (gnb_unet_save)."""
        self._chk(gnb_unet_save(self.h, path), "save")

    def load(self, path):
        """Parameters and Adam state from a checkpoint of a same-shape network."""
        self._chk(gnb_unet_load(self.h, path), "load")

    def forward(self, x, out=None):
        """x: [B, G, G, G, cin] (numpy float32 or a CUDA tensor)."""
        if isinstance(x, np.ndarray):
            x = np.ascontiguousarray(x, dtype=np.float32)
            y = np.empty(x.shape[:4] + (self.cout,), np.float32) if out is None else out
            self._chk(gnb_unet_forward(self.h, x.shape[0], x.ctypes.data, y.ctypes.data, 0), "forward")
            return y
        y = out
        self._chk(gnb_unet_forward(self.h, x.shape[0], x.data_ptr(), y.data_ptr(), 1), "forward")
        return y

    def train_step(self, x, target, lr):
        loss = C.c_double(0.0)
        if isinstance(x, np.ndarray):
            x = np.ascontiguousarray(x, dtype=np.float32)
            target = np.ascontiguousarray(target, dtype=np.float32)
            self._chk(gnb_unet_train_step(self.h, x.shape[0], x.ctypes.data, target.ctypes.data, float(lr),
                                          C.byref(loss), 0), "train_step")
        else:
            self._chk(gnb_unet_train_step(self.h, x.shape[0], x.data_ptr(), target.data_ptr(), float(lr),
                                          C.byref(loss), 1), "train_step")
        return loss.value


def gnb_set_timing(ctx, enable):
    return lib().gnb_set_timing(ctx, enable)


def gnb_set_sn_chunks(ctx, chunks):
    return lib().gnb_set_sn_chunks(ctx, chunks)


def gnb_sn_async_submit(ctx, net, nreg, centers, side, seed, sweeps):
    return lib().gnb_sn_async_submit(ctx, net, nreg, centers, side, seed, sweeps)


def gnb_sn_async_apply(ctx):
    return lib().gnb_sn_async_apply(ctx)


def gnb_sn_async_pending(ctx):
    return lib().gnb_sn_async_pending(ctx)


def gnb_phase_times(ctx, out_ms, calls, launches, reset):
    return lib().gnb_phase_times(ctx, out_ms, calls, launches, reset)


PHASES = ["SORT", "TREE", "GRAVITY", "EXTERNAL", "HYDRO_TREE", "KNN", "FORCE", "KDK", "VOXELISE", "UNET", "REMAP"]

GNB_NOALLOC_MAX_N = 262144


def gnb_morton_order_noalloc(n, x, y, z, keys, order, stream):
    """Keys and curve order of device positions with no device allocation
    (for callers that cannot allocate); all pointers are device pointers."""
    return lib().gnb_morton_order_noalloc(n, x, y, z, keys, order, stream)


# -------------------------------------------------------------- convenience wrapper
class GalnbError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"galnb error {code}: {msg}")
        self.code = code


def _ptr(a):
    """(pointer, on_device) of a numpy array or torch tensor."""
    if isinstance(a, np.ndarray):
        assert a.flags.c_contiguous
        return a.ctypes.data, 0
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous()
        return a.data_ptr(), 1 if a.is_cuda else 0
    raise TypeError(type(a))


class Context:
    """Owner of one gnb_ctx.  ``stream`` is a cudaStream_t as an int (e.g.
    ``torch.cuda.current_stream().cuda_stream``) or None."""

    _DT = {"id": np.int64, "type": np.uint8, "x": np.float64, "y": np.float64, "z": np.float64,
           "vx": np.float32, "vy": np.float32, "vz": np.float32, "m": np.float32, "eps": np.float32,
           "u": np.float32}

    def __init__(self, stream=None, **params):
        cfg = gnb_config()
        gnb_config_default(cfg)
        for k, v in params.items():
            if not hasattr(cfg, k):
                raise KeyError(k)
            setattr(cfg, k, v)
        cfg.cuda_stream = stream
        self.cfg = cfg
        h = _vp()
        rc = gnb_create(C.byref(h), cfg)
        if rc != GNB_OK:
            raise GalnbError(rc, "gnb_create failed")
        self.h = h
        self.n = 0
        self.n_gas = 0

    def close(self):
        if getattr(self, "h", None):
            gnb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, rc):
        if rc != GNB_OK:
            raise GalnbError(rc, gnb_last_error(self.h))

    def set_particles(self, p: dict):
        keys = ("id", "type", "x", "y", "z", "vx", "vy", "vz", "m", "eps", "u")
        arrs = []
        for k in keys:
            a = p[k]
            if isinstance(a, np.ndarray):
                a = np.ascontiguousarray(a, dtype=self._DT[k])
            arrs.append(a)
        ptrs = [_ptr(a) for a in arrs]
        on_dev = {d for _, d in ptrs}
        if len(on_dev) != 1:
            raise ValueError("all arrays must be on the same side (host or device)")
        n = int(arrs[2].shape[0])
        self._keep = arrs
        self._chk(gnb_set_particles(self.h, n, *[q for q, _ in ptrs], on_dev.pop()))
        self.n = n
        self.n_gas = int(self.stats()["NGAS"])

    def set_state(self, p: dict, mode=GNB_GRAV_TREE):
        """Particles with the accelerations and du/dt of their state (keys
        "ax", "ay", "az", "dudt", optionally "h2"), so that step_kdk with the
        same mode continues without evaluating the forces first."""
        keys = ("id", "type", "x", "y", "z", "vx", "vy", "vz", "m", "eps", "u", "h2", "ax", "ay", "az", "dudt")
        dt = dict(self._DT, h2=np.float64, ax=np.float32, ay=np.float32, az=np.float32, dudt=np.float32)
        arrs = []
        for k in keys:
            a = p.get(k) if k == "h2" else p[k]
            if isinstance(a, np.ndarray):
                a = np.ascontiguousarray(a, dtype=dt[k])
            arrs.append(a)
        ptrs = [_ptr(a) if a is not None else (None, None) for a in arrs]
        on_dev = {d for _, d in ptrs if d is not None}
        if len(on_dev) != 1:
            raise ValueError("all arrays must be on the same side (host or device)")
        n = int(arrs[2].shape[0])
        self._keep = arrs
        self._chk(gnb_set_state(self.h, n, *[q for q, _ in ptrs], mode, on_dev.pop()))
        self.n = n
        self.n_gas = int(self.stats()["NGAS"])

    def build_tree(self):
        self._chk(gnb_build_tree(self.h))

    def compute_gravity(self, mode=GNB_GRAV_TREE):
        self._chk(gnb_compute_gravity(self.h, mode))

    def compute_sph_density(self):
        self._chk(gnb_compute_sph_density(self.h))

    def compute_sph_force(self):
        self._chk(gnb_compute_sph_force(self.h))

    def compute_forces(self, mode=GNB_GRAV_TREE):
        self._chk(gnb_compute_forces(self.h, mode))

    def step_kdk(self, dt, nsteps=1, mode=GNB_GRAV_TREE):
        self._chk(gnb_step_kdk(self.h, float(dt), int(nsteps), mode))

    def count(self, field):
        st = self.stats()
        if field == "NBR":
            return self.n_gas * 64
        if field == "NODES":
            return 4 * st["NODES"]
        if field == "NODE_LINKS":
            return 3 * st["NODES"]
        if field == "GROUPS":
            return st["GROUPS"]
        return self.n

    def get(self, field, out=None):
        """Field in the caller's particle order as numpy (or into ``out``,
        a host array or a device tensor)."""
        fid = F[field]
        if out is None:
            out = np.empty(self.count(field), dtype=FIELD_DTYPE.get(field, np.float32))
        ptr, dev = _ptr(out)
        cap = out.numel() if hasattr(out, "numel") else out.size
        self._chk(gnb_get(self.h, fid, ptr, cap, dev))
        if field == "NBR" and isinstance(out, np.ndarray):
            return out.reshape(self.n_gas, 64)
        if field == "NODES" and isinstance(out, np.ndarray):
            return out.reshape(-1, 4)
        return out

    def get_fields(self, outs: dict):
        """Several fields at once into existing arrays ({field name: host
        array or device tensor}, all on one side), one wait for all."""
        names = list(outs)
        ptrs = [_ptr(outs[k]) for k in names]
        on_dev = {d for _, d in ptrs}
        if len(on_dev) != 1:
            raise ValueError("all arrays must be on the same side (host or device)")
        nf = len(names)
        fids = (C.c_int * nf)(*[F[k] for k in names])
        dsts = (C.c_void_p * nf)(*[q for q, _ in ptrs])
        caps = (C.c_int64 * nf)(*[(outs[k].numel() if hasattr(outs[k], "numel") else outs[k].size) for k in names])
        self._chk(gnb_get_fields(self.h, nf, fids, dsts, caps, on_dev.pop()))
        return outs

    def replace_region(self, p: dict):
        """Overwrite the particles with IDs p["id"] by p's position, velocity
        and internal energy (numpy arrays or tensors, all on one side)."""
        keys = ("id", "x", "y", "z", "vx", "vy", "vz", "u")
        arrs = []
        for k in keys:
            a = p[k]
            if isinstance(a, np.ndarray):
                a = np.ascontiguousarray(a, dtype=self._DT[k])
            arrs.append(a)
        ptrs = [_ptr(a) for a in arrs]
        on_dev = {d for _, d in ptrs}
        if len(on_dev) != 1:
            raise ValueError("all arrays must be on the same side (host or device)")
        n = int(arrs[0].shape[0])
        self._chk(gnb_replace_region(self.h, n, *[q for q, _ in ptrs], on_dev.pop()))

    def diagnostics(self):
        out = (C.c_double * 10)()
        self._chk(gnb_diagnostics(self.h, out))
        return np.array(out[:])

    def save(self, path):
        """Particle state and the last force evaluation's results to a file
        (gnb_save)."""
        self._chk(gnb_save(self.h, path))

    def load(self, path):
        """Replace the particles by a saved state (gnb_load)."""
        self._chk(gnb_load(self.h, path))
        self.n = int(self.stats()["N"])
        self.n_gas = int(self.stats()["NGAS"])

    def stats(self):
        out = (C.c_int64 * len(STATS))()
        self._chk(gnb_stats(self.h, out))
        return dict(zip(STATS, out[:]))

    def inject_energy(self, pos, energy):
        """Thermal energy into the n_ngb nearest gas particles; returns
        {weights_sum, energy_added, h, heated}."""
        p = (C.c_double * 3)(*[float(v) for v in pos])
        info = (C.c_double * 4)()
        self._chk(gnb_inject_energy(self.h, p, float(energy), info))
        return dict(zip(("weights_sum", "energy_added", "h", "heated"), info[:]))

    def cfl_timestep(self, courant=0.3):
        dt = C.c_double(0.0)
        self._chk(gnb_cfl_timestep(self.h, float(courant), C.byref(dt)))
        return dt.value

    def integrate_cfl(self, t_span, courant=0.3, max_steps=1 << 30, mode=GNB_GRAV_NONE):
        """Plain CFL-limited KDK integration over t_span; returns (t, steps)."""
        t = C.c_double(0.0)
        n = C.c_int64(0)
        self._chk(gnb_integrate_cfl(self.h, float(t_span), float(courant), int(min(max_steps, 2**31 - 1)), mode,
                                    C.byref(t), C.byref(n)))
        return t.value, n.value

    def integrate_hier(self, t_span, courant=0.3, max_level=20, max_steps=1 << 30, mode=GNB_GRAV_NONE):
        """Plain integration over t_span with hierarchical individual
        timesteps; returns (t, block steps, particle updates, wake-ups)."""
        t = C.c_double(0.0)
        info = (C.c_int64 * 3)()
        self._chk(gnb_integrate_hier(self.h, float(t_span), float(courant), int(max_level),
                                     int(min(max_steps, 2**31 - 1)), mode, C.byref(t), info))
        return t.value, int(info[0]), int(info[1]), int(info[2])

    def voxelise(self, centers, side=60.0, grid=64):
        """Standardised grids [nreg, grid, grid, grid, 5] of the regions."""
        c, cp = _centers(centers)
        nreg = c.size // 3
        out = np.empty((nreg, grid, grid, grid, 5), np.float32)
        self._chk(gnb_voxelise(self.h, nreg, cp, float(side), grid, out.ctypes.data, 0))
        return out

    def remap_regions(self, centers, pred, side=60.0, seed=0, sweeps=8):
        c, cp = _centers(centers)
        nreg = c.size // 3
        pred = np.ascontiguousarray(pred, dtype=np.float32)
        grid = int(round((pred.size // (5 * nreg)) ** (1.0 / 3.0)))
        self._chk(gnb_remap_regions(self.h, nreg, cp, float(side), grid, pred.ctypes.data, int(seed), int(sweeps), 0))

    def sn_surrogate_batch(self, net, centers, side=60.0, seed=0, sweeps=8, use_graph=True):
        c, cp = _centers(centers)
        self._chk(gnb_sn_surrogate_batch(self.h, net.h, c.size // 3, cp, float(side), int(seed), int(sweeps),
                                         1 if use_graph else 0))

    def set_params(self, **params):
        """Change configuration fields (tree and forces are recomputed later)."""
        for k, v in params.items():
            if not hasattr(self.cfg, k):
                raise KeyError(k)
            setattr(self.cfg, k, v)
        self._chk(gnb_set_config(self.h, self.cfg))

    def set_timing(self, enable=True):
        self._chk(gnb_set_timing(self.h, 1 if enable else 0))

    def set_sn_chunks(self, chunks):
        self._chk(gnb_set_sn_chunks(self.h, int(chunks)))

    def sn_async_submit(self, net, centers, side=60.0, seed=0, sweeps=8):
        """Snapshot the regions' members and start voxelise + U-Net on a side stream."""
        c, cp = _centers(centers)
        self._sna_keep = (c, net)  # the centres array and the network outlive the call
        self._chk(gnb_sn_async_submit(self.h, net.h, c.size // 3, cp, float(side), int(seed), int(sweeps)))

    def sn_async_apply(self):
        """Replace the snapshot's members from the pending batch's prediction."""
        self._chk(gnb_sn_async_apply(self.h))
        self._sna_keep = None

    def sn_async_pending(self):
        return bool(gnb_sn_async_pending(self.h))

    def phase_times(self, reset=False):
        """({phase: ms}, {phase: timed occurrences}, library kernel launches)."""
        ms = (C.c_double * len(PHASES))()
        calls = (C.c_int64 * len(PHASES))()
        launches = C.c_int64(0)
        self._chk(gnb_phase_times(self.h, ms, calls, C.byref(launches), 1 if reset else 0))
        return dict(zip(PHASES, ms[:])), dict(zip(PHASES, calls[:])), launches.value
