"""FP64 oracle of the surrogate's particle <-> grid mappings (Sec. 3.3 of
Hirashima et al., SC'25): voxelisation of the gas in a (60 pc)^3 cube around
a supernova onto 64^3 voxels (SPH kernel convolution for the density, the
Shepard method for temperature and velocity), the network's channel
standardisation, and the count-conserving Gibbs-sampling remap back to
particles.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Readings (the paper gives no formulas for these steps):
  channels  z0 = log10(max(rho, 1e-4 Msun/pc^3)) + 0.33
            z1 = (log10(max(T, 10 K)) - 2) / 2
            z2..z4 = v / (20 km/s)
  empty voxels (no kernel overlaps them) have rho = 0 (floored), T = 10 K,
  v = 0; T = u * T_PER_U with T_PER_U = (gamma-1) mu m_H / k_B in K per
  (km/s)^2 (mu = 0.6); membership: gas particles with |x - c|_inf <= side/2,
  each in the first such region.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import lib, _p, f64, GAS

T_PER_U = (2.0 / 3.0) * 0.6 * 1.67262e-24 * 1.0e10 / 1.380649e-16
RHO_FLOOR = 1e-4
T_FLOOR = 10.0


def _declare():
    L = lib()
    if getattr(L, "_sur_declared", False):
        return L
    d = C.POINTER(C.c_double)
    L.orc_voxelise.argtypes = ([C.c_int64] + [d] * 10 + [d, C.c_double, C.c_int, d])
    L.orc_uniform.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64]
    L.orc_uniform.restype = C.c_double
    L.orc_splitmix64.argtypes = [C.c_uint64]
    L.orc_splitmix64.restype = C.c_uint64
    L.orc_gibbs_remap.argtypes = [C.c_int64, C.POINTER(C.c_int64), C.POINTER(C.c_int32), d, C.c_int, d,
                                  C.c_double, C.c_uint64, C.c_int, C.POINTER(C.c_int32), d]
    L._sur_declared = True
    return L


def members(s: dict, centers, side: float):
    """Region index of every particle (-1 outside all regions or not gas)."""
    reg = np.full(s["x"].shape[0], -1, np.int64)
    gas = s["type"] == GAS
    for r, c in enumerate(np.asarray(centers, np.float64).reshape(-1, 3)):
        inside = gas & (reg < 0)
        for a, k in enumerate(("x", "y", "z")):
            inside &= np.abs(s[k] - c[a]) <= 0.5 * side
        reg[inside] = r
    return reg


def accumulate(x, y, z, m, h, rho, T, vx, vy, vz, center, side, grid):
    """Raw voxel accumulators (grid^3, 6) of the given particles."""
    L = _declare()
    lo = np.asarray(center, np.float64) - 0.5 * side
    acc = np.zeros((grid ** 3) * 6)
    arrs = [f64(a) for a in (x, y, z, m, h, rho, T, vx, vy, vz)]
    L.orc_voxelise(arrs[0].size, *(_p(a, np.float64) for a in arrs), _p(f64(lo), np.float64), float(side), grid,
                   _p(acc, np.float64))
    return acc.reshape(grid ** 3, 6)


def standardise(acc):
    """Network input channels from the accumulators (see module docstring)."""
    rho = acc[:, 0]
    den = acc[:, 1]
    safe = np.where(den > 0, den, 1.0)
    T = np.where(den > 0, acc[:, 2] / safe, T_FLOOR)
    v = np.where(den[:, None] > 0, acc[:, 3:6] / safe[:, None], 0.0)
    z = np.empty((acc.shape[0], 5))
    z[:, 0] = np.log10(np.maximum(rho, RHO_FLOOR)) + 0.33
    z[:, 1] = (np.log10(np.maximum(T, T_FLOOR)) - 2.0) / 2.0
    z[:, 2:5] = v / 20.0
    return z


def voxelise(s: dict, rho, h, center, side=60.0, grid=64, region_mask=None):
    """Standardised (grid^3, 5) cube of the gas selected by region_mask;
    rho and h (support) are per particle."""
    sel = region_mask if region_mask is not None else (s["type"] == GAS)
    T = s["u"] * T_PER_U
    acc = accumulate(s["x"][sel], s["y"][sel], s["z"][sel], s["m"][sel], h[sel], rho[sel], T[sel],
                     s["vx"][sel], s["vy"][sel], s["vz"][sel], center, side, grid)
    return standardise(acc)


def weights(pred):
    """Voxel weights of the Gibbs sampler: the predicted density."""
    return np.power(10.0, pred[:, 0].astype(np.float64) - 0.33)


def uniform(seed, pid, k):
    return _declare().orc_uniform(seed, pid, k)


def splitmix64(x):
    return int(_declare().orc_splitmix64(x))


def remap(pred, ids, pos, center, side=60.0, grid=64, seed=0, sweeps=8):
    """New positions, internal energies and velocities of the particles
    ``ids`` (old positions ``pos``, shape (n, 3)) sampled from the predicted
    standardised grid.  Returns (voxel indices (n, 3), positions, u, v)."""
    L = _declare()
    lo = np.asarray(center, np.float64) - 0.5 * side
    d = side / grid
    start = np.clip(np.floor((np.asarray(pos, np.float64) - lo) / d), 0, grid - 1).astype(np.int32)
    n = start.shape[0]
    w = np.ascontiguousarray(weights(pred))
    vox = np.zeros((n, 3), np.int32)
    newp = np.zeros((n, 3))
    idv = np.ascontiguousarray(ids, dtype=np.int64)
    L.orc_gibbs_remap(n, idv.ctypes.data_as(C.POINTER(C.c_int64)),
                      np.ascontiguousarray(start).ctypes.data_as(C.POINTER(C.c_int32)), _p(w, np.float64), grid,
                      _p(f64(lo), np.float64), float(side), int(seed), int(sweeps),
                      vox.ctypes.data_as(C.POINTER(C.c_int32)), _p(newp, np.float64))
    flat = (vox[:, 2] * grid + vox[:, 1]) * grid + vox[:, 0]
    p = pred[flat].astype(np.float64)
    T = np.power(10.0, 2.0 * p[:, 1] + 2.0)
    u = T / T_PER_U
    v = 20.0 * p[:, 2:5]
    return vox, newp, u, v
