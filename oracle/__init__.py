"""FP64 CPU oracle of the N-body/SPH interaction path and the supernova
surrogate.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package.  It shares no code with
the CUDA library (``paper_2510_23330_gb300``); the two only share the seeded
input generators of ``paper_2510_23330_gb300.ics``.

The particle part is plain C (``oracle.c``, built with
``-O2 -ffp-contract=off -fopenmp``) wrapped with ctypes; the compositions that
are a few lines of array arithmetic (external halo, leapfrog, diagnostics)
are written here with numpy in FP64.  Each function cites the passage of
Hirashima et al. (SC'25, arXiv 2510.23330) it follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

GAS = 1


def build(force: bool = False) -> str:
    """Compile oracle.c into a shared library (gcc, no FMA contraction)."""
    src = os.path.join(_HERE, "oracle.c")
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(src)):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-shared", "-fPIC", "-std=c11", "-D_GNU_SOURCE", src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            _declare(_lib)
    return _lib


_d = C.POINTER(C.c_double)
_i64 = C.POINTER(C.c_int64)
_u64 = C.POINTER(C.c_uint64)
_i32 = C.POINTER(C.c_int32)


def _declare(L):
    L.orc_direct_gravity.argtypes = [C.c_int64] + [_d] * 5 + [C.c_double] + [_d] * 5
    L.orc_direct_gravity_sample.argtypes = ([C.c_int64] + [_d] * 5 + [C.c_double, C.c_int64, _i64]
                                            + [_d] * 5)
    L.orc_root_box.argtypes = [C.c_int64, _d, _d, _d, _d, _d]
    L.orc_morton.argtypes = [C.c_int64, _d, _d, _d, _d, C.c_double, _u64, _i32, _i32, _i32]
    L.orc_sort_order.argtypes = [C.c_int64, _u64, _i64]
    L.orc_octree.argtypes = [C.c_int64, _u64, C.c_int, C.c_int64, _i32, _u64, _i64, _i64, _i64, _i32]
    L.orc_octree.restype = C.c_int64
    L.orc_moments.argtypes = [C.c_int64, _i64, _i64] + [_d] * 5 + [_d] * 4
    L.orc_groups.argtypes = [C.c_int64, _i64, _i64, _i32, C.c_int64, _i64]
    L.orc_groups.restype = C.c_int64
    L.orc_walk.argtypes = [C.c_int64, _i32, _u64, _i64, _i64, _i64, _i32, _i32, _i32, _i32,
                           C.c_double, C.c_int64, C.c_int64, _i64, _i64, C.c_int64, _i64, _i64]
    L.orc_walk.restype = C.c_int
    L.orc_tree_gravity.argtypes = ([C.c_int64] + [_d] * 5 + [C.c_double, C.c_double, C.c_int,
                                   C.c_int64, C.c_int] + [_d] * 5 + [_i64])
    L.orc_tree_gravity.restype = C.c_int
    L.orc_tree_gravity_ex.argtypes = L.orc_tree_gravity.argtypes + [C.c_int64, _d]
    L.orc_tree_gravity_ex.restype = C.c_int
    L.orc_knn.argtypes = [C.c_int64, _d, _d, _d, C.c_int, C.c_int64, _i64, _i64, _d]
    L.orc_knn.restype = C.c_int
    L.orc_kernel_eval.argtypes = [C.c_int64, _d, C.c_double, _d, _d]
    L.orc_density.argtypes = [C.c_int64, _i64, _d, _d, _d, _d, _d, C.c_int, _i64, _d,
                              C.c_double, _d, _d, _d, C.c_int]
    L.orc_sph_force.argtypes = ([C.c_int64] + [_d] * 6 + [_d] * 4 + [_d, C.c_int, _i64, C.c_double]
                                + [_d] * 5 + [_d, C.c_double, C.c_int, _d])
    L.orc_sph_force.restype = C.c_int
    L.orc_num_threads.restype = C.c_int
    L.orc_sph_vsig.argtypes = [C.c_int64] + [_d] * 7 + [C.c_int, _i64, _d]


def _p(a, dtype):
    assert a.dtype == dtype and a.flags.c_contiguous, (a.dtype, dtype)
    ct = {np.float64: C.c_double, np.int64: C.c_int64, np.uint64: C.c_uint64,
          np.int32: C.c_int32}[dtype]
    return a.ctypes.data_as(C.POINTER(ct))


def f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return int(lib().orc_num_threads())


# --------------------------------------------------------------------------
# Gravity
# --------------------------------------------------------------------------
def direct_gravity(p: dict, G: float = 1.0) -> dict:
    """O(N^2) softened gravity, Sec. 3.5 Eq. 1 (per-particle softening)."""
    n = p["x"].shape[0]
    x, y, z, m, e = (f64(p[k]) for k in ("x", "y", "z", "m", "eps"))
    out = {k: np.zeros(n) for k in ("ax", "ay", "az", "phi", "asum")}
    lib().orc_direct_gravity(n, _p(x, np.float64), _p(y, np.float64), _p(z, np.float64),
                             _p(m, np.float64), _p(e, np.float64), G,
                             *(_p(out[k], np.float64) for k in ("ax", "ay", "az", "phi", "asum")))
    return out


def direct_gravity_sample(p: dict, sample, G: float = 1.0) -> dict:
    """Eq. 1 direct sum for the listed particles only."""
    n = p["x"].shape[0]
    x, y, z, m, e = (f64(p[k]) for k in ("x", "y", "z", "m", "eps"))
    sample = np.ascontiguousarray(sample, dtype=np.int64)
    ns = sample.shape[0]
    out = {k: np.zeros(ns) for k in ("ax", "ay", "az", "phi", "asum")}
    lib().orc_direct_gravity_sample(n, _p(x, np.float64), _p(y, np.float64), _p(z, np.float64),
                                    _p(m, np.float64), _p(e, np.float64), G, ns, _p(sample, np.int64),
                                    *(_p(out[k], np.float64) for k in ("ax", "ay", "az", "phi", "asum")))
    return out


def root_box(p: dict):
    n = p["x"].shape[0]
    x, y, z = (f64(p[k]) for k in ("x", "y", "z"))
    lo = np.zeros(3)
    L = np.zeros(1)
    lib().orc_root_box(n, _p(x, np.float64), _p(y, np.float64), _p(z, np.float64),
                       _p(lo, np.float64), _p(L, np.float64))
    return lo, float(L[0])


def morton(p: dict):
    """Morton keys and grid cells of every particle (input order)."""
    n = p["x"].shape[0]
    x, y, z = (f64(p[k]) for k in ("x", "y", "z"))
    lo, L = root_box(p)
    key = np.zeros(n, np.uint64)
    c = [np.zeros(n, np.int32) for _ in range(3)]
    lib().orc_morton(n, _p(x, np.float64), _p(y, np.float64), _p(z, np.float64),
                     _p(lo, np.float64), L, _p(key, np.uint64), *(_p(a, np.int32) for a in c))
    return key, np.stack(c, axis=1), lo, L


def sort_order(key: np.ndarray) -> np.ndarray:
    n = key.shape[0]
    key = np.ascontiguousarray(key, dtype=np.uint64)
    order = np.zeros(n, np.int64)
    lib().orc_sort_order(n, _p(key, np.uint64), _p(order, np.int64))
    return order


def octree(skey: np.ndarray, n_leaf: int) -> dict:
    """Breadth-first octree over sorted keys (see oracle.c)."""
    n = skey.shape[0]
    skey = np.ascontiguousarray(skey, dtype=np.uint64)
    cap = 4 * n + 64
    t = {"level": np.zeros(cap, np.int32), "prefix": np.zeros(cap, np.uint64),
         "first": np.zeros(cap, np.int64), "count": np.zeros(cap, np.int64),
         "child": np.zeros(cap, np.int64), "nchild": np.zeros(cap, np.int32)}
    nn = lib().orc_octree(n, _p(skey, np.uint64), n_leaf, cap, _p(t["level"], np.int32),
                          _p(t["prefix"], np.uint64), _p(t["first"], np.int64),
                          _p(t["count"], np.int64), _p(t["child"], np.int64),
                          _p(t["nchild"], np.int32))
    if nn < 0:
        raise RuntimeError("octree capacity")
    return {k: v[:nn].copy() for k, v in t.items()}


def moments(tree: dict, sp: dict) -> dict:
    """Cell mass, centre of mass, traceless quadrupole and mean eps^2 over
    particles given in sorted order."""
    nn = tree["level"].shape[0]
    M, e2 = np.zeros(nn), np.zeros(nn)
    com, Q = np.zeros((nn, 3)), np.zeros((nn, 6))
    arrs = [f64(sp[k]) for k in ("x", "y", "z", "m", "eps")]
    lib().orc_moments(nn, _p(tree["first"], np.int64), _p(tree["count"], np.int64),
                      *(_p(a, np.float64) for a in arrs), _p(M, np.float64),
                      _p(com, np.float64), _p(Q, np.float64), _p(e2, np.float64))
    return {"M": M, "com": com, "Q": Q, "eps2": e2}


def groups(tree: dict, n_g: int) -> np.ndarray:
    nn = tree["level"].shape[0]
    g = np.zeros(nn, np.int64)
    ng = lib().orc_groups(nn, _p(tree["count"], np.int64), _p(tree["child"], np.int64),
                          _p(tree["nchild"], np.int32), n_g, _p(g, np.int64))
    return g[:ng].copy()


def walk(g: int, tree: dict, cells_sorted: np.ndarray, theta: float):
    """Interaction lists of group node g: (EPJ particle slots, SPJ cells)."""
    nn = tree["level"].shape[0]
    n = cells_sorted.shape[0]
    cs = [np.ascontiguousarray(cells_sorted[:, a], dtype=np.int32) for a in range(3)]
    epj = np.zeros(n + 1, np.int64)
    spj = np.zeros(nn + 1, np.int64)
    ne, ns = np.zeros(1, np.int64), np.zeros(1, np.int64)
    rc = lib().orc_walk(g, _p(tree["level"], np.int32), _p(tree["prefix"], np.uint64),
                        _p(tree["first"], np.int64), _p(tree["count"], np.int64),
                        _p(tree["child"], np.int64), _p(tree["nchild"], np.int32),
                        *(_p(a, np.int32) for a in cs), theta, nn, n + 1, _p(epj, np.int64),
                        _p(ne, np.int64), nn + 1, _p(spj, np.int64), _p(ns, np.int64))
    if rc != 0:
        raise RuntimeError("walk overflow")
    return epj[:ne[0]].copy(), spj[:ns[0]].copy()


def tree_gravity(p: dict, theta: float = 0.5, n_leaf: int = 16, n_g: int = 64,
                 quad: bool = True, G: float = 1.0) -> dict:
    """Barnes-Hut group-walk gravity, every step of the approximation in
    plain FP64 (Sec. 3.4, 5.2.2, 5.2.4)."""
    n = p["x"].shape[0]
    arrs = [f64(p[k]) for k in ("x", "y", "z", "m", "eps")]
    out = {k: np.zeros(n) for k in ("ax", "ay", "az", "phi", "asum")}
    stats = np.zeros(4, np.int64)
    rc = lib().orc_tree_gravity(n, *(_p(a, np.float64) for a in arrs), G, theta, n_leaf,
                                n_g, int(bool(quad)),
                                *(_p(out[k], np.float64) for k in ("ax", "ay", "az", "phi", "asum")),
                                _p(stats, np.int64))
    if rc != 0:
        raise RuntimeError("oracle tree gravity failed")
    out["nodes"], out["groups"], out["n_pp"], out["n_pc"] = (int(s) for s in stats)
    return out


def tree_gravity_sampled(p: dict, gstride: int, theta: float = 0.5, n_leaf: int = 16,
                         n_g: int = 64, quad: bool = True, G: float = 1.0):
    """Tree gravity walking every gstride-th group only.  Returns
    (build_seconds, walk_seconds, stats) for timing a bounded sample."""
    n = p["x"].shape[0]
    arrs = [f64(p[k]) for k in ("x", "y", "z", "m", "eps")]
    out = {k: np.zeros(n) for k in ("ax", "ay", "az", "phi", "asum")}
    stats = np.zeros(4, np.int64)
    times = np.zeros(2)
    rc = lib().orc_tree_gravity_ex(n, *(_p(a, np.float64) for a in arrs), G, theta, n_leaf, n_g,
                                   int(bool(quad)),
                                   *(_p(out[k], np.float64) for k in ("ax", "ay", "az", "phi", "asum")),
                                   _p(stats, np.int64), int(gstride), _p(times, np.float64))
    if rc != 0:
        raise RuntimeError("oracle tree gravity failed")
    return float(times[0]), float(times[1]), stats


# --------------------------------------------------------------------------
# SPH
# --------------------------------------------------------------------------
def knn(g: dict, k: int = 64, sample=None):
    """Exact k nearest gas neighbours (self included) by (d^2, index); h^2 is
    the k-th d^2 (kernel size, Sec. 5.2.5).  ``g`` holds gas particles only;
    indices refer to g's order."""
    n = g["x"].shape[0]
    x, y, z = (f64(g[a]) for a in ("x", "y", "z"))
    if sample is None:
        sample = np.arange(n, dtype=np.int64)
    sample = np.ascontiguousarray(sample, dtype=np.int64)
    ns = sample.shape[0]
    nbr = np.zeros((ns, k), np.int64)
    h2 = np.zeros(ns)
    rc = lib().orc_knn(n, _p(x, np.float64), _p(y, np.float64), _p(z, np.float64), k, ns,
                       _p(sample, np.int64), _p(nbr, np.int64), _p(h2, np.float64))
    if rc != 0:
        raise ValueError("fewer gas particles than neighbours")
    return nbr, h2


def kernel(r, h):
    r = f64(r)
    w, dw = np.zeros_like(r), np.zeros_like(r)
    lib().orc_kernel_eval(r.shape[0], _p(r, np.float64), float(h), _p(w, np.float64),
                          _p(dw, np.float64))
    return w, dw


def density(g: dict, nbr, h2, gamma: float = 5.0 / 3.0, sample=None, u=None, pressure: bool = False):
    """rho, P, c of the sampled gas particles (Table 3 "density and pressure").
    pressure=True: P is the smoothed pressure (gamma-1) sum_j m_j u_j W_ij(h_i)
    of pressure-energy SPH instead of (gamma-1) rho_i u_i."""
    n = g["x"].shape[0]
    if sample is None:
        sample = np.arange(n, dtype=np.int64)
    sample = np.ascontiguousarray(sample, dtype=np.int64)
    ns, k = nbr.shape
    x, y, z, m = (f64(g[a]) for a in ("x", "y", "z", "m"))
    uu = f64(g["u"] if u is None else u)
    nbr = np.ascontiguousarray(nbr, dtype=np.int64)
    h2 = f64(h2)
    rho, P, c = np.zeros(ns), np.zeros(ns), np.zeros(ns)
    lib().orc_density(ns, _p(sample, np.int64), _p(x, np.float64), _p(y, np.float64),
                      _p(z, np.float64), _p(m, np.float64), _p(uu, np.float64), k,
                      _p(nbr, np.int64), _p(h2, np.float64), gamma, _p(rho, np.float64),
                      _p(P, np.float64), _p(c, np.float64), int(pressure))
    return rho, P, c


def sph_force(g: dict, nbr, h2, rho, P, c, alpha: float = 1.0, v=None, u=None,
              gamma: float = 5.0 / 3.0, pressure: bool = False):
    """Symmetric SPH pressure force + artificial viscosity and du/dt over the
    union neighbour sets (Table 3 "hydro force"); pressure=True: the
    pressure-energy form with the smoothed pressure P (see oracle.c).
    Also returns the sums' scales: asum = sum_j |a_ij| and dusum = sum_j of
    the magnitudes of du/dt's pressure and viscosity terms."""
    n, k = nbr.shape
    x, y, z, m = (f64(g[a]) for a in ("x", "y", "z", "m"))
    if v is None:
        v = (g["vx"], g["vy"], g["vz"])
    vx, vy, vz = (f64(a) for a in v)
    out = {a: np.zeros(n) for a in ("ax", "ay", "az", "dudt", "asum", "dusum")}
    nbr = np.ascontiguousarray(nbr, dtype=np.int64)
    rc = lib().orc_sph_force(n, *(_p(a, np.float64) for a in (x, y, z, vx, vy, vz, m)),
                             *(_p(f64(a), np.float64) for a in (rho, P, c, h2)), k,
                             _p(nbr, np.int64), alpha,
                             *(_p(out[a], np.float64) for a in ("ax", "ay", "az", "dudt", "asum")),
                             _p(f64(g["u"] if u is None else u), np.float64), gamma, int(pressure),
                             _p(out["dusum"], np.float64))
    if rc != 0:
        raise RuntimeError("oracle sph force failed")
    return out


def sph_vsig(g: dict, nbr, c, v=None):
    """Largest pair signal velocity c_i + c_j - 3 min(w_ij, 0) per particle."""
    n, k = nbr.shape
    x, y, z = (f64(g[a]) for a in ("x", "y", "z"))
    if v is None:
        v = (g["vx"], g["vy"], g["vz"])
    vx, vy, vz = (f64(a) for a in v)
    out = np.zeros(n)
    lib().orc_sph_vsig(n, *(_p(a, np.float64) for a in (x, y, z, vx, vy, vz, f64(c))), k,
                       _p(np.ascontiguousarray(nbr, dtype=np.int64), np.int64), _p(out, np.float64))
    return out


def sph(g: dict, k: int = 64, gamma: float = 5.0 / 3.0, alpha: float = 1.0, u=None, v=None,
        pressure: bool = False):
    """kNN + density + force for a gas-only particle set (pressure=True:
    pressure-energy SPH)."""
    nbr, h2 = knn(g, k)
    rho, P, c = density(g, nbr, h2, gamma, u=u, pressure=pressure)
    f = sph_force(g, nbr, h2, rho, P, c, alpha, v=v, u=u, gamma=gamma, pressure=pressure)
    f.update(nbr=nbr, h2=h2, rho=rho, P=P, c=c, vsig=sph_vsig(g, nbr, c, v=v))
    return f


# --------------------------------------------------------------------------
# External halo, forces, leapfrog, diagnostics
# --------------------------------------------------------------------------
def nfw(p: dict, Ms: float, rs: float, G: float = 1.0):
    """Static NFW halo: M(<r) = Ms [ln(1+r/rs) - (r/rs)/(1+r/rs)],
    a = -G M(<r) x / r^3, Phi = -G Ms ln(1 + r/rs) / r."""
    x, y, z = (f64(p[k]) for k in ("x", "y", "z"))
    r = np.sqrt(x * x + y * y + z * z)
    s = r / rs
    menc = Ms * (np.log1p(s) - s / (1.0 + s))
    with np.errstate(divide="ignore", invalid="ignore"):
        f = np.where(r > 0, -G * menc / r ** 3, 0.0)
        pot = np.where(r > 0, -G * Ms * np.log1p(s) / r, -G * Ms / rs)
    return f * x, f * y, f * z, pot


class Config:
    """Parameters of one force evaluation (defaults of the disk model)."""

    def __init__(self, G=1.0, theta=0.5, n_leaf=16, n_g=64, quad=True, gravity="tree",
                 n_ngb=64, gamma=5.0 / 3.0, alpha=1.0, nfw_ms=0.0, nfw_rs=8.0, sph="density"):
        self.G, self.theta, self.n_leaf, self.n_g, self.quad = G, theta, n_leaf, n_g, quad
        self.gravity, self.n_ngb, self.gamma, self.alpha = gravity, n_ngb, gamma, alpha
        self.nfw_ms, self.nfw_rs = nfw_ms, nfw_rs
        self.sph = sph  # "density": density-energy SPH; "pressure": pressure-energy SPH


def forces(s: dict, cfg: Config, u=None, v=None) -> dict:
    """Total acceleration, self-gravity potential and du/dt of state ``s``.
    ``u`` and ``v`` override the gas internal energy and velocity used by the
    pressure and viscosity terms (the predicted values of the leapfrog)."""
    n = s["x"].shape[0]
    if cfg.gravity == "direct":
        g = direct_gravity(s, cfg.G)
    elif cfg.gravity == "none":
        g = {k: np.zeros(n) for k in ("ax", "ay", "az", "phi", "asum")}
    else:
        g = tree_gravity(s, cfg.theta, cfg.n_leaf, cfg.n_g, cfg.quad, cfg.G)
    ax, ay, az = g["ax"].copy(), g["ay"].copy(), g["az"].copy()
    pext = np.zeros(n)
    if cfg.nfw_ms > 0:
        ex, ey, ez, pext = nfw(s, cfg.nfw_ms, cfg.nfw_rs, cfg.G)
        ax += ex; ay += ey; az += ez
    dudt = np.zeros(n)
    gi = np.nonzero(s["type"] == GAS)[0]
    res = {"phi": g["phi"], "phi_ext": pext, "grav": g}
    if gi.size:
        gs = {k: s[k][gi] for k in ("x", "y", "z", "m")}
        uu = (s["u"] if u is None else u)[gi]
        vv = [(s[k] if v is None else v[a])[gi] for a, k in enumerate(("vx", "vy", "vz"))]
        gs["u"] = uu
        h = sph(gs, cfg.n_ngb, cfg.gamma, cfg.alpha, u=uu, v=vv, pressure=cfg.sph == "pressure")
        ax[gi] += h["ax"]; ay[gi] += h["ay"]; az[gi] += h["az"]
        dudt[gi] = h["dudt"]
        res["sph"] = h
        res["gas_index"] = gi
    res.update(ax=ax, ay=ay, az=az, dudt=dudt)
    return res


def state(p: dict) -> dict:
    """FP64 working copy of a particle set."""
    s = {k: f64(p[k]) for k in ("x", "y", "z", "vx", "vy", "vz", "m", "eps", "u")}
    s["type"] = np.asarray(p["type"]).copy()
    s["id"] = np.asarray(p["id"]).copy()
    return s


def kdk_step(s: dict, f: dict, dt: float, cfg: Config):
    """One kick-drift-kick leapfrog step with a shared timestep (Sec. 3.2:
    half kick, drift, force, half kick).  ``f`` holds the forces at the start
    of the step; returns the new state and its forces.  The gas pressure and
    viscosity at the end of the step use the predicted u and v."""
    h = 0.5 * dt
    ns = dict(s)
    vhx = s["vx"] + f["ax"] * h
    vhy = s["vy"] + f["ay"] * h
    vhz = s["vz"] + f["az"] * h
    uh = s["u"] + f["dudt"] * h
    ns["x"] = s["x"] + vhx * dt
    ns["y"] = s["y"] + vhy * dt
    ns["z"] = s["z"] + vhz * dt
    vp = (vhx + f["ax"] * h, vhy + f["ay"] * h, vhz + f["az"] * h)
    up = uh + f["dudt"] * h
    nf = forces(ns, cfg, u=up, v=vp)
    ns["vx"] = vhx + nf["ax"] * h
    ns["vy"] = vhy + nf["ay"] * h
    ns["vz"] = vhz + nf["az"] * h
    ns["u"] = uh + nf["dudt"] * h
    return ns, nf


def diagnostics(s: dict, f: dict) -> np.ndarray:
    """E_kin, E_pot (self-gravity, 1/2 sum m phi), E_ext, E_th, P[3], L[3]."""
    m = s["m"]
    v2 = s["vx"] ** 2 + s["vy"] ** 2 + s["vz"] ** 2
    gas = s["type"] == GAS
    ek = 0.5 * np.sum(m * v2)
    ep = 0.5 * np.sum(m * f["phi"])
    ee = np.sum(m * f["phi_ext"])
    eth = np.sum(m[gas] * s["u"][gas])
    P = [np.sum(m * s[k]) for k in ("vx", "vy", "vz")]
    x, y, z, vx, vy, vz = (s[k] for k in ("x", "y", "z", "vx", "vy", "vz"))
    L = [np.sum(m * (y * vz - z * vy)), np.sum(m * (z * vx - x * vz)),
         np.sum(m * (x * vy - y * vx))]
    return np.array([ek, ep, ee, eth, *P, *L])


# --------------------------------------------------------------------------
# Supernova region: injection and plain CFL-limited integration
# --------------------------------------------------------------------------
def inject_energy(s: dict, pos, E: float, k: int = 64):
    """Thermal energy E into the k gas particles nearest to pos (ordered by
    FP64 d^2 = (dx*dx + dy*dy) + dz*dz, then gas rank), weighted by the cubic
    spline with support h = distance to the k-th: du_j = E W_j/(m_j sum W).
    Returns the new state and {h, members, energy_added}."""
    gi = np.nonzero(s["type"] == GAS)[0]
    dx, dy, dz = (s[a][gi] - float(pos[i]) for i, a in enumerate(("x", "y", "z")))
    d2 = (dx * dx + dy * dy) + dz * dz
    order = np.lexsort((np.arange(gi.size), d2))[:k]
    h = float(np.sqrt(d2[order[-1]]))
    r = np.sqrt(d2[order])
    if h > 0:
        w, _ = kernel(r, h)
    else:
        w = np.ones(k)
    ns = dict(s)
    ns["u"] = s["u"].copy()
    members = gi[order]
    du = E * w / (s["m"][members] * w.sum())
    ns["u"][members] += du
    return ns, {"h": h, "members": members, "energy_added": float(np.sum(s["m"][members] * du)),
                "weights_sum": float(w.sum())}


def cfl_dt(f: dict, courant: float = 0.3) -> float:
    """dt = courant * min_i h_i / vsig_i over the gas of a force evaluation."""
    h = np.sqrt(f["sph"]["h2"])
    return float(courant * np.min(h / f["sph"]["vsig"]))


def integrate_cfl(s: dict, t_span: float, courant: float, cfg: Config, max_steps: int = 1 << 30):
    """Plain small-timestep integration: KDK steps of the CFL timestep, the
    last one shortened to end at t_span.  Returns (state, forces, t, steps)."""
    f = forces(s, cfg)
    t, n = 0.0, 0
    while t < t_span and n < max_steps:
        dt = min(cfl_dt(f, courant), t_span - t)
        s, f = kdk_step(s, f, dt, cfg)
        t += dt
        n += 1
    return s, f, t, n


# --------------------------------------------------------------------------
# Plain integration with hierarchical (block) individual timesteps
# --------------------------------------------------------------------------
# Sec. 1 describes the conventional scheme the surrogate competes with: every
# particle carries its own timestep and is integrated only when its step
# ends, while at each such step the positions and other quantities of all
# particles are predicted and the octree is rebuilt for the force
# calculation.  The paper gives no formulas; the reading written out here is
# the usual power-of-two block scheme on an integer time grid:
#   * ticks: the span is 2^(K+1) ticks of length t_span 2^-(K+1); level k has
#     the step dt_k = t_span 2^-k = 2^(K+1-k) ticks (k = 0 .. K);
#   * the CFL level of a gas particle is the coarsest k with dt_k <= its CFL
#     step C h_i / vsig_i (other particles: level 0); a step starting at tick
#     T takes the coarser of the finest of that level and the coarsest level
#     whose step divides T, so steps start and end on their own grid;
#   * a block step goes to the next tick T at which some step ends, drifts
#     every particle there with its half-step velocity, predicts the velocity
#     and energy of every particle from the force of its last evaluation
#     (v + a (t - t_mid), t_mid the middle of its current step), and
#     evaluates all forces at that predicted state;
#   * a particle whose step ends at T, or whose CFL level at T is finer than
#     its current level (a wake-up: the step is cut short at T, its opening
#     kick and the drift since its start are corrected to the shorter step),
#     gets the closing half kick with the new force and -- unless the span
#     is done -- a new level and the opening half kick of its next step.
def hier_cfl_level(dtc, K: int, t_span: float) -> np.ndarray:
    """The coarsest k <= K with dt_k = t_span 2^-k <= dtc; -1 where even
    dt_K exceeds dtc (the finest level does not resolve the particle)."""
    dtc = np.asarray(dtc, dtype=np.float64)
    k = np.zeros(dtc.shape, dtype=np.int64)
    for j in range(K):
        k += np.ldexp(t_span, -j) > dtc  # dt_j longer than the CFL step: one level finer
    return np.where(np.ldexp(t_span, -K) > dtc, -1, k)


def hier_align_level(T: int, K: int) -> int:
    """The coarsest level whose step 2^(K+1-k) ticks divides tick T."""
    if T == 0:
        return 0
    a = (T & -T).bit_length() - 1  # T = 2^a * odd
    return max(0, K + 1 - a)


def cfl_steps(f: dict, n: int, courant: float) -> np.ndarray:
    """Individual CFL steps: courant h_i / vsig_i for gas, infinite for the
    other particles and for gas with vsig = 0."""
    out = np.full(n, np.inf)
    if "sph" in f:
        gi = f["gas_index"]
        h = np.sqrt(f["sph"]["h2"])
        vs = f["sph"]["vsig"]
        with np.errstate(divide="ignore"):
            out[gi] = np.where(vs > 0, courant * h / np.where(vs > 0, vs, 1.0), np.inf)
    return out


def level_margin(dtc, kc, t_span: float) -> float:
    """Smallest relative distance of a CFL step to the level boundaries that
    decided its level (dt_kc <= dtc < dt_(kc-1)): how far a rounding error
    of the step would have to go to change the decision."""
    dtc = np.asarray(dtc, dtype=np.float64)
    ok = np.isfinite(dtc) & (kc >= 0)
    if not np.any(ok):
        return np.inf
    d, k = dtc[ok], kc[ok]
    lo = np.abs(d / np.ldexp(t_span, -k) - 1.0)
    hi = np.where(k > 0, np.abs(d / np.ldexp(t_span, -(k - 1)) - 1.0), np.inf)
    return float(min(lo.min(), hi.min()))


def integrate_hier(s: dict, t_span: float, courant: float, cfg: Config, max_level: int = 20,
                   max_steps: int = 1 << 30, force_fn=None, step_fn=None):
    """Plain integration over t_span with hierarchical individual timesteps
    (Sec. 1; the reading above).  force_fn(s, u, v) -> {ax, ay, az, dudt, ...}
    defaults to forces(s, cfg, u, v); step_fn(f, n) -> individual steps
    defaults to the CFL steps.  Returns (state, forces, info) with info =
    {t, steps (block steps), updates (particle updates after the start),
    wakeups, level (the last step's), margin (smallest level_margin)}."""
    if force_fn is None:
        def force_fn(st, u=None, v=None):
            return forces(st, cfg, u=u, v=v)
    if step_fn is None:
        def step_fn(ff, nn):
            return cfl_steps(ff, nn, courant)
    K = int(max_level)
    NT = 1 << (K + 1)
    tick = float(np.ldexp(t_span, -(K + 1)))
    s = dict(s)
    for k in ("x", "y", "z", "vx", "vy", "vz", "u"):
        s[k] = np.array(s[k], dtype=np.float64, copy=True)
    n = s["x"].shape[0]
    gas = s["type"] == GAS
    V = ("vx", "vy", "vz")

    def cfl_level(ff):
        dtc = step_fn(ff, n)
        kc = hier_cfl_level(dtc, K, t_span)
        return kc, level_margin(dtc, kc, t_span)

    def kick(mask, acc, half):
        for a, k in enumerate(V):
            s[k][mask] = s[k][mask] + acc[a][mask] * half[mask]
        g = mask & gas
        s["u"][g] = s["u"][g] + acc[3][g] * half[g]

    f = force_fn(s)
    acc = [np.array(f[k], dtype=np.float64, copy=True) for k in ("ax", "ay", "az", "dudt")]
    kc, margin = cfl_level(f)
    if np.any(kc < 0):
        raise ValueError("a CFL step is shorter than the finest level")
    lev = kc.copy()
    T0 = np.zeros(n, dtype=np.int64)
    T1 = np.left_shift(np.int64(1), K + 1 - lev).astype(np.int64)
    kick(np.ones(n, dtype=bool), acc, ((T1 - T0) // 2).astype(np.float64) * tick)  # opening half kicks
    T, steps, updates, wakeups = 0, 0, 0, 0
    while T < NT and steps < max_steps:
        Tn = int(T1.min())
        dd = float(Tn) * tick - float(T) * tick
        for k in ("x", "y", "z"):
            s[k] = s[k] + s["v" + k] * dd
        T = Tn
        tau = (T - (T0 + T1) // 2).astype(np.float64) * tick
        vp = [s[k] + acc[a] * tau for a, k in enumerate(V)]
        up = np.where(gas, s["u"] + acc[3] * tau, 0.0)
        f = force_fn(s, u=up, v=vp)
        kc, mg = cfl_level(f)
        if np.any(kc < 0):
            raise ValueError("a CFL step is shorter than the finest level")
        margin = min(margin, mg)
        due = T1 == T
        wake = ~due & (kc > lev)
        if np.any(wake):
            # the step [T0, T1] becomes [T0, T]: opening kick and drift redone
            cut = (T - T1).astype(np.float64) * (0.5 * tick)  # <= 0
            el = (T - T0).astype(np.float64) * tick
            for a, k in enumerate(V):
                dv = acc[a] * cut
                s[k[1]][wake] = s[k[1]][wake] + (dv * el)[wake]
                s[k][wake] = s[k][wake] + dv[wake]
            g = wake & gas
            s["u"][g] = s["u"][g] + (acc[3] * cut)[g]
        active = due | wake
        new = [np.asarray(f[k], dtype=np.float64) for k in ("ax", "ay", "az", "dudt")]
        for a in range(4):
            acc[a] = np.where(active, new[a], acc[a])
        kick(active, acc, ((T - T0) // 2).astype(np.float64) * tick)  # closing half kicks
        if T < NT:
            lev = np.where(active, np.maximum(kc, hier_align_level(T, K)), lev)
            T0 = np.where(active, T, T0)
            T1 = np.where(active, T + np.left_shift(np.int64(1), K + 1 - lev), T1)
            kick(active, acc, ((T1 - T0) // 2).astype(np.float64) * tick)  # opening half kicks
        steps += 1
        updates += int(np.count_nonzero(active))
        wakeups += int(np.count_nonzero(wake))
    info = {"t": float(T) * tick, "steps": steps, "updates": updates, "wakeups": wakeups,
            "level": lev, "margin": margin}
    return s, f, info
