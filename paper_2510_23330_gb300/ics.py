"""Seeded synthetic initial conditions shared by the CUDA path, the oracle and
the benchmark.

This module only draws particles; it holds none of the method's arithmetic
(no forces, keys, trees, kernels or integrators).  Every generator is a pure
function of its arguments and seed, so both sides of a parity test see the same
bits.  Storage precision follows the mixed-precision rule of Sec. 4.3 of the
paper (positions in FP64) with the per-particle FP32 fields of the library's
particle layout: velocity, mass, softening and internal energy are returned as
float32 so that the oracle receives exactly the values the GPU stores.

The paper's own Milky Way initial conditions come from AGAMA (Sec. 4.2) and are
not available; the generators below stand in for them with the same structure
(a centrally concentrated system, thin disks whose scale height is ~10 % of the
scale length).
"""
from __future__ import annotations

import numpy as np

STAR = 0
GAS = 1


def _pack(x, v, m, eps, u, ptype):
    n = x.shape[0]
    return {
        "id": np.arange(n, dtype=np.int64),
        "type": np.ascontiguousarray(ptype, dtype=np.uint8),
        "x": np.ascontiguousarray(x[:, 0], dtype=np.float64),
        "y": np.ascontiguousarray(x[:, 1], dtype=np.float64),
        "z": np.ascontiguousarray(x[:, 2], dtype=np.float64),
        "vx": np.ascontiguousarray(v[:, 0], dtype=np.float32),
        "vy": np.ascontiguousarray(v[:, 1], dtype=np.float32),
        "vz": np.ascontiguousarray(v[:, 2], dtype=np.float32),
        "m": np.ascontiguousarray(m, dtype=np.float32),
        "eps": np.ascontiguousarray(eps, dtype=np.float32),
        "u": np.ascontiguousarray(u, dtype=np.float32),
    }


def _isotropic(rng, n):
    cz = rng.uniform(-1.0, 1.0, n)
    ph = rng.uniform(0.0, 2.0 * np.pi, n)
    s = np.sqrt(1.0 - cz * cz)
    return np.stack([s * np.cos(ph), s * np.sin(ph), cz], axis=1)


def plummer(n: int, seed: int = 0, n_gas: int | None = None, u_gas: float = 0.05,
            eps: float = 0.01, r_max: float = 100.0) -> dict:
    """Plummer sphere with G = M = a = 1 and equal masses 1/n (Aarseth, Henon
    & Wielen 1974 sampling).  Radii above ``r_max`` are re-drawn.  The first
    ``n - n_gas`` particles are stars, the rest gas with internal energy
    ``u_gas``; ``n_gas`` defaults to n // 2."""
    rng = np.random.default_rng(seed)
    if n_gas is None:
        n_gas = n // 2
    r = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        x1 = rng.uniform(0.0, 1.0, todo.size)
        rr = np.full(todo.size, np.inf)
        ok = x1 > 0.0
        rr[ok] = 1.0 / np.sqrt(x1[ok] ** (-2.0 / 3.0) - 1.0)
        good = rr <= r_max
        r[todo[good]] = rr[good]
        todo = todo[~good]
    pos = _isotropic(rng, n) * r[:, None]
    # speed fraction q from g(q) ~ q^2 (1 - q^2)^{7/2} by rejection
    q = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        x4 = rng.uniform(0.0, 1.0, todo.size)
        x5 = rng.uniform(0.0, 0.1, todo.size)
        good = x5 < x4 * x4 * (1.0 - x4 * x4) ** 3.5
        q[todo[good]] = x4[good]
        todo = todo[~good]
    vesc = np.sqrt(2.0) * (1.0 + r * r) ** (-0.25)
    vel = _isotropic(rng, n) * (q * vesc)[:, None]
    ptype = np.full(n, STAR, np.uint8)
    ptype[n - n_gas:] = GAS
    m = np.full(n, 1.0 / n)
    ep = np.full(n, eps)
    u = np.where(ptype == GAS, u_gas, 0.0)
    return _pack(pos, vel, m, ep, u, ptype)


# Static NFW halo used by the disk model: r_s = 8, M_s = 4 pi rho_s r_s^3 = 30.
NFW_RS = 8.0
NFW_MS = 30.0


def _nfw_menc(r, ms=NFW_MS, rs=NFW_RS):
    x = r / rs
    return ms * (np.log1p(x) - x / (1.0 + x))


def exp_disk(n: int, gas_frac: float = 0.2, seed: int = 0, star_rd: float = 1.0,
             gas_rd: float = 2.0, zd: float = 0.1, eps: float = 0.01,
             u_range=(1e-3, 1e-1), sigma_frac: float = 0.1,
             nfw_ms: float = NFW_MS, nfw_rs: float = NFW_RS) -> dict:
    """Exponential stellar disk plus exponential gas disk (total mass 1, equal
    particle masses) inside a static NFW halo, G = 1.

    Surface density ~ exp(-R/R_d) is drawn as R = -R_d ln(U1 U2); the vertical
    profile ~ sech^2(z/z_d) as z = z_d atanh(2U - 1).  Circular speeds use the
    halo's enclosed mass plus the disk mass enclosed within the spherical
    radius (counted from the sample).  Stars get an isotropic Gaussian
    dispersion of ``sigma_frac`` times the circular speed; gas is on circular
    orbits with u drawn log-uniformly from ``u_range``.  Stars come first."""
    rng = np.random.default_rng(seed)
    n_gas = int(round(gas_frac * n))
    n_star = n - n_gas

    def disk(k, rd):
        u1 = rng.uniform(0.0, 1.0, k)
        u2 = rng.uniform(0.0, 1.0, k)
        u1 = np.where(u1 <= 0.0, 1e-300, u1)
        u2 = np.where(u2 <= 0.0, 1e-300, u2)
        R = -rd * np.log(u1 * u2)
        uz = rng.uniform(-1.0, 1.0, k)
        uz = np.clip(uz, -1.0 + 1e-12, 1.0 - 1e-12)
        z = zd * np.arctanh(uz)
        ph = rng.uniform(0.0, 2.0 * np.pi, k)
        return R, ph, z

    Rs, phs, zs = disk(n_star, star_rd)
    Rg, phg, zg = disk(n_gas, gas_rd)
    R = np.concatenate([Rs, Rg])
    ph = np.concatenate([phs, phg])
    z = np.concatenate([zs, zg])
    pos = np.stack([R * np.cos(ph), R * np.sin(ph), z], axis=1)
    r = np.sqrt(R * R + z * z)
    order = np.argsort(r, kind="stable")
    menc_disk = np.empty(n)
    menc_disk[order] = (np.arange(n) + 1.0) / n
    menc = menc_disk + (_nfw_menc(r, nfw_ms, nfw_rs) if nfw_ms > 0 else 0.0)
    vc = np.sqrt(menc / np.maximum(r, 1e-6)) * (R / np.maximum(r, 1e-12))
    tang = np.stack([-np.sin(ph), np.cos(ph), np.zeros(n)], axis=1)
    vel = tang * vc[:, None]
    sig = sigma_frac * vc[:n_star]
    vel[:n_star] += rng.normal(0.0, 1.0, (n_star, 3)) * sig[:, None]
    ptype = np.full(n, STAR, np.uint8)
    ptype[n_star:] = GAS
    m = np.full(n, 1.0 / n)
    ep = np.full(n, eps)
    lo, hi = np.log(u_range[0]), np.log(u_range[1])
    u = np.zeros(n)
    u[n_star:] = np.exp(rng.uniform(lo, hi, n_gas))
    return _pack(pos, vel, m, ep, u, ptype)


def lattice(n_side: int, spacing: float = 1.0, mass: float = 1.0, u: float = 1.0,
            eps: float = 0.01, jitter: float = 0.0, seed: int = 0,
            origin=(0.0, 0.0, 0.0)) -> dict:
    """Uniform cubic lattice of n_side^3 gas particles; optional uniform
    jitter of +-``jitter``*spacing per axis."""
    rng = np.random.default_rng(seed)
    g = np.arange(n_side, dtype=np.float64) * spacing
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    pos = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    pos += np.asarray(origin, dtype=np.float64)
    if jitter > 0:
        pos += rng.uniform(-jitter, jitter, pos.shape) * spacing
    n = pos.shape[0]
    return _pack(pos, np.zeros((n, 3)), np.full(n, mass), np.full(n, eps),
                 np.full(n, u), np.full(n, GAS, np.uint8))


def kepler_pair(a: float = 1.0, e: float = 0.5, m1: float = 0.5, m2: float = 0.5,
                eps: float = 0.0) -> dict:
    """Two stars on a Kepler ellipse (G = 1) started at pericentre, centre of
    mass at rest at the origin."""
    mt = m1 + m2
    rp = a * (1.0 - e)
    vp = np.sqrt(mt / a * (1.0 + e) / (1.0 - e))
    x = np.array([[-m2 / mt * rp, 0.0, 0.0], [m1 / mt * rp, 0.0, 0.0]])
    v = np.array([[0.0, -m2 / mt * vp, 0.0], [0.0, m1 / mt * vp, 0.0]])
    return _pack(x, v, np.array([m1, m2]), np.array([eps, eps]), np.zeros(2),
                 np.zeros(2, np.uint8))


def uniform_random(n: int, seed: int = 0, box: float = 1.0, gas_frac: float = 1.0,
                   eps: float = 0.01, u: float = 1.0) -> dict:
    """n particles uniform in [0, box)^3 with random velocities; the last
    round(gas_frac*n) are gas.  Used for ragged-size parity cases."""
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0.0, box, (n, 3))
    vel = rng.normal(0.0, 0.1, (n, 3))
    n_gas = int(round(gas_frac * n))
    ptype = np.full(n, STAR, np.uint8)
    ptype[n - n_gas:] = GAS
    mass = rng.uniform(0.5, 1.5, n) / n
    uu = np.where(ptype == GAS, u * rng.uniform(0.5, 1.5, n), 0.0)
    return _pack(pos, vel, mass, np.full(n, eps), uu, ptype)


def subset(p: dict, idx) -> dict:
    """Particles ``idx`` of ``p`` (ids kept)."""
    return {k: np.ascontiguousarray(v[idx]) for k, v in p.items()}


def config_tiny(seed: int = 0) -> dict:
    """8,192 particles: 4,096 stars + 4,096 gas from a Plummer sphere."""
    return plummer(8192, seed=seed, n_gas=4096, u_gas=0.05, eps=0.01)


def config_disk(n: int = 1 << 20, gas_frac: float = 0.2, seed: int = 0) -> dict:
    """Disk model: 80 % stars (R_d = 1, z_d = 0.1) and 20 % gas (R_d = 2)."""
    return exp_disk(n, gas_frac=gas_frac, seed=seed)


# ---------------------------------------------------------------- SN regions
# Units of supernova regions: pc, solar mass, km/s (time unit pc/(km/s) =
# 0.97779 Myr).  u in (km/s)^2; T = (gamma - 1) mu m_H u / k_B with mu = 0.6.
PC_KMS_MYR = 0.977792221
E_SN_CODE = 1.0e51 / 1.98847e43          # 10^51 erg in Msun (km/s)^2
T_PER_U = (2.0 / 3.0) * 0.6 * 1.67262e-24 * 1.0e10 / 1.380649e-16   # K per (km/s)^2
T_SN_END = 0.1 / PC_KMS_MYR              # 0.1 Myr in code time


def _grf(rng, ng: int, slope: float, ncomp: int = 1, solenoidal: bool = False):
    """Gaussian random field(s) on an ng^3 periodic grid with power spectrum
    P(k) ~ k^slope, zero mean, unit variance per component."""
    k = np.fft.fftfreq(ng) * ng
    kz = np.fft.rfftfreq(ng) * ng
    KX, KY, KZ = np.meshgrid(k, k, kz, indexing="ij")
    k2 = KX * KX + KY * KY + KZ * KZ
    amp = np.zeros_like(k2)
    nz = k2 > 0
    amp[nz] = k2[nz] ** (slope / 4.0)
    comps = []
    for _ in range(ncomp):
        ph = rng.normal(size=k2.shape) + 1j * rng.normal(size=k2.shape)
        comps.append(ph * amp)
    if solenoidal and ncomp == 3:
        kv = (KX, KY, KZ)
        dot = sum(kv[a] * comps[a] for a in range(3))
        with np.errstate(invalid="ignore", divide="ignore"):
            for a in range(3):
                comps[a] = np.where(nz, comps[a] - kv[a] * dot / np.where(nz, k2, 1.0), 0.0)
    out = []
    for c in comps:
        f = np.fft.irfftn(c, s=(ng, ng, ng), axes=(0, 1, 2))
        f = (f - f.mean()) / (f.std() + 1e-300)
        out.append(f)
    return out


def sn_region(n: int = 100000, seed: int = 0, side: float = 60.0, sigma: float = 1.0,
              slope: float = -11.0 / 3.0, v_rms: float = 10.0, T: float = 100.0,
              grid: int = 64, m: float = 1.0) -> dict:
    """Turbulent star-forming gas around a supernova (the training setup of
    Sec. 3.3: turbulent density fields, gas particles of 1 Msun): n gas
    particles of mass m in a cube of side `side` pc centred on the origin,
    log-normal density (sigma of ln rho) from a Gaussian random field with
    P(k) ~ k^slope (Kolmogorov by default), a solenoidal velocity field with
    the same spectrum and rms v_rms km/s, uniform temperature T."""
    rng = np.random.default_rng(seed)
    (g,) = _grf(rng, grid, slope)
    rho = np.exp(sigma * g - 0.5 * sigma * sigma).ravel()
    cell = rng.choice(rho.size, size=n, p=rho / rho.sum())
    ix, iy, iz = np.unravel_index(cell, (grid, grid, grid))
    dxv = side / grid
    pos = np.stack([ix, iy, iz], axis=1) + rng.uniform(0.0, 1.0, (n, 3))
    pos = pos * dxv - 0.5 * side
    vf = _grf(rng, grid, slope, ncomp=3, solenoidal=True)
    v = np.stack([f.ravel()[cell] for f in vf], axis=1)
    v *= v_rms / np.sqrt(np.mean(np.sum(v * v, axis=1)))
    u = np.full(n, T / T_PER_U)
    return _pack(pos, v, np.full(n, m), np.full(n, 0.1), u, np.full(n, GAS, np.uint8))


def uniform_box(n_side: int, seed: int = 0, jitter: float = 0.1, rho: float = 1.0, u: float = 1e-6) -> dict:
    """Gas on a jittered cubic lattice filling [-1/2, 1/2]^3 at density rho
    (for the Sedov-Taylor blast test)."""
    n = n_side ** 3
    d = 1.0 / n_side
    p = lattice(n_side, spacing=d, mass=rho / n, u=u, eps=0.01 * d, jitter=jitter, seed=seed,
                origin=(-0.5 + 0.5 * d,) * 3)
    return p
