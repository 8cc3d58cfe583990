"""Seeded synthetic inputs for the block-matching path.

This module only *makes inputs*: smooth MRI-like phantoms, a known smooth
displacement field, the warped and noisy "intra-operative" volume and an
ellipsoidal intracranial mask.  It contains none of the arithmetic of the
method itself (no block variance, no NCC, no search), so both the CUDA path
and the CPU oracle can take their inputs from here without sharing any of the
computation being checked.

The paper's clinical MRI (pre-operative and intra-operative scans of brain
tumour patients, with an intracranial-cavity mask; Sec. 3 and Sec. 4.1) is
not available; these phantoms stand in for it with the same layout and the
block counts the paper quotes (order 1e4..1e5 selected blocks, Sec. 4.1).

Layout of every volume: C-contiguous ``[nz][ny][nx]`` (x fastest).  ``dims``
is always given as ``(nx, ny, nz)``.
"""
from __future__ import annotations

import functools
from dataclasses import dataclass

import numpy as np

SEED_BASE = 230810868


@dataclass(frozen=True)
class Workload:
    """One synthetic registration workload (volume recipe + search settings)."""

    name: str
    dims: tuple  # (nx, ny, nz)
    umax: float  # max |u| of the displacement field, voxels
    noise: float  # sigma of additive Gaussian noise
    block: int  # full odd block edge b
    stride: int  # candidate grid stride
    frac: float  # selection fraction F_s
    radius: int  # isotropic search radius R
    seed_index: int


# The five workloads: a small single registration, the clinical-size single
# registration, the batched parameter search (on the clinical-size pair), the
# served stream, and the high-resolution variant.
WORKLOADS = {
    "small": Workload("small_64x64x48_b7_r4_f10", (64, 64, 48), 4.0, 20.0, 7, 2, 0.10, 4, 0),
    "clinical": Workload("clinical_256x256x124_b7_r5_f5", (256, 256, 124), 8.0, 30.0, 7, 2, 0.05, 5, 1),
    "highres": Workload("highres_512x512x256_b9_r7_f5_s3", (512, 512, 256), 12.0, 30.0, 9, 3, 0.05, 7, 4),
}

SERVE_SIZES = ((128, 128, 64), (192, 192, 96), (256, 256, 160))


def rng_for(seed_index: int, salt: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + seed_index + 1000 * salt))


def _g1(n: int, c: float, s: float) -> np.ndarray:
    x = np.arange(n, dtype=np.float64)
    return np.exp(-0.5 * ((x - c) / s) ** 2)


_SLAB = 16  # z-planes per slab when evaluating separable sums


def phantom_f64(dims, rng, n_gauss=40, sigma=(3.0, 10.0), amp=(0.0, 4095.0)) -> np.ndarray:
    """Sum of ``n_gauss`` isotropic 3-D Gaussians, evaluated in FP64."""
    nx, ny, nz = dims
    params = []
    for _ in range(n_gauss):
        cx, cy, cz = rng.uniform(0, nx), rng.uniform(0, ny), rng.uniform(0, nz)
        s = rng.uniform(*sigma)
        a = rng.uniform(*amp)
        params.append((cx, cy, cz, s, a))
    vol = np.zeros((nz, ny, nx), dtype=np.float64)
    for cx, cy, cz, s, a in params:
        gyx = a * np.multiply.outer(_g1(ny, cy, s), _g1(nx, cx, s))
        gz = _g1(nz, cz, s)
        for z0 in range(0, nz, _SLAB):
            z1 = min(nz, z0 + _SLAB)
            vol[z0:z1] += gz[z0:z1, None, None] * gyx[None]
    return vol


def _field_params(dims, rng, n_bumps=8):
    nx, ny, nz = dims
    m = float(min(dims))
    bumps = []
    for _ in range(n_bumps):
        c = (rng.uniform(0, nx), rng.uniform(0, ny), rng.uniform(0, nz))
        s = rng.uniform(0.15, 0.35) * m
        d = rng.standard_normal(3)
        d = d / np.linalg.norm(d)
        bumps.append((c, s, d))
    return bumps


def _field_slab(dims, bumps, z0, z1):
    """Unscaled displacement field (ux, uy, uz) on planes z0..z1-1."""
    nx, ny, nz = dims
    u = np.zeros((3, z1 - z0, ny, nx), dtype=np.float64)
    for c, s, d in bumps:
        g = np.multiply.outer(_g1(nz, c[2], s)[z0:z1], np.multiply.outer(_g1(ny, c[1], s), _g1(nx, c[0], s)))
        for k in range(3):
            u[k] += d[k] * g
    return u


def _trilinear_zero(vol: np.ndarray, px, py, pz) -> np.ndarray:
    """Sample ``vol`` at real coordinates with trilinear weights; 0 outside."""
    nz, ny, nx = vol.shape
    pad = np.zeros((nz + 2, ny + 2, nx + 2), dtype=vol.dtype)
    pad[1:-1, 1:-1, 1:-1] = vol
    x0 = np.floor(px)
    y0 = np.floor(py)
    z0 = np.floor(pz)
    fx, fy, fz = px - x0, py - y0, pz - z0
    out = np.zeros(px.shape, dtype=np.float64)
    for dz in (0, 1):
        wz = fz if dz else 1.0 - fz
        iz = np.clip(z0 + dz, -1, nz).astype(np.int64) + 1
        for dy in (0, 1):
            wy = fy if dy else 1.0 - fy
            iy = np.clip(y0 + dy, -1, ny).astype(np.int64) + 1
            for dx in (0, 1):
                wx = fx if dx else 1.0 - fx
                ix = np.clip(x0 + dx, -1, nx).astype(np.int64) + 1
                out += wz * wy * wx * pad[iz, iy, ix]
    return out


def to_u16(v: np.ndarray) -> np.ndarray:
    return np.clip(np.rint(v), 0, 65535).astype(np.uint16)


def ellipsoid_mask(dims, frac=0.45) -> np.ndarray:
    """Centered ellipsoid with semi-axes ``frac * (nx, ny, nz)``; u8 0/1."""
    nx, ny, nz = dims
    z, y, x = np.ogrid[0:nz, 0:ny, 0:nx]
    r2 = (((x - (nx - 1) / 2) / (frac * nx)) ** 2 + ((y - (ny - 1) / 2) / (frac * ny)) ** 2
          + ((z - (nz - 1) / 2) / (frac * nz)) ** 2)
    return (r2 <= 1.0).astype(np.uint8)


def make_pair(dims, umax: float, noise: float, seed_index: int, n_gauss: int = 40):
    """Return ``(preop u16, intraop u16, mask u8, scale)``.

    intraop(x) = preop_f64(x - u(x)) (trilinear, 0 outside) + N(0, noise^2),
    rounded to nearest and clamped to the uint16 range; ``u`` is a sum of 8
    Gaussian vector bumps scaled so that max |u|_2 == umax.
    """
    rng = rng_for(seed_index)
    nx, ny, nz = dims
    pre = phantom_f64(dims, rng, n_gauss)
    bumps = _field_params(dims, rng)
    # pass 1: max |u|
    umax_raw = 0.0
    for z0 in range(0, nz, _SLAB):
        u = _field_slab(dims, bumps, z0, min(nz, z0 + _SLAB))
        umax_raw = max(umax_raw, float(np.sqrt((u * u).sum(axis=0)).max()))
    scale = umax / umax_raw
    # pass 2: warp + noise, slab by slab
    intra = np.empty((nz, ny, nx), dtype=np.uint16)
    xs = np.arange(nx, dtype=np.float64)[None, None, :]
    ys = np.arange(ny, dtype=np.float64)[None, :, None]
    for z0 in range(0, nz, _SLAB):
        z1 = min(nz, z0 + _SLAB)
        u = _field_slab(dims, bumps, z0, z1) * scale
        zs = np.arange(z0, z1, dtype=np.float64)[:, None, None]
        px = np.broadcast_to(xs, u[0].shape) - u[0]
        py = np.broadcast_to(ys, u[0].shape) - u[1]
        pz = np.broadcast_to(zs, u[0].shape) - u[2]
        w = _trilinear_zero(pre, px, py, pz)
        w += rng.normal(0.0, noise, size=w.shape)
        intra[z0:z1] = to_u16(w)
    return to_u16(pre), intra, ellipsoid_mask(dims), scale


@functools.lru_cache(maxsize=8)
def workload_pair(key: str):
    """Cached ``(preop, intraop, mask)`` for one of ``WORKLOADS``."""
    w = WORKLOADS[key]
    pre, intra, mask, _ = make_pair(w.dims, w.umax, w.noise, w.seed_index)
    for a in (pre, intra, mask):
        a.setflags(write=False)
    return pre, intra, mask


@functools.lru_cache(maxsize=8)
def serve_pair(size_index: int, variant: int):
    """Volume pair for the served stream: one of SERVE_SIZES, phantom as the
    clinical workload (field max 8 voxels, noise sigma 30)."""
    dims = SERVE_SIZES[size_index]
    pre, intra, mask, _ = make_pair(dims, 8.0, 30.0, 100 + 10 * size_index + variant)
    for a in (pre, intra, mask):
        a.setflags(write=False)
    return pre, intra, mask


def as_f32(u16: np.ndarray) -> np.ndarray:
    """Float32 intensities in [0, 1] made from a uint16 volume: u / 65535."""
    return (u16.astype(np.float32) / np.float32(65535.0)).astype(np.float32)


def translate(vol: np.ndarray, t) -> np.ndarray:
    """out(x) = vol(x - t) for integer t = (tx, ty, tz); 0 where x - t leaves
    the volume."""
    tx, ty, tz = (int(v) for v in t)
    out = np.zeros_like(vol)
    nz, ny, nx = vol.shape

    def rng_(n, s):
        return (max(0, s), min(n, n + s)), (max(0, -s), min(n, n - s))

    (dz0, dz1), (sz0, sz1) = rng_(nz, tz)
    (dy0, dy1), (sy0, sy1) = rng_(ny, ty)
    (dx0, dx1), (sx0, sx1) = rng_(nx, tx)
    out[dz0:dz1, dy0:dy1, dx0:dx1] = vol[sz0:sz1, sy0:sy1, sx0:sx1]
    return out


def random_u16(dims, seed: int, hi: int = 65536) -> np.ndarray:
    """Uniform random uint16 volume (platform-independent integer draws)."""
    nx, ny, nz = dims
    g = np.random.Generator(np.random.PCG64(SEED_BASE + 7919 * seed))
    return g.integers(0, hi, size=(nz, ny, nx), dtype=np.uint16)


def parameter_settings(n: int = 64, seed: int = SEED_BASE):
    """The batched parameter search: ``n`` settings drawn without replacement
    from block {5,7,9} x radius {3..7} x fraction {2,4,6,8,10}% (stride 2)."""
    combos = [(b, r, f) for b in (5, 7, 9) for r in (3, 4, 5, 6, 7) for f in (0.02, 0.04, 0.06, 0.08, 0.10)]
    g = np.random.Generator(np.random.PCG64(seed))
    idx = g.choice(len(combos), size=n, replace=False)
    return [combos[int(i)] for i in idx]


def poisson_arrivals(n: int, rate: float, seed: int = SEED_BASE + 3):
    """Arrival times (s) of a Poisson stream with mean ``rate`` requests/s and
    per-request (size_index, variant, block, radius, frac) drawn alongside."""
    g = np.random.Generator(np.random.PCG64(seed))
    gaps = g.exponential(1.0 / rate, size=n)
    t = np.cumsum(gaps) - gaps[0]
    combos = [(b, r, f) for b in (5, 7, 9) for r in (3, 4, 5, 6, 7) for f in (0.02, 0.04, 0.06, 0.08, 0.10)]
    reqs = []
    for i in range(n):
        s = int(g.integers(0, len(SERVE_SIZES)))
        b, r, f = combos[int(g.integers(0, len(combos)))]
        reqs.append((float(t[i]), s, b, r, f))
    return reqs
