"""Python access to the CPU oracle (``nrr_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the product package.

The C source is compiled with gcc into ``oracle/_build/liboracle.so`` by
:func:`build` (``-O2 -fopenmp -ffp-contract=off``).  Every function below is
argument marshalling around the C function of the same name; the arithmetic
is all in the C file, which cites the passages of the paper it follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nrr_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, C99, OpenMP, no FMA contraction)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=c99", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        P = C.c_void_p
        i32, i64, dbl = C.c_int, C.c_int64, C.c_double
        L.oracle_num_threads.restype = i32
        L.oracle_set_threads.argtypes = [i32]
        L.oracle_block_key.restype = i64
        L.oracle_block_key.argtypes = [P, i32, i32, i32, i32, i32, i32, i32]
        L.oracle_block_key_3.restype = i64
        L.oracle_block_key_3.argtypes = [P, i32, i32, i32, i32, i32, i32, i32, i32, i32]
        L.oracle_grid_keys.restype = i64
        L.oracle_grid_keys.argtypes = [P, P, i32, i32, i32, i32, i32, P]
        L.oracle_grid_keys_3.restype = i64
        L.oracle_grid_keys_3.argtypes = [P, P, i32, i32, i32, i32, i32, i32, i32, P]
        L.oracle_n_select.restype = i64
        L.oracle_n_select.argtypes = [i64, dbl]
        L.oracle_select_blocks.restype = i64
        L.oracle_select_blocks.argtypes = [P, P, i32, i32, i32, i32, i32, dbl, P, i64, P]
        L.oracle_select_blocks_3.restype = i64
        L.oracle_select_blocks_3.argtypes = [P, P, i32, i32, i32, i32, i32, i32, i32, dbl, P, i64, P]
        L.oracle_select_blocks_spaced.restype = i64
        L.oracle_select_blocks_spaced.argtypes = [P, P, i32, i32, i32, i32, i32, dbl, i32, P, i64, P]
        for name in ("oracle_ncc_u16", "oracle_pearson_u16", "oracle_pearson_f32"):
            f = getattr(L, name)
            f.restype = i32
            f.argtypes = [P, P, i32, i32, i32, i32, i32, i32, i32, i32, i32, i32, P]
            f = getattr(L, name + "_3")
            f.restype = i32
            f.argtypes = [P, P, i32, i32, i32, i32, i32, i32, i32, i32, i32, i32, i32, i32, P]
        for name in ("oracle_match_u16", "oracle_match_f32"):
            f = getattr(L, name)
            f.restype = None
            f.argtypes = [P, P, i32, i32, i32, P, i64, i32, P, P, P, P]
            f = getattr(L, name + "_3")
            f.restype = None
            f.argtypes = [P, P, i32, i32, i32, P, i64, P, P, P, P, P]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _dims(vol: np.ndarray):
    nz, ny, nx = vol.shape
    return nx, ny, nz


def _block3(b):
    """Block edges (bx, by, bz) from an int (cubic block) or a triple."""
    if np.isscalar(b):
        return (int(b),) * 3
    bx, by, bz = (int(v) for v in b)
    return bx, by, bz


def num_threads() -> int:
    return int(lib().oracle_num_threads())


def set_threads(n: int) -> None:
    lib().oracle_set_threads(int(n))


def block_key(vol, b, x, y, z) -> int:
    """b: block edge, or (bx, by, bz)."""
    vol = np.ascontiguousarray(vol, dtype=np.uint16)
    if np.isscalar(b):
        return int(lib().oracle_block_key(_p(vol), *_dims(vol), b, x, y, z))
    return int(lib().oracle_block_key_3(_p(vol), *_dims(vol), *_block3(b), x, y, z))


def grid_keys(preop, mask, b, stride):
    preop = np.ascontiguousarray(preop, dtype=np.uint16)
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    nx, ny, nz = _dims(preop)
    g = (-(-nx // stride), -(-ny // stride), -(-nz // stride))
    keys = np.empty(g[2] * g[1] * g[0], dtype=np.int64)
    if np.isscalar(b):
        nc = lib().oracle_grid_keys(_p(preop), _p(mask), nx, ny, nz, b, stride, _p(keys))
    else:
        nc = lib().oracle_grid_keys_3(_p(preop), _p(mask), nx, ny, nz, *_block3(b), stride, _p(keys))
    return keys.reshape(g[2], g[1], g[0]), int(nc)


def n_select(n_candidates: int, frac: float) -> int:
    return int(lib().oracle_n_select(int(n_candidates), float(frac)))


def select_blocks(preop, mask, b, stride, frac):
    """b: block edge, or (bx, by, bz).  Returns (centers int32[n][3] (x,y,z)
    in raster order, n_candidates)."""
    preop = np.ascontiguousarray(preop, dtype=np.uint16)
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    nx, ny, nz = _dims(preop)
    ng = (-(-nx // stride)) * (-(-ny // stride)) * (-(-nz // stride))
    cap = max(1, ng)
    out = np.empty((cap, 3), dtype=np.int32)
    nc = C.c_int64(0)
    if np.isscalar(b):
        n = lib().oracle_select_blocks(_p(preop), _p(mask), nx, ny, nz, b, stride, float(frac), _p(out), cap,
                                       C.byref(nc))
    else:
        n = lib().oracle_select_blocks_3(_p(preop), _p(mask), nx, ny, nz, *_block3(b), stride, float(frac),
                                         _p(out), cap, C.byref(nc))
    return out[:n].copy(), int(nc.value)


def select_blocks_spaced(preop, mask, b, stride, frac, conn):
    """Selection with a connectivity pattern conn in {0, 6, 18, 26} (Sec.
    4.1).  Returns (centers int32[n][3] in raster order, n_candidates)."""
    preop = np.ascontiguousarray(preop, dtype=np.uint16)
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    nx, ny, nz = _dims(preop)
    ng = (-(-nx // stride)) * (-(-ny // stride)) * (-(-nz // stride))
    cap = max(1, ng)
    out = np.empty((cap, 3), dtype=np.int32)
    nc = C.c_int64(0)
    n = lib().oracle_select_blocks_spaced(_p(preop), _p(mask), nx, ny, nz, b, stride, float(frac), int(conn),
                                          _p(out), cap, C.byref(nc))
    return out[:n].copy(), int(nc.value)


def _ncc_at(fn, preop, intraop, b, c, d):
    nx, ny, nz = _dims(preop)
    v = C.c_double(0.0)
    if np.isscalar(b):
        ok = fn(_p(preop), _p(intraop), nx, ny, nz, b, int(c[0]), int(c[1]), int(c[2]), int(d[0]), int(d[1]),
                int(d[2]), C.byref(v))
    else:
        fn3 = getattr(lib(), fn.__name__ + "_3")
        ok = fn3(_p(preop), _p(intraop), nx, ny, nz, *_block3(b), int(c[0]), int(c[1]), int(c[2]), int(d[0]),
                 int(d[1]), int(d[2]), C.byref(v))
    return float(v.value) if ok else None


def ncc_u16(preop, intraop, b, c, d):
    """Exact-integer NCC of block at c against the shifted block at c+d."""
    preop = np.ascontiguousarray(preop, dtype=np.uint16)
    intraop = np.ascontiguousarray(intraop, dtype=np.uint16)
    return _ncc_at(lib().oracle_ncc_u16, preop, intraop, b, c, d)


def pearson_u16(preop, intraop, b, c, d):
    preop = np.ascontiguousarray(preop, dtype=np.uint16)
    intraop = np.ascontiguousarray(intraop, dtype=np.uint16)
    return _ncc_at(lib().oracle_pearson_u16, preop, intraop, b, c, d)


def pearson_f32(preop, intraop, b, c, d):
    preop = np.ascontiguousarray(preop, dtype=np.float32)
    intraop = np.ascontiguousarray(intraop, dtype=np.float32)
    return _ncc_at(lib().oracle_pearson_f32, preop, intraop, b, c, d)


def _radius3(radius):
    if np.isscalar(radius):
        return np.array([radius] * 3, dtype=np.int32)
    return np.ascontiguousarray(radius, dtype=np.int32).reshape(3)


def match(preop, intraop, centers, b, radius):
    """Exhaustive block matching.  uint16 volumes use the exact integer path,
    float32 volumes the FP64 two-pass path; b is the block edge or (bx, by,
    bz).  Returns (disp int32[n][3], ncc f64[n], valid u8[n])."""
    f32 = preop.dtype == np.float32
    dt = np.float32 if f32 else np.uint16
    preop = np.ascontiguousarray(preop, dtype=dt)
    intraop = np.ascontiguousarray(intraop, dtype=dt)
    centers = np.ascontiguousarray(centers, dtype=np.int32).reshape(-1, 3)
    n = centers.shape[0]
    disp = np.zeros((n, 3), dtype=np.int32)
    ncc = np.zeros(n, dtype=np.float64)
    valid = np.zeros(n, dtype=np.uint8)
    r = _radius3(radius)
    nx, ny, nz = _dims(preop)
    if np.isscalar(b):
        fn = lib().oracle_match_f32 if f32 else lib().oracle_match_u16
        fn(_p(preop), _p(intraop), nx, ny, nz, _p(centers), n, b, _p(r), _p(disp), _p(ncc), _p(valid))
    else:
        fn = lib().oracle_match_f32_3 if f32 else lib().oracle_match_u16_3
        bl = np.array(_block3(b), dtype=np.int32)
        fn(_p(preop), _p(intraop), nx, ny, nz, _p(centers), n, _p(bl), _p(r), _p(disp), _p(ncc), _p(valid))
    return disp, ncc, valid
