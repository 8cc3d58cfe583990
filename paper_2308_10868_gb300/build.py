"""Build ``libnrr.so`` (the CUDA library behind include/nrr.h) in-tree.

Every translation unit is compiled by nvcc for sm_103a only
(``-gencode arch=compute_103a,code=sm_103a``), in parallel, and linked into
``paper_2308_10868_gb300/_build/libnrr.so`` with the CUDA runtime linked
statically, so the library needs no libcudart at load time and no libcuda at
link time (the TMA descriptor encoder is fetched from the driver at run
time).
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libnrr.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC]

PLAIN_UNITS = ["nrr_api.cu", "nrr_select.cu", "nrr_spacing.cu", "nrr_boxsum.cu", "nrr_boxsum3.cu", "nrr_match_dispatch.cu", "nrr_tune.cu", "nrr_batch.cu", "nrr_serve.cu", "nrr_fem.cu"]
# (float32?, block edge, search lines per thread): uint16 cubic blocks come
# with one or two lines per thread, float32 with one
MATCH_VARIANTS = [(0, b, l) for b in (3, 5, 7, 9, 11) for l in (1, 2)] + [(1, b, 1) for b in (3, 5, 7, 9, 11)]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _units():
    units = []
    # the match variants first: they take longest
    for f32, b, lpt in MATCH_VARIANTS:
        name = f"nrr_match_f32_b{b}.o" if f32 else f"nrr_match_u16_b{b}_l{lpt}.o"
        defs = [f"-DNRR_INST_F32={f32}", f"-DNRR_INST_B={b}"] + ([] if f32 else [f"-DNRR_INST_LPT={lpt}"])
        units.append((os.path.join(CSRC, "nrr_match_inst.cu"), os.path.join(OUT_DIR, name), defs))
    for u in PLAIN_UNITS:
        units.append((os.path.join(CSRC, u), os.path.join(OUT_DIR, u.replace(".cu", ".o")), []))
    return units


def _deps_mtime() -> float:
    files = glob.glob(os.path.join(CSRC, "*")) + glob.glob(os.path.join(INCLUDE, "*.h")) + [__file__]
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile and link the library if any source is newer than it."""
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps_mtime():
        return LIB
    nvcc = _nvcc()
    units = _units()

    def compile_one(u):
        src, obj, defs = u
        cmd = [nvcc] + ARCH + FLAGS + defs + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed: " + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose and (r.stdout or r.stderr):
            sys.stderr.write(r.stdout + r.stderr)
        return obj

    workers = max(1, min(len(units), os.cpu_count() or 4))
    with cf.ThreadPoolExecutor(workers) as ex:
        objs = list(ex.map(compile_one, units))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed: " + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
