"""Python binding of ``libnrr.so`` (the C ABI in include/nrr.h).

Argument marshalling only: every step of selection and matching runs in the
library's CUDA kernels.  PyTorch supplies device memory and the current
stream.  There is no CPU fallback: if the library has not been built, or a
call is made without a CUDA device, the call raises.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libnrr.so")

NRR_OK, NRR_PENDING = 0, 1
NRR_U16, NRR_F32 = 0, 1

# Every entry point declared in include/nrr.h, with its ctypes signature.
_P = C.c_void_p
_I32 = C.c_int32


class Dims(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32)]


class Setting(C.Structure):
    _fields_ = [("block", C.c_int32), ("stride", C.c_int32), ("radius", C.c_int32 * 3), ("frac", C.c_double)]


class BatchView(C.Structure):
    _fields_ = [("centers", C.c_void_p), ("n_blocks", C.c_void_p), ("disp", C.c_void_p), ("ncc", C.c_void_p),
                ("valid", C.c_void_p), ("capacity", C.c_int32)]


class MatchShape(C.Structure):
    _fields_ = [("ctas_per_sm", C.c_int32), ("windows", C.c_int32), ("stage", C.c_int32), ("lines", C.c_int32)]


class Pair(C.Structure):
    _fields_ = [("d_preop", C.c_void_p), ("d_intraop", C.c_void_p), ("d_mask", C.c_void_p), ("dims", Dims)]


NRR_BATCH_GRAPH, NRR_BATCH_AUTOTUNE, NRR_BATCH_NO_DEDUP, NRR_BATCH_PLAIN_LAUNCH = 1, 2, 4, 8


class FemParams(C.Structure):
    _fields_ = [("grid", C.c_int32), ("young", C.c_double), ("poisson", C.c_double), ("n_rej", C.c_int32),
                ("n_int", C.c_int32), ("reject_frac", C.c_double), ("cg_tol", C.c_double), ("cg_max_iter", C.c_int32)]


class Request(C.Structure):
    _fields_ = [("d_preop", C.c_void_p), ("d_intraop", C.c_void_p), ("d_select", C.c_void_p),
                ("d_mask", C.c_void_p), ("dims", Dims), ("dtype", C.c_int), ("block", C.c_int32),
                ("stride", C.c_int32), ("radius", C.c_int32 * 3), ("frac", C.c_double)]


class Result(C.Structure):
    _fields_ = [("n_blocks", C.c_int32), ("centers", C.c_void_p), ("disp", C.c_void_p), ("ncc", C.c_void_p),
                ("valid", C.c_void_p), ("queued_s", C.c_double), ("latency_s", C.c_double)]

SIGNATURES = {
    "nrr_status_string": (C.c_char_p, [C.c_int]),
    "nrr_last_error": (C.c_char_p, []),
    "nrr_version": (_I32, []),
    "nrr_kernel_launches": (C.c_int64, []),
    "nrr_select_blocks": (C.c_int, [_P, _P, Dims, _I32, _I32, C.c_double, _P, _I32, _P, _P, _P]),
    "nrr_select_blocks_noalloc": (C.c_int, [_P, _P, Dims, _I32, _I32, C.c_double, _P, _I32, _P, _P, _P]),
    "nrr_select_blocks_spaced": (C.c_int, [_P, _P, Dims, _I32, _I32, C.c_double, _I32, _P, _I32, _P, _P, _P]),
    "nrr_boxsum_bytes": (C.c_int, [Dims, C.c_int, C.POINTER(C.c_size_t)]),
    "nrr_boxsums": (C.c_int, [_P, C.c_int, Dims, _I32, _P, _P]),
    "nrr_block_match": (C.c_int, [_P, _P, C.c_int, Dims, _P, _I32, _P, _I32, _P, _P, _P, _P, _P]),
    "nrr_block_match_bs": (C.c_int, [_P, _P, _P, C.c_int, Dims, _P, _I32, _P, _I32, _P, _P, _P, _P, _P]),
    "nrr_block_match_plain": (C.c_int, [_P, _P, _P, C.c_int, Dims, _P, _I32, _P, _I32, _P, _P, _P, _P, _P]),
    "nrr_select_blocks_aniso": (C.c_int, [_P, _P, Dims, _P, _I32, C.c_double, _P, _I32, _P, _P, _P]),
    "nrr_boxsums_aniso": (C.c_int, [_P, C.c_int, Dims, _P, _P, _P]),
    "nrr_block_match_aniso": (C.c_int, [_P, _P, C.c_int, Dims, _P, _I32, _P, _P, _P, _P, _P, _P, _P]),
    "nrr_block_match_bs_aniso": (C.c_int, [_P, _P, _P, C.c_int, Dims, _P, _I32, _P, _P, _P, _P, _P, _P, _P]),
    "nrr_device_status": (C.c_int, [_P]),
    "nrr_fem_grid": (C.c_int, [Dims, _I32, _P]),
    "nrr_fem_update": (C.c_int, [_P, Dims, _P, _P, _P, _P, _I32, _P, _P, _P, _P, _P, _P]),
    "nrr_test_set_wait": (C.c_int, [C.c_uint64, _I32]),
    "nrr_autotune_match": (C.c_int, [_P, _P, _P, C.c_int, Dims, _P, _I32, _I32, _P, _P, _P, _P, _P, _P, _P]),
    "nrr_tuning_get": (C.c_int, [C.c_int, _I32, _P, _P]),
    "nrr_tuning_set": (C.c_int, [C.c_int, _I32, _P, _I32]),
    "nrr_tuning_get_shape": (C.c_int, [C.c_int, _I32, _P, _P]),
    "nrr_tuning_set_shape": (C.c_int, [C.c_int, _I32, _P, _P]),
    "nrr_tuning_save": (C.c_int, [C.c_char_p]),
    "nrr_tuning_load": (C.c_int, [C.c_char_p]),
    "nrr_batch_create": (C.c_int, [_P, _P, _P, Dims, _P, _I32, _I32, _P]),
    "nrr_batch_create_pairs": (C.c_int, [_P, _I32, _P, _P, _I32, _I32, _P]),
    "nrr_batch_run": (C.c_int, [_P, _P]),
    "nrr_batch_view_get": (C.c_int, [_P, _I32, _P]),
    "nrr_batch_destroy": (C.c_int, [_P]),
    "nrr_server_start": (C.c_int, [_I32, C.c_size_t]),
    "nrr_server_start_ex": (C.c_int, [_I32, C.c_size_t, _I32]),
    "nrr_server_stop": (C.c_int, []),
    "nrr_submit": (C.c_int, [_P, _P]),
    "nrr_poll": (C.c_int, [C.c_uint64, _P]),
    "nrr_release": (C.c_int, [C.c_uint64]),
}

_lib = None


class NrrError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: status {status} ({detail})")
        self.status = status


def lib():
    """Load libnrr.so; raise if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2308_10868_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status: int, where: str):
    if status < 0:
        L = lib()
        detail = L.nrr_last_error().decode() or L.nrr_status_string(status).decode()
        raise NrrError(status, where, detail)
    return status


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _dims(vol: torch.Tensor) -> Dims:
    nz, ny, nx = vol.shape
    return Dims(nx, ny, nz)


def _dtype_code(vol: torch.Tensor) -> int:
    if vol.dtype == torch.float32:
        return NRR_F32
    if vol.dtype in (torch.uint16, torch.int16):  # int16 = same bits, reinterpreted
        return NRR_U16
    raise TypeError(f"volumes must be uint16 (or int16 bit-views) or float32, got {vol.dtype}")


def _cuda_contig(t: torch.Tensor, name: str):
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def radius3(radius):
    if isinstance(radius, int):
        return (radius, radius, radius)
    r = tuple(int(v) for v in radius)
    if len(r) != 3:
        raise ValueError("radius must be an int or 3 ints")
    return r


def block3(block):
    """Block edges (bx, by, bz) as a C int32[3], or None for a cubic block
    given as one int."""
    if isinstance(block, (tuple, list)):
        if len(block) != 3:
            raise ValueError("block must be an int or (bx, by, bz)")
        return (C.c_int32 * 3)(*(int(b) for b in block))
    return None


def max_selected(dims, stride: int, frac: float) -> int:
    """Upper bound on the number of blocks selection can return."""
    nx, ny, nz = dims
    ng = math.ceil(nx / stride) * math.ceil(ny / stride) * math.ceil(nz / stride)
    return int(math.floor(0.5 + ng * frac))


def select_blocks(preop: torch.Tensor, mask: torch.Tensor, block, stride: int, frac: float,
                  max_blocks: int | None = None, centers: torch.Tensor | None = None,
                  n_selected: torch.Tensor | None = None, sync: bool = True, stream=None,
                  connectivity: int = 0):
    """Variance-based block selection.  Returns the (n, 3) int32 centres
    (x, y, z) in raster order.  With ``sync=False`` nothing is read back:
    the full ``centers`` buffer and the device count ``n_selected`` are
    returned instead.  ``connectivity`` 6, 18 or 26 applies the face, edge
    or vertex spacing pattern (nrr_select_blocks_spaced).  ``block`` is the
    block edge, or (bx, by, bz) for nrr_select_blocks_aniso."""
    _cuda_contig(preop, "preop")
    _cuda_contig(mask, "mask")
    if _dtype_code(preop) != NRR_U16:
        raise TypeError("selection takes a uint16 volume")
    if mask.dtype not in (torch.uint8, torch.bool) or mask.shape != preop.shape:
        raise ValueError("mask must be uint8/bool with the volume's shape")
    dims = _dims(preop)
    if max_blocks is None:
        max_blocks = max_selected((dims.nx, dims.ny, dims.nz), stride, frac)
    if centers is None:
        centers = torch.empty((max(1, max_blocks), 3), dtype=torch.int32, device=preop.device)
    if n_selected is None:
        n_selected = torch.zeros(1, dtype=torch.int32, device=preop.device)
    h = C.c_int32(0)
    b3 = block3(block)
    if b3 is not None:
        if connectivity:
            raise ValueError("the connectivity pattern takes a cubic block")
        st = lib().nrr_select_blocks_aniso(_ptr(preop), _ptr(mask), dims, b3, stride, float(frac), _ptr(centers),
                                           max_blocks, _ptr(n_selected), C.byref(h) if sync else None,
                                           _stream(stream))
        _check(st, "nrr_select_blocks_aniso")
    elif connectivity:
        st = lib().nrr_select_blocks_spaced(_ptr(preop), _ptr(mask), dims, block, stride, float(frac),
                                            int(connectivity), _ptr(centers), max_blocks, _ptr(n_selected),
                                            C.byref(h) if sync else None, _stream(stream))
        _check(st, "nrr_select_blocks_spaced")
    else:
        st = lib().nrr_select_blocks(_ptr(preop), _ptr(mask), dims, block, stride, float(frac), _ptr(centers),
                                     max_blocks, _ptr(n_selected), C.byref(h) if sync else None, _stream(stream))
        _check(st, "nrr_select_blocks")
    if sync:
        return centers[:h.value]
    return centers, n_selected


def boxsum_bytes(vol: torch.Tensor) -> int:
    n = C.c_size_t(0)
    _check(lib().nrr_boxsum_bytes(_dims(vol), _dtype_code(vol), C.byref(n)), "nrr_boxsum_bytes")
    return int(n.value)


def boxsums(intraop: torch.Tensor, block, out: torch.Tensor | None = None, stream=None):
    """Box sums S_J, S_JJ of the reference volume for one block size (an
    opaque uint8 device buffer for :func:`block_match`); ``block`` is the
    edge or (bx, by, bz)."""
    _cuda_contig(intraop, "intraop")
    nbytes = boxsum_bytes(intraop)
    if out is None:
        out = torch.empty(nbytes + 256, dtype=torch.uint8, device=intraop.device)
    off = (-out.data_ptr()) % 256
    buf = out[off:off + nbytes]
    b3 = block3(block)
    if b3 is not None:
        _check(lib().nrr_boxsums_aniso(_ptr(intraop), _dtype_code(intraop), _dims(intraop), b3, _ptr(buf),
                                       _stream(stream)), "nrr_boxsums_aniso")
    else:
        _check(lib().nrr_boxsums(_ptr(intraop), _dtype_code(intraop), _dims(intraop), block, _ptr(buf),
                                 _stream(stream)), "nrr_boxsums")
    return buf


def block_match(preop: torch.Tensor, intraop: torch.Tensor, centers: torch.Tensor, block, radius,
                n_blocks: torch.Tensor | None = None, box: torch.Tensor | None = None, out=None, stream=None,
                plain: bool = False):
    """Exhaustive NCC block matching.  Returns (disp int32 (n,3), ncc f64 (n,),
    valid uint8 (n,)).  ``n_blocks`` is an optional device int32 count
    (<= len(centers)); ``box`` optional precomputed box sums; ``block`` the
    block edge or (bx, by, bz).  ``plain`` (cubic blocks, box sums given)
    calls nrr_block_match_plain: one CTA per block instead of persistent
    CTAs, same results."""
    for t, nm in ((preop, "preop"), (intraop, "intraop"), (centers, "centers")):
        _cuda_contig(t, nm)
    if preop.shape != intraop.shape or preop.dtype != intraop.dtype:
        raise ValueError("preop and intraop must have the same shape and dtype")
    if centers.dtype != torch.int32 or centers.dim() != 2 or centers.shape[1] != 3:
        raise ValueError("centers must be int32 (n, 3)")
    n = centers.shape[0]
    dev = preop.device
    if out is None:
        out = (torch.empty((n, 3), dtype=torch.int32, device=dev), torch.empty(n, dtype=torch.float64, device=dev),
               torch.empty(n, dtype=torch.uint8, device=dev))
    disp, ncc, valid = out
    r = (C.c_int32 * 3)(*radius3(radius))
    L = lib()
    b3 = block3(block)
    if plain and (b3 is not None or box is None):
        raise ValueError("the plain launch takes a cubic block and precomputed box sums")
    if plain:
        st = L.nrr_block_match_plain(_ptr(preop), _ptr(intraop), _ptr(box), _dtype_code(preop), _dims(preop),
                                     _ptr(centers), n, _ptr(n_blocks), block, r, _ptr(disp), _ptr(ncc), _ptr(valid),
                                     _stream(stream))
    elif b3 is not None:
        if box is None:
            st = L.nrr_block_match_aniso(_ptr(preop), _ptr(intraop), _dtype_code(preop), _dims(preop), _ptr(centers),
                                         n, _ptr(n_blocks), b3, r, _ptr(disp), _ptr(ncc), _ptr(valid), _stream(stream))
        else:
            st = L.nrr_block_match_bs_aniso(_ptr(preop), _ptr(intraop), _ptr(box), _dtype_code(preop), _dims(preop),
                                            _ptr(centers), n, _ptr(n_blocks), b3, r, _ptr(disp), _ptr(ncc),
                                            _ptr(valid), _stream(stream))
    elif box is None:
        st = L.nrr_block_match(_ptr(preop), _ptr(intraop), _dtype_code(preop), _dims(preop), _ptr(centers), n,
                               _ptr(n_blocks), block, r, _ptr(disp), _ptr(ncc), _ptr(valid), _stream(stream))
    else:
        st = L.nrr_block_match_bs(_ptr(preop), _ptr(intraop), _ptr(box), _dtype_code(preop), _dims(preop),
                                  _ptr(centers), n, _ptr(n_blocks), block, r, _ptr(disp), _ptr(ncc), _ptr(valid),
                                  _stream(stream))
    _check(st, "nrr_block_match")
    return disp, ncc, valid


def kernel_launches() -> int:
    """Kernels launched by the library so far in this process."""
    return int(lib().nrr_kernel_launches())


class _DeviceArray:
    """A raw device pointer seen through __cuda_array_interface__ (no copy)."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3, "strides": None}


def _wrap(ptr, shape, typestr, device):
    return torch.as_tensor(_DeviceArray(ptr, shape, typestr), device=device)


def autotune_match(preop, intraop, box, centers, block: int, radius, stream=None):
    """Time the match kernel at every feasible CTAs-per-SM on these inputs and
    keep the fastest for this (dtype, block, radius).  Returns (ctas, ms)."""
    n = centers.shape[0]
    out = (torch.empty((n, 3), dtype=torch.int32, device=preop.device),
           torch.empty(n, dtype=torch.float64, device=preop.device),
           torch.empty(n, dtype=torch.uint8, device=preop.device))
    r = (C.c_int32 * 3)(*radius3(radius))
    k, ms = C.c_int32(0), C.c_float(0)
    _check(lib().nrr_autotune_match(_ptr(preop), _ptr(intraop), _ptr(box), _dtype_code(preop), _dims(preop),
                                    _ptr(centers), n, block, r, _ptr(out[0]), _ptr(out[1]), _ptr(out[2]),
                                    C.byref(k), C.byref(ms), _stream(stream)), "nrr_autotune_match")
    return int(k.value), float(ms.value)


def tuning_get(dtype_code: int, block: int, radius) -> int:
    r = (C.c_int32 * 3)(*radius3(radius))
    v = C.c_int32(0)
    _check(lib().nrr_tuning_get(dtype_code, block, r, C.byref(v)), "nrr_tuning_get")
    return int(v.value)


def tuning_set(dtype_code: int, block: int, radius, ctas_per_sm: int):
    r = (C.c_int32 * 3)(*radius3(radius))
    _check(lib().nrr_tuning_set(dtype_code, block, r, ctas_per_sm), "nrr_tuning_set")


def tuning_get_shape(dtype_code: int, block: int, radius):
    """The tuned launch shape (ctas_per_sm, windows, stage, lines) of a variant."""
    r = (C.c_int32 * 3)(*radius3(radius))
    v = MatchShape()
    _check(lib().nrr_tuning_get_shape(dtype_code, block, r, C.byref(v)), "nrr_tuning_get_shape")
    return int(v.ctas_per_sm), int(v.windows), int(v.stage), int(v.lines)


def tuning_set_shape(dtype_code: int, block: int, radius, ctas_per_sm: int, windows: int = 0, stage: int = 0,
                     lines: int = 0):
    r = (C.c_int32 * 3)(*radius3(radius))
    v = MatchShape(ctas_per_sm, windows, stage, lines)
    _check(lib().nrr_tuning_set_shape(dtype_code, block, r, C.byref(v)), "nrr_tuning_set_shape")


class BatchPlan:
    """A batched parameter search (see nrr_batch_create_pairs) over one uint16
    volume pair (``preop, intraop, mask``) or, with ``pairs`` a list of
    (preop, intraop, mask) and ``pair_of`` each setting's pair index, over
    several pairs of different sizes.  ``settings`` is a list of (block,
    stride, radius, frac) with radius an int or 3 ints."""

    def __init__(self, preop=None, intraop=None, mask=None, settings=(), graph: bool = True,
                 autotune: bool = False, dedup: bool = True, pairs=None, pair_of=None, plain_launch: bool = False):
        if pairs is None:
            pairs = [(preop, intraop, mask)]
        parr = (Pair * len(pairs))()
        for k, (p, i, m) in enumerate(pairs):
            for t, nm in ((p, "preop"), (i, "intraop"), (m, "mask")):
                _cuda_contig(t, nm)
            parr[k].d_preop, parr[k].d_intraop, parr[k].d_mask = _ptr(p), _ptr(i), _ptr(m)
            parr[k].dims = _dims(p)
        self._keep = list(pairs)  # the plan holds their addresses
        self.device = pairs[0][0].device
        arr = (Setting * len(settings))()
        for i, (b, st, r, f) in enumerate(settings):
            arr[i].block, arr[i].stride, arr[i].frac = b, st, float(f)
            arr[i].radius[:] = list(radius3(r))
        pof = None
        if pair_of is not None:
            if len(pair_of) != len(settings):
                raise ValueError("pair_of needs one pair index per setting")
            pof = (C.c_int32 * len(settings))(*[int(x) for x in pair_of])
        self.settings = list(settings)
        flags = ((NRR_BATCH_GRAPH if graph else 0) | (NRR_BATCH_AUTOTUNE if autotune else 0) |
                 (0 if dedup else NRR_BATCH_NO_DEDUP) | (NRR_BATCH_PLAIN_LAUNCH if plain_launch else 0))
        h = C.c_void_p(0)
        _check(lib().nrr_batch_create_pairs(parr, len(pairs), arr, pof, len(settings), flags, C.byref(h)),
               "nrr_batch_create_pairs")
        self._h = h

    def run(self, stream=None):
        _check(lib().nrr_batch_run(self._h, _stream(stream)), "nrr_batch_run")

    def view(self, s: int):
        """Device tensors (no copy) of setting s: n (1,), centres, disp, ncc,
        valid, each with the plan's capacity."""
        v = BatchView()
        _check(lib().nrr_batch_view_get(self._h, s, C.byref(v)), "nrr_batch_view_get")
        cap, dev = v.capacity, self.device
        return (_wrap(v.n_blocks, (1,), "<i4", dev), _wrap(v.centers, (cap, 3), "<i4", dev),
                _wrap(v.disp, (cap, 3), "<i4", dev), _wrap(v.ncc, (cap,), "<f8", dev), _wrap(v.valid, (cap,), "|u1", dev))

    def result(self, s: int):
        """Copies of setting s's results, trimmed to its count (synchronises)."""
        n, c, d, x, v = self.view(s)
        k = int(n.item())
        return c[:k].clone(), d[:k].clone(), x[:k].clone(), v[:k].clone()

    def close(self):
        if self._h:
            lib().nrr_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Registration server with continuous batching (see nrr_server_start).
    Volumes passed to submit() must stay alive until the request is done."""

    def __init__(self, slots: int = 8, reserve_bytes: int = 1 << 30, max_group: int = 16):
        _check(lib().nrr_server_start_ex(slots, reserve_bytes, max_group), "nrr_server_start_ex")
        self._live = {}

    def submit(self, preop, intraop, mask, block: int, stride: int, radius, frac: float, select=None) -> int:
        for t, nm in ((preop, "preop"), (intraop, "intraop"), (mask, "mask")):
            _cuda_contig(t, nm)
        sel = preop if select is None else select
        if _dtype_code(sel) != NRR_U16:
            raise TypeError("selection needs a uint16 volume (pass select= for float32 requests)")
        r = Request()
        r.d_preop, r.d_intraop, r.d_select, r.d_mask = (preop.data_ptr(), intraop.data_ptr(), sel.data_ptr(),
                                                         mask.data_ptr())
        r.dims, r.dtype, r.block, r.stride, r.frac = _dims(preop), _dtype_code(preop), block, stride, float(frac)
        r.radius[:] = list(radius3(radius))
        t = C.c_uint64(0)
        _check(lib().nrr_submit(C.byref(r), C.byref(t)), "nrr_submit")
        self._live[t.value] = (preop, intraop, mask, sel)
        return int(t.value)

    def poll(self, ticket: int):
        """None while pending; else dict with device tensors (views, valid
        until release) and latencies.  Raises NrrError if the request failed."""
        res = Result()
        st = lib().nrr_poll(ticket, C.byref(res))
        if st == NRR_PENDING:
            return None
        _check(st, "nrr_poll")
        n = res.n_blocks
        dev = self._live[ticket][0].device if ticket in self._live else torch.device("cuda")
        wrap = (lambda p, sh, ty: _wrap(p, sh, ty, dev)) if n > 0 else (lambda p, sh, ty: torch.empty(
            sh, dtype={"<i4": torch.int32, "<f8": torch.float64, "|u1": torch.uint8}[ty], device=dev))
        return {"n": n, "centers": wrap(res.centers, (n, 3), "<i4"), "disp": wrap(res.disp, (n, 3), "<i4"),
                "ncc": wrap(res.ncc, (n,), "<f8"), "valid": wrap(res.valid, (n,), "|u1"),
                "queued_s": res.queued_s, "latency_s": res.latency_s}

    def release(self, ticket: int):
        _check(lib().nrr_release(ticket), "nrr_release")
        self._live.pop(ticket, None)

    def stop(self):
        lib().nrr_server_stop()
        self._live.clear()


def fem_grid(dims, grid: int):
    """Vertex counts (Nx, Ny, Nz) of the finite-element grid of a volume of
    dims (nx, ny, nz) with vertices every ``grid`` voxels."""
    out = (C.c_int32 * 3)()
    _check(lib().nrr_fem_grid(Dims(*dims), int(grid), out), "nrr_fem_grid")
    return tuple(int(v) for v in out)


def fem_update(mask: torch.Tensor, centers: torch.Tensor, disp: torch.Tensor, ncc: torch.Tensor,
               valid: torch.Tensor, grid: int = 4, young: float = 1.0, poisson: float = 0.45, n_rej: int = 2,
               n_int: int = 1, reject_frac: float = 0.05, cg_tol: float = 1e-10, cg_max_iter: int = 20000,
               stream=None):
    """The robust finite-element update on the block matches
    (nrr_fem_update).  ``mask`` uint8 (nz, ny, nx); ``centers`` int32 (n, 3),
    ``disp`` int32 (n, 3), ``ncc`` float64 (n,), ``valid`` uint8 (n,), all on
    the device.  Returns (U float64 (Nz, Ny, Nx, 3), s float64 (n,),
    rejected_step int32 (n,), the solves' iteration counts)."""
    _cuda_contig(mask, "mask")
    if mask.dtype != torch.uint8 or mask.dim() != 3:
        raise ValueError("mask must be uint8 (nz, ny, nx)")
    n = centers.shape[0]
    for t, nm, dt in ((centers, "centers", torch.int32), (disp, "disp", torch.int32), (ncc, "ncc", torch.float64),
                      (valid, "valid", torch.uint8)):
        _cuda_contig(t, nm)
        if t.dtype != dt or t.shape[0] != n:
            raise ValueError(f"{nm} must be {dt} with {n} rows")
    nz, ny, nx = mask.shape
    Nx, Ny, Nz = fem_grid((nx, ny, nz), grid)
    dev = mask.device
    U = torch.empty((Nz, Ny, Nx, 3), dtype=torch.float64, device=dev)
    s = torch.empty(n, dtype=torch.float64, device=dev)
    step = torch.empty(n, dtype=torch.int32, device=dev)
    iters = (C.c_int32 * max(1, n_rej + n_int))()
    P = FemParams(grid, young, poisson, n_rej, n_int, reject_frac, cg_tol, cg_max_iter)
    _check(lib().nrr_fem_update(_ptr(mask), Dims(nx, ny, nz), _ptr(centers), _ptr(disp), _ptr(ncc), _ptr(valid), n,
                                C.byref(P), _ptr(U), _ptr(s), _ptr(step), iters, _stream(stream)), "nrr_fem_update")
    return U, s, step, [int(v) for v in iters][: n_rej + n_int]


def device_status(stream=None) -> int:
    """Wait for the stream; raise if a kernel reported a timeout or failed
    check since the last call."""
    return _check(lib().nrr_device_status(_stream(stream)), "nrr_device_status")


def test_set_wait(limit_ns: int, missing_arrivals: int = 0):
    """Test hook (nrr_test_set_wait): the limit of later launches' bounded
    device waits (0 = the 2 s default) and arrivals that never come at the
    pattern selection's grid barriers (0 = none)."""
    _check(lib().nrr_test_set_wait(int(limit_ns), int(missing_arrivals)), "nrr_test_set_wait")


def to_device_u16(a, device="cuda") -> torch.Tensor:
    """uint16 numpy array -> CUDA tensor holding the same bits."""
    import numpy as np

    a = np.ascontiguousarray(a, dtype=np.uint16)
    return torch.from_numpy(a.view(np.int16)).to(device)
