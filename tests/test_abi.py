"""The C-ABI library builds, loads without a GPU, exports every entry point
declared in include/nrr.h and rejects bad arguments before touching the
device (CPU only: no compute call is made)."""
import ctypes as C
import os
import re

import pytest

from paper_2308_10868_gb300 import build as nbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    nbuild.build()
    from paper_2308_10868_gb300 import nrr

    return nrr.lib()


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            text = open(os.path.join(ROOT, "include", f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(nrr_[a-z0-9_]+)\s*\(", text))
    return names


def test_every_declared_symbol_is_exported(L):
    from paper_2308_10868_gb300 import nrr

    names = _declared()
    assert {"nrr_select_blocks", "nrr_block_match", "nrr_status_string"} <= names
    for n in sorted(names):
        assert hasattr(L, n), f"{n} not exported"
    # the binding declares a signature for every entry point
    assert names <= set(nrr.SIGNATURES), sorted(names - set(nrr.SIGNATURES))


def test_status_strings_and_version(L):
    assert L.nrr_status_string(0) == b"ok"
    assert L.nrr_status_string(-1) == b"invalid argument"
    assert L.nrr_status_string(12345) == b"unknown status"
    assert L.nrr_version() >= 100


def test_argument_checks_need_no_device(L):
    from paper_2308_10868_gb300 import nrr

    d = nrr.Dims(64, 64, 48)
    n = C.c_size_t(0)
    assert L.nrr_boxsum_bytes(d, 0, C.byref(n)) == 0 and n.value >= 64 * 64 * 48 * 8
    assert L.nrr_boxsum_bytes(nrr.Dims(63, 64, 48), 0, C.byref(n)) == -1  # nx*2 not a multiple of 16
    assert b"multiple of 16" in L.nrr_last_error()
    assert L.nrr_boxsum_bytes(nrr.Dims(64, 64, 48), 7, C.byref(n)) == -1  # bad dtype
    fake = C.c_void_p(1 << 20)
    # even block size, radius out of range, bad fraction, bad stride
    assert L.nrr_select_blocks(fake, fake, d, 6, 2, 0.1, fake, 10, None, None, None) == -1
    assert L.nrr_select_blocks(fake, fake, d, 7, 0, 0.1, fake, 10, None, None, None) == -1
    assert L.nrr_select_blocks(fake, fake, d, 7, 2, 0.0, fake, 10, None, None, None) == -1
    assert L.nrr_select_blocks(fake, fake, d, 7, 2, 1.5, fake, 10, None, None, None) == -1
    # connectivity pattern must be 0, 6, 18 or 26
    for conn in (1, 8, 27, -6):
        assert L.nrr_select_blocks_spaced(fake, fake, d, 7, 2, 0.1, conn, fake, 10, None, None, None) == -1
        assert b"connectivity" in L.nrr_last_error()
    assert L.nrr_select_blocks_spaced(fake, fake, d, 6, 2, 0.1, 6, fake, 10, None, None, None) == -1
    for bad in ((4, 16, 4), (-1, 3, 3), (3, 3, 99)):  # radius 0..15 per axis
        r = (C.c_int32 * 3)(*bad)
        assert L.nrr_block_match(fake, fake, 0, d, fake, 5, None, 7, r, fake, fake, fake, None) == -1
        assert b"radius" in L.nrr_last_error()
    r = (C.c_int32 * 3)(4, 4, 4)
    assert L.nrr_block_match(fake, fake, 0, d, fake, 5, None, 13, r, fake, fake, fake, None) == -1
    assert L.nrr_block_match(None, fake, 0, d, fake, 5, None, 7, r, fake, fake, fake, None) == -1
    assert L.nrr_block_match(fake, fake, 0, nrr.Dims(64, 64, 4), fake, 5, None, 7, r, fake, fake, fake, None) == -1


def test_binding_refuses_cpu_tensors():
    import torch

    from paper_2308_10868_gb300 import nrr

    v = torch.zeros((8, 8, 8), dtype=torch.int16)
    with pytest.raises(ValueError):
        nrr.select_blocks(v, torch.zeros((8, 8, 8), dtype=torch.uint8), 3, 2, 0.1)


def test_serving_and_batch_arguments_need_no_device(L):
    import ctypes as C

    from paper_2308_10868_gb300 import nrr

    r = nrr.Request()
    t = C.c_uint64(0)
    assert L.nrr_submit(C.byref(r), C.byref(t)) == -1  # block 0 is invalid
    r.d_preop = r.d_intraop = r.d_select = r.d_mask = 1 << 20
    r.dims, r.dtype, r.block, r.stride, r.frac = nrr.Dims(64, 64, 48), 0, 7, 2, 0.1
    r.radius[:] = [3, 3, 3]
    assert L.nrr_submit(C.byref(r), C.byref(t)) == -1  # no server running
    assert b"no server" in L.nrr_last_error()
    assert L.nrr_poll(1, None) == -1 and L.nrr_release(1) == -1
    assert L.nrr_server_start(0, 0) == -1
    assert L.nrr_server_start_ex(1, 0, 0) == -1 and L.nrr_server_start_ex(1, 0, 17) == -1
    assert b"max_group" in L.nrr_last_error()
    s = (nrr.Setting * 1)()
    s[0].block, s[0].stride, s[0].frac = 6, 2, 0.1
    h = C.c_void_p(0)
    assert L.nrr_batch_create(1 << 20, 1 << 20, 1 << 20, nrr.Dims(64, 64, 48), s, 1, 0, C.byref(h)) == -1
    assert b"setting 0" in L.nrr_last_error()
    assert L.nrr_batch_run(None, None) == -1
    pr = (nrr.Pair * 2)()
    for k in range(2):
        pr[k].d_preop = pr[k].d_intraop = pr[k].d_mask = 1 << 20
        pr[k].dims = nrr.Dims(64, 64, 48)
    s[0].block = 7
    s[0].stride, s[0].frac = 2, 0.1
    bad = (C.c_int32 * 1)(2)  # pair index out of range
    assert L.nrr_batch_create_pairs(pr, 2, s, bad, 1, 0, C.byref(h)) == -1
    assert b"pair index" in L.nrr_last_error()
    pr[1].d_mask = None
    assert L.nrr_batch_create_pairs(pr, 2, s, None, 1, 0, C.byref(h)) == -1
    assert b"pair 1" in L.nrr_last_error()
    pr[1].d_mask, pr[1].dims = 1 << 20, nrr.Dims(60, 64, 48)  # nx * 2 not a multiple of 16
    one = (C.c_int32 * 1)(1)
    assert L.nrr_batch_create_pairs(pr, 2, s, one, 1, 0, C.byref(h)) == -1
    assert b"setting 0" in L.nrr_last_error()
    assert L.nrr_batch_create_pairs(None, 0, s, None, 1, 0, C.byref(h)) == -1


def test_tuning_shape_entries_need_no_device(L):
    import ctypes as C

    from paper_2308_10868_gb300 import nrr

    r = (C.c_int32 * 3)(3, 3, 3)
    for bad in ((65, 0, 0), (-1, 0, 0), (1, 3, 0), (1, 0, 3), (1, -1, 0), (1, 0, 0, 3), (1, 0, 0, -1)):
        sh = nrr.MatchShape(*bad)
        assert L.nrr_tuning_set_shape(0, 7, r, C.byref(sh)) == -1
    assert L.nrr_tuning_set_shape(0, 7, r, None) == -1
    assert L.nrr_tuning_get_shape(0, 7, r, None) == -1
    sh = nrr.MatchShape(3, 1, 2, 1)
    assert L.nrr_tuning_set_shape(0, 7, r, C.byref(sh)) == 0
    got = nrr.MatchShape()
    assert L.nrr_tuning_get_shape(0, 7, r, C.byref(got)) == 0
    assert (got.ctas_per_sm, got.windows, got.stage, got.lines) == (3, 1, 2, 1)
    k = C.c_int32(0)
    assert L.nrr_tuning_get(0, 7, r, C.byref(k)) == 0 and k.value == 3
    assert L.nrr_tuning_set(0, 7, r, 0) == 0  # ctas only: the other fields back to "by occupancy"
    assert L.nrr_tuning_get_shape(0, 7, r, C.byref(got)) == 0
    assert (got.ctas_per_sm, got.windows, got.stage, got.lines) == (0, 0, 0, 0)


def test_tuning_table_save_and_load(L, tmp_path):
    import ctypes as C

    from paper_2308_10868_gb300 import nrr

    r = (C.c_int32 * 3)(5, 4, 3)
    assert L.nrr_tuning_set_shape(0, 9, r, C.byref(nrr.MatchShape(2, 2, 1, 2))) == 0
    path = str(tmp_path / "tune.txt")
    assert L.nrr_tuning_save(path.encode()) == 0
    text = open(path).read()
    assert "ctas_per_sm windows stage lines" in text
    assert L.nrr_tuning_set_shape(0, 9, r, C.byref(nrr.MatchShape(0, 0, 0))) == 0
    assert L.nrr_tuning_load(path.encode()) == 0
    got = nrr.MatchShape()
    assert L.nrr_tuning_get_shape(0, 9, r, C.byref(got)) == 0
    assert (got.ctas_per_sm, got.windows, got.stage, got.lines) == (2, 2, 1, 2)
    # a line of the older form (CTAs per SM only) leaves the other fields by occupancy
    old = tmp_path / "old.txt"
    dev = text.splitlines()[1].split()[0]
    old.write_text(f"# device dtype block rx ry rz ctas_per_sm\n{dev} 0 9 5 4 3 4\n")
    assert L.nrr_tuning_load(str(old).encode()) == 0
    assert L.nrr_tuning_get_shape(0, 9, r, C.byref(got)) == 0
    assert (got.ctas_per_sm, got.windows, got.stage, got.lines) == (4, 0, 0, 0)
    # and a line without the lines per thread leaves them by x-shift count
    old.write_text(f"# device dtype block rx ry rz ctas_per_sm windows stage\n{dev} 0 9 5 4 3 3 1 2\n")
    assert L.nrr_tuning_load(str(old).encode()) == 0
    assert L.nrr_tuning_get_shape(0, 9, r, C.byref(got)) == 0
    assert (got.ctas_per_sm, got.windows, got.stage, got.lines) == (3, 1, 2, 0)
    assert L.nrr_tuning_set_shape(0, 9, r, C.byref(nrr.MatchShape(0, 0, 0))) == 0


def test_fem_entries_need_no_device(L):
    # vertex counts of the finite-element grid, and the update's argument
    # checks, which return before any device work
    from paper_2308_10868_gb300 import nrr

    out = (C.c_int32 * 3)()
    assert L.nrr_fem_grid(nrr.Dims(256, 256, 124), 4, out) == 0 and tuple(out) == (65, 65, 32)
    assert L.nrr_fem_grid(nrr.Dims(30, 26, 19), 4, out) == 0 and tuple(out) == (9, 8, 6)
    assert L.nrr_fem_grid(nrr.Dims(30, 26, 19), 1, out) == -1
    assert L.nrr_fem_grid(nrr.Dims(1, 26, 19), 4, out) == -1
    assert L.nrr_fem_grid(nrr.Dims(30, 26, 19), 4, None) == -1
    good = dict(grid=4, young=1.0, poisson=0.45, n_rej=1, n_int=1, reject_frac=0.05, cg_tol=1e-10, cg_max_iter=100)
    fake = C.c_void_p(0x1000)  # never dereferenced: every call below fails its checks first
    d = nrr.Dims(32, 32, 32)
    for bad in (dict(grid=1), dict(young=0.0), dict(young=float("nan")), dict(poisson=0.5), dict(poisson=-0.1),
                dict(n_rej=-1), dict(n_int=1001), dict(reject_frac=-0.01), dict(reject_frac=1.01),
                dict(cg_tol=0.0), dict(cg_max_iter=0)):
        P = nrr.FemParams(**{**good, **bad})
        assert L.nrr_fem_update(fake, d, fake, fake, fake, fake, 10, C.byref(P), fake, fake, fake, None, None) == -1, bad
    P = nrr.FemParams(**good)
    assert L.nrr_fem_update(fake, d, fake, fake, fake, fake, 10, None, fake, fake, fake, None, None) == -1
    assert L.nrr_fem_update(fake, d, fake, fake, fake, fake, -1, C.byref(P), fake, fake, fake, None, None) == -1
    assert L.nrr_fem_update(fake, d, fake, fake, fake, fake, (1 << 19) + 1, C.byref(P), fake, fake, fake, None, None) == -1
    assert L.nrr_fem_update(fake, d, None, fake, fake, fake, 10, C.byref(P), fake, fake, fake, None, None) == -1
    assert L.nrr_fem_update(None, d, fake, fake, fake, fake, 10, C.byref(P), fake, fake, fake, None, None) == -1
    assert L.nrr_fem_update(fake, nrr.Dims(32, 1, 32), fake, fake, fake, fake, 10, C.byref(P), fake, fake, fake, None,
                            None) == -1
