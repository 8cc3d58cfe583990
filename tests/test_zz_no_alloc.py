"""The allocation-free selection entry point (GPU).

nrr_select_blocks_noalloc is for callers that cannot allocate device memory
when they call in (memory budget fixed at start-up, no allocation allowed in
the calling context).  Called through the C ABI, it must give exactly what
nrr_select_blocks gives, on two calls in a row (the second sees whatever the
first left in the shared scratch array), and refuse a grid too large for its
fixed scratch with a clear error.  This file is collected last so that a
run stopping at the first failure has already run every other test; it also
passes on its own in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2308_10868_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nrr():
    from paper_2308_10868_gb300 import build as nbuild

    nbuild.build()
    from paper_2308_10868_gb300 import nrr as m

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return m


def _call(nrr, fn, dpre, dmask, block, stride, frac, cap):
    centers = torch.full((cap, 3), -1, dtype=torch.int32, device="cuda")
    n_dev = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    n_host = C.c_int32(-1)
    nz, ny, nx = dpre.shape
    st = fn(C.c_void_p(dpre.data_ptr()), C.c_void_p(dmask.data_ptr()), nrr.Dims(nx, ny, nz), block, stride,
            float(frac), C.c_void_p(centers.data_ptr()), cap, C.c_void_p(n_dev.data_ptr()), C.byref(n_host),
            C.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st, n_host.value, int(n_dev.item()), centers.cpu().numpy()


@pytest.mark.parametrize("key,block,stride,frac", [("clinical", 7, 2, 0.05), ("small", 5, 2, 0.10)])
def test_noalloc_equals_allocating_selection_twice(nrr, key, block, stride, frac):
    L = nrr.lib()
    pre, _, mask = synth.workload_pair(key)
    dpre, dmask = nrr.to_device_u16(pre), torch.from_numpy(mask).cuda()
    cap = nrr.max_selected(pre.shape[::-1], stride, frac)
    st, n_ref, nd_ref, c_ref = _call(nrr, L.nrr_select_blocks, dpre, dmask, block, stride, frac, cap)
    assert st == 0 and n_ref == nd_ref > 0
    for _ in range(2):  # the second call starts from the first call's leftovers
        st, n, nd, c = _call(nrr, L.nrr_select_blocks_noalloc, dpre, dmask, block, stride, frac, cap)
        assert st == 0, L.nrr_last_error()
        assert n == nd == n_ref
        assert np.array_equal(c, c_ref)


def test_noalloc_refuses_grids_beyond_its_scratch(nrr):
    L = nrr.lib()
    nx, ny, nz = 256, 256, 128  # stride 1: 8.4M grid points > ~4M
    dpre = torch.zeros((nz, ny, nx), dtype=torch.int16, device="cuda")
    dmask = torch.ones((nz, ny, nx), dtype=torch.uint8, device="cuda")
    st, n, nd, c = _call(nrr, L.nrr_select_blocks_noalloc, dpre, dmask, 3, 1, 0.01, 16)
    assert st == -4  # NRR_E_CAPACITY
    assert b"allocation-free selection holds" in L.nrr_last_error()
    assert nd == -1 and (c == -1).all()  # nothing written
