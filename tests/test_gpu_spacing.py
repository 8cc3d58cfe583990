"""GPU parity of the selection with a connectivity pattern (Sec. 4.1, face /
edge / vertex = 6 / 18 / 26 neighbours on the candidate grid) against the CPU
oracle: the centre lists must be identical (integer work, bit-exact)."""
import itertools

import numpy as np
import pytest

import oracle
from paper_2308_10868_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CONNS = (6, 18, 26)


@pytest.fixture(scope="module")
def nrr():
    from paper_2308_10868_gb300 import build as nbuild

    nbuild.build()
    from paper_2308_10868_gb300 import nrr as m

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return m


def _select(nrr, pre, mask, b, stride, frac, conn):
    got = nrr.select_blocks(nrr.to_device_u16(pre), torch.from_numpy(np.ascontiguousarray(mask)).cuda(), b, stride,
                            frac, connectivity=conn)
    nrr.device_status()
    return got.cpu().numpy()


def _independent(centers, stride, conn):
    order = {6: 1, 18: 2, 26: 3}[conn]
    pts = {tuple(int(v) // stride for v in c) for c in centers}
    for p in pts:
        for o in itertools.product((-1, 0, 1), repeat=3):
            if 0 < sum(map(abs, o)) <= order and (p[0] + o[0], p[1] + o[1], p[2] + o[2]) in pts:
                return False
    return True


@pytest.mark.parametrize("conn", CONNS)
@pytest.mark.parametrize("key", ["small", "clinical"])
def test_spaced_selection_workloads_bit_exact(nrr, key, conn):
    pre, _, mask = synth.workload_pair(key)
    w = synth.WORKLOADS[key]
    got = _select(nrr, pre, mask, w.block, w.stride, w.frac, conn)
    ref, nc = oracle.select_blocks_spaced(pre, mask, w.block, w.stride, w.frac, conn)
    assert len(ref) > 0
    assert np.array_equal(got, ref)
    assert _independent(got, w.stride, conn)


def test_spaced_selection_highres_bit_exact(nrr):
    pre, _, mask = synth.workload_pair("highres")
    w = synth.WORKLOADS["highres"]
    got = _select(nrr, pre, mask, w.block, w.stride, w.frac, 6)
    ref, _ = oracle.select_blocks_spaced(pre, mask, w.block, w.stride, w.frac, 6)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("conn", CONNS)
@pytest.mark.parametrize("b,stride,frac", [(3, 1, 0.3), (5, 2, 1.0), (7, 3, 0.5), (9, 5, 1.0)])
def test_spaced_selection_ties_and_flat_regions(nrr, b, stride, frac, conn):
    dims = (48, 36, 30)
    pre = synth.random_u16(dims, 21, hi=6)  # tiny range: many equal keys, ranked by raster index
    pre[:, :, :10] = 4  # a flat slab: key 0, never selected
    mask = synth.ellipsoid_mask(dims, 0.5)
    got = _select(nrr, pre, mask, b, stride, frac, conn)
    ref, _ = oracle.select_blocks_spaced(pre, mask, b, stride, frac, conn)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("conn", CONNS)
def test_spaced_selection_equal_keys_lattice(nrr, conn):
    # every 3^3 block holds the same values: all keys equal, order = raster
    # order, and the greedy set is a lattice (long chains of dependence: the
    # decision at each point waits for the one before it along the raster)
    nz, ny, nx = 24, 40, 64
    x = np.arange(nx)
    pre = np.broadcast_to(1000 + 300 * (x % 3), (nz, ny, nx)).astype(np.uint16).copy()
    mask = np.ones((nz, ny, nx), np.uint8)
    got = _select(nrr, pre, mask, 3, 1, 1.0, conn)
    ref, nc = oracle.select_blocks_spaced(pre, mask, 3, 1, 1.0, conn)
    assert np.array_equal(got, ref)
    assert len(ref) * {6: 2, 18: 4, 26: 8}[conn] == nc  # the interior extents 62, 38, 22 are even


def test_spaced_selection_without_pattern_is_plain(nrr):
    pre, _, mask = synth.workload_pair("small")
    got = _select(nrr, pre, mask, 7, 2, 0.1, 0)
    ref, _ = oracle.select_blocks(pre, mask, 7, 2, 0.1)
    assert np.array_equal(got, ref)


def test_spaced_selection_empty_and_flat(nrr):
    dims = (32, 24, 20)
    pre = synth.random_u16(dims, 3)
    none = np.zeros((dims[2], dims[1], dims[0]), np.uint8)
    assert _select(nrr, pre, none, 5, 2, 0.5, 18).shape[0] == 0
    flat = np.full((dims[2], dims[1], dims[0]), 77, np.uint16)
    assert _select(nrr, flat, np.ones_like(none), 5, 2, 0.5, 26).shape[0] == 0
