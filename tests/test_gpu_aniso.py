"""GPU parity for blocks with a different edge per axis (bx, by, bz) against
the CPU oracle, through the C ABI: selection and uint16 matching bit-exact,
box sums exact, float32 within the float32 tolerances of the cubic tests."""
import numpy as np
import pytest

import oracle
from paper_2308_10868_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F32_NCC_TOL = 1e-6
F32_TIE_TOL = 2e-6


@pytest.fixture(scope="module")
def nrr():
    from paper_2308_10868_gb300 import build as nbuild

    nbuild.build()
    from paper_2308_10868_gb300 import nrr as m

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return m


def _same_ncc(a, b):
    na, nb = np.isnan(a), np.isnan(b)
    return np.array_equal(na, nb) and np.array_equal(a[~na].view(np.int64), b[~nb].view(np.int64))


def _match_u16(nrr, pre, intra, centers, bl, r, box=False):
    dpre, dintra = nrr.to_device_u16(pre), nrr.to_device_u16(intra)
    dc = torch.from_numpy(np.ascontiguousarray(centers, dtype=np.int32).reshape(-1, 3)).cuda()
    bx = nrr.boxsums(dintra, bl) if box else None
    disp, ncc, valid = nrr.block_match(dpre, dintra, dc, bl, r, box=bx)
    nrr.device_status()
    return disp.cpu().numpy(), ncc.cpu().numpy(), valid.cpu().numpy()


def _check_u16(nrr, pre, intra, centers, bl, r, box=False):
    gd, gn, gv = _match_u16(nrr, pre, intra, centers, bl, r, box)
    rd, rn, rv = oracle.match(pre, intra, centers, bl, r)
    bad = np.nonzero((gd != rd).any(axis=1))[0]
    assert bad.size == 0, f"{bad.size} displacements differ: gpu {gd[bad[:3]]} cpu {rd[bad[:3]]}"
    assert np.array_equal(gv, rv)
    assert _same_ncc(gn, rn)
    return gv


BLOCKS = [(3, 5, 7), (7, 5, 3), (9, 7, 5), (5, 9, 3), (11, 3, 5), (3, 3, 11)]


@pytest.mark.parametrize("bl", BLOCKS)
def test_selection_bit_exact(nrr, bl):
    pre, _, mask = synth.workload_pair("small")
    got = nrr.select_blocks(nrr.to_device_u16(pre), torch.from_numpy(mask).cuda(), bl, 2, 0.1)
    ref, nc = oracle.select_blocks(pre, mask, bl, 2, 0.1)
    assert len(ref) == oracle.n_select(nc, 0.1) and len(ref) > 0
    assert np.array_equal(got.cpu().numpy(), ref)


@pytest.mark.parametrize("bl,stride,frac", [((3, 5, 7), 1, 0.05), ((7, 3, 5), 3, 0.5), ((5, 5, 9), 2, 1.0)])
def test_selection_ties_and_flat_regions(nrr, bl, stride, frac):
    dims = (40, 36, 30)
    pre = synth.random_u16(dims, 21, hi=8)  # tiny range: many equal keys
    pre[:, :, :9] = 3  # flat slab: key 0 never selected
    mask = synth.ellipsoid_mask(dims, 0.5)
    got = nrr.select_blocks(nrr.to_device_u16(pre), torch.from_numpy(mask).cuda(), bl, stride, frac)
    ref, _ = oracle.select_blocks(pre, mask, bl, stride, frac)
    assert np.array_equal(got.cpu().numpy(), ref)


@pytest.mark.parametrize("bl,r", [((3, 5, 7), 4), ((7, 5, 3), (3, 2, 1)), ((9, 7, 5), (5, 4, 3)),
                                  ((5, 9, 3), (0, 2, 3)), ((11, 3, 5), (7, 1, 2)), ((3, 3, 11), (2, 7, 4))])
def test_match_small_workload_bit_exact(nrr, bl, r):
    pre, intra, mask = synth.workload_pair("small")
    centers, _ = oracle.select_blocks(pre, mask, bl, 2, 0.1)
    v = _check_u16(nrr, pre, intra, centers, bl, r)
    assert v.sum() > 0.9 * len(v)


def test_match_precomputed_box_sums_and_cubic_triple(nrr):
    pre, intra, mask = synth.workload_pair("small")
    centers, _ = oracle.select_blocks(pre, mask, (7, 5, 3), 2, 0.1)
    _check_u16(nrr, pre, intra, centers, (7, 5, 3), (3, 2, 2), box=True)
    # a cubic triple takes the cubic path: identical bits to the int form
    c7, _ = oracle.select_blocks(pre, mask, 7, 2, 0.1)
    a = _match_u16(nrr, pre, intra, c7, 7, 4)
    b = _match_u16(nrr, pre, intra, c7, (7, 7, 7), 4)
    assert all(np.array_equal(x.view(np.uint8), y.view(np.uint8)) for x, y in zip(a, b))


def test_match_border_and_invalid_blocks(nrr):
    dims = (40, 32, 24)
    pre = synth.random_u16(dims, 31, hi=4096)
    intra = synth.random_u16(dims, 32, hi=4096)
    nx, ny, nz = dims
    bl = (3, 9, 5)
    hx, hy, hz = 1, 4, 2
    centers = np.array([(hx, hy, hz), (nx - 1 - hx, ny - 1 - hy, nz - 1 - hz), (hx, ny // 2, hz),
                        (0, 10, 10), (10, hy - 1, 10), (10, 10, nz - hz), (20, 16, 12), (nx - 2, ny - 5, nz - 3)],
                       dtype=np.int32)
    v = _check_u16(nrr, pre, intra, centers, bl, (3, 2, 4))
    assert v[3] == 0 and v[4] == 0 and v[5] == 0 and v[6] == 1


def test_match_clinical_workload_bit_exact(nrr):
    pre, intra, mask = synth.workload_pair("clinical")
    bl = (9, 7, 5)
    centers, _ = oracle.select_blocks(pre, mask, bl, 2, 0.05)
    assert len(centers) > 10000
    _check_u16(nrr, pre, intra, centers, bl, (5, 5, 3))


@pytest.mark.parametrize("bl", [(3, 5, 7), (11, 7, 3)])
def test_box_sums_contents(nrr, bl):
    # uint16: S1 exact int32; A2 = N*S2 - S1^2 rounded once to float32; zero
    # where the block leaves the volume
    dims = (48, 26, 21)
    vol = synth.random_u16(dims, 33)  # full 16-bit range
    buf = nrr.boxsums(nrr.to_device_u16(vol), bl).cpu().numpy()
    nz, ny, nx = vol.shape
    nv = nx * ny * nz
    s1 = buf[:4 * nv].view(np.int32).reshape(nz, ny, nx).astype(np.int64)
    off = (4 * nv + 255) // 256 * 256
    a2 = buf[off:off + 4 * nv].view(np.float32).reshape(nz, ny, nx)
    hx, hy, hz = ((b - 1) // 2 for b in bl)
    v = vol.astype(np.int64)
    r1 = np.zeros_like(v)
    r2 = np.zeros_like(v)
    for z in range(hz, nz - hz):
        for y in range(hy, ny - hy):
            blk = v[z - hz:z + hz + 1, y - hy:y + hy + 1]
            for x in range(hx, nx - hx):
                w = blk[:, :, x - hx:x + hx + 1]
                r1[z, y, x] = w.sum()
                r2[z, y, x] = (w * w).sum()
    assert np.array_equal(s1, r1)
    ref_a2 = (bl[0] * bl[1] * bl[2] * r2 - r1 * r1).astype(np.float32)
    assert np.array_equal(a2.view(np.uint32), ref_a2.view(np.uint32))


def test_f32_small_workload(nrr):
    pre, intra, mask = synth.workload_pair("small")
    pre32, intra32 = synth.as_f32(pre), synth.as_f32(intra)
    for bl, r in (((7, 5, 3), 4), ((3, 9, 5), (5, 2, 3))):
        centers, _ = oracle.select_blocks(pre, mask, bl, 2, 0.1)
        dc = torch.from_numpy(np.ascontiguousarray(centers, np.int32)).cuda()
        disp, ncc, valid = nrr.block_match(torch.from_numpy(pre32).cuda(), torch.from_numpy(intra32).cuda(), dc, bl, r)
        nrr.device_status()
        gd, gn, gv = disp.cpu().numpy(), ncc.cpu().numpy(), valid.cpu().numpy()
        rd, rn, rv = oracle.match(pre32, intra32, centers, bl, r)
        assert np.array_equal(gv, rv)
        ok = rv == 1
        at_gpu = np.array([oracle.pearson_f32(pre32, intra32, bl, centers[i], gd[i]) if ok[i] else np.nan
                           for i in range(len(centers))], dtype=np.float64)
        assert np.abs(gn[ok] - at_gpu[ok]).max() <= F32_NCC_TOL
        diff = (gd != rd).any(axis=1) & ok
        assert (rn[diff] - at_gpu[diff] <= F32_TIE_TOL).all()


def test_argument_checks(nrr):
    pre, intra, mask = synth.workload_pair("small")
    dpre = nrr.to_device_u16(pre)
    dmask = torch.from_numpy(mask).cuda()
    for bad in ((4, 5, 7), (3, 13, 5), (1, 3, 3)):
        with pytest.raises(RuntimeError):
            nrr.select_blocks(dpre, dmask, bad, 2, 0.1)
    with pytest.raises(ValueError):
        nrr.select_blocks(dpre, dmask, (3, 5, 7), 2, 0.1, connectivity=6)
