"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

uint16 results must be bit-identical (centres, displacements, NCC bits,
valid flags).  float32 results: NCC within 1e-6 of the oracle's FP64 value
at the returned shift, and a returned shift that differs from the oracle's
only where the oracle's own scores of the two are within 2e-6.
"""
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


def _dev_u16(nrr, a):
    return nrr.to_device_u16(a)


def _same_ncc(a, b):
    na, nb = np.isnan(a), np.isnan(b)
    return np.array_equal(na, nb) and np.array_equal(a[~na].view(np.int64), b[~nb].view(np.int64))


def _check_u16(nrr, pre, intra, centers, b, r, dpre=None, dintra=None):
    dpre = _dev_u16(nrr, pre) if dpre is None else dpre
    dintra = _dev_u16(nrr, intra) if dintra is None else dintra
    dc = torch.from_numpy(np.ascontiguousarray(centers, dtype=np.int32).reshape(-1, 3)).cuda()
    disp, ncc, valid = nrr.block_match(dpre, dintra, dc, b, r)
    nrr.device_status()
    rd, rn, rv = oracle.match(pre, intra, centers, b, r)
    gd, gn, gv = disp.cpu().numpy(), ncc.cpu().numpy(), valid.cpu().numpy()
    bad = np.nonzero((gd != rd).any(axis=1))[0]
    assert bad.size == 0, f"{bad.size} displacements differ, first block {bad[:5]}: gpu {gd[bad[:3]]} cpu {rd[bad[:3]]}"
    assert np.array_equal(gv, rv)
    assert _same_ncc(gn, rn), np.nanmax(np.abs(gn - rn))
    return gd, gn, gv


@pytest.mark.parametrize("key", ["small", "clinical"])
def test_selection_bit_exact(nrr, key):
    pre, intra, mask = synth.workload_pair(key)
    w = synth.WORKLOADS[key]
    got = nrr.select_blocks(_dev_u16(nrr, pre), torch.from_numpy(mask).cuda(), w.block, w.stride, w.frac)
    ref, nc = oracle.select_blocks(pre, mask, w.block, w.stride, w.frac)
    assert got.shape[0] == ref.shape[0] == oracle.n_select(nc, w.frac)
    assert np.array_equal(got.cpu().numpy(), ref)


@pytest.mark.parametrize("b,stride,frac", [(3, 1, 0.05), (5, 3, 0.5), (9, 2, 1.0), (11, 4, 0.2)])
def test_selection_variants_and_ties(nrr, b, stride, frac):
    dims = (40, 36, 30)
    pre = synth.random_u16(dims, 11, hi=8)  # tiny range: many equal keys
    pre[:, :, :9] = 3  # a flat slab: key 0 never selected
    mask = synth.ellipsoid_mask(dims, 0.5)
    got = nrr.select_blocks(_dev_u16(nrr, pre), torch.from_numpy(mask).cuda(), b, stride, frac)
    ref, _ = oracle.select_blocks(pre, mask, b, stride, frac)
    assert np.array_equal(got.cpu().numpy(), ref)


def test_selection_capacity_and_device_count(nrr):
    pre, _, mask = synth.workload_pair("small")
    dpre, dmask = _dev_u16(nrr, pre), torch.from_numpy(mask).cuda()
    ref, _ = oracle.select_blocks(pre, mask, 7, 2, 0.1)
    with pytest.raises(nrr.NrrError) as ei:
        nrr.select_blocks(dpre, dmask, 7, 2, 0.1, max_blocks=10)
    assert ei.value.status == -4
    centers, n = nrr.select_blocks(dpre, dmask, 7, 2, 0.1, sync=False)
    torch.cuda.synchronize()
    assert int(n.item()) == len(ref)
    assert np.array_equal(centers[:len(ref)].cpu().numpy(), ref)


def test_match_small_workload_bit_exact(nrr):
    pre, intra, mask = synth.workload_pair("small")
    w = synth.WORKLOADS["small"]
    centers, _ = oracle.select_blocks(pre, mask, w.block, w.stride, w.frac)
    _check_u16(nrr, pre, intra, centers, w.block, w.radius)


def test_match_clinical_workload_bit_exact(nrr):
    pre, intra, mask = synth.workload_pair("clinical")
    w = synth.WORKLOADS["clinical"]
    centers, _ = oracle.select_blocks(pre, mask, w.block, w.stride, w.frac)
    assert len(centers) > 19000
    gd, gn, gv = _check_u16(nrr, pre, intra, centers, w.block, w.radius)
    assert gv.all() and np.nanmedian(gn) > 0.9


@pytest.mark.parametrize("key,r", [("small", None), ("clinical", None), ("small", (3, 1, 2))])
def test_match_plain_launch(nrr, key, r):
    """One CTA per block (nrr_block_match_plain) returns exactly what the
    persistent launch returns; on the small workload, the oracle's result."""
    pre, intra, mask = synth.workload_pair(key)
    w = synth.WORKLOADS[key]
    r = w.radius if r is None else r
    centers, _ = oracle.select_blocks(pre, mask, w.block, w.stride, w.frac)
    dpre, dintra = _dev_u16(nrr, pre), _dev_u16(nrr, intra)
    dc = torch.from_numpy(np.ascontiguousarray(centers, dtype=np.int32)).cuda()
    box = nrr.boxsums(dintra, w.block)
    pd, pn, pv = (t.cpu().numpy() for t in nrr.block_match(dpre, dintra, dc, w.block, r, box=box, plain=True))
    nrr.device_status()
    qd, qn, qv = (t.cpu().numpy() for t in nrr.block_match(dpre, dintra, dc, w.block, r, box=box))
    assert np.array_equal(pd, qd) and np.array_equal(pv, qv) and _same_ncc(pn, qn)
    if key == "small":
        rd, rn, rv = oracle.match(pre, intra, centers, w.block, r)
        assert np.array_equal(pd, rd) and np.array_equal(pv, rv) and _same_ncc(pn, rn)
    with pytest.raises(ValueError):
        nrr.block_match(dpre, dintra, dc, w.block, r, plain=True)  # box sums required


# windows whose (dy, dz) line grid pairs along z only, along y only (rz = 0),
# with a line left over along y or along z (ry = 0), or is a single line
@pytest.mark.parametrize("b,r", [(3, (1, 1, 1)), (5, (3, 2, 1)), (7, (0, 2, 3)), (9, (7, 7, 7)),
                                 (11, (2, 5, 4)), (5, (6, 0, 0)), (3, (7, 1, 6)), (5, (2, 0, 3)),
                                 (7, (1, 4, 0)), (3, (0, 0, 1)), (9, (3, 6, 7))])
def test_match_block_sizes_and_anisotropic_windows(nrr, b, r):
    pre, intra, mask = synth.workload_pair("small")
    centers, _ = oracle.select_blocks(pre, mask, b, 2, 0.05)
    _check_u16(nrr, pre, intra, centers[:400], b, r)


def test_match_border_and_invalid_blocks(nrr):
    pre, intra, _ = synth.workload_pair("small")
    pre = pre.copy()
    pre[10:17, 10:17, 10:17] = 1234  # flat floating block centred at (13,13,13), b=7
    nz, ny, nx = pre.shape
    centers = [(13, 13, 13), (3, 3, 3), (2, 30, 30), (nx - 4, ny - 4, nz - 4), (nx - 3, 20, 20), (5, ny - 5, 4),
               (-3, 10, 10), (30, 30, 100)]
    centers += [(x, y, z) for z in (3, 4, 5, nz - 6, nz - 5, nz - 4) for y in (3, 6, ny - 4) for x in (3, 8, nx - 4)]
    gd, gn, gv = _check_u16(nrr, pre, intra, np.array(centers, dtype=np.int32), 7, (5, 4, 6))
    assert gv[0] == 0 and gv[2] == 0 and gv[4] == 0 and gv[6] == 0 and gv[7] == 0


def test_match_random_noise_many_ties(nrr):
    dims = (48, 40, 32)
    pre = synth.random_u16(dims, 21, hi=4)  # 2-bit data: plenty of exactly equal NCC values
    intra = synth.random_u16(dims, 22, hi=4)
    cs = np.array([(x, y, z) for z in range(3, 29, 5) for y in range(3, 37, 6) for x in range(3, 45, 7)], np.int32)
    _check_u16(nrr, pre, intra, cs, 5, (3, 3, 2))


def test_match_full_range_intensities(nrr):
    dims = (48, 40, 32)
    pre = synth.random_u16(dims, 31)  # uniform over all 65536 values
    intra = synth.random_u16(dims, 32)
    cs = np.array([(x, y, z) for z in range(5, 27, 4) for y in range(5, 35, 5) for x in range(5, 43, 6)], np.int32)
    _check_u16(nrr, pre, intra, cs, 11, (3, 2, 2))
    big = (pre // 2 + 32768).astype(np.uint16)  # large mean, small spread
    _check_u16(nrr, big, (intra // 64 + 65000).astype(np.uint16), cs, 9, (4, 4, 4))


def test_self_match_and_translation(nrr):
    pre, _, mask = synth.workload_pair("small")
    centers, _ = oracle.select_blocks(pre, mask, 7, 2, 0.1)
    gd, gn, gv = _check_u16(nrr, pre, pre, centers, 7, 4)
    assert (gd == 0).all() and (gn == 1.0).all()
    t = (3, -2, 1)
    gd, gn, gv = _check_u16(nrr, pre, synth.translate(pre, t), centers, 7, 4)


def test_device_count_and_empty(nrr):
    pre, intra, mask = synth.workload_pair("small")
    centers, _ = oracle.select_blocks(pre, mask, 7, 2, 0.1)
    dpre, dintra = _dev_u16(nrr, pre), _dev_u16(nrr, intra)
    dc = torch.from_numpy(centers).cuda()
    n = torch.tensor([100], dtype=torch.int32, device="cuda")
    disp, ncc, valid = (torch.full((len(centers), 3), 77, dtype=torch.int32, device="cuda"),
                        torch.zeros(len(centers), dtype=torch.float64, device="cuda"),
                        torch.full((len(centers),), 9, dtype=torch.uint8, device="cuda"))
    nrr.block_match(dpre, dintra, dc, 7, 4, n_blocks=n, out=(disp, ncc, valid))
    nrr.device_status()
    rd, rn, rv = oracle.match(pre, intra, centers[:100], 7, 4)
    assert np.array_equal(disp[:100].cpu().numpy(), rd)
    assert (disp[100:] == 77).all() and (valid[100:] == 9).all()
    e = torch.empty((0, 3), dtype=torch.int32, device="cuda")
    d0, n0, v0 = nrr.block_match(dpre, dintra, e, 7, 4)
    assert d0.shape == (0, 3)
    n.zero_()
    nrr.block_match(dpre, dintra, dc, 7, 4, n_blocks=n, out=(disp, ncc, valid))
    nrr.device_status()
    assert (disp[:100].cpu().numpy() == rd).all()  # untouched


def test_repeatable_and_precomputed_box_sums(nrr):
    pre, intra, mask = synth.workload_pair("small")
    centers, _ = oracle.select_blocks(pre, mask, 7, 2, 0.1)
    dpre, dintra = _dev_u16(nrr, pre), _dev_u16(nrr, intra)
    dc = torch.from_numpy(centers).cuda()
    a = [t.cpu().numpy() for t in nrr.block_match(dpre, dintra, dc, 7, 4)]
    box = nrr.boxsums(dintra, 7)
    for _ in range(3):
        b = [t.cpu().numpy() for t in nrr.block_match(dpre, dintra, dc, 7, 4, box=box)]
        assert all(np.array_equal(x.view(np.uint8), y.view(np.uint8)) for x, y in zip(a, b))


def _check_f32(nrr, pre32, intra32, centers, b, r):
    dc = torch.from_numpy(np.ascontiguousarray(centers, np.int32)).cuda()
    disp, ncc, valid = nrr.block_match(torch.from_numpy(pre32).cuda(), torch.from_numpy(intra32).cuda(), dc, b, r)
    nrr.device_status()
    gd, gn, gv = disp.cpu().numpy(), ncc.cpu().numpy(), valid.cpu().numpy()
    rd, rn, rv = oracle.match(pre32, intra32, centers, b, r)
    assert np.array_equal(gv, rv)
    ok = rv == 1
    # oracle's FP64 score at the GPU's chosen shift
    at_gpu = np.array([oracle.pearson_f32(pre32, intra32, b, centers[i], gd[i]) if ok[i] else np.nan
                       for i in range(len(centers))], dtype=np.float64)
    err = np.abs(gn[ok] - at_gpu[ok])
    assert err.max() <= F32_NCC_TOL, err.max()
    diff = (gd != rd).any(axis=1) & ok
    assert (rn[diff] - at_gpu[diff] <= F32_TIE_TOL).all()
    print(f"\nfloat32 b={b} r={r}: NCC error against FP64 at the returned shift: max {err.max():.3g}, "
          f"mean {err.mean():.3g} over {int(ok.sum())} blocks; shift differs from the FP64 arg-max in "
          f"{int(diff.sum())} (within {F32_TIE_TOL:g} of its score)")
    return err.max(), diff.mean()


def test_f32_small_workload(nrr):
    pre, intra, mask = synth.workload_pair("small")
    centers, _ = oracle.select_blocks(pre, mask, 7, 2, 0.1)
    _check_f32(nrr, synth.as_f32(pre), synth.as_f32(intra), centers, 7, 4)
    _check_f32(nrr, synth.as_f32(pre), synth.as_f32(intra), centers[:300], 9, (7, 3, 5))


def test_f32_integer_valued_equals_u16(nrr):
    # Integer-valued float32 intensities: the float32 path's float-float sums
    # are exact, so its NCC must equal the uint16 path's (and the oracle's
    # canonical value) to rounding, and its displacements must be the
    # oracle's except where the oracle's own scores of the two shifts tie.
    pre, intra, mask = synth.workload_pair("small")
    centers, _ = oracle.select_blocks(pre, mask, 7, 2, 0.1)
    dc = torch.from_numpy(centers).cuda()
    d16, n16, v16 = nrr.block_match(_dev_u16(nrr, pre), _dev_u16(nrr, intra), dc, 7, 4)
    d32, n32, v32 = nrr.block_match(torch.from_numpy(pre.astype(np.float32)).cuda(),
                                    torch.from_numpy(intra.astype(np.float32)).cuda(), dc, 7, 4)
    nrr.device_status()
    rd, rn, rv = oracle.match(pre, intra, centers, 7, 4)
    g32, n32h, v32h = d32.cpu().numpy(), n32.cpu().numpy(), v32.cpu().numpy()
    assert torch.equal(v16, v32) and np.array_equal(v32h, rv)
    ok = rv == 1
    assert np.abs(n32h[ok] - rn[ok]).max() < 1e-12
    assert (n16 - n32).abs().max().item() < 1e-12
    diff = np.nonzero((g32 != rd).any(axis=1) & ok)[0]
    for i in diff:  # a different shift only on an exact tie of the canonical scores
        assert abs(oracle.ncc_u16(pre, intra, 7, centers[i], g32[i]) - rn[i]) < 1e-12, (i, g32[i], rd[i])
    print(f"\ninteger-valued float32: {len(diff)} of {int(ok.sum())} displacements differ from the oracle "
          f"(canonical-score ties only)")


@pytest.mark.parametrize("offset,spread", [(50.0, 1.0), (1000.0, 1e-2)])
def test_f32_large_offset(nrr, offset, spread):
    # Intensities on an offset large against their spread (50x and 10^5x).
    # The float box sums are of J - c with c the volume's centre value, so
    # they keep every reference block's spread and the filter bound applies
    # on both; the float-float rescoring must not lose the spread to the
    # offset either.
    pre, intra, mask = synth.workload_pair("small")
    centers, _ = oracle.select_blocks(pre, mask, 7, 2, 0.1)
    centers = centers[:160]
    off, sp = np.float32(offset), np.float32(spread)
    p32 = (off + synth.as_f32(pre) * sp).astype(np.float32)
    i32 = (off + synth.as_f32(intra) * sp).astype(np.float32)
    _check_f32(nrr, p32, i32, centers, 7, 3)



def _box_ref(vol, b):
    """Exact block sums of J and J^2 by integral volumes (int64), 0 where the
    block leaves the volume."""
    v = vol.astype(np.int64)
    h = (b - 1) // 2

    def boxsum(a):
        c = np.zeros(tuple(s + 1 for s in a.shape), np.int64)
        c[1:, 1:, 1:] = a.cumsum(0).cumsum(1).cumsum(2)
        nz, ny, nx = a.shape
        out = np.zeros(a.shape, np.int64)
        z0, y0, x0 = np.arange(nz - b + 1), np.arange(ny - b + 1), np.arange(nx - b + 1)
        Z, Y, X = np.ix_(z0, y0, x0)
        s = (c[Z + b, Y + b, X + b] - c[Z, Y + b, X + b] - c[Z + b, Y, X + b] - c[Z + b, Y + b, X]
             + c[Z, Y, X + b] + c[Z, Y + b, X] + c[Z + b, Y, X] - c[Z, Y, X])
        out[h:nz - h, h:ny - h, h:nx - h] = s
        return out

    return boxsum(v), boxsum(v * v)


@pytest.mark.parametrize("b", [3, 7, 11])
def test_box_sums_contents(nrr, b):
    # uint16 box sums: S1 exact int32; A2 = N*S2 - S1^2 rounded once to float32
    dims = (48, 26, 21)
    vol = synth.random_u16(dims, 5)  # full 16-bit range
    buf = nrr.boxsums(_dev_u16(nrr, vol), b).cpu().numpy()
    nz, ny, nx = vol.shape
    nv = nx * ny * nz
    s1 = buf[:4 * nv].view(np.int32).reshape(nz, ny, nx)
    off = (4 * nv + 255) // 256 * 256
    a2 = buf[off:off + 4 * nv].view(np.float32).reshape(nz, ny, nx)
    r1, r2 = _box_ref(vol, b)
    assert np.array_equal(s1.astype(np.int64), r1)
    ref_a2 = (b ** 3 * r2 - r1 * r1).astype(np.float32)
    assert np.array_equal(a2.view(np.uint32), ref_a2.view(np.uint32))


@pytest.mark.parametrize("b,r,nb", [(7, (8, 8, 8), 160), (5, (11, 3, 9), 160), (5, (15, 15, 15), 60),
                                    (7, (9, 0, 12), 120)])
def test_large_radius_bit_exact(nrr, b, r, nb):
    # Radii above 7 are searched as sub-windows (two per axis for 8..11,
    # three for 12..15); the best over them must be the oracle's exactly.
    pre, intra, mask = synth.workload_pair("small")
    centers, _ = oracle.select_blocks(pre, mask, b, 2, 0.1)
    _check_u16(nrr, pre, intra, centers[:nb], b, r)


def test_large_radius_recovers_a_large_translation(nrr):
    # intraop = preop shifted by t with |t| up to 14: every block whose
    # shifted block lies in the volume returns d = t with NCC exactly 1.
    pre, _, mask = synth.workload_pair("small")
    t = (12, -9, 14)
    intra = synth.translate(pre, t)
    centers, _ = oracle.select_blocks(pre, mask, 5, 2, 0.1)
    gd, gn, gv = _check_u16(nrr, pre, intra, centers[:200], 5, (15, 15, 15))
    nz, ny, nx = pre.shape
    h = 2
    full = np.array([all(h <= c[k] + t[k] <= (nx, ny, nz)[k] - 1 - h for k in range(3)) for c in centers[:200]])
    assert full.sum() > 20
    assert (gd[full] == np.array(t)).all() and (gn[full] == 1.0).all()


def test_f32_large_radius(nrr):
    pre, intra, mask = synth.workload_pair("small")
    centers, _ = oracle.select_blocks(pre, mask, 7, 2, 0.1)
    _check_f32(nrr, synth.as_f32(pre), synth.as_f32(intra), centers[:100], 7, (10, 4, 13))
