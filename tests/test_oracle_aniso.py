"""Pins of the oracle for blocks with a different edge per axis (bx, by, bz).

The paper's parameter list (Sec. 5) counts twelve tunable parameters, which
holds only when the half block size, like the half window size, is given per
anatomical axis.  These tests fix the per-axis oracle to things that do not
come from it: numpy's correlation coefficient, brute force in Python
integers, the cubic path (bx = by = bz), a known translation, and the
symmetry of the method under a permutation of the volume axes (which catches
an x/z or y/z mix-up in either direction).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2308_10868_gb300 import synth


def _half(bl):
    return tuple((b - 1) // 2 for b in bl)


def _block(vol, c, bl):
    hx, hy, hz = _half(bl)
    x, y, z = c
    return vol[z - hz:z + hz + 1, y - hy:y + hy + 1, x - hx:x + hx + 1]


def _inside(dims, c, bl):
    h = _half(bl)
    return all(h[i] <= c[i] <= dims[i] - 1 - h[i] for i in range(3))


def _shifts(r):
    rx, ry, rz = r
    for dz in range(-rz, rz + 1):
        for dy in range(-ry, ry + 1):
            for dx in range(-rx, rx + 1):
                yield (dx, dy, dz)


def _t1_better(s, d, bs, bd):
    if s != bs:
        return s > bs
    n1, n2 = sum(v * v for v in d), sum(v * v for v in bd)
    if n1 != n2:
        return n1 < n2
    return (d[2], d[1], d[0]) < (bd[2], bd[1], bd[0])


DIMS = (15, 12, 10)  # nx != ny != nz
BLOCKS = [(3, 5, 7), (7, 3, 5), (5, 7, 3), (3, 3, 9), (9, 5, 3)]


@pytest.mark.parametrize("bl", BLOCKS)
def test_block_key_is_exact_integer_form(bl):
    vol = synth.random_u16(DIMS, 11)
    h = _half(bl)
    nx, ny, nz = DIMS
    for c in [h, (nx // 2, ny // 2, nz // 2), (nx - 1 - h[0], ny - 1 - h[1], nz - 1 - h[2])]:
        vals = [int(v) for v in _block(vol, c, bl).ravel()]
        assert len(vals) == bl[0] * bl[1] * bl[2]
        assert oracle.block_key(vol, bl, *c) == len(vals) * sum(v * v for v in vals) - sum(vals) ** 2


@pytest.mark.parametrize("bl", BLOCKS[:3])
def test_ncc_equals_numpy_corrcoef(bl):
    pre = synth.random_u16(DIMS, 12)
    intra = synth.random_u16(DIMS, 13)
    h = _half(bl)
    nx, ny, nz = DIMS
    n = 0
    for c in [h, (nx // 2, ny // 2, nz // 2), (nx - 1 - h[0], ny - 1 - h[1], nz - 1 - h[2])]:
        for d in _shifts((1, 1, 1)):
            v = oracle.ncc_u16(pre, intra, bl, c, d)
            cd = tuple(c[i] + d[i] for i in range(3))
            if not _inside(DIMS, cd, bl):
                assert v is None
                continue
            I = _block(pre, c, bl).astype(np.float64).ravel()
            J = _block(intra, cd, bl).astype(np.float64).ravel()
            assert v == pytest.approx(float(np.corrcoef(I, J)[0, 1]), abs=1e-12)
            assert oracle.pearson_u16(pre, intra, bl, c, d) == pytest.approx(v, abs=1e-12)
            fv = oracle.pearson_f32(pre.astype(np.float32), intra.astype(np.float32), bl, c, d)
            assert fv == pytest.approx(v, abs=1e-12)
            n += 1
    assert n > 20


@pytest.mark.parametrize("bl,r", [((3, 5, 7), (1, 1, 1)), ((7, 3, 3), (2, 1, 0)), ((3, 3, 5), (1, 2, 1))])
def test_match_equals_brute_force(bl, r):
    pre = synth.random_u16(DIMS, 14, hi=4096)
    intra = synth.random_u16(DIMS, 15, hi=4096)
    h = _half(bl)
    nx, ny, nz = DIMS
    centers = np.array([(x, y, z) for z in range(h[2], nz - h[2], 2) for y in range(h[1], ny - h[1], 3)
                        for x in range(h[0], nx - h[0], 4)] + [(0, 5, 4), (nx - 1, 5, 4)], dtype=np.int32)
    disp, ncc, valid = oracle.match(pre, intra, centers, bl, r)
    for i, c in enumerate(centers):
        best, bd = None, (0, 0, 0)
        if _inside(DIMS, c, bl):
            I = _block(pre, c, bl).astype(np.float64).ravel()
            for d in _shifts(r):
                cd = tuple(int(c[k]) + d[k] for k in range(3))
                if not _inside(DIMS, cd, bl):
                    continue
                J = _block(intra, cd, bl).astype(np.float64).ravel()
                s = float(np.corrcoef(I, J)[0, 1])
                if best is None or _t1_better(s, d, best, bd):
                    best, bd = s, d
        if best is None:
            assert valid[i] == 0 and np.isnan(ncc[i]) and tuple(disp[i]) == (0, 0, 0)
        else:
            assert valid[i] == 1 and tuple(disp[i]) == bd
            assert ncc[i] == pytest.approx(best, abs=1e-12)


def _brute_select(pre, mask, bl, stride, frac):
    nz, ny, nx = pre.shape
    cands = []
    for z in range(0, nz, stride):
        for y in range(0, ny, stride):
            for x in range(0, nx, stride):
                if not _inside((nx, ny, nz), (x, y, z), bl) or mask[z, y, x] == 0:
                    continue
                vals = [int(v) for v in _block(pre, (x, y, z), bl).ravel()]
                cands.append((len(vals) * sum(v * v for v in vals) - sum(vals) ** 2, (z * ny + y) * nx + x, (x, y, z)))
    nsel = math.floor(0.5 + len(cands) * frac)
    pos = sorted([c for c in cands if c[0] > 0], key=lambda c: (-c[0], c[1]))
    return [c[2] for c in sorted(pos[:nsel], key=lambda c: c[1])], len(cands)


@pytest.mark.parametrize("bl,stride,frac", [((3, 5, 7), 1, 0.1), ((7, 5, 3), 2, 0.3), ((3, 7, 3), 3, 1.0)])
def test_selection_equals_brute_force(bl, stride, frac):
    dims = (19, 16, 14)
    pre = synth.random_u16(dims, 16, hi=64)  # small range: many tied keys
    pre[:, :, :4] = 9  # flat slab: key 0, never selected
    mask = synth.ellipsoid_mask(dims, 0.48)
    got, nc = oracle.select_blocks(pre, mask, bl, stride, frac)
    ref, nc_ref = _brute_select(pre, mask, bl, stride, frac)
    assert nc == nc_ref
    assert [tuple(c) for c in got] == ref


def test_cubic_triple_is_the_cubic_path():
    pre, intra, mask = synth.workload_pair("small")
    c1, n1 = oracle.select_blocks(pre, mask, 5, 2, 0.05)
    c3, n3 = oracle.select_blocks(pre, mask, (5, 5, 5), 2, 0.05)
    assert n1 == n3 and np.array_equal(c1, c3)
    a = oracle.match(pre, intra, c1[::4], 5, (2, 1, 2))
    b = oracle.match(pre, intra, c1[::4], (5, 5, 5), (2, 1, 2))
    for x, y in zip(a, b):
        assert np.array_equal(x, y, equal_nan=True)


@pytest.mark.parametrize("bl", [(3, 5, 7), (7, 5, 3)])
def test_axis_permutation_symmetry(bl):
    # swapping the x and z axes of both volumes, the block edges, the radii
    # and the centres swaps the x and z displacement components; the sums
    # are the same integers, so the NCC values are bit-identical
    pre = synth.random_u16(DIMS, 17, hi=4096)
    intra = synth.random_u16(DIMS, 18, hi=4096)
    h = _half(bl)
    nx, ny, nz = DIMS
    centers = np.array([(x, y, z) for z in range(h[2], nz - h[2], 2) for y in range(h[1], ny - h[1], 2)
                        for x in range(h[0], nx - h[0], 3)], dtype=np.int32)
    r = (2, 1, 1)
    d1, s1, v1 = oracle.match(pre, intra, centers, bl, r)
    preT = np.ascontiguousarray(pre.transpose(2, 1, 0))
    intraT = np.ascontiguousarray(intra.transpose(2, 1, 0))
    d2, s2, v2 = oracle.match(preT, intraT, centers[:, ::-1].copy(), bl[::-1], r[::-1])
    assert np.array_equal(v1, v2)
    ok = v1 == 1
    assert np.array_equal(s1[ok], s2[ok])
    # the displacement agrees unless the tie-break decided between equal
    # scores (its lexicographic part is not symmetric under the swap)
    same = (d1 == d2[:, ::-1]).all(axis=1)
    assert same[ok].mean() > 0.99
    # a wrong axis in the block extent would change the sums: compare with
    # the block rotated the wrong way on the same volume
    d3, s3, _ = oracle.match(pre, intra, centers, bl[::-1], r)
    assert not np.array_equal(s1, s3)


def test_known_translation_with_anisotropic_block():
    pre, _, mask = synth.workload_pair("small")
    t = (2, -1, 1)
    intra = synth.translate(pre, t)
    bl = (7, 5, 3)
    centers, _ = oracle.select_blocks(pre, mask, bl, 2, 0.10)
    centers = centers[::5]
    disp, ncc, valid = oracle.match(pre, intra, centers, bl, (3, 2, 2))
    nz, ny, nx = pre.shape
    checked = 0
    for i, c in enumerate(centers):
        if _inside((nx, ny, nz), tuple(int(c[k]) + t[k] for k in range(3)), bl):
            assert tuple(disp[i]) == t and ncc[i] == 1.0
            checked += 1
    assert checked > 20
