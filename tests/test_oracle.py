"""Pins of the CPU oracle to things other than itself (CPU only).

Each test checks the oracle against what the paper and the mathematics fix:
a library routine (numpy.corrcoef, numpy.var), brute force in Python on tiny
inputs, closed forms (a known integer translation), and invariants of the
NCC (self-match, affine maps of intensity).  Together they catch a dropped
term, a wrong sign, a swapped axis or operand, an off-by-one in the block or
window extent and a wrong tie-break.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_2308_10868_gb300 import synth


def _block(vol, c, b):
    h = (b - 1) // 2
    x, y, z = c
    return vol[z - h:z + h + 1, y - h:y + h + 1, x - h:x + h + 1]


def _inside(dims, c, b):
    h = (b - 1) // 2
    return all(h <= c[i] <= dims[i] - 1 - h for i in range(3))


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


def _brute_match(pre, intra, centers, b, r):
    """numpy brute force: Pearson via numpy.corrcoef over every shift."""
    nz, ny, nx = pre.shape
    dims = (nx, ny, nz)
    out = []
    for c in centers:
        best, bd = None, (0, 0, 0)
        if _inside(dims, c, b):
            I = _block(pre, c, b).astype(np.float64).ravel()
            for d in _shifts(r):
                cd = tuple(int(c[i]) + d[i] for i in range(3))
                if not _inside(dims, cd, b):
                    continue
                J = _block(intra, cd, b).astype(np.float64).ravel()
                if I.std() == 0 or J.std() == 0:
                    continue
                s = float(np.corrcoef(I, J)[0, 1])
                if best is None or _t1_better(s, d, best, bd):
                    best, bd = s, d
        out.append((bd, best))
    return out


DIMS_TINY = (13, 11, 9)  # nx != ny != nz so a swapped axis shows


@pytest.mark.parametrize("b,r", [(3, (1, 1, 1)), (3, (2, 1, 1)), (5, (1, 2, 0))])
def test_ncc_equals_numpy_corrcoef_every_shift(b, r):
    pre = synth.random_u16(DIMS_TINY, 1)
    intra = synth.random_u16(DIMS_TINY, 2)
    h = (b - 1) // 2
    nx, ny, nz = DIMS_TINY
    n = 0
    for c in [(h, h, h), (nx // 2, ny // 2, nz // 2), (nx - 1 - h, ny - 1 - h, nz - 1 - h), (h + 1, ny - 2 - h, h)]:
        for d in _shifts(r):
            v = oracle.ncc_u16(pre, intra, b, c, d)
            cd = tuple(c[i] + d[i] for i in range(3))
            if not _inside(DIMS_TINY, cd, b):
                assert v is None
                continue
            I = _block(pre, c, b).astype(np.float64).ravel()
            J = _block(intra, cd, b).astype(np.float64).ravel()
            ref = float(np.corrcoef(I, J)[0, 1])
            assert v == pytest.approx(ref, abs=1e-12)
            # the FP64 two-pass definition agrees with the exact-integer form
            assert oracle.pearson_u16(pre, intra, b, c, d) == pytest.approx(v, abs=1e-12)
            # float32 inputs holding the same integers give the same value
            fv = oracle.pearson_f32(pre.astype(np.float32), intra.astype(np.float32), b, c, d)
            assert fv == pytest.approx(v, abs=1e-12)
            n += 1
    assert n > 10


@pytest.mark.parametrize("b,r", [(3, (1, 1, 1)), (3, (1, 2, 1)), (5, (2, 1, 1))])
def test_match_equals_brute_force(b, r):
    pre = synth.random_u16(DIMS_TINY, 3, hi=4096)
    intra = synth.random_u16(DIMS_TINY, 4, hi=4096)
    h = (b - 1) // 2
    nx, ny, nz = DIMS_TINY
    centers = np.array([(x, y, z) for z in range(h, nz - h, 2) for y in range(h, ny - h, 3) for x in range(h, nx - h, 3)]
                       + [(0, 5, 4), (nx - 1, 5, 4)], dtype=np.int32)
    disp, ncc, valid = oracle.match(pre, intra, centers, b, r)
    ref = _brute_match(pre, intra, centers, b, r)
    for i, (bd, best) in enumerate(ref):
        if best is None:
            assert valid[i] == 0 and np.isnan(ncc[i]) and tuple(disp[i]) == (0, 0, 0)
        else:
            assert valid[i] == 1
            assert tuple(disp[i]) == bd
            assert ncc[i] == pytest.approx(best, abs=1e-12)
    assert valid.sum() >= len(centers) - 2


def test_tie_break_prefers_small_shift_then_lexicographic():
    nx, ny, nz = 16, 12, 10
    z, y, x = np.ogrid[0:nz, 0:ny, 0:nx]
    # constant along x, non-affine in y and z: every dx ties, dy/dz decide
    pre = np.broadcast_to((100 + 7 * y * y + 5 * z * z).astype(np.uint16), (nz, ny, nx)).copy()
    centers = np.array([[8, 6, 5]], dtype=np.int32)
    disp, ncc, valid = oracle.match(pre, pre, centers, 3, (2, 1, 1))
    assert valid[0] == 1 and ncc[0] == 1.0
    assert tuple(disp[0]) == (0, 0, 0)
    intra = synth.translate(pre, (0, 1, 0))
    disp, ncc, valid = oracle.match(pre, intra, centers, 3, (2, 1, 1))
    assert tuple(disp[0]) == (0, 1, 0) and ncc[0] == 1.0
    assert _brute_match(pre, intra, centers, 3, (2, 1, 1))[0][0] == (0, 1, 0)
    # period 2 along x, content moved by +1 in x: d=(-1,0,0) and (+1,0,0)
    # both match exactly with equal |d|^2; lexicographic order picks dx=-1
    pre2 = (100 + 50 * (x % 2) + 7 * y * y + 5 * z * z).astype(np.uint16)
    pre2 = np.broadcast_to(pre2, (nz, ny, nx)).copy()
    intra2 = synth.translate(pre2, (1, 0, 0))
    disp, ncc, valid = oracle.match(pre2, intra2, centers, 3, (2, 1, 1))
    assert tuple(disp[0]) == (-1, 0, 0) and ncc[0] == 1.0


def _small_phantom():
    pre, intra, mask = synth.workload_pair("small")
    return pre, intra, mask


def test_self_match_is_exactly_one_at_zero():
    pre, _, mask = _small_phantom()
    centers, _ = oracle.select_blocks(pre, mask, 7, 2, 0.10)
    centers = centers[::7]
    disp, ncc, valid = oracle.match(pre, pre, centers, 7, 2)
    assert valid.all()
    assert (disp == 0).all()
    assert (ncc == 1.0).all()  # sqrt(RN(v*v)) == v in binary64


def test_known_translation_is_recovered_exactly():
    pre, _, mask = _small_phantom()
    t = (2, -1, 1)
    intra = synth.translate(pre, t)
    centers, _ = oracle.select_blocks(pre, mask, 7, 2, 0.10)
    centers = centers[::5]
    disp, ncc, valid = oracle.match(pre, intra, centers, 7, 3)
    nz, ny, nx = pre.shape
    checked = 0
    for i, c in enumerate(centers):
        if _inside((nx, ny, nz), tuple(c[k] + t[k] for k in range(3)), 7):
            assert tuple(disp[i]) == t and ncc[i] == 1.0
            checked += 1
    assert checked > 20


def test_affine_maps_of_intensity():
    pre, intra, mask = _small_phantom()
    pre = (pre // 4).astype(np.uint16)
    intra = (intra // 4).astype(np.uint16)
    assert int(intra.max()) * 4 + 7 <= 65535
    centers, _ = oracle.select_blocks(pre, mask, 7, 2, 0.10)
    centers = centers[::9]
    d0, n0, v0 = oracle.match(pre, intra, centers, 7, 2)
    # power-of-two gain: bit-identical
    for a in (2, 4):
        d1, n1, v1 = oracle.match(pre, (intra * a).astype(np.uint16), centers, 7, 2)
        assert (d1 == d0).all() and (v1 == v0).all()
        assert np.array_equal(n1.view(np.int64), n0.view(np.int64))
    # gain 3 with offset: same displacements, NCC within rounding
    d3, n3, v3 = oracle.match(pre, (intra * 3 + 7).astype(np.uint16), centers, 7, 2)
    assert (d3 == d0).all() and (v3 == v0).all()
    np.testing.assert_allclose(n3, n0, rtol=0, atol=1e-15)
    # negative gain: NCC negated exactly at every shift
    neg = (65535 - intra).astype(np.uint16)
    for c in centers[:5]:
        for d in _shifts((2, 2, 2)):
            a_ = oracle.ncc_u16(pre, intra, 7, c, d)
            b_ = oracle.ncc_u16(pre, neg, 7, c, d)
            assert (a_ is None and b_ is None) or b_ == -a_
    # a positive affine map of the pre-operative volume keeps the selection
    c2, _ = oracle.select_blocks((pre * 3 + 11).astype(np.uint16), mask, 7, 2, 0.10)
    c1, _ = oracle.select_blocks(pre, mask, 7, 2, 0.10)
    assert np.array_equal(c1, c2)


def test_block_key_is_n_squared_times_variance():
    vol = synth.random_u16((12, 10, 9), 5)
    for b in (3, 5, 7):
        h = (b - 1) // 2
        for c in [(h, h, h), (6, 5, 4), (11 - h, 9 - h, 8 - h)]:
            k = oracle.block_key(vol, b, *c)
            blk = _block(vol, c, b).astype(np.float64)
            assert k == pytest.approx(blk.size ** 2 * blk.var(), rel=1e-12)
            # exact integer form, computed independently in Python ints
            vals = [int(v) for v in blk.ravel()]
            assert k == len(vals) * sum(v * v for v in vals) - sum(vals) ** 2


@pytest.mark.parametrize("nc,frac,expect", [(10, 0.25, 3), (10, 0.24, 2), (10, 0.05, 1), (10, 0.04, 0),
                                            (387, 0.05, 19), (1000, 0.1, 100), (7, 1.0, 7), (0, 0.5, 0)])
def test_selection_count_rounds_half_up(nc, frac, expect):
    assert oracle.n_select(nc, frac) == expect == math.floor(0.5 + nc * frac)


def _brute_select(pre, mask, b, stride, frac):
    nz, ny, nx = pre.shape
    h = (b - 1) // 2
    cands = []
    for z in range(0, nz, stride):
        for y in range(0, ny, stride):
            for x in range(0, nx, stride):
                if not (h <= x <= nx - 1 - h and h <= y <= ny - 1 - h and h <= z <= nz - 1 - h):
                    continue
                if mask[z, y, x] == 0:
                    continue
                vals = [int(v) for v in _block(pre, (x, y, z), b).ravel()]
                key = len(vals) * sum(v * v for v in vals) - sum(vals) ** 2
                cands.append((key, (z * ny + y) * nx + x, (x, y, z)))
    nsel = math.floor(0.5 + len(cands) * frac)
    pos = sorted([c for c in cands if c[0] > 0], key=lambda c: (-c[0], c[1]))
    chosen = sorted(pos[:nsel], key=lambda c: c[1])
    return [c[2] for c in chosen], len(cands)


@pytest.mark.parametrize("b,stride,frac", [(3, 2, 0.1), (3, 1, 0.05), (5, 2, 0.3), (3, 3, 1.0)])
def test_selection_equals_brute_force(b, stride, frac):
    dims = (17, 14, 12)
    pre = synth.random_u16(dims, 6, hi=64)  # small range: many tied keys
    pre[:, :, :4] = 9  # a flat slab: key 0, never selected
    mask = synth.ellipsoid_mask(dims, 0.48)
    got, nc = oracle.select_blocks(pre, mask, b, stride, frac)
    ref, nc_ref = _brute_select(pre, mask, b, stride, frac)
    assert nc == nc_ref
    assert [tuple(c) for c in got] == ref


def test_selection_fractions_are_nested():
    pre, _, mask = _small_phantom()
    prev = set()
    for f in (0.02, 0.04, 0.06, 0.08, 0.10):
        c, _ = oracle.select_blocks(pre, mask, 7, 2, f)
        cur = set(map(tuple, c))
        assert prev <= cur
        prev = cur


def test_invalid_blocks():
    pre = synth.random_u16((12, 12, 12), 8)
    pre[2:9, 2:9, 2:9] = 500  # flat preop block at (5,5,5), b=7
    centers = np.array([[5, 5, 5], [2, 6, 6], [6, 6, 6]], dtype=np.int32)
    disp, ncc, valid = oracle.match(pre, pre, centers, 7, 1)
    assert list(valid) == [0, 0, 1]
    assert np.isnan(ncc[0]) and np.isnan(ncc[1])
    assert (disp[:2] == 0).all()


def test_f32_path_agrees_with_integer_path():
    pre, intra, mask = _small_phantom()
    centers, _ = oracle.select_blocks(pre, mask, 7, 2, 0.10)
    centers = centers[::11]
    d16, n16, v16 = oracle.match(pre, intra, centers, 7, 2)
    d32, n32, v32 = oracle.match(pre.astype(np.float32), intra.astype(np.float32), centers, 7, 2)
    assert (v16 == v32).all()
    np.testing.assert_allclose(n32, n16, rtol=0, atol=1e-12)
    assert (d32 == d16).all()
    # scaled to [0,1] the values move by float32 rounding only
    ds, ns, vs = oracle.match(synth.as_f32(pre), synth.as_f32(intra), centers, 7, 2)
    assert (vs == v16).all()
    np.testing.assert_allclose(ns, n16, rtol=0, atol=1e-5)


# ---------------------------------------------------------------------------
# Selection with a connectivity pattern (Sec. 4.1: face / edge / vertex
# simplex patterns = 6 / 18 / 26 connectivity; greedy in selection order)
# ---------------------------------------------------------------------------
_ORDER = {6: 1, 18: 2, 26: 3}


def _phantom(dims, seed):
    """Smooth Gaussian-blob volume (dims = (nx, ny, nz)) plus a little noise,
    so that block variances vary smoothly with long monotone runs."""
    rng = synth.rng_for(seed, salt=17)
    v = synth.phantom_f64(dims, rng, n_gauss=12, sigma=(2.0, 6.0))
    return synth.to_u16(v + rng.normal(0.0, 3.0, v.shape))


def _pattern_offsets(conn):
    return [o for o in itertools.product((-1, 0, 1), repeat=3) if 0 < sum(map(abs, o)) <= _ORDER[conn]]


@pytest.mark.parametrize("b,stride,frac", [(3, 1, 0.2), (5, 2, 0.5), (3, 3, 1.0)])
def test_spaced_selection_without_pattern_is_plain_selection(b, stride, frac):
    pre = _phantom((26, 24, 22), seed=7)
    mask = np.ones(pre.shape, np.uint8)
    mask[:, :, :4] = 0
    plain, nc = oracle.select_blocks(pre, mask, b, stride, frac)
    spaced, nc2 = oracle.select_blocks_spaced(pre, mask, b, stride, frac, 0)
    assert nc == nc2 and np.array_equal(plain, spaced)


@pytest.mark.parametrize("stride", [1, 2])
@pytest.mark.parametrize("conn", [6, 18, 26])
def test_spaced_selection_equal_keys_gives_the_closed_form_lattice(conn, stride):
    # I = 1000 + 300*(x mod 3): every 3^3 block holds the same multiset of
    # values, so every candidate has the same positive key and the selection
    # order is the raster order.  Greedy exclusion in raster order then keeps,
    # in grid coordinates relative to the first candidate (a, a, a):
    #   face (6):    (u+v+w) even
    #   edge (18):   u = v = w (mod 2)
    #   vertex (26): u, v, w all even
    # (densities 1/2, 1/4, 1/8: the face pattern is the densest).
    nz, ny, nx = 13, 14, 15
    x = np.arange(nx)
    pre = np.broadcast_to(1000 + 300 * (x % 3), (nz, ny, nx)).astype(np.uint16).copy()
    mask = np.ones((nz, ny, nx), np.uint8)
    got, nc = oracle.select_blocks_spaced(pre, mask, 3, stride, 1.0, conn)
    keys, _ = oracle.grid_keys(pre, mask, 3, stride)
    cand = np.argwhere(keys >= 0)  # (k, j, i)
    assert len(cand) == nc and len(np.unique(keys[keys >= 0])) == 1 and keys.max() > 0
    a = cand.min(axis=0)
    u, v, w = (cand - a).T
    keep = {6: (u + v + w) % 2 == 0, 18: ((u % 2) == (v % 2)) & ((v % 2) == (w % 2)),
            26: (u % 2 == 0) & (v % 2 == 0) & (w % 2 == 0)}[conn]
    kji = cand[keep]
    expect = np.stack([kji[:, 2], kji[:, 1], kji[:, 0]], axis=1) * stride
    order = np.lexsort((expect[:, 0], expect[:, 1], expect[:, 2]))
    assert np.array_equal(got, expect[order].astype(np.int32))
    # a smaller fraction keeps the first n_sel lattice points in raster order
    frac = 0.1
    part, _ = oracle.select_blocks_spaced(pre, mask, 3, stride, frac, conn)
    assert np.array_equal(part, expect[order][:oracle.n_select(nc, frac)].astype(np.int32))


def _selection_ranks(keys):
    """Rank of every candidate with a positive key in selection order (key
    descending, raster index ascending), keyed by its grid point (k, j, i)."""
    gz, gy, gx = keys.shape
    flat = [(int(keys[k, j, i]), (k * gy + j) * gx + i, (int(k), int(j), int(i))) for k, j, i in np.argwhere(keys > 0)]
    flat.sort(key=lambda t: (-t[0], t[1]))
    return {kji: r for r, (_, _, kji) in enumerate(flat)}


def _greedy_violation(S, rank, conn, want):
    """Why the grid-point set S is not the greedy selection with pattern
    `conn` truncated at `want` members, or None if it is.  The greedy result
    is characterised by: (1) no two members of S are pattern neighbours;
    (2) |S| = min(want, size of the full greedy set); (3) every unselected
    candidate with a positive key that precedes the last member of S in
    selection order (or any, if |S| < want) has a member of S among its
    neighbours that precedes it.  Any set with these properties equals the
    greedy one (a first difference contradicts (1))."""
    offs = _pattern_offsets(conn)

    def nbrs(p):
        for o in offs:
            q = (p[0] + o[2], p[1] + o[1], p[2] + o[0])
            if q in rank:
                yield q

    for p in S:  # (1)
        if p not in rank:
            return f"{p} is not a candidate with a positive key"
        if any(q in S for q in nbrs(p)):
            return f"{p} has a selected neighbour"
    if len(S) > want:
        return f"{len(S)} selected, more than {want}"
    last = max(rank[p] for p in S) if S else -1
    for p, r in rank.items():  # (3)
        if p in S or (len(S) == want and r > last):
            continue
        if not any(q in S and rank[q] < r for q in nbrs(p)):
            return f"{p} was skipped without an earlier selected neighbour"
    if len(S) < want and not all(p in S or any(q in S for q in nbrs(p)) for p in rank):  # (2)
        return "the walk stopped short with candidates left to add"
    return None


@pytest.mark.parametrize("conn", [6, 18, 26])
@pytest.mark.parametrize("b,stride,frac", [(3, 1, 0.08), (3, 2, 0.3), (5, 1, 1.0), (5, 3, 0.2)])
def test_spaced_selection_is_the_greedy_independent_set(conn, b, stride, frac):
    pre = _phantom((30, 27, 25), seed=11 + conn)
    mask = np.zeros(pre.shape, np.uint8)
    mask[3:-3, 2:-2, 4:-1] = 1
    got, nc = oracle.select_blocks_spaced(pre, mask, b, stride, frac, conn)
    keys, _ = oracle.grid_keys(pre, mask, b, stride)
    rank = _selection_ranks(keys)
    S = {(int(c[2]) // stride, int(c[1]) // stride, int(c[0]) // stride) for c in got}
    assert len(S) == len(got)
    assert _greedy_violation(S, rank, conn, oracle.n_select(nc, frac)) is None


def _walk(rank, conn, want, mistake=None):
    """The greedy walk in selection order, written out in Python, with an
    optional planted mistake: "order" uses the next larger neighbourhood for
    the exclusion (face -> edge, edge -> vertex, vertex -> face), "stop"
    takes one member past `want`, "taken" marks a skipped candidate as taken
    too (so it blocks its later neighbours)."""
    use = {6: 18, 18: 26, 26: 6}[conn] if mistake == "order" else conn
    offs = _pattern_offsets(use)
    taken, S = set(), set()
    limit = want + 1 if mistake == "stop" else want
    for p, _ in sorted(rank.items(), key=lambda t: t[1]):
        if len(S) >= limit:
            break
        blocked = any((p[0] + o[2], p[1] + o[1], p[2] + o[0]) in taken for o in offs)
        if not blocked:
            S.add(p)
            taken.add(p)
        elif mistake == "taken":
            taken.add(p)
    return S


@pytest.mark.parametrize("conn", [6, 18, 26])
def test_greedy_checks_catch_planted_mistakes(conn):
    # The characterisation above must accept the correct walk (which must
    # equal the oracle's selection) and reject each planted mistake: an
    # exclusion neighbourhood one order off, a walk that does not stop at
    # n_sel, a skipped candidate wrongly marked taken.
    pre = _phantom((30, 27, 25), seed=23 + conn)
    mask = np.zeros(pre.shape, np.uint8)
    mask[3:-3, 2:-2, 4:-1] = 1
    b, stride, frac = 3, 1, 0.08
    got, nc = oracle.select_blocks_spaced(pre, mask, b, stride, frac, conn)
    keys, _ = oracle.grid_keys(pre, mask, b, stride)
    rank = _selection_ranks(keys)
    want = oracle.n_select(nc, frac)
    good = _walk(rank, conn, want)
    assert good == {(int(c[2]) // stride, int(c[1]) // stride, int(c[0]) // stride) for c in got}
    assert _greedy_violation(good, rank, conn, want) is None
    for mistake in ("order", "stop", "taken"):
        bad = _walk(rank, conn, want, mistake)
        assert bad != good, mistake
        assert _greedy_violation(bad, rank, conn, want) is not None, mistake


@pytest.mark.parametrize("conn", [6, 26])
def test_spaced_selection_fractions_are_nested(conn):
    pre = _phantom((28, 26, 24), seed=5)
    mask = np.ones(pre.shape, np.uint8)
    prev = set()
    for frac in (0.01, 0.03, 0.07, 0.2):
        s, _ = oracle.select_blocks_spaced(pre, mask, 3, 1, frac, conn)
        cur = {tuple(c) for c in s.tolist()}
        assert prev <= cur
        prev = cur
