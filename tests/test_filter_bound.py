"""The match kernel's filter, checked on the CPU: for uint16 inputs the
kernel scores every shift with an FP32 correlation and keeps for exact
rescoring only the shifts whose upper bound reaches the best lower bound.
That is exact only if, at every shift, the approximate NCC v and its bound e
satisfy |v - NCC| <= e, NCC being the exact Pearson correlation (Sec. 3, the
NCC equation).  This test emulates the kernel's float32 arithmetic in numpy,
operation by operation and in the kernel's order: the window values enter
centred by the floating block's integer mean m (the kernel forms them as the
subnormals (u - m) * 2^-149 and scales the template by 2^64, a power-of-two
rescaling that leaves every rounding unchanged, so the emulation works in
units of one), one chain of N FMAs per shift, then the box-sum terms and the
bound, each operation rounded on its own as the kernel writes it; rsqrt.approx and sqrt.approx are replaced by the exact value
perturbed to the edges of their 2^-22 relative error.  The inequality is
checked on data chosen to stress it: smooth blocks, full-range noise,
near-flat blocks with a large mean, two-level blocks and near-perfect
matches, with the FMA chain taken in both orders the kernel uses (template
rows innermost along y, or along z).  The float32 path's bound is checked the
same way further down.
"""
import numpy as np
import pytest

U = np.float32(2.0 ** -24)
F = np.float32


def f32(x):
    return np.asarray(x, dtype=np.float64).astype(np.float32)


def fma32(a, b, c):
    # a*b is exact in float64 (24 + 24 bits); one rounding to float64, then to float32
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float32)


def round_up32(x):
    f = np.float32(x)
    return f if float(f) >= x else np.nextafter(f, np.float32(np.inf))


def approx(exact64, delta):
    # an approximate unit with relative error |delta| <= 2^-22
    return f32(exact64 * (1.0 + delta))


def _chain(T, W, P, order):
    """A(d) = sum_k T_k W_{k+d} as one FMA chain per shift, the template
    walked in the kernel's order: planes outside, rows, then columns
    ("zyx"), or rows outside, planes, then columns ("yzx")."""
    bz, by, bx = T.shape
    acc = np.zeros((P, P, P), np.float32)
    outer, inner = (bz, by) if order == "zyx" else (by, bz)
    for o in range(outer):
        for i in range(inner):
            kz, ky = (o, i) if order == "zyx" else (i, o)
            for kx in range(bx):
                acc = fma32(np.full((P, P, P), T[kz, ky, kx], np.float32), W[kz:kz + P, ky:ky + P, kx:kx + P], acc)
    return acc


def kernel_bound(I, W, R, delta_rsqrt, delta_sqrt, order="zyx"):
    """Approximate NCC v, bound e and exact NCC for every shift of the block
    I (b^3, uint16 values) in the window W ((b+2R)^3), all shifts inside."""
    b = I.shape[0]
    N = b ** 3
    P = 2 * R + 1
    I64 = I.astype(np.int64)
    S_I, S_II = int(I64.sum()), int((I64 * I64).sum())
    vI = N * S_II - S_I * S_I
    m = (2 * S_I + N) // (2 * N)  # nearest integer to the block mean
    rr = N * m - S_I
    qt = int(((I64 - m) ** 2).sum())
    T = (I64 - m).astype(np.float32)  # exact
    Jc = (W.astype(np.int64) - m).astype(np.float32)  # exact
    acc = _chain(T, Jc, P, order)
    # exact sums per shift
    W64 = W.astype(np.int64)
    S_J = np.zeros((P, P, P), np.int64)
    S_JJ = np.zeros((P, P, P), np.int64)
    S_IJ = np.zeros((P, P, P), np.int64)
    for dz in range(P):
        for dy in range(P):
            for dx in range(P):
                blk = W64[dz:dz + b, dy:dy + b, dx:dx + b]
                S_J[dz, dy, dx] = blk.sum()
                S_JJ[dz, dy, dx] = (blk * blk).sum()
                S_IJ[dz, dy, dx] = (blk * I64).sum()
    vJ = N * S_JJ - S_J * S_J
    num = N * S_IJ - S_I * S_J
    with np.errstate(invalid="ignore", divide="ignore"):
        ncc = num.astype(np.float64) / np.sqrt(float(vI) * vJ.astype(np.float64))
    # the bound, as the kernel evaluates it (uint16 path)
    fN = F(N)
    GAMMA_N = N * 2.0 ** -24 / (1.0 - N * 2.0 ** -24)
    qf = F(qt)
    kq = round_up32(float(round_up32(float(F(N * GAMMA_N)) * float(round_up32(np.sqrt(float(qf)))))) * 1.000004)
    fvI, frr = F(vI), F(rr)
    vjf = f32(vJ)
    s1f = f32(S_J - N * m)
    inv_n = F(1.0) / fN
    s2u = (fma32(s1f, s1f, vjf) * inv_n) * (F(1.0) + F(16.0) * U)
    with np.errstate(invalid="ignore", divide="ignore"):
        inv = approx(1.0 / np.sqrt((fvI * vjf).astype(np.float64)), delta_rsqrt)
    na = acc * fN
    rs = frr * s1f
    v = (na + rs) * inv
    sq = approx(np.sqrt(s2u.astype(np.float64)), delta_sqrt)
    t1 = (kq * sq) * inv
    t2 = ((F(4.0) * U) * (np.abs(na) + np.abs(rs))) * inv
    e = (t1 + t2) * (F(1.0) + F(64.0) * U) + (F(40.0) * U) * np.abs(v)
    e = F(2.0) * e + F(1e-9)
    valid = vjf > 0
    return v.astype(np.float64), e.astype(np.float64), ncc, valid


def _smooth(rng, shape, lo, hi):
    z, y, x = np.meshgrid(*[np.arange(s) for s in shape], indexing="ij")
    f = np.zeros(shape)
    for _ in range(6):
        cz, cy, cx = (rng.uniform(0, s) for s in shape)
        sg = rng.uniform(2, 6)
        f += rng.uniform(-1, 1) * np.exp(-((z - cz) ** 2 + (y - cy) ** 2 + (x - cx) ** 2) / (2 * sg * sg))
    f = (f - f.min()) / (np.ptp(f) + 1e-12)
    return np.rint(lo + (hi - lo) * f).astype(np.uint16)


def _cases():
    rng = np.random.default_rng(20231)
    b, R = 7, 3
    w = b + 2 * R
    cases = []
    W = _smooth(rng, (w, w, w), 500, 4000)
    cases.append(("smooth", W[R:R + b, R:R + b, R:R + b].copy(), W))
    W2 = np.clip(W.astype(np.int64) + rng.normal(0, 30, W.shape).round().astype(np.int64), 0, 65535).astype(np.uint16)
    cases.append(("smooth + noise, matching block", W[R + 1:R + 1 + b, R:R + b, R - 1:R - 1 + b].copy(), W2))
    cases.append(("full-range noise", rng.integers(0, 65536, (b, b, b), dtype=np.uint16),
                  rng.integers(0, 65536, (w, w, w), dtype=np.uint16)))
    cases.append(("near-flat, large mean", (40000 + rng.integers(-3, 4, (b, b, b))).astype(np.uint16),
                  (40000 + rng.integers(-3, 4, (w, w, w))).astype(np.uint16)))
    cases.append(("two-level extremes", (65535 * rng.integers(0, 2, (b, b, b))).astype(np.uint16),
                  (65535 * rng.integers(0, 2, (w, w, w))).astype(np.uint16)))
    cases.append(("self-match", W[R:R + b, R:R + b, R:R + b].copy(), W))
    return cases, R


@pytest.mark.parametrize("order", ["zyx", "yzx"])
@pytest.mark.parametrize("delta_rsqrt,delta_sqrt", [(2.0 ** -22, 2.0 ** -22), (-2.0 ** -22, -2.0 ** -22),
                                                      (2.0 ** -22, -2.0 ** -22), (0.0, 0.0)])
def test_filter_bound_covers_the_error(delta_rsqrt, delta_sqrt, order):
    cases, R = _cases()
    for name, I, W in cases:
        v, e, ncc, valid = kernel_bound(I, W, R, delta_rsqrt, delta_sqrt, order)
        assert valid.any(), name
        err = np.abs(v - ncc)[valid]
        assert (err <= e[valid]).all(), (name, float((err - e[valid]).max()))


def test_filter_bound_is_tight_enough_to_filter():
    """The bound is a worst case (about fifty times the error seen here), but
    it stays small against the spread of the NCC values, so one shift
    survives on each case; and it is within a hundredfold of the error
    actually made, so a bound a hundred times smaller would be violated (the
    covering test above can fail)."""
    cases, R = _cases()
    for name, I, W in cases:
        v, e, ncc, valid = kernel_bound(I, W, R, 2.0 ** -22, 2.0 ** -22)
        lb = (v - e)[valid].max()
        survivors = int(((v + e)[valid] >= lb).sum())
        assert e[valid].max() < 1e-3, (name, e[valid].max())
        assert survivors <= 3, (name, survivors)
    name, I, W = cases[0]
    v, e, ncc, valid = kernel_bound(I, W, R, 2.0 ** -22, 2.0 ** -22)
    assert (np.abs(v - ncc)[valid] > e[valid] / 100).any()


# ---------------------------------------------------------------------------
# float32 intensities: the same check for the float32 path's bound, which also
# covers the rounding of the inputs' centring, of the float box sums (three
# levels of b-term sums of J - c, c the reference volume's centre value) and
# of the float block constants; shifts whose reference spread the float sums
# cannot resolve are rescored unconditionally (no bound is claimed for them).
# ---------------------------------------------------------------------------
def _box_f32(blk):
    """Sum of a b^3 float32 block as the box kernel forms it: b terms along
    x, then b of those along y, then b along z, each level in float32."""
    sx = blk[:, :, 0].copy()
    for x in range(1, blk.shape[2]):
        sx = sx + blk[:, :, x]
    sy = sx[:, 0].copy()
    for y in range(1, blk.shape[1]):
        sy = sy + sx[:, y]
    sz = sy[0]
    for z in range(1, blk.shape[0]):
        sz = sz + sy[z]
    return np.float32(sz)


def kernel_bound_f32(I, W, R, delta_rsqrt, delta_sqrt, cv=None):
    """cv: the box sums' centre c (the reference volume's centre value; by
    default the window's centre voxel here)."""
    bz, by, bx = I.shape  # a block with an edge per axis: the box-sum depth is bx + by + bz
    N = bx * by * bz
    P = 2 * R + 1
    fN = F(N)
    # block constants (the kernel sums I - I0 in float-float: about 2^-48
    # relative, taken here as exact)
    i0 = I[0, 0, 0]
    d = I.astype(np.float64) - float(i0)
    s1, s2 = float(d.sum()), float((d * d).sum())
    tsh = i0 + F(s1) * (F(1.0) / fN)  # any float near the mean
    ibar = float(i0) + s1 / N
    dv = max(s2 - s1 * (s1 / N), 0.0)
    em = ibar - float(tsh)
    emu, fvI = F(em), F(dv)
    # bound on emu's error beyond 2u |emu|, as the kernel forms it
    eI = F(np.nextafter(np.float32((2.0 ** -36 * np.sqrt(N * s2) / N + 2.0 ** -52 * (abs(float(i0)) + abs(s1) / N)) * 1.01),
                        np.float32(np.inf)))
    kq = F(np.sqrt((dv + 2048.0 * 1.1102230246251565e-16 * s2 + N * em * em) * (1.0 + 2.4e-7)) * (1.0 + 1e-6))
    T = I - tsh  # float32, rounded as in the kernel
    # float box sums of J - c and (J - c)^2 at every shift (J - c rounded
    # once, its square once), and the centring constant
    if cv is None:
        cv = W[W.shape[0] // 2, W.shape[1] // 2, W.shape[2] // 2]
    cv = F(cv)
    S1 = np.zeros((P, P, P), np.float32)
    S2 = np.zeros((P, P, P), np.float32)
    for dz in range(P):
        for dy in range(P):
            for dx in range(P):
                blk = (W[dz:dz + bz, dy:dy + by, dx:dx + bx] - cv).astype(np.float32)
                S1[dz, dy, dx] = _box_f32(blk)
                S2[dz, dy, dx] = _box_f32(blk * blk)
    c_f = tsh  # centring constant: the float mean
    Jc = W - c_f  # float32, rounded as in the kernel
    acc = _chain(T, Jc, P, "zyx")
    # exact Pearson correlation of the float values (two-pass, float64)
    I64 = I.astype(np.float64) - I.astype(np.float64).mean()
    ncc = np.full((P, P, P), np.nan)
    for dz in range(P):
        for dy in range(P):
            for dx in range(P):
                J64 = W[dz:dz + bz, dy:dy + by, dx:dx + bx].astype(np.float64)
                J64 = J64 - J64.mean()
                den = np.sqrt((I64 * I64).sum() * (J64 * J64).sum())
                if den > 0:
                    ncc[dz, dy, dx] = (I64 * J64).sum() / den
    # the bound, as the kernel evaluates it (float32 path): every operation
    # rounded on its own, in the kernel's order
    depth = bx + by + bz + 3  # the levels, the rounding of J - c and of its square
    GS = F(depth * 2.0 ** -24 / (1.0 - depth * 2.0 ** -24))
    GN = F(N * 2.0 ** -24 / (1.0 - N * 2.0 ** -24))
    s1b, s2b = S1, np.maximum(S2, F(0.0))
    d1 = approx(np.sqrt((fN * s2b).astype(np.float64)), delta_sqrt)
    d1 = (GS * d1) * F(1.01)
    s1sq_n = (s1b * s1b) * (F(1.0) / fN)
    vJa = s2b - s1sq_n
    dvJ = (GS * s2b + ((F(2.0) * np.abs(s1b) + d1) * d1) / fN) + (F(4.0) * U) * (s2b + s1sq_n)
    dl = c_f - cv
    s1p = s1b - fN * dl
    m2 = (s2b + (F(2.0) * np.abs(dl)) * np.abs(s1b)) + (fN * dl) * dl
    e2 = (s2b - (F(2.0) * dl) * s1b) + (fN * dl) * dl
    sj2 = (np.maximum(e2, F(0.0)) + ((GS + F(12.0) * U) * m2) * F(1.01)) * (F(1.0) + F(4.0) * U)
    resolved = (vJa - dvJ) > 0
    with np.errstate(invalid="ignore", divide="ignore"):
        rho = dvJ / (vJa - dvJ)
    bounded = resolved & (rho <= F(0.25))
    with np.errstate(invalid="ignore", divide="ignore"):
        inv = approx(1.0 / np.sqrt((fvI * vJa).astype(np.float64)), delta_rsqrt)
    sq = approx(np.sqrt(sj2.astype(np.float64)), delta_sqrt)
    A = acc
    es = emu * s1p
    num = A - es
    v = num * inv
    aem = np.abs(emu)
    ds = d1 + (F(4.0) * U) * (fN * np.abs(dl))
    sb = np.abs(s1p) + ds
    tes = sb * ((F(2.0) * U) * aem + eI) + aem * (ds + (F(2.0) * U) * np.abs(s1p))
    enum = ((((GN + F(3.0) * U) * kq) * sq + tes * F(1.01)) + U * (np.abs(A) + np.abs(es)))
    r1 = (F(1.0) + F(0.7) * rho) + F(4.0) * U
    r2 = F(0.7) * rho + F(6.0) * U
    e = ((enum * inv) * r1 + (np.abs(num) * inv) * r2) * (F(1.0) + F(64.0) * U) + (F(43.0) * U) * np.abs(v)
    e = F(2.0) * e + F(1e-9)
    return v.astype(np.float64), e.astype(np.float64), ncc, bounded & ~np.isnan(ncc)


def _cases_f32():
    cases, R = _cases()
    out = [(name, (I.astype(np.float32) / np.float32(65535.0)), (W.astype(np.float32) / np.float32(65535.0)))
           for name, I, W in cases]
    rng = np.random.default_rng(7)
    b, w = 7, 7 + 2 * R
    # offsets large against the spread: the centring matters (sums of J - c
    # with c on the offset keep the spread at 50x and at 10^5x)
    for off, spread in ((50.0, 1.0), (1000.0, 0.01)):
        I = np.float32(off) + rng.random((b, b, b)).astype(np.float32) * np.float32(spread)
        W = np.float32(off) + rng.random((w, w, w)).astype(np.float32) * np.float32(spread)
        out.append((f"offset {off:g}, spread {spread:g}", I, W))
    return out, R


@pytest.mark.parametrize("centre", ["volume", "zero", "far"])
@pytest.mark.parametrize("delta_rsqrt,delta_sqrt", [(2.0 ** -22, 2.0 ** -22), (-2.0 ** -22, -2.0 ** -22),
                                                      (2.0 ** -22, -2.0 ** -22), (0.0, 0.0)])
def test_filter_bound_f32_covers_the_error(delta_rsqrt, delta_sqrt, centre):
    # c: the volume's centre value (near the data), zero (a volume whose
    # centre is background) or a value far from the data
    cases, R = _cases_f32()
    n_bounded_cases = 0
    for name, I, W in cases:
        cv = {"volume": None, "zero": 0.0, "far": float(W.max()) * 3.0 + 1.0}[centre]
        with np.errstate(invalid="ignore", divide="ignore"):
            v, e, ncc, bounded = kernel_bound_f32(I, W, R, delta_rsqrt, delta_sqrt, cv=cv)
        if not bounded.any():  # spread not resolved: every shift is rescored exactly
            continue
        n_bounded_cases += 1
        err = np.abs(v - ncc)[bounded]
        assert (err <= e[bounded]).all(), (name, centre, float((err - e[bounded]).max()))
    # a c far from the data makes its own offset: fewer cases are resolved
    assert n_bounded_cases >= {"volume": 7, "zero": 6, "far": 4}[centre]


def test_filter_bound_f32_large_offset_is_bounded_with_the_centred_sums():
    # an offset 10^5 times the spread: with c from the volume the spread is
    # resolved and the bound filters (no shift forced to rescoring); with
    # uncentred sums (c = 0) it is not
    cases, R = _cases_f32()
    name, I, W = cases[-1]
    assert name.startswith("offset 1000")
    with np.errstate(invalid="ignore", divide="ignore"):
        v, e, ncc, bounded = kernel_bound_f32(I, W, R, 2.0 ** -22, 2.0 ** -22)
        assert bounded.all()
        lb = (v - e)[bounded].max()
        assert int(((v + e)[bounded] >= lb).sum()) <= 3
        assert not kernel_bound_f32(I, W, R, 2.0 ** -22, 2.0 ** -22, cv=0.0)[3].any()


def test_filter_bound_f32_leaves_few_survivors():
    cases, R = _cases_f32()
    for name, I, W in cases[:2]:
        with np.errstate(invalid="ignore", divide="ignore"):
            v, e, ncc, bounded = kernel_bound_f32(I, W, R, 2.0 ** -22, 2.0 ** -22)
        assert bounded.all(), name  # smooth data: every shift is bounded, none forced to rescoring
        lb = (v - e)[bounded].max()
        assert int(((v + e)[bounded] >= lb).sum()) <= 3, name


def test_filter_bound_f32_blocks_with_an_edge_per_axis():
    rng = np.random.default_rng(11)
    R = 2
    for bz, by, bx in ((3, 5, 9), (9, 7, 3), (11, 3, 5)):
        shape = (bz + 2 * R, by + 2 * R, bx + 2 * R)
        W = _smooth(rng, shape, 200, 3000).astype(np.float32) / np.float32(65535.0)
        W = W + (rng.normal(0, 3, shape) / 65535.0).astype(np.float32)
        I = W[R:R + bz, R:R + by, R:R + bx].copy()
        with np.errstate(invalid="ignore", divide="ignore"):
            v, e, ncc, bounded = kernel_bound_f32(I, W, R, 2.0 ** -22, -2.0 ** -22)
        assert bounded.any()
        err = np.abs(v - ncc)[bounded]
        assert (err <= e[bounded]).all(), ((bz, by, bx), float((err - e[bounded]).max()))
