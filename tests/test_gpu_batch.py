"""Batched parameter search and autotuning (GPU).

Every setting of a batch plan must give exactly what the single-registration
path gives for that setting (and that path is checked against the oracle
elsewhere); two settings per plan are also checked against the oracle
directly.  Graph replay, eager runs and autotuned launch shapes must not
change any bit.
"""
import numpy as np
import pytest

import oracle
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


@pytest.fixture(scope="module")
def pair(nrr):
    pre, intra, mask = synth.workload_pair("small")
    return pre, intra, mask, nrr.to_device_u16(pre), nrr.to_device_u16(intra), torch.from_numpy(mask).cuda()


SETTINGS = [(5, 2, 2, 0.05), (5, 2, 3, 0.05), (7, 2, 3, 0.10), (7, 2, 3, 0.04), (5, 3, (3, 1, 2), 0.08),
            (9, 2, 4, 0.02), (7, 2, 3, 0.10), (5, 2, 2, 0.10)]


def _single(nrr, dpre, dintra, dmask, s):
    b, st, r, f = s
    c = nrr.select_blocks(dpre, dmask, b, st, f)
    d, n, v = nrr.block_match(dpre, dintra, c, b, r)
    return [t.cpu().numpy() for t in (c, d, n, v)]


def _same(a, b):
    return all(np.array_equal(x.view(np.uint8), y.view(np.uint8)) for x, y in zip(a, b))


@pytest.mark.parametrize("graph", [True, False])
def test_batch_equals_single_calls(nrr, pair, graph):
    pre, intra, mask, dpre, dintra, dmask = pair
    plan = nrr.BatchPlan(dpre, dintra, dmask, SETTINGS, graph=graph)
    for rep in range(2):
        plan.run()
        torch.cuda.synchronize()
        nrr.device_status()
        for i, s in enumerate(SETTINGS):
            got = [t.cpu().numpy() for t in plan.result(i)]
            assert _same(got, _single(nrr, dpre, dintra, dmask, s)), (rep, i, s)
    for i in (2, 4):
        b, st, r, f = SETTINGS[i]
        rc, _ = oracle.select_blocks(pre, mask, b, st, f)
        rd, rn, rv = oracle.match(pre, intra, rc, b, r)
        c, d, n, v = [t.cpu().numpy() for t in plan.result(i)]
        assert np.array_equal(c, rc) and np.array_equal(d, rd) and np.array_equal(v, rv)
        assert np.array_equal(n[~np.isnan(n)].view(np.int64), rn[~np.isnan(rn)].view(np.int64))
    plan.close()


def test_batch_more_jobs_than_one_launch_holds(nrr, pair):
    pre, intra, mask, dpre, dintra, dmask = pair
    # 18 strides: 18 matched selections of one (b, R) variant, so two launches
    settings = [(5, st, 2, 0.3) for st in range(1, 19)]
    plan = nrr.BatchPlan(dpre, dintra, dmask, settings, graph=True)
    plan.run()
    torch.cuda.synchronize()
    nrr.device_status()
    for i in (0, 1, 15, 16, 17):
        got = [t.cpu().numpy() for t in plan.result(i)]
        assert _same(got, _single(nrr, dpre, dintra, dmask, settings[i]))
    plan.close()


def test_batch_nested_fractions_share_one_match(nrr, pair):
    # fractions of one (b, stride, R) unit are matched once (the largest) and
    # the others gathered from it: every one must equal its own single call
    pre, intra, mask, dpre, dintra, dmask = pair
    fr = [0.01, 0.02 + 0.005, 0.05, 0.05, 0.07, 0.02, 0.13]
    settings = [(7, 2, (2, 3, 1), f) for f in fr] + [(7, 3, (2, 3, 1), f) for f in fr[:3]]
    plan = nrr.BatchPlan(dpre, dintra, dmask, settings, graph=True)
    plan.run()
    torch.cuda.synchronize()
    nrr.device_status()
    for i, s in enumerate(settings):
        got = [t.cpu().numpy() for t in plan.result(i)]
        assert _same(got, _single(nrr, dpre, dintra, dmask, s)), (i, s)
    plan.close()


def test_autotune_keeps_results(nrr, pair):
    pre, intra, mask, dpre, dintra, dmask = pair
    c = nrr.select_blocks(dpre, dmask, 7, 2, 0.1)
    ref = [t.cpu().numpy() for t in nrr.block_match(dpre, dintra, c, 7, 4)]
    box = nrr.boxsums(dintra, 7)
    k, ms = nrr.autotune_match(dpre, dintra, box, c, 7, 4)
    assert k >= 1 and ms > 0
    assert nrr.tuning_get(0, 7, 4) in (0, k)
    for forced in (1, 2):
        nrr.tuning_set(0, 7, 4, forced)
        got = [t.cpu().numpy() for t in nrr.block_match(dpre, dintra, c, 7, 4)]
        assert _same(got, ref)
    nrr.tuning_set(0, 7, 4, 0)
    plan = nrr.BatchPlan(dpre, dintra, dmask, SETTINGS[:3], graph=True, autotune=True)
    plan.run()
    torch.cuda.synchronize()
    for i, s in enumerate(SETTINGS[:3]):
        assert _same([t.cpu().numpy() for t in plan.result(i)], _single(nrr, dpre, dintra, dmask, s))
    plan.close()


def test_batch_smaller_radii_reported_by_the_larger_search(nrr, pair):
    # units of one (b, stride) whose boxes nest: the largest box's job also
    # reports the best shift within each smaller box (up to 4 extra levels;
    # a fifth is matched by itself); every setting must equal its own call
    pre, intra, mask, dpre, dintra, dmask = pair
    radii = [(4, 4, 4), (3, 3, 3), (2, 2, 2), (1, 1, 1), (0, 0, 0), (3, 1, 2)]
    settings = [(5, 2, r, 0.1) for r in radii] + [(5, 2, (2, 2, 2), 0.05), (5, 2, (4, 4, 4), 0.03)]
    plan = nrr.BatchPlan(dpre, dintra, dmask, settings, graph=True)
    for rep in range(2):
        plan.run()
        torch.cuda.synchronize()
        nrr.device_status()
        for i, s in enumerate(settings):
            got = [t.cpu().numpy() for t in plan.result(i)]
            assert _same(got, _single(nrr, dpre, dintra, dmask, s)), (rep, i, s)
    # and directly against the oracle for one served level
    b, st, r, f = settings[2]
    rc, _ = oracle.select_blocks(pre, mask, b, st, f)
    rd, rn, rv = oracle.match(pre, intra, rc, b, r)
    c, d, n, v = [t.cpu().numpy() for t in plan.result(2)]
    assert np.array_equal(c, rc) and np.array_equal(d, rd) and np.array_equal(v, rv)
    plan.close()


@pytest.fixture(scope="module")
def uneven_pairs(nrr):
    out = []
    for k, dims in enumerate([(64, 64, 48), (96, 80, 56), (128, 96, 64)]):
        pre, intra, mask, _ = synth.make_pair(dims, 4.0, 20.0, 500 + k)
        out.append((pre, intra, mask, nrr.to_device_u16(pre), nrr.to_device_u16(intra), torch.from_numpy(mask).cuda()))
    return out


# settings spread over three pairs of different sizes: one launch per
# (block, radius) then holds jobs of several pairs (radius 9 needs
# sub-windows; the radius-2 settings nest in the radius-4 ones)
MULTI = [(0, (7, 2, 3, 0.1)), (1, (7, 2, 3, 0.1)), (2, (7, 2, 3, 0.05)), (2, (7, 2, 3, 0.1)),
         (1, (5, 2, 4, 0.08)), (1, (5, 2, 2, 0.08)), (0, (5, 2, 4, 0.1)), (2, (5, 3, (4, 2, 3), 0.06)),
         (0, (9, 2, 9, 0.03)), (2, (9, 2, 9, 0.02)), (1, (7, 3, (2, 3, 1), 0.04))]


@pytest.mark.parametrize("dedup", [True, False])
def test_batch_over_uneven_pairs_equals_single_calls(nrr, uneven_pairs, dedup):
    pairs = [(p[3], p[4], p[5]) for p in uneven_pairs]
    settings = [s for _, s in MULTI]
    pof = [p for p, _ in MULTI]
    plan = nrr.BatchPlan(settings=settings, pairs=pairs, pair_of=pof, graph=True, dedup=dedup)
    for rep in range(2):
        plan.run()
        torch.cuda.synchronize()
        nrr.device_status()
        for i, (p, s) in enumerate(MULTI):
            got = [t.cpu().numpy() for t in plan.result(i)]
            assert _same(got, _single(nrr, *pairs[p], s)), (dedup, rep, i, p, s)
    # one setting per pair directly against the oracle
    for i in (0, 4, 7):
        p, (b, st, r, f) = MULTI[i]
        pre, intra, mask = uneven_pairs[p][:3]
        rc, _ = oracle.select_blocks(pre, mask, b, st, f)
        rd, rn, rv = oracle.match(pre, intra, rc, b, r)
        c, d, n, v = [t.cpu().numpy() for t in plan.result(i)]
        assert np.array_equal(c, rc) and np.array_equal(d, rd) and np.array_equal(v, rv)
        assert np.array_equal(n[~np.isnan(n)].view(np.int64), rn[~np.isnan(rn)].view(np.int64))
    plan.close()


def test_batch_pairs_with_and_without_dedup_agree(nrr, uneven_pairs):
    # the sharing (nested fractions, radius levels, shared selections) must
    # not change a bit: the same plan without it gives the same results
    pairs = [(p[3], p[4], p[5]) for p in uneven_pairs]
    settings = [(5, 2, r, f) for r in (1, 2, 3) for f in (0.03, 0.06)] * 3
    pof = [k // 6 for k in range(len(settings))]
    a = nrr.BatchPlan(settings=settings, pairs=pairs, pair_of=pof, graph=True)
    b = nrr.BatchPlan(settings=settings, pairs=pairs, pair_of=pof, graph=False, dedup=False)
    a.run()
    b.run()
    torch.cuda.synchronize()
    nrr.device_status()
    for i in range(len(settings)):
        assert _same([t.cpu().numpy() for t in a.result(i)], [t.cpu().numpy() for t in b.result(i)]), i
    a.close()
    b.close()


def test_plain_launches_and_work_queue_agree(nrr, uneven_pairs):
    # persistent CTAs taking blocks from the work queue (also with one CTA
    # per SM, so each CTA takes many) against one CTA per block
    pairs = [(p[3], p[4], p[5]) for p in uneven_pairs]
    settings = [s for _, s in MULTI]
    pof = [p for p, _ in MULTI]
    ref = nrr.BatchPlan(settings=settings, pairs=pairs, pair_of=pof, graph=False, plain_launch=True)
    ref.run()
    torch.cuda.synchronize()
    want = [[t.cpu().numpy() for t in ref.result(i)] for i in range(len(settings))]
    ref.close()
    for k in (1, 0):
        for b, _, r, _ in settings:
            nrr.tuning_set(0, b, r, k)
        plan = nrr.BatchPlan(settings=settings, pairs=pairs, pair_of=pof, graph=True)
        for rep in range(2):
            plan.run()
            torch.cuda.synchronize()
            nrr.device_status()
            for i in range(len(settings)):
                assert _same([t.cpu().numpy() for t in plan.result(i)], want[i]), (k, rep, i)
        plan.close()


@pytest.mark.parametrize("dtype", ["u16", "f32"])
def test_every_launch_shape_gives_the_same_bits(nrr, pair, dtype):
    # CTAs per SM, one or two window buffers, box sums loaded at the bound
    # or staged into shared memory by asynchronous copies, one or two search
    # lines per thread (float32 ignores the field): no shape may change a
    # result bit (the autotuner picks among them)
    pre, intra, mask, dpre, dintra, dmask = pair
    p, i = (dpre, dintra) if dtype == "u16" else (torch.from_numpy(synth.as_f32(pre)).cuda(),
                                                   torch.from_numpy(synth.as_f32(intra)).cuda())
    code = 0 if dtype == "u16" else 1
    c = nrr.select_blocks(dpre, dmask, 7, 2, 0.1)
    for b, r in ((7, 4), (5, (3, 2, 5)), (7, 9)):
        ref = [t.cpu().numpy() for t in nrr.block_match(p, i, c, b, r)]
        for k, windows, stage, lines in ((1, 1, 1, 2), (2, 2, 1, 1), (1, 1, 2, 1), (0, 2, 2, 2), (3, 1, 2, 2),
                                         (0, 0, 0, 1), (0, 0, 0, 2), (0, 0, 0, 0)):
            nrr.tuning_set_shape(code, b, r, k, windows, stage, lines)
            try:
                got = [t.cpu().numpy() for t in nrr.block_match(p, i, c, b, r)]
            except nrr.NrrError as e:  # a layout that does not fit is refused, never run
                assert e.status == -1 and "does not fit" in str(e), str(e)
                continue
            nrr.device_status()
            assert _same(got, ref), (dtype, b, r, k, windows, stage, lines)
        nrr.tuning_set_shape(code, b, r, 0, 0, 0)


def test_one_and_two_lines_per_thread_agree_at_every_window_width(nrr, pair):
    # uint16 cubic blocks: every x-shift count 1..15 of one window (radius
    # 0..7) and every block size, searched with one and with two lines per
    # thread, gives the same bits (the default picks one of the two by the
    # x-shift count)
    pre, intra, mask, dpre, dintra, dmask = pair
    for b, r in ((3, 0), (5, 1), (7, 2), (9, 3), (11, 4), (5, 5), (7, 6), (3, 7), (9, (2, 5, 3))):
        c = nrr.select_blocks(dpre, dmask, b, 2, 0.02)
        outs = []
        for lines in (1, 2):
            nrr.tuning_set_shape(0, b, r, 0, 0, 0, lines)
            outs.append([t.cpu().numpy() for t in nrr.block_match(dpre, dintra, c, b, r)])
            nrr.device_status()
        nrr.tuning_set_shape(0, b, r, 0, 0, 0)
        assert _same(outs[0], outs[1]), (b, r)
        assert outs[0][2].any(), (b, r)  # some blocks found a valid match
