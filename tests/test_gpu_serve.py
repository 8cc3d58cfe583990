"""Serving with continuous batching (GPU).

Requests of mixed sizes and parameters run concurrently on several slots;
each result must equal the same registration run alone through the
synchronous calls, bit for bit (float32 requests use the same kernels, so
they are exact here too), and the oracle: uint16 selections and matches bit
for bit, float32 matches within the parity tests' tolerance.  Failures are
injected on the host (an allocation reported as failed), never on the GPU.
"""
import os
import time

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


def _pairs(nrr, host=None):
    out = []
    for k, dims in enumerate([(64, 64, 48), (96, 80, 56), (128, 96, 64)]):
        pre, intra, mask, _ = synth.make_pair(dims, 4.0, 20.0, 300 + k)
        if host is not None:
            host.append((pre, intra, mask))
        out.append((nrr.to_device_u16(pre), nrr.to_device_u16(intra), torch.from_numpy(mask).cuda(),
                    torch.from_numpy(synth.as_f32(pre)).cuda(), torch.from_numpy(synth.as_f32(intra)).cuda()))
    return out


def _check_oracle(pre, intra, mask, b, r, f, f32, got):
    """A served result against the oracle run on the host copies."""
    rc, _ = oracle.select_blocks(pre, mask, b, 2, f)
    assert np.array_equal(got["centers"].cpu().numpy(), rc)
    gd, gn, gv = (got[k].cpu().numpy() for k in ("disp", "ncc", "valid"))
    if not f32:
        rd, rn, rv = oracle.match(pre, intra, rc, b, r)
        assert np.array_equal(gd, rd) and np.array_equal(gv, rv)
        assert np.array_equal(np.isnan(gn), np.isnan(rn))
        assert np.array_equal(gn[~np.isnan(gn)].view(np.int64), rn[~np.isnan(rn)].view(np.int64))
    else:
        p32, i32 = synth.as_f32(pre), synth.as_f32(intra)
        rd, rn, rv = oracle.match(p32, i32, rc, b, r)
        assert np.array_equal(gv, rv)
        ok = rv == 1
        at = np.array([oracle.pearson_f32(p32, i32, b, rc[i], gd[i]) if ok[i] else np.nan for i in range(len(rc))])
        assert np.abs(gn[ok] - at[ok]).max(initial=0.0) <= 1e-6
        diff = (gd != rd).any(axis=1) & ok
        assert (rn[diff] - at[diff] <= 2e-6).all()


def _wait(srv, tickets, timeout=60.0):
    res, t0 = {}, time.time()
    while len(res) < len(tickets):
        for t in tickets:
            if t not in res:
                r = srv.poll(t)
                if r is not None:
                    res[t] = r
        assert time.time() - t0 < timeout, "requests did not finish"
    return res


def test_mixed_stream_equals_lone_calls(nrr):
    host = []
    pairs = _pairs(nrr, host)
    rng = np.random.default_rng(7)
    reqs = []
    for i in range(24):
        p = int(rng.integers(0, len(pairs)))
        b = int(rng.choice([5, 7, 9]))
        r = int(rng.integers(2, 6))
        f = float(rng.choice([0.02, 0.05, 0.1]))
        reqs.append((p, b, r, f, i % 5 == 4))  # every fifth request in float32
    srv = nrr.Server(slots=4, reserve_bytes=256 << 20)
    try:
        tickets = []
        for p, b, r, f, f32 in reqs:
            dp, di, dm, fp, fi = pairs[p]
            if f32:
                tickets.append(srv.submit(fp, fi, dm, b, 2, r, f, select=dp))
            else:
                tickets.append(srv.submit(dp, di, dm, b, 2, r, f))
        res = _wait(srv, tickets)
        for t, (p, b, r, f, f32) in zip(tickets, reqs):
            dp, di, dm, fp, fi = pairs[p]
            c = nrr.select_blocks(dp, dm, b, 2, f)
            d, n, v = nrr.block_match(fp if f32 else dp, fi if f32 else di, c, b, r)
            got = res[t]
            assert got["n"] == c.shape[0]
            assert torch.equal(got["centers"], c) and torch.equal(got["disp"], d) and torch.equal(got["valid"], v)
            g, e = got["ncc"].cpu().numpy(), n.cpu().numpy()
            assert np.array_equal(np.isnan(g), np.isnan(e))
            assert np.abs(g[~np.isnan(g)] - e[~np.isnan(e)]).max(initial=0.0) == 0.0
            assert 0.0 <= got["queued_s"] <= got["latency_s"]
            _check_oracle(*host[p], b, r, f, f32, got)
            srv.release(t)
        with pytest.raises(nrr.NrrError) as ei:
            srv.poll(tickets[0])
        assert ei.value.status == -7
    finally:
        srv.stop()


def test_failed_allocation_is_contained(nrr):
    dp, di, dm, _, _ = _pairs(nrr)[0]
    srv = nrr.Server(slots=2, reserve_bytes=0)
    os.environ["NRR_FAULT"] = "alloc_once"
    try:
        t_bad = srv.submit(dp, di, dm, 7, 2, 3, 0.05)
        deadline = time.time() + 30
        while True:
            try:
                r = srv.poll(t_bad)
            except nrr.NrrError as e:
                assert e.status == -2  # NRR_E_NOMEM
                break
            assert r is None, "the injected failure was not reported"
            assert time.time() < deadline
        t_ok = srv.submit(dp, di, dm, 7, 2, 3, 0.05)
        res = _wait(srv, [t_ok])
        assert res[t_ok]["n"] > 0
        srv.release(t_ok)
        srv.release(t_bad)
    finally:
        os.environ.pop("NRR_FAULT", None)
        srv.stop()


def test_server_lifecycle_errors(nrr):
    srv = nrr.Server(slots=1)
    try:
        with pytest.raises(nrr.NrrError):
            nrr.Server(slots=1)  # one server per process
        with pytest.raises(nrr.NrrError) as ei:
            srv.release(123456)
        assert ei.value.status == -7
    finally:
        srv.stop()


def test_queued_same_variant_requests_share_a_launch(nrr):
    # one slot and a burst of same-variant requests on volumes of three
    # sizes: the ones queued behind a running group join one match launch
    # (each job with its own volumes and maps); every result must equal the
    # same registration run alone, and the oracle
    host = []
    pairs = _pairs(nrr, host)
    reqs = [(k % 3, 7, 3, (0.02, 0.05, 0.08)[(k // 3) % 3], k % 4 == 3) for k in range(14)]
    srv = nrr.Server(slots=1, reserve_bytes=0)
    try:
        tickets = []
        for p, b, r, f, f32 in reqs:
            dp, di, dm, fp, fi = pairs[p]
            tickets.append(srv.submit(fp, fi, dm, b, 2, r, f, select=dp) if f32 else srv.submit(dp, di, dm, b, 2, r, f))
        res = _wait(srv, tickets)
        for t, (p, b, r, f, f32) in zip(tickets, reqs):
            dp, di, dm, fp, fi = pairs[p]
            c = nrr.select_blocks(dp, dm, b, 2, f)
            d, n, v = nrr.block_match(fp if f32 else dp, fi if f32 else di, c, b, r)
            got = res[t]
            assert torch.equal(got["centers"], c) and torch.equal(got["disp"], d) and torch.equal(got["valid"], v)
            g, e = got["ncc"].cpu().numpy(), n.cpu().numpy()
            assert np.array_equal(g.view(np.uint64), e.view(np.uint64))
            srv.release(t)
        for i in (1, 2):
            p, b, r, f, f32 = reqs[i]
            dp, di, dm, fp, fi = pairs[p]
            c = nrr.select_blocks(dp, dm, b, 2, f)
            d, n, v = nrr.block_match(dp, di, c, b, r)
            _check_oracle(*host[p], b, r, f, False, {"centers": c, "disp": d, "ncc": n, "valid": v})
    finally:
        srv.stop()
