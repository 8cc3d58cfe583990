"""Bounded device-side waits give up (GPU), without a fault or a hang.

The connectivity-pattern selection runs one cooperative launch whose CTAs
meet at grid barriers; each wait there is bounded.  Through the test hook
nrr_test_set_wait the barriers are given one arrival that never comes and a
short limit: every CTA then waits out the limit, the kernel records
NRR_E_TIMEOUT in the device error word and returns.  The host reads the
status, the context stays usable, and the next selection with the hook
cleared equals the oracle.
"""
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


def test_grid_barrier_wait_gives_up_and_is_reported(nrr):
    pre, intra, mask = synth.workload_pair("small")
    dp, dm = nrr.to_device_u16(pre), torch.from_numpy(mask).cuda()
    nrr.device_status()  # no error pending
    nrr.test_set_wait(20_000_000, 1)  # 20 ms, one arrival that never comes
    try:
        t0 = time.time()
        try:
            nrr.select_blocks(dp, dm, 5, 2, 0.1, connectivity=6)
        except nrr.NrrError:
            pass  # the selection's own result is not defined here; the status is
        with pytest.raises(nrr.NrrError) as ei:
            nrr.device_status()
        assert ei.value.status == -5  # NRR_E_TIMEOUT
        assert time.time() - t0 < 30.0
    finally:
        nrr.test_set_wait(0, 0)
    nrr.device_status()  # the error word was cleared by the report
    got = nrr.select_blocks(dp, dm, 5, 2, 0.1, connectivity=6).cpu().numpy()
    nrr.device_status()
    ref, _ = oracle.select_blocks_spaced(pre, mask, 5, 2, 0.1, 6)
    assert np.array_equal(got, ref)


def test_hook_rejects_out_of_range_values(nrr):
    with pytest.raises(nrr.NrrError) as ei:
        nrr.test_set_wait(0, -1)
    assert ei.value.status == -1
    with pytest.raises(nrr.NrrError):
        nrr.test_set_wait(61_000_000_000, 0)
    nrr.test_set_wait(0, 0)
