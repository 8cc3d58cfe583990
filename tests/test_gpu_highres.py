"""Parity at the high-resolution size (512x512x256, block 9^3, stride 3,
top 5%, radius 7: 3375 shifts), in the configuration bench.py times: the
whole selection and the whole match run on the GPU, and a sample of the
blocks is checked against the oracle (every result of the sample: uint16
bit-exact; float32 intensities u/65535 within the NCC tolerance)."""
import numpy as np
import pytest

import oracle
from paper_2308_10868_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F32_NCC_TOL = 1e-6
F32_TIE_TOL = 2e-6


@pytest.fixture(scope="module")
def setup():
    from paper_2308_10868_gb300 import build as nbuild

    nbuild.build()
    from paper_2308_10868_gb300 import nrr

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pre, intra, mask = synth.workload_pair("highres")
    w = synth.WORKLOADS["highres"]
    dpre, dintra = nrr.to_device_u16(pre), nrr.to_device_u16(intra)
    centers = nrr.select_blocks(dpre, torch.from_numpy(mask).cuda(), w.block, w.stride, w.frac)
    return nrr, w, pre, intra, mask, dpre, dintra, centers


def test_highres_selection_and_u16_match(setup):
    nrr, w, pre, intra, mask, dpre, dintra, centers = setup
    ref_c, _ = oracle.select_blocks(pre, mask, w.block, w.stride, w.frac)
    assert np.array_equal(centers.cpu().numpy(), ref_c)
    disp, ncc, valid = nrr.block_match(dpre, dintra, centers, w.block, w.radius)
    nrr.device_status()
    idx = np.arange(0, len(ref_c), 37)
    rd, rn, rv = oracle.match(pre, intra, ref_c[idx], w.block, w.radius)
    assert np.array_equal(disp.cpu().numpy()[idx], rd)
    assert np.array_equal(valid.cpu().numpy()[idx], rv)
    g = ncc.cpu().numpy()[idx]
    assert np.array_equal(g[~np.isnan(g)].view(np.int64), rn[~np.isnan(rn)].view(np.int64))


def test_highres_f32_match(setup):
    nrr, w, pre, intra, mask, dpre, dintra, centers = setup
    p32, i32 = synth.as_f32(pre), synth.as_f32(intra)
    disp, ncc, valid = nrr.block_match(torch.from_numpy(p32).cuda(), torch.from_numpy(i32).cuda(), centers, w.block,
                                       w.radius)
    nrr.device_status()
    c = centers.cpu().numpy()
    idx = np.arange(0, len(c), 53)
    gd, gn, gv = disp.cpu().numpy()[idx], ncc.cpu().numpy()[idx], valid.cpu().numpy()[idx]
    rd, rn, rv = oracle.match(p32, i32, c[idx], w.block, w.radius)
    assert np.array_equal(gv, rv)
    at = np.array([oracle.pearson_f32(p32, i32, w.block, c[i], gd[k]) for k, i in enumerate(idx)])
    ok = rv == 1
    err = np.abs(gn[ok] - at[ok])
    assert err.max() <= F32_NCC_TOL
    diff = (gd != rd).any(axis=1) & ok
    assert (rn[diff] - at[diff] <= F32_TIE_TOL).all()
    print(f"\nfloat32 high resolution: NCC error against FP64 at the returned shift: max {err.max():.3g}, "
          f"mean {err.mean():.3g} over {int(ok.sum())} sampled blocks; shift differs from the FP64 arg-max in "
          f"{int(diff.sum())}")
