"""Host-side logic of bench.py (CPU): the check that decides whether the
recorded ncu traffic still describes the match kernel, and the bit-for-bit
comparison that validates a replayed CUDA graph of a registration."""
import os
import shutil

import numpy as np
import pytest

import bench

torch = pytest.importorskip("torch")

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2308_10868_gb300", "csrc")


def _copy_sources(tmp_path):
    for f in ("nrr_match.cuh", "nrr_ptx.cuh"):
        shutil.copy(os.path.join(CSRC, f), tmp_path / f)
    return str(tmp_path)


def test_kernel_hash_ignores_comments_but_not_code(tmp_path):
    d = _copy_sources(tmp_path)
    h0 = bench._kernel_source_hash(d)
    assert h0 == bench._kernel_source_hash()
    p = tmp_path / "nrr_match.cuh"
    text = p.read_text()
    p.write_text("// a comment added at the top\n\n" + text.replace("\n", "  // trailing note\n", 3))
    assert bench._kernel_source_hash(d) == h0
    p.write_text(text.replace("constexpr int MATCH_MAX_THREADS_C = 256;", "constexpr int MATCH_MAX_THREADS_C = 128;"))
    assert bench._kernel_source_hash(d) != h0


def _results(n, cap, seed):
    rng = np.random.default_rng(seed)
    disp = torch.from_numpy(rng.integers(-5, 6, (cap, 3), dtype=np.int32))
    ncc = torch.from_numpy(rng.random(cap))
    valid = torch.from_numpy(rng.integers(0, 2, cap, dtype=np.uint8))
    return (disp, ncc, valid), torch.tensor([n], dtype=torch.int32)


def test_replay_check_covers_the_selected_blocks_only():
    out, n_sel = _results(40, 64, 1)
    ref = [t.clone() for t in out] + [n_sel.clone()]
    assert bench._same_results(out, n_sel, ref)
    for t in out:
        t[40:] = 0  # entries past the count are never written
    assert bench._same_results(out, n_sel, ref)
    out[1][7] = np.nextafter(out[1][7].item(), 2.0)  # one NCC bit
    assert not bench._same_results(out, n_sel, ref)
    out[1][7] = ref[1][7]
    out[0][39, 2] += 1  # the last selected block's displacement
    assert not bench._same_results(out, n_sel, ref)
    out[0][39, 2] -= 1
    assert bench._same_results(out, torch.tensor([39], dtype=torch.int32), [ref[0], ref[1], ref[2], ref[3]]) is False
    nan = out[1].clone()
    nan[3] = float("nan")
    ref_nan = [ref[0], nan.clone(), ref[2], ref[3]]
    assert bench._same_results((out[0], nan, out[2]), n_sel, ref_nan)  # equal NaN bit patterns compare equal
