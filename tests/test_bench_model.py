"""The bench's algorithmic byte models (the numerators of the reported roofline) equal the per-window
formulas stated for each kernel, and agree with the DRAM bytes ncu measured for those kernels (CPU;
synthetic statistics and recorded counter values, no GPU).

Fly-shaped library at full scale: R = 100, k = 31, W = 2.0677G windows, 1.4805G candidates,
0.5872G first sightings; the pass-1 model is then 49.6 B per window.
"""
import os
import sys
import types

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

W, NC, NF, NU, NO = 2_067_736_949, 1_480_518_957, 587_217_992, 168_259_571, 115_269_743


def _lib(k=31, R=100):
    return types.SimpleNamespace(k=k, n_reads=2, offsets=np.array([0, R, 2 * R], dtype=np.uint64))


def _stats(passes=2, parts=1, table_bytes=0):
    return {"n_windows": W, "n_candidates": NC, "n_firsts": NF, "n_unique": NU, "n_out": NO,
            "super_partitions": parts, "sort_passes": passes, "table_bytes": table_bytes}


def test_pass1_model_is_49_6_bytes_per_window_on_the_fly_shaped_library():
    b, launches, units = bench.stage_bytes("filter", _stats(), _lib(), True)
    packed = (100 / 4 + 100 / 8) / (100 - 31 + 1)
    assert launches == 1 and units == W
    assert b == pytest.approx(W * packed + 32 * W + 32 * NF + 8 * (NC + NF))
    assert b / W == pytest.approx(49.6, abs=0.05)


def test_sort_and_bucket_models():
    b, launches, units = bench.stage_bytes("sort", _stats(), _lib(), True)
    assert b == 2 * 2 * 8 * (NC + NF) and launches == 4 and units == 2 * (NC + NF)  # 2 passes x 2 streams
    b, launches, units = bench.stage_bytes("rle", _stats(), _lib(), True)
    assert b == 8 * (NC + NF) + 12 * NO and launches == 1 and units == NC + NF
    assert b / W == pytest.approx(8.67, abs=0.01)  # the bucket kernel's 8.67 B per window


def test_parts_multiply_the_packed_reads_only():
    one, _, _ = bench.stage_bytes("filter", _stats(parts=1), _lib(), True)
    four, launches, _ = bench.stage_bytes("filter", _stats(parts=4), _lib(), True)
    packed = (100 / 4 + 100 / 8) / (100 - 31 + 1)
    assert launches == 4 and four - one == pytest.approx(3 * W * packed)


def test_hash_form_models():
    tb = 8 << 30
    b, launches, units = bench.stage_bytes_hash("table", _stats(table_bytes=tb), _lib())
    assert b == 2 * 8 * NC + tb + 64 * NC and launches == 1 and units == NC
    b, _, units = bench.stage_bytes_hash("recount", _stats(table_bytes=tb), _lib())
    assert b == NF * (8 + 32) and units == NF
    b, launches, units = bench.stage_bytes_hash("sort", _stats(passes=8, table_bytes=tb), _lib())
    assert b == 8 * 2 * 8 * NO + NO * (8 + 36) and launches == 8 and units == 8 * NO


def test_128_bit_keys_double_the_key_bytes():
    b31, _, _ = bench.stage_bytes("sort", _stats(), _lib(k=31), True)
    b64, _, _ = bench.stage_bytes("sort", _stats(), _lib(k=64, R=150), True)
    assert b64 == 2 * b31


# ---------------------------------------------------------------- against hardware counters
# The figures below are ncu's dram__bytes_read.sum + dram__bytes_write.sum of single launches on small
# cases (profiles/*.md, which give the commands): an independent measure of the bytes each kernel moves.
# The streaming kernels must move what their model says (every key read and written once, no re-reads);
# pass 1 must move about twice its model: each 32-byte filter probe that misses L2 brings a 64-byte
# line pair from DRAM, which the algorithmic model does not count.

def test_sort_model_matches_measured_dram_bytes():
    """k_onesweep on the bucket index, fly-shaped at 1/10 scale, first pass over 145,978,999 candidates:
    1.169 GB read + 1.189 GB written (profiles/k_onesweep_bucket_fly_scale0.1.md)."""
    measured = (1.169e9 + 1.189e9) / 145_978_999
    b, _, units = bench.stage_bytes("sort", _stats(), _lib(), True)
    model = b / units  # bytes per key-pass
    assert model == 16.0
    assert abs(measured / model - 1) < 0.02


def test_bucket_kernel_model_matches_measured_dram_bytes():
    """k_bucket_count<Key128>, long-k at 1/50 scale, key range 0 of 4: 17.1 DRAM bytes per key read
    (profiles/k_bucket_count_longk_scale0.02.md). The model: a 16-byte key read per candidate or first
    sighting, 20 bytes written per reported key (380,554,878 windows, 21,057,192 reported)."""
    W_, NC_, NO_ = 380_554_878, 259_574_202, 21_057_192
    st = {"n_windows": W_, "n_candidates": NC_, "n_firsts": W_ - NC_, "n_unique": NO_, "n_out": NO_,
          "super_partitions": 4, "sort_passes": 2, "table_bytes": 0}
    b, _, units = bench.stage_bytes("rle", st, _lib(k=64, R=150), True)
    assert units == W_
    assert abs(17.1 / (b / units) - 1) < 0.03


def test_pass1_model_is_half_the_measured_dram_bytes():
    """k_pass1, fly-shaped at 1/10 scale with the full-size filter (259 MB): 16.85 GB read + 3.61 GB
    written over 206.8M windows, 98.9 B per window (profiles/k_pass1_fly_scale0.1.md); 21% of the probes
    hit L2, the rest move a 64-byte line pair for a 32-byte sector."""
    measured = (16.85e9 + 3.61e9) / 206.8e6
    b, _, units = bench.stage_bytes("filter", _stats(), _lib(), True)
    ratio = measured / (b / units)
    assert 1.8 < ratio < 2.2
