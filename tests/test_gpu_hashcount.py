"""Hash-table counting (params.compact = 2) vs the CPU oracle.

The hash-table form counts the candidates in an open-addressing table instead of sorting them
(the hash-table side of the paper's Table 1). Its own paths: the table sized from a distinct-key
estimate, a table too small for its keys (doubled and recounted until every key has a slot), key
ranges, a saturated filter, counts above 2^16, the host and streamed forms. Every result must be
the oracle's, bit for bit.
"""
import numpy as np
import pytest

import oracle
import synth
from tests import brute

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(have_gpu):
    import paper_1305_1861_gb300 as pkg

    pkg.build()
    c = pkg.Context(0)
    yield c
    c.close()


def _check(ctx, bases, offs, k, min_count, **kw):
    import torch
    import paper_1305_1861_gb300 as pkg

    b = torch.from_numpy(np.ascontiguousarray(bases)).cuda()
    o = torch.from_numpy(np.ascontiguousarray(offs).astype(np.int64)).cuda()
    keys, counts, nw = ctx.turtle_count_device(b, o, k, min_count, pkg.Params.default(compact=2, **kw))
    ok, oc, onw = oracle.count(bases, offs, k, min_count)
    gk = keys.cpu().numpy().astype(np.uint64)
    assert nw == onw
    assert gk.shape == ok.shape and np.array_equal(gk, ok)
    assert np.array_equal(counts.cpu().numpy().astype(np.uint64), oc)
    return ctx.stats()


@pytest.mark.parametrize("k", [11, 31, 32, 33, 64])
@pytest.mark.parametrize("min_count", [1, 2, 3])
def test_sized_from_estimate(ctx, k, min_count):
    """Default sizing: the table holds every distinct candidate at load <= 1/2 after one insert."""
    lib = synth.small(seed=60 + k, scale=0.05)
    st = _check(ctx, lib.bases, lib.offsets, k, min_count)
    slot = 16 if k <= 32 else 32
    assert st["n_unique"] > 0 and st["table_bytes"] >= 2 * slot * st["n_unique"]
    assert st["stage_launches"]["table"] == 3  # sketch, clear, insert: no second attempt


@pytest.mark.parametrize("k", [21, 31, 64])
@pytest.mark.parametrize("log2_slots", [3, 10])
def test_table_too_small_is_doubled(ctx, k, log2_slots):
    """A table of 8 or 1024 slots for tens of thousands of distinct keys: keys run out of probes, the
    table doubles until they fit, and the counts are still exact."""
    lib = synth.small(seed=70 + k, scale=0.05)
    st = _check(ctx, lib.bases, lib.offsets, k, 2, hash_slots_log2=log2_slots)
    slot = 16 if k <= 32 else 32
    assert st["table_bytes"] > (slot << log2_slots)  # grew
    assert st["stage_launches"]["table"] > 2  # more than one clear + insert


def test_every_kmer_twice(ctx):
    """Two error-free copies of a genome: about half the windows are distinct candidates."""
    rng = np.random.default_rng(5)
    g = "".join(rng.choice(list("ACGT"), size=200_000))
    k = 31
    reads = []
    for _ in range(2):
        for s in range(0, len(g) - k + 1, 150 - k + 1):
            reads.append(g[s:s + 150])
    bases, offs = brute.pack(reads)
    _check(ctx, bases, offs, k, 2)


def test_saturated_filter(ctx):
    """A filter far too small: most first sightings are false positives and become candidates."""
    lib = synth.small(seed=8, scale=0.05)
    st = _check(ctx, lib.bases, lib.offsets, 31, 2, filter_bits_per_window=0.01, pattern_bits=1, n_patterns=1)
    assert st["n_unique"] > st["n_out"]


def test_counts_above_2_16_and_edge_inputs(ctx):
    reads = ["A" * 100] * 1200 + ["T" * 100] * 5 + ["ACGT" * 25]
    bases, offs = brute.pack(reads)
    for k in (31, 64):
        _check(ctx, bases, offs, k, 2)
    for reads in (["ACG"], ["N" * 50], ["", ""], ["ACGTACGTAC"]):
        bases, offs = brute.pack(reads)
        if bases.size == 0:
            bases = np.zeros(1, np.uint8)
        _check(ctx, bases, offs, 5, 2)


@pytest.mark.parametrize("k,min_count", [(31, 2), (64, 3), (17, 1)])
def test_key_range_super_partitions(ctx, k, min_count):
    """A 1 MiB budget splits the key space into many ranges, each counted in its own table."""
    lib = synth.longk(seed=19, scale=0.002, k=k)
    b, o = lib.chunk(0, lib.n_reads)
    st = _check(ctx, b, o, k, min_count, budget_mib=1)
    assert st["super_partitions"] > 4


def test_fly_shaped_scaled(ctx):
    lib = synth.fly(seed=2, scale=0.01)
    _check(ctx, lib.bases, lib.offsets, 31, 2)


@pytest.mark.parametrize("k,chunk", [(31, 0), (63, 0), (45, 2)])
def test_host_form(have_gpu, k, chunk):
    """Host reads, copied at once or streamed in 2 MiB chunks: the same result."""
    import paper_1305_1861_gb300 as pkg

    lib = synth.longk(seed=23, scale=0.001, k=k)
    b, o = lib.chunk(0, lib.n_reads)
    keys, counts, nw = pkg.turtle_count(b, o, k, 2, pkg.Params.default(compact=2, stream_chunk_mib=chunk))
    ok, oc, onw = oracle.count(b, o, k, 2)
    assert nw == onw and np.array_equal(keys, ok) and np.array_equal(counts.astype(np.uint64), oc)


def test_small_config_full_size(ctx):
    """The full small configuration: 1 Mbp genome, 200,000 x 100 bp reads, k = 31, min_count = 2."""
    lib = synth.small(seed=1)
    st = _check(ctx, lib.bases, lib.offsets, 31, 2)
    assert st["n_windows"] == 200_000 * 70 and st["n_out"] > 0
