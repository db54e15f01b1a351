"""Bucketed sort-and-compact vs the CPU oracle: cases that stress its per-bucket shared-memory table.

A bucket CTA merges at most a fixed number of distinct keys per attempt; beyond that it splits
the bucket's key range and redoes each half. These inputs force that path (every k-mer exactly
twice, so distinct keys per bucket exceed the table; one narrow key range holding tens of
thousands of distinct keys; all-singleton libraries with min_count = 1) and check the output is
still exact, and equal to the global form's.
"""
import numpy as np
import pytest

import oracle
from tests import brute

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(have_gpu):
    import paper_1305_1861_gb300 as pkg

    pkg.build()
    c = pkg.Context(0)
    yield c
    c.close()


# (compact, bucket_slots, sort_tile): bucketed with both table sizes and three tile shapes (4: persistent
# sort with bulk-copied tiles), global (with both tile loads), hash table
FORMS = [(0, 0, 0), (0, 8192, 3), (0, 0, 4), (1, 0, 0), (1, 0, 4), (2, 0, 0)]


def _run(ctx, bases, offs, k, min_count, form):
    import torch
    import paper_1305_1861_gb300 as pkg

    compact, slots, tile = form
    b = torch.from_numpy(np.ascontiguousarray(bases)).cuda()
    o = torch.from_numpy(np.ascontiguousarray(offs).astype(np.int64)).cuda()
    p = pkg.Params.default(compact=compact, bucket_slots=slots, sort_tile=tile)
    keys, counts, nw = ctx.turtle_count_device(b, o, k, min_count, p)
    return keys.cpu().numpy().astype(np.uint64), counts.cpu().numpy().astype(np.uint64), nw, ctx.stats()


def _check(ctx, bases, offs, k, min_count):
    ok, oc, onw = oracle.count(bases, offs, k, min_count)
    for form in FORMS:
        gk, gc, nw, st = _run(ctx, bases, offs, k, min_count, form)
        assert nw == onw
        assert gk.shape == ok.shape and np.array_equal(gk, ok), form
        assert np.array_equal(gc, oc), form
    return ok, oc


def _genome(seed, n):
    rng = np.random.default_rng(seed)
    return "".join(rng.choice(list("ACGT"), size=n))


@pytest.mark.parametrize("k", [21, 31, 32, 45, 64])
def test_every_kmer_twice_overflows_bucket_tables(ctx, k):
    """Two error-free copies of a 300 kbp genome in 150 bp reads: about half the windows are
    distinct candidates, more per bucket than one table attempt holds."""
    g = _genome(100 + k, 300_000)
    reads = []
    for copy in range(2):
        step = 150 - k + 1  # consecutive reads overlap by k-1: every window of the genome once per copy
        for s in range(0, len(g) - k + 1, step):
            reads.append(g[s:s + 150])
    bases, offs = brute.pack(reads)
    ok, oc = _check(ctx, bases, offs, k, 2)
    assert ok.shape[0] > 250_000 and int(oc.min()) >= 2


@pytest.mark.parametrize("k", [31, 64])
def test_narrow_key_range_with_many_distinct_keys(ctx, k):
    """40,000 distinct k-mers sharing a long all-A prefix (one bucket), each seen twice or three
    times: the bucket is split into key ranges several levels deep."""
    rng = np.random.default_rng(7 + k)
    tail = k - 20 if k <= 32 else k - 40
    reads = []
    for i in range(40_000):
        t = "".join(rng.choice(list("CGT"), size=tail))  # no A: the forward strand stays the smaller one
        r = "A" * (k - tail) + t
        reads += [r] * (2 + (i % 2))
    bases, offs = brute.pack(reads)
    ok, oc = _check(ctx, bases, offs, k, 2)
    assert ok.shape[0] > 30_000  # 40,000 draws from 3^11 tails (k = 31) collide a little


@pytest.mark.parametrize("k", [25, 31, 63])
def test_min_count_one_all_singletons(ctx, k):
    """No filter (min_count = 1) on a library of mostly unique k-mers."""
    g = _genome(3 + k, 200_000)
    reads = [g[s:s + 100] for s in range(0, len(g) - 100, 37)]
    bases, offs = brute.pack(reads)
    _check(ctx, bases, offs, k, 1)
    _check(ctx, bases, offs, k, 3)


def test_single_bucket_and_empty_buckets(ctx):
    """Tiny inputs: one bucket, or keys in few buckets of many."""
    for reads in (["ACGTTGCA"] * 3, ["A" * 40] * 2 + ["C" * 40], ["ACGTACGTACGTAAAT", "ACGTACGTACGTAAAT"]):
        bases, offs = brute.pack(reads)
        for k in (3, 5, 8):
            _check(ctx, bases, offs, k, 2)
            _check(ctx, bases, offs, k, 1)
