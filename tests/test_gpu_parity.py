"""GPU path vs the CPU oracle, through the C ABI. Integer work: the bar is bit-exact.

Per step: a2 extraction (every window's canonical key and validity), a3 filter
(bit array after inserting distinct keys, membership of fresh keys), a4
sort-and-compact; whole path: turtle_count_device / turtle_count on synthetic
libraries (several tiles plus ragged tails), every key width, edge cases, and an
adversarial no-false-negative case with a saturated filter.
"""
import numpy as np
import pytest

import oracle
import synth
from tests import brute

pytestmark = pytest.mark.gpu

KS = [1, 2, 5, 15, 21, 31, 32, 33, 47, 55, 63, 64]


@pytest.fixture(scope="module")
def ctx(have_gpu):
    import paper_1305_1861_gb300 as pkg

    pkg.build()
    c = pkg.Context(0)
    yield c
    c.close()


def _dev(bases, offsets):
    import torch

    return torch.from_numpy(np.ascontiguousarray(bases)).cuda(), \
        torch.from_numpy(np.ascontiguousarray(offsets).astype(np.int64)).cuda()


def _u64(t):
    return t.cpu().numpy().astype(np.uint64)


def _mixed_reads(seed, n, lo, hi):
    rng = np.random.default_rng(seed)
    g = "".join(rng.choice(list("ACGT"), size=3000))
    reads = []
    for i in range(n):
        L = int(rng.integers(lo, hi + 1))
        s = int(rng.integers(0, max(1, 3000 - L)))
        r = list(g[s:s + L])
        for j in range(len(r)):
            u = rng.random()
            if u < 0.01:
                r[j] = "N"
            elif u < 0.02:
                r[j] = r[j].lower()
            elif u < 0.025:
                r[j] = "ACGT"[rng.integers(0, 4)]
        reads.append("".join(r))
    return reads


# ---------------------------------------------------------------- a2: extraction
@pytest.mark.parametrize("k", KS)
def test_extract_matches_oracle_windows(ctx, k):
    reads = _mixed_reads(k, 400, 0, 220) + ["", "A" * k, "acgtN" * 30]
    bases, offs = brute.pack(reads)
    pos, okeys = oracle.windows(bases, offs, k)
    b, o = _dev(bases, offs)
    keys, valid, nw = ctx.turtle_extract(b, o, k)
    assert nw == len(pos)
    v = valid.cpu().numpy().astype(np.uint64)
    bits = np.unpackbits(v.view(np.uint8), bitorder="little")[: bases.size].astype(bool)
    assert np.array_equal(np.flatnonzero(bits), pos.astype(np.int64))
    got = _u64(keys)[pos.astype(np.int64)]
    assert np.array_equal(got, okeys)


def test_extract_unaligned_base_pointer_and_leading_bytes(ctx):
    import torch

    reads = _mixed_reads(3, 200, 50, 150)
    bases, offs = brute.pack(reads)
    pad = 5  # bases start 5 bytes into the buffer; bytes before offsets[0] belong to no read
    buf = np.concatenate([np.frombuffer(b"TTTTT", dtype=np.uint8), bases])
    offs2 = offs + pad
    tb = torch.from_numpy(buf).cuda()
    to = torch.from_numpy(offs2.astype(np.int64)).cuda()
    for start in (0, 3):  # also an unaligned device pointer
        sub = tb[start:]
        o = to - start
        keys, valid, nw = ctx.turtle_extract(sub, o, 31)
        pos, okeys = oracle.windows(buf[start:], offs2 - start, 31)
        assert nw == len(pos)
        assert np.array_equal(_u64(keys)[pos.astype(np.int64)], okeys)


# ---------------------------------------------------------------- a3: filter
@pytest.mark.parametrize("words,bits,npat", [(1, 4, 1024), (2, 4, 1024), (1, 6, 4096), (1, 2, 64)])
def test_filter_bits_match_sequential_oracle(ctx, words, bits, npat):
    import torch

    import paper_1305_1861_gb300 as pkg

    rng = np.random.default_rng(words * 100 + bits)
    n_sectors = 1 << 12
    keys = np.unique(rng.integers(0, 2 ** 62, size=(60_000, words), dtype=np.uint64), axis=0)
    rng.shuffle(keys)
    ins, probe = keys[:40_000], keys[40_000:]
    if words == 1:
        ins, probe = ins[:, 0].copy(), probe[:, 0].copy()
    prm = pkg.Params.default(pattern_bits=bits, n_patterns=npat, pattern_seed=987654321)
    of = oracle.PBBF(n_sectors, bits, npat, seed=987654321)
    of.test_and_set(ins)
    words_t = torch.zeros(4 * n_sectors, dtype=torch.int64, device="cuda")
    ctx.turtle_filter(torch.from_numpy(ins.view(np.int64)).cuda(), words_t, n_sectors, prm, set=True)
    # distinct keys: the final bit array does not depend on insertion order
    assert np.array_equal(_u64(words_t), of.words)
    seen = ctx.turtle_filter(torch.from_numpy(probe.view(np.int64)).cuda(), words_t, n_sectors, prm, set=False)
    assert np.array_equal(seen.cpu().numpy(), of.test(probe))
    again = ctx.turtle_filter(torch.from_numpy(ins.view(np.int64)).cuda(), words_t, n_sectors, prm, set=False)
    assert again.cpu().numpy().all()


def test_filter_concurrent_duplicates_never_both_first(ctx):
    """Many copies of each key in one launch: exactly one copy may see 'first', never zero or two."""
    import torch

    import paper_1305_1861_gb300 as pkg

    rng = np.random.default_rng(5)
    base = rng.integers(0, 2 ** 62, size=5000, dtype=np.uint64)
    stream = np.repeat(base, 64)  # 64 adjacent copies: same warp, same CTA, neighbouring CTAs
    n_sectors = 1 << 16
    words_t = torch.zeros(4 * n_sectors, dtype=torch.int64, device="cuda")
    seen = ctx.turtle_filter(torch.from_numpy(stream.view(np.int64)).cuda(), words_t, n_sectors,
                             pkg.Params.default(), set=True).cpu().numpy().reshape(5000, 64)
    firsts = (seen == 0).sum(axis=1)
    assert firsts.max() <= 1
    # a key whose bits were all set by others already is a false positive (0 firsts): rare at this load
    assert (firsts == 0).mean() < 0.01


# ---------------------------------------------------------------- a4: sort-and-compact
@pytest.mark.parametrize("words,n,distinct,bits", [(1, 0, 1, 62), (1, 1, 1, 62), (1, 4095, 100, 62),
                                                   (1, 4097, 4097, 64), (1, 300_001, 20_000, 62),
                                                   (1, 123_457, 1 << 20, 42), (2, 2049, 50, 128),
                                                   (2, 200_003, 30_000, 128), (2, 77_777, 5_000, 66)])
def test_sort_compact_matches_oracle(ctx, words, n, distinct, bits):
    import torch

    rng = np.random.default_rng(n + words)
    if words == 1:
        pool = rng.integers(0, 2 ** 63, size=distinct, dtype=np.uint64) & np.uint64((1 << bits) - 1 if bits < 64
                                                                                     else 2 ** 64 - 1)
        pool[:1] = np.uint64((1 << bits) - 1) if bits < 64 else np.uint64(2 ** 64 - 1)
        keys = pool[rng.integers(0, distinct, size=n)] if n else np.zeros(0, np.uint64)
    else:
        hi = rng.integers(0, 2 ** 62, size=distinct, dtype=np.uint64) & np.uint64((1 << (bits - 64)) - 1)
        lo = rng.integers(0, 2 ** 64, size=distinct, dtype=np.uint64)
        pool = np.stack([hi, lo], axis=1)
        keys = pool[rng.integers(0, distinct, size=n)]
    t = torch.from_numpy(np.ascontiguousarray(keys).view(np.int64)).cuda()
    if words == 2:
        t = t.reshape(n, 2)
    uk, uc = ctx.turtle_sort_compact(t, bits)
    ok, oc = oracle.sort_compact(keys)
    assert np.array_equal(_u64(uk).reshape(ok.shape), ok)
    assert np.array_equal(uc.cpu().numpy().astype(np.uint64), oc)
    assert np.array_equal(_u64(t).reshape(keys.shape), keys)  # input untouched


# ---------------------------------------------------------------- whole path
def _check_count(ctx, bases, offs, k, min_count, params=None):
    b, o = _dev(bases, offs)
    keys, counts, nw = ctx.turtle_count_device(b, o, k, min_count, params)
    ok, oc, onw = oracle.count(bases, offs, k, min_count)
    assert nw == onw
    gk = _u64(keys)
    assert gk.shape == ok.shape and np.array_equal(gk, ok)
    assert np.array_equal(counts.cpu().numpy().astype(np.uint64), oc)
    return ctx.stats()


@pytest.mark.parametrize("k", KS)
@pytest.mark.parametrize("min_count", [1, 2, 3])
@pytest.mark.parametrize("compact", [0, 1, 2])
def test_count_small_library_all_k(ctx, k, min_count, compact):
    """All three forms of counting the candidates: bucketed (default), global sort, hash table."""
    import paper_1305_1861_gb300 as pkg

    lib = synth.small(seed=k, scale=0.02)  # 20 kbp genome, 4000 reads: many tiles, ragged tails
    st = _check_count(ctx, lib.bases, lib.offsets, k, min_count, pkg.Params.default(compact=compact))
    if compact == 0:
        assert st["sort_passes"] == 1 and st["stage_launches"]["table"] == 0


@pytest.mark.parametrize("k", [5, 31, 32, 33, 64])
def test_count_recount_by_windows(ctx, k):
    """The literal second pass (re-extract every window, count it in the table) agrees too."""
    import paper_1305_1861_gb300 as pkg

    lib = synth.small(seed=40 + k, scale=0.02)
    st = _check_count(ctx, lib.bases, lib.offsets, k, 2, pkg.Params.default(recount_windows=1))
    assert st["n_firsts"] == 0
    st = _check_count(ctx, lib.bases, lib.offsets, k, 2, pkg.Params.default(recount_windows=0))
    assert st["n_firsts"] + st["n_candidates"] == st["n_windows"]


def test_count_mixed_reads_with_ambiguous_calls(ctx):
    import paper_1305_1861_gb300 as pkg

    reads = _mixed_reads(11, 3000, 0, 300)
    bases, offs = brute.pack(reads)
    for k in (7, 31, 40, 64):
        for rw in (0, 1):
            _check_count(ctx, bases, offs, k, 2, pkg.Params.default(recount_windows=rw))


def test_count_small_config_full_size(ctx):
    """Configuration 'small': 1 Mbp genome, 200,000 x 100 bp, 1% errors, k=31, min_count=2."""
    lib = synth.small(seed=1)
    st = _check_count(ctx, lib.bases, lib.offsets, 31, 2)
    assert st["n_windows"] == 200_000 * 70 and st["n_out"] > 0


def test_count_saturated_filter_has_no_false_negatives(ctx):
    """A filter far too small (most first sightings are false positives) changes nothing in the output."""
    import paper_1305_1861_gb300 as pkg

    lib = synth.small(seed=7, scale=0.05)
    for rw in (0, 1):
        p = pkg.Params.default(filter_bits_per_window=0.01, pattern_bits=1, n_patterns=1, recount_windows=rw)
        st = _check_count(ctx, lib.bases, lib.offsets, 31, 2, p)
        assert st["filter_bytes"] <= 4096 and st["n_unique"] > st["n_out"]  # false-positive singletons recounted


def test_count_one_kmer_above_2_16(ctx):
    reads = ["A" * 100] * 1200 + ["T" * 100] * 5 + ["ACGT" * 25]
    bases, offs = brute.pack(reads)
    _check_count(ctx, bases, offs, 31, 2)
    _check_count(ctx, bases, offs, 64, 2)


def test_count_edge_inputs(ctx):
    import paper_1305_1861_gb300 as pkg

    for reads in (["ACG"], ["N" * 50], ["", ""], ["ACGTACGTAC"]):
        bases, offs = brute.pack(reads)
        if bases.size == 0:
            bases = np.zeros(1, np.uint8)
        _check_count(ctx, bases, offs, 5, 2)
    bases, offs = brute.pack(["ACGTACGT", "ACGT"])
    b, o = _dev(bases, offs[::-1].copy())
    with pytest.raises(pkg.TurtleError) as e:
        ctx.turtle_count_device(b, o, 3, 2)
    assert e.value.code == -1


def test_count_deterministic(ctx):
    lib = synth.small(seed=3, scale=0.1)
    b, o = _dev(lib.bases, lib.offsets)
    k1, c1, _ = ctx.turtle_count_device(b, o, 31, 2)
    k1, c1 = k1.clone(), c1.clone()
    k2, c2, _ = ctx.turtle_count_device(b, o, 31, 2)
    assert bool((k1 == k2).all()) and bool((c1 == c2).all())


def test_host_form_matches_oracle(have_gpu):
    import paper_1305_1861_gb300 as pkg

    lib = synth.small(seed=4, scale=0.05)
    for k in (31, 63):
        keys, counts, nw = pkg.turtle_count(lib.bases, lib.offsets, k, 2)
        ok, oc, onw = oracle.count(lib.bases, lib.offsets, k, 2)
        assert nw == onw and np.array_equal(keys, ok) and np.array_equal(counts.astype(np.uint64), oc)


@pytest.mark.parametrize("k,min_count", [(31, 2), (21, 1), (45, 3)])
def test_host_form_overlapped_copy(have_gpu, k, min_count):
    """~100 Mbase of host reads: copied in chunks while earlier chunks are packed and filtered
    (reads and windows straddle the chunk boundaries); the result is the oracle's."""
    import paper_1305_1861_gb300 as pkg

    lib = synth.fly(seed=12, scale=0.034)
    assert lib.bases.size >= 64 << 20
    keys, counts, nw = pkg.turtle_count(lib.bases, lib.offsets, k, min_count)
    ok, oc, onw = oracle.count(lib.bases, lib.offsets, k, min_count)
    assert nw == onw and np.array_equal(keys, ok) and np.array_equal(counts.astype(np.uint64), oc)


def test_fly_shaped_scaled_with_repeats_and_n(ctx):
    """Fly-shaped library at 1/100 scale (1 Mbp + repeats, 300k reads, 0.05% N): exact."""
    lib = synth.fly(seed=2, scale=0.01)
    _check_count(ctx, lib.bases, lib.offsets, 31, 2)


@pytest.mark.parametrize("budget", [1, 400])
@pytest.mark.parametrize("k,min_count,rw", [(31, 2, 0), (31, 2, 1), (31, 1, 0), (64, 2, 0), (64, 3, 1), (17, 2, 0),
                                            (16, 2, 0), (15, 2, 0), (33, 1, 0), (48, 2, 0)])
def test_count_in_key_range_super_partitions(ctx, k, min_count, rw, budget):
    """A small budget forces the key space into consecutive ranges; the output must not change
    (1 MiB: tens of ranges; 400 MiB: a few)."""
    import paper_1305_1861_gb300 as pkg

    lib = synth.longk(seed=9, scale=0.002, k=k)
    b, o = lib.chunk(0, lib.n_reads)
    p = pkg.Params.default(budget_mib=budget, recount_windows=rw)
    st = _check_count(ctx, b, o, k, min_count, p)
    assert st["super_partitions"] > (4 if budget == 1 else 1)
    st = _check_count(ctx, b, o, k, min_count, pkg.Params.default(recount_windows=rw))
    assert st["super_partitions"] == 1


@pytest.mark.parametrize("k,chunk_mib", [(31, 1), (64, 1), (45, 2)])
def test_host_form_streamed_through_pinned_chunks(have_gpu, k, chunk_mib):
    """Host reads streamed in small chunks (many chunk boundaries inside reads): same result."""
    import paper_1305_1861_gb300 as pkg

    lib = synth.longk(seed=5, scale=0.001, k=k)  # ~35 Mbase: tens of 1-2 MiB chunks
    b, o = lib.chunk(0, lib.n_reads)
    keys, counts, nw = pkg.turtle_count(b, o, k, 2, pkg.Params.default(stream_chunk_mib=chunk_mib))
    ok, oc, onw = oracle.count(b, o, k, 2)
    assert nw == onw and np.array_equal(keys, ok) and np.array_equal(counts.astype(np.uint64), oc)


@pytest.mark.parametrize("k", [15, 31, 32, 33, 64])
@pytest.mark.parametrize("budget", [0, 1])
def test_count_with_probes_ordered_by_filter_block(ctx, k, budget):
    """Pass 1 with its windows binned by filter block before the probes (probe_order = 1): same output,
    in one key range and in several (a small budget)."""
    import paper_1305_1861_gb300 as pkg

    s = synth.longk(seed=30 + k, scale=0.001, k=k)
    b, o = s.chunk(0, s.n_reads)
    st = _check_count(ctx, b, o, k, 2, pkg.Params.default(probe_order=1, budget_mib=budget))
    assert st["stage_launches"]["filter"] >= 3 * st["super_partitions"]
    reads = ["A" * 100] * 1200 + ["ACGT" * 25] * 3  # one key fills one bin
    bases, offs = brute.pack(reads)
    _check_count(ctx, bases, offs, k, 2, pkg.Params.default(probe_order=1))


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_host_transfer_modes(have_gpu, mode):
    """Host arrays copied directly (2), page-locked for their copies (1) or as the context's measured
    rates decide (0): the same results, in the single-library, overlapped-copy and batched forms."""
    import paper_1305_1861_gb300 as pkg

    p = pkg.Params.default(host_transfer=mode)
    lib = synth.fly(seed=12, scale=0.034)  # ~100 Mbase: the copy overlaps pass 1
    keys, counts, nw = pkg.turtle_count(lib.bases, lib.offsets, 31, 2, p)
    ok, oc, onw = oracle.count(lib.bases, lib.offsets, 31, 2)
    assert nw == onw and np.array_equal(keys, ok) and np.array_equal(counts.astype(np.uint64), oc)
    specs = synth.batched_specs(seed=4, n_libs=6, scale=0.05)
    libs = [synth.library_from_spec(sp) for sp in specs]
    jobs = [(l.bases, l.offsets, l.k, l.min_count) for l in libs]
    for (b, o, k, m), (keys, counts, nw) in zip(jobs, pkg.turtle_count_batch(jobs, p)):
        ok, oc, onw = oracle.count(b, o, k, m)
        assert nw == onw and np.array_equal(keys, ok) and np.array_equal(counts.astype(np.uint64), oc)


def test_trim_gives_back_cached_memory_and_calls_still_work(have_gpu):
    import torch

    import paper_1305_1861_gb300 as pkg

    lib = synth.fly(seed=13, scale=0.034)
    ok, oc, _ = oracle.count(lib.bases, lib.offsets, 31, 2)
    keys, counts, _ = pkg.turtle_count(lib.bases, lib.offsets, 31, 2)
    del keys, counts
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    pkg.turtle_trim()
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after > free_before + (256 << 20)  # the internal context's pool held its scratch between calls
    keys, counts, _ = pkg.turtle_count(lib.bases, lib.offsets, 31, 2)
    assert np.array_equal(keys, ok) and np.array_equal(counts.astype(np.uint64), oc)


# ---------------------------------------------------------------- persistent sort with bulk-copied tiles
@pytest.mark.parametrize("k", [21, 31, 45, 64])
@pytest.mark.parametrize("compact", [0, 1])
@pytest.mark.parametrize("genome", [3_000, 60_000, 700_000])
def test_bulk_copied_sort_tiles_match_oracle(ctx, k, compact, genome):
    """sort_tile = 4: one tile or many, the first and last full tiles loaded by the threads, a ragged last
    tile, first sightings starting between two 16-byte boundaries (64-bit keys), both key widths."""
    import paper_1305_1861_gb300 as pkg

    g = synth.genome_iid(900 + genome + k, genome)
    b, o = synth.reads_uniform(g, 901 + k, max(1, int(12 * genome / 120)), 120, 0.01)
    st = _check_count(ctx, b, o, k, 2, pkg.Params.default(compact=compact, sort_tile=4))
    assert st["n_candidates"] > 0


def test_host_form_large_arrays_locked_for_their_copies(have_gpu):
    """750 Mbase of host reads page-locked for their copies, which overlap pass 1 in chunks, and a fresh
    result buffer first touched and locked: the oracle's result, twice (the second call reuses the
    recycled result buffers)."""
    import paper_1305_1861_gb300 as pkg

    lib = synth.fly(seed=13, scale=0.25)
    assert lib.bases.size > (512 << 20)
    ok, oc, onw = oracle.count(lib.bases, lib.offsets, 31, 2)
    for _ in range(2):
        keys, counts, nw = pkg.turtle_count(lib.bases, lib.offsets, 31, 2, pkg.Params.default(host_transfer=1))
        assert nw == onw and np.array_equal(keys, ok) and np.array_equal(counts.astype(np.uint64), oc)
        del keys, counts
