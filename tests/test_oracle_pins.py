"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

None of these re-run the oracle's own formulas: they compare with string brute
force (Sec. 2.1.2 definitions written on characters), reverse-complement
symmetry, the window-count invariant, a closed form for tiled reads, the paper's
sort-and-compact toy example (Sec. 2.1.4) and the blocked-Bloom false-positive
formula (Sec. 2.1.3, Putze et al.) plus the 9.6-bits-per-item sizing (Sec. 2.2).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from tests import brute

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
KS = [1, 2, 3, 4, 5, 7, 16, 31, 32, 33, 48, 63, 64]


def _reads_mixed(rng, n, lo, hi):
    alpha = list("ACGTACGTACGTACGTacgtNnRY.")
    return brute.random_reads(rng, n, lo, hi, alphabet=alpha)


@pytest.mark.parametrize("k", KS)
def test_brute_force_tiny(k):
    rng = np.random.default_rng(100 + k)
    reads = _reads_mixed(rng, 40, 0, 90) + ["", "A" * (k - 1), "acgt" * 20, "N" * 5]
    bases, offs = brute.pack(reads)
    want = brute.kmer_counts(reads, k)
    for fn in (lambda: oracle.count(bases, offs, k, 1, threads=1), lambda: oracle.count(bases, offs, k, 1, threads=3),
               lambda: oracle.count_map(bases, offs, k, 1)):
        keys, counts, nw = fn()
        assert brute.as_dict(keys, counts, k) == want
        assert nw == brute.n_windows(reads, k)
        # ascending unsigned order, unique keys
        if k <= 32:
            assert np.all(np.diff(keys.astype(np.uint64)) > 0) if len(keys) > 1 else True
        else:
            tup = [(int(a), int(b)) for a, b in keys]
            assert tup == sorted(set(tup))


@pytest.mark.parametrize("k,min_count", [(3, 2), (5, 3), (31, 2), (33, 2)])
def test_min_count_cut(k, min_count):
    rng = np.random.default_rng(7)
    g = "".join(rng.choice(list("ACGT"), size=300))
    reads = [g[s:s + 60] for s in rng.integers(0, 240, size=80)] + _reads_mixed(rng, 20, 10, 70)
    bases, offs = brute.pack(reads)
    keys, counts, _ = oracle.count(bases, offs, k, min_count, threads=2)
    assert brute.as_dict(keys, counts, k) == brute.kmer_counts(reads, k, min_count)


@pytest.mark.parametrize("k", [5, 31, 32, 33, 64])
def test_reverse_complement_symmetry(k):
    rng = np.random.default_rng(11 + k)
    reads = _reads_mixed(rng, 60, 50, 120)
    rc_reads = [brute.revcomp("".join(ch.upper() if ch in "acgt" else ch for ch in r)) for r in reads]
    a = oracle.count(*brute.pack(reads), k, 1)
    b = oracle.count(*brute.pack(rc_reads), k, 1)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and a[2] == b[2]


@pytest.mark.parametrize("k", [1, 9, 31, 64])
def test_window_sum_invariant(k):
    rng = np.random.default_rng(5 + k)
    reads = _reads_mixed(rng, 200, 0, 160)
    keys, counts, nw = oracle.count(*brute.pack(reads), k, 1)
    assert int(counts.sum()) == nw == brute.n_windows(reads, k)


def test_tiled_reads_closed_form():
    """Every length-R substring of a genome with distinct canonical k-mers, each taken c times:
    the k-mer at position p is covered by min(p, G-R) - max(0, p+k-R) + 1 reads."""
    G, R, k, c = 1500, 40, 13, 3
    for seed in range(20):
        rng = np.random.default_rng(seed)
        g = "".join(rng.choice(list("ACGT"), size=G))
        canon = [min(g[p:p + k], brute.revcomp(g[p:p + k])) for p in range(G - k + 1)]
        if len(set(canon)) == len(canon):
            break
    else:
        pytest.fail("no genome with distinct canonical k-mers found")
    reads = [g[s:s + R] for s in range(G - R + 1) for _ in range(c)]
    keys, counts, nw = oracle.count(*brute.pack(reads), k, 1)
    got = brute.as_dict(keys, counts, k)
    assert len(got) == G - k + 1
    for p in range(G - k + 1):
        assert got[canon[p]] == c * (min(p, G - R) - max(0, p + k - R) + 1)


def test_single_repeated_read_large_count():
    """One homopolymer read copied many times: one k-mer (A..A, encoding 0) seen copies*(R-k+1) > 2^16 times."""
    R, k, copies = 100, 31, 1200
    reads = ["A" * R] * copies + ["T" * R] * 5
    keys, counts, nw = oracle.count(*brute.pack(reads), k, 2)
    assert keys.tolist() == [0] and counts.tolist() == [(copies + 5) * (R - k + 1)]
    assert counts[0] > 2 ** 16


def test_even_k_palindrome_counted_once_per_window():
    # ACGT is its own reverse complement; each window counts once.
    keys, counts, nw = oracle.count(*brute.pack(["ACGT", "ACGTNACGT"]), 4, 1)
    assert brute.as_dict(keys, counts, 4) == {"ACGT": 3} and nw == 3


def test_edge_inputs():
    empty_b, empty_o = brute.pack([])
    keys, counts, nw = oracle.count(empty_b, empty_o, 31, 1)
    assert keys.size == 0 and counts.size == 0 and nw == 0
    keys, counts, nw = oracle.count(*brute.pack(["ACG", "NNNN", ""]), 5, 1)
    assert keys.size == 0 and nw == 0
    with pytest.raises(ValueError):
        oracle.count(*brute.pack(["ACGT"]), 0, 1)
    with pytest.raises(ValueError):
        oracle.count(*brute.pack(["ACGT"]), 65, 1)


def test_golden_worked_examples():
    with open(os.path.join(GOLDEN, "worked_examples.json")) as f:
        cases = json.load(f)
    for case in cases["count"]:
        keys, counts, nw = oracle.count(*brute.pack(case["reads"]), case["k"], case["min_count"])
        assert brute.as_dict(keys, counts, case["k"]) == case["expect"], case["cite"]
        assert nw == case["n_windows"], case["cite"]
    for case in cases["sort_compact"]:
        k, c = oracle.sort_compact(np.array(case["items"], dtype=np.uint64))
        assert k.tolist() == case["keys"] and c.tolist() == case["counts"], case["cite"]


@pytest.mark.parametrize("words", [1, 2])
def test_sort_compact_matches_counter(words):
    rng = np.random.default_rng(3 + words)
    base = rng.integers(0, 2 ** 63, size=(500, words), dtype=np.uint64)
    pick = base[rng.integers(0, 500, size=5000)]
    keys, counts = oracle.sort_compact(pick if words == 2 else pick[:, 0])
    from collections import Counter
    want = Counter(tuple(int(x) for x in row) for row in pick)
    got = {(tuple(int(x) for x in keys[i]) if words == 2 else (int(keys[i]),)): int(counts[i])
           for i in range(len(counts))}
    assert got == dict(want)
    order = sorted(want)
    assert list(got) == order


@pytest.mark.parametrize("k", [4, 31, 40])
def test_windows_enumeration(k):
    rng = np.random.default_rng(21 + k)
    reads = _reads_mixed(rng, 30, 0, 100)
    pos, keys = oracle.windows(*brute.pack(reads), k)
    want = brute.windows(reads, k)
    assert [int(p) for p in pos] == [p for p, _ in want]
    assert [brute.decode(x, k) for x in keys] == [w for _, w in want]


@pytest.mark.parametrize("k", [7, 31, 50])
def test_count_queries(k):
    rng = np.random.default_rng(31 + k)
    g = "".join(rng.choice(list("ACGT"), size=400))
    reads = [g[s:s + 90] for s in rng.integers(0, 310, size=60)] + _reads_mixed(rng, 10, 20, 90)
    bases, offs = brute.pack(reads)
    keys, counts, _ = oracle.count(bases, offs, k, 1)
    idx = rng.choice(len(counts), size=min(40, len(counts)), replace=False)
    q = keys[idx]
    absent = np.array([[0x3FFFFFFFFFFFFFFF, 0x3FFFFFFFFFFFFFFF]] if k > 32 else [2 ** (2 * k) - 1], dtype=np.uint64)
    got = oracle.count_queries(bases, offs, k, np.concatenate([q, absent]))
    want = brute.kmer_counts(reads, k)
    assert got[:-1].tolist() == [want[brute.decode(x, k)] for x in q]
    tail = brute.decode(absent[0], k)
    assert got[-1] == want.get(min(tail, brute.revcomp(tail)), 0) * (min(tail, brute.revcomp(tail)) == tail)


# ---------------------------------------------------------------- pattern-blocked Bloom filter
@pytest.mark.parametrize("lam,h,T", [(2.0, 4, 1024), (5.0, 4, 1024), (5.0, 6, 4096), (10.0, 3, 256)])
def test_pbbf_false_positive_rate_matches_blocked_formula(lam, h, T):
    n_sectors = 1 << 13
    n = int(lam * n_sectors * 4)
    rng = np.random.default_rng(int(lam * 10) + h)
    keys = np.unique(rng.integers(0, 2 ** 64, size=n + 300_000, dtype=np.uint64))
    rng.shuffle(keys)
    ins, probe = keys[:n], keys[n:n + 200_000]
    f = oracle.PBBF(n_sectors, h, T, seed=12345)
    f.test_and_set(ins)
    before = f.words
    assert f.test(ins).all(), "an inserted key must always test as seen"
    fp = f.test(probe[:100_000]).mean()
    want = oracle.pbbf_fp_formula(lam, h, T)
    sigma = math.sqrt(want * (1 - want) / 100_000)
    assert abs(fp - want) < 4 * sigma + 1e-5, (fp, want, sigma)
    assert np.array_equal(f.words, before), "a membership test sets nothing"
    f.test_and_set(probe)
    assert np.all((f.words & before) == before), "bits are only ever set"


def test_pbbf_pattern_table_shape():
    f = oracle.PBBF(16, 5, 1024, seed=99)
    pats = f.patterns
    assert all(bin(int(p)).count("1") == 5 for p in pats)
    # each of the 64 bit positions is used about 5/64 of the time
    freq = np.array([sum((int(p) >> b) & 1 for p in pats) for b in range(64)]) / len(pats)
    assert abs(freq.mean() - 5 / 64) < 1e-9 and freq.max() < 0.16
    # one insertion touches exactly one 64-bit word, with exactly the pattern's bits
    f.test_and_set(np.array([0xDEADBEEF], dtype=np.uint64))
    w = f.words
    assert np.count_nonzero(w) == 1 and bin(int(w[w != 0][0])).count("1") == 5
    assert int(w[w != 0][0]) in set(int(p) for p in pats)


@pytest.mark.parametrize("words", [1, 2])
def test_pbbf_sequential_first_sighting(words):
    """Keys seen twice are reported seen on their second sighting (no false negatives)."""
    rng = np.random.default_rng(77)
    ks = rng.integers(0, 2 ** 62, size=(20000, words), dtype=np.uint64)
    f = oracle.PBBF(1 << 12, 4, 1024)
    stream = np.concatenate([ks, ks]) if words == 2 else np.concatenate([ks[:, 0], ks[:, 0]])
    seen = f.test_and_set(stream)
    assert seen[20000:].all()


def test_standard_bloom_sizing_quoted_in_paper():
    """Sec. 2.2: about 9.6 n bits give a 1% false-positive rate (unblocked Bloom filter)."""
    bpi = oracle.standard_bloom_bits_per_item(0.01)
    assert abs(bpi - 9.6) < 0.05
    # Monte Carlo of a plain Bloom filter of that size with the optimal 7 hashes
    rng = np.random.default_rng(0)
    n = 50_000
    m = int(bpi * n)
    bits = np.zeros(m, dtype=bool)
    bits[rng.integers(0, m, size=(n, 7))] = True
    fp = bits[rng.integers(0, m, size=(200_000, 7))].all(axis=1).mean()
    assert abs(fp - 0.01) < 4 * math.sqrt(0.01 * 0.99 / 200_000) + 5e-4


# ---------------------------------------------------------------- cTurtle (Sec. 2.2)
def _ct_reads(seed, n, G=4000):
    rng = np.random.default_rng(seed)
    g = "".join(rng.choice(list("ACGT"), size=G))
    return [g[s:s + 80] for s in rng.integers(0, G - 80, size=n)] + _reads_mixed(rng, 30, 20, 90)


@pytest.mark.parametrize("k", [5, 21, 32, 33, 64])
def test_cturtle_large_filter_reports_each_repeated_kmer_once(k):
    """With every key collision-free (a filter far larger than the key set), cTurtle reports
    exactly the k-mers seen at least twice, each once (string brute force)."""
    reads = _ct_reads(300 + k, 120)
    bases, offs = brute.pack(reads)
    n_sectors = 1 << 20
    keys, nw = oracle.cturtle(bases, offs, k, n_sectors)
    assert nw == brute.n_windows(reads, k)
    got = [brute.decode(x, k) for x in keys]
    assert len(got) == len(set(got))
    assert set(got) == set(brute.kmer_counts(reads, k, 2))
    distinct, _, _ = oracle.count(bases, offs, k, 1)
    assert oracle.cturtle_collision_free(distinct, n_sectors).all()


def test_cturtle_stages_by_hand():
    """k = 3: AAA seen 4 times, AAC once, ACG twice (its reverse complement CGT is the same
    k-mer): reported AAA then ACG, in the order of their second sightings, each once."""
    reads = ["AAAC", "AAA", "ACGT", "AAAA"]  # windows: AAA AAC | AAA | ACG CGT(=ACG) | AAA AAA
    bases, offs = brute.pack(reads)
    keys, nw = oracle.cturtle(bases, offs, 3, 1 << 16)
    assert nw == 7
    assert [brute.decode(x, 3) for x in keys] == ["AAA", "ACG"]


@pytest.mark.parametrize("n_sectors", [1 << 6, 1 << 9])
def test_cturtle_collision_free_keys_follow_their_counts(n_sectors):
    """In a crowded filter, a key no other key's patterns can cover is reported exactly when it
    occurs at least twice; colliding keys may be missed (false negatives) or reported as
    singletons (false positives), but nothing is reported twice and nothing foreign appears."""
    reads = _ct_reads(9, 200, G=3000)
    bases, offs = brute.pack(reads)
    k = 21
    keys, _ = oracle.cturtle(bases, offs, k, n_sectors)
    distinct, counts, _ = oracle.count(bases, offs, k, 1)
    free = oracle.cturtle_collision_free(distinct, n_sectors)
    assert 0 < free.sum() < len(free)  # both kinds present
    rep = set(int(x) for x in keys)
    assert len(rep) == len(keys) and rep <= set(int(x) for x in distinct)
    for key, c, f in zip(distinct, counts, free):
        if f:
            assert (int(key) in rep) == (c >= 2)


def test_cturtle_error_rates_shrink_with_the_filter():
    """Sec. 2.2: false positives plus false negatives against the exact set of k-mers seen twice
    fall as the filter grows (4,594 such k-mers here): hundreds with 64 sectors, a handful at most
    once the filter has ~15 bits per distinct k-mer."""
    reads = _ct_reads(21, 300, G=6000)
    bases, offs = brute.pack(reads)
    k = 25
    truth = set(int(x) for x in oracle.count(bases, offs, k, 2)[0])
    errs = []
    for n_sectors in (1 << 6, 1 << 8, 1 << 10, 1 << 13, 1 << 16):
        rep = set(int(x) for x in oracle.cturtle(bases, offs, k, n_sectors)[0])
        errs.append(len(rep - truth) + len(truth - rep))
    assert errs[0] > errs[1] > errs[2] and errs[0] > 0.2 * len(truth)
    assert max(errs[3:]) <= 2
