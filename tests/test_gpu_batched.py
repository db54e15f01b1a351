"""Batched form: many libraries, mixed k, one pipeline per (k, min_count) group; each result is exact."""
import numpy as np
import pytest

import oracle
import synth
from tests import brute

pytestmark = pytest.mark.gpu


def _lib(seed, G, cov, R, k, m, err=0.01):
    g = synth.genome_iid(seed, G)
    n = max(1, int(cov * G / R))
    b, o = synth.reads_uniform(g, seed, n, R, err)
    return (b, o, k, m)


@pytest.mark.parametrize("compact", [0, 1, 2])
def test_batch_matches_oracle_per_library(have_gpu, compact):
    """Every form of counting (bucketed: per-library bucket ranges; global: recount table; hash table:
    one table keyed by the library-tagged keys)."""
    import paper_1305_1861_gb300 as pkg

    jobs = []
    for i in range(10):  # one k=21 run holds all ten
        jobs.append(_lib(100 + i, 2000 + 700 * i, 15, 100, 21, 2))
    for i in range(6):  # k=31: four libraries per run -> two runs
        jobs.append(_lib(200 + i, 3000 + 500 * i, 12, 150, 31, 2 + (i == 5)))
    for i in range(5):
        jobs.append(_lib(300 + i, 2500 + 900 * i, 20, 150, 55, 2))
    jobs.append(_lib(400, 5000, 10, 100, 32, 2))
    jobs.append(_lib(401, 5000, 10, 150, 64, 2))
    jobs.append((np.zeros(0, np.uint8), np.zeros(1, np.uint64), 21, 2))  # empty library
    b, o = brute.pack(["ACGT" * 30, "NNACGTACGTAAAATTTT" * 5])
    jobs.append((np.concatenate([np.frombuffer(b"TTT", np.uint8), b]), o + 3, 21, 2))  # offsets start past 0
    got = pkg.turtle_count_batch(jobs, pkg.Params.default(compact=compact))
    assert len(got) == len(jobs)
    for (b, o, k, m), (keys, counts, nw) in zip(jobs, got):
        ok, oc, onw = oracle.count(b, o, k, m)
        assert nw == onw
        assert np.array_equal(keys, ok) and np.array_equal(counts.astype(np.uint64), oc), (k, m, len(oc))


def test_batch_equals_plain_calls(have_gpu):
    import paper_1305_1861_gb300 as pkg

    specs = synth.batched_specs(seed=4, n_libs=12, scale=0.01)
    jobs = [(l.bases, l.offsets, l.k, l.min_count) for l in map(synth.library_from_spec, specs)]
    got = pkg.turtle_count_batch(jobs)
    for (b, o, k, m), (keys, counts, nw) in zip(jobs, got):
        pk, pc, pn = pkg.turtle_count(b, o, k, m)
        assert nw == pn and np.array_equal(keys, pk) and np.array_equal(counts, pc)


def test_batch_overlapped_copy_equals_plain_calls(have_gpu):
    """A batch of more than 64 MiB copies its libraries in chunks while earlier chunks are packed
    and filtered (chunks straddle library boundaries); each result equals the plain call's."""
    import paper_1305_1861_gb300 as pkg

    specs = synth.batched_specs(seed=7, n_libs=10, scale=0.1)
    for sp in specs:
        sp["k"] = 21  # one run holds them all: ~100 Mbase
    jobs = [(l.bases, l.offsets, l.k, l.min_count) for l in map(synth.library_from_spec, specs)]
    assert sum(b.size for b, _, _, _ in jobs) >= 64 << 20
    got = pkg.turtle_count_batch(jobs)
    for (b, o, k, m), (keys, counts, nw) in zip(jobs, got):
        pk, pc, pn = pkg.turtle_count(b, o, k, m)
        assert nw == pn and np.array_equal(keys, pk) and np.array_equal(counts, pc)


def _mixed_jobs():
    """Libraries of many k (2 .. 64) and three min_counts; lengths both multiples of 128 and not, so
    some libraries follow one another without a gap and some with one."""
    jobs = []
    ks = [2, 5, 13, 21, 31, 32, 33, 45, 55, 61, 62, 64]
    for i in range(70):  # 70 libraries that a mixed run can hold with min_count 2: two mixed runs
        k = ks[i % 10]
        jobs.append(_lib(500 + i, 600 + 97 * i, 8, 64 + (i % 3) * 32, k, 2))
    for i, k in enumerate(ks):  # min_count 3 and 1, with k 62 and 64 in runs of their own
        jobs.append(_lib(600 + i, 1500 + 211 * i, 10, 100, k, 3))
        jobs.append(_lib(700 + i, 1000 + 128 * i, 6, 128, k, 1))
    jobs.append((np.zeros(0, np.uint8), np.zeros(1, np.uint64), 21, 2))  # empty library
    b, o = brute.pack(["ACGT" * 32, "NNACGTACGTAAAATTTT" * 5])
    jobs.append((np.concatenate([np.frombuffer(b"TTT", np.uint8), b]), o + 3, 45, 2))  # offsets start past 0
    b, o = brute.pack(["ACGTTGCA" * 16])  # exactly 128 bases, then the next library without a gap
    jobs.append((b, o, 31, 2))
    b, o = brute.pack(["ACGTNACGGT" * 20, "TTTT", "N" * 40])  # k = 1 (single bases), reads of Ns only
    jobs.append((b, o, 1, 2))
    b, o = brute.pack(["N" * 300])  # no valid window at all
    jobs.append((b, o, 21, 2))
    return jobs


@pytest.mark.parametrize("mixed", [1, 0, 2])
def test_mixed_k_batch_matches_oracle_per_library(have_gpu, mixed):
    """Mixed runs (batch_mixed = 1: libraries of different k share a run, keys of 128 bits tagged in
    the top 6) give every library exactly the oracle's result, as do the automatic choice (0) and
    runs grouped by k (2)."""
    import paper_1305_1861_gb300 as pkg

    jobs = _mixed_jobs()
    got = pkg.turtle_count_batch(jobs, pkg.Params.default(batch_mixed=mixed))
    assert len(got) == len(jobs)
    for (b, o, k, m), (keys, counts, nw) in zip(jobs, got):
        ok, oc, onw = oracle.count(b, o, k, m)
        assert nw == onw, (k, m)
        assert keys.ndim == ok.ndim == (1 if k <= 32 else 2)
        assert np.array_equal(keys, ok) and np.array_equal(counts.astype(np.uint64), oc), (k, m, len(oc))


def test_mixed_k_batch_other_forms_fall_back_to_grouped_runs(have_gpu):
    """batch_mixed asks for mixed runs, but the global and hash-table forms keep runs of one k."""
    import paper_1305_1861_gb300 as pkg

    jobs = _mixed_jobs()[:24]
    for compact in (1, 2):
        got = pkg.turtle_count_batch(jobs, pkg.Params.default(batch_mixed=1, compact=compact))
        for (b, o, k, m), (keys, counts, nw) in zip(jobs, got):
            ok, oc, onw = oracle.count(b, o, k, m)
            assert nw == onw and np.array_equal(keys, ok) and np.array_equal(counts.astype(np.uint64), oc)


def test_mixed_k_batch_refuses_bad_mode(have_gpu):
    import paper_1305_1861_gb300 as pkg

    with pytest.raises(pkg.TurtleError):
        pkg.turtle_count_batch(_mixed_jobs()[:4], pkg.Params.default(batch_mixed=3))
