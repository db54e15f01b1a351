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
