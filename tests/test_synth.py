"""The seeded input generator: reproducible, chunkable, and shaped as specified."""
import numpy as np

import synth
from tests import brute


def test_deterministic_and_thread_independent():
    g1 = synth.genome_iid(9, 100_000, threads=1)
    g2 = synth.genome_iid(9, 100_000, threads=7)
    assert np.array_equal(g1, g2)
    b1, o1 = synth.reads_uniform(g1, 3, 2000, 100, 0.01, 0.001, threads=1)
    b2, o2 = synth.reads_uniform(g1, 3, 2000, 100, 0.01, 0.001, threads=5)
    assert np.array_equal(b1, b2) and np.array_equal(o1, o2)
    assert set(np.unique(g1).tolist()) == set(b"ACGT")


def test_chunks_equal_the_whole():
    g = synth.genome_iid(4, 50_000)
    full, _ = synth.reads_uniform(g, 8, 1000, 150, 0.01)
    part, off = synth.reads_uniform(g, 8, 300, 150, 0.01, first=400)
    assert np.array_equal(part, full[400 * 150:700 * 150]) and off[-1] == 300 * 150


def test_error_free_reads_are_genome_substrings():
    g = synth.genome_iid(5, 20_000)
    gs = g.tobytes().decode()
    b, o = synth.reads_uniform(g, 6, 200, 100, 0.0, 0.0)
    for i in range(200):
        r = b[o[i]:o[i + 1]].tobytes().decode()
        assert r in gs or brute.revcomp(r) in gs


def test_substitution_and_n_rates():
    g = synth.genome_iid(5, 200_000)
    clean, _ = synth.reads_uniform(g, 6, 20_000, 100, 0.0, 0.0)
    noisy, _ = synth.reads_uniform(g, 6, 20_000, 100, 0.01, 0.0)
    diff = clean != noisy
    assert abs(diff.mean() - 0.01) < 0.001
    assert np.all(noisy[diff] != clean[diff])
    with_n, _ = synth.reads_uniform(g, 6, 20_000, 100, 0.01, 0.0005)
    assert abs((with_n == ord("N")).mean() - 0.0005) < 0.0001


def test_repeat_genome_shape():
    g = synth.genome_repeats(2, 1_000_000)
    assert 1_050_000 <= g.size <= 1_000_000 + 50_000 + 100_000


def test_region_plan_lognormal_coverage():
    G = 2_000_000
    prefix = synth.region_plan(3, G, 10_000, 20.0, 1.0, 150)
    per_region = np.diff(prefix.astype(np.int64)) * 150 / 10_000
    med = np.median(per_region)
    assert 16 < med < 24
    assert per_region.max() > 3 * med  # heavy right tail of the amplification skew
    lib = synth.longk(scale=0.002)
    b, o = lib.chunk(0, 100)
    assert b.size == 100 * 150 and o[-1] == 15000


def test_workload_specs():
    specs = synth.batched_specs()
    assert len(specs) == 64 and {s["k"] for s in specs} <= {21, 31, 55}
    assert all(100_000 <= s["G"] <= 20_000_000 and 10 <= s["cov"] <= 60 for s in specs)
    jobs = synth.served_jobs(n_jobs=200)
    t = np.array([j["t"] for j in jobs])
    assert np.all(np.diff(t) > 0) and 2.0 < t[-1] < 6.0
    assert {j["k"] for j in jobs} <= {25, 31, 63} and {j["min_count"] for j in jobs} <= {2, 3}
