"""Why the bucketed sort-and-compact uses f(v) = v (2^32 - v) on the top 31 key bits (CPU).

For a random k-mer, the forward and reverse-complement keys are (close to) independent and
uniform, so the canonical key (their minimum) has the distribution of the minimum of two uniforms:
with u = top31 / 2^31, P(U <= u) = 1 - (1 - u)^2 = 2u - u^2. And f(v) / 2^62 = 2u - u^2 exactly,
so f maps canonical keys to a uniform variable: equal slices of f hold about equal numbers of
keys. These tests check that algebra and measure the balance on the canonical keys the oracle
reports for a random library.
"""
import numpy as np

import oracle
import synth


def f_of(top31: np.ndarray) -> np.ndarray:
    v = top31.astype(np.uint64)
    return v * (np.uint64(1 << 32) - v)


def test_f_is_the_cdf_of_the_minimum_of_two_uniforms():
    v = np.array([0, 1, 1 << 20, 1 << 30, (1 << 31) - 1, 1 << 31], dtype=np.uint64)
    u = v.astype(np.float64) / 2.0 ** 31
    assert np.allclose(f_of(v).astype(np.float64) / 2.0 ** 62, 2 * u - u * u, rtol=1e-12, atol=1e-15)
    f = f_of(v)
    assert np.all(f[1:] > f[:-1])  # strictly increasing (in integers): buckets stay key ranges


def test_canonical_keys_of_random_reads_fill_f_buckets_evenly():
    k = 31
    lib = synth.small(seed=11, scale=0.2)  # 200 kbp genome, 40,000 reads: ~2.8M windows
    keys, counts, _ = oracle.count(lib.bases, lib.offsets, k, 1)
    top = keys >> np.uint64(2 * k - 31)
    n_buckets = 256
    by_f = (f_of(top) >> np.uint64(62 - 8)).astype(np.int64)  # 256 equal slices of f
    by_top = (top >> np.uint64(31 - 8)).astype(np.int64)  # 256 equal slices of the key itself
    occ_f = np.bincount(by_f, weights=counts.astype(np.float64), minlength=n_buckets)
    occ_top = np.bincount(by_top, weights=counts.astype(np.float64), minlength=n_buckets)
    mean = counts.sum() / n_buckets
    # f: every bucket within 15% of the mean (sampling noise at ~11k windows per bucket is ~1%,
    # plus the genome's own k-mer repeats); raw key slices: the low ones hold about twice the
    # mean and the top ones almost nothing
    assert occ_f.max() < 1.15 * mean and occ_f.min() > 0.85 * mean
    assert occ_top[:8].mean() > 1.8 * mean and occ_top[-8:].mean() < 0.2 * mean
