"""Parity at the sizes the benchmark times, in the launch configuration it times (GPU vs oracle).

* fly-shaped library at full size (105 Mbp genome with repeat copies, 30M x 100 bp, 0.05% N,
  2.07G windows, k = 31, min_count = 2): every reported (key, count) pair and the window count
  compared with the oracle's full count, element by element;
* long-k library (k = 64, 128-bit keys) at 1/10 scale with a device budget that splits the key
  space into the same four key ranges as the full-size run: compared in full with the oracle;
* long-k at full size (19.1G windows, four key ranges): properties that hold at any size (the
  window count's closed form, strictly ascending keys, counts >= min_count, their sum <= W) and a
  sampled exact check through oracle.count_queries: sampled reported keys must carry their exact
  counts, and every key of sampled random windows that is missing from the output must occur
  fewer than min_count times.

Expected values come from the oracle only (oracle.count / oracle.count_queries / oracle.windows).
"""
import os
import time

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 1


@pytest.fixture(scope="module")
def ctx(have_gpu):
    import paper_1305_1861_gb300 as pkg

    pkg.build()
    c = pkg.Context(0)
    yield c
    c.close()


def _bench_params(pkg, **kw):
    return pkg.Params.default(timing=1, **kw)  # the benchmark records stage events


def _device_count(ctx, bases, offsets, k, min_count, params):
    import torch

    b = torch.from_numpy(bases).cuda()
    o = torch.from_numpy(offsets.astype(np.int64)).cuda()
    keys, counts, nw = ctx.turtle_count_device(b, o, k, min_count, params)
    torch.cuda.synchronize()
    hk = keys.cpu().numpy().view(np.uint64)
    hc = counts.cpu().numpy().view(np.uint32)
    st = ctx.stats()
    del b, o, keys, counts
    torch.cuda.empty_cache()
    return hk, hc, nw, st


def test_fly_shaped_full_size_matches_oracle(ctx):
    """The benchmark's headline workload, compared in full."""
    import paper_1305_1861_gb300 as pkg

    lib = synth.fly(seed=2, scale=1.0)
    gk, gc, nw, st = _device_count(ctx, lib.bases, lib.offsets, 31, 2, _bench_params(pkg))
    assert st["super_partitions"] == 1 and st["n_windows"] > 2_000_000_000
    t0 = time.time()
    ok, oc, onw = oracle.count(lib.bases, lib.offsets, 31, 2, threads=THREADS)
    print("oracle: %d windows in %.1f s on %d threads" % (onw, time.time() - t0, THREADS))
    assert nw == onw
    assert gk.shape == ok.shape and np.array_equal(gk, ok)
    assert np.array_equal(gc.astype(np.uint64), oc)


def _longk_windows(offsets, k):
    lens = np.diff(offsets.astype(np.int64))
    return int(np.maximum(lens - k + 1, 0).sum())  # the long-k recipe has no ambiguous calls


def test_longk_tenth_scale_in_four_key_ranges_matches_oracle(ctx):
    """k = 64 (128-bit keys) at 1/10 scale (100 Mbp, 3.3 Gbase, 1.9G windows), with a budget that
    splits the key space into the same four key ranges as the full-size run."""
    import paper_1305_1861_gb300 as pkg

    s = synth.longk(seed=3, scale=0.1)
    b, o = s.chunk(0, s.n_reads)
    W = _longk_windows(o, 64)
    per_window = 2 * 16 + 8 + 1.0 / 8  # the bucketed form's working set per window of a key range
    budget_mib = int(W * per_window / 3.5 / (1 << 20))  # ceil(W * per_window / budget) = 4
    gk, gc, nw, st = _device_count(ctx, b, o, 64, 2, _bench_params(pkg, budget_mib=budget_mib))
    assert st["super_partitions"] == 4
    assert nw == W
    ok, oc, onw = oracle.count(b, o, 64, 2, threads=THREADS)
    assert nw == onw
    gk = gk.reshape(-1, 2)
    assert gk.shape == ok.shape and np.array_equal(gk, ok)
    assert np.array_equal(gc.astype(np.uint64), oc)


def _sorted_u128(keys):
    hi, lo = keys[:, 0], keys[:, 1]
    return bool(np.all((hi[1:] > hi[:-1]) | ((hi[1:] == hi[:-1]) & (lo[1:] > lo[:-1]))))


def _member(sorted_keys, q):
    """For 128-bit keys q[i] = (hi, lo): index in the ascending sorted_keys, or -1."""
    hi, lo = sorted_keys[:, 0], sorted_keys[:, 1]
    a = np.searchsorted(hi, q[:, 0], side="left")
    e = np.searchsorted(hi, q[:, 0], side="right")
    idx = np.full(q.shape[0], -1, np.int64)
    for i in range(q.shape[0]):
        if e[i] > a[i]:
            j = a[i] + np.searchsorted(lo[a[i]:e[i]], q[i, 1])
            if j < e[i] and lo[j] == q[i, 1]:
                idx[i] = j
    return idx


def test_longk_full_size_properties_and_sampled_counts(ctx):
    """Long-k at full size (1 Gbp, ~220M x 150 bp, 19.1G windows), the benchmark's launch
    configuration: properties at full size, then 100,000 sampled reported keys and the keys of
    ~100,000 random windows checked against exact counts by the oracle."""
    import paper_1305_1861_gb300 as pkg

    s = synth.longk(seed=3, scale=1.0)
    b, o = s.chunk(0, s.n_reads)
    W = _longk_windows(o, 64)
    gk, gc, nw, st = _device_count(ctx, b, o, 64, 2, _bench_params(pkg))
    gk = gk.reshape(-1, 2)
    print("long-k: %d windows, %d reported, %d key ranges" % (nw, gk.shape[0], st["super_partitions"]))
    assert nw == W and st["super_partitions"] > 1
    assert _sorted_u128(gk)
    assert int(gc.min()) >= 2 and int(gc.astype(np.uint64).sum()) <= W
    rng = np.random.default_rng(64)
    rep = gk[rng.choice(gk.shape[0], 100_000, replace=False)]
    reads = np.sort(rng.choice(s.n_reads, 1_200, replace=False))
    sb = np.concatenate([b[int(o[r]):int(o[r + 1])] for r in reads])
    so = np.concatenate([[0], np.cumsum(np.diff(o.astype(np.int64))[reads])]).astype(np.uint64)
    _, win = oracle.windows(sb, so, 64)
    queries = np.concatenate([rep, win])
    t0 = time.time()
    exact = oracle.count_queries(b, o, 64, queries, threads=THREADS)
    print("oracle queries: %d keys over %d windows in %.1f s" % (queries.shape[0], W, time.time() - t0))
    where = _member(gk, queries)
    found = where >= 0
    assert found[: rep.shape[0]].all()
    assert np.array_equal(gc[where[found]].astype(np.uint64), exact[found])
    assert (exact[~found] < 2).all()  # every key missing from the output occurs once
    assert (~found).sum() > 10_000  # the random windows include many once-seen (error) k-mers
