"""cTurtle (Sec. 2.2) on the GPU vs the CPU oracle.

The two-stage counting filter is approximate, and for keys whose patterns collide with other
keys' patterns the outcome depends on the order the windows are taken in, which differs between
the GPU and the sequential oracle. The oracle therefore classifies every distinct key: a key no
other key's patterns can cover is reported exactly when it occurs at least twice, under any
order, and the GPU must agree on all such keys; for the rest, the GPU may only report each key
once and only keys of the input.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(have_gpu):
    import paper_1305_1861_gb300 as pkg

    pkg.build()
    c = pkg.Context(0)
    yield c
    c.close()


def _n_sectors(W, bits):
    x = int(W * bits / 256.0) + 1
    n = 1 << (x - 1).bit_length()
    return max(n, 2)


def _keyset(keys):
    a = np.asarray(keys, dtype=np.uint64)
    return set(map(tuple, a.tolist())) if a.ndim == 2 else set(a.tolist())


def _run(ctx, bases, offs, k, bits):
    import torch
    import paper_1305_1861_gb300 as pkg

    b = torch.from_numpy(np.ascontiguousarray(bases)).cuda()
    o = torch.from_numpy(np.ascontiguousarray(offs).astype(np.int64)).cuda()
    keys, nw = ctx.turtle_frequent_device(b, o, k, pkg.Params.default(cturtle_bits_per_window=bits))
    return keys.cpu().numpy().astype(np.uint64), nw


def _check(ctx, bases, offs, k, bits, result=None):
    gk, nw = result if result is not None else _run(ctx, bases, offs, k, bits)
    distinct, counts, onw = oracle.count(bases, offs, k, 1)
    assert nw == onw
    free = oracle.cturtle_collision_free(distinct, _n_sectors(nw, bits))
    got = _keyset(gk)
    assert len(got) == len(gk)  # each key at most once
    if k <= 32 and len(gk) > 1:
        assert np.all(np.diff(gk) > 0)  # ascending
    elif len(gk) > 1:
        t = [tuple(x) for x in gk.tolist()]
        assert t == sorted(t)
    allk = _keyset(distinct)
    assert got <= allk  # nothing foreign
    dk = distinct.tolist()
    for key, c, f in zip(dk, counts.tolist(), free.tolist()):
        if f:
            kk = tuple(key) if k > 32 else key
            assert (kk in got) == (c >= 2), (kk, c)
    return free, got, counts


@pytest.mark.parametrize("k", [15, 21, 31, 32, 33, 55, 64])
def test_frequent_near_exact_with_a_large_filter(ctx, k):
    """64 bits per window: over 99.5% of keys are collision-free; the GPU result differs from the
    exact set of k-mers seen twice at most on the few colliding keys."""
    lib = synth.small(seed=60 + k, scale=0.02)
    free, got, counts = _check(ctx, lib.bases, lib.offsets, k, 64)
    assert free.mean() > 0.995
    assert abs(len(got) - int((counts >= 2).sum())) <= int((~free).sum())


@pytest.mark.parametrize("k,bits", [(21, 1), (31, 2), (31, 8), (45, 2)])
def test_frequent_collision_free_keys_in_a_crowded_filter(ctx, k, bits):
    lib = synth.small(seed=80 + k, scale=0.05)
    free, got, counts = _check(ctx, lib.bases, lib.offsets, k, bits)
    assert 0 < free.sum() < len(free)


def test_frequent_host_form(ctx):
    """Host memory in and out: the same guarantees (two runs may differ on colliding keys only)."""
    import paper_1305_1861_gb300 as pkg

    lib = synth.small(seed=5, scale=0.05)
    for k, bits in ((31, 8), (63, 4)):
        hk, hn = pkg.turtle_frequent(lib.bases, lib.offsets, k, pkg.Params.default(cturtle_bits_per_window=bits))
        _check(ctx, lib.bases, lib.offsets, k, bits, result=(np.asarray(hk, dtype=np.uint64), hn))


def test_frequent_error_rate_at_default_size(ctx):
    """Default 8 bits per window on a fly-shaped library at 1/100 scale: false positives plus false
    negatives stay under 1% of the k-mers seen twice."""
    import torch
    import paper_1305_1861_gb300 as pkg

    lib = synth.fly(seed=2, scale=0.01)
    b = torch.from_numpy(lib.bases).cuda()
    o = torch.from_numpy(lib.offsets.astype(np.int64)).cuda()
    keys, nw = ctx.turtle_frequent_device(b, o, 31)
    got = set(keys.cpu().numpy().astype(np.uint64).tolist())
    truth = set(oracle.count(lib.bases, lib.offsets, 31, 2)[0].tolist())
    err = len(got - truth) + len(truth - got)
    assert err < 0.01 * len(truth)


def test_frequent_edge_inputs(ctx):
    from tests import brute

    for reads in (["ACG"], ["N" * 40], ["ACGTACGTAC", "ACGTACGTAC"]):
        bases, offs = brute.pack(reads)
        gk, nw = _run(ctx, bases, offs, 5, 8)
        truth = oracle.count(bases, offs, 5, 2)[0]
        assert _keyset(gk) == _keyset(truth)
