"""Error paths, made to fire from the host (include/turtle_testing.h); nothing here faults a GPU.

* the n-th device scratch allocation of a call fails -> TURTLE_E_NOMEM, and the context's pool
  holds no buffer of the failed call afterwards;
* a host result allocation fails -> TURTLE_E_NOMEM;
* a look-back wait whose predecessor tile never runs expires after a short, bounded number of
  rounds -> the kernel sets its error word and returns -> TURTLE_E_DEVICE;
* pass 1 given less candidate room than it needs -> TURTLE_E_CAPACITY.
After each failure the same context (or the library) must count correctly again.
"""
import time

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

NOMEM, DEVICE, CAPACITY = -2, -7, -9


@pytest.fixture(scope="module")
def env(have_gpu):
    import torch

    import paper_1305_1861_gb300 as pkg

    pkg.build()
    lib = pkg.load()
    ctx = pkg.Context(0)
    small = synth.small(seed=17, scale=0.05)
    dev = (torch.from_numpy(small.bases).cuda(), torch.from_numpy(small.offsets.astype(np.int64)).cuda())
    ref = oracle.count(small.bases, small.offsets, 31, 2)
    yield pkg, lib, ctx, small, dev, ref
    lib.turtle_test_inject(0, 0)
    ctx.close()


def _count_ok(pkg, ctx, dev, ref, params=None):
    keys, counts, nw = ctx.turtle_count_device(dev[0], dev[1], 31, 2, params)
    assert nw == ref[2]
    assert np.array_equal(keys.cpu().numpy().astype(np.uint64), ref[0])
    assert np.array_equal(counts.cpu().numpy().astype(np.uint64), ref[1])


@pytest.mark.parametrize("compact", [0, 1, 3])
def test_device_allocation_failure_frees_everything(env, compact):
    pkg, lib, ctx, small, dev, ref = env
    p = pkg.Params.default(compact=compact, budget_mib=4 if compact == 3 else 0)
    failed = 0
    for n in (0, 1, 2, 3, 5, 8, 13, 21):
        assert lib.turtle_test_inject(1, n) == 0
        try:
            ctx.turtle_count_device(dev[0], dev[1], 31, 2, p)
        except pkg.TurtleError as e:
            assert e.code == NOMEM
            failed += 1
            used, _ = ctx.pool_bytes()
            assert used == 0  # neither the failed call's scratch nor a stale result is held
        finally:
            lib.turtle_test_inject(0, 0)
        _count_ok(pkg, ctx, dev, ref, p)
    assert failed >= 5


def test_host_result_allocation_failure(env):
    pkg, lib, ctx, small, dev, ref = env
    for n in (0, 1):
        assert lib.turtle_test_inject(2, n) == 0
        with pytest.raises(pkg.TurtleError) as e:
            pkg.turtle_count(small.bases, small.offsets, 31, 2)
        assert e.value.code == NOMEM
        lib.turtle_test_inject(0, 0)
    keys, counts, nw = pkg.turtle_count(small.bases, small.offsets, 31, 2)
    assert np.array_equal(keys, ref[0]) and np.array_equal(counts.astype(np.uint64), ref[1])


def test_expired_lookback_wait_returns_device_error(env):
    """The merge's tiles get tickets from 1: tile 0 never publishes, its successors give up after
    4096 rounds, flag the error and finish; the call reports TURTLE_E_DEVICE within a short time."""
    pkg, lib, ctx, small, dev, ref = env
    p = pkg.Params.default(compact=3, budget_mib=2)  # many chunks: merges of several tiles each
    assert lib.turtle_test_inject(3, 4096) == 0
    t0 = time.time()
    with pytest.raises(pkg.TurtleError) as e:
        ctx.turtle_count_device(dev[0], dev[1], 31, 2, p)
    assert e.value.code == DEVICE
    assert time.time() - t0 < 30
    lib.turtle_test_inject(0, 0)
    _count_ok(pkg, ctx, dev, ref, p)
    _count_ok(pkg, ctx, dev, ref)


def test_candidate_room_overflow_returns_capacity_error(env):
    pkg, lib, ctx, small, dev, ref = env
    for cap in (1, 1000):
        assert lib.turtle_test_inject(4, cap) == 0
        with pytest.raises(pkg.TurtleError) as e:
            ctx.turtle_count_device(dev[0], dev[1], 31, 2)
        assert e.value.code == CAPACITY
        lib.turtle_test_inject(0, 0)
    _count_ok(pkg, ctx, dev, ref)


def test_unknown_injection_is_refused(env):
    pkg, lib, ctx, small, dev, ref = env
    assert lib.turtle_test_inject(99, 1) == -1
    assert lib.turtle_test_inject(3, 0) == -1
