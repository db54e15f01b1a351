"""Key-range sharding across ranks (Sec. 2.1.5 routing by key), on CPU.

* turtle_shard_bounds (host code of the library, no device): the bounds follow their definition
  (shard s starts at the first part where the windows below reach s/n of all windows), are
  monotone, cover every part once, and balance shards to within one part;
* two gloo ranks: each rank counts its shard -- here the oracle's count restricted to the shard's
  key range, standing in for the GPU call, which needs a GPU -- and rank 0 gathers the shards in
  rank order; the concatenation must equal the oracle's whole-library count. The key -> part map
  f(v) = v (2^32 - v) >> 56 (v = top 31 key bits) is restated here from its definition.
"""
import os
import socket

import numpy as np
import pytest

import oracle
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pkg():
    import paper_1305_1861_gb300 as p

    p.build()
    p.load()
    return p


def _bounds_by_definition(w, n):
    w = [int(x) for x in w]
    total = sum(w)
    b = [0]
    for s in range(1, n):
        p, below = 0, 0
        while p < len(w) and below * n < total * s:
            below += w[p]
            p += 1
        b.append(p)
    b.append(len(w))
    return b


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 64, 100])
def test_shard_bounds_follow_their_definition(pkg, n):
    from paper_1305_1861_gb300 import shard

    rng = np.random.default_rng(n)
    for w in (np.full(64, 1000, np.uint64), rng.integers(0, 10 ** 9, 64).astype(np.uint64),
              np.zeros(64, np.uint64), np.array([0] * 30 + [5] + [0] * 33, np.uint64)):
        b = shard.shard_bounds(w, n)
        assert list(b) == _bounds_by_definition(w, n)
        assert b[0] == 0 and b[-1] == 64 and np.all(np.diff(b.astype(np.int64)) >= 0)
        if w.sum():
            per = np.array([w[b[s]:b[s + 1]].sum() for s in range(n)], dtype=np.float64)
            assert per.sum() == w.sum()
            assert per.max() <= w.sum() / n + w.max()  # within one part of an equal share


def test_equal_parts_split_evenly(pkg):
    from paper_1305_1861_gb300 import shard

    b = shard.shard_bounds(np.full(64, 7, np.uint64), 4)
    assert list(b) == [0, 16, 32, 48, 64]


def test_shard_bounds_reject_bad_arguments(pkg):
    import ctypes

    lib = pkg.load()
    w = np.ones(4, np.uint64)
    out = np.zeros(8, np.uint32)
    assert lib.turtle_shard_bounds(w.ctypes.data, 0, 2, out.ctypes.data) == -1
    assert lib.turtle_shard_bounds(w.ctypes.data, 4, 0, out.ctypes.data) == -1
    assert lib.turtle_shard_bounds(None, 4, 2, out.ctypes.data) == -1
    assert lib.turtle_shard_bounds(w.ctypes.data, 4, 2, ctypes.c_void_p()) == -1


def part_of(keys: np.ndarray, k: int) -> np.ndarray:
    """Part (of 64) of each canonical key: f(top 31 of the 2k key bits) >> 56."""
    if keys.ndim == 2:  # 128-bit keys, k > 32: the top 31 of 2k bits straddle hi / lo
        sh = 2 * k - 31
        hi, lo = keys[:, 0].astype(object), keys[:, 1].astype(object)
        v = np.array([((int(h) << 64 | int(l)) >> sh) & 0x7FFFFFFF for h, l in zip(hi, lo)], dtype=np.uint64)
    else:
        b = 2 * k
        v = (keys >> np.uint64(b - 31)) if b >= 31 else (keys << np.uint64(31 - b))
        v = v & np.uint64(0x7FFFFFFF)
    f = v * (np.uint64(1 << 32) - v)
    return (f >> np.uint64(56)).astype(np.int64)


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _shard_worker(rank, world, port, k, q):
    import sys

    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle as orc
        import synth as syn
        from paper_1305_1861_gb300 import shard
        from tests.test_shard import part_of

        lib = syn.small(seed=33, scale=0.02)
        _, wkeys = orc.windows(lib.bases, lib.offsets, k)  # every window's key: the per-part window counts
        pw = np.bincount(part_of(wkeys, k), minlength=64).astype(np.uint64)

        def count_one_shard(bases, offsets, kk, mc, params):  # the oracle, restricted to this shard's parts
            b = shard.shard_bounds(pw, params.shard_count)
            keys, counts, nw = orc.count(bases, offsets, kk, mc)
            p = part_of(keys, kk)
            sel = (p >= b[params.shard_index]) & (p < b[params.shard_index + 1])
            return keys[sel], counts[sel].astype(np.uint32), nw

        got = shard.count_sharded(lib.bases, lib.offsets, k, 2, count=count_one_shard)
        if rank == 0:
            ok, oc, onw = orc.count(lib.bases, lib.offsets, k, 2)
            q.put((rank, got[2] == onw and np.array_equal(got[0], ok) and np.array_equal(got[1].astype(np.uint64), oc),
                   int(len(oc))))
        else:
            q.put((rank, got is None, 0))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("k", [31, 45])
def test_two_gloo_ranks_gather_shards_in_key_order(pkg, k):
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, k, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = {}
    try:
        for _ in procs:
            rank, ok, n = q.get(timeout=300)
            got[rank] = (ok, n)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert all(p.exitcode == 0 for p in procs)
    assert got[0][0] and got[0][1] > 0  # rank 0: the concatenation equals the whole count
    assert got[1][0]                     # rank 1: sent its shard, holds nothing
