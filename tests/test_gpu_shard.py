"""Key-range shards on the GPU (params.shard_index / shard_count), through the C ABI, vs the oracle.

Every shard reads all the reads and counts only its key range; concatenating the shards in order
must give the whole result, bit-exact. The shards run one after another on one GPU (in a
multi-GPU job each rank runs one of them; nothing here waits on another shard).
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


def _concat(parts, w):
    keys = np.concatenate([p[0] for p in parts], axis=0) if parts else np.zeros((0, 2) if w == 2 else 0, np.uint64)
    counts = np.concatenate([p[1] for p in parts]) if parts else np.zeros(0, np.uint32)
    return keys, counts


@pytest.mark.parametrize("k", [15, 31, 33, 64])
@pytest.mark.parametrize("n_shards", [2, 3, 8])
@pytest.mark.parametrize("budget", [0, 1])
def test_device_shards_concatenate_to_the_whole_count(ctx, k, n_shards, budget):
    import torch

    import paper_1305_1861_gb300 as pkg
    from paper_1305_1861_gb300 import shard

    s = synth.longk(seed=21, scale=0.001, k=k)
    b, o = s.chunk(0, s.n_reads)
    db, do = torch.from_numpy(b).cuda(), torch.from_numpy(o.astype(np.int64)).cuda()
    parts, ranges = [], 0
    for r in range(n_shards):
        p = shard.shard_params(r, n_shards, pkg.Params.default(budget_mib=budget))
        keys, counts, nw = ctx.turtle_count_device(db, do, k, 2, p)
        parts.append((keys.cpu().numpy().astype(np.uint64), counts.cpu().numpy().astype(np.uint32)))
        ranges += ctx.stats()["super_partitions"]
    gk, gc = _concat(parts, 2 if k > 32 else 1)
    ok, oc, onw = oracle.count(b, o, k, 2)
    assert nw == onw
    assert gk.shape == ok.shape and np.array_equal(gk, ok)
    assert np.array_equal(gc.astype(np.uint64), oc)
    if budget:
        assert ranges > n_shards  # a small budget splits shards into further key ranges


def test_host_shards_and_argument_checks(ctx):
    import paper_1305_1861_gb300 as pkg
    from paper_1305_1861_gb300 import shard

    lib = synth.small(seed=5, scale=0.05)
    parts = [pkg.turtle_count(lib.bases, lib.offsets, 31, 3, shard.shard_params(r, 4))[:2] for r in range(4)]
    gk, gc = _concat(parts, 1)
    ok, oc, _ = oracle.count(lib.bases, lib.offsets, 31, 3)
    assert np.array_equal(gk, ok) and np.array_equal(gc.astype(np.uint64), oc)
    for bad in (dict(shard_count=2, shard_index=2), dict(shard_count=65), dict(shard_count=2, compact=3)):
        with pytest.raises(pkg.TurtleError) as e:
            pkg.turtle_count(lib.bases, lib.offsets, 31, 2, pkg.Params.default(**bad))
        assert e.value.code == -1
