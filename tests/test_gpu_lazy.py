"""Lazy sort-and-compact phases (compact = 3, the memory-capped form) vs the oracle, bit-exact.

A small device budget cuts the reads into many chunks, so the running array is merged many
times (keys present in both inputs, in one, runs of either input exhausted first, chunks whose
candidates are all new or all old); a large budget takes them in one chunk. Every case is
compared with the oracle's plain count.
"""
import numpy as np
import pytest

import oracle
import synth
from tests import brute

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(have_gpu):
    import paper_1305_1861_gb300 as pkg

    pkg.build()
    c = pkg.Context(0)
    yield c
    c.close()


def _check(ctx, bases, offs, k, min_count, params):
    import torch

    b = torch.from_numpy(np.ascontiguousarray(bases)).cuda()
    o = torch.from_numpy(np.ascontiguousarray(offs).astype(np.int64)).cuda()
    keys, counts, nw = ctx.turtle_count_device(b, o, k, min_count, params)
    ok, oc, onw = oracle.count(bases, offs, k, min_count)
    assert nw == onw
    gk = keys.cpu().numpy().astype(np.uint64)
    assert gk.shape == ok.shape and np.array_equal(gk, ok)
    assert np.array_equal(counts.cpu().numpy().astype(np.uint64), oc)
    return ctx.stats()


@pytest.mark.parametrize("k", [5, 21, 31, 32, 33, 55, 64])
@pytest.mark.parametrize("min_count", [1, 2, 3])
@pytest.mark.parametrize("budget", [1, 512])
def test_lazy_form_matches_oracle(ctx, k, min_count, budget):
    import paper_1305_1861_gb300 as pkg

    lib = synth.small(seed=100 + k, scale=0.05)  # 50 kbp genome, 10,000 reads, 1% errors
    st = _check(ctx, lib.bases, lib.offsets, k, min_count, pkg.Params.default(compact=3, budget_mib=budget))
    if budget == 1:
        assert st["chunks"] > 4
    else:
        assert st["chunks"] == 1
    merges = st["stage_launches"]["merge"] // 2  # chunks after the first that had candidates
    assert merges <= st["chunks"] - 1 and (merges > 0 or st["chunks"] == 1)


def test_lazy_form_fly_shaped_with_repeats_and_n(ctx):
    """Repeat copies and ambiguous calls, 1/100 scale, many chunks."""
    import paper_1305_1861_gb300 as pkg

    lib = synth.fly(seed=2, scale=0.01)
    st = _check(ctx, lib.bases, lib.offsets, 31, 2, pkg.Params.default(compact=3, budget_mib=16))
    assert st["chunks"] > 4


def test_lazy_form_long_k_with_skewed_coverage(ctx):
    import paper_1305_1861_gb300 as pkg

    s = synth.longk(seed=9, scale=0.002)
    b, o = s.chunk(0, s.n_reads)
    for mc in (2, 3):
        st = _check(ctx, b, o, 64, mc, pkg.Params.default(compact=3, budget_mib=64))
        assert st["chunks"] > 4


def test_lazy_form_saturated_filter(ctx):
    """A filter far too small: nearly every window becomes a candidate; counts stay exact."""
    import paper_1305_1861_gb300 as pkg

    lib = synth.small(seed=7, scale=0.05)
    p = pkg.Params.default(compact=3, budget_mib=2, filter_bits_per_window=0.01, pattern_bits=1, n_patterns=1)
    st = _check(ctx, lib.bases, lib.offsets, 31, 2, p)
    assert st["n_unique"] > st["n_out"]


def test_lazy_form_chunks_without_candidates_and_edge_inputs(ctx):
    """Stretches of ambiguous calls leave whole chunks without a window; a repeated read gives a count
    above 2^16 that is merged across many chunks; tiny and empty inputs."""
    import paper_1305_1861_gb300 as pkg

    reads = ["N" * 5000] * 40 + ["ACGT" * 25] * 3 + ["A" * 100] * 1200 + ["N" * 3000] * 40 + ["ACGT" * 25] * 2
    bases, offs = brute.pack(reads)
    p = pkg.Params.default(compact=3, budget_mib=1)
    for k in (15, 31, 64):
        for mc in (1, 2):
            _check(ctx, bases, offs, k, mc, p)
    for reads in (["ACG"], ["N" * 50], ["ACGTACGTAC"]):
        bases, offs = brute.pack(reads)
        _check(ctx, bases, offs, 5, 2, p)
