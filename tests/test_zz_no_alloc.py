"""The allocation-free sort-and-compact agrees with the allocating one and with the oracle (GPU,
through the C ABI).

turtle_sort_compact_noalloc is for callers that may not allocate device memory
(fixed budgets, host frameworks that own every allocation, latency-critical
loops); its scratch is one fixed array inside the library's device image and is
shared by every call. Each width is checked on two calls in a row, the second
smaller than the first, so anything the first call left behind in the shared
array would show up in the second result. This file is collected last.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _keys(rng, words, n, bits, distinct):
    if words == 1:
        pool = rng.integers(0, 2 ** 63, size=distinct, dtype=np.uint64) & np.uint64((1 << bits) - 1)
        return pool[rng.integers(0, distinct, size=n)]
    hi = rng.integers(0, 2 ** 62, size=distinct, dtype=np.uint64) & np.uint64((1 << (bits - 64)) - 1)
    lo = rng.integers(0, 2 ** 64, size=distinct, dtype=np.uint64)
    return np.stack([hi, lo], axis=1)[rng.integers(0, distinct, size=n)]


def test_noalloc_matches_allocating_entry_point_on_consecutive_calls(have_gpu):
    import torch

    import oracle
    import paper_1305_1861_gb300 as pkg

    pkg.build()
    lib = pkg.load()
    ctx = pkg.Context(0)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rng = np.random.default_rng(2024)
    cases = [(1, 1 << 20, 62, 60_000), (1, 300_001, 62, 1_000),      # 64-bit keys: at the limit, then smaller
             (2, 1 << 19, 128, 30_000), (2, 70_001, 100, 500)]       # 128-bit keys: at the limit, then smaller
    for words, n, bits, distinct in cases:
        host = _keys(rng, words, n, bits, distinct)
        t = torch.from_numpy(np.ascontiguousarray(host).view(np.int64)).cuda()
        ref_u, ref_c = ctx.turtle_sort_compact(t, bits)
        unique = torch.full_like(t, -1)
        counts = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        nu = ctypes.c_uint64(12345)
        rc = lib.turtle_sort_compact_noalloc(t.data_ptr(), n, words, bits, unique.data_ptr(), counts.data_ptr(),
                                             ctypes.byref(nu), stream)
        assert rc == 0, pkg.turtle_strerror(rc)
        assert nu.value == ref_u.shape[0]
        assert torch.equal(unique[: nu.value], ref_u)
        assert torch.equal(counts[: nu.value], ref_c)
        assert int(counts[: nu.value].sum()) == n
        ok, oc = oracle.sort_compact(host)  # the plain sort-and-compact of Sec. 2.1.4 on the host
        got = unique[: nu.value].cpu().numpy().view(np.uint64)
        assert np.array_equal(got.reshape(ok.shape), ok)
        assert np.array_equal(counts[: nu.value].cpu().numpy().astype(np.uint64), oc)
    ctx.close()


def test_noalloc_refuses_inputs_above_its_limit(have_gpu):
    import torch

    import paper_1305_1861_gb300 as pkg

    lib = pkg.load()
    t = torch.zeros(4, dtype=torch.int64, device="cuda")
    nu = ctypes.c_uint64(7)
    for words, limit in ((1, 1 << 20), (2, 1 << 19)):
        rc = lib.turtle_sort_compact_noalloc(t.data_ptr(), limit + 1, words, 64, t.data_ptr(), t.data_ptr(),
                                             ctypes.byref(nu), None)
        assert rc == -10 and nu.value == 0
        assert "fixed scratch" in pkg.turtle_strerror(rc)
