"""CPU oracle for the Turtle frequent k-mer method (arXiv:1305.1861).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg may import this package.  The library
under ``paper_1305_1861_gb300`` never imports or links it, and this package
imports nothing from the library.

``oracle.cpp`` writes out the plain definition of what the method computes
(exact canonical k-mer counts, Sec. 2.1.1-2.1.2 and Alg. 1), the sort-and-compact
step on its own (Sec. 2.1.4) and a sequential pattern-blocked Bloom filter
(Sec. 2.1.3).  This module adds the blocked-Bloom false-positive formula used to
pin the filter and the classic Bloom sizing rule quoted in Sec. 2.2.

Every function is pinned by ``tests/test_oracle_pins.py`` against brute force on
strings, reverse-complement symmetry, the window-count invariant, closed forms
and the paper's worked example; none of the pins re-run this code's formulas.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None

u64 = ctypes.c_uint64
_p = ctypes.c_void_p


class _Result(ctypes.Structure):
    _fields_ = [("n", u64), ("words", ctypes.c_int), ("keys", ctypes.POINTER(u64)),
                ("counts", ctypes.POINTER(u64)), ("n_windows", u64)]


def build(force: bool = False) -> str:
    """Compile liboracle.so (g++, host only)."""
    src = os.path.join(_HERE, "oracle.cpp")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread", src, "-o", _SO])
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        lib.oracle_count.argtypes = [_p, _p, u64, ctypes.c_int, u64, ctypes.c_int, ctypes.POINTER(_Result)]
        lib.oracle_count_map.argtypes = [_p, _p, u64, ctypes.c_int, u64, ctypes.POINTER(_Result)]
        lib.oracle_result_free.argtypes = [ctypes.POINTER(_Result)]
        lib.oracle_windows.argtypes = [_p, _p, u64, ctypes.c_int, _p, _p, u64]
        lib.oracle_windows.restype = u64
        lib.oracle_sort_compact.argtypes = [_p, u64, ctypes.c_int, ctypes.POINTER(_Result)]
        lib.oracle_count_queries.argtypes = [_p, _p, u64, ctypes.c_int, _p, u64, ctypes.c_int, _p]
        lib.oracle_pbbf_new.argtypes = [u64, ctypes.c_int, ctypes.c_int, u64]
        lib.oracle_pbbf_new.restype = _p
        lib.oracle_pbbf_free.argtypes = [_p]
        lib.oracle_pbbf_test_and_set.argtypes = [_p, _p, u64, ctypes.c_int, _p]
        lib.oracle_pbbf_test.argtypes = [_p, _p, u64, ctypes.c_int, _p]
        lib.oracle_cturtle.argtypes = [_p, _p, u64, ctypes.c_int, u64, ctypes.c_int, ctypes.c_int, u64,
                                       ctypes.POINTER(_Result)]
        lib.oracle_cturtle_collision_free.argtypes = [_p, u64, ctypes.c_int, u64, ctypes.c_int, ctypes.c_int, u64, _p]
        lib.oracle_cturtle_collision_free.restype = None
        lib.oracle_pbbf_words.argtypes = [_p]
        lib.oracle_pbbf_words.restype = ctypes.POINTER(u64)
        lib.oracle_pbbf_patterns.argtypes = [_p]
        lib.oracle_pbbf_patterns.restype = ctypes.POINTER(u64)
        _lib = lib
    return _lib


def _threads(t):
    return int(t or os.cpu_count() or 1)


def _prep(bases, offsets):
    bases = np.ascontiguousarray(bases, dtype=np.uint8)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    return bases, offsets


def _take(res: _Result):
    n, w = res.n, res.words
    keys = np.ctypeslib.as_array(res.keys, shape=(max(n * w, 1),))[: n * w].copy()
    counts = np.ctypeslib.as_array(res.counts, shape=(max(n, 1),))[:n].copy()
    if w == 2:
        keys = keys.reshape(n, 2)
    nw = res.n_windows
    _load().oracle_result_free(ctypes.byref(res))
    return keys, counts, nw


def count(bases, offsets, k: int, min_count: int = 1, threads=None):
    """Exact (key, count) pairs with count >= min_count, ascending by key.

    Returns (keys, counts, n_windows); keys is uint64[n] for k <= 32 and
    uint64[n, 2] (hi, lo) for k > 32.
    """
    bases, offsets = _prep(bases, offsets)
    res = _Result()
    rc = _load().oracle_count(bases.ctypes.data, offsets.ctypes.data, offsets.size - 1, k, min_count,
                              _threads(threads), ctypes.byref(res))
    if rc:
        raise ValueError("oracle_count failed (%d)" % rc)
    return _take(res)


def count_map(bases, offsets, k: int, min_count: int = 1):
    """Same definition, counted in a std::map (small inputs)."""
    bases, offsets = _prep(bases, offsets)
    res = _Result()
    rc = _load().oracle_count_map(bases.ctypes.data, offsets.ctypes.data, offsets.size - 1, k, min_count,
                                  ctypes.byref(res))
    if rc:
        raise ValueError("oracle_count_map failed (%d)" % rc)
    return _take(res)


def windows(bases, offsets, k: int, cap=None):
    """Every valid window in read order: (start offsets, canonical keys)."""
    bases, offsets = _prep(bases, offsets)
    if cap is None:
        lens = np.diff(offsets.astype(np.int64))
        cap = int(np.maximum(lens - k + 1, 0).sum())
    w = 1 if k <= 32 else 2
    pos = np.empty(max(cap, 1), dtype=np.uint64)
    keys = np.empty(max(cap, 1) * w, dtype=np.uint64)
    n = _load().oracle_windows(bases.ctypes.data, offsets.ctypes.data, offsets.size - 1, k, pos.ctypes.data,
                               keys.ctypes.data, cap)
    keys = keys[: n * w]
    return pos[:n], (keys.reshape(n, 2) if w == 2 else keys)


def sort_compact(keys):
    """Sec. 2.1.4 sort-and-compact: (unique keys ascending, run lengths)."""
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    w = 2 if keys.ndim == 2 else 1
    res = _Result()
    _load().oracle_sort_compact(keys.ctypes.data, keys.shape[0], w, ctypes.byref(res))
    k, c, _ = _take(res)
    return k, c


def count_queries(bases, offsets, k: int, queries, threads=None):
    """Exact count of each query key (any order) by enumerating every window."""
    bases, offsets = _prep(bases, offsets)
    q = np.ascontiguousarray(queries, dtype=np.uint64)
    w = 2 if q.ndim == 2 else 1
    order = np.lexsort((q[:, 1], q[:, 0])) if w == 2 else np.argsort(q, kind="stable")
    qs = np.ascontiguousarray(q[order])
    if w == 2:
        uniq, inv = np.unique(qs, axis=0, return_inverse=True)
    else:
        uniq, inv = np.unique(qs, return_inverse=True)
    uniq = np.ascontiguousarray(uniq, dtype=np.uint64)
    cnt = np.zeros(uniq.shape[0], dtype=np.uint64)
    rc = _load().oracle_count_queries(bases.ctypes.data, offsets.ctypes.data, offsets.size - 1, k, uniq.ctypes.data,
                                      uniq.shape[0], _threads(threads), cnt.ctypes.data)
    if rc:
        raise ValueError("oracle_count_queries failed (%d)" % rc)
    out = np.empty(q.shape[0], dtype=np.uint64)
    out[order] = cnt[inv.reshape(-1)]
    return out


class PBBF:
    """Sequential pattern-blocked Bloom filter (Sec. 2.1.3); geometry as in oracle.cpp."""

    def __init__(self, n_sectors: int, pattern_bits: int, n_patterns: int = 1024, seed: int = 0x7475727469):
        self.n_sectors, self.pattern_bits, self.n_patterns, self.seed = n_sectors, pattern_bits, n_patterns, seed
        self._h = _load().oracle_pbbf_new(n_sectors, pattern_bits, n_patterns, seed)
        if not self._h:
            raise ValueError("bad filter geometry")

    def __del__(self):
        if getattr(self, "_h", None):
            _load().oracle_pbbf_free(self._h)
            self._h = None

    def test_and_set(self, keys) -> np.ndarray:
        keys = np.ascontiguousarray(keys, dtype=np.uint64)
        w = 2 if keys.ndim == 2 else 1
        seen = np.empty(keys.shape[0], dtype=np.uint8)
        _load().oracle_pbbf_test_and_set(self._h, keys.ctypes.data, keys.shape[0], w, seen.ctypes.data)
        return seen

    def test(self, keys) -> np.ndarray:
        """Membership test without setting anything."""
        keys = np.ascontiguousarray(keys, dtype=np.uint64)
        w = 2 if keys.ndim == 2 else 1
        seen = np.empty(keys.shape[0], dtype=np.uint8)
        _load().oracle_pbbf_test(self._h, keys.ctypes.data, keys.shape[0], w, seen.ctypes.data)
        return seen

    @property
    def words(self) -> np.ndarray:
        return np.ctypeslib.as_array(_load().oracle_pbbf_words(self._h), shape=(self.n_sectors * 4,)).copy()

    @property
    def patterns(self) -> np.ndarray:
        return np.ctypeslib.as_array(_load().oracle_pbbf_patterns(self._h), shape=(self.n_patterns,)).copy()


def pbbf_fp_formula(lam: float, h: int, n_patterns: int, word_bits: int = 64, imax: int = 200) -> float:
    """Expected false-positive rate of a fresh key in a pattern-blocked filter.

    Putze et al.'s blocked-Bloom argument, specialised to a one-word pattern: the
    number i of inserted keys sharing the probed word is Poisson(lam); the probe's
    pattern is covered either because one of the i keys drew the same table entry
    (prob. 1 - (1 - 1/T)^i) or, failing that, because the union of i uniform
    h-subsets of the word's bits contains it, which inclusion-exclusion gives as
    sum_a (-1)^a C(h, a) [C(B-a, h) / C(B, h)]^i.
    """
    B = word_bits
    total = 0.0
    pois = math.exp(-lam)
    for i in range(imax):
        if i > 0:
            pois *= lam / i
        cover = sum((-1) ** a * math.comb(h, a) * (math.comb(B - a, h) / math.comb(B, h)) ** i for a in range(h + 1))
        same = 1.0 - (1.0 - 1.0 / n_patterns) ** i
        total += pois * (same + (1.0 - same) * cover)
    return total


def standard_bloom_bits_per_item(p: float) -> float:
    """Classic sizing of an unblocked Bloom filter with optimal hash count: m/n = -ln p / (ln 2)^2."""
    return -math.log(p) / (math.log(2) ** 2)

def cturtle(bases, offsets, k: int, n_sectors: int, pattern_bits: int = 4, n_patterns: int = 1024,
            seed: int = 0x7475727469):
    """cTurtle (Sec. 2.2): keys reported by the sequential two-stage counting filter, in report
    order (uint64[n] or uint64[n, 2]), and the number of valid windows."""
    bases, offsets = _prep(bases, offsets)
    res = _Result()
    rc = _load().oracle_cturtle(bases.ctypes.data, offsets.ctypes.data, offsets.size - 1, k, n_sectors,
                                pattern_bits, n_patterns, seed, ctypes.byref(res))
    if rc:
        raise ValueError("oracle_cturtle failed (%d)" % rc)
    keys, _, nw = _take(res)
    return keys, nw


def cturtle_collision_free(keys, n_sectors: int, pattern_bits: int = 4, n_patterns: int = 1024,
                           seed: int = 0x7475727469):
    """For distinct keys (uint64[n] or uint64[n, 2]): True where the key's cTurtle outcome cannot
    depend on the order of the windows (see oracle_cturtle_collision_free)."""
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    words = 2 if keys.ndim == 2 else 1
    n = keys.shape[0]
    out = np.zeros(max(n, 1), np.uint8)
    _load().oracle_cturtle_collision_free(keys.ctypes.data, n, words, n_sectors, pattern_bits, n_patterns, seed,
                                          out.ctypes.data)
    return out[:n].astype(bool)
