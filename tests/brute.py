"""String-level brute force for tiny inputs (tests only).

Works on Python strings, never on 2-bit integers: reverse complement by string
reversal and base translation, canonical form by lexicographic min (A<C<G<T, so
this equals the numeric min of the 2-bit encodings with A=0 C=1 G=2 T=3), reads
split at every character that is not A/C/G/T in either case (Sec. 2.1.2).
"""
from __future__ import annotations

import re
from collections import Counter

import numpy as np

_COMP = str.maketrans("ACGT", "TGCA")
_SPLIT = re.compile("[^ACGT]+")


def revcomp(s: str) -> str:
    return s[::-1].translate(_COMP)


def segments(read: str):
    up = "".join(ch.upper() if ch in "acgt" else ch for ch in read)
    return [s for s in _SPLIT.split(up) if s]


def kmer_counts(reads, k: int, min_count: int = 1) -> dict:
    c = Counter()
    for r in reads:
        for seg in segments(r):
            for p in range(len(seg) - k + 1):
                w = seg[p:p + k]
                c[min(w, revcomp(w))] += 1
    return {w: n for w, n in c.items() if n >= min_count}


def n_windows(reads, k: int) -> int:
    return sum(max(0, len(s) - k + 1) for r in reads for s in segments(r))


def windows(reads, k: int):
    """[(offset in the concatenation, canonical string)] in read order."""
    out, base = [], 0
    for r in reads:
        up = "".join(ch.upper() if ch in "acgt" else ch for ch in r)
        for p in range(len(r) - k + 1):
            w = up[p:p + k]
            if all(ch in "ACGT" for ch in w):
                out.append((base + p, min(w, revcomp(w))))
        base += len(r)
    return out


def decode(key, k: int) -> str:
    """2-bit integer key (int, or (hi, lo) pair) -> string, first base most significant."""
    if isinstance(key, (tuple, list, np.ndarray)) and np.ndim(key) == 1 and len(key) == 2:
        v = (int(key[0]) << 64) | int(key[1])
    else:
        v = int(key)
    return "".join("ACGT"[(v >> (2 * (k - 1 - j))) & 3] for j in range(k))


def pack(reads):
    """list[str] -> (bases uint8, offsets uint64) in the library's read layout."""
    data = "".join(reads).encode("latin-1")
    bases = np.frombuffer(data, dtype=np.uint8).copy() if data else np.zeros(0, dtype=np.uint8)
    offs = np.zeros(len(reads) + 1, dtype=np.uint64)
    offs[1:] = np.cumsum([len(r) for r in reads])
    return bases, offs


def as_dict(keys, counts, k: int) -> dict:
    return {decode(keys[i], k): int(counts[i]) for i in range(len(counts))}


def random_reads(rng, n, lo, hi, alphabet="ACGT", weights=None):
    out = []
    for _ in range(n):
        L = int(rng.integers(lo, hi + 1))
        out.append("".join(rng.choice(list(alphabet), size=L, p=weights)))
    return out
