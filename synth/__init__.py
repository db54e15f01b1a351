"""Seeded synthetic read libraries (input generation only).

The generator lives in ``synth.c`` (SplitMix64, counter-style, so every genome
block and read is an independent stream and generation is parallel and
reproducible).  This module holds none of the k-mer counting arithmetic: it makes
ASCII reads that the oracle and the GPU path both consume.

Workload recipes follow the five library shapes used to benchmark the method
(paper Table 2 stands behind the fly-, chicken- and human-scale data sets, which
are not available here; these synthetic libraries stand in for them):

* ``small``      1 Mbp iid genome, 200,000 x 100 bp reads, 1% substitutions.
* ``fly``        100 Mbp iid genome + 5% inserted repeat copies (1-5 kb
                 segments, 2-20 copies, 2% divergence), 30M x 100 bp reads, 1%
                 substitutions, 0.05% N calls.
* ``longk``      1 Gbp iid genome, per-10-kb log-normal coverage (median 20x,
                 sigma 1), 150 bp reads, 0.5% substitutions (k=64 workload).
* ``batched``    64 libraries, genome log-uniform 0.1-20 Mbp, coverage
                 U(10, 60), 100 or 150 bp, 1% substitutions, k in {21, 31, 55}.
* ``served``     Poisson arrivals (50 jobs/s) of 1-50 Mbp libraries (100 bp,
                 1% substitutions), k in {25, 31, 63}, min_count in {2, 3}.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libsynth.so")
_lib = None

u64 = ctypes.c_uint64
_p = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile libsynth.so next to this file (plain C, host only)."""
    src = os.path.join(_HERE, "synth.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-pthread", src, "-o", _SO, "-lm"])
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        lib.synth_genome_iid.argtypes = [u64, u64, _p, ctypes.c_int]
        lib.synth_genome_repeats_cap.argtypes = [u64, ctypes.c_double, ctypes.c_int, ctypes.c_int]
        lib.synth_genome_repeats_cap.restype = u64
        lib.synth_genome_repeats.argtypes = [u64, u64, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_int, ctypes.c_double, _p, u64, ctypes.c_int]
        lib.synth_genome_repeats.restype = u64
        lib.synth_reads_uniform.argtypes = [_p, u64, u64, u64, u64, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                            _p, _p, ctypes.c_int]
        lib.synth_region_plan.argtypes = [u64, u64, u64, ctypes.c_double, ctypes.c_double, ctypes.c_int, _p]
        lib.synth_region_plan.restype = u64
        lib.synth_reads_regions.argtypes = [_p, u64, u64, _p, u64, u64, u64, u64, ctypes.c_int, ctypes.c_double,
                                            ctypes.c_double, _p, _p, ctypes.c_int]
        _lib = lib
    return _lib


def _threads(threads):
    return int(threads or os.cpu_count() or 1)


def genome_iid(seed: int, length: int, threads=None) -> np.ndarray:
    out = np.empty(length, dtype=np.uint8)
    _load().synth_genome_iid(seed, length, out.ctypes.data, _threads(threads))
    return out


def genome_repeats(seed: int, base_len: int, repeat_frac=0.05, seg=(1000, 5000), copies=(2, 20), divergence=0.02,
                   threads=None) -> np.ndarray:
    lib = _load()
    cap = lib.synth_genome_repeats_cap(base_len, repeat_frac, seg[1], copies[1])
    out = np.empty(cap, dtype=np.uint8)
    n = lib.synth_genome_repeats(seed, base_len, repeat_frac, seg[0], seg[1], copies[0], copies[1], divergence,
                                 out.ctypes.data, cap, _threads(threads))
    return out[:n]


def reads_uniform(genome: np.ndarray, seed: int, n_reads: int, R: int, err=0.01, nrate=0.0, first=0, threads=None):
    """Reads `first .. first+n_reads-1` of the uniform-start stream; returns (bases, offsets)."""
    assert genome.dtype == np.uint8 and genome.size >= R
    bases = np.empty(n_reads * R, dtype=np.uint8)
    offsets = np.empty(n_reads + 1, dtype=np.uint64)
    _load().synth_reads_uniform(genome.ctypes.data, genome.size, seed, first, n_reads, R, err, nrate,
                                bases.ctypes.data, offsets.ctypes.data, _threads(threads))
    return bases, offsets


def region_plan(seed: int, G: int, region_len=10_000, median=20.0, sigma=1.0, R=150) -> np.ndarray:
    n_regions = (G + region_len - 1) // region_len
    prefix = np.empty(n_regions + 1, dtype=np.uint64)
    _load().synth_region_plan(seed, G, region_len, median, sigma, R, prefix.ctypes.data)
    return prefix


def reads_regions(genome: np.ndarray, seed: int, prefix: np.ndarray, region_len: int, first: int, n_reads: int, R: int,
                  err=0.005, nrate=0.0, threads=None):
    bases = np.empty(n_reads * R, dtype=np.uint8)
    offsets = np.empty(n_reads + 1, dtype=np.uint64)
    _load().synth_reads_regions(genome.ctypes.data, genome.size, seed, prefix.ctypes.data, prefix.size - 1,
                                region_len, first, n_reads, R, err, nrate, bases.ctypes.data, offsets.ctypes.data,
                                _threads(threads))
    return bases, offsets


# ---------------------------------------------------------------- workloads
@dataclass
class Library:
    """One read library: concatenated ASCII bases + offsets[n_reads+1] (read i = bases[off[i]:off[i+1]])."""
    name: str
    bases: np.ndarray
    offsets: np.ndarray
    k: int
    min_count: int
    meta: dict = field(default_factory=dict)

    @property
    def n_reads(self) -> int:
        return self.offsets.size - 1

    def window_upper_bound(self) -> int:
        lens = np.diff(self.offsets.astype(np.int64))
        return int(np.maximum(lens - self.k + 1, 0).sum())


def small(seed=1, scale=1.0, k=31, min_count=2, threads=None) -> Library:
    """1 Mbp iid genome; 200,000 x 100 bp uniform reads, either strand; 1% errors; no N."""
    G = max(200, int(1_000_000 * scale))
    n = max(1, int(200_000 * scale))
    g = genome_iid(seed, G, threads)
    b, o = reads_uniform(g, seed, n, 100, 0.01, 0.0, threads=threads)
    return Library("small", b, o, k, min_count, dict(G=G, n_reads=n, R=100, err=0.01, seed=seed))


def fly(seed=2, scale=1.0, k=31, min_count=2, threads=None) -> Library:
    """100 Mbp genome + 5% repeat copies; 30M x 100 bp (30x); 1% errors; 0.05% N."""
    base_len = max(10_000, int(100_000_000 * scale))
    g = genome_repeats(seed, base_len, 0.05, (1000, 5000), (2, 20), 0.02, threads)
    n = max(1, int(30_000_000 * scale))
    b, o = reads_uniform(g, seed, n, 100, 0.01, 0.0005, threads=threads)
    return Library("fly", b, o, k, min_count, dict(G=int(g.size), n_reads=n, R=100, err=0.01, nrate=0.0005,
                                                     seed=seed))


@dataclass
class StreamedLibrary:
    """A library too large to hold at once: reads are produced chunk by chunk."""
    name: str
    genome: np.ndarray
    prefix: np.ndarray
    seed: int
    region_len: int
    R: int
    err: float
    k: int
    min_count: int

    @property
    def n_reads(self) -> int:
        return int(self.prefix[-1])

    def chunk(self, first: int, n: int, threads=None):
        n = min(n, self.n_reads - first)
        return reads_regions(self.genome, self.seed, self.prefix, self.region_len, first, n, self.R, self.err,
                             0.0, threads)


def longk(seed=3, scale=1.0, k=64, min_count=2, threads=None) -> StreamedLibrary:
    """1 Gbp iid genome; per-10-kb log-normal coverage (median 20x, sigma 1); 150 bp; 0.5% errors; k=64."""
    G = max(20_000, int(1_000_000_000 * scale))
    g = genome_iid(seed, G, threads)
    prefix = region_plan(seed, G, 10_000, 20.0, 1.0, 150)
    return StreamedLibrary("longk", g, prefix, seed, 10_000, 150, 0.005, k, min_count)


def batched_specs(seed=4, n_libs=64, scale=1.0):
    """64 library specs: genome log-uniform 0.1-20 Mbp, coverage U(10,60), R in {100,150}, k in {21,31,55}."""
    rng = np.random.Generator(np.random.PCG64(seed))
    specs = []
    for i in range(n_libs):
        G = int(math.exp(rng.uniform(math.log(100_000), math.log(20_000_000))) * scale)
        cov = float(rng.uniform(10, 60))
        R = int(rng.choice([100, 150]))
        k = int(rng.choice([21, 31, 55]))
        specs.append(dict(G=max(G, 1000), cov=cov, R=R, k=k, err=0.01, seed=seed * 1000 + i, min_count=2))
    return specs


def library_from_spec(spec, threads=None) -> Library:
    g = genome_iid(spec["seed"], spec["G"], threads)
    n = max(1, int(round(spec["cov"] * spec["G"] / spec["R"])))
    b, o = reads_uniform(g, spec["seed"], n, spec["R"], spec["err"], 0.0, threads=threads)
    return Library("lib%d" % spec["seed"], b, o, spec["k"], spec.get("min_count", 2), dict(spec, n_reads=n))


def served_jobs(seed=5, n_jobs=1000, rate=50.0, scale=1.0):
    """Poisson arrivals (rate jobs/s); read bases log-uniform 1-50 Mbp; 100 bp; 1% errors;
    k in {25, 31, 63}; min_count in {2, 3}; genome = bases / 20 (20x coverage)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    jobs = []
    for i in range(n_jobs):
        t += float(rng.exponential(1.0 / rate))
        bases = int(math.exp(rng.uniform(math.log(1e6), math.log(50e6))) * scale)
        R = 100
        G = max(1000, bases // 20)
        jobs.append(dict(t=t, G=G, cov=bases / G, R=R, k=int(rng.choice([25, 31, 63])),
                         min_count=int(rng.choice([2, 3])), err=0.01, seed=seed * 100000 + i))
    return jobs
