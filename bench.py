"""Benchmark: canonical k-mers/s of the Turtle hot path on one GB300 (or N independent replicas).

A step is one whole pass of the path (pack, extract, Bloom filter, radix sort and
compaction, exact recount, threshold) over one synthetic library already resident
in HBM. Default workload: the fly-shaped library (100 Mbp genome + 5% repeat
copies, 30M x 100 bp reads, 1% substitutions, 0.05% N), k=31, min_count=2.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload fly|small|longk|batched|served] [--scale S] [--blocks k64,batched,served]

Prints one JSON line (rank 0). Without --workload the line is the fly-shaped headline and,
on one GPU, nested blocks for the other measured workloads: "k64" (long-k at full size, k = 64,
with its own roofline, streamed end to end and oracle baseline), "batched" (64 libraries in one
batched call vs 64 plain calls) and "served" (Poisson arrivals and a saturated queue, continuous
batching vs one job at a time). Under torchrun each rank counts its own replica library (different
seed, same shape): weak scaling, no data-path collective; the blocks run at N = 1 only.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "canonical k-mers/s"
HEADLINE = "canonical k-mers/s and HBM roofline fraction at k=31/k=64; batched/served vs plain"
# DRAM bytes (read + write) per unit of each kernel, from ncu captures of the current kernels on the
# fly-shaped library at 1/10 scale (profiles/); scaled to a full launch by the units it processes.
# A kernel is left out (traffic null) until it has been captured again after a change.
NCU_BYTES_PER_UNIT = {"k_pass1": 98.96, "k_onesweep": 16.0, "k_bucket_count": 8.66, "k_hash_insert": 221.8}
# long-k (k = 64, 128-bit keys, four key ranges), from a capture at 1/50 scale whose ranges have the full-size
# 1 GiB filter (profiles/k_pass1_range_longk_scale0.02.md): k_pass1_range per library window per launch (every
# launch tests every window for its range; the mean of the first launch, which also writes the range ids, 17.87,
# and the other three, 17.23-17.26), k_bucket_count per key of its range (the range's keys taken as W/4)
NCU_BYTES_PER_UNIT_U128 = {"k_pass1_range": 17.40, "k_bucket_count": 17.09}
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=None, choices=["fly", "small", "longk", "served", "batched"],
                    help="one workload alone (default: the fly-shaped headline plus the --blocks)")
    ap.add_argument("--method", default="scturtle", choices=["scturtle", "cturtle"],
                    help="cturtle: the approximate two-stage counting filter (k-mers seen twice, no counts)")
    ap.add_argument("--cturtle-bits", type=int, default=0, help="cturtle filter bits per window (0 = default 8)")
    ap.add_argument("--jobs", type=int, default=1000, help="served: number of jobs (Poisson arrivals, 50/s)")
    ap.add_argument("--max-batch", type=int, default=4, help="served: most queued jobs batched into one run")
    ap.add_argument("--saturate-jobs", type=int, default=300,
                    help="served: also submit this many jobs at once (no arrival gaps) to compare capacity")
    ap.add_argument("--scale", type=float, default=1.0)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--blocks", default="tuned,batched,served,k64",
                    help="default run: also measure these workloads as nested blocks of the same line "
                         "(k64, batched, served; 'none' for the headline alone)")
    ap.add_argument("--block-steps", type=int, default=3, help="timed steps of the k64 and batched blocks")
    ap.add_argument("--cpu-sample-reads", type=int, default=0, help="reads in the oracle sample (0 = auto)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--filter-bits", type=float, default=0.0, help="Bloom bits per window (0 = library default)")
    ap.add_argument("--l2-fetch", type=int, default=-1, help="L2 fetch granularity hint in bytes (-1 = default)")
    ap.add_argument("--recount-windows", action="store_true", help="recount by re-extracting every window")
    ap.add_argument("--member-filter", action="store_true", help="screen first sightings with a membership bitmap")
    ap.add_argument("--sort-tile", type=int, default=-1, help="onesweep tile shape 0..4 (4: persistent, bulk-copied tiles; -1 = default)")
    ap.add_argument("--bucket-slots", type=int, default=0, help="bucket CTA table slots: 4096 or 8192 (0 = default)")
    ap.add_argument("--bucket-windows", type=int, default=0, help="windows per bucket, about (0 = default 16384)")
    ap.add_argument("--compact", type=int, default=-1,
                    help="0 = bucketed, 1 = global sort-and-compact, 2 = hash-table counting, "
                         "3 = lazy sort-and-compact phases (memory-capped, chunked)")
    ap.add_argument("--budget-mib", type=int, default=0, help="device-memory budget per key range (0 = automatic)")
    ap.add_argument("--pattern-bits", type=int, default=0, help="Bloom pattern bits (0 = library default)")
    ap.add_argument("--host-transfer", type=int, default=-1,
                    help="host copies: 0 = measured choice, 1 = page-lock the arrays, 2 = pageable (-1 = default)")
    ap.add_argument("--probe-order", type=int, default=-1,
                    help="pass 1 probes: 0 = in window order, 1 = by filter block (binned) (-1 = default)")
    ap.add_argument("--micro", action="store_true",
                    help="measure the random 32-byte-sector read / atomic ceiling with torch gathers instead")
    return ap.parse_args()


def workload(name: str, scale: float, rank: int):
    seed_shift = 1000 * rank
    if name == "fly":
        lib = synth.fly(seed=2 + seed_shift, scale=scale)
        desc = "fly-shaped: %.0f Mbp genome incl. 5%% repeat copies (1-5 kb, 2-20 copies, 2%% divergence), " \
               "%d x 100 bp reads, 1%% substitutions, 0.05%% N; k=31, min_count=2" % (lib.meta["G"] / 1e6,
                                                                                     lib.n_reads)
    elif name == "small":
        lib = synth.small(seed=1 + seed_shift, scale=scale)
        desc = "small: 1 Mbp iid genome, %d x 100 bp reads, 1%% substitutions; k=31, min_count=2" % lib.n_reads
    else:
        s = synth.longk(seed=3 + seed_shift, scale=scale)
        n = s.n_reads
        b, o = s.chunk(0, n)
        lib = synth.Library("longk", b, o, 64, 2, dict(G=s.genome.size, n_reads=n, R=150))
        desc = "long-k: %.0f Mbp iid genome, log-normal coverage (median 20x, sigma 1), %d x 150 bp, " \
               "0.5%% substitutions; k=64, min_count=2" % (s.genome.size / 1e6, n)
    return lib, desc


def reduce_over_ranks(values, ops, device):
    """Combine per-rank scalars over the process group: values[i] by ops[i] ("max" or "sum"). Without an
    initialised group of more than one rank the values come back unchanged."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    mx, sm = t.clone(), t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return [float(mx[i]) if op == "max" else float(sm[i]) for i, op in enumerate(ops)]


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms during the timed region."""

    FIELDS = "clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown," \
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown," \
             "clocks_event_reasons.sw_power_cap"

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(lib, sample_reads: int):
    """The oracle as it stands, on the host cores, over the first `sample_reads` reads of the workload."""
    import oracle

    n = min(sample_reads, lib.n_reads)
    end = int(lib.offsets[n])
    b, o = lib.bases[:end], lib.offsets[: n + 1]
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    _, _, nw = oracle.count(b, o, lib.k, lib.min_count, threads=cores)
    dt = time.perf_counter() - t0
    return {"value": nw / dt, "unit": METRIC, "cores": cores, "kind": "oracle",
            "sample": "first %d reads (%d windows) of the same library, %.1f s" % (n, nw, dt)}


# The kernel behind each timed stage (bucketed form / global form of sort-and-compact).
STAGE_KERNEL = {"filter": "k_pass1", "sort": "k_onesweep", "rle": "k_bucket_count", "recount": "k_add_firsts"}
STAGE_KERNEL_GLOBAL = {"filter": "k_pass1", "sort": "k_onesweep", "rle": "k_rle", "recount": "k_add_firsts"}
STAGE_KERNEL_HASH = {"filter": "k_pass1", "table": "k_hash_insert", "recount": "k_hash_firsts",
                     "threshold": "k_hash_extract", "sort": "k_onesweep"}
STAGE_KERNEL_LAZY = {"filter": "k_pass1", "sort": "k_onesweep", "rle": "k_bucket_count", "merge": "k_merge_counts",
                     "recount": "k_pass2", "threshold": "k_threshold"}


def stage_bytes_lazy(stage: str, st: dict, lib):
    """Byte model of the lazy form (compact = 3), as stage_bytes: (bytes, launches, units).

      filter    k_pass1 over each chunk: packed reads, one filter sector per window, a first sighting's
                sector written back, a candidate key written; unit = window
      sort      bucket-index radix passes over each chunk's candidates; unit = key-pass
      rle       k_bucket_count: each chunk's candidates read, its distinct keys and counts written; the
                distinct keys of all chunks are taken as (chunks x the final distinct count), an upper
                bound; unit = candidate
      merge     k_merge_counts: the running array and a chunk's distinct keys read, the merged array
                written, each (key + count), taken as 3 x the final distinct count per merge; unit = key
      recount   k_pass2: packed reads, one 32-byte table sector per window; unit = window
      threshold k_threshold: the distinct keys read, one table sector each, kept keys written; unit = key
    """
    W = st["n_windows"]
    kw = 8 if lib.k <= 32 else 16
    R = float(np.diff(lib.offsets[:2].astype(np.int64))[0]) if lib.n_reads else 100.0
    packed = (R / 4.0 + R / 8.0) / max(R - lib.k + 1, 1)
    nc, nu, no = st["n_candidates"], st["n_unique"], st["n_out"]
    ch = max(st.get("chunks", 1), 1)
    passes = max(st["sort_passes"], 1)
    if stage == "filter":
        return W * packed + W * 32.0 + 32.0 * (W - nc) + kw * nc, ch, W
    if stage == "sort":
        return passes * 2.0 * kw * nc, passes * ch, passes * nc
    if stage == "rle":
        return kw * nc + (kw + 4.0) * min(nc, ch * nu), ch, nc
    if stage == "merge":
        m = max(ch - 1, 1)
        return m * 3.0 * (kw + 4.0) * nu, m, m * 3 * nu
    if stage == "recount":
        return W * packed + W * 32.0, 1, W
    if stage == "threshold":
        return nu * (kw + 32.0) + no * (kw + 4.0), 1, nu
    return 0.0, 1, 0


def stage_bytes_hash(stage: str, st: dict, lib):
    """Byte model of the hash-table form (compact = 2), as stage_bytes: (bytes, launches, units).

      table     sketch (candidates read), clear (table written), k_hash_insert: candidates read, one
                slot sector read and written back each; unit = candidate
      recount   k_hash_firsts: first sightings read, one slot sector each; unit = first sighting
      threshold k_hash_extract: table read, kept keys written; unit = kept key
      sort      onesweep passes over the kept keys, then one slot sector and a count per kept key;
                unit = key-pass
    """
    W = st["n_windows"]
    kw = 8 if lib.k <= 32 else 16
    parts = max(st["super_partitions"], 1)
    nc, nf, no = st["n_candidates"], st["n_firsts"], st["n_out"]
    tb = st["table_bytes"]
    passes = max(st["sort_passes"], 1)
    if stage == "table":
        return 2.0 * kw * nc + tb + 64.0 * nc, parts, nc
    if stage == "recount":
        return nf * (kw + 32.0), parts, nf
    if stage == "threshold":
        return tb + kw * no, parts, no
    if stage == "sort":
        return passes * 2.0 * kw * no + no * (kw + 36.0), passes * parts, passes * no
    return stage_bytes(stage, st, lib, False)


def stage_bytes(stage: str, st: dict, lib, bucketed: bool):
    """(algorithmic HBM bytes of the stage's main kernel over one step, its launches per step, its units
    per step: windows for filter and rle, key-passes for sort, first sightings for recount).

    Byte model (one unit = one valid window; kw = key bytes; parts = key-range super-partitions):
      filter  k_pass1: every part re-reads the packed reads (2-bit codes + validity bits), each window
              probes one 32-byte filter sector in its own part, a first sighting writes its sector
              back, every probed window leaves as one key (candidate or first sighting)
      sort    k_onesweep: every key read and written once per digit pass (bucketed: candidates and
              first sightings, two sorts per part; global: candidates)
      rle     k_bucket_count: candidates and first sightings read once, kept keys and counts written
              (global form k_rle: candidates read, distinct keys and run starts written)
      recount k_add_firsts (global form): first sightings streamed, one table sector each
    """
    W = st["n_windows"]
    kw = 8 if lib.k <= 32 else 16
    parts = max(st["super_partitions"], 1)
    R = float(np.diff(lib.offsets[:2].astype(np.int64))[0]) if lib.n_reads else 100.0
    packed = (R / 4.0 + R / 8.0) / max(R - lib.k + 1, 1)
    nc, nf, nu, no = st["n_candidates"], st["n_firsts"], st["n_unique"], st["n_out"]
    passes = max(st["sort_passes"], 1)
    if stage == "filter":
        return parts * W * packed + W * 32.0 + 32.0 * (nf if nf else W - nc) + kw * (nc + nf), parts, W
    if stage == "sort":
        if bucketed:
            return passes * 2.0 * kw * (nc + nf), passes * parts * ((nc > 1) + (nf > 1)), passes * (nc + nf)
        return passes * 2.0 * kw * nc, passes * parts, passes * nc
    if stage == "rle":
        if bucketed:
            return kw * (nc + nf) + (kw + 4.0) * no, parts, nc + nf
        return kw * nc + (kw + 8.0) * nu, parts, nc
    if stage == "recount":
        return nf * (kw + 32.0) + 32.0 * nu, parts, nf
    return 0.0, 1, 0


def make_params(pkg, args, **kw):
    prm = pkg.Params.default(timing=1, **kw)
    if args.filter_bits > 0:
        prm.filter_bits_per_window = args.filter_bits
    if args.l2_fetch >= 0:
        prm.l2_fetch_bytes = args.l2_fetch
    if args.recount_windows:
        prm.recount_windows = 1
    if args.member_filter:
        prm.member_filter = 1
    if args.sort_tile >= 0:
        prm.sort_tile = args.sort_tile
    if args.bucket_slots:
        prm.bucket_slots = args.bucket_slots
    if args.compact >= 0:
        prm.compact = args.compact
    if args.budget_mib:
        prm.budget_mib = args.budget_mib
    if args.pattern_bits:
        prm.pattern_bits = args.pattern_bits
    if args.probe_order >= 0:
        prm.probe_order = args.probe_order
    if args.host_transfer >= 0:
        prm.host_transfer = args.host_transfer
    if args.bucket_windows:
        prm.bucket_windows = args.bucket_windows
    return prm


def time_device(pkg, ctx, lib, prm, steps, warmup, world=1, dev=0):
    """Device-resident steps: W untimed, then K timed between CUDA events on the launching stream, with
    clocks sampled meanwhile. Returns (ms per step (max over ranks), windows (sum over ranks), last stats,
    per-stage average ms, launches in the timed region, clocks)."""
    import torch

    bases = torch.from_numpy(lib.bases).cuda()
    offs = torch.from_numpy(lib.offsets.astype(np.int64)).cuda()
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        ctx.turtle_count_device(bases, offs, lib.k, lib.min_count, prm, stream)
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    sampler = ClockSampler(dev)
    stage_ms = {s: [] for s in pkg.STAGES}
    launches = 0
    barrier()
    torch.cuda.synchronize()
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        ctx.turtle_count_device(bases, offs, lib.k, lib.min_count, prm, stream)
        st = ctx.stats()
        launches += st["launches"]
        for s in pkg.STAGES:
            stage_ms[s].append(st["stage_ms"][s])
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / steps
    W = st["n_windows"]
    ms_all, W_all = reduce_over_ranks([ms, W], ["max", "sum"], "cuda")  # slowest rank, all ranks' windows
    del bases, offs
    torch.cuda.empty_cache()
    return ms_all, W_all, st, {s: float(np.mean(v)) for s, v in stage_ms.items()}, launches, clocks


def time_e2e(pkg, lib, prm, steps, W_all, world=1, dev=0):
    """End to end through the C ABI (turtle_ctx_count) on the caller's pageable NumPy arrays, as a user
    calls it: the reads' copy to the device and the result's copy back are inside the timed region.
    Each result is released before the next call (a streaming consumer). Reports the host-side phases."""
    import torch

    prm_e2e = pkg.Params.from_buffer_copy(prm)  # the same form and knobs, without stage events
    prm_e2e.timing = 0
    ctx = pkg.Context(dev)
    keys, counts, nw = ctx.turtle_count(lib.bases, lib.offsets, lib.k, lib.min_count, prm_e2e)  # warm the context
    keys_n = len(counts)
    del keys, counts
    phases = {p: [] for p in pkg.HOST_PHASES}
    h2d, locked = [], 0
    t0 = time.perf_counter()
    for _ in range(steps):
        keys, counts, nw = ctx.turtle_count(lib.bases, lib.offsets, lib.k, lib.min_count, prm_e2e)
        keys_n = len(counts)
        del keys, counts
        st = ctx.stats()
        for p in pkg.HOST_PHASES:
            phases[p].append(st["host_ms"][p])
        h2d.append(st["h2d_ms"])
        locked += st["host_locked"]
    e2e_s = (time.perf_counter() - t0) / steps
    ctx.close()
    torch.cuda.empty_cache()
    e2e_s = reduce_over_ranks([e2e_s], ["max"], "cuda")[0]
    kw = 8 if lib.k <= 32 else 16
    return {"value": W_all / e2e_s, "unit": METRIC, "h2d_bytes_per_step": int(lib.bases.nbytes + lib.offsets.nbytes),
            "d2h_bytes_per_step": int(keys_n * (kw + 4)), "ms_per_step": e2e_s * 1e3, "steps": steps,
            "host": "pageable NumPy arrays (the caller's own memory), turtle_ctx_count",
            "stages_ms": {p: round(float(np.mean(v)), 3) for p, v in phases.items()},
            "h2d_copy_span_ms": round(float(np.mean(h2d)), 3),
            "transfer_gbs_measured": st["transfer_gbs"], "calls_page_locked": locked,
            "stages_note": "input: device buffers + offsets copy + queueing the reads' copy; path: device path until "
                           "the result is in HBM (an overlapped or streamed copy of the reads runs inside it); "
                           "touch: first touch of fresh host result pages; output: result copy to host"}


def roofline_of(lib, prm, st, avg, args):
    bucketed = prm.compact == 0 and not prm.recount_windows
    hashed = prm.compact == 2
    lazy = prm.compact == 3
    kernels = (STAGE_KERNEL_LAZY if lazy else STAGE_KERNEL_HASH if hashed else
               (STAGE_KERNEL if bucketed else STAGE_KERNEL_GLOBAL))
    dom = max(kernels, key=lambda s: avg[s])
    hbm, src = peaks()
    total_bytes, n_launch, units = (stage_bytes_lazy(dom, st, lib) if lazy else stage_bytes_hash(dom, st, lib)
                                    if hashed else stage_bytes(dom, st, lib, bucketed))
    ach = total_bytes / (avg[dom] / 1e3) / 1e9  # = bytes per launch / average launch time
    kern = kernels[dom]
    if kern == "k_pass1" and st["super_partitions"] > 1 and not lazy:
        kern = "k_pass1_range"  # one key range per launch: the compacting form of pass 1
    table = NCU_BYTES_PER_UNIT if lib.k <= 32 else NCU_BYTES_PER_UNIT_U128
    # per-unit DRAM bytes were captured on the fly-shaped (k = 31) and long-k (k = 64) libraries at
    # default parameters only
    per_unit = (table.get(kern) if lib.name in ("fly", "longk") and (bucketed or hashed) and not lazy
                and args.filter_bits <= 0 and args.scale == 1.0 and not args.budget_mib else None)
    if per_unit and kern == "k_pass1_range":
        traffic = per_unit * st["n_windows"]  # every range's launch tests every window
    else:
        traffic = per_unit * units / n_launch if per_unit else None
    return {"bound": "hbm", "kernel": kern, "achieved": round(ach, 1), "peak": hbm, "peak_source": src,
            "unit": "GB/s", "frac": round(ach / hbm, 4), "traffic": traffic,
            "bytes_per_launch": total_bytes / n_launch, "launches_per_step": n_launch,
            "traffic_note": ("ncu dram bytes per unit of this kernel (profiles/) x units per launch"
                             if traffic else None),
            "stage_ms": {s: round(v, 3) for s, v in avg.items()}}


def config_of(lib, desc, st, prm, world):
    bucketed = prm.compact == 0 and not prm.recount_windows
    hashed = prm.compact == 2
    return {"workload": desc, "k": lib.k, "min_count": lib.min_count, "windows": st["n_windows"],
            "n_reads": lib.n_reads, "bases": int(lib.bases.size), "candidates": st["n_candidates"],
            "unique_candidates": st["n_unique"], "reported": st["n_out"],
            "form": ("lazy sort-and-compact phases (%d chunks)" % st.get("chunks", 0) if prm.compact == 3 else
                     "hash table" if hashed else ("bucketed" if bucketed else "global sort")),
            "scratch_bytes": st["scratch_bytes"], "table_bytes": st["table_bytes"],
            "l2": "inputs larger than L2 (%.1f GB of reads resident)" % (lib.bases.nbytes / 1e9),
            "parallelism": "replicas%d" % world if world > 1 else "single"}


def run_ours(args, rank, world):
    import torch

    import paper_1305_1861_gb300 as pkg

    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    pkg.load()
    lib, desc = workload(args.workload, args.scale, rank)
    ctx = pkg.Context(dev)
    prm = make_params(pkg, args)
    ms_all, W_all, st, avg, launches, clocks = time_device(pkg, ctx, lib, prm, args.steps, args.warmup, world, dev)
    ctx.close()  # give the device-resident context's memory back before the host-form calls
    torch.cuda.empty_cache()
    value = W_all / (ms_all / 1e3)
    e2e = time_e2e(pkg, lib, prm, args.e2e_steps, W_all, world, dev)
    out = {"metric": HEADLINE, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_all, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "u64" if lib.k <= 32 else "u128", "data": "synthetic",
           "config": config_of(lib, desc, st, prm, world),
           "e2e": e2e, "roofline": roofline_of(lib, prm, st, avg, args), "clocks": clocks, "gpu_launches": launches,
           "sort_passes": st["sort_passes"], "super_partitions": st["super_partitions"],
           # digit passes over each key per bit of the key (eight 8-bit passes would be 8 / (2k))
           "sort_passes_per_key_bit": round(st["sort_passes"] / (2.0 * lib.k), 4)}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        frac = 0.01 if lib.k > 32 else 0.1  # about 10-30 s of oracle work
        sample = args.cpu_sample_reads or max(1, int(lib.n_reads * frac))
        out["cpu_baseline"] = cpu_baseline(lib, sample)
    return out


KNOBS = ("filter_bits_per_window", "pattern_bits", "sort_tile", "bucket_slots", "bucket_windows")


def run_tuned_block(args):
    """Autotuner A/B on the fly-shaped library, device-resident: turtle_autotune chooses the knobs, then the
    default and the tuned params alternate step by step (CUDA events on the launching stream)."""
    import torch

    import paper_1305_1861_gb300 as pkg

    lib, desc = workload("fly", 1.0, 0)
    pkg.load().turtle_tune_cache_clear()
    ctx = pkg.Context(0)
    b = torch.from_numpy(lib.bases).cuda()
    o = torch.from_numpy(lib.offsets.astype(np.int64)).cuda()
    base = make_params(pkg, args)
    base.timing = 0
    t0 = time.perf_counter()
    best, rep = ctx.autotune(b, o, lib.k, lib.min_count, base)
    tune_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    times = {"default": [], "tuned": []}
    for p in (base, best):
        ctx.turtle_count_device(b, o, lib.k, lib.min_count, p, stream)
    for step in range(2 * max(1, min(args.steps, 10))):
        name, p = (("default", base), ("tuned", best))[step % 2]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.turtle_count_device(b, o, lib.k, lib.min_count, p, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        times[name].append(e0.elapsed_time(e1))
    W = ctx.stats()["n_windows"]
    ctx.close()
    del b, o
    torch.cuda.empty_cache()
    d, t = float(np.median(times["default"])), float(np.median(times["tuned"]))
    return {"metric": "autotuned vs default knobs, fly-shaped k=31, device-resident", "unit": METRIC,
            "default_ms": d, "tuned_ms": t, "speedup_vs_default": d / t, "value": W / (t / 1e3),
            "knobs_default": {k: getattr(base, k) for k in KNOBS}, "knobs_tuned": {k: getattr(best, k) for k in KNOBS},
            "evaluations": rep.evaluations, "tune_wall_s": round(tune_s, 2),
            "tuner_ms": {"start": rep.default_ms, "best": rep.best_ms}, "steps_each": len(times["tuned"])}


def run_k64_block(args):
    """The long-k workload (k = 64, 128-bit keys) at full size, device-resident, with its own roofline, its
    end to end streamed through two device staging buffers in 1 GiB chunks, and its oracle baseline."""
    import torch

    import paper_1305_1861_gb300 as pkg

    lib, desc = workload("longk", 1.0, 0)
    ctx = pkg.Context(0)
    prm = make_params(pkg, args)
    steps, warmup = max(1, min(args.steps, args.block_steps)), max(3, min(args.warmup, 3))
    ms, W, st, avg, launches, clocks = time_device(pkg, ctx, lib, prm, steps, warmup)
    ctx.close()
    torch.cuda.empty_cache()
    e2e = time_e2e(pkg, lib, pkg.Params.default(stream_chunk_mib=1024, timing=1), 2, W)
    e2e["host"] += ", reads streamed in 1 GiB chunks through two device staging buffers (stream_chunk_mib = 1024)"
    out = {"metric": "canonical k-mers/s at k=64", "value": W / (ms / 1e3), "unit": METRIC, "steps": steps,
           "warmup": warmup, "ms_per_step": ms, "dtype": "u128", "config": config_of(lib, desc, st, prm, 1),
           "e2e": e2e, "roofline": roofline_of(lib, prm, st, avg, args), "clocks": clocks,
           "gpu_launches": launches, "super_partitions": st["super_partitions"], "sort_passes": st["sort_passes"],
           "sort_passes_per_key_bit": round(st["sort_passes"] / (2.0 * lib.k), 4)}
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(lib, max(1, int(lib.n_reads * 0.01)))
    del lib
    return out


def run_reference(args, rank, world):
    """The oracle (plain CPU exact counter) on host cores, bounded sample per step."""
    lib, desc = workload(args.workload, min(args.scale, 1.0), 0)
    sample = args.cpu_sample_reads or max(1, int(lib.n_reads * 0.05))
    for _ in range(args.warmup):
        cpu_baseline(lib, max(1, sample // 10))
    vals = []
    t_all = 0.0
    last = None
    for _ in range(args.steps):
        r = cpu_baseline(lib, sample)
        vals.append(r["value"])
        last = r
    v = float(np.median(vals))
    return {"impl": "reference", "metric": HEADLINE, "value": v, "unit": METRIC, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u64" if lib.k <= 32 else "u128", "data": "synthetic",
            "config": {"workload": desc, "k": lib.k, "min_count": lib.min_count},
            "cpu_baseline": {"value": v, "unit": METRIC, "cores": last["cores"], "kind": "oracle",
                             "sample": last["sample"]},
            "e2e": {"value": v, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def _set_l2_fetch(nbytes: int):
    """cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, nbytes) through the CUDA runtime torch loaded."""
    import ctypes
    import glob

    import torch

    cands = glob.glob(os.path.join(os.path.dirname(torch.__file__), "..", "nvidia", "cu*", "lib", "libcudart.so*"))
    cands += ["libcudart.so.13", "libcudart.so"]
    for c in cands:
        try:
            rt = ctypes.CDLL(c)
            return rt.cudaDeviceSetLimit(ctypes.c_int(0x05), ctypes.c_size_t(nbytes))
        except OSError:
            continue
    return -1


def micro():
    """Practical ceiling for the hash-probe kernels: random 8-byte reads (one 32-byte sector each) and
    random 4-byte atomic adds over a table far larger than L2, with torch's gather / index_add kernels,
    under several L2 fetch-granularity hints (0 = the context default)."""
    import torch

    n_words = 1 << 29  # 4 GiB of int64
    table = torch.zeros(n_words, dtype=torch.int64, device="cuda")
    idx = torch.randint(0, n_words, (1 << 28,), device="cuda")
    ones = torch.ones(idx.numel(), dtype=torch.int32, device="cuda")
    t32 = table.view(torch.int32)
    res = {}

    def timeit(fn):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(5):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 5

    for fetch in (0, 32, 64, 128):
        rc = _set_l2_fetch(fetch) if fetch else 0
        for name, fn in (("gather_8B", lambda: table[idx]), ("index_add_4B", lambda: t32.index_add_(0, idx * 2, ones))):
            ms = timeit(fn)
            res["%s_fetch%d" % (name, fetch)] = {"ms": round(ms, 3), "G_accesses_per_s": round(idx.numel() / ms / 1e6, 2),
                                                 "set_limit_rc": rc}
    print(json.dumps({"micro": "random 32-byte sectors over a 4 GiB table", "accesses": idx.numel(), **res}))


def run_served(args):
    """Served form: Poisson arrivals (50 jobs/s) of 1-50 Mbase libraries, k in {25,31,63}, min_count in {2,3}.

    The same arrival stream is driven through the server twice: with up to `--max-batch` queued jobs
    batched into one run (continuous batching) and with every job run alone (the plain per-library
    form behind a FIFO queue), each over both halves of the trace in the order served, FIFO, FIFO,
    served.
    """
    import queue

    import paper_1305_1861_gb300 as pkg

    specs = synth.served_jobs(seed=5, n_jobs=args.jobs, rate=50.0, scale=args.scale)
    jobs = []
    for sp in specs:
        lib = synth.library_from_spec(sp)
        jobs.append((lib.bases, lib.offsets, sp["k"], sp["min_count"], sp["t"]))

    def drive(workers, jobs=jobs, paced=True):
        srv = pkg.Server(0, hbm_budget_bytes=0, max_batch=workers)
        for b, o, k, m, _ in jobs[:4]:  # warm every worker's context
            srv.poll(srv.submit(b, o, k, m))
        pending = queue.Queue()
        lat, windows, done_at = [], 0, [0.0]

        def collect():
            nonlocal windows
            while True:
                t = pending.get()
                if t is None:
                    return
                _, _, nw, tm = srv.poll(t)
                lat.append(tm.total_ms)
                windows += nw
                done_at[0] = time.perf_counter()

        th = threading.Thread(target=collect)
        th.start()
        t0 = time.perf_counter()
        for b, o, k, m, at in jobs:
            delay = at - (time.perf_counter() - t0)
            if paced and delay > 0:
                time.sleep(delay)
            pending.put(srv.submit(b, o, k, m))
        pending.put(None)
        th.join()
        st = srv.stats()
        srv.close()
        span = done_at[0] - t0
        return summary([{"lat": lat, "windows": windows, "span": span, "stats": st}])

    def summary(parts):
        lat = [x for p in parts for x in p["lat"]]
        windows = sum(p["windows"] for p in parts)
        span = sum(p["span"] for p in parts)
        return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_ms": float(np.mean(lat)), "kmers_per_s": windows / span, "makespan_s": span,
                "windows": windows, "peak_running": max(p["stats"]["peak_running"] for p in parts),
                "peak_queued": max(p["stats"]["peak_queued"] for p in parts),
                "peak_admitted_gb": max(p["stats"]["peak_admitted_bytes"] for p in parts) / 1e9,
                "_parts": parts}

    def rebased(part):  # arrival times measured from the part's first arrival
        t_first = part[0][4]
        return [(b, o, k, m, at - t_first) for b, o, k, m, at in part]

    # Poisson arrivals, in the order A B B A: served and FIFO each run both halves of the trace, so a
    # drift of the host's speed during the run (boxes vary by up to 2x on the host side) hits both.
    half = len(jobs) // 2
    h1, h2 = rebased(jobs[:half]), rebased(jobs[half:])
    s1 = drive(args.max_batch, h1)
    p1 = drive(1, h1)
    p2 = drive(1, h2)
    s2 = drive(args.max_batch, h2)
    served = summary(s1["_parts"] + s2["_parts"])
    plain = summary(p1["_parts"] + p2["_parts"])
    burst = jobs[: args.saturate_jobs]
    # saturated: the two modes alternate twice and the second run of each counts (host-side warm-up
    # and page-cache effects otherwise favour whichever mode runs later)
    drive(1, burst, paced=False)
    drive(args.max_batch, burst, paced=False)
    sat_plain = drive(1, burst, paced=False)
    sat_served = drive(args.max_batch, burst, paced=False)
    for d in (served, plain, sat_plain, sat_served):
        d.pop("_parts")
    return {"metric": "served: p50/p99 job latency and aggregate canonical k-mers/s", "value": served["kmers_per_s"],
            "unit": METRIC, "n_gpus": 1, "higher_is_better": True, "data": "synthetic",
            "config": {"workload": "served: %d jobs, Poisson arrivals 50/s, read bases log-uniform %.1f-%.0f Mbase, "
                                   "100 bp, 1%% substitutions, k in {25,31,63}, min_count in {2,3}"
                                   % (len(jobs), 1.0 * args.scale, 50.0 * args.scale),
                       "max_batch": args.max_batch},
            "served": served, "plain_fifo_1_worker": plain,
            "p99_speedup_vs_plain": plain["p99_ms"] / served["p99_ms"],
            "saturated": {"jobs": len(burst), "served": sat_served, "plain_fifo_1_worker": sat_plain,
                          "throughput_vs_plain": sat_served["kmers_per_s"] / sat_plain["kmers_per_s"]}}


def run_batched(args):
    """Batched form: 64 libraries (genome log-uniform 0.1-20 Mbp, coverage U(10,60), 100/150 bp, 1% errors,
    k in {21,31,55}) counted by turtle_count_batch vs 64 sequential turtle_count calls (host memory, end to end);
    at full scale also the same recipe at 1/50 scale ("small_libraries")."""
    import paper_1305_1861_gb300 as pkg

    def compare(scale):
        specs = synth.batched_specs(seed=4, n_libs=64, scale=scale)
        libs = [synth.library_from_spec(sp) for sp in specs]
        jobs = [(lib.bases, lib.offsets, lib.k, lib.min_count) for lib in libs]
        res, ok = batched_vs_plain(pkg, jobs, args)
        return res, ok, sum(l.bases.size for l in libs)

    res, ok, n_bases = compare(args.scale)
    out = {"metric": "batched vs plain: canonical k-mers/s over 64 libraries", "value": res["batched"]["kmers_per_s"],
           "unit": METRIC, "n_gpus": 1, "higher_is_better": True, "data": "synthetic", "steps": args.steps,
           "config": {"workload": "batched: 64 libraries, genome log-uniform %.3g-%.3g Mbp, coverage U(10,60), "
                                  "R in {100,150}, 1%% substitutions, k in {21,31,55}, min_count 2; %.2f Gbase"
                                  % (0.1 * args.scale, 20 * args.scale, n_bases / 1e9)},
           "batched": res["batched"], "plain": res["plain_64_calls"], "batched_autotune": res["batched_autotune"],
           "batched_mixed": res["batched_mixed"],
           "speedup_vs_plain": res["plain_64_calls"]["s_per_batch"] / res["batched"]["s_per_batch"],
           "autotune_speedup_vs_plain": res["plain_64_calls"]["s_per_batch"] / res["batched_autotune"]["s_per_batch"],
           "mixed_speedup_vs_plain": res["plain_64_calls"]["s_per_batch"] / res["batched_mixed"]["s_per_batch"],
           "identical_results": ok}
    if args.scale == 1.0:  # the same recipe at 1/50 scale: small libraries, where per-call costs dominate
        res_s, ok_s, nb_s = compare(0.02)
        out["small_libraries"] = {"bases": nb_s, "batched": res_s["batched"], "plain": res_s["plain_64_calls"],
                                  "batched_autotune": res_s["batched_autotune"],
                                  "batched_mixed": res_s["batched_mixed"],
                                  "speedup_vs_plain": res_s["plain_64_calls"]["s_per_batch"]
                                  / res_s["batched"]["s_per_batch"],
                                  "autotune_speedup_vs_plain": res_s["plain_64_calls"]["s_per_batch"]
                                  / res_s["batched_autotune"]["s_per_batch"],
                                  "mixed_speedup_vs_plain": res_s["plain_64_calls"]["s_per_batch"]
                                  / res_s["batched_mixed"]["s_per_batch"], "identical_results": ok_s}
    return out


def batched_vs_plain(pkg, jobs, args):
    """64 sequential turtle_count calls vs one turtle_count_batch on the same jobs (runs of one k chosen
    automatically, autotuned, and mixed-k runs): medians of alternating steps, and whether every result
    is identical."""

    def plain():
        return [pkg.turtle_count(b, o, k, m) for b, o, k, m in jobs]

    def batched():
        return pkg.turtle_count_batch(jobs)

    tuned_params = pkg.Params.default(autotune=1)
    mixed_params = pkg.Params.default(batch_mixed=1)

    def batched_tuned():
        return pkg.turtle_count_batch(jobs, tuned_params)

    def batched_mixed():  # libraries of every k (<= 61) in shared runs of up to 64, 128-bit keys
        return pkg.turtle_count_batch(jobs, mixed_params)

    # The forms alternate step by step and each reports its median, so a drift in the host's speed
    # during the run (boxes differ and vary by up to 2x on the host side) hits all alike. The autotuned
    # batch tunes each group's class in its warm-up call; the timed calls reuse the cached knobs.
    pkg.load().turtle_tune_cache_clear()
    fns = (("plain_64_calls", plain), ("batched", batched), ("batched_autotune", batched_tuned),
           ("batched_mixed", batched_mixed))
    for _ in range(max(1, args.warmup)):
        for _, fn in fns:
            out = fn()
            del out
    times = {name: [] for name, _ in fns}
    W = 0
    for step in range(args.steps):
        for name, fn in (fns if step % 2 == 0 else fns[::-1]):
            t0 = time.perf_counter()
            out = fn()
            times[name].append(time.perf_counter() - t0)
            W = sum(o[2] for o in out)
            del out
    res = {}
    for name, _ in fns:
        dt = float(np.median(times[name]))
        res[name] = {"s_per_batch": dt, "kmers_per_s": W / dt, "windows": W,
                     "s_per_batch_all": [round(t, 4) for t in times[name]]}
    ok = all(all(np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) for b in others)
             for a, *others in zip(plain(), batched(), batched_tuned(), batched_mixed()))
    return res, ok


def run_cturtle(args):
    """cTurtle (Sec. 2.2) on the chosen library, device-resident: k-mers/s, and its false positives and
    false negatives against the exact set of k-mers seen at least twice (from the exact path)."""
    import torch

    import paper_1305_1861_gb300 as pkg

    if args.workload not in ("fly", "small"):
        raise SystemExit("--method cturtle runs on the in-memory workloads (fly, small)")
    torch.cuda.set_device(0)
    lib, desc = workload(args.workload, args.scale, 0)
    bases = torch.from_numpy(lib.bases).cuda()
    offs = torch.from_numpy(lib.offsets.astype(np.int64)).cuda()
    ctx = pkg.Context(0)
    prm = pkg.Params.default(timing=1, cturtle_bits_per_window=args.cturtle_bits)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        ctx.turtle_frequent_device(bases, offs, lib.k, prm, stream)
    torch.cuda.synchronize()
    sampler = ClockSampler(0)
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        keys, W = ctx.turtle_frequent_device(bases, offs, lib.k, prm, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / args.steps
    st = ctx.stats()
    got = keys.clone()
    ek, _, _ = ctx.turtle_count_device(bases, offs, lib.k, 2, pkg.Params.default())
    exact = ek.clone()

    if got.dim() == 1:
        hit = torch.isin(got, exact)
        n_fp = int((~hit).sum())
        n_fn = int(exact.numel() - hit.sum())
    else:  # 128-bit keys: compare on the host
        a = set(map(tuple, got.cpu().numpy().tolist()))
        b = set(map(tuple, exact.cpu().numpy().tolist()))
        n_fp, n_fn = len(a - b), len(b - a)
    n_true = int(exact.shape[0])
    return {"metric": "cTurtle: canonical k-mers/s (k-mers seen twice, no counts)", "value": W / (ms / 1e3),
            "unit": METRIC, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "data": "synthetic", "dtype": "u64" if lib.k <= 32 else "u128",
            "config": {"workload": desc, "k": lib.k, "windows": W,
                       "filter_bytes": st["filter_bytes"], "bits_per_window": args.cturtle_bits or 8},
            "reported": int(got.shape[0]), "exact_seen_twice": n_true,
            "false_positives": n_fp, "false_negatives": n_fn,
            "fp_rate": n_fp / max(n_true, 1), "fn_rate": n_fn / max(n_true, 1),
            "stage_ms": {k: round(v, 3) for k, v in st["stage_ms"].items() if v > 0}, "clocks": clocks}


def run_blocks(args, out):
    """Nested blocks of the default line: long-k at full size, batched vs plain, served vs plain."""
    import copy

    import torch

    import paper_1305_1861_gb300 as pkg

    blocks = [b for b in args.blocks.split(",") if b and b != "none"]
    for name in blocks:
        pkg.turtle_trim()  # each block starts with the device memory earlier blocks' calls kept given back
        torch.cuda.empty_cache()
        t0 = time.perf_counter()
        if name == "k64":
            res = run_k64_block(args)
        elif name == "batched":
            a = copy.copy(args)
            a.scale, a.steps, a.warmup = 1.0, max(1, min(args.steps, args.block_steps)), 1
            res = run_batched(a)
        elif name == "tuned":
            res = run_tuned_block(args)
        elif name == "served":
            a = copy.copy(args)
            a.scale, a.jobs, a.saturate_jobs = 1.0, min(args.jobs, 400), min(args.saturate_jobs, 150)
            res = run_served(a)
        else:
            raise SystemExit("unknown block %r" % name)
        res["block_wall_s"] = round(time.perf_counter() - t0, 1)
        out[name] = res


def main():
    args = parse()
    nested = args.workload is None
    if nested:
        args.workload = "fly"
    if args.workload == "batched":
        print(json.dumps(run_batched(args)), flush=True)
        return
    if args.method == "cturtle":
        print(json.dumps(run_cturtle(args)), flush=True)
        return
    if args.workload == "served":
        print(json.dumps(run_served(args)), flush=True)
        return
    if args.micro:
        micro()
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank != 0:
            return
        print(json.dumps(run_reference(args, rank, world)), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group("nccl")
    out = run_ours(args, rank, world)
    if nested and world == 1 and args.method == "scturtle":
        run_blocks(args, out)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
