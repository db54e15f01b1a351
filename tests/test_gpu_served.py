"""Served form (continuous batching): each result is the same alone and in the mix (bit-exact)."""
import time

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _jobs(n, seed=5):
    specs = synth.served_jobs(seed=seed, n_jobs=n, scale=0.2)  # 0.2-10 Mbase each
    libs = []
    for sp in specs:
        lib = synth.library_from_spec(sp)
        libs.append((lib.bases, lib.offsets, sp["k"], sp["min_count"]))
    return libs


def test_results_alone_equal_results_in_the_mix(have_gpu):
    import paper_1305_1861_gb300 as pkg

    jobs = _jobs(24)
    alone = [pkg.turtle_count(b, o, k, m) for b, o, k, m in jobs]
    srv = pkg.Server(0, hbm_budget_bytes=3 << 30, max_batch=4)
    tickets = [srv.submit(b, o, k, m) for b, o, k, m in jobs]
    for t, (ak, ac, an) in zip(tickets, alone):
        keys, counts, nw, tm = srv.poll(t)
        assert nw == an and np.array_equal(keys, ak) and np.array_equal(counts, ac)
        assert tm.total_ms >= tm.run_ms >= 0
    st = srv.stats()
    assert st["completed"] == 24 and st["failed"] == 0 and st["peak_admitted_bytes"] <= 3 << 30
    assert st["largest_batch"] >= 2 and st["batches"] < 24  # queued jobs shared runs
    srv.close()
    for (b, o, k, m), (ak, ac, an) in zip(jobs, alone):  # every job, alone (and so in the mix), is the oracle's
        ok, oc, onw = oracle.count(b, o, k, m)
        assert an == onw and np.array_equal(ak, ok) and np.array_equal(ac.astype(np.uint64), oc)


def test_admission_refuses_a_job_larger_than_the_budget(have_gpu):
    import paper_1305_1861_gb300 as pkg

    b, o, k, m = _jobs(1)[0]
    srv = pkg.Server(0, hbm_budget_bytes=1 << 20, max_batch=1)
    with pytest.raises(pkg.TurtleError) as e:
        srv.submit(b, o, k, m)
    assert e.value.code == -6
    srv.close()


def test_poll_times_out_then_completes(have_gpu):
    import paper_1305_1861_gb300 as pkg

    big = synth.fly(seed=3, scale=0.05)  # ~150 Mbase: tens of ms on the single worker
    small = _jobs(1)[0]
    srv = pkg.Server(0, hbm_budget_bytes=64 << 30, max_batch=1)
    t_big = srv.submit(big.bases, big.offsets, 31, 2)
    t_small = srv.submit(*small)
    with pytest.raises(pkg.TurtleError) as e:
        srv.poll(t_small, timeout_ms=0)  # still queued behind the big job
    assert e.value.code == -5
    srv.poll(t_big)
    keys, counts, nw, tm = srv.poll(t_small, timeout_ms=60_000)
    assert tm.queue_ms > 0
    with pytest.raises(pkg.TurtleError) as e:
        srv.poll(t_small, timeout_ms=0)  # already collected: unknown ticket
    assert e.value.code == -1
    srv.close()


def test_runs_of_different_jobs_overlap_on_the_device(have_gpu):
    """Jobs of different k cannot share a run; with two executors, two runs are in flight at once
    (their [start, end) intervals intersect), and every result is still the oracle's."""
    import paper_1305_1861_gb300 as pkg

    libs = [synth.fly(seed=60 + i, scale=0.02) for i in range(6)]
    ks = [31, 63, 31, 63, 25, 63]
    srv = pkg.Server(0, hbm_budget_bytes=64 << 30, max_batch=1, executors=2)
    tickets = [srv.submit(l.bases, l.offsets, k, 2) for l, k in zip(libs, ks)]
    res = [srv.poll(t) for t in tickets]
    st = srv.stats()
    srv.close()
    assert st["executors"] == 2 and st["peak_running_batches"] == 2 and st["failed"] == 0
    spans = [(tm.start_ms, tm.end_ms) for _, _, _, tm in res]
    overlap = [(i, j) for i in range(6) for j in range(i + 1, 6)
               if ks[i] != ks[j] and spans[i][0] < spans[j][1] and spans[j][0] < spans[i][1]]
    assert overlap, spans
    for l, k, (keys, counts, nw, _) in zip(libs, ks, res):
        ok, oc, onw = oracle.count(l.bases, l.offsets, k, 2)
        assert nw == onw and np.array_equal(keys, ok) and np.array_equal(counts.astype(np.uint64), oc)


def test_one_executor_runs_one_batch_at_a_time(have_gpu):
    import paper_1305_1861_gb300 as pkg

    libs = [synth.fly(seed=60 + i, scale=0.02) for i in range(4)]
    srv = pkg.Server(0, hbm_budget_bytes=64 << 30, max_batch=1, executors=1)
    tickets = [srv.submit(l.bases, l.offsets, k, 2) for l, k in zip(libs, [31, 63, 31, 63])]
    for t in tickets:
        srv.poll(t)
    st = srv.stats()
    srv.close()
    assert st["executors"] == 1 and st["peak_running_batches"] == 1 and st["batches"] == 4


def test_queued_jobs_of_different_k_share_a_mixed_run(have_gpu):
    """With batch_mixed = 1, queued jobs of different k (and the same min_count) join one run; every
    result is still the oracle's."""
    import paper_1305_1861_gb300 as pkg

    big = synth.fly(seed=3, scale=0.05)  # keeps the one executor busy while the others queue
    small = _jobs(8, seed=9)
    ks = [15, 25, 31, 45] * 2
    jobs = [(b, o, k, 2) for (b, o, _, _), k in zip(small, ks)]
    srv = pkg.Server(0, hbm_budget_bytes=64 << 30, max_batch=8, params=pkg.Params.default(batch_mixed=1),
                     executors=1)
    t_big = srv.submit(big.bases, big.offsets, 31, 2)
    tickets = [srv.submit(*j) for j in jobs]
    srv.poll(t_big)
    got = [srv.poll(t) for t in tickets]
    st = srv.stats()
    srv.close()
    assert st["completed"] == 9 and st["failed"] == 0
    assert st["largest_batch"] >= 3  # runs of one k would hold at most the two jobs of that k
    for (b, o, k, m), (keys, counts, nw, _) in zip(jobs, got):
        ok, oc, onw = oracle.count(b, o, k, m)
        assert nw == onw and np.array_equal(keys, ok) and np.array_equal(counts.astype(np.uint64), oc)
