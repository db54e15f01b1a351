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
