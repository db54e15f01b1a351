"""Autotuner selection logic (turtle_tune_select), on CPU with synthetic timers.

The selection is coordinate descent over five knobs; with a cost that is a sum of one term per
knob it must reach the global optimum in its single sweep, it must never return params slower
than the start, gains under 2% are noise and are not taken, and configurations whose timer fails
are skipped.
"""
import ctypes

import pytest

KNOBS = {  # knob -> candidate values, in the tuner's order
    "filter_bits_per_window": [1.0, 0.5, 2.0],
    "pattern_bits": [4, 3, 6],
    "sort_tile": [0, 2, 3],
    "bucket_slots": [0, 4096],
    "bucket_windows": [16384, 8192, 32768],
}


@pytest.fixture(scope="module")
def pkg():
    import paper_1305_1861_gb300 as p

    p.build()
    p.load()
    return p


def _knob(p, name):
    v = getattr(p, name)
    return 16384 if name == "bucket_windows" and v == 0 else v


def _select(pkg, cost, base=None):
    calls = []

    def timer(ptr, user):
        p = pkg.Params.from_address(ptr)
        calls.append({n: _knob(p, n) for n in KNOBS})
        return cost(calls[-1])

    cb = pkg.TUNE_TIMER(timer)
    base = base or pkg.Params.default()
    best, rep = pkg.Params(), pkg.TuneReport()
    rc = pkg.load().turtle_tune_select(ctypes.byref(base), cb, None, ctypes.byref(best), ctypes.byref(rep))
    return rc, {n: _knob(best, n) for n in KNOBS}, rep, calls


def test_separable_cost_reaches_its_optimum_in_one_sweep(pkg):
    pref = {"filter_bits_per_window": 2.0, "pattern_bits": 3, "sort_tile": 2, "bucket_slots": 4096,
            "bucket_windows": 32768}

    def cost(c):
        return 100.0 + sum(0.0 if c[n] == pref[n] else 5.0 + KNOBS[n].index(c[n]) for n in KNOBS)

    rc, best, rep, calls = _select(pkg, cost)
    assert rc == 0 and best == pref
    sweep = 1 + sum(len(v) - 1 for v in KNOBS.values())
    assert rep.evaluations == len(calls) == sweep + 2 * 3  # the sweep, then 3 interleaved confirmations
    assert rep.best_ms == pytest.approx(100.0) and rep.default_ms == pytest.approx(100.0 + 5 * 5)


def test_never_slower_than_the_start_and_ignores_noise(pkg):
    default = {n: v[0] for n, v in KNOBS.items()}

    def cost(c):  # every change is slower, or faster by only 1%
        return 50.0 if c == default else (49.6 if c["pattern_bits"] == 6 else 60.0)

    rc, best, rep, _ = _select(pkg, cost)
    assert rc == 0 and best == default and rep.best_ms == rep.default_ms == pytest.approx(50.0)


def test_failing_configurations_are_skipped(pkg):
    def cost(c):
        if c["sort_tile"] == 3 or c["bucket_windows"] == 8192:
            return -1.0  # cannot run
        return 10.0 - (1.0 if c["sort_tile"] == 2 else 0.0)

    rc, best, rep, _ = _select(pkg, cost)
    assert rc == 0 and best["sort_tile"] == 2 and best["bucket_windows"] == 16384


def test_failing_start_is_an_error(pkg):
    rc, _, _, calls = _select(pkg, lambda c: -1.0)
    assert rc == -7 and len(calls) == 1
    bad = pkg.Params()  # struct_size unset
    best = pkg.Params()
    assert pkg.load().turtle_tune_select(ctypes.byref(bad), pkg.TUNE_TIMER(lambda p, u: 1.0), None,
                                         ctypes.byref(best), None) == -1


def test_one_lucky_timing_is_not_kept(pkg):
    """A candidate that measured fast once (noise) but not in the interleaved confirmation is dropped."""
    default = {n: v[0] for n, v in KNOBS.items()}
    seen = set()

    def cost(c):
        key = tuple(sorted(c.items()))
        if c["sort_tile"] == 2 and key not in seen:
            seen.add(key)
            return 40.0  # the first timing of this configuration is lucky
        return 50.0

    rc, best, rep, calls = _select(pkg, cost)
    assert rc == 0 and best == default and rep.best_ms == pytest.approx(50.0)
