"""Served stream (continuous batching) and batched ensembles: results equal
the solo runs bit for bit; admission respects the memory budget."""
import numpy as np
import pytest

import paper_1005_4713_gb300 as sp
from paper_1005_4713_gb300 import ensemble, serve
from paper_1005_4713_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def solo_key(spec, cycles):
    with sp.Lattice(spec.L, spec.d, spec.J, spec.H, spec.T, spec.seed, cold=spec.cold) as lat:
        lat.run(cycles)
        o = lat.observables()
        return (o.cycle, o.clock, o.M, o.B, o.n_flip, o.n_null, int(o.sum_null_rate_fx[0]),
                int(o.sum_null_rate_fx[1])), lat.spins()


def small_stream(n=24, seed=9):
    return wl.request_stream(n=n, rate=1000.0, seed=seed, sizes=(16, 32, 48), cycles_range=(10, 300))


def test_served_results_equal_solo_runs():
    reqs = small_stream()
    srv = serve.Server(budget_bytes=1 << 30, capacity=8, step_cycles=37, keep_spins=True)
    stats = srv.serve(reqs, realtime=False)
    assert len(stats.completions) == len(reqs) and not stats.rejected
    assert stats.peak_live > 1  # the work of several requests overlapped on the device
    by_id = {r.rid: r for r in reqs}
    for c in stats.completions:
        r = by_id[c.rid]
        key, spins = solo_key(r.spec, r.cycles)
        assert c.obs == key
        assert np.array_equal(c.spins, spins)


def test_admission_respects_a_small_memory_budget():
    reqs = small_stream(n=12, seed=3)
    largest = max(sp.spkmc_bytes_required(sp.make_params(r.spec.L, r.spec.d)) for r in reqs)
    budget = 2 * largest + 1  # at most two of the largest at a time
    srv = serve.Server(budget_bytes=budget, capacity=16, step_cycles=50)
    stats = srv.serve(reqs, realtime=False)
    assert stats.peak_bytes <= budget
    assert len(stats.completions) + len(stats.rejected) == len(reqs)
    assert len(stats.completions) == len(reqs)


def test_request_too_large_for_the_budget_is_rejected():
    reqs = small_stream(n=4, seed=4)
    srv = serve.Server(budget_bytes=1024, capacity=4, step_cycles=50)
    stats = srv.serve(reqs, realtime=False)
    assert sorted(stats.rejected) == sorted(r.rid for r in reqs)


def test_cancelled_request_stops_early():
    reqs = small_stream(n=3, seed=5)
    for r in reqs:
        r.cycles = 5000
    srv = serve.Server(budget_bytes=1 << 30, capacity=4, step_cycles=20)
    srv.cancel(reqs[0].rid)
    stats = srv.serve(reqs, realtime=False)
    c0 = next(c for c in stats.completions if c.rid == reqs[0].rid)
    assert c0.cancelled and c0.cycles < 5000
    assert all(c.cycles == 5000 for c in stats.completions if c.rid != reqs[0].rid)


def test_batched_ensemble_equals_one_at_a_time():
    specs = wl.ensemble_specs(12, seed=11)
    a = ensemble.run_batched(specs, cycles=120, sample_every=40, burn_in=40)
    b = ensemble.run_one_at_a_time(specs, cycles=120, sample_every=40, burn_in=40)
    assert a.final == b.final
    for x, y in zip(a.binder, b.binder):
        assert x["samples"] == y["samples"] == 2
        assert x["U4"] == y["U4"]


def test_ensemble_samples_equal_plain_read_outs():
    """The recorded samples (and a last, shorter sample) equal m^2 and m^4
    read synchronously after plain runs to the same cycles."""
    specs = wl.ensemble_specs(5, seed=13)
    a = ensemble.run_batched(specs, cycles=130, sample_every=40, burn_in=50)
    for s, got in zip(specs, a.binder):
        with sp.Lattice(s.L, s.d, s.J, s.H, s.T, s.seed, cold=s.cold) as lat:
            m2, m4 = [], []
            for c in (40, 40, 40, 10):  # samples after cycles 80, 120, 130
                lat.run(c)
                if lat.observables().cycle > 50:
                    o = lat.observables()
                    m2.append(o.m2)
                    m4.append(o.m4)
        assert got["samples"] == 3
        assert got["m2"] == sum(m2) / 3 and got["m4"] == sum(m4) / 3


def test_one_at_a_time_baseline_equals_the_served_results():
    """The baseline of continuous batching (each request alone with the plain
    single-lattice path, first come first served) gives the same result for
    every request, and reports its own queue and run times."""
    reqs = small_stream(n=10, seed=4)
    batched = serve.Server(budget_bytes=1 << 30, capacity=8, step_cycles=25).serve(reqs, realtime=False)
    alone = serve.serve_one_at_a_time(reqs, realtime=False)
    assert sorted(c.rid for c in alone.completions) == sorted(r.rid for r in reqs)
    got = {c.rid: c.obs for c in batched.completions}
    for c in alone.completions:
        assert c.obs == got[c.rid]
        assert c.finished >= c.admitted >= c.arrival
    b = alone.breakdown(50)
    assert b["queue_s"] >= 0.0 and b["run_s"] > 0.0
    assert set(alone.by_size()) <= {"16", "32", "48"}
