"""GPU parity for the paper's two-colour sublattice (Sec. 3.2 step 4a): half
of the domains active per cycle, the colour drawn at random each cycle, the
class counts of each active domain recounted from its spins at the start of
its cycle.  Spins, event logs and counters bit-identical to the oracle, the
clock to 1e-12 relative."""
import os

import numpy as np
import pytest

import oracle
import paper_1005_4713_gb300 as sp
from paper_1005_4713_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

CLOCK_RTOL = 1e-12
THREADS = max(1, min(16, os.cpu_count() or 1))
TWO = sp.SPKMC_SUBLATTICE_2_RANDOM


def oracle_state(spec, mode=0):
    return oracle.State(spec.L, spec.d, spec.J, spec.H, spec.T, spec.seed, cold=spec.cold, rmax_mode=mode,
                        sublattice=oracle.SUB_2_RANDOM)


def gpu_lattice(spec, mode=0, log=0, config=None):
    return sp.Lattice(spec.L, spec.d, spec.J, spec.H, spec.T, spec.seed, cold=spec.cold,
                      event_log_capacity=log, config=config, rmax_mode=mode, sublattice=TWO)


def assert_same(lat, st):
    o = lat.observables()
    assert o.cycle == st.cycle
    assert (o.n_flip, o.n_null) == (st.n_flip, st.n_null)
    assert int(o.sum_null_rate_fx[0]) | (int(o.sum_null_rate_fx[1]) << 64) == st.null_fx
    assert o.clock == pytest.approx(st.clock, rel=CLOCK_RTOL, abs=0.0), (o.clock, st.clock)
    s = lat.spins()
    assert np.array_equal(s, st.spins), int(np.sum(s != st.spins))
    assert (o.M, o.B) == st.observables()


def log_as_array(ev):
    return np.stack([ev["domain"], ev["cls"], ev["site"]], axis=-1).astype(np.int32)


@pytest.mark.parametrize("mode", [sp.SPKMC_RMAX_EXACT, sp.SPKMC_RMAX_PRESCRIBED])
@pytest.mark.parametrize("spec", [
    wl.LatticeSpec(L=16, d=4, seed=1),
    wl.LatticeSpec(L=16, d=4, seed=1, cold=True),
    wl.LatticeSpec(L=4, d=2, seed=3),                     # nd = 2
    wl.LatticeSpec(L=32, d=2, seed=7, T=6.0),
    wl.LatticeSpec(L=64, d=8, seed=9, H=0.01),
    wl.LatticeSpec(L=48, d=8, seed=10, T=1.5, H=-0.2),
    wl.LatticeSpec(L=16, d=8, seed=5, J=-0.7, H=0.1, T=2.0),
    wl.LatticeSpec(L=96, d=16, seed=11),
])
def test_two_colour_matches_oracle_with_event_log(mode, spec):
    st = oracle_state(spec, mode)
    n, chunk = 111, 37
    with gpu_lattice(spec, mode, log=n * st.k_act) as lat:
        assert lat.K_act == (spec.L // spec.d) ** 3 // 2
        logs = []
        for _ in range(n // chunk):
            lat.run(chunk)
            logs.append(st.run(chunk, log=True, threads=THREADS))
            assert_same(lat, st)
        assert np.array_equal(log_as_array(lat.event_log()), np.concatenate(logs).reshape(-1, 3))
        assert lat.check_counts() == 0
        assert np.array_equal(lat.class_counts(), oracle.class_counts(spec.L, spec.d, st.spins))


def test_two_colour_128():
    spec = wl.CONFIG_128_HOT
    st = oracle_state(spec)
    with gpu_lattice(spec) as lat:
        for _ in range(3):
            lat.run(100)
            st.run(100, threads=THREADS)
            assert_same(lat, st)


def test_two_colour_1024_first_cycles():
    """1024^3, d = 16: 131 072 events per cycle, CTAs of several staging
    rounds (the recount stages its own rounds)."""
    spec = wl.CONFIG_1024
    st = oracle_state(spec)
    with gpu_lattice(spec) as lat:
        lat.run(4)
        st.run(4, threads=THREADS)
        assert_same(lat, st)


@pytest.mark.parametrize("kw", [dict(max_ctas=1), dict(items_per_cta=7), dict(items_per_cta=1000)])
def test_two_colour_launch_geometry(kw):
    spec = wl.LatticeSpec(L=64, d=4, seed=22)
    st = oracle_state(spec)
    st.run(30, threads=THREADS)
    with gpu_lattice(spec, config=sp.make_config(**kw)) as lat:
        lat.run(30)
        assert_same(lat, st)


def test_batch_mixing_sublattice_schemes():
    specs = [(wl.LatticeSpec(L=32, d=4, seed=41), 0, 0), (wl.LatticeSpec(L=48, d=8, seed=42, H=0.01), 1, 0),
             (wl.LatticeSpec(L=16, d=2, seed=43, T=3.0), 1, 1), (wl.LatticeSpec(L=64, d=16, seed=44, cold=True), 0, 2),
             (wl.LatticeSpec(L=32, d=16, seed=45), 1, 0)]
    with sp.Batch(8) as b:
        slots = [b.admit(s.L, s.d, s.J, s.H, s.T, s.seed, cold=s.cold, rmax_mode=m, sublattice=sub)
                 for s, sub, m in specs]
        b.run(23)
        b.run(30)
        for (s, sub, m), sl in zip(specs, slots):
            st = oracle.State(s.L, s.d, s.J, s.H, s.T, s.seed, cold=s.cold, rmax_mode=m, sublattice=sub)
            st.run(53)
            o = b.observables(sl)
            assert (o.cycle, o.n_flip, o.n_null) == (st.cycle, st.n_flip, st.n_null)
            assert o.clock == pytest.approx(st.clock, rel=CLOCK_RTOL, abs=0.0)
            assert np.array_equal(b.spins(sl), st.spins)


def test_two_colour_checkpoint_resume():
    spec = wl.LatticeSpec(L=64, d=8, seed=61)
    with gpu_lattice(spec) as a:
        a.run(17)
        state, spins = a.state(), a.spins()
        a.run(20)
        with gpu_lattice(wl.LatticeSpec(L=64, d=8, seed=61, cold=True)) as b:
            b.set_spins(spins)
            b.set_state(state)
            b.run(20)
            assert np.array_equal(a.spins(), b.spins())
            oa, ob = a.observables(), b.observables()
            assert (oa.cycle, oa.clock, oa.n_flip, oa.n_null) == (ob.cycle, ob.clock, ob.n_flip, ob.n_null)
