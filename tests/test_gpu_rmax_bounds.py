"""GPU parity for the bounds that replace the exact R_max (Sec. 3.2 step 4b):
the prescribed maximum aggregate rate and the bound learned from the exact
R_max of the colour's previous visit.  Both paths skip the device-wide
reduction before the events; the trajectories must still equal the oracle's
bit for bit (clock to 1e-12 relative), and the recorded R_max history must
match the oracle's exactly."""
import math
import os

import numpy as np
import pytest

import oracle
import paper_1005_4713_gb300 as sp
from paper_1005_4713_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

CLOCK_RTOL = 1e-12
THREADS = max(1, min(16, os.cpu_count() or 1))
MODES = [sp.SPKMC_RMAX_PRESCRIBED, sp.SPKMC_RMAX_LEARNED]


def oracle_state(spec, mode):
    return oracle.State(spec.L, spec.d, spec.J, spec.H, spec.T, spec.seed, cold=spec.cold, rmax_mode=mode)


def gpu_lattice(spec, mode, log=0, config=None):
    return sp.Lattice(spec.L, spec.d, spec.J, spec.H, spec.T, spec.seed, cold=spec.cold,
                      event_log_capacity=log, config=config, rmax_mode=mode)


def assert_same(lat, st, spins=True):
    o = lat.observables()
    assert o.cycle == st.cycle
    assert (o.n_flip, o.n_null) == (st.n_flip, st.n_null)
    assert int(o.sum_null_rate_fx[0]) | (int(o.sum_null_rate_fx[1]) << 64) == st.null_fx
    assert o.clock == pytest.approx(st.clock, rel=CLOCK_RTOL, abs=0.0), (o.clock, st.clock)
    assert list(lat.state().rmax_hist) == list(st.rmax_hist)
    if spins:
        s = lat.spins()
        assert np.array_equal(s, st.spins), int(np.sum(s != st.spins))
        assert (o.M, o.B) == st.observables()


def log_as_array(ev):
    return np.stack([ev["domain"], ev["cls"], ev["site"]], axis=-1).astype(np.int32)


@pytest.mark.parametrize("mode", MODES)
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
def test_bounds_match_oracle_with_event_log(mode, spec):
    """Runs in chunks of 37 cycles (launches start at both parities and the
    learned bound reads history across launches), event log compared whole."""
    st = oracle_state(spec, mode)
    n, chunk = 185, 37
    with gpu_lattice(spec, mode, log=n * st.k_act) as lat:
        logs = []
        for _ in range(n // chunk):
            lat.run(chunk)
            logs.append(st.run(chunk, log=True, threads=THREADS))
            assert_same(lat, st)
        assert np.array_equal(log_as_array(lat.event_log()), np.concatenate(logs).reshape(-1, 3))
        assert lat.check_counts() == 0


@pytest.mark.parametrize("mode", MODES)
def test_config_128_with_bounds(mode):
    spec = wl.CONFIG_128_HOT
    st = oracle_state(spec, mode)
    with gpu_lattice(spec, mode) as lat:
        for _ in range(4):
            lat.run(100)
            st.run(100, threads=THREADS)
            assert_same(lat, st)


def test_config_1024_learned_first_sixteen_cycles():
    """1024^3, 16^3-site domains, in the benchmark's launch configuration:
    8 cycles on the prescribed bound, then 8 on the learned one."""
    spec = wl.CONFIG_1024
    st = oracle_state(spec, sp.SPKMC_RMAX_LEARNED)
    with gpu_lattice(spec, sp.SPKMC_RMAX_LEARNED) as lat:
        lat.run(16)
        st.run(16, threads=THREADS)
        assert_same(lat, st)


def test_learned_bound_is_tight_and_prescribed_is_not():
    """Null fraction: learned close to exact, prescribed far above it."""
    spec = wl.LatticeSpec(L=64, d=16, seed=31)
    ur = {}
    for mode in (sp.SPKMC_RMAX_EXACT, sp.SPKMC_RMAX_PRESCRIBED, sp.SPKMC_RMAX_LEARNED):
        with sp.Lattice(spec.L, spec.d, seed=spec.seed, rmax_mode=mode) as lat:
            lat.run(800)
            o = lat.observables()
            ur[mode] = o.n_flip / (o.n_flip + o.n_null)
    assert ur[sp.SPKMC_RMAX_LEARNED] > 0.97 * ur[sp.SPKMC_RMAX_EXACT]
    assert ur[sp.SPKMC_RMAX_PRESCRIBED] < 0.7 * ur[sp.SPKMC_RMAX_EXACT]


def test_batch_mixing_modes_equals_solo_oracle_runs():
    """Exact lattices keep the reduction before the events; the others ride
    along in the same launch.  Each lattice equals its own oracle run."""
    specs = [(wl.LatticeSpec(L=32, d=4, seed=41), sp.SPKMC_RMAX_EXACT),
             (wl.LatticeSpec(L=48, d=8, seed=42, H=0.01), sp.SPKMC_RMAX_LEARNED),
             (wl.LatticeSpec(L=16, d=2, seed=43, T=3.0), sp.SPKMC_RMAX_PRESCRIBED),
             (wl.LatticeSpec(L=64, d=16, seed=44, cold=True), sp.SPKMC_RMAX_LEARNED)]
    with sp.Batch(8) as b:
        slots = [b.admit(s.L, s.d, s.J, s.H, s.T, s.seed, cold=s.cold, rmax_mode=m) for s, m in specs]
        b.run(29)
        b.run(40)
        obs = b.observables_all()
        for (s, m), sl in zip(specs, slots):
            st = oracle_state(s, m)
            st.run(69, threads=THREADS)
            o = obs[sl]
            assert (o.cycle, o.n_flip, o.n_null) == (st.cycle, st.n_flip, st.n_null)
            assert o.clock == pytest.approx(st.clock, rel=CLOCK_RTOL, abs=0.0)
            assert np.array_equal(b.spins(sl), st.spins)


def test_batch_of_bound_lattices_only():
    """No lattice needs the exact R_max: the launch has no barrier before
    the events at all."""
    specs = [wl.LatticeSpec(L=L, d=d, seed=50 + i, T=T)
             for i, (L, d, T) in enumerate([(16, 4, 4.5), (32, 8, 4.4), (24, 4, 4.6), (64, 16, 4.51)])]
    with sp.Batch(8) as b:
        slots = [b.admit(s.L, s.d, s.J, s.H, s.T, s.seed, rmax_mode=sp.SPKMC_RMAX_LEARNED) for s in specs]
        b.run(57)
        obs = b.observables_all()
        for s, sl in zip(specs, slots):
            st = oracle_state(s, sp.SPKMC_RMAX_LEARNED)
            st.run(57)
            assert (obs[sl].n_flip, obs[sl].n_null) == (st.n_flip, st.n_null)
            assert np.array_equal(b.spins(sl), st.spins)


def test_learned_checkpoint_resume_is_bit_exact():
    spec = wl.LatticeSpec(L=64, d=8, seed=61)
    mode = sp.SPKMC_RMAX_LEARNED
    with gpu_lattice(spec, mode) as a:
        a.run(21)
        state, spins = a.state(), a.spins()
        assert all(h > 0 for h in state.rmax_hist)
        a.run(30)
        with gpu_lattice(wl.LatticeSpec(L=64, d=8, seed=61, cold=True), mode) as b:
            b.set_spins(spins)
            b.set_state(state)
            b.run(30)
            assert np.array_equal(a.spins(), b.spins())
            oa, ob = a.observables(), b.observables()
            assert (oa.cycle, oa.clock, oa.n_flip, oa.n_null) == (ob.cycle, ob.clock, ob.n_flip, ob.n_null)
            assert list(a.state().rmax_hist) == list(b.state().rmax_hist)


def test_set_spins_clears_the_history():
    spec = wl.LatticeSpec(L=32, d=4, seed=62)
    mode = sp.SPKMC_RMAX_LEARNED
    st = oracle_state(spec, mode)
    with gpu_lattice(spec, mode) as lat:
        lat.run(20)
        st.run(20)
        lat.set_spins(lat.spins())
        assert list(lat.state().rmax_hist) == [0.0] * 8
        st.rmax_hist[:] = 0.0
        lat.run(12)
        st.run(12)
        assert_same(lat, st)


def test_exceeded_bound_is_reported_and_the_context_survives():
    """A history too small for the lattice (set through the checkpoint
    interface) makes the device's tolerance check fail: the host reads
    EBOUND, and a valid state makes the handle usable again."""
    spec = wl.LatticeSpec(L=32, d=8, seed=63)
    mode = sp.SPKMC_RMAX_LEARNED
    with gpu_lattice(spec, mode) as lat:
        good = lat.state()
        bad = lat.state()
        for i in range(8):
            bad.rmax_hist[i] = 1.0
        lat.set_state(bad)
        lat.run(3)
        with pytest.raises(sp.SpkmcError) as e:
            lat.synchronize()
        assert e.value.code == sp.SPKMC_EBOUND
    with gpu_lattice(spec, mode) as lat:
        lat.set_state(good)
        lat.run(10)
        st = oracle_state(spec, mode)
        st.run(10)
        assert_same(lat, st)


def test_noalloc_entry_point_with_learned_bound():
    torch = pytest.importorskip("torch")
    spec = wl.LatticeSpec(L=32, d=4, seed=64)
    mode = sp.SPKMC_RMAX_LEARNED
    st = oracle_state(spec, mode)
    spins = torch.from_numpy(st.spins.copy()).cuda()
    p = sp.make_params(spec.L, spec.d, spec.J, spec.H, spec.T, spec.seed, rmax_mode=mode)
    state = sp.spkmc_state()
    sp.spkmc_run_cycles_noalloc(p, spins.data_ptr(), state, 13)
    sp.spkmc_run_cycles_noalloc(p, spins.data_ptr(), state, 14)
    torch.cuda.synchronize()
    st.run(27)
    assert np.array_equal(spins.cpu().numpy(), st.spins)
    assert (state.cycle, state.n_flip, state.n_null) == (st.cycle, st.n_flip, st.n_null)
    assert math.isclose(state.clock, st.clock, rel_tol=CLOCK_RTOL)
    assert list(state.rmax_hist) == list(st.rmax_hist)


def test_noalloc_error_leaves_the_spins_and_the_state_as_they_were():
    """A history too small for the lattice makes the device's tolerance check
    stop the no-allocation run with EBOUND: the caller's spin buffer still
    holds its input and the state its old values, and a call with a valid
    state then runs as the oracle."""
    torch = pytest.importorskip("torch")
    spec = wl.LatticeSpec(L=32, d=4, seed=65)
    mode = sp.SPKMC_RMAX_LEARNED
    st = oracle_state(spec, mode)
    spins0 = st.spins.copy()
    dev = torch.from_numpy(spins0.copy()).cuda()
    p = sp.make_params(spec.L, spec.d, spec.J, spec.H, spec.T, spec.seed, rmax_mode=mode)
    bad = sp.spkmc_state()
    for i in range(8):
        bad.rmax_hist[i] = 1.0
    with pytest.raises(sp.SpkmcError) as e:
        sp.spkmc_run_cycles_noalloc(p, dev.data_ptr(), bad, 20)
    assert e.value.code == sp.SPKMC_EBOUND
    torch.cuda.synchronize()
    assert np.array_equal(dev.cpu().numpy(), spins0)
    assert (bad.cycle, bad.n_flip, bad.n_null, bad.clock) == (0, 0, 0, 0.0)
    assert list(bad.rmax_hist) == [1.0] * 8
    good = sp.spkmc_state()
    sp.spkmc_run_cycles_noalloc(p, dev.data_ptr(), good, 20)
    st.run(20)
    assert np.array_equal(dev.cpu().numpy(), st.spins)
    assert (good.cycle, good.n_flip, good.n_null) == (st.cycle, st.n_flip, st.n_null)


@pytest.mark.parametrize("mode", MODES + [sp.SPKMC_RMAX_EXACT])
@pytest.mark.parametrize("L,d,cycles", [(1024, 16, 2000), (256, 16, 20000), (128, 8, 20000), (64, 4, 20000)])
def test_long_runs_keep_counts_consistent(mode, L, d, cycles):
    """Long runs in launches of many cycles (where CTAs drift apart most
    across the cycles without a grid barrier): the class counts, ghost faces,
    M and B kept flip by flip still equal a recount from the spins."""
    spec = wl.LatticeSpec(L=L, d=d, seed=71)
    with gpu_lattice(spec, mode) as lat:
        lat.run(cycles)
        assert lat.check_counts() == 0
        o = lat.observables()
        assert o.cycle == cycles and o.n_flip + o.n_null == cycles * lat.K_act
