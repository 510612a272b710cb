"""GPU tests of the recorded run (spkmc_run_recorded): every * nrec cycles of
Sec. 3.1 in one persistent launch, with the observables recorded on the
device after every `every` cycles.  Each record must equal, bit for bit, the
synchronous read-out of a lattice stepped to the same cycle by plain runs,
and the oracle's counters and clock at that cycle."""
import os

import numpy as np
import pytest

import oracle
import paper_1005_4713_gb300 as sp
from paper_1005_4713_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

CLOCK_RTOL = 1e-12
THREADS = max(1, min(16, os.cpu_count() or 1))
FIELDS = ("cycle", "clock", "M", "B", "E", "m", "m2", "m4", "n_flip", "n_null", "sum_null_rate", "L",
          "domain_edge")


def gpu_lattice(spec, mode=sp.SPKMC_RMAX_EXACT, sub=sp.SPKMC_SUBLATTICE_8_ROTATING):
    return sp.Lattice(spec.L, spec.d, spec.J, spec.H, spec.T, spec.seed, cold=spec.cold, rmax_mode=mode,
                      sublattice=sub)


def assert_equal_obs(x, y):
    for f in FIELDS:
        assert getattr(x, f) == getattr(y, f), (f, getattr(x, f), getattr(y, f))
    assert list(x.sum_null_rate_fx) == list(y.sum_null_rate_fx)


@pytest.mark.parametrize("mode,sub", [
    (sp.SPKMC_RMAX_EXACT, sp.SPKMC_SUBLATTICE_8_ROTATING),
    (sp.SPKMC_RMAX_LEARNED, sp.SPKMC_SUBLATTICE_8_ROTATING),
    (sp.SPKMC_RMAX_PRESCRIBED, sp.SPKMC_SUBLATTICE_8_ROTATING),
    (sp.SPKMC_RMAX_EXACT, sp.SPKMC_SUBLATTICE_2_RANDOM),
])
@pytest.mark.parametrize("spec,every,nrec,pre", [
    (wl.LatticeSpec(L=4, d=2, seed=3), 1, 9, 0),         # nd = 2, a record every cycle
    (wl.LatticeSpec(L=32, d=4, seed=41, H=0.01), 3, 7, 1),  # starts on an odd cycle
    (wl.LatticeSpec(L=64, d=8, seed=42, cold=True), 10, 5, 0),
    (wl.LatticeSpec(L=96, d=16, seed=43, T=3.9), 7, 4, 5),
])
def test_records_equal_synchronous_read_outs(mode, sub, spec, every, nrec, pre):
    """Records of one launch equal the read-outs of plain runs of `every`
    cycles, field for field; the lattice then continues as the plain one."""
    rec = sp.obs_buffer(nrec)
    with gpu_lattice(spec, mode, sub) as a, gpu_lattice(spec, mode, sub) as b:
        if pre:
            a.run(pre)
            b.run(pre)
        a.run_recorded(every, nrec, rec)
        ref = []
        for _ in range(nrec):
            b.run(every)
            ref.append(b.observables())
        a.synchronize()
        for r in range(nrec):
            assert_equal_obs(rec[r], ref[r])
        assert rec[nrec - 1].cycle == pre + every * nrec
        assert np.array_equal(a.spins(), b.spins())
        assert a.check_counts() == 0
        a.run(3)
        b.run(3)
        assert_equal_obs(a.observables(), b.observables())
        assert np.array_equal(a.spins(), b.spins())


@pytest.mark.parametrize("spec,every,nrec", [
    (wl.LatticeSpec(L=16, d=4, seed=44), 5, 6),
    (wl.LatticeSpec(L=64, d=16, seed=45, H=-0.05), 4, 5),
])
def test_records_match_the_oracle(spec, every, nrec):
    """Each record against the oracle stepped to the same cycle: counters and
    M, B exact, the clock to 1e-12 relative."""
    rec = sp.obs_buffer(nrec)
    st = oracle.State(spec.L, spec.d, spec.J, spec.H, spec.T, spec.seed, cold=spec.cold)
    with gpu_lattice(spec) as a:
        a.run_recorded(every, nrec, rec)
        a.synchronize()
        for r in range(nrec):
            st.run(every, threads=THREADS)
            o = rec[r]
            assert o.cycle == st.cycle
            assert (o.n_flip, o.n_null) == (st.n_flip, st.n_null)
            assert int(o.sum_null_rate_fx[0]) | (int(o.sum_null_rate_fx[1]) << 64) == st.null_fx
            assert (o.M, o.B) == st.observables()
            assert o.clock == pytest.approx(st.clock, rel=CLOCK_RTOL, abs=0.0)
        assert np.array_equal(a.spins(), st.spins)


def test_records_at_the_benchmark_size():
    """1024^3, d = 16, records every 10 cycles (the benchmark's launch):
    each record equals the read-out after plain 10-cycle runs."""
    spec = wl.LatticeSpec(L=1024, d=16, seed=3)
    nrec = 3
    rec = sp.obs_buffer(nrec)
    with gpu_lattice(spec) as a, gpu_lattice(spec) as b:
        a.run_recorded(10, nrec, rec)
        ref = []
        for _ in range(nrec):
            b.run(10)
            ref.append(b.observables())
        a.synchronize()
        for r in range(nrec):
            assert_equal_obs(rec[r], ref[r])
        assert a.check_counts() == 0


def test_recorded_arguments_are_checked():
    spec = wl.LatticeSpec(L=32, d=4, seed=46)
    rec = sp.obs_buffer(4)
    with gpu_lattice(spec) as lat:
        for every, nrec in [(0, 4), (4, 0), (-1, 2), (1 << 17, 4)]:
            with pytest.raises(sp.SpkmcError) as e:
                sp._check(sp.lib().spkmc_run_recorded(lat.h, every, nrec, rec.records))
            assert e.value.code == sp.SPKMC_EINVAL
        with pytest.raises(sp.SpkmcError) as e:
            sp._check(sp.lib().spkmc_run_recorded(lat.h, 2, 2, None))
        assert e.value.code == sp.SPKMC_EINVAL
        with pytest.raises(ValueError):
            lat.run_recorded(2, 5, rec)  # more records than the buffer holds
        # nothing ran
        assert lat.observables().cycle == 0
        # a larger run after a smaller one grows the device buffers
        lat.run_recorded(1, 2, rec)
        big = sp.obs_buffer(40)
        lat.run_recorded(2, 40, big)
        lat.synchronize()
        assert [big[i].cycle for i in (0, 39)] == [4, 82]


def test_batch_records_equal_solo_read_outs():
    """A batch of uneven lattices (edges, bounds, colours, one budget ending
    within the run) recorded in one launch: each record equals the read-out
    of the same lattice run alone to that cycle (or to its last cycle)."""
    every, nrec = 5, 4
    specs = [
        (wl.LatticeSpec(L=32, d=4, seed=51), sp.SPKMC_RMAX_EXACT, sp.SPKMC_SUBLATTICE_8_ROTATING, -1),
        (wl.LatticeSpec(L=64, d=16, seed=52, H=0.02), sp.SPKMC_RMAX_LEARNED, sp.SPKMC_SUBLATTICE_8_ROTATING, -1),
        (wl.LatticeSpec(L=16, d=2, seed=53, T=3.0), sp.SPKMC_RMAX_PRESCRIBED, sp.SPKMC_SUBLATTICE_8_ROTATING, 13),
        (wl.LatticeSpec(L=48, d=8, seed=54), sp.SPKMC_RMAX_EXACT, sp.SPKMC_SUBLATTICE_2_RANDOM, 10),
    ]
    b = sp.Batch(len(specs))
    try:
        slots = [b.admit(s.L, s.d, s.J, s.H, s.T, s.seed, cold=s.cold, cycles=budget, rmax_mode=mode,
                         sublattice=sub) for s, mode, sub, budget in specs]
        b.run(3)  # records start after a few cycles (t = 3, an odd cycle)
        rec = b.run_recorded(every, nrec)
        b.synchronize()
        for slot, (s, mode, sub, budget) in zip(slots, specs):
            part = every * nrec if budget < 0 else min(budget - 3, every * nrec)
            with gpu_lattice(s, mode, sub) as a:
                a.run(3)
                done = 0
                for r in range(nrec):
                    upto = min((r + 1) * every, part)
                    if upto > done:
                        a.run(upto - done)
                        done = upto
                    assert_equal_obs(rec[slot * nrec + r], a.observables())
                assert np.array_equal(b.spins(slot), a.spins())
    finally:
        b.close()
