"""GPU parity at the full sizes of the 1024^3 and 128^3 workloads, in the
launch configuration the benchmark times: all cycles of each run as one
persistent recorded launch (observables recorded on the device every few
cycles), every record compared with the oracle stepped to the same cycle,
then the final spins and the class counts.

The oracle runs on all host cores (OpenMP over the active domains, Sec. 3.1
steps 1-6 with the 8-colour rotation of Sec. 3.2 step 4a); its trajectory
does not depend on the thread count.  Spins, M, B, the event and flip
counters and the fixed-point null-rate sum must be bit-identical; the clock
agrees to 1e-12 relative (CUDA log against libm log)."""
import os

import numpy as np
import pytest

import oracle
import paper_1005_4713_gb300 as sp
from paper_1005_4713_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

CLOCK_RTOL = 1e-12
THREADS = max(1, os.cpu_count() or 1)


def compare_records(rec, nrec, every, st):
    for r in range(nrec):
        st.run(every, threads=THREADS)
        o = rec[r]
        assert o.cycle == st.cycle, (r, o.cycle, st.cycle)
        assert (o.n_flip, o.n_null) == (st.n_flip, st.n_null), r
        assert int(o.sum_null_rate_fx[0]) | (int(o.sum_null_rate_fx[1]) << 64) == st.null_fx, r
        assert (o.M, o.B) == st.observables(), r
        assert o.clock == pytest.approx(st.clock, rel=CLOCK_RTOL, abs=0.0), r


def test_config_1024_all_500_cycles_in_one_recorded_launch():
    """1024^3, 16^3-site domains, hot start seed 3: 500 cycles in one launch
    with the observables every 10 cycles (50 records), as the benchmark runs
    its timed steps; each record, the final spins and the device's own
    recheck of counts, ghost faces, M and B."""
    spec = wl.CONFIG_1024
    every, nrec = wl.OBS_EVERY_1024, wl.CYCLES_1024 // wl.OBS_EVERY_1024
    rec = sp.obs_buffer(nrec)
    with sp.Lattice(spec.L, spec.d, spec.J, spec.H, spec.T, spec.seed) as lat:
        lat.run_recorded(every, nrec, rec)
        lat.synchronize()
        st = oracle.State(spec.L, spec.d, spec.J, spec.H, spec.T, spec.seed)
        compare_records(rec, nrec, every, st)
        assert st.cycle == 500 and st.n_flip + st.n_null == 500 * st.k_act
        assert np.array_equal(lat.spins(), st.spins)
        assert lat.check_counts() == 0


@pytest.mark.parametrize("spec", [wl.CONFIG_128_COLD, wl.CONFIG_128_HOT], ids=["cold", "hot"])
def test_config_128_all_16000_cycles_in_one_recorded_launch(spec):
    """128^3, 8^3-site domains, cold and hot start seed 2: the whole run of
    16 000 cycles (2000 visits of each colour) in one launch with the series
    every 100 cycles (160 records); each record, the final spins and class
    counts against the oracle."""
    every, nrec = 100, wl.CYCLES_128 // 100
    rec = sp.obs_buffer(nrec)
    with sp.Lattice(spec.L, spec.d, spec.J, spec.H, spec.T, spec.seed, cold=spec.cold) as lat:
        lat.run_recorded(every, nrec, rec)
        lat.synchronize()
        st = oracle.State(spec.L, spec.d, spec.J, spec.H, spec.T, spec.seed, cold=spec.cold)
        compare_records(rec, nrec, every, st)
        assert st.cycle == wl.CYCLES_128
        assert np.array_equal(lat.spins(), st.spins)
        assert np.array_equal(lat.class_counts(), oracle.class_counts(spec.L, spec.d, st.spins))
        assert lat.check_counts() == 0


def mem_available_gib() -> float:
    with open("/proc/meminfo") as f:
        for line in f:
            if line.startswith("MemAvailable:"):
                return int(line.split()[1]) / 2**20
    return 0.0


def test_2048_cube_beyond_32_bit_site_indices():
    """2048^3 (8.6e9 sites, past 32-bit site indices), 16^3-site domains,
    hot start seed 5: 262 144 active domains per cycle, so each CTA holds
    several hundred and stages them in rounds, its frequency lines going
    through the scratch lines.  One visit of each colour (8 cycles) in one
    recorded launch, records every 2 cycles against the oracle, then the
    spins bit for bit (one bit per site, compared in slabs) and the device's
    own recheck of counts, ghost faces, M and B."""
    if mem_available_gib() < 48:
        pytest.skip("the oracle's 2048^3 lattice needs about 10 GB of host memory; less than 48 GB is free")
    L, d, seed = 2048, 16, 5
    every, nrec = 2, 4
    rec = sp.obs_buffer(nrec)
    with sp.Lattice(L, d, 1.0, 0.0, 4.5115, seed) as lat:
        lat.run_recorded(every, nrec, rec)
        lat.synchronize()
        info = lat.info()  # the grid is sized at the first launch
        assert info.K_act == (L // d // 2) ** 3 and info.grid_ctas > 0
        assert -(-info.K_act // info.grid_ctas) > 256  # more than one staging round per CTA
        st = oracle.State(L, d, 1.0, 0.0, 4.5115, seed)
        compare_records(rec, nrec, every, st)
        assert st.n_flip + st.n_null == 8 * info.K_act
        bits = lat.spins_packed()
        flat = st.spins.reshape(-1)
        step = 1 << 27  # sites per slab, a multiple of 8
        for i in range(0, flat.size, step):
            want = np.packbits(flat[i:i + step] > 0, bitorder="little")
            assert np.array_equal(bits[i // 8:i // 8 + want.size], want), i
        assert lat.check_counts() == 0
