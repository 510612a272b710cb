"""Batched ensembles: many lattices of uneven L, T and H in one persistent
launch; each one's trajectory must equal its solo run and the oracle."""
import os

import numpy as np
import pytest

import oracle
import paper_1005_4713_gb300 as sp
from paper_1005_4713_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def obs_tuple(o):
    return (o.cycle, o.clock, o.M, o.B, o.n_flip, o.n_null, o.sum_null_rate_fx[0], o.sum_null_rate_fx[1])


def test_batch_matches_solo_and_oracle():
    specs = [
        wl.LatticeSpec(L=16, d=4, seed=1),
        wl.LatticeSpec(L=24, d=4, seed=2, T=4.45, H=0.01),
        wl.LatticeSpec(L=32, d=8, seed=3, cold=True),
        wl.LatticeSpec(L=8, d=2, seed=4, T=3.0),
        wl.LatticeSpec(L=48, d=8, seed=5, T=4.6),
        wl.LatticeSpec(L=64, d=16, seed=6, H=0.01),
        wl.LatticeSpec(L=16, d=2, seed=7, J=-1.0, T=2.5),
    ]
    budgets = [50, 37, 50, 12, -1, 50, 29]
    n = 50
    with sp.Batch(len(specs)) as b:
        slots = [b.admit(s.L, s.d, s.J, s.H, s.T, s.seed, cold=s.cold, cycles=c,
                         event_log_capacity=n * (s.L // s.d // 2) ** 3)
                 for s, c in zip(specs, budgets)]
        b.run(20)
        b.run(30)
        done = sorted(b.poll())
        assert done == sorted(slots[i] for i, c in enumerate(budgets) if c >= 0)
        for s, c, slot in zip(specs, budgets, slots):
            ncyc = n if c < 0 else min(n, c)
            with sp.Lattice(s.L, s.d, s.J, s.H, s.T, s.seed, cold=s.cold) as solo:
                solo.run(ncyc)
                assert obs_tuple(b.observables(slot)) == obs_tuple(solo.observables())
                assert np.array_equal(b.spins(slot), solo.spins())
            st = oracle.State(s.L, s.d, s.J, s.H, s.T, s.seed, cold=s.cold)
            ev = st.run(ncyc, log=True)
            assert np.array_equal(b.spins(slot), st.spins)
            got = b.event_log(slot)
            assert np.array_equal(np.stack([got["domain"], got["cls"], got["site"]], -1), ev.reshape(-1, 3))


def test_admit_retire_readmit_keeps_results_independent():
    """Lattices admitted later (different grid cycles, reused slots) follow
    their own lattice-local cycle counters: identical to running alone."""
    a = wl.LatticeSpec(L=32, d=4, seed=31)
    c = wl.LatticeSpec(L=16, d=4, seed=32, T=4.4)
    with sp.Batch(2) as b:
        sa = b.admit(a.L, a.d, a.J, a.H, a.T, a.seed, cycles=10)
        b.run(3)
        sc = b.admit(c.L, c.d, c.J, c.H, c.T, c.seed, cycles=25)
        b.run(30)
        assert sorted(b.poll()) == sorted([sa, sc])
        ref_a = oracle.State(a.L, a.d, a.J, a.H, a.T, a.seed)
        ref_a.run(10)
        ref_c = oracle.State(c.L, c.d, c.J, c.H, c.T, c.seed)
        ref_c.run(25)
        assert np.array_equal(b.spins(sa), ref_a.spins)
        assert np.array_equal(b.spins(sc), ref_c.spins)
        b.retire(sa)
        s2 = b.admit(a.L, a.d, a.J, a.H, a.T, a.seed, cycles=10)
        b.run(10)
        assert np.array_equal(b.spins(s2), ref_a.spins)
        assert b.usage()[0] == 2


def test_batch_full_and_empty():
    with sp.Batch(1) as b:
        b.run(5)  # nothing admitted: a no-op
        b.admit(16, 4, cycles=3)
        with pytest.raises(sp.SpkmcError) as e:
            b.admit(16, 4, cycles=3)
        assert e.value.code == sp.SPKMC_EBUSY


def test_many_small_lattices_in_one_launch():
    specs = wl.ensemble_specs(40, seed=7)
    with sp.Batch(len(specs)) as b:
        slots = [b.admit(s.L, s.d, s.J, s.H, s.T, s.seed, cycles=24) for s in specs]
        b.run(24)
        for s, slot in zip(specs[:6], slots[:6]):
            st = oracle.State(s.L, s.d, s.J, s.H, s.T, s.seed)
            st.run(24)
            assert np.array_equal(b.spins(slot), st.spins)
            o = b.observables(slot)
            assert (o.n_flip, o.n_null) == (st.n_flip, st.n_null)


@pytest.mark.parametrize("kw", [dict(max_ctas=1), dict(items_per_cta=5)])
def test_mixed_edges_share_warps(kw):
    """Lattices of every edge in few CTAs: the four domains a warp searches
    together belong to lattices of different edges (the per-octet branch of
    the site search); each lattice still equals its oracle run."""
    specs = [wl.LatticeSpec(L=8, d=2, seed=71), wl.LatticeSpec(L=16, d=4, seed=72, T=4.0),
             wl.LatticeSpec(L=16, d=8, seed=73, H=0.1), wl.LatticeSpec(L=32, d=16, seed=74),
             wl.LatticeSpec(L=12, d=2, seed=75, T=3.0), wl.LatticeSpec(L=32, d=8, seed=76),
             wl.LatticeSpec(L=8, d=4, seed=77), wl.LatticeSpec(L=64, d=16, seed=78, cold=True)]
    n = 40
    with sp.Batch(len(specs), sp.make_config(**kw)) as b:
        slots = [b.admit(s.L, s.d, s.J, s.H, s.T, s.seed, cold=s.cold) for s in specs]
        b.run(n)
        for s, slot in zip(specs, slots):
            st = oracle.State(s.L, s.d, s.J, s.H, s.T, s.seed, cold=s.cold)
            st.run(n)
            o = b.observables(slot)
            assert (o.n_flip, o.n_null) == (st.n_flip, st.n_null)
            assert np.array_equal(b.spins(slot), st.spins)


def test_batch_of_multi_round_ctas():
    """One CTA per SM, so each CTA holds more domains than one staging round
    (a dozen uneven lattices with 2^3-site domains): every lattice equals its
    oracle run."""
    specs = [wl.LatticeSpec(L=s.L, d=2, T=s.T, H=s.H, seed=s.seed) for s in wl.ensemble_specs(12)]
    n = 40
    with sp.Batch(len(specs), sp.make_config(items_per_cta=64, ctas_per_sm=1)) as b:
        slots = [b.admit(s.L, s.d, s.J, s.H, s.T, s.seed) for s in specs]
        b.run(n)
        for s, slot in zip(specs, slots):
            st = oracle.State(s.L, s.d, s.J, s.H, s.T, s.seed)
            st.run(n, threads=min(16, os.cpu_count() or 1))
            o = b.observables(slot)
            assert (o.n_flip, o.n_null) == (st.n_flip, st.n_null), s
            assert np.array_equal(b.spins(slot), st.spins)
