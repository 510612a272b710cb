"""A seeded random sweep of small lattices against the oracle.

Each case draws the domain edge d, the number of domains per axis, the
coupling J, the field H, the temperature T, a cold or hot start, the rate R
the frequency lines are padded to (the exact R_max of Sec. 3.1 step 2, or the
prescribed or self-learned bound of Sec. 3.2 step 4b), the colour scheme
(eight rotating colours or two random ones, Sec. 3.2 step 4a) and the launch
geometry.  The run is split into launches of random length.  After each
launch the spins, M, B, the flip and null counters, the fixed-point null-rate
sum and the clock are compared with the oracle; at the end, the whole event
log and the device's recheck of its class counts and ghost faces.  A third
of the cases with several launches resume from a checkpoint in a new handle
after their first launch.  The same
random lattices also run together in batches (one persistent launch over
all of them), each checked against its own oracle run."""
import os

import numpy as np
import pytest

import oracle
import paper_1005_4713_gb300 as sp

pytestmark = pytest.mark.gpu

THREADS = max(1, min(16, os.cpu_count() or 1))
CLOCK_RTOL = 1e-12
NCASES = 160

MODES = {oracle.RMAX_EXACT: sp.SPKMC_RMAX_EXACT, oracle.RMAX_PRESCRIBED: sp.SPKMC_RMAX_PRESCRIBED,
         oracle.RMAX_LEARNED: sp.SPKMC_RMAX_LEARNED}
SCHEMES = {oracle.SUB_8_ROTATING: sp.SPKMC_SUBLATTICE_8_ROTATING, oracle.SUB_2_RANDOM: sp.SPKMC_SUBLATTICE_2_RANDOM}


def draw_case(i):
    rng = np.random.default_rng([1005, 4713, i])
    d = int(rng.choice([2, 4, 8, 16]))
    nd = int(rng.choice([2, 4, 6, 8] if d >= 8 else [2, 4, 6, 8, 10, 12, 16, 20]))
    J = float(rng.choice([1.0, -1.0, rng.uniform(-1.5, 1.5)]))
    H = 0.0 if rng.random() < 0.5 else float(rng.uniform(-0.5, 0.5))
    geometry = [{}, {"items_per_cta": int(rng.integers(1, 40))}, {"max_ctas": int(rng.integers(1, 5))},
                {"ctas_per_sm": 1}][int(rng.integers(0, 4))]
    scheme = int(rng.choice(list(SCHEMES), p=[0.7, 0.3]))
    # the learned bound rests on the eight-colour rotation (both sides reject
    # it with two random colours)
    modes = list(MODES) if scheme == oracle.SUB_8_ROTATING else [oracle.RMAX_EXACT, oracle.RMAX_PRESCRIBED]
    return dict(L=d * nd, d=d, J=J, H=H, T=float(rng.uniform(1.0, 8.0)), seed=int(rng.integers(1, 2**31)),
                cold=bool(rng.random() < 0.25), mode=int(rng.choice(modes)), scheme=scheme, geometry=geometry,
                chunks=[int(c) for c in rng.integers(1, 60, size=int(rng.integers(1, 4)))])


def log_as_array(ev):
    return np.stack([ev["domain"], ev["cls"], ev["site"]], axis=-1).astype(np.int32)


@pytest.mark.parametrize("i", range(NCASES))
def test_random_case_matches_oracle(i):
    c = draw_case(i)
    st = oracle.State(c["L"], c["d"], c["J"], c["H"], c["T"], c["seed"], cold=c["cold"], rmax_mode=c["mode"],
                      sublattice=c["scheme"])
    chunks = c["chunks"]
    # every third case with more than one launch moves to a new handle after
    # its first launch: a checkpoint (state and spins) restored into a lattice
    # created cold, whose event log restarts at the restored cycle
    parts = [chunks[:1], chunks[1:]] if len(chunks) > 1 and i % 3 == 0 else [chunks]
    state = spins = None
    for k, part in enumerate(parts):
        with sp.Lattice(c["L"], c["d"], c["J"], c["H"], c["T"], c["seed"], cold=c["cold"] or k > 0,
                        event_log_capacity=sum(part) * st.k_act, config=sp.make_config(**c["geometry"]),
                        rmax_mode=MODES[c["mode"]], sublattice=SCHEMES[c["scheme"]], tuned=False) as lat:
            if k > 0:
                lat.set_spins(spins)
                lat.set_state(state)
                assert lat.check_counts() == 0, c
            logs = []
            for n in part:
                lat.run(n)
                logs.append(st.run(n, log=True, threads=THREADS))
                o = lat.observables()
                assert o.cycle == st.cycle, c
                assert (o.n_flip, o.n_null) == (st.n_flip, st.n_null), c
                assert int(o.sum_null_rate_fx[0]) | (int(o.sum_null_rate_fx[1]) << 64) == st.null_fx, c
                assert o.clock == pytest.approx(st.clock, rel=CLOCK_RTOL, abs=0.0), c
                assert (o.M, o.B) == st.observables(), c
                assert np.array_equal(lat.spins(), st.spins), c
            ev = lat.event_log()
            assert len(ev) == sum(part) * st.k_act, c
            assert np.array_equal(ev["cycle"], np.repeat(np.arange(st.cycle - sum(part), st.cycle), st.k_act)), c
            assert np.array_equal(log_as_array(ev), np.concatenate(logs).reshape(-1, 3)), c
            assert lat.check_counts() == 0, c
            state, spins = lat.state(), lat.spins()

NBATCHES = 32


def k_act(c):
    nd = c["L"] // c["d"]
    return (nd // 2) ** 3 if c["scheme"] == oracle.SUB_8_ROTATING else nd ** 3 // 2


@pytest.mark.parametrize("i", range(NBATCHES))
def test_random_batch_matches_oracle(i):
    """2 to 12 random lattices (any mix of edges, modes and colour schemes) in
    one batch, some admitted after the first launch (so the batch runs
    lattices at different cycle parities), each with a random budget or
    none, over launches of random length; each lattice must end where its own
    oracle run of the same number of cycles does, event log included."""
    rng = np.random.default_rng([1005, 4713, 99, i])
    n = int(rng.integers(2, 13))
    cases = [draw_case(100000 + 64 * i + j) for j in range(n)]
    runs = [int(x) for x in rng.integers(1, 40, size=int(rng.integers(2, 4)))]
    late = [bool(rng.random() < 0.3) for _ in range(n)]
    budgets = [-1 if rng.random() < 0.3 else int(rng.integers(1, sum(runs) + 1)) for _ in range(n)]
    geometry = [{}, {"items_per_cta": int(rng.integers(1, 40))}, {"max_ctas": int(rng.integers(1, 5))}][
        int(rng.integers(0, 3))]
    slots, avail = [None] * n, [0] * n
    with sp.Batch(n, config=sp.make_config(**geometry)) as b:
        def admit(j):
            c = cases[j]
            slots[j] = b.admit(c["L"], c["d"], c["J"], c["H"], c["T"], c["seed"], cold=c["cold"], cycles=budgets[j],
                               event_log_capacity=sum(runs) * k_act(c), rmax_mode=MODES[c["mode"]],
                               sublattice=SCHEMES[c["scheme"]])

        for j in range(n):
            if not late[j]:
                admit(j)
        for r, cyc in enumerate(runs):
            b.run(cyc)
            for j in range(n):
                if slots[j] is not None:
                    avail[j] += cyc
            if r == 0:
                for j in range(n):
                    if late[j]:
                        admit(j)
        for j, c in enumerate(cases):
            ncyc = avail[j] if budgets[j] < 0 else min(budgets[j], avail[j])
            st = oracle.State(c["L"], c["d"], c["J"], c["H"], c["T"], c["seed"], cold=c["cold"],
                              rmax_mode=c["mode"], sublattice=c["scheme"])
            ev = st.run(ncyc, log=True, threads=THREADS)
            o = b.observables(slots[j])
            assert o.cycle == ncyc, (j, c)
            assert (o.n_flip, o.n_null) == (st.n_flip, st.n_null), (j, c)
            assert int(o.sum_null_rate_fx[0]) | (int(o.sum_null_rate_fx[1]) << 64) == st.null_fx, (j, c)
            assert o.clock == pytest.approx(st.clock, rel=CLOCK_RTOL, abs=0.0), (j, c)
            assert (o.M, o.B) == st.observables(), (j, c)
            assert np.array_equal(b.spins(slots[j]), st.spins), (j, c)
            assert np.array_equal(log_as_array(b.event_log(slots[j])), ev.reshape(-1, 3)), (j, c)
