"""GPU parity: the CUDA path through the C ABI against the CPU oracle, element
by element, on the same seeded inputs.  Spins, event logs, counters and the
exact null-rate sum must be bit-identical; the clock (the only value that goes
through a transcendental function on the device) must agree to 1e-12
relative, the tolerance stated for the clock."""
import ctypes
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


def oracle_state(spec, **kw):
    return oracle.State(spec.L, spec.d, spec.J, spec.H, spec.T, spec.seed, cold=spec.cold, **kw)


def gpu_lattice(spec, log=0, config=None):
    return sp.Lattice(spec.L, spec.d, spec.J, spec.H, spec.T, spec.seed, cold=spec.cold,
                      event_log_capacity=log, config=config)


def same_clock(a, b):
    if math.isinf(a) or math.isinf(b):
        return a == b
    return a == pytest.approx(b, rel=CLOCK_RTOL, abs=0.0)


def assert_same(lat, st, spins=True):
    o = lat.observables()
    assert o.cycle == st.cycle
    assert (o.n_flip, o.n_null) == (st.n_flip, st.n_null)
    assert int(o.sum_null_rate_fx[0]) | (int(o.sum_null_rate_fx[1]) << 64) == st.null_fx
    assert same_clock(o.clock, st.clock), (o.clock, st.clock)
    if spins:
        s = lat.spins()
        assert np.array_equal(s, st.spins), int(np.sum(s != st.spins))
        assert (o.M, o.B) == st.observables()


def log_as_array(ev):
    return np.stack([ev["domain"], ev["cls"], ev["site"]], axis=-1).astype(np.int32)


@pytest.mark.parametrize("spec", [
    wl.LatticeSpec(L=16, d=4, seed=1), wl.LatticeSpec(L=16, d=4, seed=1, cold=True),
    wl.LatticeSpec(L=32, d=2, seed=7), wl.LatticeSpec(L=64, d=8, seed=9),
    wl.LatticeSpec(L=96, d=16, seed=11), wl.LatticeSpec(L=24, d=4, seed=5),
])
def test_initial_state_and_counts_match_oracle(spec):
    with gpu_lattice(spec) as lat:
        st = oracle_state(spec)
        assert np.array_equal(lat.spins(), st.spins)
        assert np.array_equal(lat.class_counts(), oracle.class_counts(spec.L, spec.d, st.spins))
        o = lat.observables()
        assert (o.M, o.B) == st.observables()
        assert lat.check_counts() == 0


def test_config_16_ten_thousand_cycles_with_event_log():
    """16^3, 4^3-site domains, hot start seed 1: 10^4 cycles, spins, clock and
    counters compared every 100 cycles, the whole event log compared."""
    spec = wl.CONFIG_16
    st = oracle_state(spec)
    kact = st.k_act
    with gpu_lattice(spec, log=wl.CYCLES_16 * kact) as lat:
        logs = []
        for _ in range(wl.CYCLES_16 // 100):
            lat.run(100)
            logs.append(st.run(100, log=True))
            assert_same(lat, st)
        ev = lat.event_log()
        assert len(ev) == wl.CYCLES_16 * kact
        ref = np.concatenate(logs).reshape(-1, 3)
        assert np.array_equal(log_as_array(ev), ref)
        assert np.array_equal(ev["cycle"], np.repeat(np.arange(wl.CYCLES_16), kact))
        assert lat.check_counts() == 0


@pytest.mark.parametrize("spec", [wl.CONFIG_128_COLD, wl.CONFIG_128_HOT])
def test_config_128_against_oracle(spec):
    """128^3, 8^3-site domains, cold and hot start: 800 cycles (100 visits per
    colour) compared every 100 cycles, event log of the first 200 cycles."""
    st = oracle_state(spec)
    with gpu_lattice(spec, log=200 * st.k_act) as lat:
        ref_log = []
        for i in range(8):
            lat.run(100)
            ev = st.run(100, log=i < 2, threads=THREADS)
            if ev is not None:
                ref_log.append(ev)
            assert_same(lat, st)
        assert np.array_equal(log_as_array(lat.event_log()), np.concatenate(ref_log).reshape(-1, 3))
        assert np.array_equal(lat.class_counts(), oracle.class_counts(spec.L, spec.d, st.spins))


def test_config_1024_first_eight_cycles():
    """1024^3 with 16^3-site domains (32768 events per cycle) in the launch
    configuration the benchmark times (one recorded launch, records every few
    cycles): one visit of every colour, the records and the final state
    compared in full with the oracle."""
    spec = wl.CONFIG_1024
    st = oracle_state(spec)
    rec = sp.obs_buffer(2)
    with gpu_lattice(spec) as lat:
        lat.run_recorded(4, 2, rec)
        lat.synchronize()
        for r in range(2):
            st.run(4, threads=THREADS)
            o = rec[r]
            assert o.cycle == st.cycle
            assert (o.n_flip, o.n_null) == (st.n_flip, st.n_null)
            assert (o.M, o.B) == st.observables()
            assert int(o.sum_null_rate_fx[0]) | (int(o.sum_null_rate_fx[1]) << 64) == st.null_fx
            assert o.clock == pytest.approx(st.clock, rel=CLOCK_RTOL, abs=0.0)
        assert_same(lat, st)
        o = lat.observables()
        assert o.n_flip + o.n_null == 8 * st.k_act


@pytest.mark.parametrize("spec", [
    wl.LatticeSpec(L=4, d=2, seed=3),                    # nd = 2: both x neighbours are one domain
    wl.LatticeSpec(L=8, d=4, seed=4, H=0.3),
    wl.LatticeSpec(L=16, d=8, seed=5, J=-0.7, H=0.1, T=2.0),
    wl.LatticeSpec(L=32, d=16, seed=6, cold=True),
    wl.LatticeSpec(L=64, d=16, seed=7, T=3.0),
    wl.LatticeSpec(L=24, d=4, seed=8, H=0.01, T=4.45),  # nd = 6
    wl.LatticeSpec(L=40, d=2, seed=9, T=6.0),           # nd = 20
    wl.LatticeSpec(L=48, d=8, seed=10, T=1.5, H=-0.2),
])
def test_geometries_and_fields(spec):
    st = oracle_state(spec)
    n = 64
    with gpu_lattice(spec, log=n * st.k_act) as lat:
        lat.run(n)
        ev = st.run(n, log=True, threads=THREADS)
        assert_same(lat, st)
        assert np.array_equal(log_as_array(lat.event_log()), ev.reshape(-1, 3))
        assert lat.check_counts() == 0


def test_frozen_lattice_has_infinite_clock_and_only_nulls():
    """Cold start at T -> 0: every rate underflows to 0, so R_max = 0, every
    event is null and dt = -ln(xi)/0 = +inf (the degenerate case of step 5)."""
    spec = wl.LatticeSpec(L=16, d=4, T=0.01, cold=True)
    st = oracle_state(spec)
    with gpu_lattice(spec) as lat:
        lat.run(3)
        st.run(3)
        o = lat.observables()
        assert o.n_flip == 0 and o.n_null == 3 * st.k_act
        assert math.isinf(o.clock) and math.isinf(st.clock)
        assert_same(lat, st)


def test_zero_cycles_is_a_noop():
    spec = wl.CONFIG_16
    with gpu_lattice(spec) as lat:
        s0 = lat.spins()
        lat.run(0)
        o = lat.observables()
        assert o.cycle == 0 and o.clock == 0.0
        assert np.array_equal(lat.spins(), s0)


def test_event_log_capacity_truncates():
    spec = wl.CONFIG_16
    st = oracle_state(spec)
    with gpu_lattice(spec, log=20) as lat:
        lat.run(10)
        ev = lat.event_log()
        assert len(ev) == 20
        ref = st.run(10, log=True).reshape(-1, 3)[:20]
        assert np.array_equal(log_as_array(ev), ref)


def test_chunked_runs_equal_one_run():
    spec = wl.LatticeSpec(L=32, d=4, seed=21)
    with gpu_lattice(spec) as a, gpu_lattice(spec) as b:
        a.run(5)
        a.run(7)
        a.run(1)
        b.run(13)
        assert np.array_equal(a.spins(), b.spins())
        oa, ob = a.observables(), b.observables()
        assert (oa.clock, oa.n_flip, oa.n_null) == (ob.clock, ob.n_flip, ob.n_null)


@pytest.mark.parametrize("kw", [dict(max_ctas=1), dict(items_per_cta=1), dict(items_per_cta=7),
                                dict(items_per_cta=1000), dict(ctas_per_sm=1)])
def test_launch_geometry_does_not_change_the_trajectory(kw):
    spec = wl.LatticeSpec(L=64, d=4, seed=22)
    st = oracle_state(spec)
    st.run(40, threads=THREADS)
    with gpu_lattice(spec, config=sp.make_config(**kw)) as lat:
        lat.run(40)
        assert_same(lat, st)


@pytest.mark.parametrize("kw", [dict(items_per_cta=1000), dict(items_per_cta=300), dict(max_ctas=2)])
def test_multi_round_ctas_in_a_grid(kw):
    """More active domains per CTA than one staging round holds, in a grid of
    several CTAs (each CTA stages, ranks and flips its domains in rounds,
    between grid barriers): 64^3 with 2^3-site domains, 4096 per cycle."""
    spec = wl.LatticeSpec(L=64, d=2, seed=31)
    st = oracle_state(spec)
    st.run(40, threads=THREADS)
    with gpu_lattice(spec, config=sp.make_config(**kw)) as lat:
        lat.run(40)
        assert lat.info().grid_ctas > 1
        assert_same(lat, st)
        assert lat.check_counts() == 0


def test_checkpoint_resume_is_bit_exact():
    spec = wl.LatticeSpec(L=64, d=8, seed=23)
    with gpu_lattice(spec) as a:
        a.run(30)
        state, spins = a.state(), a.spins()
        a.run(30)
        with gpu_lattice(wl.LatticeSpec(L=64, d=8, seed=23, cold=True)) as b:
            b.set_spins(spins)
            b.set_state(state)
            assert b.check_counts() == 0
            b.run(30)
            assert np.array_equal(a.spins(), b.spins())
            oa, ob = a.observables(), b.observables()
            assert (oa.cycle, oa.clock, oa.n_flip, oa.n_null) == (ob.cycle, ob.clock, ob.n_flip, ob.n_null)
            assert list(oa.sum_null_rate_fx) == list(ob.sum_null_rate_fx)


def test_set_spins_roundtrip_and_recount():
    spec = wl.LatticeSpec(L=32, d=8, seed=24)
    rng = np.random.default_rng(0)
    s = rng.choice(np.array([-1, 1], dtype=np.int8), size=32 ** 3)
    with gpu_lattice(spec) as lat:
        lat.set_spins(s)
        assert np.array_equal(lat.spins(), s)
        assert np.array_equal(lat.class_counts(), oracle.class_counts(32, 8, s))


def test_torch_stream_and_caching_allocator():
    torch = pytest.importorskip("torch")
    spec = wl.LatticeSpec(L=32, d=4, seed=25)
    st = oracle_state(spec)
    st.run(16)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        cfg = sp.torch_config(caching_allocator=True)
        with gpu_lattice(spec, config=cfg) as lat:
            lat.run(16)
            assert_same(lat, st)


def test_barrier_timeout_is_reported_and_the_context_survives():
    """Fault test without a GPU fault: one CTA never arrives at the grid
    barrier, the others give up after 50 ms, the host reads ETIMEOUT, and a
    fresh lattice on the same context still runs correctly."""
    spec = wl.LatticeSpec(L=64, d=4, seed=26)
    cfg = sp.make_config(barrier_timeout_ns=50_000_000, debug_skip_arrival_cta=0, items_per_cta=64)
    lat = gpu_lattice(spec, config=cfg)
    lat.run(2)
    with pytest.raises(sp.SpkmcError) as e:
        lat.synchronize()
    assert e.value.code == sp.SPKMC_ETIMEOUT
    with pytest.raises(sp.SpkmcError):
        lat.run(1)
    lat.close()
    st = oracle_state(spec)
    st.run(4)
    with gpu_lattice(spec) as ok:
        ok.run(4)
        assert_same(ok, st)


def test_asynchronous_observables_equal_the_synchronous_ones():
    """Observables enqueued after each chunk without waiting equal, bit for
    bit, those read synchronously at the same points of another run."""
    spec = wl.LatticeSpec(L=64, d=8, seed=26, H=0.01)
    buf = sp.obs_buffer(5)
    with gpu_lattice(spec) as a, gpu_lattice(spec) as b:
        ref = []
        for i in range(5):
            a.run(7 + i)
            a.observables_async(buf[i])
            b.run(7 + i)
            ref.append(b.observables())
        a.synchronize()
        for i in range(5):
            x, y = buf[i], ref[i]
            for f in ("cycle", "clock", "M", "B", "E", "m", "m2", "m4", "n_flip", "n_null", "sum_null_rate",
                      "L", "domain_edge"):
                assert getattr(x, f) == getattr(y, f), f
            assert list(x.sum_null_rate_fx) == list(y.sum_null_rate_fx)


def test_graph_replay_equals_plain_runs():
    """Two replays of a captured graph of 4 steps x 7 cycles with observables
    equal 8 plain steps, spins and observables bit for bit."""
    spec = wl.LatticeSpec(L=64, d=8, seed=27)
    rec = sp.obs_buffer(4)
    with gpu_lattice(spec) as a, gpu_lattice(spec) as b:
        with a.graph(7, 4, rec) as g:
            ref = []
            for rep in range(2):
                g.launch()
                for i in range(4):
                    b.run(7)
                    ref.append(b.observables())
                a.synchronize()
                for i in range(4):
                    x, y = rec[i], ref[4 * rep + i]
                    assert (x.cycle, x.clock, x.M, x.B, x.n_flip, x.n_null) == \
                           (y.cycle, y.clock, y.M, y.B, y.n_flip, y.n_null)
            assert a.observables().cycle == 56
            assert np.array_equal(a.spins(), b.spins())
            a.run(3)  # plain runs continue from the replayed state
            b.run(3)
            assert np.array_equal(a.spins(), b.spins())


def test_graph_arguments_are_checked():
    spec = wl.LatticeSpec(L=32, d=4, seed=28)
    with gpu_lattice(spec) as lat:
        for args in [(7, 3), (0, 4), (4, 0)]:
            with pytest.raises(sp.SpkmcError) as e:
                lat.graph(*args)
            assert e.value.code == sp.SPKMC_EINVAL
        pageable = (sp.spkmc_obs * 2)()
        with pytest.raises(sp.SpkmcError) as e:
            sp.spkmc_graph_create(lat.h, 2, 2, ctypes.addressof(pageable))
        assert e.value.code == sp.SPKMC_EINVAL


def test_graph_whose_lattice_was_destroyed_is_refused():
    """Destroying a lattice first releases the replay of the graphs captured
    on it: launching such a graph is refused (SPKMC_EINVAL) before any device
    work, its handle can still be freed, and a new lattice and graph run as
    before (and as the oracle)."""
    spec = wl.LatticeSpec(L=32, d=8, seed=41)
    lat = gpu_lattice(spec)
    g = lat.graph(2, 2)
    g.launch()
    lat.synchronize()
    lat.close()
    with pytest.raises(sp.SpkmcError) as e:
        g.launch()
    assert e.value.code == sp.SPKMC_EINVAL
    assert "destroyed" in sp.spkmc_last_error()
    g.close()
    with gpu_lattice(spec) as lat2, lat2.graph(2, 2) as g2:
        g2.launch()
        g2.launch()
        lat2.synchronize()
        st = oracle_state(spec)
        st.run(8)
        assert_same(lat2, st)


@pytest.mark.parametrize("L,d", [
    (80, 2),    # nd = 40: a full and a partial tile of domains along x, byte lines
    (160, 4),   # word lines (L % 32 == 0)
    (288, 8),
    (544, 16),  # nd = 34: the second tile two domains wide
    (64, 2),    # nd = 32: one full tile
    (640, 16),  # 16-byte lines (L % 128 == 0), the second tile 8 domains wide
    (384, 4),   # 16-byte lines, three full tiles
    (256, 2),   # L % 128 == 0 but 8-byte segments: word lines
])
@pytest.mark.parametrize("pinned", [False, True])
def test_packed_spins_tiles(L, d, pinned):
    """Packed spins written and read back through tiles of up to 32 domains
    along x, from pageable buffers (staged through device memory) and from
    page-locked ones (read and written by the kernels in place): random bytes
    come back unchanged, the int8 read-out is their little-endian bits, and
    M and B of Eq. 1 / Eq. 4, refreshed on writing, equal the sums over the
    lattice."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(L + d)
    bits = rng.integers(0, 256, size=L ** 3 // 8, dtype=np.uint8)
    src, out = bits, np.empty_like(bits)
    if pinned:
        src = torch.empty(bits.size, dtype=torch.uint8, pin_memory=True).numpy()
        src[:] = bits
        out = torch.empty(bits.size, dtype=torch.uint8, pin_memory=True).numpy()
    with gpu_lattice(wl.LatticeSpec(L=L, d=d, seed=66)) as a:
        a.set_spins_packed(src)
        assert np.array_equal(a.spins_packed(out), bits)
        s = np.unpackbits(bits, bitorder="little").astype(np.int8) * 2 - 1
        assert np.array_equal(a.spins(), s)
        s = s.reshape(L, L, L)  # [Z, Y, X]
        B = sum(int(np.sum(s * np.roll(s, -1, axis=ax), dtype=np.int64)) for ax in range(3))
        o = a.observables()
        assert (o.M, o.B) == (int(np.sum(s, dtype=np.int64)), B)
        assert a.check_counts() == 0


def test_transfers_at_the_benchmark_size():
    """1024^3, d = 16, through page-locked buffers read and written in place:
    random packed spins come back unchanged, packed and as int8; the refresh
    that follows the write leaves counts, ghost faces and M, B as the
    device's independent recount finds them, and M is 2 (ones) - L^3."""
    torch = pytest.importorskip("torch")
    L = 1024
    n = L ** 3
    rng = np.random.default_rng(1024)
    bits = torch.empty(n // 8, dtype=torch.uint8, pin_memory=True).numpy()
    bits[:] = rng.integers(0, 256, size=n // 8, dtype=np.uint8)
    out = torch.empty(n // 8, dtype=torch.uint8, pin_memory=True).numpy()
    s8 = torch.empty(n, dtype=torch.int8, pin_memory=True).numpy()
    with gpu_lattice(wl.LatticeSpec(L=L, d=16, seed=68, cold=True)) as a:
        a.set_spins_packed(bits)
        assert a.check_counts() == 0
        ones = int(np.unpackbits(bits).sum(dtype=np.int64))
        assert a.observables().M == 2 * ones - n
        a.spins_packed(out)
        assert np.array_equal(out, bits)
        sp.spkmc_get_spins(a.h, s8)
        assert np.array_equal(np.packbits(s8 > 0, bitorder="little"), bits)
        a.run(20)
        a.spins_packed(out)
        sp.spkmc_get_spins(a.h, s8)
        assert np.array_equal(np.packbits(s8 > 0, bitorder="little"), out)
        a.set_spins(s8)  # int8 in place: the same lattice again
        assert a.check_counts() == 0
        a.spins_packed(bits)
        assert np.array_equal(bits, out)


@pytest.mark.parametrize("L,d", [(80, 2), (12, 2), (160, 4), (288, 8), (544, 16), (96, 16)])
@pytest.mark.parametrize("buf", ["pageable", "pinned", "pinned_unaligned"])
def test_int8_spins_tiles(L, d, buf):
    """int8 spins written and read back through the same tiles: any byte
    value > 0 is +1 and any other -1; the read-out is +1 / -1.  Page-locked
    buffers are used in place (at d = 16, one that is not 16-byte aligned
    takes the per-row kernels)."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(L * d)
    raw = rng.integers(-128, 128, size=L ** 3, dtype=np.int16).astype(np.int8)
    want = np.where(raw > 0, 1, -1).astype(np.int8)
    if buf == "pageable":
        src, out = raw, np.empty_like(raw)
    else:
        off = 1 if buf == "pinned_unaligned" else 0
        src = torch.empty(L ** 3 + off, dtype=torch.int8, pin_memory=True).numpy()[off:]
        out = torch.empty(L ** 3 + off, dtype=torch.int8, pin_memory=True).numpy()[off:]
        src[:] = raw
    with gpu_lattice(wl.LatticeSpec(L=L, d=d, seed=67)) as a:
        a.set_spins(src)
        sp.spkmc_get_spins(a.h, out)
        assert np.array_equal(out, want)
        assert np.array_equal(a.spins_packed(), np.packbits(want > 0, bitorder="little"))
        s = want.reshape(L, L, L)
        B = sum(int(np.sum(s * np.roll(s, -1, axis=ax), dtype=np.int64)) for ax in range(3))
        o = a.observables()
        assert (o.M, o.B) == (int(np.sum(s, dtype=np.int64)), B)
        assert a.check_counts() == 0


@pytest.mark.parametrize("spec", [
    wl.LatticeSpec(L=4, d=2, seed=61),    # L^3 / 8 bytes cross x-lines
    wl.LatticeSpec(L=12, d=2, seed=62),   # L not a multiple of 8
    wl.LatticeSpec(L=24, d=4, seed=63),
    wl.LatticeSpec(L=48, d=8, seed=64),
    wl.LatticeSpec(L=96, d=16, seed=65),
])
def test_packed_spins_round_trip(spec):
    """One bit per site in global order, little-endian within a byte: the
    packed read-out equals np.packbits of the int8 one, and writing packed
    spins has the effect of writing the same spins as int8."""
    with gpu_lattice(spec) as a, gpu_lattice(spec) as b:
        a.run(13)
        s = a.spins()
        bits = a.spins_packed()
        assert bits.size == spec.L ** 3 // 8
        assert np.array_equal(bits, np.packbits(s > 0, bitorder="little"))
        rng = np.random.default_rng(spec.seed)
        new = np.where(rng.random(spec.L ** 3) < 0.3, 1, -1).astype(np.int8)
        a.set_spins_packed(np.packbits(new > 0, bitorder="little"))
        b.set_spins(new)
        assert np.array_equal(a.spins(), new)
        assert a.check_counts() == 0
        oa, ob = a.observables(), b.observables()
        assert (oa.M, oa.B) == (ob.M, ob.B)
        a.set_state(b.state())
        a.run(9)
        b.run(9)
        assert np.array_equal(a.spins(), b.spins())
        with pytest.raises(sp.SpkmcError):
            a.set_spins_packed(np.zeros(spec.L ** 3 // 8 + 1, dtype=np.uint8))
