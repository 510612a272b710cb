"""Pins for the CPU oracle (arXiv:1005.4713), checked against things other
than the oracle itself: numpy's Philox, closed forms, invariants, brute force
on tiny lattices with numpy, exact enumeration of the Boltzmann distribution,
and the numbers the paper prints.  No GPU needed."""
import itertools
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
M64 = (1 << 64) - 1


def paper_constant(name):
    with open(os.path.join(GOLDEN, "paper_constants.txt")) as f:
        for line in f:
            if line.startswith(name + " "):
                return float(line.split()[1])
    raise KeyError(name)


def numpy_philox(ctr, key):
    """Philox4x64-10 block for counter ``ctr`` via numpy, which advances its
    counter by one before producing a block, so it is seeded with ctr - 1."""
    v = (ctr[0] | ctr[1] << 64 | ctr[2] << 128 | ctr[3] << 192) - 1
    v %= 1 << 256
    cc = np.array([(v >> (64 * i)) & M64 for i in range(4)], dtype=np.uint64)
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=cc)
    return [int(x) for x in bg.random_raw(4)]


def numpy_classes(L, s):
    """class = 7*[sigma=+1] + number of up neighbours, by np.roll."""
    a = (s.reshape(L, L, L) > 0).astype(np.int64)
    u = sum(np.roll(a, sh, axis=ax) for ax in (0, 1, 2) for sh in (1, -1))
    return (7 * a + u).reshape(-1)


# --------------------------------------------------------------------------
# RNG (Sec. 3.1 step 4: independent parallel random streams)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("ctr,key", [
    ((0, 0, 0, 0), (1, 0)),
    ((7, 3, 1, 0), (1, 0)),
    ((12345, 0, 2, 0), (2, 0)),
    ((4095, 0, 3, 0), (3, 0)),
    ((2**63 + 5, 2**40, 1, 0), (2**64 - 1, 0)),
    ((1, 2, 3, 4), (5, 6)),
])
def test_philox_matches_numpy(ctr, key):
    assert [int(x) for x in oracle.philox(ctr, key)] == numpy_philox(ctr, key)


# --------------------------------------------------------------------------
# Rates (Eq. 3, read as Glauber dynamics)
# --------------------------------------------------------------------------
def test_rates_tanh_form():
    """Eq. 3 in its tanh form, (1/2)[1 - sigma tanh((J S + H)/T)], is the
    same function as the table's 1/(1 + exp(2 sigma (J S + H)/T))."""
    for J, H, T in [(1.0, 0.0, 4.5115), (1.0, 0.01, 4.4), (-0.5, 0.3, 2.0), (1.0, -0.2, 10.0)]:
        r = oracle.rates(J, H, T)
        for c in range(14):
            sigma = 1.0 if c >= 7 else -1.0
            S = 2 * (c % 7) - 6
            ref = 0.5 * (1.0 - sigma * math.tanh((J * S + H) / T))
            assert r[c] == pytest.approx(ref, rel=1e-13, abs=1e-300)


def test_rates_at_critical_point_values():
    """Flip rates of an up spin at T = 1/beta_c, beta_c printed in Sec. 2 and 6."""
    Tc = 1.0 / paper_constant("beta_c")
    r = oracle.rates(1.0, 0.0, Tc)
    up = r[7:]
    assert up[3] == 0.5  # S = 0: no field, the flip is as likely as not
    assert np.all(np.diff(up) < 0)  # more aligned neighbours, slower flips
    # r(+1, S=6) = 1/(1+exp(12 beta_c)), written through tanh
    assert up[6] == pytest.approx(0.5 * (1 - math.tanh(6 * 0.2216546)), rel=1e-12)


def test_rates_detailed_balance():
    """r(+1,S)/r(-1,S) = exp(-dE/T) with dE = 2(J S + H): the Boltzmann
    weight ratio of the two states (detailed balance of Eq. 2)."""
    for J, H, T in [(1.0, 0.0, 4.5115), (1.0, 0.01, 4.6), (-1.0, 0.5, 3.0)]:
        r = oracle.rates(J, H, T)
        for u in range(7):
            S = 2 * u - 6
            ratio = r[7 + u] / r[u]
            assert ratio == pytest.approx(math.exp(-2.0 * (J * S + H) / T), rel=1e-13)


def test_rates_glauber_identity():
    """r(+1,S) + r(-1,S) = lambda = 1 for every S and field."""
    for J, H, T in [(1.0, 0.0, 4.5115), (1.0, 0.01, 4.4), (2.0, -0.7, 1.3)]:
        r = oracle.rates(J, H, T)
        for u in range(7):
            assert abs(r[7 + u] + r[u] - 1.0) <= 2 * np.finfo(float).eps


def test_rates_infinite_temperature_and_no_coupling():
    assert np.all(oracle.rates(0.0, 0.0, 3.0) == 0.5)
    assert np.allclose(oracle.rates(1.0, 0.2, 1e12), 0.5, atol=1e-11)


# --------------------------------------------------------------------------
# Initial state and observables (Eq. 1, Eq. 4)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("L,seed", [(8, 1), (16, 3), (12, 77)])
def test_hot_start_bits_from_numpy_philox(L, seed):
    s = oracle.init_spins(L, seed)
    N = L ** 3
    exp = np.empty(N, dtype=np.int8)
    for blk in range((N + 255) // 256):
        w = numpy_philox((blk, 0, 3, 0), (seed, 0))
        for b in range(256):
            g = 256 * blk + b
            if g < N:
                exp[g] = 1 if (w[b // 64] >> (b % 64)) & 1 else -1
    assert np.array_equal(s, exp)


def test_cold_start_all_up():
    assert np.all(oracle.init_spins(8, 5, cold=True) == 1)


@pytest.mark.parametrize("L,seed", [(4, 1), (8, 2), (10, 9)])
def test_observables_bruteforce(L, seed):
    s = oracle.init_spins(L, seed)
    a = s.reshape(L, L, L).astype(np.int64)
    M = int(a.sum())
    B = int(sum((a * np.roll(a, -1, axis=ax)).sum() for ax in (0, 1, 2)))
    assert oracle.observables(L, s) == (M, B)


@pytest.mark.parametrize("L,d,seed", [(8, 2, 1), (8, 4, 2), (12, 3, 4), (16, 4, 5)])
def test_class_counts_bruteforce(L, d, seed):
    s = oracle.init_spins(L, seed)
    cls = numpy_classes(L, s)
    nd = L // d
    Z, Y, X = np.meshgrid(np.arange(L), np.arange(L), np.arange(L), indexing="ij")
    k = (X // d + nd * (Y // d + nd * (Z // d))).reshape(-1)
    exp = np.zeros((nd ** 3, 14), dtype=np.int64)
    np.add.at(exp, (k, cls), 1)
    assert np.array_equal(oracle.class_counts(L, d, s), exp)


# --------------------------------------------------------------------------
# One spkMC cycle by brute force on tiny lattices (Sec. 3.1 steps 1-6,
# Sec. 3.2 steps 4a/4b), independent Python + numpy code
# --------------------------------------------------------------------------
SLACK = 1.0 + 2.0 ** -32  # relative slack of the Sec. 3.2 bounds


def drift_margin(r):
    """Largest growth of a domain's R_k between two visits of its colour:
    the flipped site (sigma -> -sigma at fixed S) plus 12 sites whose S moves
    by 2 (its neighbours in the domain and one site per face neighbour)."""
    own = max(abs(r[7 + u] - r[u]) for u in range(7))
    step = max(abs(r[7 * sg + u + 1] - r[7 * sg + u]) for sg in (0, 1) for u in range(6))
    return own + 12 * step


def brute_bound(mode, d, r, prev8, Rmax):
    """The rate the lines are padded to: exact R_max (mode 0), the prescribed
    d^3 max_c r_c (mode 1), or the learned min(prescribed, R_max(t-8) +
    drift margin) (mode 2), both bounds times SLACK."""
    if mode == 0:
        return Rmax
    pres = (d ** 3 * max(r)) * SLACK
    if mode == 2 and prev8 > 0:
        return min(pres, (prev8 + drift_margin(r)) * SLACK)
    return pres


def brute_colour(sublattice, t, seed):
    """Sec. 3.2 step 4a: colour t mod 8 (rotation), or the top bit of a
    Philox draw (two random colours)."""
    if sublattice == 0:
        return t % 8
    return numpy_philox((t, 0, 5, 0), (seed, 0))[0] >> 63


def brute_colour_of(sublattice, dx, dy, dz):
    if sublattice == 0:
        return (dx & 1) | (dy & 1) << 1 | (dz & 1) << 2
    return (dx + dy + dz) & 1


def brute_cycles(L, d, J, H, T, seed, s, ncycles, clock=0.0, t0=0, null_sum=None, mode=0, hist=None,
                 sublattice=0):
    s = s.copy()
    hist = [0.0] * 8 if hist is None else hist
    r = [1.0 / (1.0 + math.exp(2.0 * (1 if c >= 7 else -1) * (J * (2 * (c % 7) - 6) + H) / T))
         for c in range(14)]
    nd = L // d
    log = []
    nflip = nnull = 0
    for t in range(t0, t0 + ncycles):
        cls = numpy_classes(L, s)
        col = brute_colour(sublattice, t, seed)
        active = []
        for k in range(nd ** 3):
            dx, dy, dz = k % nd, (k // nd) % nd, k // (nd * nd)
            if brute_colour_of(sublattice, dx, dy, dz) == col:
                active.append((k, dx, dy, dz))
        lines = []
        for k, dx, dy, dz in active:
            sites = []
            for l in range(d ** 3):
                x, y, z = l % d, (l // d) % d, l // (d * d)
                g = (dx * d + x) + L * ((dy * d + y) + L * (dz * d + z))
                sites.append((g, int(cls[g])))
            n = [0] * 14
            for _, c in sites:
                n[c] += 1
            cum, acc = [], 0.0
            for c in range(14):
                acc = acc + n[c] * r[c]
                cum.append(acc)
            lines.append((k, sites, n, cum))
        Rmax = max(cum[13] for _, _, _, cum in lines)
        Rpad = brute_bound(mode, d, r, hist[0], Rmax)
        assert Rpad >= Rmax
        hist[:] = hist[1:] + [Rmax]
        if null_sum is not None:
            null_sum.append(sum(int(math.ldexp(Rpad - cum[13], 64)) for _, _, _, cum in lines))
        flips = []
        for k, sites, n, cum in lines:
            w = numpy_philox((t, k, 1, 0), (seed, 0))
            target = (w[0] >> 11) * 2.0 ** -53 * Rpad
            chosen = next((c for c in range(14) if target < cum[c]), -1)
            if chosen < 0:
                log.append((k, -1, -1))
                nnull += 1
                continue
            j = (w[1] * n[chosen]) >> 64
            members = [l for l, (_, c) in enumerate(sites) if c == chosen]
            l = members[j]
            log.append((k, chosen, l))
            flips.append(sites[l][0])
            nflip += 1
        for g in flips:
            s[g] = -s[g]
        wc = numpy_philox((t, 0, 2, 0), (seed, 0))
        xi = (2 * (wc[0] >> 12) + 1) * 2.0 ** -53
        clock = clock + (-math.log(xi) / Rpad)
    return s, np.array(log, dtype=np.int32).reshape(ncycles, -1, 3), clock, nflip, nnull


@pytest.mark.parametrize("L,d,J,H,T,seed,cold", [
    (8, 2, 1.0, 0.0, 4.5115, 11, False),
    (8, 4, 1.0, 0.3, 3.0, 12, False),
    (12, 3, -0.7, 0.1, 2.5, 13, False),
    (8, 2, 1.0, 0.0, 4.5115, 14, True),
])
def test_cycles_bruteforce(L, d, J, H, T, seed, cold):
    st = oracle.State(L, d, J, H, T, seed, cold=cold)
    s0 = st.spins.copy()
    ev = st.run(17, log=True)
    s_ref, log_ref, clock_ref, nf, nn = brute_cycles(L, d, J, H, T, seed, s0, 17)
    assert np.array_equal(ev, log_ref)
    assert np.array_equal(st.spins, s_ref)
    assert st.clock == pytest.approx(clock_ref, rel=1e-15)
    assert (st.n_flip, st.n_null) == (nf, nn)


def test_cold_start_first_cycle_closed_form():
    """All +1 at H = 0: every site has class (sigma=+1, S=6), so R_k = d^3 r(+1,6)
    for every active domain, R_max = R_k (no nulls, Sec. 3.1 step 3 equality
    case), M drops by 2 per active domain, dt = -ln(xi_0)/R_max."""
    L, d, T = 16, 4, 4.5115
    st = oracle.State(L, d, 1.0, 0.0, T, 21, cold=True)
    ev = st.run(1, log=True)
    kact = (L // d // 2) ** 3
    assert np.all(ev[0, :, 1] == 13)
    assert st.n_null == 0 and st.n_flip == kact
    M, _ = st.observables()
    assert M == L ** 3 - 2 * kact
    r_up6 = 0.5 * (1.0 - math.tanh(6.0 / T))
    wc = numpy_philox((0, 0, 2, 0), (21, 0))
    xi = (2 * (wc[0] >> 12) + 1) * 2.0 ** -53
    assert st.clock == pytest.approx(-math.log(xi) / (d ** 3 * r_up6), rel=1e-13)


def test_first_clock_step_exactly():
    """Step 5 with the reading of xi (never 0 or 1): xi = (2 (w0 >> 12) + 1)
    2^-53 from the clock's own Philox word (numpy's generator).  From all +1
    at H = 0 only class 13 is populated, so R_max = d^3 r_13 exactly (d^3 a
    power of two, r_13 pinned by the closed form above), and the first clock
    step is -ln(xi) / R_max bit for bit (the same libm logarithm).  Eight
    seeds, so that some words have bit 11 clear: a xi built from w0 >> 11
    differs from the reading by 2^-53 there."""
    L, d, T = 16, 4, 4.5115
    r13 = oracle.rates(1.0, 0.0, T)[13]
    bit11_clear = 0
    for seed in range(21, 29):
        st = oracle.State(L, d, 1.0, 0.0, T, seed, cold=True)
        st.run(1)
        w0 = numpy_philox((0, 0, 2, 0), (seed, 0))[0]
        xi = (2 * (w0 >> 12) + 1) * 2.0 ** -53
        assert st.clock == -math.log(xi) / (d ** 3 * r13), seed
        bit11_clear += (w0 >> 11) & 1 == 0
    assert bit11_clear > 0


def test_no_coupling_uniform_flips_and_clock():
    """J = H = 0: all rates 1/2, R_k = d^3/2 everywhere, never a null event,
    the flipped site is uniform over the domain, E[clock] = 2 n / d^3."""
    from scipy import stats
    L, d, n = 8, 2, 4000
    st = oracle.State(L, d, 0.0, 0.0, 3.0, 31)
    ev = st.run(n, log=True)
    assert st.n_null == 0
    sites = ev[:, :, 2].reshape(-1)
    hist = np.bincount(sites, minlength=d ** 3)
    assert stats.chisquare(hist).pvalue > 1e-4
    mean, sd = 2.0 * n / d ** 3, math.sqrt(n) * 2.0 / d ** 3
    assert abs(st.clock - mean) < 5 * sd


@pytest.mark.parametrize("mode", [0, 1])
def test_one_cycle_law_chi2(mode):
    """Sec. 3.1 step 4: in each active domain the event i is chosen with
    probability r_i/R and the null event with (R - R_k)/R, where R is R_max
    (exact) or the prescribed bound d^3 max r of Sec. 3.2 step 4b."""
    from scipy import stats
    L, d, J, H, T = 8, 2, 1.0, 0.2, 3.0
    base = oracle.init_spins(L, 5)
    cls = numpy_classes(L, base)
    r = np.array([0.5 * (1 - (1 if c >= 7 else -1) * math.tanh((J * (2 * (c % 7) - 6) + H) / T))
                  for c in range(14)])
    nd = L // d
    active = [k for k in range(nd ** 3)
              if ((k % nd) & 1) | (((k // nd) % nd) & 1) << 1 | ((k // nd // nd) & 1) << 2 == 0]
    site_rates = []
    for k in active:
        dx, dy, dz = k % nd, (k // nd) % nd, k // (nd * nd)
        rr = []
        for l in range(d ** 3):
            x, y, z = l % d, (l // d) % d, l // (d * d)
            rr.append(r[cls[(dx * d + x) + L * ((dy * d + y) + L * (dz * d + z))]])
        site_rates.append(rr)
    Rk = np.array([sum(v) for v in site_rates])
    Rmax = Rk.max() if mode == 0 else d ** 3 * r.max()
    nseeds = 60000 if mode == 0 else 30000
    hist = np.zeros((len(active), d ** 3 + 1), dtype=np.int64)
    for seed in range(1, nseeds + 1):
        st = oracle.State(L, d, J, H, T, seed, spins=base, rmax_mode=mode)
        ev = st.run(1, log=True)[0]
        for a in range(len(active)):
            hist[a, ev[a, 2] if ev[a, 1] >= 0 else d ** 3] += 1
    for a in range(len(active)):
        p = np.array(site_rates[a] + [Rmax - Rk[a]]) / Rmax
        keep = p > 0
        exp = p[keep] * nseeds
        assert hist[a, ~keep].sum() == 0
        assert stats.chisquare(hist[a, keep], exp).pvalue > 1e-5


def test_threads_do_not_change_the_trajectory():
    a = oracle.State(32, 4, 1.0, 0.0, 4.5115, 41)
    b = oracle.State(32, 4, 1.0, 0.0, 4.5115, 41)
    ea = a.run(20, log=True, threads=1)
    eb = b.run(20, log=True, threads=4)
    assert np.array_equal(ea, eb) and np.array_equal(a.spins, b.spins)
    assert a.clock == b.clock and a.null_fx == b.null_fx


def test_null_rate_sum_matches_definition():
    """Eq. 10 numerator, sum_k r_0k with r_0k = R_max - R_k (step 3),
    accumulated as floor(r_0k 2^64) per domain and cycle."""
    L, d, J, H, T, seed = 8, 2, 1.0, 0.0, 4.5115, 51
    st = oracle.State(L, d, J, H, T, seed)
    s0 = st.spins.copy()
    st.run(5)
    sums = []
    brute_cycles(L, d, J, H, T, seed, s0, 5, null_sum=sums)
    assert st.null_fx == sum(sums)
    assert st.null_fx > 0


# --------------------------------------------------------------------------
# Bounds that replace the exact R_max (Sec. 3.2 step 4b)
# --------------------------------------------------------------------------
def test_prescribed_bound_closed_form():
    """R' = n_k lambda e^{-dE}/(1+e^{-dE}), dE = -2(6|J| + |H|)/T: at T_c and
    H = 0 the single-site factor is r(+1, S=-6) = 0.9346166754684477 (rate
    table pin above); elsewhere it is (1 + tanh((6|J|+|H|)/T))/2."""
    Rp, m = oracle.rmax_bounds(4, 1.0, 0.0, 4.5115)
    assert Rp == (64 * 0.9346166754684477) * SLACK
    # a = r(-1,6) - r(+1,6); b = r(+1,0) - r(+1,2) (the steepest step is at S = 0)
    assert m == pytest.approx((0.9346166754684477 - 0.06538332453155232)
                              + 12 * (0.5 - 0.29180719760737955), rel=1e-14)
    for J, H, T, d in [(1.0, 0.01, 4.5115, 16), (-0.7, 0.3, 2.5, 8), (0.0, -0.2, 1.0, 2),
                       (2.0, 0.0, 50.0, 4), (1.0, -0.5, 0.7, 8)]:
        Rp, m = oracle.rmax_bounds(d, J, H, T)
        x = (6 * abs(J) + abs(H)) / T
        top = 0.5 * (1 + math.tanh(x))
        assert Rp / SLACK == pytest.approx(d ** 3 * top, rel=1e-14)
        th = [math.tanh((J * (2 * u - 6) + H) / T) for u in range(7)]
        a = max(abs(v) for v in th)                       # |r(+1,S) - r(-1,S)| = |tanh|
        b = max(0.5 * abs(th[u + 1] - th[u]) for u in range(6))
        assert m == pytest.approx(a + 12 * b, rel=1e-12)
        # the largest Glauber rate is the formula's, bit for bit
        assert Rp == (d ** 3 * oracle.rates(J, H, T).max()) * SLACK


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("L,d,J,H,T,seed,cold", [
    (8, 2, 1.0, 0.0, 4.5115, 61, False),
    (8, 4, 1.0, 0.3, 3.0, 62, False),
    (12, 3, -0.7, 0.1, 2.5, 63, False),
    (8, 2, 1.0, 0.0, 4.5115, 64, True),
])
def test_bound_modes_bruteforce(mode, L, d, J, H, T, seed, cold):
    st = oracle.State(L, d, J, H, T, seed, cold=cold, rmax_mode=mode)
    s0 = st.spins.copy()
    ev = st.run(21, log=True)
    sums, hist = [], [0.0] * 8
    s_ref, log_ref, clock_ref, nf, nn = brute_cycles(L, d, J, H, T, seed, s0, 21, null_sum=sums,
                                                     mode=mode, hist=hist)
    assert np.array_equal(ev, log_ref)
    assert np.array_equal(st.spins, s_ref)
    assert st.clock == pytest.approx(clock_ref, rel=1e-15)
    assert (st.n_flip, st.n_null) == (nf, nn)
    assert st.null_fx == sum(sums)
    assert list(st.rmax_hist) == hist


def _rates_per_domain(L, d, spins, r):
    n = oracle.class_counts(L, d, spins)
    out = np.zeros(len(n))
    for k in range(len(n)):
        acc = 0.0
        for c in range(14):
            acc = acc + int(n[k, c]) * float(r[c])
        out[k] = acc
    return out


@pytest.mark.parametrize("L,d,J,H,T,seed,cold", [
    (8, 2, 1.0, 0.0, 4.5115, 71, False),
    (16, 4, 1.0, 0.2, 3.0, 72, False),
    (12, 2, -1.0, 0.0, 2.0, 73, True),
    (8, 2, 1.0, 0.0, 1.2, 74, False),
])
def test_rate_drift_over_one_rotation_is_bounded(L, d, J, H, T, seed, cold):
    """Over any 8 consecutive cycles a domain is active once and each of its
    face neighbours once, so R_k(t+8) - R_k(t) is at most the drift margin
    a + 12 b: the growth bound behind the learned R.  Checked on every
    domain, over windows that start at every phase of the rotation."""
    r = oracle.rates(J, H, T)
    m = drift_margin(list(r))
    st = oracle.State(L, d, J, H, T, seed, cold=cold)
    hist = [_rates_per_domain(L, d, st.spins, r)]
    worst = 0.0
    for _ in range(120):
        st.run(1)
        hist.append(_rates_per_domain(L, d, st.spins, r))
        if len(hist) > 8:
            worst = max(worst, np.abs(hist[-1] - hist[-9]).max() / m)
    assert worst <= 1 + 1e-12
    assert worst > 0.1  # the walk moved the rates


def test_rate_drift_bound_is_attained():
    """The margin a + 12 b is reached: in domain (0,0,0) of a 32^3 lattice
    with d = 8, an up spin i at (4,4,4) whose 6 neighbours each have two down
    neighbours (S = 2) flips (a), its neighbours step from S = 2 to S = 0
    (6 b), and the site across the middle of each face flips while the face
    site next to it has S = 2 (6 b)."""
    L, d, J, H, T = 32, 8, 1.0, 0.0, 4.5115
    r = oracle.rates(J, H, T)
    g = lambda x, y, z: x % L + L * ((y % L) + L * (z % L))
    s = np.ones(L ** 3, dtype=np.int8)
    down = [(5, 5, 4), (4, 5, 5), (5, 4, 5), (3, 3, 4), (4, 3, 3), (3, 4, 3)]
    faces = [((0, 4, 4), (-1, 4, 4), [(0, 3, 4), (0, 5, 4)]), ((7, 4, 4), (8, 4, 4), [(7, 3, 4), (7, 5, 4)]),
             ((4, 0, 4), (4, -1, 4), [(3, 0, 4), (5, 0, 4)]), ((4, 7, 4), (4, 8, 4), [(3, 7, 4), (5, 7, 4)]),
             ((4, 4, 0), (4, 4, -1), [(3, 4, 0), (5, 4, 0)]), ((4, 4, 7), (4, 4, 8), [(3, 4, 7), (5, 4, 7)])]
    for p in down:
        s[g(*p)] = -1
    for _, _, dn in faces:
        for p in dn:
            s[g(*p)] = -1
    before = _rates_per_domain(L, d, s, r)[0]
    s[g(4, 4, 4)] = -1
    for _, across, _ in faces:
        s[g(*across)] = -1
    after = _rates_per_domain(L, d, s, r)[0]
    _, margin = oracle.rmax_bounds(d, J, H, T)
    assert after - before == pytest.approx(margin, rel=1e-12)


def test_history_records_the_exact_rmax():
    L, d, J, H, T = 16, 4, 1.0, 0.1, 3.5
    st = oracle.State(L, d, J, H, T, 91)
    r = oracle.rates(J, H, T)
    nd = L // d
    seen = []
    for t in range(11):
        R = _rates_per_domain(L, d, st.spins, r)
        act = [k for k in range(nd ** 3)
               if ((k % nd) & 1) | (((k // nd) % nd) & 1) << 1 | ((k // nd // nd) & 1) << 2 == t % 8]
        seen.append(max(R[act]))
        st.run(1)
    assert list(st.rmax_hist) == seen[-8:]


def test_learned_equals_prescribed_until_a_colour_has_history():
    a = oracle.State(32, 4, 1.0, 0.0, 4.5115, 93, rmax_mode=oracle.RMAX_PRESCRIBED)
    b = oracle.State(32, 4, 1.0, 0.0, 4.5115, 93, rmax_mode=oracle.RMAX_LEARNED)
    assert np.array_equal(a.run(8, log=True), b.run(8, log=True))
    assert a.clock == b.clock and np.array_equal(a.spins, b.spins)
    ca, cb = a.clock, b.clock
    a.run(1)
    b.run(1)
    assert b.clock - cb > a.clock - ca  # same xi, smaller learned R


@pytest.mark.parametrize("L,d,T,H,cold", [
    (16, 2, 4.5115, 0.0, False), (16, 2, 3.0, 0.3, True), (16, 4, 8.0, 0.0, False),
    (16, 4, 1.0, 0.0, False), (16, 2, 0.6, -0.4, False), (32, 8, 4.5115, 0.01, True),
])
def test_learned_bound_holds_over_long_runs(L, d, T, H, cold):
    """The self-learned R never falls below an active domain's R_k (the run
    raises BoundExceeded otherwise), and it sits close to R_max: the null
    fraction is near that of the exact-R_max run."""
    st = oracle.State(L, d, 1.0, H, T, 81, cold=cold, rmax_mode=oracle.RMAX_LEARNED)
    ex = oracle.State(L, d, 1.0, H, T, 81, cold=cold)
    st.run(1200)
    ex.run(1200)
    ur_l = st.n_flip / (st.n_flip + st.n_null)
    ur_e = ex.n_flip / (ex.n_flip + ex.n_null)
    assert ur_l <= ur_e * 1.05
    if d == 8:
        assert ur_l > 0.85 * ur_e


def test_bound_exceeded_is_reported():
    """A recorded history that is too small for the lattice trips the check."""
    st = oracle.State(16, 4, 1.0, 0.0, 4.5115, 95, rmax_mode=oracle.RMAX_LEARNED)
    st.rmax_hist[:] = 1.0
    with pytest.raises(oracle.BoundExceeded):
        st.run(1)


# --------------------------------------------------------------------------
# The paper's two-colour sublattice, chosen at random each cycle (Sec. 3.2
# step 4a)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("L,d,J,H,T,seed,cold", [
    (8, 2, 1.0, 0.0, 4.5115, 101, False),
    (8, 4, 1.0, 0.3, 3.0, 102, False),
    (12, 3, -0.7, 0.1, 2.5, 103, False),
    (8, 2, 1.0, 0.0, 4.5115, 104, True),
])
def test_two_colour_bruteforce(mode, L, d, J, H, T, seed, cold):
    st = oracle.State(L, d, J, H, T, seed, cold=cold, rmax_mode=mode, sublattice=oracle.SUB_2_RANDOM)
    s0 = st.spins.copy()
    ev = st.run(19, log=True)
    assert ev.shape == (19, (L // d) ** 3 // 2, 3)
    sums = []
    s_ref, log_ref, clock_ref, nf, nn = brute_cycles(L, d, J, H, T, seed, s0, 19, null_sum=sums, mode=mode,
                                                     sublattice=1)
    assert np.array_equal(ev, log_ref)
    assert np.array_equal(st.spins, s_ref)
    assert st.clock == pytest.approx(clock_ref, rel=1e-15)
    assert (st.n_flip, st.n_null) == (nf, nn)
    assert st.null_fx == sum(sums)


def test_two_colour_draw_is_fair_and_not_alternating():
    """The cycle colours come from the log: half of the cycles on each colour
    (binomial, 5 sigma) and as many repeats as changes."""
    L, d, n = 8, 2, 20000
    st = oracle.State(L, d, 1.0, 0.0, 4.5115, 105, sublattice=oracle.SUB_2_RANDOM)
    ev = st.run(n, log=True)
    nd = L // d
    k = ev[:, 0, 0]
    col = ((k % nd) + (k // nd) % nd + k // (nd * nd)) & 1
    ones = int(col.sum())
    assert abs(ones - n / 2) < 5 * math.sqrt(n / 4)
    same = int(np.sum(col[1:] == col[:-1]))
    assert abs(same - (n - 1) / 2) < 5 * math.sqrt((n - 1) / 4)
    # every active domain of a cycle has that cycle's colour
    kk = ev[:, :, 0]
    c_all = ((kk % nd) + (kk // nd) % nd + kk // (nd * nd)) & 1
    assert np.all(c_all == col[:, None])


def test_two_colour_rejects_the_learned_bound():
    st = oracle.State(8, 2, 1.0, 0.0, 4.5115, 106, rmax_mode=oracle.RMAX_LEARNED, sublattice=oracle.SUB_2_RANDOM)
    with pytest.raises(ValueError):
        st.run(1)


# --------------------------------------------------------------------------
# Exact enumeration (Boltzmann) and serial BKL (the serial reference, Sec. 4)
# --------------------------------------------------------------------------
def test_enumeration_no_coupling_closed_forms():
    N = 18
    for H, T in [(0.0, 2.0), (0.4, 1.5)]:
        E, E2, m2, m4, am, m = oracle.enumerate_exact((3, 3, 2), 0.0, H, T)
        mu = math.tanh(H / T)
        assert m == pytest.approx(mu, abs=1e-12)
        assert E == pytest.approx(-H * N * mu, abs=1e-9)
        assert m2 == pytest.approx((N + N * (N - 1) * mu * mu) / N ** 2, rel=1e-12)
        if H == 0.0:
            assert m4 == pytest.approx((3 * N * N - 2 * N) / N ** 4, rel=1e-12)


def test_enumeration_bruteforce_2x2x2():
    J, H, T = 1.0, 0.1, 3.0
    states = np.array(list(itertools.product([-1, 1], repeat=8)), dtype=np.int64)
    a = states.reshape(-1, 2, 2, 2)  # (state, Z, Y, X)
    bonds = sum((a * np.roll(a, -1, axis=ax)).sum(axis=(1, 2, 3)) for ax in (1, 2, 3))
    M = a.sum(axis=(1, 2, 3))
    E = -J * bonds - H * M
    w = np.exp(-(E - E.min()) / T)
    w /= w.sum()
    m = M / 8.0
    ref = [np.dot(w, E), np.dot(w, E * E), np.dot(w, m ** 2), np.dot(w, m ** 4),
           np.dot(w, np.abs(m)), np.dot(w, m)]
    assert np.allclose(oracle.enumerate_exact((2, 2, 2), J, H, T), ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("T", [3.5, 4.5115, 6.0])
def test_serial_bkl_matches_exact_enumeration(T):
    """Time averages of the serial BKL chain with the Glauber table equal the
    Boltzmann averages of Eq. 1 on a 3x3x2 lattice (2^18 states)."""
    shape, J, H = (3, 3, 2), 1.0, 0.0
    exact = oracle.enumerate_exact(shape, J, H, T)
    s = oracle.init_spins(3, 0)[:18].copy()
    nb = 40
    sums = oracle.bkl_run(shape, J, H, T, 1000 + int(T * 10), s, 2_000_000, nb)
    w = sums[:, 0]
    for col, idx in [(1, 0), (3, 2), (4, 3)]:
        means = sums[:, col] / w
        mu = sums[:, col].sum() / w.sum()
        err = means.std(ddof=1) / math.sqrt(nb)
        assert abs(mu - exact[idx]) < 4.5 * err + 1e-12, (col, mu, exact[idx], err)


# --------------------------------------------------------------------------
# Serial BKL with the sites grouped by class (the n-fold way; the serial
# reference of Sec. 4 for relaxation runs)
# --------------------------------------------------------------------------
def numpy_classes_shape(shape, s):
    """class = 7*[sigma=+1] + up neighbours on an Lx x Ly x Lz periodic
    lattice (x fastest); an axis of length 2 lists its partner twice."""
    Lx, Ly, Lz = shape
    a = (s.reshape(Lz, Ly, Lx) > 0).astype(np.int64)
    u = sum(np.roll(a, sh, axis=ax) for ax in (0, 1, 2) for sh in (1, -1))
    return (7 * a + u).reshape(-1)


def brute_bkl(shape, J, H, T, seed, s, times, nevents):
    r = [1.0 / (1.0 + math.exp(2.0 * (1 if c >= 7 else -1) * (J * (2 * (c % 7) - 6) + H) / T))
         for c in range(14)]
    s = s.copy()
    N = s.size
    t, g, out, sites = 0.0, 0, [], []
    for e in range(nevents):
        cls = numpy_classes_shape(shape, s)
        n = [int(np.sum(cls == c)) for c in range(14)]
        cum, R = [], 0.0
        for c in range(14):
            R = R + n[c] * r[c]
            cum.append(R)
        w = numpy_philox((e, 0, 6, 0), (seed, 0))
        xi = (2 * (w[2] >> 12) + 1) * 2.0 ** -53
        dt = -math.log(xi) / R
        while g < len(times) and times[g] < t + dt:
            out.append(int(s.sum()) / N)
            g += 1
        if g >= len(times):
            break
        target = (w[0] >> 11) * 2.0 ** -53 * R
        c = next((q for q in range(14) if target < cum[q]), None)
        if c is None:
            c = max(q for q in range(14) if n[q] > 0)
        j = (w[1] * n[c]) >> 64
        site = int(np.flatnonzero(cls == c)[j])
        sites.append(site)
        t = t + dt
        s[site] = -s[site]
    return np.array(out), np.array(sites, dtype=np.int32)


@pytest.mark.parametrize("shape,J,H,T,seed", [
    ((4, 4, 4), 1.0, 0.0, 4.5115, 7),
    ((3, 3, 2), 1.0, 0.2, 3.0, 8),
    ((4, 2, 3), -0.8, 0.0, 2.5, 9),
])
def test_class_bkl_bruteforce(shape, J, H, T, seed):
    rng = np.random.default_rng(seed)
    s0 = rng.choice(np.array([-1, 1], dtype=np.int8), size=int(np.prod(shape)))
    times = np.linspace(0.01, 40.0, 60)
    n = 300
    m_ref, sites_ref = brute_bkl(shape, J, H, T, seed, s0, times, n)
    s = s0.copy()
    m, ne, sites = oracle.bkl_relax(shape, J, H, T, seed, s, times, record_sites=n)
    assert np.array_equal(sites, sites_ref[:ne])
    k = len(m_ref)
    assert np.array_equal(m[:k], m_ref)
    assert ne == len(sites_ref)


@pytest.mark.parametrize("T", [3.5, 4.5115, 6.0])
def test_class_bkl_matches_exact_enumeration(T):
    """The state sampled on a uniform time grid of a long run averages to
    the Boltzmann <m^2>, <m^4> and <|m|> of Eq. 1 on 3x3x2 (2^18 states)."""
    shape, J, H = (3, 3, 2), 1.0, 0.0
    exact = oracle.enumerate_exact(shape, J, H, T)
    s = np.ones(18, dtype=np.int8)
    times = np.arange(1, 400_001, dtype=np.float64) * 0.5
    m, _, _ = oracle.bkl_relax(shape, J, H, T, 2000 + int(T * 10), s, times)
    m = m[1000:]  # past the start from all +1
    nb = 40
    for vals, idx in [(m ** 2, 2), (m ** 4, 3), (np.abs(m), 4)]:
        means = vals[: len(vals) // nb * nb].reshape(nb, -1).mean(axis=1)
        err = means.std(ddof=1) / math.sqrt(nb)
        assert abs(vals.mean() - exact[idx]) < 4.5 * err, (idx, vals.mean(), exact[idx], err)
