"""The critical point of the 3D Ising model seen through spkMC (paper Sec. 2:
the Binder ratio of Eq. 7 and T_c = 1/beta_c with beta_c = 0.2216546).

Ensembles of 64 replicas of L = 8, 12 and 16 (2^3-site domains) at five
temperatures around T_c run as one batch from hot starts (eight colours,
exact R_max).  After a burn-in, m^2 and m^4 are sampled every 200 cycles
and the cumulant U = 1 - <m^4> / (3 <m^2>^2) of every (L, T) is formed from
the pooled samples, with a jackknife error over the replicas.  Below T_c the
larger lattice orders more (U grows with L), above T_c it disorders more (U
falls with L), so the curves of different L cross near T_c, at a value near
the universal U* = 0.465 (shifted a little by corrections to scaling at these
small sizes).

This is a statistical check of the whole method (rates, selection, clock
and the decomposition together) against physics the paper states, not a
bit comparison; the trajectory is still fixed by the seeds, so the numbers
are the same on every run.
"""
import numpy as np
import pytest

import paper_1005_4713_gb300 as sp

pytestmark = pytest.mark.gpu

T_C = 1.0 / 0.2216546
LS = (8, 12, 16)
TS = (4.40, 4.48, T_C, 4.54, 4.60)
REPLICAS = 64
BURN, CYCLES, EVERY = 20_000, 100_000, 200


def cumulant(m2, m4):
    return 1.0 - m4.mean() / (3.0 * m2.mean() ** 2)


def binder_points():
    specs = [(L, T) for L in LS for T in TS for _ in range(REPLICAS)]
    nrec = CYCLES // EVERY
    with sp.Batch(len(specs)) as b:
        slots = [b.admit(L, 2, 1.0, 0.0, T, 7000 + i) for i, (L, T) in enumerate(specs)]
        b.run(BURN)
        rec = b.run_recorded(EVERY, nrec)
        b.synchronize()
        o = np.ctypeslib.as_array(rec.records)  # record r of slot s at s * nrec + r
        m2 = o["m2"].reshape(len(specs), nrec)[slots]
        m4 = o["m4"].reshape(len(specs), nrec)[slots]
    out = {}
    for i, (L, T) in enumerate(specs[::REPLICAS]):
        a2, a4 = m2[i * REPLICAS:(i + 1) * REPLICAS], m4[i * REPLICAS:(i + 1) * REPLICAS]
        u = cumulant(a2, a4)
        keep = np.ones(REPLICAS, bool)
        jk = []
        for k in range(REPLICAS):
            keep[k] = False
            jk.append(cumulant(a2[keep], a4[keep]))
            keep[k] = True
        jk = np.array(jk)
        out[(L, T)] = (u, float(np.sqrt((REPLICAS - 1) / REPLICAS * np.sum((jk - jk.mean()) ** 2))))
    return out


def crossing(pts, la, lb):
    """Temperature and cumulant where U(lb) - U(la) changes sign (linear
    interpolation between the bracketing temperatures)."""
    diff = [pts[(lb, T)][0] - pts[(la, T)][0] for T in TS]
    signs = [d > 0 for d in diff]
    flips = [i for i in range(len(TS) - 1) if signs[i] != signs[i + 1]]
    assert len(flips) == 1, (la, lb, diff)
    i = flips[0]
    f = diff[i] / (diff[i] - diff[i + 1])
    tx = TS[i] + f * (TS[i + 1] - TS[i])
    ua = pts[(la, TS[i])][0] + f * (pts[(la, TS[i + 1])][0] - pts[(la, TS[i])][0])
    ub = pts[(lb, TS[i])][0] + f * (pts[(lb, TS[i + 1])][0] - pts[(lb, TS[i])][0])
    return tx, 0.5 * (ua + ub)


def test_binder_cumulants_cross_near_the_critical_point():
    pts = binder_points()
    for (L, T), (u, e) in sorted(pts.items()):
        print(f"L={L:2d} T={T:.4f} U={u:.4f} +- {e:.4f}")
    # ordered side: U grows with L; disordered side: U falls with L
    lo, hi = TS[0], TS[-1]
    for a, b in ((8, 12), (12, 16)):
        assert pts[(b, lo)][0] > pts[(a, lo)][0]
        assert pts[(b, hi)][0] < pts[(a, hi)][0]
    for T, sign in ((lo, 1), (hi, -1)):
        d = sign * (pts[(16, T)][0] - pts[(8, T)][0])
        err = np.hypot(pts[(16, T)][1], pts[(8, T)][1])
        assert d > 6 * err, (T, d, err)
    # the curves cross near T_c, at a cumulant near the universal value
    for la, lb in ((8, 16), (12, 16)):
        tx, ux = crossing(pts, la, lb)
        print(f"crossing of L={la} and L={lb}: T={tx:.4f} (T_c = {T_C:.4f}), U={ux:.4f} (U* = 0.465)")
        assert abs(tx - T_C) < 0.04, tx
        assert 0.40 < ux < 0.50, ux
