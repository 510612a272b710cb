"""Relaxation of the magnetisation from all spins +1 at the critical point
(Sec. 4 and Sec. 6 of arXiv:1005.4713).

``relax`` runs independent spkMC replicas (seeds seed0 + i) of one lattice in
one batch and samples every replica after each chunk of cycles, recorded on
the device: each launch runs ``records_per_launch`` chunks and records the
observables after each.  Its m(t) is on a grid of physical time
t = clock / n_colours: every domain is active in one cycle out of n_colours
(8 in rotation, or 2 on average with the two random colours), and the spkMC
clock advances by the step of an active domain, so a domain has lived
clock / n_colours when the clock reads ``clock``.  Between samples m is
interpolated linearly in time; the chunks are sized, launch by launch, so
that the clock advances by at most ``rel_step`` of its value per chunk.  The utilisation ratio UR of Eq. 10 over each grid interval is
estimated by the fraction of non-null events (its expectation in a cycle is
sum_k R_k / (K R_max)).

``bias`` is Eq. 8 for a set of parallel and serial curves, with the
deviation of the time-integrated bias of Eq. 9.  ``effective_z`` is Eq. 13:
z(t) = -(beta/nu) / (d log m / d log t), the slope fitted over a sliding
window of grid points.

Command line: ``python -m paper_1005_4713_gb300.relax --L 256 --d 16
--t-end 20`` prints one JSON object (t, m, UR and z(t)).
"""
from __future__ import annotations

import argparse
import json
import math
from dataclasses import dataclass, field

import numpy as np

from . import (Batch, SPKMC_RMAX_EXACT, SPKMC_SUBLATTICE_2_RANDOM, SPKMC_SUBLATTICE_8_ROTATING, obs_buffer)

T_CRITICAL = 1.0 / 0.2216546  # J/k_B, Sec. 2 and Sec. 6
BETA_OVER_NU = 0.515          # the ratio taken in Sec. 6


@dataclass
class Relaxation:
    t: np.ndarray                 # physical time grid
    m: np.ndarray                 # [runs, len(t)] magnetisation per spin
    ur: np.ndarray                # [runs, len(t)] UR over (t[i-1], t[i]] (t[-1] = 0)
    cycles: list = field(default_factory=list)  # cycles run per replica
    n_colours: int = 8


def _interp(clock, values, c):
    return np.interp(c, clock, values)


def relax(L, d, t_grid, n_runs=1, seed0=1, T=T_CRITICAL, J=1.0, H=0.0,
          sublattice=SPKMC_SUBLATTICE_8_ROTATING, rmax_mode=SPKMC_RMAX_EXACT, rel_step=0.02,
          max_chunk=4096, records_per_launch=8, config=None) -> Relaxation:
    t_grid = np.asarray(t_grid, dtype=np.float64)
    if t_grid.ndim != 1 or len(t_grid) == 0 or np.any(np.diff(t_grid) <= 0) or t_grid[0] <= 0:
        raise ValueError("t_grid must be positive and increasing")
    ncol = 2 if sublattice == SPKMC_SUBLATTICE_2_RANDOM else 8
    c_end = t_grid[-1] * ncol
    c_first = t_grid[0] * ncol
    N = L ** 3
    with Batch(n_runs, config) as b:
        slots = [b.admit(L, d, J, H, T, seed0 + i, cold=True, rmax_mode=rmax_mode, sublattice=sublattice)
                 for i in range(n_runs)]
        clock = [[0.0] for _ in slots]
        mag = [[1.0] for _ in slots]
        flips = [[0] for _ in slots]
        nulls = [[0] for _ in slots]
        done_cycles = 0
        chunk = 1
        nrec = records_per_launch
        rec = obs_buffer(n_runs * nrec)
        while min(c[-1] for c in clock) < c_end:
            start = [c[-1] for c in clock]
            b.run_recorded(chunk, nrec, rec)
            b.synchronize()
            done_cycles += chunk * nrec
            adv = 0.0
            for i, sl in enumerate(slots):
                for r in range(nrec):
                    o = rec[sl * nrec + r]
                    clock[i].append(o.clock)
                    mag[i].append(o.M / N)
                    flips[i].append(o.n_flip)
                    nulls[i].append(o.n_null)
                adv = max(adv, (clock[i][-1] - start[i]) / (chunk * nrec))
            now = min(c[-1] for c in clock)
            if adv > 0 and math.isfinite(adv):
                chunk = int(max(1, min(max_chunk, rel_step * max(now, c_first) / adv)))
                # near the end, no more chunks than the clock still needs
                nrec = int(max(1, min(records_per_launch, math.ceil((c_end - now) / (adv * chunk)))))
    m = np.empty((n_runs, len(t_grid)))
    ur = np.empty((n_runs, len(t_grid)))
    cg = t_grid * ncol
    for i in range(n_runs):
        c = np.asarray(clock[i])
        m[i] = _interp(c, np.asarray(mag[i]), cg)
        f = _interp(c, np.asarray(flips[i], dtype=np.float64), np.concatenate([[0.0], cg]))
        n = _interp(c, np.asarray(nulls[i], dtype=np.float64), np.concatenate([[0.0], cg]))
        df, dn = np.diff(f), np.diff(n)
        with np.errstate(invalid="ignore", divide="ignore"):
            ur[i] = np.where(df + dn > 0, df / (df + dn), np.nan)
    return Relaxation(t=t_grid, m=m, ur=ur, cycles=[done_cycles] * n_runs, n_colours=ncol)


def bias(t, m_par, m_ser, window):
    """Eq. 8 per grid point (mean over the parallel runs minus mean over the
    serial runs) and, over the time window (lo, hi), the time-integrated bias
    with its deviation sigma_b = sqrt(sigma_p^2 + sigma_s^2) of Eq. 9, where
    sigma_p and sigma_s are the standard errors of the two means of the
    window-averaged m.  Returns (bias(t), serial deviation(t), integrated
    bias, sigma_b)."""
    t = np.asarray(t)
    m_par, m_ser = np.atleast_2d(m_par), np.atleast_2d(m_ser)
    b_t = m_par.mean(axis=0) - m_ser.mean(axis=0)
    s_t = m_ser.std(axis=0, ddof=1) if m_ser.shape[0] > 1 else np.zeros_like(b_t)
    lo, hi = window
    sel = (t >= lo) & (t <= hi)
    if sel.sum() < 2:
        raise ValueError("the window holds fewer than two grid points")
    tw = t[sel]

    def window_mean(m):  # trapezoidal time average over the window
        y = m[:, sel]
        return np.sum(0.5 * (y[:, 1:] + y[:, :-1]) * np.diff(tw), axis=1) / (tw[-1] - tw[0])

    ap, as_ = window_mean(m_par), window_mean(m_ser)
    var_p = ap.var(ddof=1) / len(ap) if len(ap) > 1 else 0.0
    var_s = as_.var(ddof=1) / len(as_) if len(as_) > 1 else 0.0
    return b_t, s_t, float(ap.mean() - as_.mean()), float(math.sqrt(var_p + var_s))


def effective_z(t, m, beta_over_nu=BETA_OVER_NU, window=5):
    """Eq. 13 on a grid: the slope of log m against log t fitted by least
    squares over `window` consecutive points centred on each point (NaN at
    the ends and where m <= 0)."""
    t = np.asarray(t, dtype=np.float64)
    m = np.asarray(m, dtype=np.float64)
    z = np.full(len(t), np.nan)
    h = window // 2
    with np.errstate(invalid="ignore", divide="ignore"):
        lt, lm = np.log(t), np.log(m)
    for i in range(h, len(t) - h):
        x, y = lt[i - h:i + h + 1], lm[i - h:i + h + 1]
        if not np.all(np.isfinite(y)):
            continue
        slope = np.polyfit(x, y, 1)[0]
        if slope < 0:
            z[i] = -beta_over_nu / slope
    return z


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--L", type=int, default=256)
    ap.add_argument("--d", type=int, default=16)
    ap.add_argument("--t-start", type=float, default=0.05)
    ap.add_argument("--t-end", type=float, default=20.0)
    ap.add_argument("--points", type=int, default=60)
    ap.add_argument("--runs", type=int, default=1)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--two-colour", action="store_true")
    ap.add_argument("--window", type=int, default=9)
    args = ap.parse_args(argv)
    t = np.geomspace(args.t_start, args.t_end, args.points)
    sub = SPKMC_SUBLATTICE_2_RANDOM if args.two_colour else SPKMC_SUBLATTICE_8_ROTATING
    r = relax(args.L, args.d, t, n_runs=args.runs, seed0=args.seed, sublattice=sub)
    mm = r.m.mean(axis=0)
    z = effective_z(t, mm, window=args.window)
    print(json.dumps({"L": args.L, "d": args.d, "colours": r.n_colours, "runs": args.runs,
                      "cycles": r.cycles[0], "t": t.tolist(), "m": mm.tolist(),
                      "ur": np.nanmean(r.ur, axis=0).tolist(),
                      "z": [None if not math.isfinite(v) else v for v in z]}))


if __name__ == "__main__":
    main()
