"""Relaxation studies of Sec. 4 and Sec. 6 (not collected by pytest; run as a
command on a GPU machine).

  python tests/relaxation_study.py bias --L 64 --d 8 --colours 2 --runs 20
      spkMC replicas from all +1 at T_c against serial BKL runs of the
      oracle (the serial reference of Sec. 4): the time-integrated bias of
      Eq. 9 with its deviation sigma_b, the largest |bias(t)| of Eq. 8, m at
      the last time on both sides, and UR of Eq. 10 early and late.
  python tests/relaxation_study.py z --L 1024 --d 16 --t-end 300 --points 80
      the effective dynamic exponent z(t) of Eq. 13 from one relaxation,
      summarised over three time windows.

Each prints one JSON object.  The serial curves need the oracle, which only
test code may use; hence this file lives with the tests.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1005_4713_gb300 import relax as rx  # noqa: E402


def serial_curves(L, times, n, seed0, T=rx.T_CRITICAL, workers=None):
    def one(i):
        s = np.ones(L ** 3, dtype=np.int8)
        m, _, _ = oracle.bkl_relax((L, L, L), 1.0, 0.0, T, seed0 + i, s, times)
        return m
    with ThreadPoolExecutor(max_workers=workers or (os.cpu_count() or 1)) as ex:  # the C calls release the GIL
        return np.array(list(ex.map(one, range(n))))


def bias_study(L, d, colours, runs, t_end=4.0, points=30, window=(0.1, 4.0), seed_par=100, seed_ser=5000):
    t = np.geomspace(0.05, t_end, points)
    sub = rx.SPKMC_SUBLATTICE_2_RANDOM if colours == 2 else rx.SPKMC_SUBLATTICE_8_ROTATING
    t0 = time.perf_counter()
    par = rx.relax(L, d, t, n_runs=runs, seed0=seed_par, sublattice=sub)
    t1 = time.perf_counter()
    ser = serial_curves(L, t, runs, seed_ser)
    t2 = time.perf_counter()
    b_t, _, bi, sb = rx.bias(t, par.m, ser, window)
    late = t > 0.3
    ur = np.nanmean(par.ur, axis=0)
    return {"study": "bias", "L": L, "d": d, "colours": colours, "runs_each": runs, "window": list(window),
            "integrated_bias": bi, "sigma_b": sb, "bias_over_sigma": bi / sb if sb > 0 else None,
            "max_abs_bias_t": float(np.max(np.abs(b_t[(t >= window[0]) & (t <= window[1])]))),
            "m_last": {"spkmc": float(par.m[:, -1].mean()), "serial": float(ser[:, -1].mean())},
            "ur_late_start_end": [float(ur[late][0]), float(ur[late][-1])],
            "spkmc_cycles": par.cycles[0], "gpu_s": t1 - t0, "serial_s": t2 - t1,
            "serial_cores": os.cpu_count()}


def z_study(L, d, t_end, points, window=9, t_start=0.05):
    t = np.geomspace(t_start, t_end, points)
    t0 = time.perf_counter()
    r = rx.relax(L, d, t, n_runs=1, seed0=1)
    dt = time.perf_counter() - t0
    m = r.m.mean(axis=0)
    z = rx.effective_z(t, m, window=window)

    def mean_z(lo, hi):
        sel = (t >= lo) & (t <= hi) & np.isfinite(z)
        return float(np.mean(z[sel])) if sel.any() else None

    return {"study": "z", "L": L, "d": d, "colours": 8, "cycles": r.cycles[0], "gpu_s": dt,
            "beta_over_nu": rx.BETA_OVER_NU, "fit_points": window,
            "z_20_60": mean_z(20, 60), "z_60_150": mean_z(60, 150), "z_150_300": mean_z(150, 300),
            "m_end": float(m[-1]), "t_end": float(t[-1])}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    sub = ap.add_subparsers(dest="cmd", required=True)
    b = sub.add_parser("bias")
    b.add_argument("--L", type=int, default=64)
    b.add_argument("--d", type=int, default=8)
    b.add_argument("--colours", type=int, choices=(2, 8), default=2)
    b.add_argument("--runs", type=int, default=20)
    z = sub.add_parser("z")
    z.add_argument("--L", type=int, default=1024)
    z.add_argument("--d", type=int, default=16)
    z.add_argument("--t-end", type=float, default=300.0)
    z.add_argument("--points", type=int, default=80)
    args = ap.parse_args(argv)
    if args.cmd == "bias":
        out = bias_study(args.L, args.d, args.colours, args.runs)
    else:
        out = z_study(args.L, args.d, args.t_end, args.points)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
