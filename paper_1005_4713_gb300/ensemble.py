"""Batched ensembles of independent lattices (finite-size-scaling replicas).

``run_batched`` advances every lattice of the ensemble in one persistent
launch (one flat table of all active domains, a separate R_max, clock and
random streams per lattice); ``run_one_at_a_time`` runs the same lattices
one after the other with the single-lattice entry points.  Both sample m^2
and m^4 every ``sample_every`` cycles after ``burn_in`` cycles, recorded on
the device inside the launch, for the Binder ratio U_4 = <m^4>/<m^2>^2 of
Eq. 7 (and the cumulant U = 1 - U_4/3), and return bit-comparable final
observables.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

from . import Batch, Lattice, make_config, obs_buffer


@dataclass
class EnsembleResult:
    seconds: float
    events: int
    final: list = field(default_factory=list)   # (cycle, clock, M, B, n_flip, n_null, fx_lo, fx_hi)
    binder: list = field(default_factory=list)  # dicts per lattice

    @property
    def events_per_s(self):
        return self.events / self.seconds if self.seconds > 0 else 0.0

    @property
    def flips(self):
        return sum(f[4] for f in self.final)

    @property
    def flips_per_s(self):
        return self.flips / self.seconds if self.seconds > 0 else 0.0


def _obs_key(o):
    return (o.cycle, o.clock, o.M, o.B, o.n_flip, o.n_null, int(o.sum_null_rate_fx[0]), int(o.sum_null_rate_fx[1]))


def _binder(L, m2s, m4s):
    n = len(m2s)
    if n == 0:
        return {"L": L, "samples": 0, "U4": None, "U": None}
    a2 = sum(m2s) / n
    a4 = sum(m4s) / n
    u4 = a4 / (a2 * a2) if a2 > 0 else float("nan")
    return {"L": L, "samples": n, "m2": a2, "m4": a4, "U4": u4, "U": 1.0 - u4 / 3.0}


def batch_config(specs, config=None):
    """``config`` with the autotuner's cached launch geometry for this mix of
    lattices, when the caller set none and the mix was tuned on this device."""
    if config is not None and (config.items_per_cta or config.ctas_per_sm):
        return config
    from . import autotune, with_launch
    hit = autotune.cached_batch(specs)
    return config if hit is None else with_launch(config, *hit)


def run_batched(specs, cycles: int, sample_every: int = 50, burn_in: int = 0, config=None,
                tuned: bool = True) -> EnsembleResult:
    n = len(specs)
    if tuned:
        config = batch_config(specs, config)
    sample_every = max(1, min(sample_every, cycles)) if cycles > 0 else 1
    with Batch(n, config) as b:
        slots = [b.admit(s.L, s.d, s.J, s.H, s.T, s.seed, cold=s.cold, cycles=cycles) for s in specs]
        m2 = [[] for _ in specs]
        m4 = [[] for _ in specs]
        b.synchronize()
        t0 = time.perf_counter()
        done = 0
        # the samples are recorded on the device, many per launch
        per_launch = max(1, (1 << 18) // sample_every)
        rec = obs_buffer(n * min(per_launch, max(1, cycles // sample_every)))
        while cycles - done >= sample_every:
            nrec = min(per_launch, (cycles - done) // sample_every)
            b.run_recorded(sample_every, nrec, rec)
            b.synchronize()
            for r in range(nrec):
                done += sample_every
                if done > burn_in:
                    for i, sl in enumerate(slots):
                        o = rec[sl * nrec + r]
                        m2[i].append(o.m2)
                        m4[i].append(o.m4)
        if done < cycles:  # a last, shorter sample
            b.run(cycles - done)
            done = cycles
            if done > burn_in:
                obs = b.observables_all()
                for i, sl in enumerate(slots):
                    m2[i].append(obs[sl].m2)
                    m4[i].append(obs[sl].m4)
        b.synchronize()
        dt = time.perf_counter() - t0
        obs = b.observables_all()
        final = [_obs_key(obs[sl]) for sl in slots]
    events = sum(f[4] + f[5] for f in final)  # flips + nulls: one event per active domain and cycle
    binder = [dict(_binder(s.L, m2[i], m4[i]), T=s.T, H=s.H, d=s.d, seed=s.seed) for i, s in enumerate(specs)]
    return EnsembleResult(seconds=dt, events=events, final=final, binder=binder)


def run_one_at_a_time(specs, cycles: int, sample_every: int = 50, burn_in: int = 0, config=None) -> EnsembleResult:
    sample_every = max(1, min(sample_every, cycles)) if cycles > 0 else 1
    final, binder = [], []
    total = 0.0
    for s in specs:
        with Lattice(s.L, s.d, s.J, s.H, s.T, s.seed, cold=s.cold, config=config) as lat:
            m2, m4 = [], []
            lat.synchronize()
            t0 = time.perf_counter()
            done = 0
            per_launch = max(1, (1 << 18) // sample_every)
            rec = obs_buffer(min(per_launch, max(1, cycles // sample_every)))
            while cycles - done >= sample_every:
                nrec = min(per_launch, (cycles - done) // sample_every)
                lat.run_recorded(sample_every, nrec, rec)
                lat.synchronize()
                for r in range(nrec):
                    done += sample_every
                    if done > burn_in:
                        m2.append(rec[r].m2)
                        m4.append(rec[r].m4)
            if done < cycles:
                lat.run(cycles - done)
                done = cycles
                if done > burn_in:
                    o = lat.observables()
                    m2.append(o.m2)
                    m4.append(o.m4)
            lat.synchronize()
            total += time.perf_counter() - t0
            final.append(_obs_key(lat.observables()))
            binder.append(dict(_binder(s.L, m2, m4), T=s.T, H=s.H, d=s.d, seed=s.seed))
    events = sum(f[4] + f[5] for f in final)
    return EnsembleResult(seconds=total, events=events, final=final, binder=binder)


def default_config():
    return make_config()
