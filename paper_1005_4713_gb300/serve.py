"""Continuous-batching service for spkMC simulation requests.

Requests (a lattice spec and a cycle budget) arrive over time.  The server
keeps one batch (``spkmc_batch_t``) resident on the device and loops:

1. admit waiting requests, first come first served, while a slot is free and
   the device bytes of the admitted lattices stay within the memory budget
   (a request that can never fit, or whose admission fails with nothing else
   on the device, is rejected; one that meets a full device waits);
2. advance every admitted lattice by up to ``step_cycles`` cycles in one
   persistent launch (lattices stop at their own budget);
3. poll for finished lattices, read their observables (and spins if asked),
   free their memory, and record completion.

Spin and class state stay on the device between steps; a lattice's
trajectory depends only on its own parameters and seed, so its result is the
same alone and in any mix.  Latency is completion time minus arrival time.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from . import (Batch, Lattice, SpkmcError, make_params, spkmc_bytes_required, SPKMC_ENOMEM, SPKMC_INIT_COLD,
               SPKMC_INIT_HOT)


@dataclass
class Completion:
    rid: int
    arrival: float
    admitted: float
    finished: float
    cycles: int
    events: int
    obs: tuple
    spins: np.ndarray | None = None
    cancelled: bool = False
    L: int = 0

    @property
    def latency(self):
        return self.finished - self.arrival


@dataclass
class ServeStats:
    completions: list = field(default_factory=list)
    rejected: list = field(default_factory=list)
    wall: float = 0.0
    peak_bytes: int = 0
    peak_live: int = 0
    steps: int = 0

    @property
    def events(self):
        return sum(c.events for c in self.completions)

    @property
    def events_per_s(self):
        return self.events / self.wall if self.wall > 0 else 0.0

    def latency_percentile(self, q):
        lat = [c.latency for c in self.completions if not c.cancelled]
        return float(np.percentile(lat, q)) if lat else None

    def breakdown(self, q):
        """Percentile q of the time spent waiting for admission (queue) and
        of the time from admission to completion (run)."""
        done = [c for c in self.completions if not c.cancelled]
        if not done:
            return None
        return {"queue_s": float(np.percentile([c.admitted - c.arrival for c in done], q)),
                "run_s": float(np.percentile([c.finished - c.admitted for c in done], q))}

    def by_size(self):
        """Latency percentiles per lattice edge."""
        out = {}
        for c in self.completions:
            if not c.cancelled:
                out.setdefault(c.L, []).append(c.latency)
        return {str(L): {"n": len(v), "p50_s": float(np.percentile(v, 50)), "p99_s": float(np.percentile(v, 99))}
                for L, v in sorted(out.items())}


def _obs_key(o):
    return (o.cycle, o.clock, o.M, o.B, o.n_flip, o.n_null, int(o.sum_null_rate_fx[0]), int(o.sum_null_rate_fx[1]))


class Server:
    def __init__(self, budget_bytes: int, capacity: int = 256, step_cycles: int = 100, config=None,
                 keep_spins: bool = False):
        self.budget = int(budget_bytes)
        self.capacity = int(capacity)
        self.step_cycles = int(step_cycles)
        self.config = config
        self.keep_spins = keep_spins
        self._cancel = set()

    def cancel(self, rid: int) -> None:
        """Ask for request ``rid`` to be dropped at the next step boundary."""
        self._cancel.add(rid)

    def serve(self, requests, realtime: bool = True, on_step=None) -> ServeStats:
        """Serve ``requests`` (objects with rid, arrival, spec, cycles).  With
        ``realtime`` the arrivals follow the wall clock; otherwise every
        request counts as arrived at its turn (for tests)."""
        stats = ServeStats()
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        waiting = deque()
        active = {}  # slot -> (request, admit time, bytes)
        live_bytes = 0
        t0 = time.perf_counter()
        with Batch(self.capacity, self.config) as b:
            while pending or waiting or active:
                now = time.perf_counter() - t0
                while pending and (not realtime or pending[0].arrival <= now):
                    waiting.append(pending.popleft())
                # 1. admission by memory budget and free slots
                while waiting:
                    r = waiting[0]
                    s = r.spec
                    p = make_params(s.L, s.d, s.J, s.H, s.T, s.seed, SPKMC_INIT_COLD if s.cold else SPKMC_INIT_HOT)
                    need = spkmc_bytes_required(p)
                    if need <= 0 or need > self.budget:
                        stats.rejected.append(r.rid)
                        waiting.popleft()
                        continue
                    if live_bytes + need > self.budget or len(active) >= self.capacity:
                        break
                    try:
                        slot = b.admit(s.L, s.d, s.J, s.H, s.T, s.seed, cold=s.cold, cycles=r.cycles)
                    except SpkmcError as e:
                        if e.code == SPKMC_ENOMEM and active:
                            break  # the device is short of memory: admit again as lattices finish
                        stats.rejected.append(r.rid)
                        waiting.popleft()
                        continue
                    active[slot] = (r, time.perf_counter() - t0, need)
                    live_bytes += need
                    waiting.popleft()
                stats.peak_bytes = max(stats.peak_bytes, live_bytes)
                stats.peak_live = max(stats.peak_live, len(active))
                if not active:
                    if pending and realtime:
                        time.sleep(min(0.01, max(0.0, pending[0].arrival - (time.perf_counter() - t0))))
                    continue
                # 2. one step for every admitted lattice
                b.run(self.step_cycles)
                stats.steps += 1
                if on_step:
                    on_step(stats, active)
                # 3. completions (and cancellations)
                finished = b.poll()
                for slot, (r, _, _) in list(active.items()):
                    if r.rid in self._cancel and slot not in finished:
                        finished.append(slot)
                if finished:
                    all_obs = b.observables_all()
                    t = time.perf_counter() - t0
                    for slot in finished:
                        r, t_adm, need = active.pop(slot)
                        o = all_obs[slot]
                        spins = b.spins(slot) if self.keep_spins else None
                        s = r.spec
                        stats.completions.append(Completion(
                            rid=r.rid, arrival=r.arrival if realtime else 0.0, admitted=t_adm, finished=t,
                            cycles=o.cycle, events=o.n_flip + o.n_null, obs=_obs_key(o), spins=spins,
                            cancelled=r.rid in self._cancel, L=s.L))
                        b.retire(slot)
                        live_bytes -= need
        stats.wall = time.perf_counter() - t0
        return stats


def serve_one_at_a_time(requests, realtime: bool = True, config=None) -> ServeStats:
    """The same requests served one at a time with the plain single-lattice
    path (spkmc_create_ex, spkmc_run_cycles, spkmc_observables), first come
    first served on the same arrival times: the baseline of continuous
    batching.  Each result is bit-comparable with the batched one."""
    stats = ServeStats()
    t0 = time.perf_counter()
    for r in sorted(requests, key=lambda r: r.arrival):
        now = time.perf_counter() - t0
        if realtime and r.arrival > now:
            time.sleep(r.arrival - now)
        t_start = time.perf_counter() - t0
        s = r.spec
        with Lattice(s.L, s.d, s.J, s.H, s.T, s.seed, cold=s.cold, config=config) as lat:
            lat.run(r.cycles)
            o = lat.observables()
        t_end = time.perf_counter() - t0
        stats.completions.append(Completion(
            rid=r.rid, arrival=r.arrival if realtime else 0.0, admitted=t_start, finished=t_end, cycles=o.cycle,
            events=o.n_flip + o.n_null, obs=_obs_key(o), L=s.L))
        stats.peak_live = 1
        stats.steps += 1
    stats.wall = time.perf_counter() - t0
    return stats
