"""Autotuner for the persistent cycle launch and the domain edge.

Choices are made by timed trials on the GPU at hand and cached per device in
a JSON file (``$SPKMC_TUNE_CACHE``, default ``~/.cache/spkmc/autotune.json``):

* launch geometry: active domains per CTA (``items_per_cta``) and CTAs per SM
  (``ctas_per_sm``) of the persistent grid, for one lattice (L, d) or for a
  batch keyed by its mix of domain edges and its size.  Geometry changes only
  speed, never results: a trajectory is fixed by (L, d, J, H, T, seed), so
  the objective is the time per cycle.  :class:`Lattice` and the batched
  ensemble read the cached choice when the caller sets neither knob.
* the domain edge d for a lattice edge L (for batched ensembles).  d is part
  of a lattice's definition (it sets the sublattice decomposition of Sec. 3.2
  and the random streams), so once chosen it is recorded and every run that
  is compared with another uses the same resolved d.  The objective is spin
  flips per second: null events (Sec. 3.1 step 4, the padding R_max - R_k)
  advance no spin, and smaller domains waste a larger share of the events on
  them (Eq. 10), so events per second would favour edges that do less.

Threads per domain are not a knob: one octet of lanes per domain ranks the
sites (every edge fits one octet's words) and one thread per domain flips,
and both alternatives measured slower (a whole warp for the search, a pair of
threads for the flip).

Every ``measure`` argument is a callable that times one candidate; tests pass
fakes, the default runs the candidate on the GPU.
"""
from __future__ import annotations

import functools
import json
import math
import os
import time

EDGES = (16, 8, 4, 2)
LAUNCH_CANDIDATES = ((32, 0), (48, 0), (64, 0), (96, 0), (128, 0), (64, 1))


def cache_path() -> str:
    return os.environ.get("SPKMC_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "spkmc", "autotune.json"))


@functools.lru_cache(maxsize=None)
def device_key() -> str:
    try:
        import torch
        return torch.cuda.get_device_name(0).replace(" ", "_")
    except Exception:
        return "cuda"


def load_cache(path: str | None = None) -> dict:
    path = path or cache_path()
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(cache: dict, path: str | None = None) -> None:
    path = path or cache_path()
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def valid_edges(L: int):
    return [d for d in EDGES if L % (2 * d) == 0]


def launch_key(L: int, d: int, device: str | None = None) -> str:
    return f"{device or device_key()}|launch|L={L}|d={d}"


def spec_edge(s) -> int:
    """The domain edge a lattice spec runs with: its own, or the library's
    choice for its L when it leaves the edge to the library (d = 0)."""
    if s.d:
        return int(s.d)
    from . import spkmc_resolve_domain_edge
    return int(spkmc_resolve_domain_edge(s.L))


def batch_key(specs, device: str | None = None) -> str:
    """Batches are keyed by their set of domain edges and the power of two
    nearest their active domains per cycle (the grid fills by that count)."""
    edges = sorted({spec_edge(s) for s in specs})
    q = sum((s.L // spec_edge(s) // 2) ** 3 for s in specs)
    return f"{device or device_key()}|batch|edges={','.join(map(str, edges))}|Q=2^{round(math.log2(max(q, 1)))}"


def edge_key(L: int, device: str | None = None) -> str:
    return f"{device or device_key()}|edge|L={L}"


# ---------------------------------------------------------------------------
# measurements on the GPU (the defaults of the ``measure`` arguments)
# ---------------------------------------------------------------------------
def measure_lattice(L, d, cycles, items_per_cta=0, ctas_per_sm=0, seed=12345):
    """Events/s and flips/s of cycles of one lattice at T_c, after a warm-up."""
    from . import Lattice, make_config
    cfg = make_config(items_per_cta=items_per_cta, ctas_per_sm=ctas_per_sm)
    with Lattice(L, d, 1.0, 0.0, 4.5115, seed, config=cfg, tuned=False) as lat:
        lat.run(max(2, cycles // 4))  # warm up (and move away from the start state)
        o0 = lat.observables()
        t0 = time.perf_counter()
        lat.run(cycles)
        lat.synchronize()
        dt = time.perf_counter() - t0
        o1 = lat.observables()
    flips = o1.n_flip - o0.n_flip
    return {"events_per_s": cycles * lat.K_act / dt, "flips_per_s": flips / dt, "s_per_cycle": dt / cycles}


def measure_batch(specs, cycles, items_per_cta=0, ctas_per_sm=0):
    """Time per cycle of one batch of the given lattices."""
    from . import Batch, make_config
    cfg = make_config(items_per_cta=items_per_cta, ctas_per_sm=ctas_per_sm)
    with Batch(len(specs), cfg) as b:
        for s in specs:
            b.admit(s.L, s.d, s.J, s.H, s.T, s.seed, cold=s.cold)
        b.run(max(2, cycles // 4))
        b.synchronize()
        t0 = time.perf_counter()
        b.run(cycles)
        b.synchronize()
        dt = time.perf_counter() - t0
    q = sum((s.L // spec_edge(s) // 2) ** 3 for s in specs)
    return {"events_per_s": cycles * q / dt, "s_per_cycle": dt / cycles}


# ---------------------------------------------------------------------------
# tuning and look-ups
# ---------------------------------------------------------------------------
def _pick_launch(trials):
    return min(trials, key=lambda r: r["s_per_cycle"])


def tune_launch(L: int, d: int, cycles: int = 64, candidates=LAUNCH_CANDIDATES, cache: dict | None = None,
                persist: bool = True, measure=None, device: str | None = None) -> dict:
    """Fastest (items_per_cta, ctas_per_sm) for lattice (L, d), measured once
    per device and cached."""
    own = cache is None
    cache = load_cache() if own else cache
    key = launch_key(L, d, device)
    if key in cache:
        return cache[key]
    measure = measure or (lambda ipc, cps: measure_lattice(L, d, cycles, ipc, cps))
    trials = [dict(measure(ipc, cps), items_per_cta=ipc, ctas_per_sm=cps) for ipc, cps in candidates]
    best = _pick_launch(trials)
    entry = {"items_per_cta": best["items_per_cta"], "ctas_per_sm": best["ctas_per_sm"],
             "objective": "seconds per cycle (geometry does not change the trajectory)", "trials": trials}
    cache[key] = entry
    if persist:
        save_cache(cache)
    return entry


def tune_batch(specs, cycles: int = 64, candidates=LAUNCH_CANDIDATES, cache: dict | None = None,
               persist: bool = True, measure=None, device: str | None = None) -> dict:
    """Fastest launch geometry for a batch with this mix of lattices."""
    own = cache is None
    cache = load_cache() if own else cache
    key = batch_key(specs, device)
    if key in cache:
        return cache[key]
    measure = measure or (lambda ipc, cps: measure_batch(specs, cycles, ipc, cps))
    trials = [dict(measure(ipc, cps), items_per_cta=ipc, ctas_per_sm=cps) for ipc, cps in candidates]
    best = _pick_launch(trials)
    entry = {"items_per_cta": best["items_per_cta"], "ctas_per_sm": best["ctas_per_sm"],
             "objective": "seconds per cycle (geometry does not change the trajectory)", "trials": trials}
    cache[key] = entry
    if persist:
        save_cache(cache)
    return entry


def cached_launch(L: int, d: int, cache: dict | None = None, device: str | None = None):
    """The cached geometry of lattice (L, d) as (items_per_cta, ctas_per_sm),
    or None if it was never tuned on this device."""
    e = (load_cache() if cache is None else cache).get(launch_key(L, d, device))
    return (int(e["items_per_cta"]), int(e["ctas_per_sm"])) if e else None


def cached_batch(specs, cache: dict | None = None, device: str | None = None):
    e = (load_cache() if cache is None else cache).get(batch_key(specs, device))
    return (int(e["items_per_cta"]), int(e["ctas_per_sm"])) if e else None


def choose_domain_edge(L: int, cycles: int = 64, cache: dict | None = None, persist: bool = True,
                       measure=None, device: str | None = None) -> int:
    """Domain edge with the most spin flips per second for an L^3 lattice
    (events per second, nulls included, are recorded beside it)."""
    own = cache is None
    cache = load_cache() if own else cache
    key = edge_key(L, device)
    if key in cache and "flips_per_s" in cache[key]:
        return int(cache[key]["d"])
    measure = measure or (lambda d: measure_lattice(L, d, cycles))
    trials = {d: measure(d) for d in valid_edges(L)}
    if not trials:
        raise ValueError(f"no domain edge fits L={L}")
    best = max(trials, key=lambda d: trials[d]["flips_per_s"])
    cache[key] = {"d": best, "objective": "flips_per_s",
                  "flips_per_s": {str(d): t["flips_per_s"] for d, t in trials.items()},
                  "events_per_s": {str(d): t["events_per_s"] for d, t in trials.items()}}
    if persist:
        save_cache(cache)
    return best


def edge_map(Ls, cycles: int = 64, measure=None, device: str | None = None, cache: dict | None = None) -> dict:
    """Domain edge for every distinct L (measured once per device, cached)."""
    own = cache is None
    cache = load_cache() if own else cache
    out = {int(L): choose_domain_edge(int(L), cycles, cache=cache, persist=False,
                                      measure=(lambda d, L=L: measure(L, d)) if measure else None, device=device)
           for L in sorted(set(Ls))}
    if own:
        save_cache(cache)
    return out


def edge_report(Ls, cache: dict | None = None, device: str | None = None) -> dict:
    """Per L: the chosen edge and the measured flips/s and events/s of each
    candidate edge (from the cache)."""
    cache = load_cache() if cache is None else cache
    return {str(L): cache.get(edge_key(int(L), device)) for L in sorted(set(int(x) for x in Ls))}
