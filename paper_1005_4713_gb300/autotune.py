"""Autotuner for the persistent cycle launch and the domain edge.

Two choices are made by timed trials on the GPU at hand and cached per device
in a JSON file (``$SPKMC_TUNE_CACHE``, default ``~/.cache/spkmc/autotune.json``):

* launch geometry for a lattice (L, d): active domains per CTA and CTAs per
  SM of the persistent grid.  It changes only speed, never results: the
  trajectory is fixed by (L, d, J, H, T, seed).
* the domain edge d for a lattice edge L (used for batched ensembles).  d is
  part of a lattice's definition (it sets the sublattice decomposition of
  Sec. 3.2 and the random streams), so once chosen it is recorded and every
  run that is compared with another uses the same resolved d.
"""
from __future__ import annotations

import json
import os
import time

from . import Lattice, make_config

EDGES = (16, 8, 4, 2)
LAUNCH_CANDIDATES = ((32, 0), (48, 0), (64, 0), (96, 0), (128, 0), (64, 1))


def cache_path() -> str:
    return os.environ.get("SPKMC_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "spkmc", "autotune.json"))


def _device_key() -> str:
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
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def valid_edges(L: int):
    return [d for d in EDGES if L % (2 * d) == 0]


def _events_per_second(L, d, cycles, items_per_cta=0, ctas_per_sm=0, seed=12345):
    cfg = make_config(items_per_cta=items_per_cta, ctas_per_sm=ctas_per_sm)
    with Lattice(L, d, 1.0, 0.0, 4.5115, seed, config=cfg) as lat:
        lat.run(max(2, cycles // 4))  # warm up (and move away from the start state)
        lat.synchronize()
        t0 = time.perf_counter()
        lat.run(cycles)
        lat.synchronize()
        dt = time.perf_counter() - t0
        return cycles * lat.K_act / dt


def tune_launch(L: int, d: int, cycles: int = 64, candidates=LAUNCH_CANDIDATES, cache: dict | None = None,
                persist: bool = True) -> dict:
    """Best (items_per_cta, ctas_per_sm) for lattice (L, d), measured."""
    own = cache is None
    cache = load_cache() if own else cache
    key = f"{_device_key()}|launch|L={L}|d={d}"
    if key in cache:
        return cache[key]
    trials = []
    for ipc, cps in candidates:
        eps = _events_per_second(L, d, cycles, ipc, cps)
        trials.append({"items_per_cta": ipc, "ctas_per_sm": cps, "events_per_s": eps})
    best = max(trials, key=lambda r: r["events_per_s"])
    entry = {"items_per_cta": best["items_per_cta"], "ctas_per_sm": best["ctas_per_sm"],
             "events_per_s": best["events_per_s"], "trials": trials}
    cache[key] = entry
    if persist:
        save_cache(cache)
    return entry


def choose_domain_edge(L: int, cycles: int = 64, cache: dict | None = None, persist: bool = True) -> int:
    """Domain edge with the highest measured event rate for an L^3 lattice."""
    own = cache is None
    cache = load_cache() if own else cache
    key = f"{_device_key()}|edge|L={L}"
    if key in cache:
        return int(cache[key]["d"])
    trials = {d: _events_per_second(L, d, cycles) for d in valid_edges(L)}
    if not trials:
        raise ValueError(f"no domain edge fits L={L}")
    best = max(trials, key=trials.get)
    cache[key] = {"d": best, "events_per_s": trials}
    if persist:
        save_cache(cache)
    return best


def edge_map(Ls, cycles: int = 64) -> dict:
    """Domain edge for every distinct L (measured once per device, cached)."""
    cache = load_cache()
    out = {int(L): choose_domain_edge(int(L), cycles, cache=cache, persist=False) for L in sorted(set(Ls))}
    save_cache(cache)
    return out
