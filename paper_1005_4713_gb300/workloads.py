"""Seeded synthetic workloads shaped like the paper's runs (no method arithmetic).

The paper measures synthetic Ising lattices at the critical point (Sec. 4-6);
these generators give the lattice sizes, domain edges, temperatures, fields,
seeds and request streams used by the tests, the benchmark and the serving
loop.  Nothing here evaluates a rate, a class or an event.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

T_CRITICAL = 4.5115  # 1/beta_c with beta_c = 0.2216546 (Sec. 2, Sec. 6), rounded as in the configs


@dataclass(frozen=True)
class LatticeSpec:
    L: int
    d: int
    J: float = 1.0
    H: float = 0.0
    T: float = T_CRITICAL
    seed: int = 1
    cold: bool = False


# Single-lattice workloads.
CONFIG_16 = LatticeSpec(L=16, d=4, seed=1)             # 16^3, 4^3-site domains, hot start
CONFIG_128_HOT = LatticeSpec(L=128, d=8, seed=2)       # 128^3, 8^3-site domains, hot start
CONFIG_128_COLD = LatticeSpec(L=128, d=8, seed=2, cold=True)
CONFIG_1024 = LatticeSpec(L=1024, d=16, seed=3)        # 1024^3, 16^3-site domains, hot start

CYCLES_16 = 10_000
CYCLES_128 = 16_000   # 2000 visits of each of the 8 colours
CYCLES_1024 = 500
OBS_EVERY_1024 = 10


def ensemble_specs(n: int = 256, seed: int = 20100504, domain_edge=None):
    """Batched ensemble: L from {16,24,32,48,64,96,128}, T ~ U[4.40, 4.60],
    H in {0, 0.01}, per-lattice seeds 1000+i.  ``domain_edge`` maps L -> d
    (default: the largest of 16, 8, 4, 2 with L % 2d == 0)."""
    rng = np.random.default_rng(seed)
    Ls = rng.choice([16, 24, 32, 48, 64, 96, 128], size=n)
    Ts = rng.uniform(4.40, 4.60, size=n)
    Hs = rng.choice([0.0, 0.01], size=n)
    out = []
    for i in range(n):
        L = int(Ls[i])
        d = domain_edge(L) if domain_edge else default_edge(L)
        out.append(LatticeSpec(L=L, d=d, T=float(Ts[i]), H=float(Hs[i]), seed=1000 + i))
    return out


def default_edge(L: int) -> int:
    for d in (16, 8, 4, 2):
        if L % (2 * d) == 0:
            return d
    raise ValueError(f"no domain edge fits L={L}")


@dataclass
class Request:
    rid: int
    arrival: float          # seconds after the stream starts
    spec: LatticeSpec
    cycles: int
    meta: dict = field(default_factory=dict)


def request_stream(n: int = 2000, rate: float = 200.0, seed: int = 5, sizes=(32, 64, 128, 256),
                   t_range=(4.3, 4.7), cycles_range=(1e2, 1e4), domain_edge=None):
    """Served stream: Poisson arrivals (mean ``rate`` per second), L uniform over
    ``sizes``, T uniform in ``t_range``, H = 0, cycle budgets log-uniform."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=n)
    arrivals = np.cumsum(gaps) - gaps[0]
    Ls = rng.choice(list(sizes), size=n)
    Ts = rng.uniform(*t_range, size=n)
    cyc = np.exp(rng.uniform(np.log(cycles_range[0]), np.log(cycles_range[1]), size=n))
    out = []
    for i in range(n):
        L = int(Ls[i])
        d = domain_edge(L) if domain_edge else default_edge(L)
        out.append(Request(rid=i, arrival=float(arrivals[i]),
                           spec=LatticeSpec(L=L, d=d, T=float(Ts[i]), seed=50_000 + i),
                           cycles=int(round(cyc[i]))))
    return out
