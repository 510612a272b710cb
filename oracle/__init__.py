"""CPU oracle for the spkMC cycle (arXiv:1005.4713, Sec. 3) -- test infrastructure.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library under
``paper_1005_4713_gb300``) never imports it, and the two share no source.

The arithmetic lives in ``spkmc_oracle.c`` (plain C, FP64, -ffp-contract=off);
this module compiles it with gcc and wraps it with ctypes, returning numpy
arrays.  Parity pins for every function are in ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import platform
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spkmc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libspkmc_oracle.so")
_lock = threading.Lock()
_lib = None

_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_u64 = ctypes.c_uint64
_dbl = ctypes.c_double
_ptr = ctypes.c_void_p


_FLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared", "-std=c11"]


def _digest() -> str:
    """Hash of the oracle's source, its gcc flags and the host architecture."""
    h = hashlib.sha256()
    with open(_SRC, "rb") as f:
        h.update(f.read())
    h.update(" ".join(_FLAGS).encode())
    h.update(platform.machine().encode())
    return h.hexdigest()


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2 -ffp-contract=off -fopenmp),
    unless the one in place was built from the current source and flags."""
    os.makedirs(_BUILD, exist_ok=True)
    stamp = _LIB + ".sha256"
    digest = _digest()
    if not force and os.path.exists(_LIB) and os.path.exists(stamp):
        with open(stamp) as f:
            if f.read().strip() == digest:
                return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", *_FLAGS, "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    if os.path.exists(stamp):
        os.remove(stamp)
    os.replace(tmp, _LIB)
    with open(stamp + f".tmp{os.getpid()}", "w") as f:
        f.write(digest + "\n")
    os.replace(stamp + f".tmp{os.getpid()}", stamp)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            L.oracle_philox.argtypes = [_u64] * 6 + [_ptr]
            L.oracle_philox.restype = None
            L.oracle_rates.argtypes = [_dbl, _dbl, _dbl, _ptr]
            L.oracle_rates.restype = None
            L.oracle_init_spins.argtypes = [_i32, _u64, _i32, _ptr]
            L.oracle_init_spins.restype = None
            L.oracle_observables.argtypes = [_i32, _ptr, _ptr, _ptr]
            L.oracle_observables.restype = None
            L.oracle_class_counts.argtypes = [_i32, _i32, _ptr, _ptr]
            L.oracle_class_counts.restype = None
            L.oracle_spkmc_run.argtypes = [_i32, _i32, _dbl, _dbl, _dbl, _u64, _ptr,
                                           _i64, _i64, _ptr, _ptr, _ptr, _ptr, _ptr, _i32,
                                           _i32, _ptr, _i32]
            L.oracle_spkmc_run.restype = _i32
            L.oracle_rmax_bounds.argtypes = [_i32, _dbl, _dbl, _dbl, _ptr, _ptr]
            L.oracle_rmax_bounds.restype = None
            L.oracle_bkl_run.argtypes = [_i32, _i32, _i32, _dbl, _dbl, _dbl, _u64, _ptr,
                                         _i64, _i32, _ptr]
            L.oracle_bkl_run.restype = _i32
            L.oracle_enumerate.argtypes = [_i32, _i32, _i32, _dbl, _dbl, _dbl, _ptr]
            L.oracle_bkl_relax.argtypes = [_i32, _i32, _i32, _dbl, _dbl, _dbl, _u64, _ptr, _i32, _ptr, _ptr,
                                           _i64, _ptr, _ptr]
            L.oracle_bkl_relax.restype = _i32
            L.oracle_enumerate.restype = _i32
            _lib = L
        return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def philox(ctr, key) -> np.ndarray:
    """Philox4x64-10 block for counter ``ctr`` (4 words) and key (2 words)."""
    out = np.zeros(4, dtype=np.uint64)
    c = [int(x) & (2**64 - 1) for x in ctr]
    k = [int(x) & (2**64 - 1) for x in key]
    lib().oracle_philox(*c, *k, _p(out))
    return out


def rates(J: float, H: float, T: float) -> np.ndarray:
    """Glauber rate table r[c], c = 7*[sigma=+1] + u (Eq. 3, corrected sign)."""
    out = np.zeros(14, dtype=np.float64)
    lib().oracle_rates(J, H, T, _p(out))
    return out


def init_spins(L: int, seed: int, cold: bool = False) -> np.ndarray:
    """int8 spins in global order g = X + L*(Y + L*Z)."""
    s = np.empty(L * L * L, dtype=np.int8)
    lib().oracle_init_spins(L, seed, 1 if cold else 0, _p(s))
    return s


def observables(L: int, s: np.ndarray):
    """(M, B): magnetisation sum and forward bond sum (Eq. 1, Eq. 4)."""
    s = np.ascontiguousarray(s, dtype=np.int8)
    M = np.zeros(1, dtype=np.int64)
    B = np.zeros(1, dtype=np.int64)
    lib().oracle_observables(L, _p(s), _p(M), _p(B))
    return int(M[0]), int(B[0])


def class_counts(L: int, d: int, s: np.ndarray) -> np.ndarray:
    """Per-domain class counts, shape (K, 14), domain order k."""
    s = np.ascontiguousarray(s, dtype=np.int8)
    nd = L // d
    out = np.zeros((nd ** 3, 14), dtype=np.int32)
    lib().oracle_class_counts(L, d, _p(s), _p(out))
    return out


RMAX_EXACT, RMAX_PRESCRIBED, RMAX_LEARNED = 0, 1, 2
SUB_8_ROTATING, SUB_2_RANDOM = 0, 1


class BoundExceeded(RuntimeError):
    """An active domain's R_k exceeded the bound of Sec. 3.2 step 4b."""


def rmax_bounds(d: int, J: float, H: float, T: float):
    """(prescribed bound R', learned margin a + 12 b), Sec. 3.2: a is the
    largest rate change of a flipped site, b the largest change of a site
    whose neighbour sum moves by 2."""
    a = np.zeros(1)
    b = np.zeros(1)
    lib().oracle_rmax_bounds(d, J, H, T, _p(a), _p(b))
    return float(a[0]), float(b[0])


class State:
    """Mutable spkMC state: spins plus the cycle counter, clock and counters.

    ``rmax_mode`` picks the rate the frequency lines are padded to: the exact
    R_max of the cycle (Sec. 3.1 step 2) or a bound of Sec. 3.2 step 4b.
    ``rmax_hist[i]`` holds the exact R_max of cycle ``cycle - 8 + i``.
    ``sublattice``: eight colours in rotation, or the paper's two colours
    drawn at random each cycle (Sec. 3.2 step 4a)."""

    def __init__(self, L, d, J, H, T, seed, cold=False, spins=None, rmax_mode=RMAX_EXACT,
                 sublattice=SUB_8_ROTATING):
        self.L, self.d, self.J, self.H, self.T, self.seed = L, d, J, H, T, seed
        self.rmax_mode = rmax_mode
        self.sublattice = sublattice
        self.rmax_hist = np.zeros(8, dtype=np.float64)
        self.spins = (init_spins(L, seed, cold) if spins is None
                      else np.array(spins, dtype=np.int8, copy=True))
        self.cycle = 0
        self.clock = 0.0
        self.n_flip = 0
        self.n_null = 0
        self.null_fx = 0  # sum of null rates r_0k, fixed point with 2^-64 units

    @property
    def k_act(self):
        nd = self.L // self.d
        return (nd // 2) ** 3 if self.sublattice == SUB_8_ROTATING else nd ** 3 // 2

    def run(self, ncycles: int, log: bool = False, threads: int = 1):
        """Advance ``ncycles`` cycles.  With ``log`` returns an int32 array of
        shape (ncycles, K_act, 3) holding (k, class or -1, site or -1)."""
        clock = np.array([self.clock], dtype=np.float64)
        nf = np.array([self.n_flip], dtype=np.int64)
        nn = np.array([self.n_null], dtype=np.int64)
        fx = np.array([self.null_fx & (2**64 - 1), self.null_fx >> 64], dtype=np.uint64)
        ev = np.zeros((max(ncycles, 0), self.k_act, 3), dtype=np.int32) if log else None
        rc = lib().oracle_spkmc_run(self.L, self.d, self.J, self.H, self.T, self.seed,
                                    _p(self.spins), self.cycle, ncycles, _p(clock),
                                    _p(nf), _p(nn), _p(fx),
                                    _p(ev) if log else None, threads,
                                    self.rmax_mode, _p(self.rmax_hist), self.sublattice)
        if rc == -2:
            raise BoundExceeded("an active domain exceeded the R_max bound")
        if rc != 0:
            raise ValueError("oracle_spkmc_run rejected its arguments")
        self.cycle += ncycles
        self.clock = float(clock[0])
        self.n_flip = int(nf[0])
        self.n_null = int(nn[0])
        self.null_fx = int(fx[0]) | (int(fx[1]) << 64)
        return ev

    def observables(self):
        return observables(self.L, self.spins)


def bkl_run(shape, J, H, T, seed, spins, nevents, nbatches):
    """Serial BKL on a periodic Lx x Ly x Lz lattice; returns per-batch
    time-weighted sums, shape (nbatches, 6) = (sum dt, E dt, E^2 dt, m^2 dt,
    m^4 dt, |m| dt).  ``spins`` (int8, x fastest) is updated in place."""
    Lx, Ly, Lz = shape
    out = np.zeros((nbatches, 6), dtype=np.float64)
    assert spins.dtype == np.int8 and spins.flags.c_contiguous
    rc = lib().oracle_bkl_run(Lx, Ly, Lz, J, H, T, seed, _p(spins), nevents, nbatches, _p(out))
    if rc != 0:
        raise ValueError("oracle_bkl_run rejected its arguments")
    return out


def enumerate_exact(shape, J, H, T):
    """Exact Boltzmann averages (<E>, <E^2>, <m^2>, <m^4>, <|m|>, <m>)."""
    Lx, Ly, Lz = shape
    out = np.zeros(6, dtype=np.float64)
    rc = lib().oracle_enumerate(Lx, Ly, Lz, J, H, T, _p(out))
    if rc != 0:
        raise ValueError("oracle_enumerate rejected its arguments")
    return out


def bkl_relax(shape, J, H, T, seed, spins, times, max_events=1 << 62, record_sites=0):
    """Serial BKL with sites grouped by class (the n-fold way, Sec. 4's
    serial reference), from ``spins`` (modified in place): m at each of the
    ascending ``times``.  Returns (m, events run, flipped sites or None)."""
    Lx, Ly, Lz = shape
    times = np.ascontiguousarray(times, dtype=np.float64)
    m = np.full(len(times), np.nan)
    ne = np.zeros(1, dtype=np.int64)
    sites = np.zeros(record_sites, dtype=np.int32) if record_sites else None
    if record_sites:
        max_events = min(max_events, record_sites)
    g = lib().oracle_bkl_relax(Lx, Ly, Lz, J, H, T, seed, _p(spins), len(times), _p(times), _p(m),
                               int(max_events), _p(ne), _p(sites) if record_sites else None)
    if g < 0:
        raise ValueError("oracle_bkl_relax rejected its arguments")
    return m, int(ne[0]), (sites[:int(ne[0])] if record_sites else None)
