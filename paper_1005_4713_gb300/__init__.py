"""GB300 spkMC: synchronous parallel kinetic Monte Carlo on the 3D Ising lattice.

Python binding of ``libspkmc.so`` (C ABI in ``include/spkmc.h``).  Every
function named ``spkmc_*`` here marshals its arguments to the C entry point
of the same name; all work of the spkMC cycle (arXiv:1005.4713, Sec. 3.1
steps 1-6, Sec. 3.2 steps 4a/4b) runs in the library's CUDA kernels.  There is
no other implementation: if the library cannot be loaded, every call raises.

PyTorch is optional plumbing: :func:`torch_config` points the library at the
current torch stream and, if asked, at torch's caching allocator.
"""
from __future__ import annotations

import ctypes
import threading

import numpy as np

from . import _abi
from ._abi import (SPKMC_EBOUND, SPKMC_EBUSY, SPKMC_ECUDA, SPKMC_EINTERNAL, SPKMC_EINVAL,  # noqa: F401
                   SPKMC_ENOMEM, SPKMC_RMAX_EXACT, SPKMC_RMAX_LEARNED, SPKMC_RMAX_PRESCRIBED,
                   SPKMC_SUBLATTICE_2_RANDOM, SPKMC_SUBLATTICE_8_ROTATING,
                   SPKMC_INIT_COLD, SPKMC_INIT_HOT, SPKMC_OK, SPKMC_ETIMEOUT, spkmc_config,
                   spkmc_event, spkmc_info, spkmc_obs, spkmc_params, spkmc_state)

__all__ = [n for n in _abi.PROTOTYPES] + ["Lattice", "Batch", "Graph", "SpkmcError", "torch_config", "obs_buffer",
                                            "make_params", "make_config", "EVENT_DTYPE", "tuned_config", "with_launch"]

_lock = threading.Lock()
_lib = None

EVENT_DTYPE = np.dtype([("cycle", "<i8"), ("domain", "<i4"), ("cls", "<i4"), ("site", "<i4"),
                        ("reserved", "<i4")])


class SpkmcError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"{_abi.STATUS_NAMES.get(code, code)}: {message}")
        self.code = code


def lib() -> ctypes.CDLL:
    """The loaded library, built in tree on first use if missing or stale."""
    global _lib
    with _lock:
        if _lib is None:
            from . import build as _build
            _build.build()
            _lib = _abi.load()
        return _lib


def _check(rc: int) -> None:
    if rc != SPKMC_OK:
        raise SpkmcError(rc, lib().spkmc_last_error().decode(errors="replace"))


def make_params(L, domain_edge=0, J=1.0, H=0.0, T=4.5115, seed=1, init=SPKMC_INIT_HOT,
                event_log_capacity=0, rmax_mode=SPKMC_RMAX_EXACT,
                sublattice=SPKMC_SUBLATTICE_8_ROTATING) -> spkmc_params:
    p = spkmc_params()
    lib().spkmc_params_init(ctypes.byref(p))
    p.L, p.domain_edge, p.J, p.H, p.T, p.seed = int(L), int(domain_edge), float(J), float(H), float(T), int(seed)
    p.init = int(init)
    p.event_log_capacity = int(event_log_capacity)
    p.rmax_mode = int(rmax_mode)
    p.sublattice = int(sublattice)
    return p


def make_config(stream=None, device=-1, ctas_per_sm=0, max_ctas=0, items_per_cta=0,
                barrier_timeout_ns=0, debug_skip_arrival_cta=-1) -> spkmc_config:
    c = spkmc_config()
    lib().spkmc_config_init(ctypes.byref(c))
    c.stream = stream
    c.device = int(device)
    c.ctas_per_sm = int(ctas_per_sm)
    c.max_ctas = int(max_ctas)
    c.items_per_cta = int(items_per_cta)
    c.barrier_timeout_ns = int(barrier_timeout_ns)
    c.debug_skip_arrival_cta = int(debug_skip_arrival_cta)
    return c


_keepalive = []


def torch_config(caching_allocator: bool = False, **kw) -> spkmc_config:
    """Config on torch's current CUDA stream (and optionally its caching
    allocator for all device memory the library holds)."""
    import torch
    dev = torch.cuda.current_device()
    stream = torch.cuda.current_stream(dev)
    c = make_config(stream=stream.cuda_stream, device=dev, **kw)
    if caching_allocator:
        def _alloc(nbytes, s, ctx):
            try:
                return torch.cuda.caching_allocator_alloc(int(nbytes), dev, s)
            except Exception:
                return None

        def _free(ptr, nbytes, s, ctx):
            torch.cuda.caching_allocator_delete(ptr)

        fa, ff = _abi.ALLOC_FN(_alloc), _abi.FREE_FN(_free)
        _keepalive.append((fa, ff))
        c.alloc, c.free = fa, ff
    return c


# ---------------------------------------------------------------------------
# Entry points with the C names (handles are ctypes.c_void_p)
# ---------------------------------------------------------------------------
def spkmc_params_init(p: spkmc_params) -> None:
    lib().spkmc_params_init(ctypes.byref(p))


def spkmc_config_init(c: spkmc_config) -> None:
    lib().spkmc_config_init(ctypes.byref(c))


def spkmc_rate_table(J: float, H: float, T: float) -> np.ndarray:
    out = np.zeros(14, dtype=np.float64)
    _check(lib().spkmc_rate_table(J, H, T, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return out


def spkmc_rmax_bounds(d: int, J: float, H: float, T: float):
    """(prescribed bound, learned growth margin) of Sec. 3.2 step 4b."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(lib().spkmc_rmax_bounds(int(d), J, H, T, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def spkmc_resolve_domain_edge(L: int) -> int:
    return int(lib().spkmc_resolve_domain_edge(int(L)))


def spkmc_bytes_required(p: spkmc_params) -> int:
    return int(lib().spkmc_bytes_required(ctypes.byref(p)))


def spkmc_create(L, domain_edge, J, H, T, seed) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(lib().spkmc_create(int(L), int(domain_edge), float(J), float(H), float(T), int(seed),
                              ctypes.byref(h)))
    return h


def spkmc_create_ex(p: spkmc_params, cfg: spkmc_config | None = None) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(lib().spkmc_create_ex(ctypes.byref(p), ctypes.byref(cfg) if cfg is not None else None,
                                 ctypes.byref(h)))
    return h


def spkmc_destroy(h) -> None:
    if h:
        lib().spkmc_destroy(h)


def spkmc_run_cycles(h, ncycles: int) -> None:
    _check(lib().spkmc_run_cycles(h, int(ncycles)))


def spkmc_synchronize(h) -> None:
    _check(lib().spkmc_synchronize(h))


def spkmc_observables(h) -> spkmc_obs:
    o = spkmc_obs()
    _check(lib().spkmc_observables(h, ctypes.byref(o)))
    return o


def spkmc_observables_async(h, out: spkmc_obs) -> spkmc_obs:
    """Enqueue the observables into ``out`` (read it after a synchronise;
    see obs_buffer for pinned storage)."""
    _check(lib().spkmc_observables_async(h, ctypes.byref(out)))
    return out


def spkmc_run_recorded(h, every: int, nrec: int, records) -> None:
    """Enqueue every * nrec cycles in one launch with the observables after
    every `every` cycles into records[0 .. nrec) (an obs_buffer; read it
    after a synchronise)."""
    if len(records) < nrec:
        raise ValueError("records holds fewer than nrec entries")
    _check(lib().spkmc_run_recorded(h, int(every), int(nrec),
                                    ctypes.cast(ctypes.addressof(records.records), ctypes.POINTER(spkmc_obs))))


def spkmc_batch_run_recorded(b, every: int, nrec: int, records) -> None:
    """Enqueue every * nrec cycles of all the batch's lattices in one launch,
    with the observables after every `every` cycles into
    records[slot * nrec + r] (an obs_buffer of capacity * nrec entries)."""
    _check(lib().spkmc_batch_run_recorded(b, int(every), int(nrec),
                                          ctypes.cast(ctypes.addressof(records.records), ctypes.POINTER(spkmc_obs))))


def spkmc_graph_create(h, cycles_per_step: int, steps: int, host_obs=None) -> ctypes.c_void_p:
    g = ctypes.c_void_p()
    obs = ctypes.cast(host_obs, ctypes.POINTER(spkmc_obs)) if host_obs is not None else None
    _check(lib().spkmc_graph_create(h, int(cycles_per_step), int(steps), obs, ctypes.byref(g)))
    return g


def spkmc_graph_launch(g) -> None:
    _check(lib().spkmc_graph_launch(g))


def spkmc_graph_destroy(g) -> None:
    lib().spkmc_graph_destroy(g)


class Graph:
    """A captured sequence of steps of one lattice (spkmc_graph_create):
    `steps` x (cycles_per_step cycles, then the observables into
    records[i] of an obs_buffer when one is given), replayed by launch()."""

    def __init__(self, lattice, cycles_per_step: int, steps: int, records=None):
        self.lattice = lattice
        self.records = records
        addr = ctypes.addressof(records.records) if records is not None else None
        self.g = spkmc_graph_create(lattice.h, cycles_per_step, steps, addr)

    def launch(self) -> None:
        spkmc_graph_launch(self.g)

    def close(self) -> None:
        if self.g:
            spkmc_graph_destroy(self.g)
            self.g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class obs_buffer:
    """An array of n spkmc_obs records in pinned host memory (through the
    PyTorch allocator; plain host memory without PyTorch), for
    spkmc_observables_async."""

    def __init__(self, n: int):
        size = ctypes.sizeof(spkmc_obs) * n
        try:
            import torch
            self._keep = torch.empty(size, dtype=torch.uint8, pin_memory=torch.cuda.is_available())
            addr = self._keep.data_ptr()
        except ImportError:
            self._keep = ctypes.create_string_buffer(size)
            addr = ctypes.addressof(self._keep)
        self.records = (spkmc_obs * n).from_address(addr)

    def __getitem__(self, i) -> spkmc_obs:
        return self.records[i]

    def __len__(self):
        return len(self.records)


def spkmc_get_spins(h, out: np.ndarray) -> np.ndarray:
    assert out.dtype == np.int8 and out.flags.c_contiguous
    _check(lib().spkmc_get_spins(h, out.ctypes.data, out.size))
    return out


def spkmc_set_spins(h, spins: np.ndarray) -> None:
    s = np.ascontiguousarray(spins, dtype=np.int8)
    _check(lib().spkmc_set_spins(h, s.ctypes.data, s.size))


def spkmc_get_spins_packed(h, out: np.ndarray) -> np.ndarray:
    """Spins as bits (np.packbits(spins > 0, bitorder='little') of the int8
    read-out) into a uint8 array of L^3 / 8 bytes."""
    assert out.dtype == np.uint8 and out.flags.c_contiguous
    _check(lib().spkmc_get_spins_packed(h, out.ctypes.data, out.size))
    return out


def spkmc_set_spins_packed(h, bits: np.ndarray) -> None:
    b = np.ascontiguousarray(bits, dtype=np.uint8)
    _check(lib().spkmc_set_spins_packed(h, b.ctypes.data, b.size))


def spkmc_get_event_log(h, cap: int) -> np.ndarray:
    buf = np.zeros(max(int(cap), 0), dtype=EVENT_DTYPE)
    n = ctypes.c_size_t()
    _check(lib().spkmc_get_event_log(h, buf.ctypes.data if cap > 0 else None, buf.size, ctypes.byref(n)))
    return buf[: n.value]


def spkmc_clear_event_log(h) -> None:
    _check(lib().spkmc_clear_event_log(h))


def spkmc_get_state(h) -> spkmc_state:
    st = spkmc_state()
    _check(lib().spkmc_get_state(h, ctypes.byref(st)))
    return st


def spkmc_set_state(h, st: spkmc_state) -> None:
    _check(lib().spkmc_set_state(h, ctypes.byref(st)))


def spkmc_class_counts(h, K: int) -> np.ndarray:
    out = np.zeros((K, 14), dtype=np.int32)
    _check(lib().spkmc_class_counts(h, out.ctypes.data, out.size))
    return out


def spkmc_check_counts(h) -> int:
    n = ctypes.c_int64()
    _check(lib().spkmc_check_counts(h, ctypes.byref(n)))
    return int(n.value)


def spkmc_info_get(h) -> spkmc_info:
    i = spkmc_info()
    _check(lib().spkmc_info_get(h, ctypes.byref(i)))
    return i


def spkmc_batch_create(capacity: int, cfg: spkmc_config | None = None) -> ctypes.c_void_p:
    b = ctypes.c_void_p()
    _check(lib().spkmc_batch_create(int(capacity), ctypes.byref(cfg) if cfg is not None else None,
                                    ctypes.byref(b)))
    return b


def spkmc_batch_destroy(b) -> None:
    if b:
        lib().spkmc_batch_destroy(b)


def spkmc_batch_admit(b, p: spkmc_params, cycles: int) -> int:
    slot = ctypes.c_int32()
    _check(lib().spkmc_batch_admit(b, ctypes.byref(p), int(cycles), ctypes.byref(slot)))
    return int(slot.value)


def spkmc_batch_run(b, cycles: int) -> None:
    _check(lib().spkmc_batch_run(b, int(cycles)))


def spkmc_batch_poll(b, cap: int = 4096) -> list:
    buf = (ctypes.c_int32 * max(cap, 1))()
    n = ctypes.c_int32()
    _check(lib().spkmc_batch_poll(b, buf, int(cap), ctypes.byref(n)))
    return [int(buf[i]) for i in range(n.value)]


def spkmc_batch_retire(b, slot: int) -> None:
    _check(lib().spkmc_batch_retire(b, int(slot)))


def spkmc_batch_synchronize(b) -> None:
    _check(lib().spkmc_batch_synchronize(b))


def spkmc_batch_observables(b, slot: int) -> spkmc_obs:
    o = spkmc_obs()
    _check(lib().spkmc_batch_observables(b, int(slot), ctypes.byref(o)))
    return o


def spkmc_batch_get_spins(b, slot: int, out: np.ndarray) -> np.ndarray:
    assert out.dtype == np.int8 and out.flags.c_contiguous
    _check(lib().spkmc_batch_get_spins(b, int(slot), out.ctypes.data, out.size))
    return out


def spkmc_batch_get_event_log(b, slot: int, cap: int) -> np.ndarray:
    buf = np.zeros(max(int(cap), 0), dtype=EVENT_DTYPE)
    n = ctypes.c_size_t()
    _check(lib().spkmc_batch_get_event_log(b, int(slot), buf.ctypes.data if cap > 0 else None, buf.size,
                                           ctypes.byref(n)))
    return buf[: n.value]


def spkmc_batch_observables_all(b, capacity: int):
    """Observables of all slots (list indexed by slot; L == 0 for free slots)."""
    arr = (spkmc_obs * max(int(capacity), 1))()
    n = ctypes.c_int32()
    _check(lib().spkmc_batch_observables_all(b, arr, int(capacity), ctypes.byref(n)))
    return [arr[i] for i in range(n.value)]


def spkmc_batch_usage(b):
    n = ctypes.c_int32()
    by = ctypes.c_int64()
    _check(lib().spkmc_batch_usage(b, ctypes.byref(n), ctypes.byref(by)))
    return int(n.value), int(by.value)


def spkmc_run_cycles_noalloc(p: spkmc_params, dev_spins_ptr: int, state: spkmc_state, ncycles: int,
                             stream=None) -> spkmc_state:
    """Cycles on a caller-owned device int8 spin buffer with no allocation
    (see include/spkmc.h); ``state`` is updated in place and returned."""
    _check(lib().spkmc_run_cycles_noalloc(ctypes.byref(p), ctypes.c_void_p(dev_spins_ptr), ctypes.byref(state),
                                          int(ncycles), stream))
    return state


def spkmc_last_error() -> str:
    return lib().spkmc_last_error().decode(errors="replace")


# ---------------------------------------------------------------------------
# Convenience wrappers
# ---------------------------------------------------------------------------
def with_launch(config: spkmc_config | None, items_per_cta: int, ctas_per_sm: int) -> spkmc_config:
    """A copy of ``config`` (or of the defaults) with the given launch geometry."""
    c = make_config() if config is None else spkmc_config.from_buffer_copy(config)
    c.items_per_cta, c.ctas_per_sm = int(items_per_cta), int(ctas_per_sm)
    return c


def tuned_config(L: int, domain_edge: int, config: spkmc_config | None = None):
    """``config`` with the autotuner's cached launch geometry for (L, d) filled
    in, when the caller set neither knob and the geometry was tuned on this
    device; otherwise ``config`` itself.  Geometry never changes results."""
    if config is not None and (config.items_per_cta or config.ctas_per_sm):
        return config
    from . import autotune
    d = int(domain_edge) or spkmc_resolve_domain_edge(int(L))
    hit = autotune.cached_launch(int(L), d)
    return config if hit is None else with_launch(config, *hit)


class Lattice:
    """One lattice on the GPU (owns a spkmc_t handle).  With ``tuned`` (the
    default) the autotuner's cached launch geometry is used when ``config``
    sets none."""

    def __init__(self, L, domain_edge=0, J=1.0, H=0.0, T=4.5115, seed=1, cold=False,
                 event_log_capacity=0, config: spkmc_config | None = None, rmax_mode=SPKMC_RMAX_EXACT,
                 sublattice=SPKMC_SUBLATTICE_8_ROTATING, tuned: bool = True):
        self.params = make_params(L, domain_edge, J, H, T, seed,
                                  SPKMC_INIT_COLD if cold else SPKMC_INIT_HOT, event_log_capacity, rmax_mode,
                                  sublattice)
        if tuned:
            config = tuned_config(L, domain_edge, config)
        self.config = config
        self.h = spkmc_create_ex(self.params, config)
        info = spkmc_info_get(self.h)
        self.L, self.d, self.K, self.K_act = info.L, info.domain_edge, info.K, info.K_act

    def run(self, ncycles: int) -> None:
        spkmc_run_cycles(self.h, ncycles)

    def synchronize(self) -> None:
        spkmc_synchronize(self.h)

    def observables(self) -> spkmc_obs:
        return spkmc_observables(self.h)

    def observables_async(self, out: spkmc_obs) -> spkmc_obs:
        return spkmc_observables_async(self.h, out)

    def run_recorded(self, every: int, nrec: int, records) -> None:
        spkmc_run_recorded(self.h, every, nrec, records)

    def graph(self, cycles_per_step: int, steps: int, records=None) -> "Graph":
        return Graph(self, cycles_per_step, steps, records)

    def spins(self) -> np.ndarray:
        return spkmc_get_spins(self.h, np.empty(self.L ** 3, dtype=np.int8))

    def set_spins(self, s) -> None:
        spkmc_set_spins(self.h, s)

    def spins_packed(self, out=None) -> np.ndarray:
        """The spins as L^3 / 8 bytes, one bit per site (1 = +1), little-endian
        bit order within a byte."""
        return spkmc_get_spins_packed(self.h, np.empty(self.L ** 3 // 8, dtype=np.uint8) if out is None else out)

    def set_spins_packed(self, bits) -> None:
        spkmc_set_spins_packed(self.h, bits)

    def event_log(self, cap=None) -> np.ndarray:
        return spkmc_get_event_log(self.h, self.params.event_log_capacity if cap is None else cap)

    def state(self) -> spkmc_state:
        return spkmc_get_state(self.h)

    def set_state(self, st: spkmc_state) -> None:
        spkmc_set_state(self.h, st)

    def class_counts(self) -> np.ndarray:
        return spkmc_class_counts(self.h, self.K)

    def check_counts(self) -> int:
        return spkmc_check_counts(self.h)

    def info(self) -> spkmc_info:
        return spkmc_info_get(self.h)

    def close(self) -> None:
        if self.h:
            spkmc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch:
    """Many independent lattices advanced by one persistent launch."""

    def __init__(self, capacity: int, config: spkmc_config | None = None):
        self.b = spkmc_batch_create(capacity, config)
        self.capacity = capacity
        self.params = {}

    def admit(self, L, domain_edge=0, J=1.0, H=0.0, T=4.5115, seed=1, cold=False, cycles=-1,
              event_log_capacity=0, rmax_mode=SPKMC_RMAX_EXACT, sublattice=SPKMC_SUBLATTICE_8_ROTATING) -> int:
        p = make_params(L, domain_edge, J, H, T, seed, SPKMC_INIT_COLD if cold else SPKMC_INIT_HOT,
                        event_log_capacity, rmax_mode, sublattice)
        slot = spkmc_batch_admit(self.b, p, cycles)
        self.params[slot] = p
        return slot

    def run(self, cycles: int) -> None:
        spkmc_batch_run(self.b, cycles)

    def poll(self) -> list:
        return spkmc_batch_poll(self.b, self.capacity)

    def retire(self, slot: int) -> None:
        spkmc_batch_retire(self.b, slot)
        self.params.pop(slot, None)

    def synchronize(self) -> None:
        spkmc_batch_synchronize(self.b)

    def observables(self, slot: int) -> spkmc_obs:
        return spkmc_batch_observables(self.b, slot)

    def spins(self, slot: int) -> np.ndarray:
        L = self.params[slot].L
        return spkmc_batch_get_spins(self.b, slot, np.empty(L ** 3, dtype=np.int8))

    def event_log(self, slot: int, cap=None) -> np.ndarray:
        c = self.params[slot].event_log_capacity if cap is None else cap
        return spkmc_batch_get_event_log(self.b, slot, c)

    def observables_all(self):
        return spkmc_batch_observables_all(self.b, self.capacity)

    def run_recorded(self, every: int, nrec: int, records=None):
        """every * nrec cycles in one launch with the observables after every
        `every` cycles: records[slot * nrec + r] of an obs_buffer of
        capacity * nrec entries (allocated if None; read it after
        synchronize())."""
        if records is None:
            records = obs_buffer(self.capacity * nrec)
        if len(records) < self.capacity * nrec:
            raise ValueError("records holds fewer than capacity * nrec entries")
        spkmc_batch_run_recorded(self.b, every, nrec, records)
        return records

    def usage(self):
        return spkmc_batch_usage(self.b)

    def close(self) -> None:
        if self.b:
            spkmc_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
