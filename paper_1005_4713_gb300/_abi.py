"""ctypes mirror of include/spkmc.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libspkmc.so")

SPKMC_OK = 0
SPKMC_EINVAL = 1
SPKMC_ENOMEM = 2
SPKMC_ECUDA = 3
SPKMC_ETIMEOUT = 4
SPKMC_EBUSY = 5
SPKMC_EINTERNAL = 6
SPKMC_EBOUND = 7
SPKMC_INIT_HOT = 0
SPKMC_INIT_COLD = 1
SPKMC_RMAX_EXACT = 0
SPKMC_RMAX_PRESCRIBED = 1
SPKMC_RMAX_LEARNED = 2
SPKMC_SUBLATTICE_8_ROTATING = 0
SPKMC_SUBLATTICE_2_RANDOM = 1

SPKMC_NOALLOC_SCRATCH_BYTES = 16 << 20

STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "EBUSY", 6: "EINTERNAL",
                7: "EBOUND"}

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class spkmc_params(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("domain_edge", ctypes.c_int32), ("J", ctypes.c_double),
                ("H", ctypes.c_double), ("T", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("init", ctypes.c_int32), ("rmax_mode", ctypes.c_int32),
                ("event_log_capacity", ctypes.c_int64), ("sublattice", ctypes.c_int32),
                ("reserved1", ctypes.c_int32)]


class spkmc_config(ctypes.Structure):
    _fields_ = [("stream", ctypes.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN),
                ("alloc_ctx", ctypes.c_void_p), ("device", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("max_ctas", ctypes.c_int32),
                ("items_per_cta", ctypes.c_int32), ("barrier_timeout_ns", ctypes.c_int64),
                ("debug_skip_arrival_cta", ctypes.c_int32), ("reserved1", ctypes.c_int32)]


class spkmc_obs(ctypes.Structure):
    _fields_ = [("cycle", ctypes.c_int64), ("clock", ctypes.c_double), ("M", ctypes.c_int64),
                ("B", ctypes.c_int64), ("E", ctypes.c_double), ("m", ctypes.c_double),
                ("m2", ctypes.c_double), ("m4", ctypes.c_double), ("n_flip", ctypes.c_int64),
                ("n_null", ctypes.c_int64), ("sum_null_rate", ctypes.c_double),
                ("sum_null_rate_fx", ctypes.c_uint64 * 2), ("L", ctypes.c_int32),
                ("domain_edge", ctypes.c_int32)]


class spkmc_event(ctypes.Structure):
    _fields_ = [("cycle", ctypes.c_int64), ("domain", ctypes.c_int32), ("cls", ctypes.c_int32),
                ("site", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class spkmc_state(ctypes.Structure):
    _fields_ = [("cycle", ctypes.c_int64), ("clock", ctypes.c_double), ("n_flip", ctypes.c_int64),
                ("n_null", ctypes.c_int64), ("sum_null_rate_fx", ctypes.c_uint64 * 2),
                ("rmax_hist", ctypes.c_double * 8)]


class spkmc_info(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("domain_edge", ctypes.c_int32), ("nd", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("K", ctypes.c_int64), ("K_act", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("grid_ctas", ctypes.c_int32),
                ("threads_per_cta", ctypes.c_int32)]


P = ctypes.POINTER
_h = ctypes.c_void_p
_i32, _i64, _u64, _dbl, _sz = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_size_t

# name -> (restype, argtypes), exactly the entry points declared in include/spkmc.h
PROTOTYPES = {
    "spkmc_params_init": (None, [P(spkmc_params)]),
    "spkmc_config_init": (None, [P(spkmc_config)]),
    "spkmc_rate_table": (ctypes.c_int, [_dbl, _dbl, _dbl, P(_dbl)]),
    "spkmc_rmax_bounds": (ctypes.c_int, [ctypes.c_int32, _dbl, _dbl, _dbl, P(_dbl), P(_dbl)]),
    "spkmc_resolve_domain_edge": (_i32, [_i32]),
    "spkmc_bytes_required": (_i64, [P(spkmc_params)]),
    "spkmc_create": (ctypes.c_int, [_i32, _i32, _dbl, _dbl, _dbl, _u64, P(_h)]),
    "spkmc_create_ex": (ctypes.c_int, [P(spkmc_params), P(spkmc_config), P(_h)]),
    "spkmc_destroy": (None, [_h]),
    "spkmc_run_cycles": (ctypes.c_int, [_h, _i64]),
    "spkmc_synchronize": (ctypes.c_int, [_h]),
    "spkmc_observables": (ctypes.c_int, [_h, P(spkmc_obs)]),
    "spkmc_observables_async": (ctypes.c_int, [_h, P(spkmc_obs)]),
    "spkmc_run_recorded": (ctypes.c_int, [_h, _i64, _i32, P(spkmc_obs)]),
    "spkmc_batch_run_recorded": (ctypes.c_int, [_h, _i64, _i32, P(spkmc_obs)]),
    "spkmc_graph_create": (ctypes.c_int, [_h, ctypes.c_int64, ctypes.c_int32, P(spkmc_obs), P(ctypes.c_void_p)]),
    "spkmc_graph_launch": (ctypes.c_int, [ctypes.c_void_p]),
    "spkmc_graph_destroy": (None, [ctypes.c_void_p]),
    "spkmc_get_spins": (ctypes.c_int, [_h, ctypes.c_void_p, _sz]),
    "spkmc_set_spins": (ctypes.c_int, [_h, ctypes.c_void_p, _sz]),
    "spkmc_get_spins_packed": (ctypes.c_int, [_h, ctypes.c_void_p, _sz]),
    "spkmc_set_spins_packed": (ctypes.c_int, [_h, ctypes.c_void_p, _sz]),
    "spkmc_get_event_log": (ctypes.c_int, [_h, ctypes.c_void_p, _sz, P(_sz)]),
    "spkmc_clear_event_log": (ctypes.c_int, [_h]),
    "spkmc_get_state": (ctypes.c_int, [_h, P(spkmc_state)]),
    "spkmc_set_state": (ctypes.c_int, [_h, P(spkmc_state)]),
    "spkmc_class_counts": (ctypes.c_int, [_h, ctypes.c_void_p, _sz]),
    "spkmc_check_counts": (ctypes.c_int, [_h, P(_i64)]),
    "spkmc_info_get": (ctypes.c_int, [_h, P(spkmc_info)]),
    "spkmc_batch_create": (ctypes.c_int, [_i32, P(spkmc_config), P(_h)]),
    "spkmc_batch_destroy": (None, [_h]),
    "spkmc_batch_admit": (ctypes.c_int, [_h, P(spkmc_params), _i64, P(_i32)]),
    "spkmc_batch_run": (ctypes.c_int, [_h, _i64]),
    "spkmc_batch_poll": (ctypes.c_int, [_h, P(_i32), _i32, P(_i32)]),
    "spkmc_batch_retire": (ctypes.c_int, [_h, _i32]),
    "spkmc_batch_synchronize": (ctypes.c_int, [_h]),
    "spkmc_batch_observables": (ctypes.c_int, [_h, _i32, P(spkmc_obs)]),
    "spkmc_batch_get_spins": (ctypes.c_int, [_h, _i32, ctypes.c_void_p, _sz]),
    "spkmc_batch_get_event_log": (ctypes.c_int, [_h, _i32, ctypes.c_void_p, _sz, P(_sz)]),
    "spkmc_batch_observables_all": (ctypes.c_int, [_h, P(spkmc_obs), _i32, P(_i32)]),
    "spkmc_batch_usage": (ctypes.c_int, [_h, P(_i32), P(_i64)]),
    "spkmc_run_cycles_noalloc": (ctypes.c_int, [P(spkmc_params), ctypes.c_void_p, P(spkmc_state), _i64,
                                                 ctypes.c_void_p]),
    "spkmc_last_error": (ctypes.c_char_p, []),
}


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libspkmc.so and attach the prototypes.  Raises if it is missing:
    there is no other implementation of the hot path."""
    if not os.path.exists(path):
        raise RuntimeError(f"libspkmc.so not built at {path}; run paper_1005_4713_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in PROTOTYPES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib
