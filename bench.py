#!/usr/bin/env python3
"""Benchmark of the spkMC cycle on the 1024^3 Ising lattice (16^3-site domains).

Metric: spin-flip events per second, null events included (one event per
active domain per cycle, arXiv:1005.4713 Sec. 3.1 step 4).  A step is one
pass of the whole hot path over the lattice: 10 spkMC cycles (every colour
visited in turn) plus the observables M, E, M^2, M^4, as in the 500-cycle
run with observables every 10 cycles.  The timed steps run as one persistent
launch that records each step's observables on the device
(spkmc_run_recorded); the same steps launched one at a time, and replayed
from a CUDA graph, are reported beside it.

Arms:
  default           the CUDA library through its C ABI (this package);
  --impl reference  the CPU oracle on the host cores (no GPU), one cycle per
                    step, same lattice and metric.

Multi-GPU (torchrun, one rank per GPU): independent replicas with their own
seeds, no collective on the data path (weak scaling); rank 0 prints the line.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L_BENCH, D_BENCH, SEED_BENCH = 1024, 16, 3
CYCLES_PER_STEP = 10
# Algorithmic bytes per event of this design (restated from the paper's
# linear frequency-line pass, Sec. 5): the domain's 14 class counts (int32)
# plus its spins and one-site halo bit-packed, (d^3 + 6 d^2)/8 bytes.
def bytes_per_event(d: int) -> int:
    return 14 * 4 + (d ** 3 + 6 * d * d) // 8


def int8_bytes_per_event(d: int) -> int:
    return d ** 3 + 6 * d * d


# The bytes a design would move if it staged only what the site search reads:
# the count line, the d/2 planes of the chosen half, the plane beyond them and
# that half's x, y and z ghost words (this design stages the whole block before
# the half is known, to hide the copies under step 1).
def half_domain_floor_bytes(d: int) -> int:
    half = d // 2
    plane = d * d // 8
    ghosts = (2 * half * d + 2 * half * d + d * d) // 8
    return 14 * 4 + half * plane + plane + ghosts


# ---------------------------------------------------------------------------
# Clock sampling (NVML through ctypes, falling back to nvidia-smi)
# ---------------------------------------------------------------------------
REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
           0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown", 0x2: "applications_clocks",
           0x1: "gpu_idle", 0x10: "sync_boost", 0x100: "display_clock"}


class ClockSampler:
    def __init__(self, device_index: int = 0, period_s: float = 0.002):
        self.period = period_s
        self.samples = []  # (t, sm_mhz, reasons_mask)
        self.max_mhz = None
        self._stop = threading.Event()
        self._thread = None
        self._smi = None
        self._nvml = None
        self._handle = ctypes.c_void_p()
        try:
            nv = ctypes.CDLL("libnvidia-ml.so.1")
            if nv.nvmlInit_v2() != 0:
                raise OSError("nvmlInit failed")
            handle = ctypes.c_void_p()
            bus = self._pci_bus_id(device_index)
            rc = 1
            if bus:
                rc = nv.nvmlDeviceGetHandleByPciBusId_v2(bus.encode(), ctypes.byref(handle))
            if rc != 0:
                rc = nv.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(device_index), ctypes.byref(handle))
            if rc != 0:
                raise OSError("no NVML handle")
            mx = ctypes.c_uint()
            if nv.nvmlDeviceGetMaxClockInfo(handle, 1, ctypes.byref(mx)) == 0:
                self.max_mhz = int(mx.value)
            self._nvml, self._handle = nv, handle
        except OSError:
            self._nvml = None

    @staticmethod
    def _pci_bus_id(idx):
        try:
            import torch
            return getattr(torch.cuda.get_device_properties(idx), "pci_bus_id", None)
        except Exception:
            return None

    def _read(self):
        nv, h = self._nvml, self._handle
        clk = ctypes.c_uint()
        rs = ctypes.c_ulonglong()
        nv.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(clk))
        fn = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            nv.nvmlDeviceGetCurrentClocksThrottleReasons
        fn(h, ctypes.byref(rs))
        return int(clk.value), int(rs.value)

    def _loop(self):
        while not self._stop.is_set():
            try:
                c, r = self._read()
                self.samples.append((time.perf_counter(), c, r))
            except Exception:
                pass
            time.sleep(self.period)

    def start(self):
        if self._nvml is not None:
            self._thread = threading.Thread(target=self._loop, daemon=True)
            self._thread.start()
        else:
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active")
            try:
                self._smi = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                              "-lms", "50"], stdout=subprocess.PIPE, text=True)
            except OSError:
                self._smi = None
        return self

    def stop(self):
        self._stop.set()
        if self._thread:
            self._thread.join()
        if self._smi:
            self._smi.terminate()
            out, _ = self._smi.communicate()
            for line in out.splitlines():
                parts = [p.strip() for p in line.split(",")]
                try:
                    self.samples.append((0.0, int(float(parts[1])), int(parts[4], 16)))
                    self.max_mhz = int(float(parts[2]))
                except (ValueError, IndexError):
                    pass

    def summary(self, t0=None, t1=None):
        s = [x for x in self.samples if t0 is None or (t0 <= x[0] <= t1) or x[0] == 0.0]
        if not s:
            s = self.samples
        if not s:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": [], "samples": 0}
        mask = 0
        for _, _, r in s:
            mask |= r
        names = sorted(n for b, n in REASONS.items() if mask & b and n != "gpu_idle")
        return {"sm_mhz": statistics.median(c for _, c, _ in s), "sm_max_mhz": self.max_mhz,
                "reasons": names, "samples": len(s)}


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------
def dist_setup(n_gpus):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if os.environ.get("SPKMC_BENCH_BACKEND", "nccl") == "nccl" else "gloo"
        dist.init_process_group(backend=backend)
        pg = dist
    return world, rank, local, pg


def replica_seed(rank: int) -> int:
    """Replicas (one lattice per GPU) differ only in their seed."""
    return SEED_BENCH + rank


def max_over_ranks(value: float, pg, device=None) -> float:
    if pg is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def barrier(pg, device=None):
    if pg is None:
        return
    if device is not None:
        pg.barrier(device_ids=[device.index])
    else:
        pg.barrier()


def _code_text(src: str) -> str:
    """The code of a C++ source without its comments (string and character
    literals kept as they are), one stripped line per non-empty line."""
    out, i, n, quote = [], 0, len(src), None
    while i < n:
        c = src[i]
        if quote:
            out.append(c)
            if c == "\\" and i + 1 < n:
                out.append(src[i + 1])
                i += 2
                continue
            if c == quote:
                quote = None
            i += 1
        elif c in "\"'":
            quote = c
            out.append(c)
            i += 1
        elif src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        else:
            out.append(c)
            i += 1
    lines = (line.strip() for line in "".join(out).splitlines())
    return "\n".join(line for line in lines if line)


def kernel_source_hash() -> str:
    """Hash of the code the cycle kernel is compiled from (its translation
    unit and the headers it includes), without comments or blank lines: an
    edit of a comment leaves the captured traffic of the kernel valid."""
    h = hashlib.sha256()
    for f in ("spkmc_kernels.cu", "spkmc_device.cuh", "spkmc_internal.h"):
        with open(os.path.join(ROOT, "paper_1005_4713_gb300", "csrc", f), encoding="utf-8") as fh:
            h.update(f.encode() + b"\0" + _code_text(fh.read()).encode() + b"\0")
    return h.hexdigest()[:16]


def measured_peak():
    for path in (os.path.join(ROOT, "MEASURED_PEAKS.json"),):
        try:
            with open(path) as f:
                j = json.load(f)
            return float(j["hbm_gbs"]), "measured"
        except (OSError, KeyError, ValueError):
            pass
    return 6800.0, "fallback"


def ncu_traffic(workload: str, cycles: int):
    """DRAM bytes of one launch of the cycle kernel over `cycles` cycles, from
    the committed ncu capture (scaled by the cycles: every cycle moves the
    same blocks and count lines), only if it was taken on the current kernel
    source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            j = json.load(f)
    except (OSError, ValueError):
        return None
    e = j.get(workload)
    if not e or e.get("kernel_source_hash") != kernel_source_hash():
        return None
    return round(e["dram_bytes_per_launch"] * cycles / e["cycles_per_launch"])


def cpu_baseline(rank: int, world: int, cycles: int = 8):
    import oracle
    cores = os.cpu_count() or 1
    st = oracle.State(L_BENCH, D_BENCH, 1.0, 0.0, 4.5115, SEED_BENCH)
    t0 = time.perf_counter()
    st.run(cycles, threads=cores)
    dt = time.perf_counter() - t0
    return {"value": cycles * st.k_act / dt, "unit": "events/s", "cores": cores, "kind": "oracle",
            "sample": f"{L_BENCH}^3, d={D_BENCH}, hot start seed {SEED_BENCH}, cycles 0..{cycles - 1} "
                      f"(one visit of each colour), OpenMP over active domains, {dt:.2f} s"}


def cpu_baseline_extras(cycles_128: int = 40):
    """The oracle single-threaded on one cycle of the 1024^3 lattice, and on
    all cores on the 128^3 lattice with 8^3-site domains."""
    import oracle
    cores = os.cpu_count() or 1
    st = oracle.State(L_BENCH, D_BENCH, 1.0, 0.0, 4.5115, SEED_BENCH)
    t0 = time.perf_counter()
    st.run(1, threads=1)
    dt1 = time.perf_counter() - t0
    st2 = oracle.State(128, 8, 1.0, 0.0, 4.5115, 2)
    t0 = time.perf_counter()
    st2.run(cycles_128, threads=cores)
    dt2 = time.perf_counter() - t0
    return {"single_thread": {"value": st.k_act / dt1, "unit": "events/s", "cores": 1,
                              "sample": f"cycle 0 of {L_BENCH}^3, d={D_BENCH}, {dt1:.2f} s"},
            "config_128_d8": {"value": cycles_128 * st2.k_act / dt2, "unit": "events/s", "cores": cores,
                              "sample": f"{cycles_128} cycles of 128^3, d=8, hot start seed 2, {dt2:.2f} s"}}


def small_configs(cfg, stream, every=100, nrec=20):
    """Cycles of the two small lattices that live in L2 and shared memory
    (16^3 with 4^3-site domains, 128^3 with 8^3-site domains), bound by the
    per-cycle latency: microseconds per cycle and events/s of one recorded
    launch of every * nrec cycles, CUDA events on the launch stream."""
    import torch

    import paper_1005_4713_gb300 as sp

    out = {}
    for name, (L, d, seed) in (("config_16_d4", (16, 4, 1)), ("config_128_d8", (128, 8, 2))):
        with sp.Lattice(L, d, 1.0, 0.0, 4.5115, seed, config=cfg) as lat:
            rec = sp.obs_buffer(nrec)
            lat.run_recorded(every, nrec, rec)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lat.run_recorded(every, nrec, rec)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            cycles = every * nrec
            out[name] = {"us_per_cycle": ms * 1e3 / cycles, "events_per_s": cycles * lat.K_act / (ms / 1e3),
                         "events_per_cycle": lat.K_act, "cycles": cycles}
    return out


def binder_table(binder, t_edges=(4.40, 4.45, 4.50, 4.55, 4.60)):
    """Binder cumulant U = 1 - <m^4>/(3 <m^2>^2) (Eq. 7 and the cumulant form)
    per lattice edge and temperature bin: the mean over the lattices in the
    bin and its standard error."""
    import numpy as np
    rows = []
    for L in sorted({b["L"] for b in binder}):
        for lo, hi in zip(t_edges[:-1], t_edges[1:]):
            us = [b["U"] for b in binder if b["L"] == L and lo <= b["T"] < hi + (1e-12 if hi == t_edges[-1] else 0)
                  and b["U"] is not None]
            if us:
                rows.append({"L": L, "T_lo": lo, "T_hi": hi, "n": len(us), "U": float(np.mean(us)),
                             "err": float(np.std(us, ddof=1) / np.sqrt(len(us))) if len(us) > 1 else None})
    return rows


def batched_summary(n_lattices=256, cycles=5000):
    """Ensemble of uneven lattices in one persistent launch per chunk against
    the same lattices run one at a time with the single-lattice path: all of
    them, each bit-equal.  The domain edge of each L is the autotuner's (most
    flips per second), the batch's launch geometry too (least time per
    cycle); both are measured on this GPU first."""
    import paper_1005_4713_gb300 as sp  # noqa: F401
    from paper_1005_4713_gb300 import autotune, ensemble
    from paper_1005_4713_gb300 import workloads as wl
    Ls = [s.L for s in wl.ensemble_specs(n_lattices)]
    edges = autotune.edge_map(Ls)
    specs = wl.ensemble_specs(n_lattices, domain_edge=lambda L: edges[L])
    launch = autotune.tune_batch(specs)
    bat = ensemble.run_batched(specs, cycles, sample_every=50, burn_in=cycles // 5)
    solo = ensemble.run_one_at_a_time(specs, cycles, sample_every=50, burn_in=cycles // 5)
    same = [a == b for a, b in zip(solo.final, bat.final)]
    if not all(same):
        raise RuntimeError(f"batched results differ from the solo runs for {same.count(False)} lattices")
    return {"workload": f"{n_lattices} lattices, L in {{16..128}}, T~U[4.40,4.60], H in {{0,0.01}}, {cycles} cycles",
            "edges": {str(k): v for k, v in edges.items()},
            "edge_objective": "flips_per_s (null events excluded), measured per L on this GPU",
            "edge_trials": autotune.edge_report(Ls),
            "launch": {"items_per_cta": launch["items_per_cta"], "ctas_per_sm": launch["ctas_per_sm"],
                       "objective": launch["objective"]},
            "batched_s": bat.seconds, "batched_events_per_s": bat.events_per_s,
            "batched_flips_per_s": bat.flips_per_s,
            "solo_all_s": solo.seconds, "solo_events_per_s": solo.events_per_s, "solo_flips_per_s": solo.flips_per_s,
            "speedup_vs_solo": solo.seconds / bat.seconds,
            "bit_exact_vs_solo": f"{len(same)} of {len(same)} lattices",
            "binder_U_by_L_T": binder_table(bat.binder),
            "binder_note": "U per lattice from samples every 50 cycles after 1000 cycles; at 5000 cycles the "
                           "larger lattices have not relaxed, so this is a throughput workload, not an "
                           "estimate of the critical point (the crossing is measured on L = 8, 12, 16)"}


def served_summary(n_requests=2000, rate=200.0, budget=120 << 30, step_cycles=100, sweep=(25, 100, 400),
                   sweep_requests=400):
    """Poisson stream of simulation requests served with continuous batching,
    against the same requests served one at a time with the plain
    single-lattice path on the same arrival times; every result bit-equal.
    A short sweep of the cycles per batch step on the first requests."""
    from paper_1005_4713_gb300 import serve
    from paper_1005_4713_gb300 import workloads as wl
    reqs = wl.request_stream(n=n_requests, rate=rate)
    srv = serve.Server(budget_bytes=budget, capacity=512, step_cycles=step_cycles)
    st = srv.serve(reqs, realtime=True)
    one = serve.serve_one_at_a_time(reqs, realtime=True)
    mine = {c.rid: c.obs for c in st.completions}
    same = sum(1 for c in one.completions if mine.get(c.rid) == c.obs)
    if same != len(one.completions):
        raise RuntimeError(f"served results differ from the one-at-a-time runs for {len(one.completions) - same}")

    def arm(x):
        return {"completed": len(x.completions), "p50_latency_s": x.latency_percentile(50),
                "p99_latency_s": x.latency_percentile(99), "events_per_s": x.events_per_s, "wall_s": x.wall,
                "p50_breakdown": x.breakdown(50), "p99_breakdown": x.breakdown(99), "by_L": x.by_size()}

    sw = []
    for sc in sweep:
        x = serve.Server(budget_bytes=budget, capacity=512, step_cycles=sc).serve(reqs[:sweep_requests], realtime=True)
        sw.append({"step_cycles": sc, "p50_latency_s": x.latency_percentile(50),
                   "p99_latency_s": x.latency_percentile(99), "events_per_s": x.events_per_s, "steps": x.steps})
    cb = arm(st)
    cb.update(rejected=len(st.rejected), peak_live=st.peak_live, steps=st.steps, step_cycles=step_cycles)
    oa = arm(one)
    return {"workload": f"{n_requests} requests, Poisson {rate:g}/s, L in {{32,64,128,256}}, T~U[4.3,4.7], "
                        f"cycles log-uniform 1e2..1e4, budget {budget >> 30} GiB",
            "continuous_batching": cb, "one_at_a_time": oa,
            "speedup": {"events_per_s": st.events_per_s / one.events_per_s,
                        "p50_latency": oa["p50_latency_s"] / cb["p50_latency_s"],
                        "p99_latency": oa["p99_latency_s"] / cb["p99_latency_s"]},
            "bit_exact_vs_one_at_a_time": f"{same} of {len(one.completions)} requests",
            "step_cycles_sweep": {"requests": sweep_requests, "runs": sw}}


# ---------------------------------------------------------------------------
# arms
# ---------------------------------------------------------------------------
def variants_summary(cfg, stream, steps, cps):
    """Variants of Sec. 3.2 on the same workload.  The R_max bounds of step
    4b (learned, prescribed): the launch has no grid barrier before the
    events.  The paper's two random colours of step 4a: half of the domains
    active per cycle, each recounted at its visit.  Events/s counts nulls
    like the headline; flips/s and the useful fraction (flips / events) say
    what a bound costs in null events."""
    import torch

    import paper_1005_4713_gb300 as sp

    out = {}
    for name, kw in (("learned", dict(rmax_mode=sp.SPKMC_RMAX_LEARNED)),
                     ("prescribed", dict(rmax_mode=sp.SPKMC_RMAX_PRESCRIBED)),
                     ("two_colour", dict(sublattice=sp.SPKMC_SUBLATTICE_2_RANDOM))):
        with sp.Lattice(L_BENCH, D_BENCH, 1.0, 0.0, 4.5115, SEED_BENCH, config=cfg, **kw) as lat:
            rec = sp.obs_buffer(max(steps, 3))
            lat.run_recorded(cps, 3, rec)
            o0 = lat.observables()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lat.run_recorded(cps, steps, rec)
            e1.record(stream)
            torch.cuda.synchronize()
            s = e0.elapsed_time(e1) / 1e3
            o = lat.observables()
            nf, nn = o.n_flip - o0.n_flip, o.n_null - o0.n_null
            out[name] = {"events_per_s": (nf + nn) / s, "flips_per_s": nf / s,
                         "useful_fraction": nf / (nf + nn), "us_per_cycle": s / (steps * cps) * 1e6,
                         "events_per_cycle": lat.K_act}
    return out


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    import oracle
    cores = os.cpu_count() or 1
    st = oracle.State(L_BENCH, D_BENCH, 1.0, 0.0, 4.5115, SEED_BENCH)
    for _ in range(args.warmup):
        st.run(1, threads=cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        st.run(1, threads=cores)
    dt = time.perf_counter() - t0
    value = args.steps * st.k_act / dt
    line = {
        "impl": "reference", "metric": "spin-flip events/s (incl. null) at 1024^3",
        "value": value, "unit": "events/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u1 spins, int32 counts, f64 clock",
        "data": "synthetic (hot start from Philox)",
        "config": {"workload": "spkmc-1024^3-d16", "L": L_BENCH, "domain_edge": D_BENCH, "J": 1.0,
                   "H": 0.0, "T": 4.5115, "seed": SEED_BENCH, "cycles_per_step": 1,
                   "impl": "CPU oracle (plain C, FP64), OpenMP over active domains"},
        "cpu_baseline": {"value": value, "unit": "events/s", "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} cycles of the {L_BENCH}^3 lattice after "
                                   f"{args.warmup} warm-up cycles"},
        "e2e": {"value": value, "unit": "events/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line))
    return 0


def run_gpu(args, world, rank, local, pg):
    import numpy as np
    import torch

    import paper_1005_4713_gb300 as sp

    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    # a stream of our own (the legacy default stream has handle 0, which the
    # library would replace by a private stream that these events cannot see)
    stream = torch.cuda.Stream(device)
    torch.cuda.set_stream(stream)
    cfg = sp.torch_config()
    seed = replica_seed(rank)
    lat = sp.Lattice(L_BENCH, D_BENCH, 1.0, 0.0, 4.5115, seed, config=cfg)
    kact = lat.K_act
    cps = args.cycles_per_step

    # one step = cps cycles and the observables after them.  The timed steps
    # run as one recorded launch: the kernel records each step's observables
    # on the device (no host synchronisation, no launch per step) and one
    # copy brings the records to pinned host memory
    obs_rec = sp.obs_buffer(max(args.steps, args.warmup))
    lat.run_recorded(cps, args.warmup, obs_rec)
    torch.cuda.synchronize(device)
    barrier(pg, device)
    torch.cuda.synchronize(device)

    obs0 = lat.observables()
    sampler = ClockSampler(local).start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    t_host0 = time.perf_counter()
    e0.record(stream)
    lat.run_recorded(cps, args.steps, obs_rec)
    e1.record(stream)
    torch.cuda.synchronize(device)
    torch.cuda.synchronize(device)
    t_host1 = time.perf_counter()
    barrier(pg, device)
    sampler.stop()
    ms = e0.elapsed_time(e1)
    # the cycle kernel's launch: the events also hold the two one-pass record
    # kernels and the records' copy (a few microseconds)
    kernel_ms = ms
    ms_max = max_over_ranks(ms, pg, device)
    events = world * args.steps * cps * kact
    value = events / (ms_max / 1e3)
    lat_info = lat.info()
    obs1 = lat.observables()
    last = obs_rec[args.steps - 1]
    if (last.cycle, last.M, last.B, last.clock) != (obs1.cycle, obs1.M, obs1.B, obs1.clock):
        raise RuntimeError("recorded observables differ from the synchronous read-out")
    flips = obs1.n_flip - obs0.n_flip
    useful = flips / max(1, (obs1.n_flip + obs1.n_null) - (obs0.n_flip + obs0.n_null))

    # the same steps launched one at a time (a persistent launch and an
    # asynchronous observables record per step)
    per_step = None
    if not args.no_graph:
        for i in range(2):
            lat.run(cps)
            lat.observables_async(obs_rec[i])
        torch.cuda.synchronize(device)
        k0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        k1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        p0 = torch.cuda.Event(enable_timing=True)
        p1 = torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        for i in range(args.steps):
            k0[i].record(stream)
            lat.run(cps)
            k1[i].record(stream)
            lat.observables_async(obs_rec[i])
        p1.record(stream)
        torch.cuda.synchronize(device)
        pms = p0.elapsed_time(p1)
        per_step = {"value": world * args.steps * cps * kact / (max_over_ranks(pms, pg, device) / 1e3),
                    "unit": "events/s", "ms_per_step": pms / args.steps,
                    "kernel_ms_per_launch": sum(a.elapsed_time(b) for a, b in zip(k0, k1)) / args.steps,
                    "note": "one cycle-kernel launch and one observables record per step"}
    graph = None
    if not args.no_graph and (args.steps * cps) % 2 == 0:
        # the same steps captured once in a CUDA graph and replayed with one
        # host launch (CUDA events around the replay)
        graph_rec = sp.obs_buffer(args.steps)
        g = lat.graph(cps, args.steps, graph_rec)
        g.launch()  # warm-up replay
        torch.cuda.synchronize(device)
        ge0 = torch.cuda.Event(enable_timing=True)
        ge1 = torch.cuda.Event(enable_timing=True)
        ge0.record(stream)
        g.launch()
        ge1.record(stream)
        torch.cuda.synchronize(device)
        gms = ge0.elapsed_time(ge1)
        g.close()
        graph = {"value": world * args.steps * cps * kact / (max_over_ranks(gms, pg, device) / 1e3),
                 "unit": "events/s", "ms_per_step": gms / args.steps,
                 "note": "the per-step launches captured in one CUDA graph (cycles + observables per step)"}

    # end to end through the C ABI with host buffers: upload the start
    # lattice from pinned memory (one bit per site), run the steps with their
    # recorded observables, read the final lattice back (one bit per site);
    # the same with one int8 per site is reported beside it
    e2e = None
    if not args.no_e2e:
        n = L_BENCH ** 3
        obs_bytes = ctypes.sizeof(sp.spkmc_obs)
        lat2 = sp.Lattice(L_BENCH, D_BENCH, 1.0, 0.0, 4.5115, seed, cold=True, config=cfg)

        def timed(upload, download, host, out):
            upload(host)
            lat2.run(cps)
            lat2.observables()
            barrier(pg, device)
            torch.cuda.synchronize(device)
            t0 = time.perf_counter()
            upload(host)
            lat2.run_recorded(cps, args.steps, obs_rec)
            download(out)  # synchronises: the records have landed
            t1 = time.perf_counter()
            barrier(pg, device)
            return max_over_ranks(t1 - t0, pg, device)

        bits = torch.empty(n // 8, dtype=torch.uint8, pin_memory=True).numpy()
        lat.spins_packed(bits)
        bits_out = torch.empty(n // 8, dtype=torch.uint8, pin_memory=True).numpy()
        s_bits = timed(lat2.set_spins_packed, lat2.spins_packed, bits, bits_out)
        host = torch.empty(n, dtype=torch.int8, pin_memory=True).numpy()
        host[:] = lat.spins()
        out = torch.empty(n, dtype=torch.int8, pin_memory=True).numpy()
        s_int8 = timed(lat2.set_spins, lambda o: sp.spkmc_get_spins(lat2.h, o), host, out)
        e2e = {"value": events / s_bits, "unit": "events/s",
               "h2d_bytes_per_step": n // 8 // args.steps,
               "d2h_bytes_per_step": n // 8 // args.steps + obs_bytes,
               "spins": "one bit per site (spkmc_set_spins_packed / spkmc_get_spins_packed), page-locked host "
                        "buffers read and written in place by the transposing kernels",
               "int8_spins": {"value": events / s_int8, "h2d_bytes_per_step": n // args.steps,
                              "d2h_bytes_per_step": n // args.steps + obs_bytes}}
        lat2.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(rank, world)
        cpu.update(cpu_baseline_extras())
    small = small_configs(cfg, stream) if rank == 0 and world == 1 else None
    batched = served = variants = None
    if rank == 0 and world == 1 and not args.no_ensembles:
        batched = batched_summary()
        served = served_summary()
    if rank == 0 and world == 1 and not args.no_variants:
        variants = variants_summary(cfg, stream, args.steps, cps)

    if rank == 0:
        peak, peak_kind = measured_peak()
        bpe = bytes_per_event(D_BENCH)
        launch_cycles = args.steps * cps
        per_launch = launch_cycles * kact * bpe
        achieved = per_launch / (kernel_ms / 1e3) / 1e9
        clocks = sampler.summary(t_host0, t_host1)
        line = {
            "metric": "spin-flip events/s (incl. null) at 1024^3",
            "value": value, "unit": "events/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "u1 spins (bit-packed), int32 counts, f64 rates and clock",
            "data": "synthetic (hot start from Philox, seed 3 + rank)",
            "config": {"workload": "spkmc-1024^3-d16", "L": L_BENCH, "domain_edge": D_BENCH,
                       "J": 1.0, "H": 0.0, "T": 4.5115, "seed": SEED_BENCH,
                       "cycles_per_step": cps, "events_per_cycle": kact,
                       "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                       "l2": "working set %.0f MB > 126 MB L2, no flush" % (lat_info.device_bytes / 1e6),
                       "grid_ctas": lat_info.grid_ctas, "threads_per_cta": lat_info.threads_per_cta},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": ncu_traffic("spkmc-1024^3-d16", launch_cycles),
                         "peak_kind": peak_kind, "kernel": "spkmc_cycles_kernel",
                         "bytes_per_event": bpe, "kernel_ms_per_launch": kernel_ms,
                         "frac_vs_half_domain_floor": launch_cycles * kact * half_domain_floor_bytes(D_BENCH)
                         / (kernel_ms / 1e3) / 1e9 / peak,
                         "half_domain_floor_bytes_per_event": half_domain_floor_bytes(D_BENCH),
                         "cycles_per_launch": launch_cycles,
                         "int8_equivalent_GBps": launch_cycles * kact * int8_bytes_per_event(D_BENCH) / (kernel_ms / 1e3) / 1e9},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": 3,  # record set-up, the persistent cycle kernel, record read-out
            "clocks": clocks,
            "exact_rmax": {"flips_per_s": flips * world / (ms_max / 1e3), "useful_fraction": useful},
            "per_step_launches": per_step,
            "graph": graph,
            "variants": variants,
            "small_configs": small,
            "batched": batched,
            "served": served,
        }
        print(json.dumps(line))
    lat.close()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--cycles-per-step", type=int, default=CYCLES_PER_STEP)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ensembles", action="store_true", help="skip the batched and served summaries")
    ap.add_argument("--no-graph", action="store_true", help="skip the per-step launches and their CUDA-graph replay")
    ap.add_argument("--no-variants", "--no-bounds", dest="no_variants", action="store_true",
                    help="skip the R_max-bound and two-colour summaries")
    ap.add_argument("--only-small", action="store_true",
                    help="time only the 16^3 and 128^3 lattices (no contract line; for profiling)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.only_small:
        import torch

        import paper_1005_4713_gb300 as sp
        torch.cuda.set_device(0)
        stream = torch.cuda.Stream()
        torch.cuda.set_stream(stream)
        print(json.dumps({"small_configs": small_configs(sp.torch_config(), stream)}))
        return 0
    world, rank, local, pg = dist_setup(args.gpus)
    try:
        if args.impl == "reference":
            return run_reference(args, world, rank)
        return run_gpu(args, world, rank, local, pg)
    finally:
        if pg is not None:
            pg.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
