#!/usr/bin/env python
"""Far-field maps/s at 1e-8 relative residual on the 2D 1025x1025 workload.

Workload (one "step"): four far-field maps on [-20,20]^2, rotation pi/6,
chi = -exp(-|x|^2/4), k in {5, 10, 20, 40}, eta = +x: for each k the
scattered wave is solved to ||b - A u|| <= 1e-8 ||b|| (FP32 red-black
Gauss-Seidel V(1,1) cycles inside an FP64 iterative refinement -- FP64 outer
residual, update and coarsest-grid solve -- 8 levels, 9x9 coarsest grid) and
its far field evaluated at 720 equispaced outgoing angles.  Inputs are
synthetic (analytic potential and plane waves).

Prints one JSON line (rank 0).  --impl reference times the CPU FP64 oracle on
the same workload instead (its four solves in full, the far field on a
quarter of the angles, on the host cores).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import threading
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

KS = W.MIXED_2D_KS
METRIC = "far-field maps/s at 1e-8 residual"
UNIT = "maps/s"
WORKLOAD = "2D 1025x1025 on [-20,20]^2, rotation pi/6, chi=-exp(-|x|^2/4), k in {5,10,20,40}, 720 angles"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


# FP64 FMA throughput of this part, measured with an FMA-loop kernel
# (0.599e12 DFMA/s over 152 SMs; 2 flops per FMA).
FP64_PEAK_TFLOPS = 1.198
# FP32 operation rate derived from unit counts and clock: 152 SMs x 128 FP32
# lanes x 2.07 GHz (a packed two-lane instruction counts two operations).  The
# double-float contraction spends 36 FP32 operations (three double-float
# multiply-adds of 12, Gauss's complex product) per complex multiply-add, i.e.
# 4.5 per FP64-equivalent flop (8 per complex multiply-add), so its arithmetic
# ceiling in FP64-equivalent flops is that rate / 4.5.
FP32_INSTR_PER_S = 152 * 128 * 2.07e9
DF_INSTR_PER_FLOP = 36.0 / 8.0
DF_PEAK_TFLOPS = FP32_INSTR_PER_S / DF_INSTR_PER_FLOP / 1e12
# DRAM bytes (read + write) per launch of the dominant kernels, from one ncu
# capture of the current kernels on this workload (None when no capture of
# the current kernels exists): the double-float far-field contraction and the
# fused FP32 V(1,1) tiles (all levels, and those of the 1025^2 level).
FF_DF_DRAM_BYTES = 10.67e6
TILES_DRAM_BYTES = 0.223e6
TILES_FINE_DRAM_BYTES = 0.771e6


# FP32 V-cycles per refinement step on the headline workload (at most, with
# the adaptive schedule).  With the double-float refinement a sweep of 3, 4, 5,
# 6, 8 fixed cycles gave 522, 543, 530, 549, 533 maps/s: each step is a graph
# launch and a host round trip for its norm, and a solve stops only after a
# step.  Sizing each step from the previous step's reduction factor (the
# default) gave 652 (at most 6) and 656 (at most 8) against 635 fixed, same box.
# With the FP64 refinement each step also costs an FP64-bound residual pass:
# caps of 6, 8, 10, 12 gave 648, 664, 682, 682 maps/s with the same cycle
# counts (18, 24, 28, 27) and fewer steps.
INNER_CYCLES = 10
# concurrent plans (streams and host threads) sharing the 3D step's directions
GROUPS_3D = 4


def _cases(precision, ks=None, inner=INNER_CYCLES, adaptive=False, refine_fp64=False):
    out = []
    for k in (ks or KS):
        c = W.mixed_2d(k)
        c["opts"]["precision"] = precision
        c["opts"]["inner_cycles"] = inner
        c["opts"]["adaptive_inner"] = int(adaptive and precision == "mixed")
        c["opts"]["refine_fp64"] = int(refine_fp64 and precision == "mixed")
        out.append(c)
    return out


def _config(args, extra=None):
    cfg = {"workload": WORKLOAD, "maps_per_step": len(KS), "n": 1025, "levels": 8, "angles": 720,
           "rel_tol": 1e-8, "smoother": "rbgs V(1,1)", "precision": args.precision,
           "inner_cycles": args.inner_cycles if args.precision == "mixed" else None,
           "adaptive_inner": bool(args.adaptive_inner) if args.precision == "mixed" else None,
           "refinement": ("fp64 (outer residual, update and coarsest solve in FP64)" if args.refine_fp64
                          else "double-float") if args.precision == "mixed" else None,
           "l2": "flushed between timed steps (512 MiB write)", "parallelism": f"replicas x{args.gpus}",
           "concurrency": ("the maps of a step solved one after another" if args.sequential else
                           "the maps of a step solved concurrently: one host thread and one CUDA stream per map")}
    if extra:
        cfg.update(extra)
    return cfg


class _Nvml:
    """The read-only NVML calls the clock sampler needs, through ctypes (the
    driver's libnvidia-ml; no Python package needed): the SM clock, its
    maximum and the clock-event (throttle) reason bits of one device."""
    SM = 1                                   # NVML_CLOCK_SM
    REASONS = ((0x8, "hw_slowdown"), (0x40, "hw_thermal_slowdown"), (0x20, "sw_thermal_slowdown"),
               (0x4, "sw_power_cap"))

    def __init__(self, index, pci_bus_id=None):
        import ctypes
        self.ct = ctypes
        lib = ctypes.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        h = ctypes.c_void_p()
        rc = 1
        if pci_bus_id:
            rc = lib.nvmlDeviceGetHandleByPciBusId_v2(pci_bus_id.encode(), ctypes.byref(h))
        if rc != 0:
            rc = lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(index), ctypes.byref(h))
        if rc != 0:
            lib.nvmlShutdown()
            raise OSError("no NVML handle for the device")
        self.lib, self.h = lib, h
        self.reasons_fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            getattr(lib, "nvmlDeviceGetCurrentClocksThrottleReasons")
        mx = ctypes.c_uint()
        self.max_mhz = mx.value if lib.nvmlDeviceGetMaxClockInfo(h, self.SM, ctypes.byref(mx)) == 0 else None

    def sample(self):
        c, r = self.ct.c_uint(), self.ct.c_ulonglong()
        if self.lib.nvmlDeviceGetClockInfo(self.h, self.SM, self.ct.byref(c)) != 0:
            return None
        bits = r.value if self.reasons_fn(self.h, self.ct.byref(r)) == 0 else 0
        return c.value, [n for b, n in self.REASONS if bits & b]

    def close(self):
        self.lib.nvmlShutdown()


def _pci_bus_id(dev_index):
    """NVML's bus-id string of a CUDA device, from torch's properties (None
    where this torch does not report them)."""
    try:
        import torch
        p = torch.cuda.get_device_properties(dev_index)
        return f"{p.pci_domain_id:08X}:{p.pci_bus_id:02X}:{p.pci_device_id:02X}.0"
    except Exception:
        return None


class ClockSampler:
    """SM clocks and throttle reasons sampled during the timed region: NVML
    every 10 ms from a thread (ctypes releases the GIL during the calls), or
    nvidia-smi every 200 ms where NVML cannot be loaded."""

    def __init__(self, index, dev_index=None):
        self.index = index
        self.dev_index = index if dev_index is None else dev_index
        self.p = None
        self.nvml = None

    def _poll(self):
        while not self.stop.is_set():
            x = self.nvml.sample()
            if x is not None:
                self.samples.append(x)
            self.stop.wait(0.01)

    def __enter__(self):
        try:
            self.nvml = _Nvml(self.index, _pci_bus_id(self.dev_index))
        except Exception:
            self.nvml = None
        if self.nvml is not None:
            self.samples = []
            self.stop = threading.Event()
            self.thread = threading.Thread(target=self._poll, daemon=True)
            self.thread.start()
            return self
        q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        self.result = None
        if self.nvml is not None:
            self.stop.set()
            self.thread.join()
            self.nvml.close()
            if self.samples:
                sm = [x[0] for x in self.samples]
                self.result = {"sm_mhz": statistics.median(sm),
                               "sm_max_mhz": self.nvml.max_mhz if self.nvml.max_mhz else max(sm),
                               "samples": len(sm), "reasons": sorted({n for x in self.samples for n in x[1]}),
                               "source": "NVML every 10 ms during the timed steps"}
            return
        if self.p is None:
            return
        time.sleep(0.25)
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
            out, _ = self.p.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 6:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[2:6]):
                if v.lower() == "active":
                    reasons.add(n)
        if sm:
            self.result = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                           "reasons": sorted(reasons), "source": "nvidia-smi every 200 ms"}


# ---------------------------------------------------------------------------
# reference arm: the CPU FP64 oracle on the host cores
# ---------------------------------------------------------------------------
ORACLE_ANGLE_STRIDE = 4      # the oracle's far field runs on every 4th of the 720 angles


def _oracle_solve(k):
    """Worker: the oracle's RB-GS V(1,1) solve of one map to 1e-8 (one thread)."""
    from oracle import csff_oracle as O
    c = W.mixed_2d(k)
    p = O.problem_from_dict(c["problem"])
    t0 = time.perf_counter()
    res = O.mg_solve(p, O.rhs(p, c["eta"][0]), O.opts_from_dict(c["opts"]))
    return res.u, time.perf_counter() - t0, res.cycles


def _oracle_far_field(k, u, idx):
    """Worker: the oracle's far-field sum of one map at the angles idx."""
    from oracle import csff_oracle as O
    c = W.mixed_2d(k)
    p = O.problem_from_dict(c["problem"])
    t0 = time.perf_counter()
    O.far_field(p, u, c["eta"][0], c["alphas"][idx])
    return time.perf_counter() - t0


class OracleStep:
    """The step's four maps by the oracle on the host cores: a pool of
    single-threaded worker processes (spawned, so safe after CUDA use) solves
    the four maps at once, then evaluates their far fields at every
    ORACLE_ANGLE_STRIDE-th angle, split over all workers.  run() returns the
    measured wall time, the time with the far-field phase scaled to all 720
    angles (only the angles are scaled), and the summed single-thread task
    times (the same work on one core)."""

    def __init__(self, workers=None):
        import multiprocessing as mp
        self.workers = int(workers or min(os.cpu_count() or 1, 16))
        for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[v] = "1"          # inherited by the spawned workers: one thread each
        self.pool = mp.get_context("spawn").Pool(self.workers)

    def close(self):
        self.pool.close()
        self.pool.join()

    def run(self):
        t0 = time.perf_counter()
        solves = self.pool.map(_oracle_solve, KS)
        t1 = time.perf_counter()
        idx = np.arange(0, 720, ORACLE_ANGLE_STRIDE)
        per_map = max(1, self.workers // len(KS))
        tasks = [(k, u, ch) for k, (u, _, _) in zip(KS, solves) for ch in np.array_split(idx, per_map)]
        ff = self.pool.starmap(_oracle_far_field, tasks)
        t2 = time.perf_counter()
        return {"wall_s": t2 - t0, "solve_wall_s": t1 - t0, "ff_wall_s": t2 - t1,
                "scaled_s": (t1 - t0) + (t2 - t1) * ORACLE_ANGLE_STRIDE,
                "single_thread_s": sum(x[1] for x in solves) + sum(ff) * ORACLE_ANGLE_STRIDE,
                "solve_s": [round(x[1], 3) for x in solves], "cycles": [x[2] for x in solves]}


ORACLE_SAMPLE = ("the step's four maps (k = 5, 10, 20, 40) by the FP64 oracle: each RB-GS V(1,1) solve to 1e-8 in "
                 "full, in its own single-threaded worker process; the far fields at every 4th of the 720 angles, "
                 "split over the workers, their time scaled by 4 (only the angles are scaled)")


def cpu_baseline_record(r, workers):
    """cpu_baseline entry from one OracleStep.run() result r."""
    return {"value": len(KS) / r["scaled_s"], "unit": UNIT, "cores": workers, "kind": "oracle",
            "sample": ORACLE_SAMPLE,
            "single_thread": {"value": len(KS) / r["single_thread_s"], "unit": UNIT, "cores": 1,
                              "how": "the summed times of the single-threaded worker tasks (far-field part "
                                     "scaled by 4)"},
            "detail": {k: r[k] for k in ("wall_s", "solve_wall_s", "ff_wall_s", "solve_s", "cycles")}}


def max_over_ranks(x: float, dist, device) -> float:
    """The largest x over the ranks of the process group (x itself without one)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Units all ranks processed (each rank the same share) per second of the
    slowest rank: the whole-job throughput of a weak-scaling run."""
    return units_per_rank * world / seconds


def run_reference(args, rank, world):
    """The oracle on this host's cores, each step one OracleStep.run() of the
    headline workload; printed by rank 0 only.  ms_per_step is the measured
    wall time of a step; value scales only the far-field angles."""
    if rank != 0:
        return
    runner = OracleStep()
    try:
        for _ in range(args.warmup):
            runner.run()
        runs = [runner.run() for _ in range(args.steps)]
    finally:
        runner.close()
    scaled = sum(r["scaled_s"] for r in runs) / len(runs)
    value = len(KS) / scaled
    rec = cpu_baseline_record({**runs[-1], "scaled_s": scaled,
                               "single_thread_s": sum(r["single_thread_s"] for r in runs) / len(runs)},
                              runner.workers)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(r["wall_s"] for r in runs) / len(runs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": _config(args),
            "cpu_baseline": rec,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args, rank, world, local_rank):
    import torch
    import paper_1211_4461_gb300 as csff

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
    stream = torch.cuda.current_stream()
    ks = tuple(float(k) for k in args.ks.split(",")) if args.ks else KS
    cases = _cases(args.precision, ks, args.inner_cycles, args.adaptive_inner, args.refine_fp64)
    # one stream and one host thread per map: the four solves are independent
    # and each alone leaves most SMs idle on its coarse levels
    streams = [torch.cuda.Stream(device=dev) for _ in cases]
    t0 = time.perf_counter()
    plans = [csff.Plan(c["problem"], c["opts"], stream=st) for c, st in zip(cases, streams)]
    torch.cuda.synchronize()
    plan_ms = (time.perf_counter() - t0) * 1e3
    N = plans[0].N
    us = [torch.zeros(N, dtype=torch.complex128, device=dev) for _ in cases]
    Fs = [torch.zeros(720, dtype=torch.complex128, device=dev) for _ in cases]
    Fe = [torch.zeros(720, dtype=torch.int32, device=dev) for _ in cases]
    # host-side inputs/outputs for the end-to-end measurement, in pinned memory
    eta_h = [torch.from_numpy(np.ascontiguousarray(c["eta"])).pin_memory() for c in cases]
    al_h = [torch.from_numpy(np.ascontiguousarray(c["alphas"])).pin_memory() for c in cases]
    F_h = [torch.zeros(720, dtype=torch.complex128).pin_memory() for _ in cases]
    Fe_h = [torch.zeros(720, dtype=torch.int32).pin_memory() for _ in cases]
    flush = torch.empty(512 * 2 ** 20, dtype=torch.uint8, device=dev)
    infos = {}

    def one_map(i, e2e):
        p, c = plans[i], cases[i]
        with torch.cuda.stream(streams[i]):
            eta = eta_h[i].numpy() if e2e else c["eta"]
            al = al_h[i].numpy() if e2e else c["alphas"]
            st, info = p.solve(eta, us[i], ok=(csff.OK,))
            infos[i] = info[0]
            p.far_field(eta, us[i], al, Fs[i], Fe[i])
            if e2e:
                F_h[i].copy_(Fs[i], non_blocking=True)
                Fe_h[i].copy_(Fe[i], non_blocking=True)

    def step(e2e=False, concurrent=not args.sequential):
        start = torch.cuda.Event()
        start.record(stream)
        for st in streams:
            st.wait_event(start)
        if concurrent:
            th = [threading.Thread(target=one_map, args=(i, e2e)) for i in range(len(plans))]
            for t in th:
                t.start()
            for t in th:
                t.join()
        else:
            for i in range(len(plans)):
                one_map(i, e2e)
        for st in streams:
            stream.wait_stream(st)
        if e2e:
            stream.synchronize()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # ---- timed region (device time, CUDA events on the launching stream) ----
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = csff.kernel_launches()
    step_ms = []
    with ClockSampler(local_rank) as clk:
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    launches = csff.kernel_launches() - launches0
    if dist:
        dist.barrier()
    total_ms = max_over_ranks(sum(step_ms), dist, dev)
    value = whole_job_rate(len(cases) * args.steps, world, total_ms / 1e3)

    # ---- the dominant kernels alone: one sequential step timing only the
    # fused FP32 V(1,1) tile launches (the largest share of device time) and the
    # far-field contraction launches (CUDA events on each launch's stream) ----
    flush.zero_()
    torch.cuda.synchronize()
    csff.prof_begin(csff.PROF_TILES32 | csff.PROF_TILES32_FINE | csff.PROF_FF_CONTRACT)
    step(concurrent=False)
    torch.cuda.synchronize()
    prof_timed = csff.prof_end()
    # fraction of the contraction each map's launch computed (negligible
    # blocks are skipped; the rest of the algorithmic flops were not executed)
    ff_work = [p.far_field_work() for p in plans]

    # ---- per-family breakdown (one extra sequential profiled step) ----------
    flush.zero_()
    torch.cuda.synchronize()
    csff.prof_begin(csff.PROF_FF_CONTRACT | csff.PROF_MG32 | csff.PROF_MG64)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    step(concurrent=False)
    e1.record(stream)
    torch.cuda.synchronize()
    breakdown = csff.prof_end()
    breakdown_step_ms = e0.elapsed_time(e1)

    # ---- end to end through the public API with host buffers ----------------
    for _ in range(2):
        step(e2e=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step(e2e=True)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist, dev)
    e2e_val = whole_job_rate(len(cases) * args.steps, world, e2e_s)
    h2d = sum(int(eta_h[i].numel() * 8 + al_h[i].numel() * 8) for i in range(len(cases)))
    d2h = sum(int(F_h[i].numel() * 16 + Fe_h[i].numel() * 4) for i in range(len(cases)))

    if rank != 0:
        return
    peaks = _peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    ff = prof_timed["ff_contract"]
    ff_avg_ms = ff["ms"] / max(1, ff["launches"])
    ff_flops_all = ff["alg_flops"] / max(1, ff["launches"])
    ff_flops = ff_flops_all * sum(ff_work) / max(1, len(ff_work))      # executed, per launch
    achieved_tf = ff_flops / (ff_avg_ms * 1e-3) / 1e12 if ff_avg_ms > 0 else 0.0
    def tiles_roofline(rec, traffic, kernel, note):
        avg = rec["ms"] / max(1, rec["launches"])
        byt = rec["alg_bytes"] / max(1, rec["launches"])
        gbs = byt / (avg * 1e-3) / 1e9 if avg > 0 else 0.0
        return {"kernel": kernel, "bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                "traffic": traffic, "peak_source": "measured HBM copy bandwidth (burst; each launch timed alone)",
                "avg_launch_ms": avg, "launches": rec["launches"], "alg_bytes_per_launch": byt, "note": note}

    fine = prof_timed["tiles32_fine"]
    allt = prof_timed["tiles32"]
    rest = {k: allt[k] - fine[k] for k in ("launches", "ms", "alg_bytes")}
    alg_note = ("algorithmic bytes = 8 B x (3 fine-level points + 1 coarse point) per launch (iterate and right-hand "
                "side read, iterate written, coarse right-hand side or correction); each launch bracketed by CUDA "
                "events on its stream in a step run one map after another (in the timed step the maps' kernels "
                "overlap on four streams)")
    roofline = tiles_roofline(fine, TILES_FINE_DRAM_BYTES,
                              "k_down2 / k_up2 on the 1025^2 level (fused FP32 V(1,1) red-black tiles of 16 coarse "
                              "points; the largest share of the step's device time)",
                              alg_note + "; the 1025^2 level's FP32 arrays (8.4 MB each) stay in the 129 MB L2 "
                                         "through a V-cycle, so this fraction measures algorithmic throughput")
    roofline_levels = {"1025": roofline,
                       "513_to_65": tiles_roofline(rest, None, "k_down2 / k_up2 on the 513^2 ... 65^2 levels",
                                                   alg_note + "; these launches last about one CTA's lifetime"),
                       "all": tiles_roofline(allt, TILES_DRAM_BYTES, "k_down2 / k_up2, every fused level",
                                             alg_note)}
    roofline_ff = {"kernel": "k_ff_stage1_df (double-float far-field contraction)", "bound": "alu",
                "achieved": achieved_tf, "peak": DF_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved_tf / DF_PEAK_TFLOPS, "traffic": FF_DF_DRAM_BYTES,
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2.07 GHz / 4.5 FP32 operations per "
                               "FP64-equivalent flop (36 per complex multiply-add: three double-float "
                               "multiply-adds, Gauss's product; a packed two-lane instruction counts two)",
                "avg_launch_ms": ff_avg_ms, "launches": ff["launches"],
                "alg_flops_per_launch": ff_flops_all, "executed_flops_per_launch": ff_flops,
                "executed_fraction_per_map": ff_work,
                "note": "achieved counts the executed flops: blocks whose terms stay below 2^-55 of each "
                        "far-field value's sum of term magnitudes are skipped"}
    mg32, mg64 = breakdown["mg32"], breakdown["mg64"]
    cycles = sum(infos[i]["cycles"] for i in infos)
    vc = {"fp32_kernels_ms": mg32["ms"], "fp32_alg_bytes": mg32["alg_bytes"],
          "fp32_achieved_gbs": mg32["alg_bytes"] / (mg32["ms"] * 1e-3) / 1e9 if mg32["ms"] else 0.0,
          # mixed: the double-float refinement kernels; fp64: the FP64 V-cycles
          ("refine" if args.precision == "mixed" else "fp64") + "_kernels_ms": mg64["ms"],
          ("refine" if args.precision == "mixed" else "fp64") + "_achieved_gbs":
              mg64["alg_bytes"] / (mg64["ms"] * 1e-3) / 1e9 if mg64["ms"] else 0.0,
          "hbm_peak_gbs": hbm, "fp32_vcycles_per_step": cycles,
          "step_ms_profiled": breakdown_step_ms, "ff_contract_ms": breakdown["ff_contract"]["ms"]}
    vc["fp32_hbm_frac"] = vc["fp32_achieved_gbs"] / hbm
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32" if args.precision == "mixed" else "f64",
            "data": "synthetic", "config": _config(args, {"plan_ms": plan_ms}),
            "roofline": roofline, "roofline_levels": roofline_levels, "roofline_ff_contraction": roofline_ff,
            "vcycle": vc,
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": int(launches),
            "clocks": clk.result,
            "solve": {str(ks[i]): {"cycles": infos[i]["cycles"], "refinements": infos[i]["refinements"],
                                   "rel_res": infos[i]["rel_res"]} for i in infos}}
    if args.variants:
        line["variants"] = measure_variants(csff, torch, dev, stream, flush, total_ms / args.steps)
    if args.cpu_baseline and world == 1:
        runner = OracleStep()
        try:
            r = runner.run()
        finally:
            runner.close()
        line["cpu_baseline"] = cpu_baseline_record(r, runner.workers)
    print(json.dumps(line), flush=True)


def _time_events(torch, stream, fn, flush, reps):
    ms = []
    for _ in range(reps):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    return sum(ms) / len(ms)


def _concurrent_maps(csff, torch, dev, stream, flush, cases, reps=3):
    """The four maps of `cases` scheduled as the headline step (one host thread
    and CUDA stream per map); returns (ms per step, cycles per map)."""
    streams = [torch.cuda.Stream(device=dev) for _ in cases]
    plans = [csff.Plan(c["problem"], c["opts"], stream=st) for c, st in zip(cases, streams)]
    N = plans[0].N
    us = [torch.zeros(N, dtype=torch.complex128, device=dev) for _ in cases]
    Fs = [torch.zeros(720, dtype=torch.complex128, device=dev) for _ in cases]
    Fe = [torch.zeros(720, dtype=torch.int32, device=dev) for _ in cases]
    cyc = {}

    def one(i):
        p, c = plans[i], cases[i]
        with torch.cuda.stream(streams[i]):
            _, info = p.solve(c["eta"], us[i])
            cyc[i] = (info[0]["cycles"], info[0]["rel_res"])
            p.far_field(c["eta"], us[i], c["alphas"], Fs[i], Fe[i])

    def step():
        start = torch.cuda.Event()
        start.record(stream)
        for st in streams:
            st.wait_event(start)
        th = [threading.Thread(target=one, args=(i,)) for i in range(len(plans))]
        for t in th:
            t.start()
        for t in th:
            t.join()
        for st in streams:
            stream.wait_stream(st)

    for _ in range(3):
        step()
    ms = _time_events(torch, stream, step, flush, reps)
    for p in plans:
        p.close()
    return ms, [cyc[i][0] for i in range(len(cases))], [cyc[i][1] for i in range(len(cases))]


def measure_variants(csff, torch, dev, stream, flush, headline_ms):
    """The same four maps with the double-float refinement and in plain FP64
    (V-cycles in FP64), and the 64-instance uneven batch solved in one
    persistent launch against the same instances solved one after the other
    through the single-problem mixed path."""
    out = {}
    ms, cyc, rel = _concurrent_maps(csff, torch, dev, stream, flush,
                                    _cases("mixed", inner=INNER_CYCLES, adaptive=True, refine_fp64=False))
    out["double_float_refinement"] = {
        "value": len(KS) / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "cycles": cyc, "rel_res": rel,
        "speedup_vs_headline": headline_ms / ms,
        "note": "outer residual and update in double-float (pairs of FP32 words, about 48 bits) on the FP32 "
                "pipes, coarsest solve in FP32; same stopping test; its solutions re-checked to 1e-11 with "
                "the oracle's FP64 operator in the tests"}
    ms, cyc, rel = _concurrent_maps(csff, torch, dev, stream, flush, _cases("fp64"), reps=2)
    out["fp64_plain"] = {"value": len(KS) / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "cycles": cyc,
                         "rel_res": rel, "headline_speedup_vs_fp64_plain": ms / headline_ms}
    # ---- 64 uneven instances
    bc = W.batch_2d(64, seed=4461)
    for c in bc:
        c["opts"].update(precision="mixed", inner_cycles=INNER_CYCLES, adaptive_inner=1, coarsest_n=5)
    eta = np.vstack([c["eta"] for c in bc])
    al = [c["alphas"] for c in bc]
    b = csff.Batch([c["problem"] for c in bc], bc[0]["opts"], stream=stream)
    tc, per = b.autotune(eta)
    Fb = [torch.zeros(720, dtype=torch.complex128, device=dev) for _ in bc]
    Eb = [torch.zeros(720, dtype=torch.int32, device=dev) for _ in bc]
    binfo = {}

    def batch_step():
        _, inf = b.solve(eta)
        binfo["inf"] = inf
        b.far_field(eta, al, Fb, Eb)

    batch_step()
    ms_b = _time_events(torch, stream, batch_step, flush, 3)
    ms_bs = _time_events(torch, stream, lambda: b.solve(eta), flush, 3)
    sizes = {}
    for c in bc:
        sizes[c["problem"]["n"]] = sizes.get(c["problem"]["n"], 0) + 1
    out["batched_64"] = {"value": len(bc) / (ms_b / 1e3), "unit": UNIT, "ms_per_step": ms_b,
                         "solve_ms": ms_bs, "autotuned": {"tile_coarse_points": tc, "ctas_per_sm": per},
                         "sizes": {str(k): v for k, v in sorted(sizes.items())},
                         "all_converged": all(x["rel_res"] <= 1e-8 for x in binfo["inf"]),
                         "cycles_total": int(sum(x["cycles"] for x in binfo["inf"]))}
    b.close()
    # the same instances, one plan at a time: the single-problem mixed path
    # with the batch's iteration (FP64 refinement, adaptive schedule), then the
    # plain FP64 V-cycles (the plain GPU form) to the same tolerance
    def one_at_a_time(opts_update):
        sp = [csff.Plan(c["problem"], dict(c["opts"], **opts_update), stream=stream) for c in bc]
        su = [torch.zeros(p.N, dtype=torch.complex128, device=dev) for p in sp]
        cyc = {}

        def seq_step():
            for i, (p, c) in enumerate(zip(sp, bc)):
                _, inf = p.solve(c["eta"], su[i])
                cyc[i] = inf[0]["cycles"]
                p.far_field(c["eta"], su[i], c["alphas"], Fb[i], Eb[i])

        seq_step()
        ms = _time_events(torch, stream, seq_step, flush, 2)
        for p in sp:
            p.close()
        return ms, int(sum(cyc.values()))

    ms_s, cyc_s = one_at_a_time({"refine_fp64": 1})
    out["sequential_64"] = {"value": len(bc) / (ms_s / 1e3), "unit": UNIT, "ms_per_step": ms_s,
                            "cycles_total": cyc_s}
    out["batched_speedup_vs_sequential"] = ms_s / ms_b
    ms_p, cyc_p = one_at_a_time({"precision": "fp64"})
    out["plain_fp64_64"] = {"value": len(bc) / (ms_p / 1e3), "unit": UNIT, "ms_per_step": ms_p,
                            "cycles_total": cyc_p,
                            "note": "the same 64 instances by plain FP64 V-cycles to 1e-8, one after another"}
    out["batched_mixed_speedup_vs_plain_fp64"] = ms_p / ms_b
    out["batched_learned"] = measure_batched_learned(csff, torch, dev, stream, flush, bc, ms_p, ms_b)
    out["3d_257_16dirs"] = measure_3d(csff, torch, dev, stream, flush)
    out["vcycle_4097"] = measure_vcycle_bandwidth(csff, torch, dev, stream, flush)
    out["learned_2049"] = measure_learned(csff, torch, dev, stream, flush)
    out["gmres3_table2"] = measure_gmres_table2(csff, torch, dev, stream, flush)
    out["partial_wave_fig8"] = measure_partial_wave(csff, torch, dev, stream, flush)
    return out


def measure_batched_learned(csff, torch, dev, stream, flush, bc, ms_plain, ms_batched):
    """The combined form: the 64 uneven instances in one persistent launch
    with FP32 cycles inside the FP64 refinement and the learned step ending
    every cycle on each instance's finest level (the network trained on the GPU
    on residual patches of 257^2 problems at k h = 1.17, 32 seeded solves),
    against the plain FP64 V-cycles one instance after another (ms_plain) and
    the classical batched form (ms_batched), maps with far fields, all at 1e-8.
    Instances far from the network's k h hand themselves back to plain cycles
    (the fallback); a second batch of 16 instances at the network's k h
    (n in {257, 513, 1025}, k = 7.5 (n-1)/256) shows the cycle saving where the
    network applies."""
    from paper_1211_4461_gb300 import learned as LR
    opts = {"smoother": "rbgs", "omega": 1.0, "nu1": 1, "nu2": 1, "coarsest_n": 5, "rel_tol": 1e-8,
            "max_cycles": 400, "inner_cycles": 3}
    data = LR.collect_patches(_learned_problems(32, 7.5), opts, n_cycles=5, patch=64, per_field=6, seed=1)
    net = csff.Net(LR.init_weights(7))
    LR.train(net, data, steps=1000, batch=32, lr=2e-3, margin=4, seed=2)
    out = {}

    def run(cases, learned, far_field):
        eta = np.vstack([c["eta"] for c in cases])
        b = csff.Batch([c["problem"] for c in cases], cases[0]["opts"], stream=stream)
        if learned:
            b.set_learned(net)
        tc, per = b.autotune(eta)
        Fs = [torch.zeros(720, dtype=torch.complex128, device=dev) for _ in cases]
        Es = [torch.zeros(720, dtype=torch.int32, device=dev) for _ in cases]
        info = {}

        def step():
            _, inf = b.solve(eta)
            info["inf"] = inf
            if far_field:
                b.far_field(eta, [c["alphas"] for c in cases], Fs, Es)

        step()
        ms = _time_events(torch, stream, step, flush, 3)
        inf = info["inf"]
        b.close()
        return {"value": len(cases) / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
                "autotuned": {"tile_coarse_points": tc, "ctas_per_sm": per},
                "all_converged": all(x["rel_res"] <= 1e-8 for x in inf),
                "cycles_total": int(sum(x["cycles"] for x in inf)),
                "fell_back": int(sum(1 for x in inf if x["flags"] & 2))}

    out["config4_64"] = run(bc, True, True)
    out["config4_64"]["speedup_vs_plain_fp64"] = ms_plain / out["config4_64"]["ms_per_step"]
    out["config4_64"]["speedup_vs_batched_classical"] = ms_batched / out["config4_64"]["ms_per_step"]
    kh = W.batch_2d(16, seed=11, sizes=(257, 513, 1025))
    for c in kh:
        c["problem"]["k"] = 7.5 * (c["problem"]["n"] - 1) / 256
        c["opts"].update(precision="mixed", inner_cycles=3, coarsest_n=5, refine_fp64=1)
    out["kh117_16_classical"] = run(kh, False, False)
    out["kh117_16_learned"] = run(kh, True, False)
    out["kh117_16_learned"]["speedup_vs_classical"] = (out["kh117_16_classical"]["ms_per_step"] /
                                                       out["kh117_16_learned"]["ms_per_step"])
    out["note"] = ("solve and far field per step for config4_64, solve only for the k h = 1.17 batch (fixed "
                   "three cycles a refinement step in both of its forms); the learned step costs a residual "
                   "pass, the network pass and two grid barriers per cycle")
    net.close()
    return out


def measure_3d(csff, torch, dev, stream, flush):
    """257^3 on [-15,15]^3, k = 4, 16 incident directions, 64 x 32 angles,
    FP32-inner / FP64 refinement (the 2D headline's adaptive schedule of at
    most INNER_CYCLES cycles a step).  The step as the workload states it: the far field's
    z-contraction on the tensor cores (four-term BF16 splits, FP32 accumulation
    in tensor memory).  Scheduled like the 2D headline: four plans of four
    directions each, every plan on its own CUDA stream and host thread (the
    small levels' launches of one plan hide under another's fine-level work);
    one plan solving the sixteen directions in turn beside it, and the
    concurrent step with the FP64-class sum-factorised far field; then the far
    field alone in both modes and the relative L2 distance of their maps; last
    the concurrent step with the double-float refinement."""
    c = W.big_3d(n=257, n_rhs=16)
    c["opts"].update(precision="mixed", refine_fp64=1, inner_cycles=INNER_CYCLES, adaptive_inner=1)
    nr, na = c["eta"].shape[0], c["alphas"].shape[0]
    G = GROUPS_3D
    streams = [torch.cuda.Stream(device=dev) for _ in range(G)]
    plans = [csff.Plan(c["problem"], c["opts"], stream=st) for st in streams]
    N = plans[0].N
    per = nr // G
    us = [torch.zeros(per * N, dtype=torch.complex128, device=dev) for _ in range(G)]
    Fs = [torch.zeros(per * na, dtype=torch.complex128, device=dev) for _ in range(G)]
    Es = [torch.zeros(per * na, dtype=torch.int32, device=dev) for _ in range(G)]
    info = {}

    def group(i):
        eta = c["eta"][i * per:(i + 1) * per]
        with torch.cuda.stream(streams[i]):
            _, inf = plans[i].solve(eta, us[i])
            info[i] = inf
            plans[i].far_field(eta, us[i], c["alphas"], Fs[i], Es[i])

    def step():
        start = torch.cuda.Event()
        start.record(stream)
        for st in streams:
            st.wait_event(start)
        th = [threading.Thread(target=group, args=(i,)) for i in range(G)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        for st in streams:
            stream.wait_stream(st)

    def set_mode(mode):
        for p in plans:
            p.set_far_field_mode(mode)

    set_mode(csff.FF_TC_BF16X4)
    step()
    ms = _time_events(torch, stream, step, flush, 2)
    infs = [x for i in range(G) for x in info[i]]
    out = {"value": nr / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "maps_per_step": nr,
           "far_field": "tensor cores (z-contraction, four-term BF16 splits, FP32 accumulation)",
           "concurrency": "four plans of four directions, each on its own stream and host thread",
           "cycles": [x["cycles"] for x in infs], "all_converged": all(x["rel_res"] <= 1e-8 for x in infs)}
    set_mode(csff.FF_FP64)
    step()
    ms64 = _time_events(torch, stream, step, flush, 2)
    out["fp64_far_field"] = {"value": nr / (ms64 / 1e3), "unit": UNIT, "ms_per_step": ms64}
    for p in plans[1:]:
        p.close()
    plan = plans[0]
    u = torch.zeros(nr * N, dtype=torch.complex128, device=dev)
    F = torch.zeros(nr * na, dtype=torch.complex128, device=dev)
    Fe = torch.zeros(nr * na, dtype=torch.int32, device=dev)

    def seq_step():
        plan.solve(c["eta"], u)
        plan.far_field(c["eta"], u, c["alphas"], F, Fe)

    def ff():
        plan.far_field(c["eta"], u, c["alphas"], F, Fe)

    plan.set_far_field_mode(csff.FF_TC_BF16X4)
    with torch.cuda.stream(streams[0]):
        seq_step()
        mss = _time_events(torch, streams[0], seq_step, flush, 1)
        out["one_plan_in_turn"] = {"value": nr / (mss / 1e3), "unit": UNIT, "ms_per_step": mss}
        maps = {}
        for mode, name in ((csff.FF_FP64, "fp64"), (csff.FF_TC_BF16X4, "tc_bf16x4")):
            plan.set_far_field_mode(mode)
            ff()
            ff_ms = _time_events(torch, streams[0], ff, flush, 3)
            csff.prof_begin(csff.PROF_FF_CONTRACT)
            ff()
            torch.cuda.synchronize()
            prof = csff.prof_end()["ff_contract"]
            maps[name] = (F.cpu().numpy() * 2.0 ** Fe.cpu().numpy().astype(np.float64)).reshape(nr, na)
            out[f"ff_{name}_ms_per_16_maps"] = ff_ms
            out[f"ff_{name}_stageA_ms_per_map"] = prof["ms"] / max(1, nr)
            out[f"ff_{name}_stageA_tflops"] = prof["alg_flops"] / (prof["ms"] * 1e-3) / 1e12 if prof["ms"] else 0.0
    out["ff_fp64_stageA_fp64_frac"] = out["ff_fp64_stageA_tflops"] / FP64_PEAK_TFLOPS
    rel = np.linalg.norm(maps["tc_bf16x4"] - maps["fp64"], axis=1) / np.linalg.norm(maps["fp64"], axis=1)
    out["tc_vs_fp64_rel_l2"] = {"max": float(rel.max()), "median": float(np.median(rel)),
                                "maps_below_1e-5": int((rel <= 1e-5).sum())}
    plan.set_far_field_mode(csff.FF_FP64)
    plan.close()
    # beside the stated FP64 refinement: the double-float one (outer residual
    # and update as FP32 pairs on the FP32 pipes, coarsest solve in FP32), the
    # same concurrent step and tensor-core far field on four new plans
    opts_df = dict(c["opts"], refine_fp64=0)
    plans[:] = [csff.Plan(c["problem"], opts_df, stream=st) for st in streams]
    set_mode(csff.FF_TC_BF16X4)
    step()
    msdf = _time_events(torch, stream, step, flush, 2)
    infs = [x for i in range(G) for x in info[i]]
    out["double_float_refinement"] = {"value": nr / (msdf / 1e3), "unit": UNIT, "ms_per_step": msdf,
                                      "cycles": [x["cycles"] for x in infs],
                                      "all_converged": all(x["rel_res"] <= 1e-8 for x in infs)}
    for p in plans:
        p.close()
    return out


def measure_vcycle_bandwidth(csff, torch, dev, stream, flush):
    """Fused V(1,1) cycles on a grid whose FP32 arrays exceed the 129 MB L2
    (4097^2 on [-20,20]^2, k = 40, 10 levels, 9^2 coarsest; 134 MB per FP32
    array): algorithmic bytes of the multigrid kernels (u and b read and u
    written per tile pass, plus the next level's right-hand side) over their
    CUDA-event time, against the measured HBM copy bandwidth; the same for
    the FP64 cycle."""
    c = W.mixed_2d(40.0, n=4097)
    c["opts"].update(coarsest_n=9, precision="mixed")
    plan = csff.Plan(c["problem"], c["opts"], stream=stream)
    out = {"grid": "4097^2, 10 levels", "fp32_array_mb": plan.N * 8 / 1e6}
    peaks = _peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    for name, dt, mask in (("fp32", torch.complex64, csff.PROF_MG32), ("fp64", torch.complex128, csff.PROF_MG64)):
        u = torch.zeros(plan.N, dtype=dt, device=dev)
        b = torch.randn(plan.N, dtype=dt, device=dev)
        plan.vcycle(u, b)
        torch.cuda.synchronize()
        reps = 10 if name == "fp32" else 3
        csff.prof_begin(mask)
        for _ in range(reps):
            plan.vcycle(u, b)
        torch.cuda.synchronize()
        st = csff.prof_end()["mg32" if name == "fp32" else "mg64"]
        gbs = st["alg_bytes"] / (st["ms"] * 1e-3) / 1e9 if st["ms"] else 0.0
        out[name] = {"ms_per_cycle": st["ms"] / reps, "alg_gb_per_cycle": st["alg_bytes"] / reps / 1e9,
                     "achieved_gbs": gbs, "hbm_frac": gbs / hbm}
        del u, b
    plan.close()
    # the 3D workload's grid (257^3, 66 MB per FP32 array): per-level kernels
    c3 = W.big_3d(n=257, n_rhs=1)
    c3["opts"]["precision"] = "mixed"
    p3 = csff.Plan(c3["problem"], c3["opts"], stream=stream)
    for name, dt, mask in (("fp32_3d_257", torch.complex64, csff.PROF_MG32),
                           ("fp64_3d_257", torch.complex128, csff.PROF_MG64)):
        u = torch.zeros(p3.N, dtype=dt, device=dev)
        b = torch.randn(p3.N, dtype=dt, device=dev)
        p3.vcycle(u, b)
        torch.cuda.synchronize()
        reps = 5
        csff.prof_begin(mask)
        for _ in range(reps):
            p3.vcycle(u, b)
        torch.cuda.synchronize()
        st = csff.prof_end()["mg32" if "fp32" in name else "mg64"]
        gbs = st["alg_bytes"] / (st["ms"] * 1e-3) / 1e9 if st["ms"] else 0.0
        out[name] = {"ms_per_cycle": st["ms"] / reps, "alg_gb_per_cycle": st["alg_bytes"] / reps / 1e9,
                     "achieved_gbs": gbs, "hbm_frac": gbs / hbm}
        del u, b
    p3.close()
    return out


def _learned_problems(n_solves, k, n=257):
    """Training problems for the learned smoother: seeds 0 .. n_solves-1, chi
    and the incident angle drawn from the batch ranges, k fixed (so that k h
    matches the level the network serves)."""
    import math as _m
    out = []
    for seed in range(n_solves):
        rng = np.random.Generator(np.random.PCG64(seed))
        amp = float(rng.uniform(-2.0, -0.2))
        w = float(rng.uniform(1.0, 6.0))
        t = float(rng.uniform(0, 2 * _m.pi))
        out.append((W.problem(2, n, 20.0, _m.pi / 6, k, [W.gauss(amp, w)]), np.array([_m.cos(t), _m.sin(t)])))
    return out


def measure_learned(csff, torch, dev, stream, flush):
    """2049^2 on [-20,20]^2, k = 60 (k h = 1.17 on the finest level): plain
    red-black V(1,1) cycles against red-black + learned step u += N(h^2 r) on
    the finest level, both inside the FP64 refinement.  The networks are
    trained on the GPU on residual patches from 257^2 problems with the same
    k h (k = 7.5), chi drawn from the batch ranges: on 8, 32 and 2,000 seeded
    solves (the last is the reported network); in units of h^2 the operator is
    the same on both grids.  A second network trained at level 1's k h (257^2,
    k = 15) serves level 1 in the levels-0-1 variant."""
    from paper_1211_4461_gb300 import learned as LR
    opts = {"smoother": "rbgs", "omega": 1.0, "nu1": 1, "nu2": 1, "coarsest_n": 5, "rel_tol": 1e-8,
            "max_cycles": 400, "inner_cycles": 3}

    def train(n_solves, k, steps):
        t0 = time.perf_counter()
        data = LR.collect_patches(_learned_problems(n_solves, k), opts, n_cycles=5, patch=64,
                                  per_field=6 if n_solves <= 32 else 1, seed=1)
        net = csff.Net(LR.init_weights(7))
        hist = LR.train(net, data, steps=steps, batch=32, lr=2e-3, margin=4, seed=2)
        torch.cuda.synchronize()
        return net, {"solves": n_solves, "patches": int(data[0].shape[0]), "steps": steps,
                     "train_s": time.perf_counter() - t0, "loss_first": float(np.mean(hist[:5])),
                     "loss_last": float(np.mean(hist[-20:]))}

    case = W.mixed_2d(60.0, n=2049)
    case["opts"].update(precision="mixed", inner_cycles=3, max_cycles=400, refine_fp64=1)
    plan = csff.Plan(case["problem"], case["opts"], stream=stream)
    u = torch.zeros(plan.N, dtype=torch.complex128, device=dev)
    F = torch.zeros(720, dtype=torch.complex128, device=dev)
    Fe = torch.zeros(720, dtype=torch.int32, device=dev)
    info = {}

    def step():
        _, inf = plan.solve(case["eta"], u)
        info["inf"] = inf[0]
        plan.far_field(case["eta"], u, case["alphas"], F, Fe)

    def run(name):
        step()
        ms = _time_events(torch, stream, step, flush, 2)
        return {"value": 1.0 / (ms / 1e3), "unit": UNIT, "ms_per_map": ms, "cycles": info["inf"]["cycles"],
                "rel_res": info["inf"]["rel_res"], "flags": info["inf"]["flags"]}, \
            (F.cpu().numpy(), Fe.cpu().numpy().astype(np.int64))

    out = {}
    plan.set_learned(None)
    out["classical"], map_c = run("classical")
    curve = []
    nets = []
    for n_solves, steps in ((8, 1000), (32, 1000), (2000, 3000)):
        net, tinfo = train(n_solves, 7.5, steps)
        nets.append(net)
        plan.set_learned(net, levels=1)
        res, map_l = run("learned")
        curve.append(dict(tinfo, cycles=res["cycles"], ms_per_map=res["ms_per_map"]))
    out["training_curve"] = curve
    out["learned"] = res
    out["train"] = curve[-1]
    # the learned map against the classical one, angle by angle (mantissa and
    # power-of-two exponent: the map's terms pass the FP64 range at this k).
    # Both solutions meet 1e-8; the per-angle check against the oracle on the
    # well-conditioned cone runs in the tests (513^2).
    (f0, e0), (f1, e1) = map_c, map_l
    d = np.abs(f1 * 2.0 ** (e1 - e0).astype(np.float64) - f0) / np.abs(f0)
    out["far_field_learned_vs_classical"] = {"median_rel_diff": float(np.median(d)),
                                             "p90_rel_diff": float(np.quantile(d, 0.9)),
                                             "max_rel_diff": float(d.max())}
    out["cycle_ratio_learned_vs_classical"] = out["learned"]["cycles"] / max(1, out["classical"]["cycles"])
    out["speedup_learned_vs_classical"] = out["classical"]["ms_per_map"] / out["learned"]["ms_per_map"]
    net1, t1 = train(32, 15.0, 1000)
    plan.set_learned(nets[-1], levels=2)
    plan.set_learned_level(1, net1)
    out["learned_levels_0_1"], _ = run("learned01")
    out["learned_levels_0_1"]["level1_train"] = t1
    plan.close()
    for n in nets + [net1]:
        n.close()
    # the network forward alone on the 2049^2 finest level (4.2 M pixels)
    y = torch.empty((1, 2047, 2047), dtype=torch.complex64, device=dev)
    r = torch.randn((1, 2047, 2047), dtype=torch.complex64, device=dev)
    netf = csff.Net(LR.init_weights(7))
    out["forward_ms_2047sq"] = _time_events(torch, stream, lambda: netf.forward(r, y, stream=stream), flush, 5)
    netf.close()
    out["small_grid_129"] = measure_learned_small(csff, torch, dev, stream)
    out["3d_257_k6"] = measure_learned_3d(csff, torch, dev, stream, flush)
    return out


def measure_learned_3d(csff, torch, dev, stream, flush):
    """The 3D learned smoother on the 257^3 grid of the 3D workload at k = 6
    (k h = 0.70 on the finest level), both solves inside the FP64 refinement
    with three FP32 cycles a step: plain red-black V(1,1) against red-black +
    learned step u += N(h^2 r) (3x3x3 network on the CUDA cores) on the finest
    level.  The network is trained on the GPU on residual windows (16^3, at
    least a fifth of their energy inside the loss's 12^3 core) of 65^3 problems
    with the same grid spacing and wavenumber (box [-3.75, 3.75]^3, k = 6),
    chi and the incident direction drawn from the batch ranges, 32 seeded
    solves."""
    from paper_1211_4461_gb300 import learned as LR
    import math as _m
    opts = {"smoother": "rbgs", "omega": 1.0, "nu1": 1, "nu2": 1, "coarsest_n": 5, "rel_tol": 1e-8,
            "max_cycles": 400, "inner_cycles": 3}
    probs = []
    for seed in range(32):
        rng = np.random.Generator(np.random.PCG64(seed))
        amp = float(rng.uniform(-2.0, -0.2))
        w = float(rng.uniform(1.0, 6.0))
        th, ph = float(rng.uniform(0, _m.pi)), float(rng.uniform(0, 2 * _m.pi))
        probs.append((W.problem(3, 65, 3.75, _m.pi / 6, 6.0, [W.gauss(amp, w)]),
                      np.array([_m.sin(th) * _m.cos(ph), _m.sin(th) * _m.sin(ph), _m.cos(th)])))
    t0 = time.perf_counter()
    data = LR.collect_patches(probs, opts, n_cycles=4, patch=16, per_field=8, seed=1, core_margin=2, min_core=0.2)
    net = csff.Net(LR.init_weights(7, dim=3), dim=3)
    hist = LR.train(net, data, steps=600, batch=8, lr=3e-4, margin=2, seed=2)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    c = W.big_3d(n=257, n_rhs=1)
    c["problem"]["k"] = 6.0
    plan = csff.Plan(c["problem"], dict(c["opts"], precision="mixed", refine_fp64=1, inner_cycles=3),
                     stream=stream)
    u = torch.zeros(plan.N, dtype=torch.complex128, device=dev)
    info = {}

    def step():
        _, inf = plan.solve(c["eta"], u)
        info["inf"] = inf[0]

    out = {"train": {"solves": 32, "patches": int(data[0].shape[0]), "steps": 600, "train_s": train_s,
                     "loss_first": float(np.mean(hist[:5])), "loss_last": float(np.mean(hist[-20:]))}}
    for name, learned in (("classical", False), ("learned", True)):
        plan.set_learned(net if learned else None, levels=1)
        step()
        ms = _time_events(torch, stream, step, flush, 1)
        out[name] = {"value": 1.0 / (ms / 1e3), "unit": UNIT, "ms_per_solve": ms, "cycles": info["inf"]["cycles"],
                     "rel_res": info["inf"]["rel_res"], "flags": info["inf"]["flags"]}
    r = torch.randn(plan.N, dtype=torch.complex64, device=dev).view(1, 255, 255, 255)
    y = torch.empty_like(r)
    out["forward_ms_255cube"] = _time_events(torch, stream, lambda: net.forward(r, y, stream=stream), flush, 2)
    out["speedup_learned_vs_classical"] = out["classical"]["ms_per_solve"] / out["learned"]["ms_per_solve"]
    out["note"] = ("solve only (the far field is the same for both); the 3x3x3 network's forward pass runs "
                   "on the CUDA cores")
    plan.close()
    net.close()
    return out


def measure_learned_small(csff, torch, dev, stream):
    """129^2 on [-20,20]^2, k ~ U[3,5] (k h 0.9-1.6): trained on 24 seeded
    problems, evaluated on 4 held-out seeds (V-cycles to 1e-8)."""
    from paper_1211_4461_gb300 import learned as LR
    import math as _m
    opts = {"smoother": "rbgs", "omega": 1.0, "nu1": 1, "nu2": 1, "coarsest_n": 5, "rel_tol": 1e-8,
            "max_cycles": 300, "inner_cycles": 3}

    def probs(seeds):
        out = []
        for s in seeds:
            rng = np.random.Generator(np.random.PCG64(1000 + s))
            k = float(rng.uniform(3.0, 5.0))
            amp = float(rng.uniform(-1.5, -0.5))
            w = float(rng.uniform(2.0, 5.0))
            t = float(rng.uniform(0, 2 * _m.pi))
            out.append((W.problem(2, 129, 20.0, _m.pi / 6, k, [W.gauss(amp, w)]),
                        np.array([_m.cos(t), _m.sin(t)])))
        return out

    data = LR.collect_patches(probs(range(24)), opts, n_cycles=5, patch=48, per_field=6, seed=1)
    net = csff.Net(LR.init_weights(7))
    hist = LR.train(net, data, steps=800, batch=32, lr=2e-3, margin=4, seed=2)
    rows = []
    for prob, eta in probs([100, 101, 102, 103]):
        plan = csff.Plan(prob, dict(opts, precision="mixed"), stream=stream)
        u = torch.zeros(plan.N, dtype=torch.complex128, device=dev)
        _, b = plan.solve(np.atleast_2d(eta), u)
        plan.set_learned(net, levels=1)
        _, l = plan.solve(np.atleast_2d(eta), u)
        rows.append({"classical": b[0]["cycles"], "learned": l[0]["cycles"], "flags": l[0]["flags"]})
        plan.close()
    net.close()
    return {"loss_first": float(np.mean(hist[:5])), "loss_last": float(np.mean(hist[-20:])), "held_out": rows,
            "cycle_ratio": sum(r["learned"] for r in rows) / max(1, sum(r["classical"] for r in rows))}


def measure_gmres_table2(csff, torch, dev, stream, flush):
    """The paper's V(1,1)/GMRES(3) configuration of Table 2 (eq. chi3D on
    [-20,20]^3, rotation 9.9 degrees, residual reduction 1e-6, FP64) on the
    64^3, 128^3 and 256^3 grids for k0 = 1/4 ... 4: V-cycles, average
    convergence factor and time per solve, beside the values Table 2 prints
    (tests/golden/table2_vcycle_gmres3.txt).  At this angle the red-black
    V-cycle diverges (checked in the tests).  The same problems by full
    multigrid (nested iteration, 1e-6 on every level): V-cycles per level, time
    per solve against the V-cycles from zero, and the finest-level count Table 3
    prints (tests/golden/table3_fmg_gmres3.txt)."""
    gold = {}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tests", "golden", "table2_vcycle_gmres3.txt")
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            k, pts, cyc, fac = line.split()
            gold[(float(k), int(pts))] = (int(cyc), float(fac))
    # Table 3 (FMG cycle, same setting): V-cycles on the designated finest grid
    fmg_gold = {}
    for line in open(os.path.join(os.path.dirname(path), "table3_fmg_gmres3.txt")):
        if line.strip() and not line.startswith("#"):
            k, pts, cyc = line.split()[:3]
            fmg_gold[(float(k), int(pts))] = int(cyc)
    out = {}
    for pts in (64, 128, 256):
        rows = []
        for k in (0.25, 0.5, 1.0, 2.0, 4.0):
            c = W.paper_gmres(dim=3, k=k, n=pts + 1)
            c["opts"]["precision"] = "fp64"
            plan = csff.Plan(c["problem"], c["opts"], stream=stream)
            u = torch.zeros(plan.N, dtype=torch.complex128, device=dev)
            info = {}

            def solve():
                _, inf = plan.solve(c["eta"], u)
                info["i"] = inf[0]

            solve()
            ms = _time_events(torch, stream, solve, flush, 2)
            i = info["i"]
            pc, pf = gold[(k, pts)]

            def solve_fmg():
                _, inf, cyc = plan.solve_fmg(c["eta"], u)
                info["f"] = (inf[0], cyc[0])

            solve_fmg()
            ms_f = _time_events(torch, stream, solve_fmg, flush, 2)
            fi, fc = info["f"]
            rows.append({"k0": k, "cycles": i["cycles"], "conv_factor": round(i["conv_factor"], 3),
                         "paper_cycles": pc, "paper_factor": pf, "ms_per_solve": ms,
                         "converged": i["rel_res"] <= c["opts"]["rel_tol"],
                         "fmg": {"level_cycles_coarse_to_fine": fc, "finest_cycles": fi["cycles"],
                                 "paper_finest_cycles": fmg_gold[(k, pts)], "ms_per_solve": ms_f,
                                 "speedup_vs_vcycles_from_zero": ms / ms_f,
                                 "converged": fi["status"] == csff.OK}})
            plan.close()
            del u
        out[f"{pts}^3"] = rows
    return out


def measure_partial_wave(csff, torch, dev, stream, flush):
    """Fig. 8's cross-section curve along the contour (Sec. 5.2-5.3): for each
    energy of the figure's contour points above the threshold, the 2D
    partial-wave problem on [0,15]^2 (513^2 nodes, rotation 8.5 degrees) is
    solved by V(1,1)/GMRES(3) cycles (FP64, 1e-10; an energy whose cycles
    diverge is reported as such, as Fig. 9 reports for -1 < E < 0) with its potential and
    right-hand side given as samples, the 1D bound state and regular
    solutions come from the library, and the single and double ionization
    integrals (1 + 32 angles) run on the device.  Reports the time per energy
    and the cross sections beside the printed ones (readings: single 4|s_0|^2,
    double (4/pi) int |f|^2 k1 k2 da)."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tests", "golden",
                        "fig8_cross_sections_contour.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    rows = [(float(a), float(b), float(c)) for a, b, c in rows][1:]
    n, n_al = 513, 32
    m = n - 2
    al = (np.arange(n_al) + 0.5) * (math.pi / 2) / n_al
    out = {"grid": f"{n}^2 on [0,15]^2, rotation 8.5 deg", "energies": []}
    t_all = 0.0
    for E, ps, pd in rows:
        c = W.partial_wave(E, n=n)
        c["opts"].update(rel_tol=1e-10, max_cycles=100)
        plan = csff.Plan(c["problem"], c["opts"], stream=stream)
        V, f, w = (torch.from_numpy(np.ascontiguousarray(x).ravel()).to(dev) for x in (c["V"], c["f"], c["w"]))
        u = torch.zeros(plan.N, dtype=torch.complex128, device=dev)
        res = {}

        def run():
            plan.set_schroedinger(E, V)
            st, info = plan.solve_schroedinger(f, u, ok=(csff.OK, csff.ERR_DIVERGED, csff.ERR_NOT_CONVERGED))
            g = c["gamma"]
            lam, phi0 = csff.contour_bound_state(c["v1"], c["h"], g, -1.0)
            kn = math.sqrt(2.0 * (E - lam.real))
            X = [csff.contour_regular_solution(c["v1"], c["h"], g, kn)]
            Y = [phi0]
            if E > 0:
                k = math.sqrt(2.0 * E)
                for a in al:
                    X.append(csff.contour_regular_solution(c["v1"], c["h"], g, k * math.sin(a)))
                    Y.append(csff.contour_regular_solution(c["v1"], c["h"], g, k * math.cos(a)))
            Xd = torch.from_numpy(np.ascontiguousarray(np.stack(X))).to(dev)
            Yd = torch.from_numpy(np.ascontiguousarray(np.stack(Y))).to(dev)
            amp = plan.separable_sum(Xd, Yd, f, w, u).cpu().numpy()
            res.update(st=st, info=info, amp=amp)

        run()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        run()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        t_all += dt
        amp = res["amp"]
        single = 4.0 * abs(amp[0]) ** 2
        double = 0.0
        if E > 0:
            k2 = 2.0 * E
            double = (4.0 / math.pi) * float(np.sum(np.abs(amp[1:]) ** 2 * k2 * np.sin(al) * np.cos(al))) \
                * (math.pi / 2) / n_al
        out["energies"].append({"E": E, "cycles": res["info"]["cycles"], "conv_factor": round(res["info"]["conv_factor"], 3),
                                "converged": res["st"] == csff.OK, "single": single, "paper_single": ps,
                                "double": double, "paper_double": pd, "ms": dt * 1e3})
        plan.close()
    out["s_per_curve"] = t_all
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-variants", dest="variants", action="store_false",
                    help="skip the plain-FP64 and batched comparison runs")
    ap.add_argument("--ks", default="", help="comma-separated subset of the wavenumbers (profiling runs)")
    ap.add_argument("--inner-cycles", type=int, default=INNER_CYCLES,
                    help="FP32 V-cycles per refinement step of the mixed solve")
    ap.add_argument("--adaptive-inner", dest="adaptive_inner", action="store_true", default=True,
                    help="size each refinement step from the previous step's reduction factor (default)")
    ap.add_argument("--fixed-inner", dest="adaptive_inner", action="store_false",
                    help="always inner-cycles FP32 V-cycles per refinement step")
    ap.add_argument("--refine-fp64", dest="refine_fp64", action="store_true", default=True,
                    help="mixed solve with the FP64 outer residual, update and coarsest solve (default)")
    ap.add_argument("--refine-df", dest="refine_fp64", action="store_false",
                    help="mixed solve with the outer residual and update in double-float (pairs of FP32 words)")
    ap.add_argument("--sequential", action="store_true",
                    help="solve the maps of a step one after another on one host thread (for profilers, "
                         "which serialise kernels anyway and do not follow several capturing threads)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
