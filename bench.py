"""Benchmark of the FMM self-gravity solve on GB300 (one JSON line on stdout).

Metric: cell-interactions/s = (ordered same-level M2L + cross-level M2L +
same-level P2P + cross-level P2P interactions of one solve) / time of one solve.
A step is one full solve (P2M, M2M, M2L + correction, cross-level, P2P, L2L,
L2P) over the synthetic input, replayed from the library's CUDA graph.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
                  [--precision mixed|fp64] [--impl ours|reference]

Default workload: adaptive7 (7-level adaptive octree of a q=0.7 binary of n=1.5
polytropes, ~8000 leaf subgrids of 8^3 cells), mixed precision, with the float64
path timed beside it.  N > 1 runs one independent replica per GPU (the solve
needs no exchange between GPUs); `value` sums the replicas' work over the
slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-interactions/s"
L2_FLUSH_BYTES = 256 << 20  # twice the 129 MB L2

# Nominal peaks (per GPU, at the 2070 MHz maximum SM clock): float64 1.25 TFLOP/s
# -> 4 flop / clock / SM = 152 * 4 * 2.07e9; float32 128 lanes x 2 flop / clock / SM
# -> 152 * 256 * 2.07e9.  The roofline uses the peaks measured on the device by the
# library's fused multiply-add probe (octo_fmm_measure_peak); these are the fallback.
PEAK_FP64_TFLOPS = 152 * 4 * 2.07e9 / 1e12
PEAK_FP32_TFLOPS = 152 * 256 * 2.07e9 / 1e12
NOMINAL_ALU = {"fp64": PEAK_FP64_TFLOPS, "fp32": PEAK_FP32_TFLOPS,
               "source": "derived: 152 SMs x (4 fp64 | 256 fp32) flop/clk x 2.07 GHz"}


def measure_alu_peaks(gpu_index: int, stream):
    """float64 and float32 FMA rates of this GPU in TFLOP/s (the library's probe),
    with the SM clocks sampled while the probe ran."""
    from paper_2304_11002_gb300 import binding
    with ClockSampler(gpu_index) as clk:
        f64 = max(binding.octo_fmm_measure_peak(True, stream) for _ in range(2))
        f32 = max(binding.octo_fmm_measure_peak(False, stream) for _ in range(2))
    c = clk.summary()
    return {"fp64": f64 / 1e12, "fp32": f32 / 1e12,
            "source": f"measured: FMA-chain probe octo_fmm_measure_peak (best of 2 x 3 launches), "
                      f"SM clock median {c['sm_mhz']} MHz of max {c['sm_max_mhz']}",
            "clocks": c}


def _measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# DRAM traffic of the roofline kernel comes from one ncu capture (profiles/
# roofline_traffic.json); it is reported only while the kernel code is that the
# capture was taken with (sha256 over these files without their // comments and
# blank lines), else null.
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "roofline_traffic.json")
KERNEL_SOURCES = ("capi.cu", "cross.cuh", "device.cuh", "halo.h", "interact.cuh", "items.cuh", "kernels.h",
                  "kernels_boundary.cu", "kernels_interact.cu", "kernels_interact_b64.cu", "pair_x2.cuh", "tables.cpp",
                  "tables.h", "tma.cuh")


def code_lines(text: str):
    """The lines of a C++/CUDA source without // comments, trailing blanks and empty
    lines (a comment edit leaves the compiled kernel, and so a capture, valid)."""
    for line in text.splitlines():
        code = line.split("//", 1)[0].rstrip()
        if code:
            yield code


def kernel_sources_sha256(read=None):
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        if read is None:
            with open(os.path.join(ROOT, "paper_2304_11002_gb300", "csrc", f)) as fh:
                text = fh.read()
        else:
            text = read(f)
        for code in code_lines(text):
            h.update(code.encode() + b"\n")
    return h.hexdigest()


def recorded_traffic(stage: str, workload: str, shape=None, blocks=None, paced=None):
    """(bytes per launch, source) of a matching capture, or (None, reason).  shape
    (entries per float32 partial, split), blocks (register budget) and paced (queue)
    must match the capture's when both are known."""
    try:
        with open(TRAFFIC_FILE) as f:
            entries = json.load(f)["entries"]
    except Exception:
        return None, "no capture recorded"
    sha = kernel_sources_sha256()
    for e in entries:
        if e["stage"] == stage and e["workload"] == workload:
            if e["sources_sha256"] != sha:
                return None, "kernel changed since the capture"
            if shape is not None and e.get("interior_shape") is not None and list(shape) != e["interior_shape"]:
                return None, "the capture is of another interior shape"
            if blocks is not None and e.get("blocks_per_sm") is not None and blocks != e["blocks_per_sm"]:
                return None, "the capture is of another register budget"
            if paced is not None and e.get("paced") is not None and bool(paced) != bool(e["paced"]):
                return None, "the capture is of the other queue"
            return int(e["bytes"]), e["command"]
    return None, "no capture for this kernel and workload"


def aggregate_over_ranks(t_rank_s: float, units_per_step: float, steps: int, ws: int, reduce_max=None):
    """Whole-job throughput of ws replicas (each rank solves the same workload on its
    own GPU): units all ranks processed over the slowest rank's time.  reduce_max
    maps this rank's time to the maximum over ranks (None for one rank).  Returns
    (value, max time)."""
    t = float(t_rank_s if reduce_max is None else reduce_max(t_rank_s))
    return units_per_step * steps * ws / t, t


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine type)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


class OracleSampler:
    """The oracle as it stands, over seeded samples of leaf cells of a workload: it
    evaluates the full upward pass, then the interaction lists of the sampled cells
    and of their ancestors, and counts the ordered interactions it evaluated."""

    def __init__(self, w, theta: float = 0.5, seed: int = 123):
        import oracle
        self.oracle = oracle
        self.w, self.theta = w, theta
        self.nl = w.tree.n_leaf * 512
        self.rng = np.random.default_rng(seed)

    def run(self, n_cells: int):
        """(interactions evaluated, seconds) of one sample of n_cells leaf cells."""
        n_cells = int(min(self.nl, max(1, n_cells)))
        mask = np.zeros(self.nl, np.uint8)
        mask[self.rng.choice(self.nl, size=n_cells, replace=False)] = 1
        work = np.zeros(1, np.int64)
        t0 = time.perf_counter()
        self.oracle.fmm(self.w.tree, self.w.rho, self.theta, leaf_mask=mask, work=work)
        return int(work[0]), time.perf_counter() - t0

    def calibrate(self, seconds_target: float, n_probe: int = 64) -> int:
        """Sample size that takes about seconds_target (the upward pass is a fixed cost
        of every sample, so the size is scaled on the interaction part).  The probe
        runs once per thread count."""
        key = self.oracle.set_threads(0)
        if getattr(self, "_probe", (None,))[0] != key:
            _, t_fixed = self.run(1)
            _, t_probe = self.run(n_probe)
            self._probe = (key, t_fixed, max(t_probe - t_fixed, 1e-4) / n_probe)
        _, t_fixed, per_cell = self._probe
        return int(min(self.nl, max(n_probe, (seconds_target - t_fixed) / per_cell)))


def cpu_baseline(w, seconds_target: float = 15.0, theta: float = 0.5, one_thread_seconds: float = 8.0):
    """The oracle timed on the host cores (all of them, then one thread) over bounded
    samples of the workload; value in ordered interactions per second."""
    s = OracleSampler(w, theta)
    threads = s.oracle.set_threads(0)
    n = s.calibrate(seconds_target)
    work, dt = s.run(n)
    out = {"value": work / dt, "unit": METRIC, "cores": threads, "kind": "oracle",
           "sample": f"{n} of {s.nl} leaf cells of {w.name} (their and their ancestors' interaction lists, "
                     f"{work} interactions, {dt:.1f} s, including the full upward pass)",
           "cpu_model": cpu_model(), "seconds": dt}
    if one_thread_seconds > 0:
        s.oracle.set_threads(1)
        try:
            n1 = s.calibrate(one_thread_seconds)
            work1, dt1 = s.run(n1)
        finally:
            s.oracle.set_threads(threads)
        out["one_thread"] = {"value": work1 / dt1, "cores": 1,
                             "sample": f"{n1} leaf cells, {work1} interactions, {dt1:.1f} s"}
    return out


def run_reference(args):
    """The oracle as the reference arm: every step is one bounded sample of the
    workload (the warm-up steps short ones), timed on the host cores; ms_per_step is
    the samples' own mean time and value their interactions per second."""
    ws, rank, _ = dist_env()
    if ws > 1 and rank != 0:
        return 0
    from paper_2304_11002_gb300 import workloads as W
    w = W.make(args.workload)
    s = OracleSampler(w, w.theta)
    threads = s.oracle.set_threads(0)
    per_step = min(args.ref_seconds, max(2.0, args.ref_budget / max(args.steps, 1)))
    n_warm = s.calibrate(1.0)
    n_step = s.calibrate(per_step)
    for _ in range(args.warmup):
        s.run(n_warm)
    works, secs = [], []
    for _ in range(args.steps):
        wk, dt = s.run(n_step)
        works.append(wk)
        secs.append(dt)
    value = float(np.sum(works)) / float(np.sum(secs))
    sample = (f"{args.steps} samples of {n_step} of {s.nl} leaf cells of {w.name} (each: the full upward pass, "
              f"then the sampled cells' and their ancestors' interaction lists; {int(np.mean(works))} "
              f"interactions, {np.mean(secs):.1f} s per sample)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(secs)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "note": w.note, "theta": w.theta, "order": 3,
                       "step": "one bounded sample of the workload (see cpu_baseline.sample)"},
            "cpu_baseline": {"value": value, "unit": METRIC, "cores": threads, "kind": "oracle", "sample": sample,
                             "cpu_model": cpu_model()},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


_COUNTS_CACHE = {}


def counts_total(w):
    from paper_2304_11002_gb300 import binding
    key = id(w)
    if key not in _COUNTS_CACHE:
        _COUNTS_CACHE[key] = int(binding.octo_fmm_plan_counts(w.tree, w.theta).sum())
    return _COUNTS_CACHE[key]


STRATEGY = {"auto": 0, "per-kind": 1, "persistent": 2}


def time_solver(w, precision, steps, warmup, torch, flush, stream, strategy="auto", blocks=0, corr64=False,
                shape=None, paced=None):
    from paper_2304_11002_gb300 import binding
    fmm = binding.OctoFMM(w.tree, w.theta, precision)
    h = fmm.handle
    binding.octo_fmm_set_option(h, 2, 1)  # stage events inside the captured graph
    if corr64:  # the float64-correction variant of the mixed path (per-kind launches)
        binding.octo_fmm_set_option(h, 5, 1)
    if shape and precision == binding.OCTO_MIXED:  # interior shape fixed instead of autotuned
        binding.octo_fmm_set_option(h, 6, shape[0])
        binding.octo_fmm_set_option(h, 7, shape[1])
    if paced is not None and precision == binding.OCTO_MIXED:  # queue fixed instead of autotuned
        binding.octo_fmm_set_option(h, 8, paced)
    if strategy != "auto":
        binding.octo_fmm_set_option(h, 3, STRATEGY[strategy])
        if blocks:
            binding.octo_fmm_set_option(h, 4, blocks)
    rho = torch.from_numpy(np.ascontiguousarray(w.rho.reshape(-1))).cuda()
    phi = torch.empty(fmm.n_leaf_cells, dtype=torch.float64, device="cuda")
    g = torch.empty((3, fmm.n_leaf_cells), dtype=torch.float64, device="cuda")
    with torch.cuda.stream(stream):
        for _ in range(warmup):  # the first call also runs the autotuner, which may change the stages
            fmm.forces(rho, phi, g, stream)
        stream.synchronize()
        nst = binding.octo_fmm_stage_count(h)
        info = [binding.octo_fmm_stage_info(h, i) for i in range(nst)]
        step_ms, stage_ms = [], []
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for _ in range(steps):
            flush.zero_()  # evict L2 (outside the timed events)
            e0.record(stream)
            fmm.forces(rho, phi, g, stream)
            e1.record(stream)
            stream.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            stage_ms.append(binding.octo_fmm_stage_times(h))
    launches = binding.octo_fmm_launches_per_solve(h)
    return fmm, info, np.array(step_ms), np.array(stage_ms), launches, (rho, phi, g)


def roofline_of(info, mean_stage_ms, peaks, alu=None):
    """Roofline of the stage that takes longest (CUDA-event time per solve).  alu:
    float64 / float32 peaks in TFLOP/s (default: the nominal ones)."""
    alu = alu or NOMINAL_ALU
    k = int(np.argmax(mean_stage_ms))
    st = info[k]
    dur_s = mean_stage_ms[k] / 1e3
    if st["flops"] > 0:
        # A stage may mix float32 (far field) and float64 (near field) work: the
        # binding unit is the one whose work takes longer at its peak.
        f64, f32 = st["flops64"], st["flops"] - st["flops64"]
        fp32_bound = f32 / alu["fp32"] > f64 / alu["fp64"]
        peak = alu["fp32"] if fp32_bound else alu["fp64"]
        achieved = (f32 if fp32_bound else f64) / dur_s / 1e12
        return {"bound": "alu", "kernel": st["name"], "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None,
                "pipe": "fp32" if fp32_bound else "fp64",
                "other_pipe_frac": ((f64 / dur_s / 1e12) / alu["fp64"] if fp32_bound else
                                    (f32 / dur_s / 1e12) / alu["fp32"]),
                "peak_source": alu["source"],
                "peak_nominal": PEAK_FP32_TFLOPS if fp32_bound else PEAK_FP64_TFLOPS}
    peak = float(peaks.get("hbm_gbs", 6800.0))
    achieved = st["bytes"] / dur_s / 1e9
    return {"bound": "hbm", "kernel": st["name"], "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": None, "peak_source": "measured" if peaks else "fallback"}


def stage_rates(info, mean_stage_ms, peaks, alu=None):
    """Per stage: time, the float32 / float64 flop rates as fractions of their peaks,
    and for the tree passes also HBM GB/s as a fraction of the measured copy
    bandwidth (algorithmic bytes, every value read or written once)."""
    alu = alu or NOMINAL_ALU
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    out = {}
    for i, st in enumerate(info):
        ms = float(mean_stage_ms[i])
        if ms <= 0:
            continue
        d = {"ms": round(ms, 4)}
        if st["flops"] > 0:
            f64 = st["flops64"]
            f32 = st["flops"] - f64
            d["fp32_frac"] = round(f32 / (ms / 1e3) / 1e12 / alu["fp32"], 4)
            d["fp64_frac"] = round(f64 / (ms / 1e3) / 1e12 / alu["fp64"], 4)
        if st["bytes"] > 0:
            gbs = st["bytes"] / (ms / 1e3) / 1e9
            d["gbs"] = round(gbs, 1)
            d["hbm_frac"] = round(gbs / hbm, 4)
        out[st["name"]] = d
    return out


def interaction_fp64_frac(info, mean_stage_ms, alu=None):
    """float64 flop rate of all interaction stages together (their float64 flops over
    their summed event time) as a fraction of the float64 peak."""
    alu = alu or NOMINAL_ALU
    f64 = sum(st["flops64"] for st in info if st["pairs"] > 0)
    ms = sum(float(mean_stage_ms[i]) for i, st in enumerate(info) if st["pairs"] > 0)
    return f64 / (ms / 1e3) / 1e12 / alu["fp64"] if ms > 0 else None


def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    from paper_2304_11002_gb300 import binding, build
    from paper_2304_11002_gb300 import workloads as W
    build.build()
    w = W.make(args.workload)
    n_inter = counts_total(w)
    counts = binding.octo_fmm_plan_counts(w.tree, w.theta)
    precision = binding.OCTO_MIXED if args.precision == "mixed" else binding.OCTO_FP64
    stream = torch.cuda.Stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    alu = NOMINAL_ALU if args.nominal_peaks else measure_alu_peaks(local, stream)

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()

    barrier()
    with ClockSampler(local) as clk:
        fmm, info, step_ms, stage_ms, launches, bufs = time_solver(w, precision, args.steps, args.warmup, torch,
                                                                   flush, stream, args.strategy, args.blocks,
                                                                   args.corr64, args.interior_shape, args.paced)
    barrier()
    t_step = float(np.mean(step_ms))

    def reduce_max(x):
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        return float(t.item())

    rmax = reduce_max if ws > 1 else None
    value, _ = aggregate_over_ranks(float(np.sum(step_ms)) / 1e3, n_inter, args.steps, ws, rmax)

    # dominant kernel of the step and its roofline
    mean_stage = stage_ms.mean(axis=0)
    roof = roofline_of(info, mean_stage, _measured_peaks(), alu)
    gopt = lambda k: binding.octo_fmm_get_option(fmm.handle, k)  # noqa: E731
    shape = (gopt(6), gopt(7)) if precision == binding.OCTO_MIXED else None
    roof["traffic"], roof["traffic_source"] = recorded_traffic(roof["kernel"], w.name, shape, gopt(4),
                                                               gopt(8) if precision == binding.OCTO_MIXED else None)

    # end to end through the C ABI with host buffers (copies inside the timed region)
    nlc = fmm.n_leaf_cells
    rho_h = np.ascontiguousarray(w.rho.reshape(-1))
    phi_h = np.empty(nlc)
    g_h = np.empty((3, nlc))
    with torch.cuda.stream(stream):
        for _ in range(2):
            binding.octo_fmm_forces_host(fmm.handle, rho_h, phi_h, g_h, stream)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            binding.octo_fmm_forces_host(fmm.handle, rho_h, phi_h, g_h, stream)
        barrier()
        e2e_s = time.perf_counter() - t0
    e2e_value, _ = aggregate_over_ranks(e2e_s, n_inter, args.steps, ws, rmax)
    e2e = {"value": e2e_value, "unit": METRIC, "h2d_bytes_per_step": int(rho_h.nbytes),
           "d2h_bytes_per_step": int(phi_h.nbytes + g_h.nbytes)}

    # the float64 path on the same workload, for the mixed-vs-float64 comparison
    fp64 = None
    strategy = {"chosen": {1: "per-kind launches", 2: "persistent work queue"}[gopt(3)],
                "register_budget_blocks_per_sm": gopt(4),
                "autotune_us": {"per_kind": gopt(10), "persistent_1": gopt(11), "persistent_2": gopt(12),
                                "persistent_3": gopt(13), "interior_chunk_64": gopt(14),
                                "interior_quarter_node": gopt(15), "paced_queue": gopt(16)}}
    if precision == binding.OCTO_MIXED:
        strategy["interior_shape"] = {"entries_per_float32_partial": gopt(6),
                                      "items": {1: "half node", 2: "quarter node"}[gopt(7)]}
        strategy["paced_queue"] = bool(gopt(8))

    if precision == binding.OCTO_MIXED and not args.no_fp64:
        del fmm
        fmm64, info64, s_ms, st_ms, _, bufs64 = time_solver(w, binding.OCTO_FP64, max(3, args.steps // 2), 3, torch,
                                                            flush, stream, args.strategy)
        m64 = st_ms.mean(axis=0)
        # the hand-written adjoint (d loss / d rho for given d loss / d phi, d loss / d g)
        # after the last forward solve of this handle
        gen = torch.Generator(device="cuda").manual_seed(7)
        dphi = torch.randn(nlc, dtype=torch.float64, device="cuda", generator=gen)
        dg = torch.randn((3, nlc), dtype=torch.float64, device="cuda", generator=gen)
        drho = torch.empty(nlc, dtype=torch.float64, device="cuda")
        with torch.cuda.stream(stream):
            binding.octo_fmm_backward(fmm64.handle, dphi, dg, drho, stream)  # allocates the adjoint workspace
            b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            b0.record(stream)
            for _ in range(3):
                binding.octo_fmm_backward(fmm64.handle, dphi, dg, drho, stream)
            b1.record(stream)
            stream.synchronize()
        backward_ms = b0.elapsed_time(b1) / 3.0
        del fmm64, bufs64
        fp64 = {"value": n_inter / (float(np.mean(s_ms)) / 1e3), "ms_per_step": float(np.mean(s_ms)),
                "stages_ms": {info64[i]["name"]: round(float(m64[i]), 4) for i in range(len(info64))},
                "roofline": roofline_of(info64, m64, _measured_peaks(), alu),
                "interaction_fp64_frac": interaction_fp64_frac(info64, m64, alu),
                "backward_ms": backward_ms}

    if rank != 0:
        return 0
    clocks = clk.summary()
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if precision == binding.OCTO_MIXED else "f64",
        "mixed_correction": ("float64 (option 5)" if args.corr64 else "float32") if precision == binding.OCTO_MIXED
        else None,
        "data": "synthetic",
        "config": {"workload": w.name, "note": w.note, "precision": args.precision, "theta": w.theta, "order": 3,
                   "n_leaf_subgrids": int(w.tree.n_leaf), "n_nodes": int(w.tree.n_nodes),
                   "interactions_per_step": n_inter,
                   "counts": {"m2l_same": int(counts[0]), "m2l_cross": int(counts[1]), "p2p_same": int(counts[2]),
                              "p2p_cross": int(counts[3])},
                   "l2": "flushed before every timed step (256 MB write, outside the timed events)",
                   "parallelism": f"replicas{ws}" if ws > 1 else "single GPU"},
        "roofline": roof,
        "interaction_strategy": strategy,
        "stages_ms": {info[i]["name"]: round(float(mean_stage[i]), 4) for i in range(len(info))},
        "stage_rates": stage_rates(info, mean_stage, _measured_peaks(), alu),
        "alu_peaks_tflops": {"fp64": alu["fp64"], "fp32": alu["fp32"], "source": alu["source"],
                             "nominal_fp64": PEAK_FP64_TFLOPS, "nominal_fp32": PEAK_FP32_TFLOPS},
        "e2e": e2e,
        "gpu_launches": int(launches * args.steps),
        "clocks": clocks,
    }
    if fp64 is not None:
        line["fp64_path"] = fp64
        line["mixed_over_fp64"] = value / ws / fp64["value"]
    if not args.no_cpu_baseline and ws == 1:
        cb = cpu_baseline(w, seconds_target=args.ref_seconds)
        line["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample", "cpu_model",
                                                   "one_thread")}
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_oracle_timing(args):
    """Full (unsampled) oracle solves of the small configurations on the host cores,
    at all cores and at one thread: 16^3 lognormal (seeds 0-2), the 64^3 binary and
    the ~1e3-leaf adaptive sweep tree; cell-interactions/s from the interactions the
    oracle evaluated.  One JSON line; no GPU is used."""
    import oracle
    from paper_2304_11002_gb300 import workloads as W
    cases = [("uniform16_s0", lambda: W.uniform16(0)), ("uniform16_s1", lambda: W.uniform16(1)),
             ("uniform16_s2", lambda: W.uniform16(2)), ("binary64", W.binary64),
             ("sweep1000_q0.7_s0", lambda: W.sweep(1000, q=0.7, seed=0))]
    all_cores = oracle.set_threads(0)
    out = {"kind": "oracle", "cpu_model": cpu_model(), "cores": all_cores, "unit": METRIC, "runs": []}
    for name, make in cases:
        w = make()
        for threads in (all_cores, 1):
            if threads == 1 and name not in args.oracle_one_thread:
                continue
            oracle.set_threads(threads)
            work = np.zeros(1, np.int64)
            t0 = time.perf_counter()
            oracle.fmm(w.tree, w.rho, w.theta, work=work)
            dt = time.perf_counter() - t0
            out["runs"].append({"config": name, "threads": threads, "interactions": int(work[0]), "seconds": dt,
                                "value": float(work[0]) / dt})
            print(json.dumps(out["runs"][-1]), file=sys.stderr, flush=True)
    oracle.set_threads(all_cores)
    print(json.dumps(out), flush=True)
    return 0


def run_backward(args):
    """The hand-written adjoint alone: d(loss)/d(rho) for random d(loss)/d(phi) and
    d(loss)/d(g) after one float64 forward solve, timed over the steps with CUDA
    events (L2 flushed before every step).  One JSON line; value = the solve's
    ordered interactions per second of adjoint time."""
    import torch
    torch.cuda.set_device(0)
    from paper_2304_11002_gb300 import binding, build
    from paper_2304_11002_gb300 import workloads as W
    build.build()
    w = W.make(args.workload)
    n_inter = counts_total(w)
    stream = torch.cuda.Stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    alu = NOMINAL_ALU if args.nominal_peaks else measure_alu_peaks(0, stream)
    fmm = binding.OctoFMM(w.tree, w.theta, binding.OCTO_FP64)
    nlc = fmm.n_leaf_cells
    rho = torch.from_numpy(np.ascontiguousarray(w.rho.reshape(-1))).cuda()
    gen = torch.Generator(device="cuda").manual_seed(7)
    dphi = torch.randn(nlc, dtype=torch.float64, device="cuda", generator=gen)
    dg = torch.randn((3, nlc), dtype=torch.float64, device="cuda", generator=gen)
    drho = torch.empty(nlc, dtype=torch.float64, device="cuda")
    with torch.cuda.stream(stream):
        fmm.forces(rho, stream=stream)
        for _ in range(args.warmup):
            binding.octo_fmm_backward(fmm.handle, dphi, dg, drho, stream)
        stream.synchronize()
        ms = []
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(0) as clk:
            for _ in range(args.steps):
                flush.zero_()
                e0.record(stream)
                binding.octo_fmm_backward(fmm.handle, dphi, dg, drho, stream)
                e1.record(stream)
                stream.synchronize()
                ms.append(e0.elapsed_time(e1))
    binding.octo_fmm_stats(fmm.handle)  # raises on a failed device-side check
    t = float(np.mean(ms))
    f64 = binding.octo_fmm_get_option(fmm.handle, 24)  # counted float64 flops of one backward
    line = {"metric": "adjoint " + METRIC, "value": n_inter / (t / 1e3), "unit": METRIC, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t, "higher_is_better": True,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "note": w.note, "theta": w.theta, "order": 3,
                       "step": "octo_fmm_backward after one float64 forward solve",
                       "l2": "flushed before every timed step"},
            "roofline": {"bound": "alu", "pipe": "fp64", "achieved": f64 / (t / 1e3) / 1e12, "peak": alu["fp64"],
                         "unit": "TFLOP/s", "frac": f64 / (t / 1e3) / 1e12 / alu["fp64"],
                         "flops_per_step": f64, "peak_source": alu["source"]},
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="adaptive7")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--interior-shape", type=int, nargs=2, metavar=("CHUNK", "SPLIT"), default=None,
                    help="mixed precision: fix the interior shape (32|64 entries per float32 partial, "
                         "1|2 = half|quarter-node items) instead of autotuning it")
    ap.add_argument("--oracle-timing", action="store_true",
                    help="full oracle solves of the small configurations on the host cores (no GPU)")
    ap.add_argument("--oracle-one-thread", nargs="*", default=["uniform16_s0", "binary64"],
                    help="configurations of --oracle-timing also timed on one thread")
    ap.add_argument("--backward-only", action="store_true",
                    help="time the float64 adjoint (octo_fmm_backward) alone on the workload")
    ap.add_argument("--paced", type=int, choices=(0, 1), default=None,
                    help="mixed precision: fix the persistent queue (1 = paced, 0 = merged) instead of autotuning it")
    ap.add_argument("--corr64", action="store_true",
                    help="mixed precision with the angular-momentum correction in float64 (per-kind launches)")
    ap.add_argument("--nominal-peaks", action="store_true",
                    help="use the nominal float64/float32 peaks instead of measuring them on the device")
    ap.add_argument("--ref-seconds", type=float, default=15.0,
                    help="oracle seconds of the cpu_baseline sample and at most per reference step")
    ap.add_argument("--ref-budget", type=float, default=150.0,
                    help="oracle seconds of all timed reference steps together")
    ap.add_argument("--strategy", default="auto", choices=sorted(STRATEGY),
                    help="interaction phase: autotuned (default), per-kind launches or persistent queue")
    ap.add_argument("--blocks", type=int, default=0, choices=(0, 1, 2, 3),
                    help="register budget of a forced persistent launch (blocks per SM; 3: mixed only)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.backward_only:
        return run_backward(args)
    if args.oracle_timing:
        return run_oracle_timing(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
