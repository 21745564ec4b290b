#!/usr/bin/env python3
"""MLUPS benchmark of the fused D2Q37 time step on GB300.

Workload (N = 1): the FP64 Rayleigh-Taylor lattice of 2304 x 8192 sites (37 FP64 populations,
double-buffered, ~11.2 GB), tau = 0.9, temperature ratio 2, walls top/bottom, periodic in x.
One bench step = one fused LB time step (pull propagate + collide + wall halo write) over the
whole lattice. MLUPS = sites x steps / seconds / 1e6 (Table 1's unit).

Printed JSON line (rank 0): value = device-timed MLUPS of K steps with the lattice resident in
HBM (CUDA events on the library's stream, max over ranks); e2e = the same metric through the C
ABI from pinned host fields (lb_init upload, K steps, lb_moments download, wall clock);
roofline of the step kernel; cpu_baseline = the CPU oracle on a bounded sample; forms = the
FP32-deviation form's MLUPS and relative L2 errors; clocks sampled during the timed region.

Multi-GPU (torchrun): one independent lattice per rank (replicas, weak scaling), no collective on
the data path; barrier + max-over-ranks timing.

--impl reference times the CPU oracle (the only reference this method has: the paper ships no
code) on the same metric, rank 0 only.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

LX, LY, TAU, RATIO = 2304, 8192, 0.9, 2.0
NPOP = 37
# FP64 work of the fused step per site in this kernel's formulation: 86.2 FP64-pipe instructions
# (65.0 fused + 21.1 non-fused; ncu on step_fp64_kernel, per site), i.e. 151 flops with FMA = 2.
# The moment sums run as exact 96-bit integer sums on the integer pipe, rounded to FP64 there too,
# and each pair's equilibrium term is formed in 64-bit fixed point there (one FP64 FMA per
# population remains). The FP64 pipe issues one such instruction per lane-slot whatever its kind, so the
# ALU roofline is the FP64 instruction rate: 152 SMs x 2 per clock per SM x f_max (the 1.25 TFLOP/s
# nominal FP64 rate counts an FMA as 2 flops).
FP64_INST_PER_SITE = 86.2
FP64_FLOP_PER_SITE = 151
# The binding unit of this kernel is the integer ALU pipe (16 lanes per SM sub-partition, i.e. 64
# thread-instructions per clock per SM). Its instructions per site follow from the same capture:
# ALU share of peak 70.53 % (elapsed) x 1.0822 M cycles x 64 lanes x 152 SMs / 2359296 sites = 3147
# (of 5694 instructions per site; the FMA pipe takes the 64-bit multiplies, the FP64 pipe 86).
ALU_INST_PER_SITE = 3147
ALU_LANES_PER_CLK_SM = 64
# Pipe shares of the same capture (ncu, % of peak, active): since the pair terms and most shell
# coefficients moved to fixed point, the integer ALU pipe is the busiest.
FP64_PIPE_SHARES = {"fp64": 0.627, "alu": 0.716, "fma": 0.215, "issue": 0.648}
# The kernel sources those counts were profiled on (code_digest, below): when the code differs the
# counts are stale and the roofline's achieved and frac are reported as null
# (tests/test_bench_host.py fails on a stale table, so a committed tree carries matching counts).
FP64_INST_SOURCES = {"step_fp64.cu": "85ffbf362e557f7acf45bbbfdab6c7fd84155e6352c689134d8472c27fe87275",
                     "d2q37_gpu.cuh": "d3baaae19fce2cc02e2e1c94f075d125d5d01659018f115a632612b46c4fc86c",
                     "fixed96.cuh": "223c1f873d175ecc44292e1d48cb1cfb717e8884e9503cfe3f056c32c7b33788"}
# The algorithmic work of one site update in the oracle's plain formulation (moments, the Hermite
# equilibrium written per population, BGK relaxation with the gravity shift): 2763 flops, counted
# by compiling the oracle's collide with an operation-counting scalar type
# (oracle/count_collide_flops.cpp; tests/test_oracle_flops.py re-derives the number). The
# kernel's factored formulation needs 151 of them in FP64 (the rest runs on the integer pipes).
ORACLE_FLOP_PER_SITE = 2763
FP64_BYTES_PER_SITE = 2 * NPOP * 8       # 37 reads + 37 writes (Table 1's propagate accounting)
FP32DEV_BYTES_PER_SITE = 2 * NPOP * 4
FP64_INST_PER_CLK_SM = 2
# DRAM bytes of one step_fp64_kernel launch measured by ncu (dram__bytes_read.sum +
# dram__bytes_write.sum) on the 1152x2048 capture (profiles/step_fp64_1152x2048_full.md):
# 698.482 MB + 692.198 MB for 2359296 sites, scaled per site. Valid only for the kernel source
# it was taken on (code_digest of the files below: sha256 of the code without comments);
# otherwise reported as null.
TRAFFIC_FP64 = {"bytes_per_site": (698.482176e6 + 692.197888e6) / 2359296,
                "sources": {"step_fp64.cu": "85ffbf362e557f7acf45bbbfdab6c7fd84155e6352c689134d8472c27fe87275",
                            "d2q37_gpu.cuh": "d3baaae19fce2cc02e2e1c94f075d125d5d01659018f115a632612b46c4fc86c",
                            "fixed96.cuh": "223c1f873d175ecc44292e1d48cb1cfb717e8884e9503cfe3f056c32c7b33788"}}


# The same for step_fp32split_kernel: ncu DRAM bytes of one launch on a 1152x2048 capture
# (profiles/step_fp32split_1152x2048_full.md), 349.264 MB + 303.117 MB for 2359296 sites.
TRAFFIC_FP32SPLIT = {"bytes_per_site": (349.264128e6 + 303.117056e6) / 2359296,
                     "sources": {"step_fp32dev.cu": "9bd8776f652ce5402527ff8a5eb09373b1db75d7a1be4418d81624f303f67877",
                                 "site_fp32dev.cuh": "ed58b9d3cc6f5e6464749fb716c6985c34642f9abdd0ca704ee46d6a60204ae1",
                                 "d2q37_gpu.cuh": "d3baaae19fce2cc02e2e1c94f075d125d5d01659018f115a632612b46c4fc86c"}}


def code_digest(path):
    """sha256 of a CUDA source with its comments and whitespace removed: the measured counters stay
    valid across comment edits but not across any change of the code itself."""
    import hashlib
    import re
    with open(path, encoding="utf-8") as fh:
        text = fh.read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return hashlib.sha256(" ".join(text.split()).encode()).hexdigest()


def sources_match(table):
    csrc = os.path.join(ROOT, "paper_1804_01918_gb300", "csrc")
    for name, digest in table["sources"].items():
        try:
            if code_digest(os.path.join(csrc, name)) != digest:
                return False
        except OSError:
            return False
    return True


def env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            return json.load(fh)
    except OSError:
        return None


NVML_CLOCK_SM = 1
# clock-event reason bits of NVML's current-clocks-event-reasons mask
NVML_REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
                0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}


class Nvml:
    """Read-only NVML queries through ctypes (libnvidia-ml): SM clock, maximum SM clock, board
    power, clock-event reasons and the cumulative energy counter of one GPU. Nothing is set."""

    def __init__(self, uuid=None, index=0):
        import ctypes as C
        self.C = C
        self.lib = C.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        self.h = C.c_void_p()
        rc = 1
        if uuid:
            rc = self.lib.nvmlDeviceGetHandleByUUID(uuid.encode(), C.byref(self.h))
        if rc != 0:
            rc = self.lib.nvmlDeviceGetHandleByIndex_v2(C.c_uint(index), C.byref(self.h))
        if rc != 0:
            raise OSError("no NVML handle for the GPU")
        self._reasons = (getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None)
                         or self.lib.nvmlDeviceGetCurrentClocksThrottleReasons)

    def _uint(self, fn, *args):
        v = self.C.c_uint()
        return v.value if fn(self.h, *args, self.C.byref(v)) == 0 else None

    def sm_mhz(self):
        return self._uint(self.lib.nvmlDeviceGetClockInfo, self.C.c_int(NVML_CLOCK_SM))

    def sm_max_mhz(self):
        return self._uint(self.lib.nvmlDeviceGetMaxClockInfo, self.C.c_int(NVML_CLOCK_SM))

    def power_w(self):
        mw = self._uint(self.lib.nvmlDeviceGetPowerUsage)
        return None if mw is None else mw / 1000.0

    def reasons(self):
        v = self.C.c_ulonglong()
        return v.value if self._reasons(self.h, self.C.byref(v)) == 0 else None

    def energy_mj(self):
        v = self.C.c_ulonglong()
        return v.value if self.lib.nvmlDeviceGetTotalEnergyConsumption(self.h, self.C.byref(v)) == 0 else None


class GpuSampler:
    """Samples (host monotonic time, SM MHz, max SM MHz, board W, reason names) of one GPU on a
    background thread every `interval` s while running: through NVML, or through an nvidia-smi
    CSV stream (100 ms, host-stamped on arrival) when NVML cannot be loaded. Only the samples
    inside a window given later are used (samples_in_window)."""

    QUERY = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")

    def __init__(self, nvml=None, gpu_index=0, interval=0.02):
        self.nvml = nvml
        self.gpu_index = gpu_index
        self.interval = interval
        self.samples = []
        self._stop = None
        self._thread = None
        self._proc = None

    def start(self):
        import threading
        self._stop = threading.Event()
        if self.nvml is not None:
            target = self._run_nvml
        else:
            cmd = ["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                   "-lms", "100", "-i", str(self.gpu_index)]
            try:
                self._proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                              text=True)
            except OSError:
                self._proc = None
                return
            target = self._run_smi
        self._thread = threading.Thread(target=target, daemon=True)
        self._thread.start()

    def _run_nvml(self):
        n = self.nvml
        while not self._stop.is_set():
            mask = n.reasons()
            names = [] if mask is None else [v for b, v in NVML_REASONS.items() if mask & b]
            self.samples.append((time.monotonic(), n.sm_mhz(), n.sm_max_mhz(), n.power_w(), names))
            self._stop.wait(self.interval)

    def _run_smi(self):
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self._proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                vals = [float(parts[0]), float(parts[1]), float(parts[2])]
            except ValueError:
                continue
            active = [nm for nm, v in zip(names, parts[3:7]) if v.lower().startswith("active")]
            self.samples.append((time.monotonic(), *vals, active))
            if self._stop.is_set():
                break

    def stop(self):
        if self._stop is not None:
            self._stop.set()
        if self._proc is not None:
            self._proc.terminate()
            try:
                self._proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self._proc.kill()
        if self._thread is not None:
            self._thread.join(timeout=5)


def samples_in_window(samples, t0, t1):
    """The samples taken at host times t0 <= t <= t1."""
    return [s for s in samples if t0 <= s[0] <= t1]


def summarize_clocks(samples, source):
    """Clock record of a window's samples: median SM clock, the maximum clock, median board power
    and every throttle reason seen."""
    sm = [s[1] for s in samples if s[1] is not None]
    if not sm:
        return {"sm_mhz": None, "sm_max_mhz": None, "samples": 0, "reasons": ["no samples in the window"],
                "source": source}
    smax = [s[2] for s in samples if s[2] is not None]
    power = [s[3] for s in samples if s[3] is not None]
    reasons = sorted({r for s in samples for r in s[4]})
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax) if smax else None,
            "samples": len(sm), "power_w_median": statistics.median(power) if power else None,
            "reasons": reasons, "source": source}


def energy_from_counter(e0_mj, e1_mj, seconds, steps, sites):
    """Energy to solution per step from a cumulative energy counter read before and after `steps`
    steps that took `seconds` (the analog of the paper's RAPL package + DRAM energy per iteration,
    Sec. 5 and Fig. 5; on GB300 the board energy includes the HBM)."""
    if e0_mj is None or e1_mj is None or e1_mj <= e0_mj or steps <= 0 or seconds <= 0:
        return None
    j = (e1_mj - e0_mj) * 1e-3
    return {"joules_per_step": round(j / steps, 4), "nJ_per_site_update": round(j / steps / sites * 1e9, 3),
            "power_w": round(j / seconds, 1), "window_s": round(seconds, 3), "window_steps": steps}


def energy_from_power(samples, seconds, steps, sites):
    """The same from board-power samples inside the window (median power x window time)."""
    power = [s[3] for s in samples if s[3] is not None]
    if not power or steps <= 0 or seconds <= 0:
        return None
    j = statistics.median(power) * seconds
    return {"joules_per_step": round(j / steps, 4), "nJ_per_site_update": round(j / steps / sites * 1e9, 3),
            "power_w": round(statistics.median(power), 1), "window_s": round(seconds, 3),
            "window_steps": steps, "samples": len(power)}


def energy_window_steps(ms_per_step, min_seconds=2.0, at_least=1):
    """Steps of the energy window: enough for min_seconds at the measured step time."""
    return int(max(at_least, math.ceil(min_seconds * 1e3 / max(ms_per_step, 1e-6))))


def measure_energy(run, sync, ms_per_step, sites, nvml, sampler):
    """Energy per step over its own window of >= 2 s of steps (after the timed region), from NVML's
    cumulative energy counter read before and after, else from the power samples in the window."""
    steps = energy_window_steps(ms_per_step)
    sync()
    e0 = nvml.energy_mj() if nvml else None
    t0 = time.monotonic()
    run(steps)
    sync()
    t1 = time.monotonic()
    e1 = nvml.energy_mj() if nvml else None
    out = energy_from_counter(e0, e1, t1 - t0, steps, sites)
    win = samples_in_window(sampler.samples, t0, t1)
    if out is not None:
        out["source"] = "NVML cumulative energy counter over a window of steps after the timed region"
    else:
        out = energy_from_power(win, t1 - t0, steps, sites)
        if out is not None:
            out["source"] = "median board power sampled in a window of steps after the timed region"
    if out is not None:
        out["clocks_in_window"] = summarize_clocks(win, "in the energy window")
    return out


def open_nvml(local_rank):
    """NVML handle of this rank's GPU (by UUID from torch), or None if NVML is unavailable."""
    try:
        import torch
        uuid = getattr(torch.cuda.get_device_properties(local_rank), "uuid", None)
        uuid = f"GPU-{uuid}" if uuid is not None and not str(uuid).startswith("GPU-") else uuid
        return Nvml(uuid=None if uuid is None else str(uuid), index=visible_gpu_index(local_rank))
    except (OSError, AttributeError):
        return None


def sites_of(lx, ly):
    return lx * ly


def visible_gpu_index(local_rank):
    cvd = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    ids = [s for s in cvd.split(",") if s.strip() != ""]
    if ids and local_rank < len(ids) and ids[local_rank].strip().isdigit():
        return int(ids[local_rank])
    return local_rank


# ----------------------------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline leg and --impl reference)
# ----------------------------------------------------------------------------------------------

def oracle_mlups(rows, steps, nthreads):
    """Oracle MLUPS on a band of `rows` rows of the 2304-wide Rayleigh-Taylor workload."""
    from oracle import oracle as orc
    from paper_1804_01918_gb300 import inputs
    st = inputs.rayleigh_taylor(LX, LY, R=RATIO, seed=0)
    y0 = LY // 2 - rows // 2
    sub = [a[y0:y0 + rows] for a in (st.rho, st.ux, st.uy, st.T)]
    f0 = orc.equilibrium(*sub)
    t0 = time.perf_counter()
    orc.run(f0, tau=TAU, nsteps=steps, gy=st.gy, T_top=st.T_top, T_bottom=st.T_bottom,
            nthreads=nthreads)
    dt = time.perf_counter() - t0
    return LX * rows * steps / dt / 1e6, dt


def cpu_baseline(target_s=20.0):
    """The oracle on the same workload, as many whole steps as fit ~target_s of CPU time (a
    band of rows instead when even one full step would take longer)."""
    from oracle import oracle as orc
    nthreads = orc.default_threads()
    rate, _ = oracle_mlups(min(LY, 2048), 3, nthreads)      # calibration: 3 steps of a 2048-row band
    full_step_s = LX * LY / (rate * 1e6)
    if full_step_s <= target_s:
        rows, steps = LY, int(max(1, min(50, round(target_s / full_step_s))))
    else:
        rows, steps = int(max(64, LY * target_s / full_step_s)), 1
    v, dt = oracle_mlups(rows, steps, nthreads)
    if rows == LY and dt < 0.5 * target_s and steps < 50:  # calibration was pessimistic: redo once
        steps = int(min(50, max(steps + 1, round(steps * target_s / dt))))
        v, dt = oracle_mlups(rows, steps, nthreads)
    what = ("the whole" if rows == LY else f"a {LX}x{rows} band (walls at the band edges) of the")
    return {"value": round(v, 3), "unit": "MLUPS", "cores": nthreads, "kind": "oracle",
            "sample": f"{steps} steps of {what} {LX}x{LY} FP64 Rayleigh-Taylor workload, "
                      f"{dt:.1f} s of CPU time"}


def run_reference(args):
    rank = env_int("RANK", 0)
    if rank != 0:
        return 0
    from oracle import oracle as orc
    nthreads = orc.default_threads()
    # calibration on a 512-row band: large enough (~0.7 GB of populations) to run at the
    # memory-bound rate of the full lattice rather than from the caches
    rate, _ = oracle_mlups(512, 1, nthreads)
    per_step = 150.0 / max(1, args.steps + args.warmup)
    rows = int(max(16, min(LY, rate * 1e6 * per_step / LX)))
    from paper_1804_01918_gb300 import inputs
    st = inputs.rayleigh_taylor(LX, LY, R=RATIO, seed=0)
    y0 = LY // 2 - rows // 2
    f = orc.equilibrium(*[a[y0:y0 + rows] for a in (st.rho, st.ux, st.uy, st.T)])
    kw = dict(tau=TAU, gy=st.gy, T_top=st.T_top, T_bottom=st.T_bottom, nthreads=nthreads)
    f = orc.run(f, nsteps=args.warmup, **kw)
    t0 = time.perf_counter()
    orc.run(f, nsteps=args.steps, **kw)
    dt = time.perf_counter() - t0
    value = LX * rows * args.steps / dt / 1e6
    sample = (f"each step a {LX}x{rows} band of the {LX}x{LY} FP64 Rayleigh-Taylor workload "
              f"(walls at the band edges)")
    line = {"impl": "reference", "metric": metric_name("fp64"),
            "value": round(value, 3), "unit": "MLUPS", "n_gpus": 0, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(1),
            "cpu_baseline": {"value": round(value, 3), "unit": "MLUPS", "cores": nthreads,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(value, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


PRECISION_LABEL = {"fp64": "FP64", "fp32dev": "FP32-deviation", "fp32split": "FP32 exact-split"}


def workload_config(world, precision="fp64"):
    bpv = 8 if precision == "fp64" else 4
    half = 37 * LX * (LY + 6) * bpv / 1e9
    return {"workload": f"D2Q37 {PRECISION_LABEL[precision]} Rayleigh-Taylor {LX}x{LY} (18.9M "
                        f"sites, ~{2 * half:.1f} GB double-buffered), tau {TAU}, T ratio 1:{RATIO}, "
                        f"walls top/bottom, periodic x, fused propagate+collide+walls",
            "Lx": LX, "Ly": LY, "tau": TAU, "precision": precision,
            "replicas": world, "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
            "l2": f"inputs larger than L2 ({half:.1f} GB read + {half:.1f} GB written per step vs "
                  f"129 MB L2)"}


# The headline metric: the plain FP64 step's MLUPS on one GB300, with the FP32, batched and learned
# forms beside it (under "forms", each with its L2 error against the FP64 step).
HEADLINE_METRIC = "D2Q37 MLUPS on 1 GB300: FP64 plain vs FP32/batched/NN-collide at stated L2 err"


def metric_name(precision="fp64"):
    if precision == "fp64":
        return HEADLINE_METRIC
    return f"D2Q37 MLUPS, fused {PRECISION_LABEL[precision]} LB step (propagate+collide+walls)"


# ----------------------------------------------------------------------------------------------

def device_peak_terms(torch, local, nvml, clocks):
    """(SM count, maximum SM clock in MHz, where they came from) of this rank's GPU: the SM count
    from the CUDA device properties, the maximum SM clock from NVML (else from the clock samples,
    else the recipe's 2070 MHz)."""
    sms = int(torch.cuda.get_device_properties(local).multi_processor_count)
    mhz, src = None, None
    if nvml is not None:
        mhz = nvml.sm_max_mhz()
        src = "SM count from cudaDeviceProp, max SM clock from NVML"
    if not mhz and clocks.get("sm_max_mhz"):
        mhz, src = clocks["sm_max_mhz"], "SM count from cudaDeviceProp, max SM clock from the clock samples"
    if not mhz:
        mhz, src = 2070.0, "SM count from cudaDeviceProp, max SM clock the recipe's 2070 MHz"
    return sms, float(mhz), src


def fp64_probe(lb, torch, stream, kind="fp64"):
    """Achieved FP64 FMA rate of the library's probe (TFLOP/s, FMA = 2 flops). kind "fp64": chains
    that settle on a fixed point; "fp64_varying": operands that keep changing."""
    blocks, threads, iters = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count * 8, 256, 2048
    out = torch.empty(blocks * threads, dtype=torch.float64, device="cuda")
    with torch.cuda.stream(stream):
        lb.probe_fma(kind, blocks, threads, iters, out, stream)   # warm-up
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lb.probe_fma(kind, blocks, threads, iters, out, stream)
        e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    return blocks * threads * 16 * iters / (ms * 1e-3) / 1e12


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-forms", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--only", choices=["ensemble", "learned"], default=None,
                    help="run only this form (profiling): the ensemble or the learned step")
    ap.add_argument("--members", type=int, default=64, help="ensemble members (with --only ensemble)")
    ap.add_argument("--pairs", type=int, default=10_000_000, help="training pairs (with --only learned)")
    ap.add_argument("--epochs", type=int, default=20, help="training epochs (with --only learned)")
    ap.add_argument("--lattice", default=None,
                    help="LXxLY of a smaller case for profiling (default: the 2304x8192 workload)")
    ap.add_argument("--precision", choices=["fp64", "fp32dev", "fp32split"], default="fp64")
    ap.add_argument("--staging", choices=["plain", "tma"], default="plain",
                    help="fp32split: read the pulled rows with plain loads or TMA-staged tiles")
    args = ap.parse_args()
    if args.lattice:
        global LX, LY
        LX, LY = (int(v) for v in args.lattice.lower().split("x"))
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.only:
        return run_only(args)

    import numpy as np
    import torch

    from paper_1804_01918_gb300 import build as pkg_build
    from paper_1804_01918_gb300 import inputs, lb

    from paper_1804_01918_gb300 import replicas
    rank, world, local = replicas.rank_env()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl" if torch.cuda.is_available() else "gloo")
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (no CPU fallback)")
    torch.cuda.set_device(local)
    pkg_build.build()

    st = inputs.rayleigh_taylor(LX, LY, R=RATIO, seed=replicas.replica_seed(rank))
    stream = torch.cuda.Stream()
    lat = lb.Lattice.from_fields(st, tau=TAU, stream=stream, precision=args.precision)
    if args.precision == "fp32split" and args.staging == "tma":
        lat.set_staging(True)
    lat.step(args.warmup)
    lat.sync()
    probe_tf = fp64_probe(lb, torch, stream)
    probe_var_tf = fp64_probe(lb, torch, stream, "fp64_varying")

    nvml = open_nvml(local)
    sampler = GpuSampler(nvml, visible_gpu_index(local))
    sampler.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_start = time.monotonic()
    e0.record(stream)
    lat.step(args.steps)
    e1.record(stream)
    e1.synchronize()
    t_end = time.monotonic()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    lat.sync()    # raises on a non-finite state
    clocks = summarize_clocks(samples_in_window(sampler.samples, t_start, t_end),
                              "NVML every 20 ms in the timed region" if nvml else
                              "nvidia-smi every 100 ms in the timed region")
    energy = measure_energy(lat.step, lat.sync, ms / args.steps, sites_of(LX, LY), nvml, sampler)
    sampler.stop()
    ms = replicas.max_over_ranks(ms, dist, device="cuda")
    sites = LX * LY
    value = replicas.aggregate_mlups(sites, args.steps, ms, world)
    kernel_s = ms * 1e-3 / args.steps
    lat.close()
    del lat

    # ---- end to end through the C ABI from pinned host buffers ----
    e2e = None
    if not args.no_e2e:
        pin = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
               for a in (st.rho, st.ux, st.uy, st.T)]
        outs = [torch.empty((LY, LX), dtype=torch.float64).pin_memory() for _ in range(4)]
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        lat2 = lb.Lattice(LX, LY, TAU, *pin, gy=st.gy, T_top=st.T_top, T_bottom=st.T_bottom,
                          stream=stream)
        lat2.step(args.steps)
        lat2.moments(out=outs)
        t1 = time.perf_counter()
        lat2.close()
        del lat2
        dt = replicas.max_over_ranks(t1 - t0, dist, device="cuda")
        e2e = {"value": round(world * sites * args.steps / dt / 1e6, 2), "unit": "MLUPS",
               "h2d_bytes_per_step": round(4 * 8 * sites / args.steps, 1),
               "d2h_bytes_per_step": round(4 * 8 * sites / args.steps, 1),
               "note": "one lb_init upload of rho,u,T (32 B/site) and one lb_moments download "
                       "(32 B/site) per K-step run, amortised per step"}

    # ---- roofline of the step kernel ----
    hbm = (measured_peaks() or {}).get("hbm_gbs", 6800.0)
    if args.precision == "fp64":
        sm_count, sm_max_mhz, peak_src = device_peak_terms(torch, local, nvml, clocks)
        peak = sm_count * FP64_INST_PER_CLK_SM * sm_max_mhz * 1e6 / 1e12
        counts_valid = sources_match({"sources": FP64_INST_SOURCES})
        if not counts_valid:
            print("bench.py: step_fp64 sources changed since FP64_INST_PER_SITE was profiled; "
                  "roofline achieved/frac reported as null", file=sys.stderr)
        inst_rate = FP64_INST_PER_SITE * sites / kernel_s / 1e12 if counts_valid else None
        traffic = (round(TRAFFIC_FP64["bytes_per_site"] * sites) if sources_match(TRAFFIC_FP64)
                   and (LX, LY) == (2304, 8192) else None)
        alu_rate = ALU_INST_PER_SITE * sites / kernel_s / 1e12 if counts_valid else None
        alu_peak = sm_count * ALU_LANES_PER_CLK_SM * sm_max_mhz * 1e6 / 1e12
        roofline = {"bound": "alu", "kernel": "step_fp64_kernel",
                    "achieved": None if alu_rate is None else round(alu_rate, 3),
                    "peak": round(alu_peak, 3), "unit": "T integer-ALU instructions/s",
                    "frac": None if alu_rate is None else round(alu_rate / alu_peak, 4), "traffic": traffic,
                    "peak_note": f"integer ALU pipe: {sm_count} SMs x 64 instructions per clock per SM x "
                                 f"{sm_max_mhz:.0f} MHz ({peak_src}); the step's binding unit since its pair "
                                 "terms and most shell coefficients run in fixed point; ALU instructions per "
                                 "site from ncu's ALU-pipe share of the 1152x2048 capture",
                    "alu_inst_per_site": ALU_INST_PER_SITE,
                    "fp64_pipe": {"achieved": None if inst_rate is None else round(inst_rate, 4),
                                  "peak": round(peak, 4), "unit": "T FP64-instructions/s",
                                  "frac": None if inst_rate is None else round(inst_rate / peak, 4),
                                  "peak_note": f"FP64 pipe: {sm_count} SMs x 2 FP64 instructions per clock per "
                                               f"SM x {sm_max_mhz:.0f} MHz, the recipe's 1.25 TFLOP/s nominal "
                                               "with FMA = 2 flops"},
                    "sm_count": sm_count, "sm_max_mhz": sm_max_mhz, "peak_terms_source": peak_src,
                    "algorithmic_fp64_inst_per_site": FP64_INST_PER_SITE,
                    "pipe_shares_ncu": FP64_PIPE_SHARES if counts_valid else None,
                    "inst_count_matches_sources": counts_valid,
                    "achieved_tflops": round(FP64_FLOP_PER_SITE * sites / kernel_s / 1e12, 4),
                    "oracle_flop_per_site": ORACLE_FLOP_PER_SITE,
                    "achieved_tflops_oracle_formulation": round(ORACLE_FLOP_PER_SITE * sites / kernel_s / 1e12, 4),
                    "peak_tflops": round(2 * peak, 4),
                    "probe_fp64_tflops": round(probe_tf, 4),
                    "probe_fp64_varying_tflops": round(probe_var_tf, 4),
                    "frac_of_varying_probe": (None if inst_rate is None
                                              else round(inst_rate / (probe_var_tf / 2), 4)),
                    "probe_note": "FMA chains that settle on a fixed point reach nearly the nominal "
                                  "rate; with operands that keep changing GB300's FP64 pipe sustains "
                                  "less (varying probe), the rate real data sees",
                    "traffic_note": "ncu dram bytes of a 1152x2048 launch scaled to 2304x8192 by sites",
                    "hbm_achieved_gbs": round(FP64_BYTES_PER_SITE * sites / kernel_s / 1e9, 1),
                    "hbm_frac": round(FP64_BYTES_PER_SITE * sites / kernel_s / 1e9 / hbm, 4)}
    else:
        gbs = FP32DEV_BYTES_PER_SITE * sites / kernel_s / 1e9
        kname = "step_fp32split_tma_kernel" if args.staging == "tma" else f"step_{args.precision}_kernel"
        traffic32 = (round(TRAFFIC_FP32SPLIT["bytes_per_site"] * sites)
                     if args.precision == "fp32split" and args.staging == "plain"
                     and sources_match(TRAFFIC_FP32SPLIT) and (LX, LY) == (2304, 8192) else None)
        roofline = {"bound": "hbm", "kernel": kname, "achieved": round(gbs, 1),
                    "peak": hbm, "unit": "GB/s", "frac": round(gbs / hbm, 4), "traffic": traffic32,
                    "peak_note": "MEASURED_PEAKS.json hbm_gbs (of measured)"}

    # ---- FP32-deviation form: MLUPS and L2 error against the FP64 path ----
    forms = None
    if not args.no_forms and rank == 0 and args.precision == "fp64":  # forms are compared with FP64
        forms = measure_forms(lb, torch, np, st, stream, value / world)
        net = None
        if not args.no_learned:
            forms["learned"], net = measure_learned(lb, torch, np, inputs, st, stream,
                                                    forms["fp32split"]["mlups"])
            forms["learned"]["speedup_vs_fp64"] = round(forms["learned"]["mlups"] / (value / world), 3)
        for form, e in measure_accuracy(lb, np, st, stream, learned_net=net).items():
            forms[form]["rel_l2_vs_fp64"] = e
        if net is not None:
            net.close()
        if not args.no_ensemble:
            forms["ensemble"] = measure_ensemble(lb, torch, np, inputs, value / world)
            forms["ensemble_per_item"] = measure_ensemble(lb, torch, np, inputs, value / world,
                                                          per_item=True,
                                                          tile=tuple(forms["ensemble"]["tile"]))
        forms["table1_1024x8192"] = measure_table1(lb, torch, np, inputs)

    line = {"metric": metric_name(args.precision),
            "value": round(value, 2), "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "f32",
            "data": "synthetic (seeded Rayleigh-Taylor fields)",
            "config": workload_config(world, args.precision),
            "roofline": roofline, "clocks": clocks, "gpu_launches": args.steps,
            "energy": energy,
            "e2e": e2e,
            "paper_context": {"KNL 7230 flat/quad Global MLUPS 1024x8192": 119,
                              "P100 Global MLUPS 1024x8192": 232}}
    if forms:
        line["forms"] = forms
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_only(args):
    """One form alone, for profiling: prints its measurement as one JSON line."""
    import numpy as np
    import torch

    from paper_1804_01918_gb300 import build as pkg_build
    from paper_1804_01918_gb300 import inputs, lb
    pkg_build.build()
    if args.only == "ensemble":
        out = measure_ensemble(lb, torch, np, inputs, 1.0, n=args.members, steps=args.steps)
    else:
        st = inputs.rayleigh_taylor(LX, LY, R=RATIO, seed=0)
        out, net = measure_learned(lb, torch, np, inputs, st, torch.cuda.Stream(), 1.0,
                                   epochs=args.epochs, steps=args.steps, pairs=args.pairs)
        net.close()
    print(json.dumps({"only": args.only, "config": {"Lx": LX, "Ly": LY}, **out}), flush=True)
    return 0


def measure_forms(lb, torch, np, st, stream, fp64_mlups):
    """MLUPS (device-timed, 1000 steps) and HBM fraction of both FP32-deviation forms on the bench
    workload."""
    sites = LX * LY
    hbm = (measured_peaks() or {}).get("hbm_gbs", 6800.0)
    out = {}
    for form in ("fp32dev", "fp32split"):
        lat = lb.Lattice.from_fields(st, tau=TAU, stream=stream, precision=form)
        lat.step(10)
        lat.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lat.step(1000)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        lat.sync()
        lat.close()
        mlups = sites * 1000 / (ms * 1e-3) / 1e6
        gbs = FP32DEV_BYTES_PER_SITE * mlups * 1e6 / 1e9
        out[form] = {"mlups": round(mlups, 1), "speedup_vs_fp64": round(mlups / fp64_mlups, 3),
                     "hbm_gbs": round(gbs, 1), "hbm_frac": round(gbs / hbm, 4)}
    return out


def measure_accuracy(lb, np, st, stream, learned_net=None):
    """Relative L2 error of rho and T of the FP32 forms (and of the learned collide) against the
    FP64 path at steps 100, 500 and 1000, all from the same initial state. The FP64 path is the
    reference at this size: it matches the CPU oracle to 1e-12 in the tests, including sampled
    sites of this very workload."""
    lats = {form: lb.Lattice.from_fields(st, tau=TAU, stream=stream, precision=form)
            for form in ("fp64", "fp32dev", "fp32split")}
    compared = ["fp32dev", "fp32split"]
    if learned_net is not None:
        lats["learned"] = lb.Lattice.from_fields(st, tau=TAU, stream=stream, precision="fp32split")
        lats["learned"].set_collide_learned(learned_net, bound=1e-4, check_every=1)
        compared.append("learned")
    done = 0
    errs = {form: {} for form in compared}
    for mark in (100, 500, 1000):
        for lat in lats.values():
            lat.step(mark - done)
        done = mark
        ra, _, _, Ta = lats["fp64"].moments()
        for form in compared:
            rb, _, _, Tb = lats[form].moments()
            errs[form][str(mark)] = {"rho": float(np.linalg.norm(rb - ra) / np.linalg.norm(ra)),
                                     "T": float(np.linalg.norm(Tb - Ta) / np.linalg.norm(Ta))}
    for lat in lats.values():
        lat.close()
    return errs


def collect_training_pairs(lb, torch, np, inputs, total=10_000_000, seed=0):
    """(pre, post) FP32-deviation pairs from the plain collide, as configured: every site of the
    64x256 Rayleigh-Taylor run at each of its 100 steps (1.64 M pairs), and the rest sampled at
    random sites of the 2304x8192 run every 100 of its 1000 steps (FP32 storage, exact-split
    accumulation)."""
    pre, post = [], []
    st1 = inputs.rayleigh_taylor(64, 256, R=RATIO, seed=seed)
    lat = lb.Lattice.from_fields(st1, tau=TAU, precision="fp32split")
    sites = torch.arange(64 * 256, dtype=torch.int32, device="cuda")
    for _ in range(100):
        a = torch.empty((sites.numel(), NPOP), dtype=torch.float32, device="cuda")
        b = torch.empty_like(a)
        with torch.cuda.stream(lat.stream):
            lat.collect_pairs(sites, a, b)
        lat.step(1)
        pre.append(a)
        post.append(b)
    lat.sync()
    lat.close()
    remaining = max(1280, total - sum(a.shape[0] for a in pre))
    st3 = inputs.rayleigh_taylor(LX, LY, R=RATIO, seed=seed + 1)
    lat = lb.Lattice.from_fields(st3, tau=TAU, precision="fp32split")
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    per = remaining // 10
    for k in range(10):
        m = per if k < 9 else remaining - 9 * per
        idx = torch.randint(0, LX * LY, (m,), dtype=torch.int32, device="cuda", generator=gen)
        a = torch.empty((m, NPOP), dtype=torch.float32, device="cuda")
        b = torch.empty_like(a)
        torch.cuda.current_stream().synchronize()
        with torch.cuda.stream(lat.stream):
            lat.collect_pairs(idx, a, b)
        lat.step(100)
        pre.append(a)
        post.append(b)
    lat.sync()
    lat.close()
    return torch.cat(pre), torch.cat(post)


def measure_learned(lb, torch, np, inputs, st, stream, fp32split_mlups, epochs=20, steps=1000,
                    pairs=10_000_000):
    """Learned collide at the bench size: train the MLP (20 epochs, batch 4096, Adam 1e-3) on 10 M
    pairs, then run the learned LB step (bound 1e-4 per 32x32 tile, checked every step) and report
    its MLUPS, the fraction of tiles kept on the network and its error against the FP64 path."""
    t0 = time.perf_counter()
    pre, post = collect_training_pairs(lb, torch, np, inputs, total=pairs)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    net = lb.MLP(seed=0)
    t0 = time.perf_counter()
    losses = net.train(pre, post, epochs=epochs, batch=4096, lr=1e-3, seed=0)
    t_train = time.perf_counter() - t0
    npairs = int(pre.shape[0])
    del pre, post
    torch.cuda.empty_cache()
    sites = LX * LY
    lat = lb.Lattice.from_fields(st, tau=TAU, stream=stream, precision="fp32split")
    lat.set_collide_learned(net, bound=1e-4, check_every=1)
    lat.step(10)
    lat.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    lat.step(steps)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    lat.sync()
    stats = lat.learned_stats()
    lat.close()
    mlups = sites * steps / (ms * 1e-3) / 1e6
    kept = 1.0 - stats["tiles_fallback"] / max(1, stats["tiles_checked"])
    # the same network with the check amortised over 10 steps (tiles keep their last decision in
    # between): what the learned collide costs when it does not also run the plain one every step
    lat = lb.Lattice.from_fields(st, tau=TAU, stream=stream, precision="fp32split")
    lat.set_collide_learned(net, bound=1e-4, check_every=10)
    lat.step(10)
    lat.sync()
    e0.record(stream)
    lat.step(steps)
    e1.record(stream)
    e1.synchronize()
    ms10 = e0.elapsed_time(e1)
    lat.sync()
    stats10 = lat.learned_stats()
    lat.close()
    kept10 = 1.0 - stats10["tiles_fallback"] / max(1, stats10["tiles_checked"])
    out = {"mlups": round(mlups, 1), "speedup_vs_fp32split": round(mlups / fp32split_mlups, 3),
           "tiles_kept_learned": round(kept, 4), "max_tile_residual": stats["max_residual"],
           "mlups_check_every_10": round(sites * steps / (ms10 * 1e-3) / 1e6, 1),
           "tiles_kept_learned_check_every_10": round(kept10, 4),
           "bound": 1e-4, "check_every": 1, "train_pairs": npairs, "epochs": epochs,
           "final_loss": float(losses[-1]), "first_epoch_loss": float(losses[0]),
           "train_s": round(t_train, 1), "pair_generation_s": round(t_data, 1),
           "train_samples_per_s": round(npairs * epochs / t_train, 0)}
    return out, net


def measure_table1(lb, torch, np, inputs, reps=20):
    """The paper's per-kernel metrics (Table 1) on GB300 at its 1024 x 8192 lattice, FP64:
    separate propagate and collide kernels timed launch by launch (CUDA events), propagate GB/s
    with 592 B per site, collide MLUPS and GF/s (with the paper's ~6600 flop/site, as Table 1
    derives it, and with this kernel's FP64 flops per site), and Global MLUPS of the two-kernel step and of the
    fused step."""
    Lx, Ly = 1024, 8192
    sites = Lx * Ly
    st = inputs.rayleigh_taylor(Lx, Ly, R=RATIO, seed=0)
    stream = torch.cuda.Stream()
    lat = lb.Lattice.from_fields(st, tau=TAU, stream=stream)
    for _ in range(3):
        lat.propagate()
        lat.collide()
    lat.sync()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3 * reps)]
    for k in range(reps):
        ev[3 * k].record(stream)
        lat.propagate()
        ev[3 * k + 1].record(stream)
        lat.collide()
        ev[3 * k + 2].record(stream)
    ev[-1].synchronize()
    lat.sync()
    t_prop = sum(ev[3 * k].elapsed_time(ev[3 * k + 1]) for k in range(reps)) / reps
    t_coll = sum(ev[3 * k + 1].elapsed_time(ev[3 * k + 2]) for k in range(reps)) / reps
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    lat.step(16)
    e0.record(stream)
    lat.step(10 * 16)
    e1.record(stream)
    e1.synchronize()
    t_fused = e0.elapsed_time(e1) / 160
    lat.sync()
    lat.close()
    coll_mlups = sites / (t_coll * 1e-3) / 1e6
    return {"lattice": [Lx, Ly], "T_prop_ms": round(t_prop, 4), "T_coll_ms": round(t_coll, 4),
            "propagate_GBs": round(FP64_BYTES_PER_SITE * sites / (t_prop * 1e-3) / 1e9, 1),
            "collide_MLUPS": round(coll_mlups, 1),
            "collide_GFs_at_6600_flop_per_site": round(coll_mlups * 6600 / 1e3, 1),
            f"collide_GFs_at_{FP64_FLOP_PER_SITE}_flop_per_site": round(coll_mlups * FP64_FLOP_PER_SITE / 1e3, 1),
            "global_MLUPS_two_kernel": round(sites / ((t_prop + t_coll) * 1e-3) / 1e6, 1),
            "global_MLUPS_fused": round(sites / (t_fused * 1e-3) / 1e6, 1),
            "paper_KNL_7230_flat": {"T_prop_ms": 12.5, "T_coll_ms": 50.3, "propagate_GBs": 398,
                                    "collide_GFs": 1100, "collide_MLUPS": 166, "global_MLUPS": 119},
            "paper_P100": {"T_prop_ms": 12.5, "T_coll_ms": 24.1, "propagate_GBs": 396,
                           "collide_GFs": 2253, "collide_MLUPS": 340, "global_MLUPS": 232}}


def measure_ensemble(lb, torch, np, inputs, fp64_mlups, n=64, seed=0, steps=300, per_item=False,
                     tile=None):
    """Batched ensemble: n seed-drawn Rayleigh-Taylor lattices (Lx uniform over multiples of 32 in
    [128, 1024], Ly = 4 Lx, Atwood in [0.05, 0.5], tau in [tau_min(A), 1.2]), FP32 storage (exact-split
    accumulation), autotuned tile shape (or the given one), 100-step CUDA graphs; MLUPS = sum of
    sites x steps / s. The launch: one persistent grid per step whose co-resident blocks claim
    the work items in list order (default), or per_item: one block per work item."""
    descs = inputs.ensemble_members(n, seed=seed)
    specs = []
    for d in descs:
        st = inputs.rayleigh_taylor(d["Lx"], d["Ly"], R=d["R"], seed=d["seed"])
        specs.append({"Lx": d["Lx"], "Ly": d["Ly"], "tau": d["tau"], "gy": st.gy,
                      "T_top": st.T_top, "T_bottom": st.T_bottom, "rho": st.rho, "ux": st.ux,
                      "uy": st.uy, "T": st.T})
    stream = torch.cuda.Stream()
    ens = lb.Ensemble(specs, precision="fp32split", graph_steps=100, stream=stream,
                      per_item=per_item, tile=tile or (0, 0))
    specs = None
    if tile is None:
        tx, ty, tune_mlups = ens.autotune(steps=3)
    else:
        (tx, ty), tune_mlups = tile, None
    ens.step(100)
    ens.sync()
    sites = ens.info()["sites"]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ens.step(steps)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    ens.sync()
    info = ens.info()
    ens.close()
    mlups = sites * steps / (ms * 1e-3) / 1e6
    hbm = (measured_peaks() or {}).get("hbm_gbs", 6800.0)
    gbs = FP32DEV_BYTES_PER_SITE * mlups * 1e6 / 1e9
    return {"members": n, "sites": sites, "steps": steps, "mlups": round(mlups, 1),
            "speedup_vs_fp64": round(mlups / fp64_mlups, 3), "hbm_gbs": round(gbs, 1),
            "hbm_frac": round(gbs / hbm, 4), "tile": [tx, ty], "work_items": info["items"],
            "autotune_best_mlups": None if tune_mlups is None else round(tune_mlups, 1),
            "graph_steps": 100, "precision": "fp32split",
            "launch": "one block per work item" if per_item
                      else "persistent grid (co-resident blocks claim the work items in order)"}


if __name__ == "__main__":
    sys.exit(main())
