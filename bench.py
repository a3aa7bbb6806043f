#!/usr/bin/env python
"""Benchmark of the APH DPD filter on GB300.

One step = one pass of the predistorter (basis, branch FIRs, accumulation with
the LO-leakage constant) over one batch of 2^24 complex64 samples of a
synthetic two-carrier OFDM signal, P = Q = 9, M = 4 (K = 51 coefficients).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  ``value`` is device-timed throughput (CUDA
events on the launching stream, inputs resident in HBM, two alternating buffer
sets so that no step reads data the previous step left in L2); ``e2e`` is the
same metric through the library's host-buffer path with the host<->device
copies inside the timed region.  With N > 1 (torchrun) every rank runs an
independent replica on its own batch: weak scaling, no collective on the data
path.  ``--impl reference`` times the FP64 CPU oracle on a bounded sample.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DPD Gsamples/s and % of roofline, plain vs batched; adjoint step ms; Gram TFLOP/s"
P, Q, M = 9, 9, 4
N_SAMPLES = 1 << 24
BYTES_PER_SAMPLE = 16            # 8 B complex64 read + 8 B written
FLOPS_ALG = lambda P, Q, M: 8 * (((P + 1) // 2) + ((Q + 1) // 2)) * (M + 1) + 3 * ((P + 1) // 2) + 2
FLOPS_WL = lambda P, Q, M: 8 * max((P + 1) // 2, (Q + 1) // 2) * (M + 1) + 3
SM_COUNT_NOMINAL, FP32_LANES_PER_SM = 152, 128
FALLBACK_HBM_GBS = 6800.0
WORKLOAD = ("APH DPD filter (Eq. 1), 2^24-sample two-carrier OFDM (1024-pt IFFT, 600 QPSK "
            "subcarriers, 72-sample CP, +-0.3 Nyquist, RMS 0.25), P=Q=9, M=4, K=51, complex64")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-patterns", action="store_true",
                    help="skip the batched / adjoint / Gram side measurements")
    ap.add_argument("--fwd-launch", default=None, metavar="MODE,V,WARPS,STAGES[,GROUP]",
                    help="fix the forward launch shape instead of tuning it (profiling runs)")
    ap.add_argument("--pattern", choices=["small", "batched", "adjoint", "grad", "gram", "gram_one", "ila", "cpu", "sweep",
                                          "fma", "estimate", "estimate_batched",
                                          "oracle"],
                    default=None,
                    help="run only this side measurement (1 GPU) and print its JSON; for profiling")
    ap.add_argument("--grad-log2n", type=int, default=24, help="samples (log2) of --pattern grad")
    ap.add_argument("--gram-precision", default="bf16x3", choices=["fp32", "tf32x3", "bf16x3"],
                    help="precision of --pattern gram_one")
    ap.add_argument("--batched-launch", default=None, metavar="V,WARPS,STAGES,CTAS_PER_SM[,GROUP]",
                    help="fix the batched launch shape of --pattern batched instead of tuning it (profiling runs)")
    ap.add_argument("--min-warmup-s", type=float, default=1.5,
                    help="keep warming up for at least this long so clocks settle and get sampled")
    return ap.parse_args()


# ----------------------------------------------------------------------------- helpers
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": FALLBACK_HBM_GBS}, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for fn in ("dpd_fwd.cuh", "dpd_device.cuh", "dpd_internal.h"):
        with open(os.path.join(ROOT, "paper_1612_09001_gb300", "csrc", fn), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel source; else None."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as f:
            d = json.load(f).get(kernel)
    except (OSError, ValueError):
        return None
    if not d or d.get("source_hash") != kernel_source_hash():
        return None
    return d


class ClockSampler:
    """nvidia-smi sampling (200 ms) of SM clock and throttle reasons."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,utilization.gpu,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [s.strip() for s in line.split(",")]
                if len(parts) < 10:
                    continue
                try:
                    rows.append(dict(sm=float(parts[1]), smax=float(parts[2]), util=float(parts[4]),
                                     hw=parts[6], hwt=parts[7], swt=parts[8], pcap=parts[9]))
                except ValueError:
                    continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        load = [r for r in rows if r["util"] > 0] or rows
        reasons = set()
        for r in load:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                              ("swt", "sw_thermal_slowdown"), ("pcap", "sw_power_cap")):
                if r[key].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in load), "sm_max_mhz": max(r["smax"] for r in rows),
                "reasons": sorted(reasons), "samples": len(load)}


class Ranks:
    """The replicas' coordination: barrier, max over ranks, rank 0 prints.

    With one process it does nothing.  Under torchrun every rank runs an
    independent replica (no collective on the data path); only the timing uses
    the process group: a barrier on both sides of the timed region and the
    maximum of the per-rank durations.  backend "nccl" reduces a tensor on the
    rank's GPU, "gloo" one in host memory (the CPU tests)."""

    def __init__(self, world: int, rank: int, backend: str = "nccl", device=None):
        self.world, self.rank, self.device = world, rank, device
        self.pg = None
        if world > 1:
            import torch.distributed as dist
            if backend == "nccl":
                dist.init_process_group("nccl", device_id=device)
            else:
                dist.init_process_group(backend)
            self.pg = dist

    @property
    def root(self) -> bool:
        return self.rank == 0

    def barrier(self):
        if self.pg is not None:
            self.pg.barrier()

    def max_over_ranks(self, v: float) -> float:
        if self.pg is None:
            return v
        import torch
        t = torch.tensor([v], dtype=torch.float64, device=self.device)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg is not None:
            self.pg.destroy_process_group()
            self.pg = None


def whole_job_rate(world: int, steps: int, units_per_step: int, seconds_max: float) -> float:
    """Units per second of the whole job: every rank processed steps x units in
    at most seconds_max (weak scaling), in 1e9 units/s."""
    return world * steps * units_per_step / seconds_max / 1e9


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ----------------------------------------------------------------------------- reference arm
def cpu_oracle_throughput(n_sample: int, min_seconds: float, nthreads: int = 0):
    """Time the FP64 oracle (as it stands) on the first n_sample samples of the workload."""
    import oracle
    import dpd_synth as synth
    x = synth.ofdm2(n_sample, key=(0, 0))
    h = synth.coeffs(P, Q, M, key=(0, 1))
    oracle.apply(x[:4096], h, P, Q, M, nthreads=nthreads)    # load + warm
    reps, t0 = 0, time.perf_counter()
    while True:
        oracle.apply(x, h, P, Q, M, nthreads=nthreads)
        reps += 1
        el = time.perf_counter() - t0
        if el >= min_seconds:
            break
    return reps * n_sample / el / 1e9, el, reps, oracle.threads(nthreads)


def cpu_oracle_configs(nthreads_multi: int):
    """The FP64 oracle, as it stands, on bounded samples of every workload:
    median of 5 timed runs, with all host cores and with one thread."""
    import numpy as np
    import oracle
    import dpd_synth as synth

    def med(fn, nt):
        fn(nt)
        ts = []
        for _ in range(5):
            t0 = time.perf_counter()
            fn(nt)
            ts.append(time.perf_counter() - t0)
        return statistics.median(ts)

    out = {"kind": "oracle", "threads_multi": oracle.threads(nthreads_multi), "cpu": _cpu_model(),
           "note": "median of 5 runs; value = units / median seconds"}
    x0 = synth.clipped_gaussian(1 << 16, 0.3, key=(0, 0))
    h0 = synth.coeffs(5, 5, 2, key=(0, 1))
    x1 = synth.ofdm2(1 << 20, key=(0, 0))
    h1 = synth.coeffs(P, Q, M, key=(0, 1))
    specs = synth.batch_streams(64, seed=0)
    cut = 1 << 14
    h3 = synth.coeffs(7, 7, 3, key=(0, 1))
    x3 = x1[: 1 << 18]
    g3 = synth.ofdm2(1 << 18, key=(0, 2))
    u4, th4 = synth.ls_problem(1 << 15)
    t4 = oracle.apply(u4, th4, 11, 11, 7, nthreads=nthreads_multi)
    cases = [
        ("cfg0_2p16_P5M2", "full 2^16 samples", 1 << 16, "Gsamples/s",
         lambda nt: oracle.apply(x0, h0, 5, 5, 2, nthreads=nt)),
        ("cfg1_2p24_P9M4", "first 2^20 of the 2^24 samples", 1 << 20, "Gsamples/s",
         lambda nt: oracle.apply(x1, h1, P, Q, M, nthreads=nt)),
        ("cfg2_batched_64", f"first {cut} samples of each of the 64 streams", sum(min(cut, len(sp['x'])) for sp in specs),
         "Gsamples/s",
         lambda nt: [oracle.apply(sp["x"][:cut], sp["h"], sp["P"], sp["Q"], sp["M"], nthreads=nt) for sp in specs]),
        ("cfg3_fwd_grad_P7M3", "forward + coefficient and input gradient, first 2^18 samples", 1 << 18,
         "Gsamples/s",
         lambda nt: (oracle.apply(x3, h3, 7, 7, 3, nthreads=nt), oracle.grad(x3, h3, g3, 7, 7, 3, nthreads=nt))),
        ("cfg4_ls_P11M7", "Gram + FP64 Cholesky solve, 2^15 of the 2^22 rows, K=97", 1 << 15, "Grows/s",
         lambda nt: oracle.ls(u4, t4, 11, 11, 7, nthreads=nt)),
    ]
    res = {}
    for name, sample, units, unit, fn in cases:
        tm = med(fn, nthreads_multi)
        t1 = med(fn, 1)
        res[name] = {"sample": sample, "unit": unit, "multi": units / tm / 1e9, "single_thread": units / t1 / 1e9,
                     "seconds_multi": tm, "seconds_single": t1}
    out["configs"] = res
    return out


def _cpu_model():
    arm_parts = {"0xd4f": "Arm Neoverse V2", "0xd40": "Arm Neoverse V1", "0xd0c": "Arm Neoverse N1"}
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                key, _, val = line.partition(":")
                key, val = key.strip().lower(), val.strip()
                if key == "model name":
                    return val
                if key == "cpu part":
                    return f"{arm_parts.get(val, 'Arm')} (CPU part {val})"
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    import oracle
    import dpd_synth as synth
    n_sample = 1 << 20
    nth = os.cpu_count() or 1   # every host core, as the main line's cpu_baseline
    x = synth.ofdm2(n_sample, key=(0, 0))
    h = synth.coeffs(P, Q, M, key=(0, 1))
    for _ in range(max(args.warmup, 0)):
        oracle.apply(x, h, P, Q, M, nthreads=nth)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.apply(x, h, P, Q, M, nthreads=nth)
    el = time.perf_counter() - t0
    v = args.steps * n_sample / el / 1e9
    cores = oracle.threads(nth)
    sample = f"first 2^20 samples of the workload per step, FP64 C oracle, {cores} threads"
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "Gsamples/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "P": P, "Q": Q, "M": M,
                                        "n_samples_per_step": n_sample},
        "cpu_baseline": {"value": v, "unit": "Gsamples/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "Gsamples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- our arm
def _time_graph(fn, reps, dev):
    """Capture fn() in a CUDA graph, replay it reps times, return seconds per replay."""
    import torch
    s = torch.cuda.Stream(dev)
    s.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(s):
        fn()
    torch.cuda.synchronize(dev)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        fn()
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    cur = torch.cuda.current_stream(dev)
    e0.record(cur)
    for _ in range(reps):
        g.replay()
    e1.record(cur)
    torch.cuda.synchronize(dev)
    return e0.elapsed_time(e1) * 1e-3 / reps


def measure_fma_ceiling(dev, reps=5, gpu_index=0):
    """The FP32 FMA pipe's ceiling on this GPU: dpd_probe_fma (independent FMA
    chains only, scalar and packed f32x2), 4 CTAs of 256 threads per SM, about
    10 ms per launch, CUDA events, median of `reps` launches after two warm-up
    launches, with the SM clock sampled during the launches."""
    import ctypes
    import torch
    from paper_1612_09001_gb300 import _lib
    lib = _lib.load()
    props = torch.cuda.get_device_properties(dev)
    blocks, iters = props.multi_processor_count * 4, 1 << 17
    sink = torch.empty(blocks * 256, dtype=torch.float32, device=dev)
    sp = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    fmas = blocks * 256 * iters * 16
    out = {"kernel": "dpd_probe_fma", "blocks": blocks, "threads": 256, "fmas_per_launch": fmas,
           "timing": f"CUDA events, median of {reps} launches after 2 warm-up launches"}
    sampler = ClockSampler(gpu_index)
    sampler.start()
    time.sleep(0.3)
    for packed in (1, 0):
        def launch():
            _lib.check("dpd_probe_fma", lib.dpd_probe_fma(blocks, iters, packed, ctypes.c_void_p(sink.data_ptr()), sp))
        for _ in range(2):
            launch()
        torch.cuda.synchronize(dev)
        ts = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            launch()
            e1.record()
            torch.cuda.synchronize(dev)
            ts.append(e0.elapsed_time(e1) * 1e-3)
        sec = statistics.median(ts)
        out["packed" if packed else "scalar"] = {"ms": sec * 1e3, "fma_per_s": fmas / sec}
    clk = sampler.stop()
    out["clocks"] = clk
    best = max(out["packed"]["fma_per_s"], out["scalar"]["fma_per_s"])
    out["fma_per_s"] = best
    out["tflops"] = 2.0 * best / 1e12
    if clk and clk.get("sm_mhz"):
        out["fma_per_clock_per_sm"] = best / (clk["sm_mhz"] * 1e6) / props.multi_processor_count
    return out


def measure_sweep(dev, log2_min=10, log2_max=26):
    """Throughput against length (the paper's throughput-vs-samples experiment):
    graph-replayed dpd_apply at N = 2^10 .. 2^26, at the 2^16 workload's model
    (clipped Gaussian, P=Q=5, M=2) and at the 2^24 workload's (OFDM, P=Q=9, M=4).
    Up to 2^22 samples the data stay in L2 between replays."""
    import torch
    import dpd_synth as synth
    import paper_1612_09001_gb300 as dpd
    nmax = 1 << log2_max
    out = {"unit": "Gsamples/s", "timing": "CUDA graph of 20 calls, replayed; events on the replay stream"}
    for name, (Pm, Qm, Mm), gen in (("P5M2_clipped_gaussian", (5, 5, 2), lambda n: synth.clipped_gaussian(n, 0.3, key=(0, 0))),
                                     ("P9M4_ofdm", (9, 9, 4), lambda n: synth.ofdm2(n, key=(0, 0)))):
        xa = torch.from_numpy(gen(nmax)).to(dev)
        ya = torch.empty_like(xa)
        f = dpd.DPD(Pm, Qm, Mm)
        f.set_coeffs(synth.coeffs(Pm, Qm, Mm, key=(0, 1)))
        rows = []
        for lg in range(log2_min, log2_max + 1):
            n = 1 << lg
            x, y = xa[:n], ya[:n]
            calls = 20
            reps = max(3, min(200, (1 << 27) // (n * calls)))

            def body():
                for _ in range(calls):
                    f.apply(x, out=y)

            t = _time_graph(body, reps, dev) / calls
            rows.append({"log2_n": lg, "us_per_call": t * 1e6, "gsamples_per_s": n / t / 1e9})
        f.sync_status()
        f.close()
        out[name] = rows
        del xa, ya
    return out


def measure_grad(dev, log2_n=24, reps=20):
    """dpd_grad alone (the adjoint kernels): input gradient, coefficient
    gradient and both, on 2^log2_n OFDM samples with an OFDM-like output
    gradient, at the 2^24 workload's model and at the direct-learning model."""
    import torch
    import dpd_synth as synth
    import paper_1612_09001_gb300 as dpd
    n = 1 << log2_n
    x = torch.from_numpy(synth.ofdm2(n, key=(0, 0))).to(dev)
    gy = torch.from_numpy(synth.ofdm2(n, key=(0, 1))).to(dev)
    gx = torch.empty_like(x)
    out = {"n": n, "unit": "us per call", "timing": f"{reps} back-to-back calls after 3 warm-up calls, CUDA events"}
    for (Pm, Qm, Mm) in ((9, 9, 4), (7, 7, 3)):
        f = dpd.DPD(Pm, Qm, Mm)
        f.set_coeffs(synth.coeffs(Pm, Qm, Mm, key=(0, 1)))
        gh = torch.empty(f.K, dtype=torch.complex64, device=dev)
        row = {}
        for name, kw in (("gx", dict(gx=gx)), ("gh", dict(gh=gh)), ("gx_and_gh", dict(gx=gx, gh=gh))):
            for _ in range(3):
                f.grad(x, gy, **kw)
            torch.cuda.synchronize(dev)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                f.grad(x, gy, **kw)
            e1.record()
            torch.cuda.synchronize(dev)
            us = e0.elapsed_time(e1) * 1e3 / reps
            row[name] = {"us": us, "gsamples_per_s": n / us / 1e3}
        # Coefficients set from device memory: the derived tables are copied
        # back to host memory behind the set, and once that copy has landed the
        # input gradient takes them by value as well.
        f.set_coeffs(torch.from_numpy(synth.coeffs(Pm, Qm, Mm, key=(0, 1)).astype("complex64")).to(dev))
        torch.cuda.synchronize(dev)
        for _ in range(3):
            f.grad(x, gy, gx=gx)
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            f.grad(x, gy, gx=gx)
        e1.record()
        torch.cuda.synchronize(dev)
        us = e0.elapsed_time(e1) * 1e3 / reps
        row["gx_device_set_coeffs"] = {"us": us, "gsamples_per_s": n / us / 1e3}
        f.sync_status()
        f.close()
        # The allocation-free entry point (no handle: plain-load kernel) on the
        # same inputs, for comparison with the handle's staged kernel.
        import ctypes
        from paper_1612_09001_gb300 import _lib
        lib = _lib.load()
        sp = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)

        def noalloc():
            _lib.check("dpd_grad_coeffs_noalloc", lib.dpd_grad_coeffs_noalloc(
                Pm, Qm, Mm, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(gy.data_ptr()), n,
                ctypes.c_void_p(gh.data_ptr()), sp))
        for _ in range(3):
            noalloc()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            noalloc()
        e1.record()
        torch.cuda.synchronize(dev)
        us = e0.elapsed_time(e1) * 1e3 / reps
        row["gh_noalloc"] = {"us": us, "gsamples_per_s": n / us / 1e3,
                             "kernel": "plain-load adj_gh_kernel (dpd_grad_coeffs_noalloc)"}
        out[f"P{Pm}Q{Qm}M{Mm}"] = row
    return out


def measure_small(dev, calls=200):
    """2^16 clipped-Gaussian samples, P=Q=5, M=2 (L2-resident, launch-bound):
    microseconds per dpd_apply, back to back and replayed from a CUDA graph."""
    import torch
    import dpd_synth as synth
    import paper_1612_09001_gb300 as dpd
    n = 1 << 16
    x = torch.from_numpy(synth.clipped_gaussian(n, 0.3, key=(0, 0))).to(dev)
    y = torch.empty_like(x)
    f = dpd.DPD(5, 5, 2)
    f.set_coeffs(synth.coeffs(5, 5, 2, key=(0, 1)))
    s = torch.cuda.Stream(dev)
    with torch.cuda.stream(s):
        for _ in range(10):
            f.apply(x, out=y, stream=s)
    s.synchronize()

    def timed(fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        fn()
        e1.record(s)
        e1.synchronize()
        return e0.elapsed_time(e1) * 1e3

    def plain():
        for _ in range(calls):
            f.apply(x, out=y, stream=s)

    t_plain = timed(plain) / calls
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        for _ in range(calls):
            f.apply(x, out=y, stream=s)
    def replay():
        with torch.cuda.stream(s):   # a graph replays on the current stream
            g.replay()

    replay()
    s.synchronize()
    t_graph = timed(replay) / calls
    f.sync_status(s)
    return {"workload": "2^16 clipped Gaussian (RMS 0.3), P=Q=5, M=2 (K=19), L2-resident",
            "us_per_call_plain": t_plain, "us_per_call_graph": t_graph,
            "gsamples_per_s_graph": n / (t_graph * 1e-6) / 1e9, "calls": calls}


def measure_ila(dev, n=1 << 20):
    """Indirect learning (Sec. 2.2) around the Eq. 3 WARP PA on LTE-like signals
    (one 10 MHz carrier; two 3 MHz carriers 10 MHz apart; 4x oversampled, RMS 0.2):
    time per ILA iteration and out-of-band suppression (the paper's Fig. 8 test)."""
    import torch
    import dpd_synth as synth
    import paper_1612_09001_gb300 as dpd
    from paper_1612_09001_gb300 import direct, spectrum
    P, Q, M = 7, 3, 1
    tx, G = direct.warp_pa_transmitter(device=dev)
    out = {"model": f"DPD P={P} Q={Q} M={M}; PA of Eq. 3; 3 ILA iterations, TF32x3, orthogonal basis",
           "signals": {}}
    for name, gen in (("10MHz_single", synth.lte_single), ("2x3MHz_noncontiguous", synth.lte_two)):
        x, band = gen(n, key=(8, 0), rms=0.2)
        xd = torch.from_numpy(x).to(dev)
        direct.ila_train(xd, tx, P, Q, M, gain=G, iterations=1, precision="tf32x3", basis="orthogonal")
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        h, hist = direct.ila_train(xd, tx, P, Q, M, gain=G, iterations=3, precision="tf32x3", basis="orthogonal")
        torch.cuda.synchronize(dev)
        t_ila = (time.perf_counter() - t0) / 3
        f = dpd.DPD(P, Q, M)
        f.set_coeffs(h)
        y_plain = (tx.apply(xd) / G).cpu().numpy()
        y_dpd = (tx.apply(f.apply(xd)) / G).cpu().numpy()
        f.close()
        rep = spectrum.suppression_report(x, y_plain, y_dpd, band)
        out["signals"][name] = {"samples": n, "ms_per_ila_iteration": t_ila * 1e3,
                                "nmse_db_per_iteration": [r["nmse_db_before"] for r in hist],
                                "oob_total_dbc": {k: rep[k]["oob_total_dbc"] for k in ("input", "no_dpd", "dpd")},
                                "oob_peak_dbc": {k: rep[k]["oob_peak_dbc"] for k in ("input", "no_dpd", "dpd")},
                                "suppression_total_db": rep["suppression_total_db"],
                                "suppression_peak_db": rep["suppression_peak_db"]}
    return out


def measure_cpu_simd(n=1 << 24):
    """The portable SIMD + OpenMP CPU filter on the host cores (a like-for-like
    CPU comparison, not the oracle): the benchmark workload and the paper's
    Table 2 model (P=5, Q=3, L=5) on 1, 4 and all threads."""
    import numpy as np
    import dpd_synth as synth
    from paper_1612_09001_gb300 import build, cpu
    build.build_cpu()
    x = synth.ofdm2(n, key=(0, 0))
    y = np.empty_like(x)
    out = {"host_threads": cpu.max_threads(), "samples": n, "dtype": "f32", "results": {}}
    for name, (P, Q, M) in (("P9_Q9_M4", (9, 9, 4)), ("table2_P5_Q3_L5", (5, 3, 4))):
        h = synth.coeffs(P, Q, M, key=(0, 1))
        r = {}
        for th in sorted({1, 4, cpu.max_threads()}):
            cpu.apply(x[: 1 << 16], h, P, Q, M, threads=th, out=y[: 1 << 16])
            reps, t0 = 0, time.perf_counter()
            while True:
                cpu.apply(x, h, P, Q, M, threads=th, out=y)
                reps += 1
                el = time.perf_counter() - t0
                if el > 1.0 or reps >= 20:
                    break
            r[f"{th}_threads_gsamples_per_s"] = reps * n / el / 1e9
        out["results"][name] = r
    return out


def measure_batched(dev, reps=20, launch=None):
    """64 antenna streams, lengths U[2^12, 2^20], P in {5,7,9}, M in {2..6}:
    one persistent launch (CUDA graph) against 64 plain launches."""
    import torch
    import dpd_synth as synth
    import paper_1612_09001_gb300 as dpd
    specs = synth.batch_streams(64, seed=0)
    streams, handles = [], []
    for sp in specs:
        x = torch.from_numpy(sp["x"]).to(dev)
        streams.append(dict(x=x, y=torch.empty_like(x), P=sp["P"], Q=sp["Q"], M=sp["M"], h=sp["h"]))
        f = dpd.DPD(sp["P"], sp["Q"], sp["M"])
        f.set_coeffs(sp["h"])
        handles.append(f)
    total = sum(len(sp["x"]) for sp in specs)
    plan = dpd.BatchedPlan(streams)
    from paper_1612_09001_gb300 import tune
    if launch:                                 # fixed shape (profiling runs)
        best = tuple(launch)
        plan.set_launch(*best)
    else:                                      # tile / stage / grid picked by timing, before the timed region
        best, _ = tune.tune_batched(plan)
    l0 = dpd.kernel_launches()
    t_plan = _time_graph(lambda: plan.execute(), reps, dev)
    launches_plan = (dpd.kernel_launches() - l0) // 2   # captured twice (warm-up + capture)

    def plain():
        for f, st in zip(handles, streams):
            f.apply(st["x"], out=st["y"])

    t_graph64 = _time_graph(plain, reps, dev)
    for _ in range(3):
        plain()
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        plain()
    e1.record()
    torch.cuda.synchronize(dev)
    t_plain = e0.elapsed_time(e1) * 1e-3 / reps
    plan.sync_status()
    for f in handles:
        f.sync_status()
        f.close()
    plan.close()
    return {"workload": "64 streams, n ~ U[2^12, 2^20], P=Q in {5,7,9}, M in {2..6}, clipped Gaussian RMS 0.3",
            "total_samples": total, "unit": "Gsamples/s",
            "persistent_graph": total / t_plan / 1e9, "persistent_launches_per_step": launches_plan,
            "persistent_launch_shape": {"V": best[0], "warps": best[1], "stages": best[2], "ctas_per_sm": best[3],
                                        "group": best[4] if len(best) > 4 else 0},
            "plain_64_launches": total / t_plain / 1e9, "plain_64_in_one_graph": total / t_graph64 / 1e9,
            "persistent_us": t_plan * 1e6, "plain_64_us": t_plain * 1e6, "plain_64_graph_us": t_graph64 * 1e6,
            "hbm_gbs_persistent": 16 * total / t_plan / 1e9}


def measure_direct(dev, steps=400, lr=5e-3):
    """Direct learning, 2^20 OFDM samples, DPD P=Q=7, M=3 through the synthetic
    I/Q + PA transmitter: one graph-replayed Adam step, and the NMSE reached
    against indirect learning (3 LS iterations)."""
    import torch
    import dpd_synth as synth
    from paper_1612_09001_gb300.direct import DirectLearner, Transmitter, indirect_learning, nmse_db
    import paper_1612_09001_gb300 as dpd
    t = synth.synthetic_pa(seed=1)
    tx = Transmitter([t["iq"], t["pa"]], device=dev)
    x = torch.from_numpy(synth.ofdm2(1 << 20, key=(0, 0))).to(dev)
    base = nmse_db(tx.apply(x), x)
    learner = DirectLearner(x, tx, 7, 7, 3, lr=lr).capture()
    l0 = dpd.kernel_launches()
    learner.step()
    torch.cuda.synchronize(dev)
    ms = learner.time_step(50)
    learner.train(steps)
    with torch.no_grad():
        direct = nmse_db(tx.apply(learner.filt.apply(x)), x)
    h_ila = indirect_learning(x, tx, 7, 7, 3, iterations=3)
    f = dpd.DPD(7, 7, 3)
    f.set_coeffs(h_ila)
    ila = nmse_db(tx.apply(f.apply(x)), x)
    return {"workload": "2^20 OFDM samples, DPD P=Q=7 M=3 (K=33), transmitter: I/Q (g=1.02, 2 deg, LO 0.005) + PA P=7 M=3",
            "adjoint_step_ms": ms, "step": "graph replay: DPD -> I/Q -> PA -> loss -> adjoint PA, I/Q, DPD -> Adam",
            "nmse_db_no_dpd": base, "nmse_db_direct": direct, "direct_steps": steps + 54,
            "direct_optimizer": f"Adam, learning rate {lr:g} (constant), graph-replayed steps",
            "nmse_db_ila_3_iterations": ila, "direct_minus_ila_db": direct - ila}


def measure_estimate(dev, reps=5, refine_iters=3):
    """One least-squares estimate of 2^22 rows x K = 97 (P = Q = 11, M = 7,
    BF16x3 and TF32x3, monomial basis, statistics on): wall time per call
    (median of `reps` after two warm-up calls), the device time of the same
    call (CUDA events around it), the library kernel launches it makes, and
    the host time in between (wall minus device)."""
    import numpy as np
    import torch
    import dpd_synth as synth
    import paper_1612_09001_gb300 as dpd
    P, Q, M, n = 11, 11, 7, 1 << 22
    u, theta = synth.ls_problem(n, P, Q, M, seed=0)
    ud = torch.from_numpy(u).to(dev)
    g = dpd.DPD(P, Q, M)
    g.set_coeffs(theta)
    td = g.apply(ud)
    f = dpd.DPD(P, Q, M)
    out = {"workload": "LS estimate, Psi 2^22 rows x 97 complex columns (P=Q=11, M=7), t = Psi theta",
           "refine_iters": refine_iters, "timing": f"median of {reps} calls after 2 warm-up calls"}
    for prec in ("bf16x3", "tf32x3"):
        for _ in range(2):
            f.estimate(ud, td, precision=prec, refine_iters=refine_iters)
        torch.cuda.synchronize(dev)
        walls, devs = [], []
        launches = 0
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            l0 = dpd.kernel_launches()
            t0 = time.perf_counter()
            e0.record()
            h, st = f.estimate(ud, td, precision=prec, refine_iters=refine_iters)
            e1.record()
            torch.cuda.synchronize(dev)
            walls.append(time.perf_counter() - t0)
            devs.append(e0.elapsed_time(e1) * 1e-3)
            launches = dpd.kernel_launches() - l0
        err = float(np.linalg.norm(h.cpu().numpy() - theta) / np.linalg.norm(theta))
        out[prec] = {"wall_ms": statistics.median(walls) * 1e3, "events_ms": statistics.median(devs) * 1e3,
                     "library_launches": launches, "coef_rel_error_vs_true": err, "cond_est_DGD": st["cond_est"]}
    f.close()
    g.close()
    return out


def measure_estimate_batched(dev, reps=5, refine_iters=2):
    """One batched least-squares estimate of 256 problems of 2^16 rows x K = 97
    (P = Q = 11, M = 7, BF16x3 and TF32x3, monomial basis, 2 refinements, the
    per-problem info codes copied to the host): device time (CUDA events
    around the call, median of `reps` after two warm-up calls), wall time and
    the library kernel launches the call makes."""
    import numpy as np
    import torch
    import dpd_synth as synth
    import paper_1612_09001_gb300 as dpd
    P, Q, M, nb, nr = 11, 11, 7, 256, 1 << 16
    g = dpd.DPD(P, Q, M)
    us, ts, thetas = [], [], []
    for b in range(nb):
        ub, thb = synth.ls_problem(nr, P, Q, M, seed=b)
        ubd = torch.from_numpy(ub).to(dev)
        g.set_coeffs(thb)
        us.append(ubd)
        ts.append(g.apply(ubd))
        thetas.append(thb)
    us, ts = torch.stack(us), torch.stack(ts)   # equal lengths: one (problems x rows) tensor each
    f = dpd.DPD(P, Q, M)
    out = {"workload": f"{nb} LS estimates of {nr} rows x 97 complex columns (P=Q=11, M=7), t = Psi theta, "
                       f"monomial basis",
           "refine_iters": refine_iters, "timing": f"median of {reps} calls after 2 warm-up calls"}
    for prec in ("bf16x3", "tf32x3"):
        for _ in range(2):
            f.estimate_batched(us, ts, precision=prec, refine_iters=refine_iters)
        torch.cuda.synchronize(dev)
        walls, devs = [], []
        launches = 0
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            l0 = dpd.kernel_launches()
            t0 = time.perf_counter()
            e0.record()
            hb, info = f.estimate_batched(us, ts, precision=prec, refine_iters=refine_iters)
            e1.record()
            torch.cuda.synchronize(dev)
            walls.append(time.perf_counter() - t0)
            devs.append(e0.elapsed_time(e1) * 1e-3)
            launches = dpd.kernel_launches() - l0
        hb = hb.cpu().numpy()
        errs = [float(np.linalg.norm(hb[i] - thetas[i]) / np.linalg.norm(thetas[i])) for i in range(nb)]
        out[prec] = {"wall_ms": statistics.median(walls) * 1e3, "events_ms": statistics.median(devs) * 1e3,
                     "library_launches": launches, "coef_rel_error_median": float(np.median(errs)),
                     "not_spd": int(sum(1 for i in info if i))}
    f.close()
    g.close()
    return out


def measure_gram_one(dev, precision, reps=10):
    """The Gram contraction alone (dpd_gram: tensor or FP32 kernel, FP64
    reduction and assembly) of 2^22 rows x K = 97 (P = Q = 11, M = 7) in one
    precision: two warm-up calls, then `reps` back-to-back calls between CUDA
    events."""
    import torch
    import dpd_synth as synth
    import paper_1612_09001_gb300 as dpd
    P, Q, M, n = 11, 11, 7, 1 << 22
    u, theta = synth.ls_problem(n, P, Q, M, seed=0)
    ud = torch.from_numpy(u).to(dev)
    g = dpd.DPD(P, Q, M)
    g.set_coeffs(theta)
    td = g.apply(ud)
    f = dpd.DPD(P, Q, M)
    for _ in range(2):
        f.gram(ud, td, precision=precision, want_tt=False)
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        f.gram(ud, td, precision=precision, want_tt=False)
    e1.record()
    torch.cuda.synchronize(dev)
    f.sync_status()
    ms = e0.elapsed_time(e1) / reps
    f.close()
    g.close()
    return {"workload": "Psi 2^22 rows x 97 complex columns (P=Q=11, M=7)", "precision": precision,
            "gram_ms": ms, "timing": f"{reps} back-to-back dpd_gram calls after 2 warm-up calls, CUDA events"}


def measure_gram(dev, reps=5):
    """LS Gram of 2^22 rows x K=97 (P=Q=11, M=7) in every precision, and the
    batch of 256 estimations of 2^16 rows."""
    import numpy as np
    import torch
    import dpd_synth as synth
    import paper_1612_09001_gb300 as dpd
    P, Q, M, n = 11, 11, 7, 1 << 22
    u, theta = synth.ls_problem(n, P, Q, M, seed=0)
    f = dpd.DPD(P, Q, M)
    K = f.K
    ud = torch.from_numpy(u).to(dev)
    g = dpd.DPD(P, Q, M)
    g.set_coeffs(theta)
    td = g.apply(ud)
    useful = 8.0 * n * K * K
    out = {"workload": "Psi 2^22 rows x 97 complex columns (P=Q=11, M=7), clipped Gaussian RMS 0.3, t = Psi theta",
           "flops_convention": "useful = 8 n K^2 (the complex Gram by its definition); the tensor path computes the "
                               "lagged correlations of the 15 basis / target signals instead, executing three "
                               "128 x 224 x 16 MMAs per 128 samples = 21504 flops per sample (fewer than the "
                               "definition's, so 'useful' can exceed the tensor peak); rates over the whole dpd_gram "
                               "call (Gram kernel + FP64 reduction + assembly)",
           "single": {}, "batch": {}}
    for prec in ("fp32", "tf32x3", "bf16x3"):
        f.gram(ud, td, precision=prec, want_tt=False)
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            f.gram(ud, td, precision=prec, want_tt=False)   # Gram + FP64 reduction + assembly, no host sync
        e1.record()
        torch.cuda.synchronize(dev)
        t_gram = e0.elapsed_time(e1) * 1e-3 / reps
        est = {}
        for basis in ("monomial", "orthogonal"):
            f.estimate(ud, td, precision=prec, refine_iters=3, basis=basis)
            walls = []
            for _ in range(reps):
                torch.cuda.synchronize(dev)
                t0 = time.perf_counter()
                h, st = f.estimate(ud, td, precision=prec, refine_iters=3, basis=basis)
                walls.append(time.perf_counter() - t0)
            t_est = statistics.median(walls)
            h0, _ = f.estimate(ud, td, precision=prec, refine_iters=0, basis=basis)
            est[basis] = {"estimate_ms_3_refinements": t_est * 1e3,
                          "coef_rel_error_vs_true": float(np.linalg.norm(h.cpu().numpy() - theta) / np.linalg.norm(theta)),
                          "coef_rel_error_no_refinement": float(np.linalg.norm(h0.cpu().numpy() - theta)
                                                                / np.linalg.norm(theta)),
                          "cond_est_DGD": st["cond_est"], "rel_residual": st["rel_residual"]}
        f.set_estimate_basis("monomial")
        executed = None
        if prec != "fp32":   # three 128 x 224 x 16 MMAs per 128 samples
            executed = 21504.0 * n
        out["single"][prec] = {"gram_ms": t_gram * 1e3, "gram_tflops_useful": useful / t_gram / 1e12,
                               "tensor_tflops_executed": (executed / t_gram / 1e12) if executed else None,
                               "estimate": est}
    # batch: 256 antennas x 2^16 rows
    nb, nr = 256, 1 << 16
    us, ts, thetas = [], [], []
    for b in range(nb):
        ub, thb = synth.ls_problem(nr, P, Q, M, seed=b)
        ubd = torch.from_numpy(ub).to(dev)
        g.set_coeffs(thb)
        us.append(ubd)
        ts.append(g.apply(ubd))
        thetas.append(thb)
    us, ts = torch.stack(us), torch.stack(ts)   # equal lengths: one (problems x rows) tensor each
    useful_b = 8.0 * nb * nr * K * K
    batch_refine = 2
    out["batch_timing"] = (f"one estimate_batched call over all {nb} problems ((basis,) Gram, FP64 Cholesky, solve, "
                           f"{batch_refine} refinements, info copied to the host): median of {reps} calls after 2 "
                           f"warm-up calls; CUDA events around the call and wall time")
    for prec in ("tf32x3", "bf16x3"):
        out["batch"][prec] = {}
        for basis in ("monomial", "orthogonal"):
            f.set_estimate_basis(basis)
            for _ in range(2):
                f.estimate_batched(us, ts, precision=prec, refine_iters=batch_refine)
            torch.cuda.synchronize(dev)
            walls, devs = [], []
            for _ in range(reps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                t0 = time.perf_counter()
                e0.record()
                f.estimate_batched(us, ts, precision=prec, refine_iters=batch_refine)
                e1.record()
                torch.cuda.synchronize(dev)
                walls.append(time.perf_counter() - t0)
                devs.append(e0.elapsed_time(e1) * 1e-3)
            t_b = statistics.median(devs)
            r = {"problems": nb, "rows_each": nr, "refine_iters": batch_refine, "events_ms": t_b * 1e3,
                 "wall_ms": statistics.median(walls) * 1e3, "tflops_useful": useful_b / t_b / 1e12}
            for it in (0, 2):
                hb, info = f.estimate_batched(us, ts, precision=prec, refine_iters=it)
                hb = hb.cpu().numpy()
                errs = [float(np.linalg.norm(hb[i] - thetas[i]) / np.linalg.norm(thetas[i])) for i in range(nb)]
                r[f"coef_rel_error_median_{it}_refinements"] = float(np.median(errs))
                r[f"coef_rel_error_max_{it}_refinements"] = float(np.max(errs))
                r["not_spd"] = int(sum(1 for i in info if i))
            out["batch"][prec][basis] = r
        f.set_estimate_basis("monomial")
    peaks, kind = measured_peaks()
    bf = out["single"]["bf16x3"]
    bf["tensor_frac_of_bf16_peak"] = bf["tensor_tflops_executed"] / peaks.get("bf16_tflops", 1900.0)
    bf["peak_kind"] = f"of {kind} BF16 burst (dense cuBLAS)"
    tf = out["single"]["tf32x3"]   # TF32 peak: the BF16 one x the nominal dense ratio 1.1 / 2.25
    tf["tensor_frac_of_tf32_peak"] = tf["tensor_tflops_executed"] / (peaks.get("bf16_tflops", 1900.0) * 1.1 / 2.25)
    tf["peak_kind"] = f"of {kind} BF16 burst x 1.1 / 2.25 (nominal TF32 / BF16 dense ratio)"
    return out


def run_ours(args, world, rank, local):
    import numpy as np
    import torch
    import dpd_synth as synth
    import paper_1612_09001_gb300 as dpd

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ranks = Ranks(world, rank, "nccl", dev)
    barrier, max_over_ranks = ranks.barrier, ranks.max_over_ranks

    n = N_SAMPLES
    x_host = synth.ofdm2(n, key=(rank, 0))
    h = synth.coeffs(P, Q, M, key=(0, 1))
    f = dpd.DPD(P, Q, M)
    f.set_coeffs(h)   # estimated offline, installed from host memory (the paper's use)
    xs = [torch.from_numpy(x_host).to(dev) for _ in range(2)]
    ys = [torch.empty_like(xs[0]) for _ in range(2)]
    stream = torch.cuda.current_stream(dev)
    from paper_1612_09001_gb300 import tune
    if args.fwd_launch:
        vals = [int(v) for v in args.fwd_launch.split(",")]
        mode, V, warps, stages = vals[:4]
        f.set_fwd_launch(mode=mode, V=V, warps=warps, stages=stages, group=vals[4] if len(vals) > 4 else 0)
        picked_by = "--fwd-launch"
    else:
        tune.tune_forward(f, xs[0], ys[0])   # launch shape picked by timing, before the timed region
        picked_by = "autotuner (tune.tune_forward)"

    sampler = ClockSampler(local)
    sampler.start()
    # warm-up: at least W steps and at least min_warmup_s of the same work
    t0 = time.perf_counter()
    i = 0
    while i < args.warmup or time.perf_counter() - t0 < args.min_warmup_s:
        f.apply(xs[i % 2], out=ys[i % 2])
        i += 1
        if i % 64 == 0:
            torch.cuda.synchronize(dev)
    f.sync_status()

    K = args.steps
    e_start = torch.cuda.Event(enable_timing=True)
    e_end = torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize(dev)
    launches0 = dpd.kernel_launches()
    w0 = time.perf_counter()
    e_start.record(stream)
    for k in range(K):
        f.apply(xs[k % 2], out=ys[k % 2])
    e_end.record(stream)
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - w0
    barrier()
    launches = dpd.kernel_launches() - launches0
    clocks = sampler.stop()
    f.sync_status()
    total = e_start.elapsed_time(e_end) * 1e-3
    total_max = max_over_ranks(total)
    value = whole_job_rate(world, K, n, total_max)
    mean_launch = total / K   # one kernel launch per step

    # ---- end to end through the library's host path (dpd_apply_host): pinned
    # host input in, pinned host output back, copies inside the timed region
    xh = torch.from_numpy(x_host).pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    K2 = max(3, min(K, 20))

    def timed_host(step):
        for _ in range(2):
            step()
        torch.cuda.synchronize(dev)
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(K2):
            step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return max_over_ranks(e0.elapsed_time(e1) * 1e-3)

    l0 = dpd.kernel_launches()
    t_zc = timed_host(lambda: f.apply_host(xh, out=yh, zero_copy=True))
    e2e_launches = (dpd.kernel_launches() - l0) // (K2 + 2)
    t_pipe = timed_host(lambda: f.apply_host(xh, out=yh))
    xd, yd = xs[0], ys[0]

    def explicit():
        xd.copy_(xh, non_blocking=True)
        f.apply(xd, out=yd)
        yh.copy_(yd, non_blocking=True)

    t_cp = timed_host(explicit)

    # host-link ceiling: both copy directions at once on two streams (copy engines)
    s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)

    def link_copies():
        s_in.wait_stream(stream)
        s_out.wait_stream(stream)
        with torch.cuda.stream(s_in):
            xd.copy_(xh, non_blocking=True)
        with torch.cuda.stream(s_out):
            yh.copy_(ys[1], non_blocking=True)
        stream.wait_stream(s_in)
        stream.wait_stream(s_out)

    t_link = timed_host(link_copies)
    link_gbs = 2 * n * 8 / (t_link / K2) / 1e9
    e2e = {"value": whole_job_rate(world, K2, n, t_zc), "unit": "Gsamples/s",
           "h2d_bytes_per_step": n * 8, "d2h_bytes_per_step": n * 8,
           "path": "dpd_apply_host (zero copy): one kernel reads the pinned host input and writes the pinned "
                   "host output in place over the CPU-GPU link, staged through shared memory in whole lines",
           "gpu_launches_per_step": e2e_launches,
           "link": {"h2d_plus_d2h_gbs": link_gbs, "frac": (2 * n * 8 / (t_zc / K2) / 1e9) / link_gbs,
                    "how": "cudaMemcpyAsync H2D and D2H of the same buffers concurrently on two streams"},
           "pipelined_value": whole_job_rate(world, K2, n, t_pipe),
           "pipelined_path": "dpd_apply_host (pipelined): 2^21-sample chunks copied in, filtered and copied out "
                             "on three streams, overlapping both copy directions with the kernels",
           "explicit_copy_value": whole_job_rate(world, K2, n, t_cp),
           "explicit_copy_path": "cudaMemcpyAsync H2D -> dpd_apply -> cudaMemcpyAsync D2H, one after the other"}

    if not ranks.root:
        f.close()
        ranks.close()
        return 0

    peaks, peak_kind = measured_peaks()
    achieved = BYTES_PER_SAMPLE * n / mean_launch / 1e9
    fl = f.fwd_launch
    kname = f"fwd_tma_kernel<B=5,T=5,V={fl['V']},MODE={fl['mode']}>"
    tr = recorded_traffic(kname)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": tr["dram_bytes_per_launch"] if tr else None,
                "peak_kind": f"of {peak_kind} (copy bandwidth)",
                "kernel": kname, "bytes_per_sample": BYTES_PER_SAMPLE}
    sm_mhz = clocks["sm_mhz"] if clocks and clocks.get("sm_mhz") else peaks.get("sm_max_mhz", 2070.0)
    props = torch.cuda.get_device_properties(dev)
    nominal = props.multi_processor_count * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
    fma = measure_fma_ceiling(dev, gpu_index=local)
    fp32_peak = fma["tflops"]
    rate = n / mean_launch
    alu = {"bound": "alu", "fp32_peak_tflops": fp32_peak,
           "peak_basis": "measured: dpd_probe_fma (FMA chains only) on this GPU, CUDA events, median of 5",
           "peak_probe": fma,
           "nominal_tflops": nominal,
           "nominal_basis": f"{props.multi_processor_count} SMs x 128 FP32 lanes x 2 x {sm_mhz:.0f} MHz",
           "flops_per_sample_alg1": FLOPS_ALG(P, Q, M), "flops_per_sample_executed": FLOPS_WL(P, Q, M),
           "achieved_tflops_alg1": rate * FLOPS_ALG(P, Q, M) / 1e12,
           "achieved_tflops_executed": rate * FLOPS_WL(P, Q, M) / 1e12,
           "frac_executed": rate * FLOPS_WL(P, Q, M) / 1e12 / fp32_peak,
           "frac_executed_of_nominal": rate * FLOPS_WL(P, Q, M) / 1e12 / nominal}

    patterns = {}
    if not args.no_patterns:
        b = measure_batched(dev)
        b["hbm_frac_persistent"] = b["hbm_gbs_persistent"] / peaks["hbm_gbs"]
        patterns["batched"] = b
        patterns["small_2p16"] = measure_small(dev)
        patterns["adjoint"] = measure_direct(dev)
        patterns["grad_kernels"] = measure_grad(dev)
        patterns["gram"] = measure_gram(dev)
        patterns["ila_spectral"] = measure_ila(dev)
        patterns["length_sweep"] = measure_sweep(dev)
        if world == 1:
            patterns["cpu_simd"] = measure_cpu_simd()

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        ncores = os.cpu_count() or 1
        v, el, reps, cores = cpu_oracle_throughput(1 << 22, 10.0, nthreads=ncores)
        cpu = {"value": v, "unit": "Gsamples/s", "cores": cores, "kind": "oracle",
               "sample": f"first 2^22 samples of the workload, repeated {reps}x ({el:.1f} s), FP64 C oracle",
               "all_workloads": cpu_oracle_configs(ncores)}

    line = {
        "metric": METRIC, "value": value, "unit": "Gsamples/s", "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": total_max / K * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "P": P, "Q": Q, "M": M, "n_samples_per_step": n,
                   "l2": "inputs larger than L2: 134 MB in + 134 MB out per step, two alternating buffer sets",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "launch": dict(f.fwd_launch), "launch_picked_by": picked_by},
        "wall_s_timed": wall, "gpu_launches": launches, "clocks": clocks, "roofline": roofline, "alu": alu,
        "e2e": e2e, "cpu_baseline": cpu, "patterns": patterns,
        "samples_per_s_per_gpu": K * n / total / 1e9,
    }
    print(json.dumps(line), flush=True)
    f.close()
    ranks.close()
    return 0


def main():
    args = parse()
    world, rank, local = dist_init()
    if args.impl == "reference":
        return run_reference(args, world, rank)
    if args.pattern == "cpu":
        print(json.dumps({"pattern": "cpu", "result": measure_cpu_simd()}))
        return 0
    if args.pattern == "oracle":
        print(json.dumps({"pattern": "oracle", "result": cpu_oracle_configs(os.cpu_count() or 1)}))
        return 0
    if args.pattern:
        import torch
        dev = torch.device("cuda", local)
        torch.cuda.set_device(dev)
        blaunch = [int(v) for v in args.batched_launch.split(",")] if args.batched_launch else None
        fn = {"small": measure_small, "batched": lambda d: measure_batched(d, launch=blaunch),
              "adjoint": measure_direct,
              "gram": measure_gram, "ila": measure_ila, "sweep": measure_sweep,
              "gram_one": lambda d: measure_gram_one(d, args.gram_precision),
              "grad": lambda d: measure_grad(d, args.grad_log2n),
              "fma": lambda d: measure_fma_ceiling(d, gpu_index=local),
              "estimate": measure_estimate, "estimate_batched": measure_estimate_batched}[args.pattern]
        print(json.dumps({"pattern": args.pattern, "result": fn(dev)}, default=float))
        return 0
    return run_ours(args, world, rank, local)


if __name__ == "__main__":
    sys.exit(main())
