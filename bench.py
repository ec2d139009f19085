#!/usr/bin/env python
"""Benchmark of the low-rank NUFFT-II on one GB300: N = M = 2^20, eps = 1e-9.

One step = the whole online hot path on one batch of synthetic input, as a training
step runs it: the forward NUFFT-II f = A c together with f' = df/dx (pass 1 + pass 2
with one more rank), then the backward of a loss through it: the adjoint A^H g
(pass A + pass B) for dL/dc and Re(conj(g) f') for dL/dx.  The plan (rounding, rank, coefficients, bucketing) is built once
before the timed region, as the paper's planning stage is (section 2.3); its time
is reported separately.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Inputs: x_j = j/N + 0.5 u_j / N with u_j ~ U[-1, 1] (the perturbed grid), c, g ~ CN(0,1)
complex64, all seeded (paper_1701_04492_gb300.workloads).  L2 is flushed (a 512 MiB
write) before every timed step; only the step itself is inside the CUDA events.
Rank 0 prints one JSON line.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "NUFFT-II Gpts/s at N=2^20, ε=1e-9 (fwd, fwd+bwd); % HBM roofline vs plain"
N_LOG2 = 20
EPS = 1e-9
SEED = 2024
FLUSH_BYTES = 512 << 20
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
# the nominal FP32 rate (context only): SMs x 128 FP32 lanes x 2 flops (FMA) x the maximum
# SM clock; the roofline's denominator is the rate measured by nufft_fp32_fma_peak
FP32_LANES = 128


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload_config(N, M, K, gamma, L, ws):
    """The bench line's config, the same for both arms."""
    return {"workload": "1D NUFFT-II fwd+bwd (fwd with df/dx, adjoint A^H, dL/dx), N=M=2^20, "
                        "eps=1e-9, perturbed grid x_j=j/N+0.5u_j/N, c,g~CN(0,1) complex64",
            "N": N, "M": M, "eps": EPS, "K": K, "gamma": gamma, "L": L,
            "parallelism": "replicas" if ws > 1 else "single-gpu",
            "l2": "flushed before every timed step (512 MiB write)"}


def _workload():
    from paper_1701_04492_gb300 import workloads as wl
    N = 1 << N_LOG2
    x = wl.samples_perturbed(N, SEED, 0.5)
    c = wl.coeffs_cn(N, SEED).astype(np.complex64)
    g = wl.cotangent_cn(N, SEED).astype(np.complex64)
    return N, x, c, g


# ---------------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.uuid, "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "20"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def wait_first(self, busy, limit_s=3.0):
        """Run busy() (untimed GPU work) until the sampler has reported once, so that its
        samples cover the timed region that follows."""
        t0 = time.perf_counter()
        while self.proc is not None and not self.lines and time.perf_counter() - t0 < limit_s:
            busy()

    def __exit__(self, *exc):
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
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) != 6:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[2:]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------------
# traffic from the committed ncu summary (null when the kernels changed since)
# ---------------------------------------------------------------------------------

def kernel_source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1701_04492_gb300", "csrc")
    for name in ("fft_team.cuh", "passes.cuh"):
        with open(os.path.join(csrc, name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def committed_traffic(kernel):
    """DRAM bytes per launch of `kernel` inside a running step (ncu, --cache-control none),
    from the committed summary, while the kernel sources still hash as they did then."""
    path = os.path.join(ROOT, "profiles", "ncu_step_kernels_n2e20.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m = re.search(r"source_hash:\s*(\w+)", txt)
    if not m or m.group(1) != kernel_source_hash():
        return None
    # | kernel | dram read MB | dram write MB | in-step dram bytes per launch | ...
    m = re.search(r"^\|\s*%s\s*\|[^|]*\|[^|]*\|\s*([0-9]+)\s*\|" % re.escape(kernel), txt, re.M)
    return float(m.group(1)) if m else None


# ---------------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------------

def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_1701_04492_gb300 import api

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=dev)

    N, x, c_np, g_np = _workload()
    M = x.size
    stream = torch.cuda.current_stream(dev)
    c = torch.tensor(c_np, device=dev)
    g = torch.tensor(g_np, device=dev)
    f = torch.empty(M, dtype=torch.complex64, device=dev)
    gc = torch.empty(N, dtype=torch.complex64, device=dev)
    gx = torch.empty(M, dtype=torch.float32, device=dev)
    fp = torch.empty(M, dtype=torch.complex64, device=dev)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    plan = api.Plan(N, x, EPS, "f32", device=dev)
    torch.cuda.synchronize(dev)
    plan_ms = (time.perf_counter() - t0) * 1e3

    def step():
        plan.forward_deriv(c, f, fp)   # f and df/dx
        plan.adjoint(g, gc)            # dL/dc = A^H g
        plan.grad_x(g, fp, gx)         # dL/dx = Re(conj(g) f')

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize(dev)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for a, b in evs:
            flush.fill_(1.0)
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize(dev)
        return [a.elapsed_time(b) for a, b in evs]

    if args.only == "batch":
        if rank == 0:
            print(json.dumps({"batch_c5": batch_c5(api, dev, timed, args.steps),
                              "nufft2d_c3": bench_2d(api, dev, timed, args.steps),
                              "inverse": bench_inverse(api, dev),
                              "worst_grid_e3": worst_grid_sweep(api, dev, timed, args.steps),
                              "autograd_c4": bench_autograd_c4(api, dev, timed, args.steps)}), flush=True)
        return
    if args.only:
        # profiling mode: only the named operation, no extra measurements
        op = {"step": step, "fwd": lambda: plan.forward(c, f), "adj": lambda: plan.adjoint(g, gc),
              "dx": lambda: plan.dx(c, g, gx)}[args.only]
        for _ in range(args.warmup + args.steps):
            op()
        torch.cuda.synchronize(dev)
        if rank == 0:
            print(json.dumps({"only": args.only, "steps": args.steps, "warmup": args.warmup, "K": plan.K}))
        return

    uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(uuid) as clk:
        clk.wait_first(lambda: (step(), torch.cuda.synchronize(dev)))   # extra untimed steps
        step_ms = timed(step, args.steps, args.warmup)
    if ws > 1:
        dist.barrier()
    total_ms, value = job_throughput(sum(step_ms), ws, M * args.steps, dev)

    extra = {}
    if rank == 0:
        # forward only, and the uniform-x forward
        fwd_ms = timed(lambda: plan.forward(c, f), args.steps, args.warmup)
        extra["fwd_gpts"] = M * len(fwd_ms) / (sum(fwd_ms) * 1e-3) / 1e9
        extra["fwd_ms"] = float(np.mean(fwd_ms))
        from paper_1701_04492_gb300 import workloads as wl
        xu = wl.samples_uniform(M, SEED)
        plan_u = api.Plan(N, xu, EPS, "f32", device=dev)
        fu_ms = timed(lambda: plan_u.forward(c, f), args.steps, args.warmup)
        extra["fwd_uniform_x_gpts"] = M * len(fu_ms) / (sum(fu_ms) * 1e-3) / 1e9
        del plan_u
        # the plain unfused FP64 form of the method, and the fused FP64 path
        c64 = c.to(torch.complex128)
        f64 = torch.empty(M, dtype=torch.complex128, device=dev)
        plan64 = api.Plan(N, x, EPS, "f64", unfused=True, device=dev)
        st = max(3, args.steps // 4)
        pl_ms = timed(lambda: plan64.forward_unfused(c64, f64), st, 2)
        fu64_ms = timed(lambda: plan64.forward(c64, f64), st, 2)
        extra["plain_unfused_fp64_fwd_gpts"] = M * st / (sum(pl_ms) * 1e-3) / 1e9
        extra["fused_fp64_fwd_gpts"] = M * st / (sum(fu64_ms) * 1e-3) / 1e9
        # the comparison at equal accuracy: both FP64 (their errors against the oracle are in
        # cpu_baseline); the FP32 path is faster still but at FP32 accuracy
        extra["fused_fp64_vs_plain_fp64_fwd_speedup"] = extra["fused_fp64_fwd_gpts"] / extra["plain_unfused_fp64_fwd_gpts"]
        extra["fused_fp32_vs_plain_fp64_fwd_speedup_unequal_accuracy"] = \
            extra["fwd_gpts"] / extra["plain_unfused_fp64_fwd_gpts"]
        # for information: the FFT stage alone of a cuFFT-based plain form (torch.fft on the
        # K x L rank matrix), a lower bound on that form's time, in both precisions
        cuf = {}
        for name, dt in (("fp32", torch.complex64), ("fp64", torch.complex128)):
            Xr = torch.randn((plan.K, plan.L), dtype=dt, device=dev)   # not constant: the GPU compresses constant data
            cuf[name + "_K_ffts_ms"] = float(np.median(timed(lambda: torch.fft.fft(Xr, dim=1), args.steps, 3)))
            del Xr
        cuf["fused_fp32_fwd_ms"] = extra["fwd_ms"]
        cuf["fused_fp64_fwd_ms"] = M / (extra["fused_fp64_fwd_gpts"] * 1e9) * 1e3
        cuf["note"] = ("torch.fft (cuFFT) of K x L complex values, the FFT stage alone of a plain form "
                       "that calls cuFFT: a lower bound on its time, beside the whole fused forward")
        extra["cufft_comparator"] = cuf
        plan64.forward_unfused(c64, f64)
        f64_plain = f64.cpu().numpy()
        plan64.forward(c64, f64)
        f64_fused = f64.cpu().numpy()
        del plan64
        # per-kernel device time from events around each launch
        tplan = api.Plan(N, x, EPS, "f32", timing=True, device=dev)
        kt = {"pass1": [], "pass2": [], "passA": [], "passB": [], "pass1_deriv": [], "pass2_deriv": []}
        for i in range(args.warmup + args.steps):
            flush.fill_(1.0)
            tplan.forward(c, f)
            a1, a2 = tplan.kernel_times()
            flush.fill_(1.0)
            tplan.adjoint(g, gc)
            b1, b2 = tplan.kernel_times()
            flush.fill_(1.0)
            tplan.forward_deriv(c, f, fp)
            d1, d2 = tplan.kernel_times()
            if i >= args.warmup:
                for k, v in zip(kt, (a1, a2, b1, b2, d1, d2)):
                    kt[k].append(v)
        kavg = {k: float(np.mean(v)) for k, v in kt.items()}
        extra["kernel_ms"] = kavg
        K, L = tplan.K, tplan.L
        L1 = 1 << ((N_LOG2 + 1) // 2)
        L2 = L // L1
        flops = {
            "pass1": 5.0 * K * L * np.log2(L2) + 2.0 * K * N,
            "pass2": 5.0 * K * L * np.log2(L1) + 8.0 * K * M,
        }
        flops["passA"], flops["passB"] = flops["pass2"], flops["pass1"]
        flops["pass1_deriv"] = 5.0 * (K + 1) * L * np.log2(L2) + 2.0 * (K + 1) * N
        flops["pass2_deriv"] = 5.0 * (K + 1) * L * np.log2(L1) + 8.0 * (2 * K + 1) * M
        dom = max(("pass1_deriv", "pass2_deriv", "passA", "passB"), key=lambda k: kavg[k])
        peak = measure_fp32_peak(dev)
        peak_tf = peak["tflops"]
        ach = flops[dom] / (kavg[dom] * 1e-3) / 1e12
        traffic = committed_traffic(dom)
        roof = {"kernel": dom, "bound": "alu", "achieved": ach, "peak": peak_tf, "unit": "TFLOP/s",
                "frac": ach / peak_tf, "traffic": traffic,
                "peak_source": "measured (of measured): " + peak["how"],
                "peak_measurement": peak,
                "frac_of_nominal": ach / peak["nominal_tflops"],
                "flops_per_launch": flops[dom],
                "alu_frac_per_kernel": {k: flops[k] / (kavg[k] * 1e-3) / 1e12 / peak_tf for k in kavg}}
        hbm = json.load(open(PEAKS_PATH))["hbm_gbs"] if os.path.exists(PEAKS_PATH) else 6800.0
        if traffic is not None:
            # the DRAM bytes ncu counted for one launch inside a step over its measured time
            roof["dram_GBps"] = traffic / (kavg[dom] * 1e-3) / 1e9
            roof["dram_frac_of_measured_hbm"] = roof["dram_GBps"] / hbm
            roof["dram_bytes_per_point"] = traffic / M
        fwd_s = extra["fwd_ms"] * 1e-3
        extra["hbm_algorithmic"] = {
            "bytes_per_point": 24, "fwd_GBps": 24.0 * M / fwd_s / 1e9,
            "frac_of_measured_hbm": 24.0 * M / fwd_s / 1e9 / hbm, "hbm_peak_GBps": hbm}
        del tplan
        extra["peak_tflops_fp32"] = peak_tf

        # end to end through the API with host buffers: H2D c, g; fwd + bwd; D2H f, gc, gx
        ch = torch.tensor(c_np).pin_memory()
        ghost = torch.tensor(g_np).pin_memory()
        fh = torch.empty(M, dtype=torch.complex64).pin_memory()
        gch = torch.empty(N, dtype=torch.complex64).pin_memory()
        gxh = torch.empty(M, dtype=torch.float32).pin_memory()

        def e2e_step():   # one C-ABI call with host buffers (copies overlap the transforms)
            plan.step_host(ch, ghost, fh, gch, gxh)
        e_ms = timed(e2e_step, args.steps, args.warmup)
        torch.cuda.synchronize(dev)
        e2e = {"value": M * len(e_ms) / (sum(e_ms) * 1e-3) / 1e9, "unit": "Gpts/s",
               "h2d_bytes_per_step": ch.numel() * 8 + ghost.numel() * 8,
               "d2h_bytes_per_step": fh.numel() * 8 + gch.numel() * 8 + gxh.numel() * 4}

        line = {
            "metric": METRIC, "value": value, "unit": "Gpts/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(N, M, K, plan.gamma, L, ws),
            "plan_ms": plan_ms,
            "roofline": roof,
            "e2e": e2e,
            "gpu_launches": 5 * args.steps,
            "clocks": clk.summary(),
        }
        line.update(extra)
        if not args.no_batch:
            line["batch_c5"] = batch_c5(api, dev, timed, args.steps)
            line["nufft2d_c3"] = bench_2d(api, dev, timed, args.steps, peak_tf)
            line["inverse"] = bench_inverse(api, dev)
            line["worst_grid_e3"] = worst_grid_sweep(api, dev, timed, args.steps)
            line["autograd_c4"] = bench_autograd_c4(api, dev, timed, args.steps)
        if ws == 1 and not args.no_cpu_baseline:
            plan.forward(c, f)   # the plain forward's f for the accuracy record
            line["cpu_baseline"] = cpu_baseline(plan, c_np, g_np, x, f, {"fp64_fused": f64_fused,
                                                                          "fp64_plain_unfused": f64_plain})
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()


def job_throughput(local_ms, ws, units_per_rank, device):
    """Whole-job throughput of N replicas: the timed region is the slowest rank's
    (max over ranks), and the job processed ws x units_per_rank points in it.
    Returns (max ms, Gpts/s)."""
    import torch
    import torch.distributed as dist
    tot = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    if ws > 1:
        dist.all_reduce(tot, op=dist.ReduceOp.MAX)
    total_ms = float(tot.item())
    return total_ms, ws * units_per_rank / (total_ms * 1e-3) / 1e9


def measure_fp32_peak(dev, seconds=2.0):
    """The FP32 FMA rate of this GPU, measured: nufft_fp32_fma_peak (two 1024-thread CTAs
    per SM, 16 independent FMA chains per thread) launched back to back for about
    `seconds`, each launch timed by CUDA events; the median launch gives TFLOP/s.  The SM
    clock is sampled meanwhile, so the figure comes with the clock it was measured at."""
    import ctypes
    import torch
    from paper_1701_04492_gb300 import _lib
    lib = _lib.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    ms, fl = ctypes.c_float(), ctypes.c_double()
    _lib.check(lib.nufft_fp32_fma_peak(1000, 2, stream, ctypes.byref(ms), ctypes.byref(fl)), "fma peak")
    iters = max(1000, int(1000 * 0.2 / max(ms.value * 1e-3, 1e-6)))   # about 0.2 s per launch
    props = torch.cuda.get_device_properties(dev)
    uuid = "GPU-" + str(props.uuid)
    rates = []
    with ClockSampler(uuid) as clk:
        clk.wait_first(lambda: lib.nufft_fp32_fma_peak(1000, 2, stream, ctypes.byref(ms), ctypes.byref(fl)))
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < seconds or len(rates) < 3:
            _lib.check(lib.nufft_fp32_fma_peak(iters, 2, stream, ctypes.byref(ms), ctypes.byref(fl)), "fma peak")
            rates.append(fl.value / (ms.value * 1e-3) / 1e12)
    c = clk.summary()
    sms = props.multi_processor_count
    nominal = sms * FP32_LANES * 2 * (c["sm_max_mhz"] or 2070.0) * 1e6 / 1e12
    return {"tflops": float(np.median(rates)), "launches": len(rates), "ms_per_launch": float(ms.value),
            "sm_mhz_median": c["sm_mhz"], "sm_max_mhz": c["sm_max_mhz"], "clock_reasons": c["reasons"],
            "sms": sms, "nominal_tflops": nominal,
            "how": "nufft_fp32_fma_peak: %d SMs x 2 CTAs x 1024 threads x 16 FMA chains, %d launches of "
                   "%.0f ms, median, CUDA events" % (sms, len(rates), ms.value)}


def batch_c5(api, dev, timed, steps):
    """The serving workload: 512 independent problems, N log-uniform in [2^10, 2^18]
    (integers, M = N), eps drawn from {1e-4, 1e-7, 1e-12}, uniform x, complex64 c.
    Packed c, f (sum N values each); the same work run five ways."""
    import torch
    from paper_1701_04492_gb300 import workloads as wl
    Ns, epss = wl.uneven_batch(512, SEED)
    Ns = [int(n) for n in Ns]
    xs = [wl.samples_uniform(n, SEED + 1 + i) for i, n in enumerate(Ns)]
    tot = int(sum(Ns))
    c = torch.tensor(wl.coeffs_cn(tot, SEED).astype(np.complex64), device=dev)
    g = torch.tensor(wl.cotangent_cn(tot, SEED).astype(np.complex64), device=dev)
    f = torch.empty(tot, dtype=torch.complex64, device=dev)
    cc = torch.empty(tot, dtype=torch.complex64, device=dev)
    out = {"workload": "512 problems, N=M=round(2^U[10,18]), eps in {1e-4,1e-7,1e-12}, uniform x, complex64",
           "sum_N": tot, "unit": "Gpts/s (sum M / time)"}
    variants = [("per_problem_launches", {"per_problem": True}, True),
                ("per_problem_graph", {"per_problem": True, "graph": True}, False),
                ("batched", {}, False),
                ("batched_graph", {"graph": True}, False),
                ("batched_autotuned", {"autotune": True}, False),
                ("batched_graph_autotuned", {"graph": True, "autotune": True}, False),
                ("persistent", {"persistent": True}, False),
                ("persistent_graph", {"persistent": True, "graph": True}, False),
                ("persistent_graph_autotuned", {"persistent": True, "graph": True, "autotune": True}, False)]
    for name, kw, each in variants:
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        b = api.Batch(Ns, xs, epss, "f32", device=dev, **kw)
        torch.cuda.synchronize(dev)
        plan_s = time.perf_counter() - t0
        if each:
            fw, bw = (lambda: b.forward_each(c, f)), (lambda: b.adjoint_each(f, cc))
        else:
            fw, bw = (lambda: b.forward(c, f)), (lambda: b.adjoint(f, cc))
        ms_f = timed(fw, steps, 3)
        ms_fb = timed(lambda: (fw(), bw()), steps, 3)
        b.check()
        out[name] = {"fwd": tot * len(ms_f) / (sum(ms_f) * 1e-3) / 1e9,
                     "fwd_bwd": tot * len(ms_fb) / (sum(ms_fb) * 1e-3) / 1e9,
                     "fwd_ms": float(np.mean(ms_f)), "plan_s": plan_s,
                     "launches_per_fwd": 2 * b.count if each else b.launches_per_direction,
                     "grid_doubled": int(sum(int(L) > max(1024, 1 << (n - 1).bit_length()) for L, n in zip(b.L, Ns)))}
        b.close()
    return out


def bench_2d(api, dev, timed, steps, peak_tf=None):
    """The 2D workload of section 4: m = n = 1024, M = 2^20 uniform samples in [0,1)^2,
    eps = 1e-6 (K_x = K_y = 10 at eps/2), C[k1][k2] ~ CN(0,1)/(1 + k1^2 + k2^2)^(1/2)
    complex64; forward Gpts/s with per-pass device times and algorithmic flops."""
    import torch
    from paper_1701_04492_gb300 import workloads as wl
    m = n = 1024
    M = 1 << 20
    x, y = wl.samples_2d_uniform(M, SEED)
    C = torch.tensor(wl.coeffs_2d_decay(m, n, SEED).astype(np.complex64), device=dev)
    f = torch.empty(M, dtype=torch.complex64, device=dev)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    p = api.Plan2D(m, n, x, y, 1e-6, device=dev, timing=True)
    torch.cuda.synchronize(dev)
    plan_s = time.perf_counter() - t0
    g = torch.tensor(wl.cotangent_cn(M, SEED).astype(np.complex64), device=dev)
    Ca = torch.empty((m, n), dtype=torch.complex64, device=dev)
    ms = timed(lambda: p.forward(C, f), steps, 3)
    msa = timed(lambda: p.adjoint(g, Ca), steps, 3)
    kt, kta = [], []
    for _ in range(steps):
        p.forward(C, f)
        kt.append(p.kernel_times())
        p.adjoint(g, Ca)
        kta.append(p.kernel_times())
    k1, k2 = float(np.median([k[0] for k in kt])), float(np.median([k[1] for k in kt]))
    a_rows, a_cols = float(np.median([k[0] for k in kta])), float(np.median([k[1] for k in kta]))
    p.check()
    Kx, Ky, Lx, Ly = p.Kx, p.Ky, p.Lx, p.Ly
    L = Lx * Ly
    fl_cols = 5.0 * Kx * L * np.log2(Lx) + 2.0 * Kx * m * n
    fl_rows = 5.0 * Kx * Ky * L * np.log2(Ly) + 8.0 * Kx * Ky * M
    if peak_tf is None:
        peak_tf = measure_fp32_peak(dev)["tflops"]
    return {"workload": "2D NUFFT-II m=n=1024, M=2^20 uniform (x,y), eps=1e-6, C~CN(0,1)/sqrt(1+k1^2+k2^2) complex64",
            "Kx": Kx, "Ky": Ky, "fwd_gpts": M * len(ms) / (sum(ms) * 1e-3) / 1e9, "fwd_ms": float(np.mean(ms)),
            "adj_gpts": M * len(msa) / (sum(msa) * 1e-3) / 1e9, "adj_ms": float(np.mean(msa)),
            "plan_s": plan_s, "kernel_ms": {"cols": k1, "rows": k2, "adj_rows": a_rows, "adj_cols": a_cols},
            "alu_frac": {"cols": fl_cols / (k1 * 1e-3) / 1e12 / peak_tf, "rows": fl_rows / (k2 * 1e-3) / 1e12 / peak_tf,
                         "adj_rows": fl_rows / (a_rows * 1e-3) / 1e12 / peak_tf,
                         "adj_cols": fl_cols / (a_cols * 1e-3) / 1e12 / peak_tf},
            "launches_per_fwd": 2, "launches_per_adj": 2}


def worst_grid_sweep(api, dev, timed, steps):
    """Section 2.4's worst grid at N = M = 2^20, eps = 1e-9: two shifted halves,
    x_j = (j + gamma)/N for j <= N/2 and (j - gamma)/N above, so every |delta_j| = gamma.
    gamma in {1/2, 1/8, 1/32, 0} sets K (12, 9, 7, 1); forward and forward+adjoint Gpts/s."""
    import torch
    from paper_1701_04492_gb300 import workloads as wl
    N = 1 << 20
    c = torch.tensor(wl.coeffs_cn(N, SEED).astype(np.complex64), device=dev)
    f = torch.empty(N, dtype=torch.complex64, device=dev)
    gc = torch.empty(N, dtype=torch.complex64, device=dev)
    out = {"workload": "1D NUFFT-II on the worst grid, N=M=2^20, eps=1e-9, c~CN(0,1) complex64"}
    for gname, gamma in (("1/2", 0.5), ("1/8", 1 / 8), ("1/32", 1 / 32), ("0", 0.0)):
        p = api.Plan(N, wl.samples_worst(N, gamma), EPS, "f32", device=dev)
        fw = timed(lambda: p.forward(c, f), steps, 3)
        fb = timed(lambda: (p.forward(c, f), p.adjoint(f, gc)), steps, 3)
        out[gname] = {"K": p.K, "gamma": p.gamma, "fwd_gpts": N * len(fw) / (sum(fw) * 1e-3) / 1e9,
                      "fwd_adj_gpts": N * len(fb) / (sum(fb) * 1e-3) / 1e9}
        del p
    return out


def bench_inverse(api, dev):
    """The inverse NUFFT-II of section 3.3 at N = 2^20 on the perturbed grid with
    gamma = 1/8 (Fig. 3.1's middle case): f = A c for a known c, then CG to tol, timed end
    to end on the device (the solver's per-iteration host check included), FP64 and FP32."""
    import torch
    from paper_1701_04492_gb300 import workloads as wl
    N = 1 << 20
    x = wl.samples_perturbed(N, SEED, 1 / 8)
    out = {"workload": "inverse NUFFT-II, N=M=2^20, perturbed grid gamma=1/8, CG on A^H A (Toeplitz, 2N circulant)"}
    for prec, eps, tol, cdt in (("f64", 1e-14, 1e-12, torch.complex128), ("f32", 1e-7, 1e-5, torch.complex64)):
        c = torch.tensor(wl.coeffs_cn(N, SEED), dtype=cdt, device=dev)
        p = api.Plan(N, x, eps, prec, device=dev)
        f = p.forward(c)
        p.inverse(f, tol=tol, maxit=1)          # builds the solver state
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        cs, it, rr = p.inverse(f, tol=tol, maxit=1000)
        torch.cuda.synchronize(dev)
        sec = time.perf_counter() - t0
        err = float(torch.linalg.vector_norm(cs - c) / torch.linalg.vector_norm(c))
        out[prec] = {"tol": tol, "iterations": it, "relres": rr, "ms": sec * 1e3, "ms_per_iteration": sec * 1e3 / max(it, 1),
                     "rel_err_vs_c": err}
        del p
    return out


def bench_autograd_c4(api, dev, timed, steps):
    """The differentiable workload: N = M = 2^18, 64 complex64 coefficient vectors sharing
    uniform x, loss = sum |f - f*|^2; one step = forward (with f' for dL/dx) + backward
    (A^H g per member, dL/dx summed), through torch.autograd; all 64 members run in one
    launch per pass."""
    import torch
    from paper_1701_04492_gb300 import workloads as wl
    N = M = 1 << 18
    B = 64
    x = wl.samples_uniform(M, SEED)
    plan = api.Plan(N, x, 1e-9, "f32", device=dev)
    c0 = torch.tensor(np.stack([wl.coeffs_cn(N, SEED + b) for b in range(B)]).astype(np.complex64), device=dev)
    ft = plan.forward(torch.tensor(wl.coeffs_cn(N, SEED + B).astype(np.complex64), device=dev))
    xt = torch.tensor(x, dtype=torch.float64, device=dev, requires_grad=True)
    c = c0.clone().requires_grad_(True)

    def train_step():
        c.grad = None
        xt.grad = None
        f = api.nufft2(c, xt, plan=plan)
        ((f - ft[None, :]).abs() ** 2).sum().backward()
    ms = timed(train_step, steps, 3)
    return {"workload": "autograd NUFFT-II, N=M=2^18, batch 64 complex64, x shared, loss sum|f-f*|^2, grads to c and x",
            "ms_per_step": float(np.mean(ms)), "gpts_per_s": B * M * len(ms) / (sum(ms) * 1e-3) / 1e9,
            "gpu_launches_per_step": 5}   # batched forward+f' (2), batched adjoint (2), dL/dx summed (1)


def _oracle_worker(L, seconds, steps, warmup, ready, start, out):
    """One process of the CPU baseline: plan the workload with the oracle (untimed), run
    `warmup` steps, report ready, wait for the common start, then run fwd+bwd steps of the
    oracle as it stands -- exactly `steps` of them, or (steps = 0) as many as fit in
    `seconds` -- and report (steps done, seconds taken)."""
    sys.path.insert(0, ROOT)
    from oracle import lowrank
    N, x, c_np, g_np = _workload()
    c, g = c_np.astype(np.complex128), g_np.astype(np.complex128)
    P = lowrank.plan(N, x, EPS, L)

    def step():
        f = lowrank.nufft2(P, c)
        lowrank.nufft2_adjoint(P, f)
        lowrank.nufft2_dx(P, c, g)
    for _ in range(warmup):
        step()
    ready.put(P.K)
    start.wait()
    t0 = time.perf_counter()
    n = 0
    while (n < steps) if steps > 0 else (n < 1 or time.perf_counter() - t0 < seconds):
        step()
        n += 1
    out.put((n, time.perf_counter() - t0))


def oracle_pool(L, seconds=10.0, steps=0, warmup=0, procs=None):
    """The oracle on every host core: `procs` (default: all cores) spawned processes, each
    running the whole workload's fwd+bwd steps single-threaded (BLAS and OpenMP limited to
    one thread each), started together.  Throughput = all the points they processed over
    the slowest one's time.  Spawned, not forked, so the GPU context of this process is
    not inherited."""
    import multiprocessing as mp
    procs = procs or os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    ready, out, start = ctx.Queue(), ctx.Queue(), ctx.Event()
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        ps = [ctx.Process(target=_oracle_worker, args=(L, seconds, steps, warmup, ready, start, out))
              for _ in range(procs)]
        for p in ps:
            p.start()
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    K = [ready.get(timeout=900) for _ in ps][0]
    start.set()
    res = [out.get(timeout=1800) for _ in ps]
    for p in ps:
        p.join(timeout=60)
    n_tot = sum(n for n, _ in res)
    wall = max(dt for _, dt in res)
    return {"steps_total": n_tot, "wall_s": wall, "procs": procs, "K": K,
            "gpts": (1 << N_LOG2) * n_tot / wall / 1e9, "steps_per_proc": [n for n, _ in res]}


def cpu_baseline(plan, c_np, g_np, x, f_gpu, others=None):
    """The oracle as it stands on all of this host's cores, for about 10 s (see
    oracle_pool); also the GPU results' errors against the oracle (the FP32 step's
    forward, and the FP64 fused and plain forwards in `others`)."""
    from oracle import lowrank
    N = c_np.size
    c = c_np.astype(np.complex128)
    P = lowrank.plan(N, x, EPS, plan.L)
    f_cpu = lowrank.nufft2(P, c)
    fg = f_gpu.cpu().numpy().astype(np.complex128)
    err2 = float(np.linalg.norm(fg - f_cpu) / np.linalg.norm(f_cpu))
    errinf = float(np.max(np.abs(fg - f_cpu)) / np.sum(np.abs(c)))
    errs = {k + "_rel2_err_vs_oracle": float(np.linalg.norm(v - f_cpu) / np.linalg.norm(f_cpu))
            for k, v in (others or {}).items()}
    pool = oracle_pool(plan.L, seconds=10.0)
    return {"value": pool["gpts"], "unit": "Gpts/s", "cores": pool["procs"], "nproc": os.cpu_count(),
            "kind": "oracle",
            "sample": "%d processes (one per host core), each running full fwd+bwd steps of the same workload "
                      "(N=M=2^20, K=%d) with the numpy FP64 oracle, single-threaded, for about 10 s: %d steps in "
                      "%.1f s, plan excluded" % (pool["procs"], P.K, pool["steps_total"], pool["wall_s"]),
            "gpu_f32_fwd_rel2_err_vs_oracle": err2, "gpu_f32_fwd_inf_err_over_c1": errinf, **errs,
            "eps_note": "the FP32 path's error is set by FP32 rounding: its infinity-norm error over ||c||_1 "
                        "is the number above, next to eps = 1e-9"}


# ---------------------------------------------------------------------------------
# reference arm: the oracle, on this host's cores
# ---------------------------------------------------------------------------------

def run_reference(args):
    """The reference arm: the oracle as it stands on all host cores.  One step = every
    process runs one full fwd+bwd step of the workload (so a step processes procs x M
    points); `steps` timed steps after `warmup` untimed ones, the slowest process's time."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    from oracle import lowrank
    N, x, _, _ = _workload()
    gamma = float(np.max(np.abs(lowrank.round_to_grid(x, N)[2])))
    pool = oracle_pool(N, steps=args.steps, warmup=args.warmup, procs=args.cpu_procs)
    v = pool["gpts"]
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Gpts/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": pool["wall_s"] / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": workload_config(N, x.size, pool["K"], gamma, N, ws),
            "cpu_baseline": {"value": v, "unit": "Gpts/s", "cores": pool["procs"], "nproc": os.cpu_count(),
                             "kind": "oracle",
                             "sample": "%d processes (one per host core), each running full fwd+bwd steps of the "
                                       "workload with the numpy FP64 oracle, single-threaded; a step is one such "
                                       "step in every process (%d x M points), plan excluded"
                                       % (pool["procs"], pool["procs"])},
            "e2e": {"value": v, "unit": "Gpts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-procs", type=int, default=None,
                    help="processes of the oracle in the CPU baseline and the reference arm (default: all cores)")
    ap.add_argument("--no-batch", action="store_true", help="skip the 512-problem batch measurement")
    ap.add_argument("--only", choices=["step", "fwd", "adj", "dx", "batch"], default=None,
                    help="profiling mode: run only this operation warmup+steps times, untimed "
                         "(batch: only the 512-problem batch, 2D and inverse measurements, timed)")
    args = ap.parse_args()
    if args.warmup < 3 and not args.only:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
