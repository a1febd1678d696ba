#!/usr/bin/env python
"""Benchmark of the calibrate-and-peel cadence on GB300.

Workload (a synthetic MWA cadence with the shape of the paper's Table 1):
512 antennas (130816 baselines), 768 channels x 40 kHz from 167 MHz, 8 times x
1 s, 4 polarisations, complex64 (25.7 GB cube), 1000 sources peeled with 20 ALS
sweeps each.  The cube is the library's own prediction of the 1000 sources with
their true Jones matrices plus Gaussian noise (sigma = 0.01 Jy), resident in HBM
before timing.  One step = one rts_peel_cadence call over that cube (out of
place: the input stays intact, the residual goes to a second cube).

Metric: source x visibility peel updates per second = K N_bl N_chan N_t / time.
Extra legs in the same run: end to end through rts_peel_cadence_host (pinned
host buffers, copies timed), the plain FP64 GPU path on the same input for a
bounded number of sources, the adjoint step (config with 300 sources,
perturbed positions; mixed and FP64 paths), the ionospheric offset step at the
same shape, and the FP64 CPU oracle on a bounded sample (the CPU baseline).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
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

METRIC = "source×visibility peel updates/s (512 ant, 768 ch); adjoint step ms vs FP64 path"
UNIT = "updates/s"
BYTES_PER_UPDATE = 64          # complex64 2x2 read + write per source x visibility
FLOPS_PER_UPDATE = 32          # 2x2 complex times a complex phasor: 4 complex multiply-adds
ADJ_FLOPS_PER_UPDATE = 80      # adjoint: model MACs 32 + R e^{+i phi} 24 + plain and channel-weighted sums 24
MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def workload_config(cad, n_src, n_iter):
    return {
        "workload": (f"MWA cadence {cad.n_ant} ant ({cad.n_bl} baselines) x {cad.n_chan} ch x "
                     f"{cad.n_time} t x 4 pol complex64, {n_src} sources peeled, {n_iter} ALS sweeps"),
        "n_ant": cad.n_ant, "n_baselines": cad.n_bl, "n_chan": cad.n_chan, "n_time": cad.n_time,
        "n_sources": n_src, "n_iter": n_iter,
        "cube_bytes": cad.n_vis * 32,
        "l2": "inputs larger than L2 (25.7 GB cube vs 129 MB L2); no flush needed",
        "precision": "mixed: FP32 streaming, FP64 phase argument and normal-equation sums",
    }


# ---------------------------------------------------------------------------
# clocks (nvidia-smi sampled during the timed region)

class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


KERNEL_SOURCES = {"k_stream_mixed<true,true>": ("common.cuh", "stream_kernels.cuh"),
                  "k_block_pass<64,true,true>": ("common.cuh", "stream_kernels.cuh", "block_kernels.cuh"),
                  "k_block_pass_tc05<true,true>": ("common.cuh", "stream_kernels.cuh", "block_kernels.cuh",
                                                   "tc05.cuh", "block_tc05_kernels.cuh"),
                  "k_block_pass_tc05<true,true,true>": ("common.cuh", "stream_kernels.cuh", "block_kernels.cuh",
                                                        "tc05.cuh", "block_tc05_kernels.cuh"),
                  "k_grad_sweep_fac<false>": ("common.cuh", "kahan.cuh", "grad_kernels.cuh"),
                  "k_stream_taylor<true,true>": ("common.cuh", "stream_kernels.cuh", "als_kernels.cuh",
                                                 "taylor_kernels.cuh"),
                  "k_integrate": ("rts_integrate.cu",)}


def kernel_source_hash(kernel: str) -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        h.update(open(os.path.join(ROOT, "paper_1003_5575_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, if it still matches the kernel source."""
    try:
        t = json.load(open(TRAFFIC_FILE))
        e = t[kernel]
        if e.get("source_hash") == kernel_source_hash(kernel):
            return e["dram_bytes_per_launch"]
    except (OSError, KeyError, ValueError):
        pass
    return None


def fp32_peak_tflops(sm_mhz: float) -> float:
    """FP32 (non-tensor) peak: the device's SMs x 128 FP32 lanes x 2 flop (FMA) x clock."""
    import torch
    n_sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    return n_sm * 128 * 2 * sm_mhz * 1e6 / 1e12


# ---------------------------------------------------------------------------
# CPU oracle (baseline leg and the reference arm)

def oracle_sample(n_chan=16, n_src=4):
    """A bounded sample of the same workload for the FP64 CPU oracle: the full
    512-antenna geometry and 8 times, the first n_chan channels, n_src sources."""
    import numpy as np
    import oracle
    from synth import config
    cad = config(3).with_(n_chan=n_chan, n_src=n_src)
    V = oracle.simulate(cad)
    V = V.astype(np.complex64).astype(np.complex128)
    return cad, V


def time_oracle(cad, V, reps=1):
    import oracle
    t0 = time.perf_counter()
    for _ in range(reps):
        oracle.peel(cad.uvw(), cad.freqs(), V, cad.sources(), n_iter=20)
    dt = (time.perf_counter() - t0) / reps
    return cad.n_src * cad.n_vis / dt, dt


def run_cpu_baselines():
    """The CPU-baseline plan: the FP64 oracle on the machine's host cores, all cores and
    one core; configurations 1, 2 and 4 peeled in full, the full-size
    configuration 3 on its first 20 sources and extrapolated linearly to 1000
    (labelled so).  One JSON line; minutes of CPU time."""
    import numpy as np
    import oracle
    from synth import config
    oracle.build()
    n_all = oracle.num_threads()
    rows = []
    plan = [("config 1", config(1), None, True), ("config 2", config(2), None, True),
            ("config 4", config(4).with_(pos_sigma_rad=0.0), None, False),
            ("config 3, first 20 sources", config(3), 20, False)]
    for label, cad, k, single in plan:
        run = cad.with_(n_src=k) if k else cad
        V = oracle.simulate(run)
        if run.precision == "mixed":
            V = V.astype(np.complex64).astype(np.complex128)
        row = {"workload": label, "n_ant": run.n_ant, "n_chan": run.n_chan, "n_time": run.n_time,
               "sources_timed": run.n_src}
        for threads in ([n_all, 1] if single else [n_all]):
            oracle.set_num_threads(threads)
            rate, dt = time_oracle(run, V)
            row[f"{threads}_cores"] = {"s": dt, "updates_per_s": rate}
        oracle.set_num_threads(n_all)
        if k:
            row["extrapolated_to_sources"] = cad.n_src
            row["extrapolated_s"] = row[f"{n_all}_cores"]["s"] * cad.n_src / k
        rows.append(row)
    print(json.dumps({"cpu_baselines": rows, "cores": n_all, "os_cpu_count": os.cpu_count(),
                      "kind": "oracle (plain FP64 C, OpenMP over baselines)"}), flush=True)
    return 0


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    from synth import config
    oracle.build()
    cad, V = oracle_sample(n_chan=8, n_src=2)
    for _ in range(args.warmup):
        time_oracle(cad, V)
    times = []
    for _ in range(args.steps):
        _, dt = time_oracle(cad, V)
        times.append(dt)
    ms = 1e3 * sum(times) / len(times)
    value = cad.n_src * cad.n_vis / (ms / 1e3)
    sample = (f"512 ant, 8 t, first {cad.n_chan} of 768 channels, {cad.n_src} sources per step "
              "(FP64 C oracle, OpenMP over baselines)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(config(3), 1000, 20),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU legs

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-baselines", action="store_true",
                    help="time the FP64 CPU oracle on configurations 1, 2, 4 and 3 (first 20 sources) instead")
    ap.add_argument("--sources", type=int, default=1000, help="sources peeled per cadence")
    ap.add_argument("--n-iter", type=int, default=20)
    ap.add_argument("--antennas", type=int, default=512,
                    help="antennas (512 = the workload; fewer only for small profiling cases)")
    ap.add_argument("--channels", type=int, default=768,
                    help="channels (768 = the workload; fewer only for small profiling cases)")
    ap.add_argument("--per-pass", type=int, default=0,
                    help="sources per streaming pass: 1, 64 (blocked) or 0 (library default)")
    ap.add_argument("--block-kernel", type=int, default=0, choices=[0, 1, 2, 3],
                    help="blocked pass: 0 library choice, 1 FP32 FMA pass, 2 mma.sync pass, 3 tcgen05 pass")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the FP64 / adjoint / CPU legs")
    ap.add_argument("--profile-case", choices=["adjoint", "taylor", "grid", "integrate"], default=None,
                    help="only this workload, twice, at --antennas antennas (small ncu captures; "
                         "adjoint: 300 sources of the config-5 cadence, taylor: --sources sources (one pass per "
                         "source, blocked with --per-pass 64), "
                         "grid: the gridder leg on random values, integrate: the integrator leg); prints "
                         "its own one-line summary, "
                         "not the benchmark line")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.cpu_baselines:
        return run_cpu_baselines()
    if args.profile_case:
        return run_profile_case(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_1003_5575_gb300 import replicas
    barrier = replicas.barrier

    def max_over_ranks(x: float) -> float:
        return replicas.max_over_ranks(x, device="cuda")

    import __graft_entry__
    __graft_entry__.build()
    from paper_1003_5575_gb300 import Peeler, _abi
    from synth import config

    cad = config(3).with_(n_src=args.sources, n_chan=args.channels, n_ant=args.antennas,
                          seed=replicas.rank_seed(config(3).seed, rank))
    src = cad.sources()
    K = cad.n_src
    log(f"[rank {rank}] building cadence: {cad.n_ant} ant, {cad.n_chan} ch, {cad.n_time} t, {K} sources")
    p = Peeler(cad.uvw(), cad.freqs(), n_iter=args.n_iter, precision="mixed", max_sources=K,
               sources_per_pass=args.per_pass, block_kernel=args.block_kernel)
    J_true = torch.from_numpy(cad.jones().astype(np.complex64)).cuda()
    stream = torch.cuda.current_stream()
    d_vis = p.predict(src, J_true)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(cad.seed)
    noise = torch.randn(d_vis.shape + (2,), generator=gen, device="cuda", dtype=torch.float32)
    d_vis.view(torch.float32).view(noise.shape).add_(noise, alpha=cad.noise_sigma)
    del noise
    d_resid = p.empty_cube()
    d_jones = torch.empty((K, cad.n_ant, 4), dtype=torch.complex64, device="cuda")
    torch.cuda.synchronize()
    updates_per_step = K * cad.n_vis

    for _ in range(args.warmup):
        p.cadence(d_vis, src, resid=d_resid, jones=d_jones, status=False)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    _abi.rts_peel_timing(p.h, 1)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        p.cadence(d_vis, src, resid=d_resid, jones=d_jones, status=False)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    _abi.rts_peel_timing(p.h, 0)
    ktimes = _abi.rts_peel_timing_read(p.h)
    ms_total = max_over_ranks(e0.elapsed_time(e1))
    ms_step = ms_total / args.steps
    value = replicas.job_rate(updates_per_step * args.steps, ms_total / 1e3, world)
    launches = sum(v[2] for v in ktimes.values())

    # results of the timed cadence: statuses (untimed re-run with status)
    _, _, st = p.cadence(d_vis, src, resid=d_resid, jones=d_jones, status=True)
    n_nonconv = int(np.sum(st == 1))

    # roofline of the dominant kernel
    peaks = json.load(open(MEASURED_PEAKS)) if os.path.exists(MEASURED_PEAKS) else {}
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    shares = {k: round(v[0] / max(1e-9, sum(x[0] for x in ktimes.values())), 4) for k, v in ktimes.items()
              if v[2]}
    block_kernel, solve_kernel = _abi.rts_peel_kernels(p.h)
    if ktimes["block_pass"][2]:
        # blocked path: the fused pass (subtract a block + average the next block)
        ms_bp, n_bp, _ = ktimes["block_pass"]
        flops = 2 * K * cad.n_vis * FLOPS_PER_UPDATE * args.steps        # every source subtracted and averaged once
        achieved = flops / (ms_bp / 1e3) / 1e12
        sm_mhz = clk.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
        name = {1: "k_block_pass<64,SUB,ACC> (FP32 FMA)", 2: "k_block_pass_tc<SUB,ACC> (TF32 mma.sync)",
                3: "k_block_pass_tc05<SUB,ACC> (tcgen05.mma kind::tf32, TMEM accumulators)"}[block_kernel]
        if block_kernel == 1:
            peak = fp32_peak_tflops(sm_mhz)
            bound, peak_source = "alu", (f"derived: the device's SMs x 128 FP32 lanes x 2 flop x {sm_mhz:.0f} MHz "
                                         "(median SM clock under load)")
        else:
            # TF32 dense peak: measured bf16 (sustained: the pass runs inside a long step)
            # x the nominal TF32/BF16 ratio 1.1/2.25
            bf16 = peaks.get("bf16_tflops_sustained") or 1700.0
            peak = bf16 * 1.1 / 2.25
            bound = "tensor"
            peak_source = (f"MEASURED_PEAKS.json bf16_tflops_sustained {bf16:.0f} x nominal TF32/BF16 ratio 1.1/2.25 "
                           "(of measured)")
        roofline = {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak,
                    "traffic": (ncu_traffic("k_block_pass<64,true,true>") if block_kernel == 1 else
                                ncu_traffic("k_block_pass_tc05<true,true>") if block_kernel == 3 else None),
                    "kernel": name + ": subtract 64 solved sources + average the next 64",
                    "algorithmic_flops_per_update": FLOPS_PER_UPDATE,
                    "algorithmic_flops_note": ("32 FP32 flop per source x visibility for each of the subtraction and "
                                               "the average (4 complex multiply-adds); the tensor-core passes execute "
                                               "3 TF32 MMAs per product (split operands), so the tensor pipes do 3x "
                                               "the algorithmic work"),
                    "algorithmic_bytes_per_launch": cad.n_vis * BYTES_PER_UPDATE,
                    "avg_launch_ms": ms_bp / n_bp,
                    "hbm_GBps_of_the_pass": cad.n_vis * BYTES_PER_UPDATE / (ms_bp / n_bp / 1e3) / 1e9,
                    "peak_source": peak_source,
                    "device_time_share": shares}
    else:
        ms_k3, n_k3, _ = ktimes["sub_average"]
        per_launch_s = (ms_k3 / n_k3) / 1e3 if n_k3 else float("nan")
        alg_bytes = cad.n_vis * BYTES_PER_UPDATE
        achieved = alg_bytes / per_launch_s / 1e9
        roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                    "frac": achieved / hbm_peak, "traffic": ncu_traffic("k_stream_mixed<true,true>"),
                    "kernel": "k_stream_mixed<SUB,ACC> (subtract source k + rotate/average source k+1)",
                    "algorithmic_bytes_per_launch": alg_bytes,
                    "avg_launch_ms": per_launch_s * 1e3,
                    "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks else "fallback",
                    "device_time_share": shares}
    log(f"[rank {rank}] {ms_step:.1f} ms/step, {value:.3e} updates/s, roofline {roofline['achieved']:.1f} "
        f"{roofline['unit']} ({roofline['frac']:.2f} of {roofline['bound']} peak)")

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded MWA-shaped cadence, library-predicted sky + noise)",
        "config": dict(workload_config(cad, K, args.n_iter), parallelism=f"replicas{world}"),
        "clocks": clk, "gpu_launches": int(launches), "roofline": roofline,
        "kernels": {"block_pass": {0: "one source per pass", 1: "fp32-fma", 2: "tf32-mma.sync",
                                   3: "tcgen05-tf32"}[block_kernel],
                    "block_solve": {0: "cooperative (one launch per block)", 1: "one launch per step"}[solve_kernel]},
        "kernel_ms": {k: round(v[0], 3) for k, v in ktimes.items() if v[2]},
        "status": {"not_converged": n_nonconv, "sources": K},
    }

    # ---- end to end through the pipelined host-buffer C-ABI calls -----------
    if not args.no_e2e:
        import ctypes
        cube_bytes = cad.n_vis * 32
        h_in = _abi.rts_host_alloc(cube_bytes)
        h_out = [_abi.rts_host_alloc(cube_bytes), _abi.rts_host_alloc(cube_bytes)]
        try:
            arr = np.ctypeslib.as_array((ctypes.c_float * (cad.n_vis * 8)).from_address(h_in))
            torch.from_numpy(arr).copy_(d_vis.view(torch.float32).reshape(-1))
            # raw copy bandwidth of the same buffers (context for the e2e number)
            arr_o = np.ctypeslib.as_array((ctypes.c_float * (cad.n_vis * 8)).from_address(h_out[0]))
            e_a, e_b, e_c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e_a.record(stream)
            d_resid.view(torch.float32).reshape(-1).copy_(torch.from_numpy(arr), non_blocking=True)
            e_b.record(stream)
            torch.from_numpy(arr_o).copy_(d_resid.view(torch.float32).reshape(-1), non_blocking=True)
            e_c.record(stream)
            torch.cuda.synchronize()
            h2d_gbs = cube_bytes / (e_a.elapsed_time(e_b) / 1e3) / 1e9
            d2h_gbs = cube_bytes / (e_b.elapsed_time(e_c) / 1e3) / 1e9
            src_c = np.ascontiguousarray(src, dtype=np.float64)
            h_jones = [np.zeros((K, cad.n_ant, 4), np.complex64) for _ in range(2)]
            h_st = [np.zeros(K, np.int32) for _ in range(2)]
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int32)

            def submit(i):
                _abi.rts_peel_pipeline_submit(p.h, ctypes.c_void_p(h_in), ctypes.c_void_p(h_out[i % 2]), K,
                                              src_c.ctypes.data_as(dp),
                                              ctypes.c_void_p(h_jones[i % 2].ctypes.data),
                                              h_st[i % 2].ctypes.data_as(ip))
            submit(0)
            _abi.rts_peel_pipeline_wait(p.h)
            # a stream of cadences, as the real-time pipeline runs: the first copy-in and the
            # last copy-out (the pipeline's fill and drain) spread over 8 cadences at least
            n_e2e = max(8, args.steps)
            barrier()
            t0 = time.perf_counter()
            for i in range(n_e2e):
                submit(i)
            _abi.rts_peel_pipeline_wait(p.h)
            dt = max_over_ranks((time.perf_counter() - t0) / n_e2e)
            line["e2e"] = {"value": world * updates_per_step / dt, "unit": UNIT,
                           "h2d_bytes_per_step": cube_bytes + K * 24,
                           "d2h_bytes_per_step": cube_bytes + K * cad.n_ant * 32 + K * 4,
                           "ms_per_step": dt * 1e3, "steps": n_e2e,
                           "h2d_GBps": h2d_gbs, "d2h_GBps": d2h_gbs,
                           "api": ("rts_peel_pipeline_submit / rts_peel_pipeline_wait: each cadence copied in "
                                   "from pinned host memory, peeled, copied out; copies of one cadence overlap "
                                   "the peel of the other; the timed region holds every submit and the final "
                                   "wait, so the first copy-in and the last copy-out are inside it")}
        finally:
            _abi.rts_host_free(h_in)
            for hb in h_out:
                _abi.rts_host_free(hb)

    if not args.no_extra:
        line.update(extra_legs(args, p, cad, d_vis, d_resid, src, rank, value / world,
                               clk.get("sm_mhz") or 2070.0))

    p.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_profile_case(args):
    """A small case of one extra-leg workload for profiling captures."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1003_5575_gb300 import Peeler
    from synth import config
    if args.profile_case == "integrate":
        c = config(3).with_(n_ant=args.antennas)
        vals = torch.randn((c.n_time, c.n_bl, c.n_chan, 4), dtype=torch.complex64, device="cuda")
        res = integrator_leg(c, vals, lambda: torch.cuda.Event(enable_timing=True), reps=1)
        print(json.dumps({"profile_case": "integrate", "antennas": c.n_ant, "ms": res["ms"]}), flush=True)
        return 0
    if args.profile_case == "grid":
        c = config(3).with_(n_ant=args.antennas)
        vals = torch.randn((c.n_time, c.n_bl, 12, 4), dtype=torch.complex64, device="cuda")
        res = gridder_leg(c, vals, lambda: torch.cuda.Event(enable_timing=True), reps=1)
        print(json.dumps({"profile_case": "grid", "antennas": c.n_ant, "ms_per_12_channels": res["ms_per_12_channels"]}),
              flush=True)
        return 0
    if args.profile_case == "adjoint":
        c = config(5).with_(n_ant=args.antennas)
        p = Peeler(c.uvw(), c.freqs(), n_iter=args.n_iter, precision="mixed", max_sources=c.n_src)
        J = torch.from_numpy(c.jones().astype(np.complex64)).cuda()
        d = p.predict(c.sources(), J)
        s_fit = torch.from_numpy(c.perturbed_sources()).cuda()
        for _ in range(2):
            loss = p.grad(d, J, s_fit)[0]
        summary = {"loss": float(loss.item())}
    else:
        c = config(3).with_(n_ant=args.antennas, n_src=args.sources)
        # one pass per source unless --per-pass 64 (the blocked Taylor schedule)
        p = Peeler(c.uvw(), c.freqs(), n_iter=args.n_iter, precision="mixed", max_sources=c.n_src,
                   sources_per_pass=args.per_pass or 1)
        J = torch.from_numpy(c.jones().astype(np.complex64)).cuda()
        d = p.predict(c.sources(), J)
        for _ in range(2):
            _, _, _, st = p.cadence_taylor(d, c.sources())
        summary = {"status": [int(x) for x in st]}
    torch.cuda.synchronize()
    p.close()
    print(json.dumps({"profile_case": args.profile_case, "antennas": c.n_ant, "channels": c.n_chan,
                      "times": c.n_time, "sources": c.n_src, **summary}), flush=True)
    return 0


def integrator_leg(cad, d_vis, ev, reps=3):
    """Time the integrator on a 16-sample (0.5 s) cadence built from the bench cube: groups of
    16, 8 or 4 samples (8, 4, 2 s) by baseline length (cuts 699 m and 1398 m: at most 0.05 turn
    of fringe drift at the 21.4 deg field edge and 198 MHz over the group)."""
    import numpy as np
    import torch
    from paper_1003_5575_gb300 import Integrator, integration_lengths
    fine = d_vis.repeat_interleave(2, dim=0)                 # [16][n_bl][n_chan][4]
    L = integration_lengths(cad.uvw()[cad.n_time // 2], [699.0, 1398.0], [16, 8, 4])
    ig = Integrator(16, cad.n_chan, L, n_slot=4)
    out = ig.run(fine)
    torch.cuda.synchronize()
    a, b = ev(), ev()
    a.record()
    for _ in range(reps):
        ig.run(fine, out=out)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / reps
    ig.close()
    nbytes = (16 + 4) * cad.n_bl * cad.n_chan * 32
    del fine, out
    torch.cuda.empty_cache()
    peaks = json.load(open(MEASURED_PEAKS)) if os.path.exists(MEASURED_PEAKS) else {}
    hbm = peaks.get("hbm_gbs", 6800.0)
    gbs = nbytes / (ms / 1e3) / 1e9
    return {"workload": f"{cad.n_ant} ant x {cad.n_chan} ch, 16 samples of 0.5 s -> groups of 8/4/2 s "
                        f"({int(np.sum(L == 16))}/{int(np.sum(L == 8))}/{int(np.sum(L == 4))} baselines), 4 slots",
            "ms": ms, "visibilities_per_s": 16 * cad.n_bl * cad.n_chan / (ms / 1e3),
            "roofline": {"bound": "hbm", "kernel": "k_integrate", "achieved": gbs, "peak": hbm, "unit": "GB/s",
                         "frac": gbs / hbm, "traffic": ncu_traffic("k_integrate"),
                         "algorithmic_bytes_per_launch": nbytes}}


def gridder_leg(cad, d_resid, ev, n_pix=1125, r_max=12.0, n_grid_chan=12, fov_deg=21.4, reps=3, bin=24):
    """Time the gridder over n_grid_chan channels of the residual cube."""
    import numpy as np
    import torch
    from paper_1003_5575_gb300 import Gridder
    from synth import baseline_pairs
    r = np.linspace(0.0, 1.0, 1025)
    kb = np.i0(8.0 * np.sqrt(np.clip(1.0 - r * r, 0.0, None)))
    gcf = (kb - kb[-1]) / (kb[0] - kb[-1])                  # Kaiser-Bessel, vanishing at r_max
    pairs = baseline_pairs(cad.n_ant)
    t_mid = cad.n_time // 2
    uvw = cad.uvw()[t_mid]
    duv = uvw[pairs[:, 0]] - uvw[pairs[:, 1]]               # metres
    cell = math.radians(fov_deg)                            # pixels per wavelength
    freqs = cad.freqs()[:n_grid_chan]
    xy, vis, n_in = [], [], 0
    for c, f in enumerate(freqs):
        pix = duv[:, :2] * (f / 299792458.0) * cell + n_pix / 2.0
        n_in += int(np.sum(np.all((pix >= 0) & (pix < n_pix), axis=1)))
        xy.append(torch.from_numpy(pix.astype(np.float32)).cuda())
        vis.append(d_resid[t_mid, :, c, :].contiguous())
    g = Gridder(n_pix, r_max, gcf, bin=bin, n_pol=4, max_vis=cad.n_bl)
    grids = torch.empty((n_grid_chan, 4, n_pix, n_pix), dtype=torch.complex64, device="cuda")
    for c in range(n_grid_chan):
        g.run(xy[c], vis[c], out=grids[c])
    torch.cuda.synchronize()
    a, b = ev(), ev()
    ms_sort = ms_gather = 0.0
    a.record()
    for _ in range(reps):
        for c in range(n_grid_chan):
            g.run(xy[c], vis[c], out=grids[c])
    b.record()
    torch.cuda.synchronize()
    for c in range(n_grid_chan):                            # sort / gather split of one pass
        g.run(xy[c], vis[c], out=grids[c])
        s_ms, g_ms = g.last_ms()
        ms_sort += s_ms
        ms_gather += g_ms
    ms = a.elapsed_time(b) / reps
    g.close()
    flops = n_in * math.pi * r_max * r_max * 16              # 4 complex values x real weight per pair
    peak = fp32_peak_tflops(2070.0)
    return {"workload": f"{n_pix} x {n_pix} pixels, r_max {r_max:g} (24 x 24 convolution function), {bin} x {bin} bins, "
                        f"{n_grid_chan} channels x {cad.n_bl} visibilities (one per baseline, middle time), 4 pol, "
                        f"{fov_deg} deg field",
            "ms_per_12_channels": ms, "ms_sort": ms_sort, "ms_gather": ms_gather,
            "visibilities_per_s": n_grid_chan * cad.n_bl / (ms / 1e3), "visibilities_in_grid": n_in,
            "roofline": {"bound": "alu", "kernel": "k_grid_gather<4>", "achieved": flops / (ms_gather / 1e3) / 1e12,
                         "peak": peak, "unit": "TFLOP/s", "frac": flops / (ms_gather / 1e3) / 1e12 / peak,
                         "algorithmic_flops": flops, "traffic": None,
                         "note": "algorithmic = visibilities in the grid x pi r_max^2 pixels x 16 flop"},
            "paper_tesla_c1060_ms": 590, "paper_note": "the paper's CUDA gridding work time for 12 channels "
                                                      "(Table of work times; another machine: context only)"}


def refine_leg(pa, c5, vis, J_true, ms_adj, ev, n_steps=20):
    """The adjoint-refinement workload at full size: 20 gradient steps of a joint
    Jones + position fit of 300 sources through the autograd Function PeelLoss
    (phasors recomputed in every backward), from positions perturbed by
    N(0, (1 arcmin)^2) and the true Jones matrices, on the noise-free cube of the
    true sky.  Steps are Gauss-Newton scaled: each antenna's Jones matrix moves
    by -gJ / (2 S^2 n_t n_c (n_ant - 1)), halved (its block of the normal matrix
    with J ~ I; all antennas move at once), and (l, m) by -H^-1 g with H the
    position normal matrix of the six-number statistics (rts_peel_offsets,
    alpha = 0) at the start.  Also the forward peel of the same 300 sources."""
    import numpy as np
    import torch
    from paper_1003_5575_gb300 import PeelLoss
    torch.cuda.synchronize()
    torch.cuda.reset_peak_memory_stats()
    base_alloc = torch.cuda.memory_allocated()
    truth = torch.from_numpy(c5.sources()).cuda()
    src = torch.from_numpy(c5.perturbed_sources()).cuda().requires_grad_(True)
    J = J_true.clone().requires_grad_(True)
    S = truth[:, 2]
    scale_J = (1.0 / (2.0 * S * S * c5.n_time * c5.n_chan * (c5.n_ant - 1)) * 0.5).to(torch.float32)
    six, _ = pa.offsets(vis, J.detach(), src.detach(), alpha=0.0)
    Hll, Hlm, Hmm = six[:, 0], six[:, 1], six[:, 2]
    det = Hll * Hmm - Hlm * Hlm
    arcsec = 180.0 / math.pi * 3600.0

    def pos_err():
        d = (src.detach()[:, :2] - truth[:, :2]) * arcsec
        return float(torch.sqrt(torch.mean(d * d)).item())

    err0 = pos_err()
    losses = []
    a, b = ev(), ev()
    a.record()
    for _ in range(n_steps):
        loss = PeelLoss.apply(pa, vis, J, src)
        loss.backward()
        with torch.no_grad():
            losses.append(loss.detach())
            J -= J.grad * scale_J[:, None, None]
            gl, gm = src.grad[:, 0], src.grad[:, 1]
            src[:, 0] -= (Hmm * gl - Hlm * gm) / det
            src[:, 1] -= (Hll * gm - Hlm * gl) / det
        J.grad = None
        src.grad = None
    b.record()
    torch.cuda.synchronize()
    ms_fit = a.elapsed_time(b)
    final = PeelLoss.apply(pa, vis, J.detach(), src.detach())
    # the fit's working set: its cube, what torch allocated for it, the library's
    # adjoint workspace (88 bytes per source and baseline)
    fit_gb = (vis.numel() * vis.element_size() + torch.cuda.max_memory_allocated() - base_alloc
              + 88 * c5.n_src * c5.n_bl) / 1e9
    # the forward peel of the same 300 sources (default blocked schedule), for the
    # adjoint-step / forward-peel ratio
    resid = torch.empty_like(vis)
    pa.cadence(vis, c5.sources(), resid=resid, status=False)
    a, b = ev(), ev()
    a.record()
    pa.cadence(vis, c5.sources(), resid=resid, status=False)
    b.record()
    torch.cuda.synchronize()
    ms_fwd = a.elapsed_time(b)
    del resid
    return {"workload": "512 ant x 768 ch x 8 t, 300 sources: 20 Gauss-Newton-scaled gradient steps of a joint "
                        "Jones + (l, m) fit through PeelLoss (autograd Function), from (l, m) perturbed by "
                        "N(0, 1 arcmin^2) per coordinate and the true Jones matrices, noise-free cube of the true sky",
            "steps": n_steps, "ms_per_step": ms_fit / n_steps,
            "loss_curve": [float(x.item()) for x in losses] + [float(final.item())],
            "position_rms_error_arcsec": {"before": err0, "after": pos_err()},
            "fit_working_set_GB": fit_gb,
            "forward_peel_ms_300_sources": ms_fwd,
            "adjoint_step_over_forward_peel": ms_adj / ms_fwd}


def extra_legs(args, p, cad, d_vis, d_resid, src, rank, mixed_rate, sm_mhz):
    """One-source-per-pass path, gains Taylor-expanded in frequency, FP64-path
    comparison, adjoint step, integrator, gridder, ionospheric offsets, CPU baseline
    (rank 0 at N=1 only)."""
    import numpy as np
    import torch
    from paper_1003_5575_gb300 import Peeler
    from synth import config
    out = {}
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    from paper_1003_5575_gb300 import _abi
    # the one-source-per-pass path (HBM-bound fused subtract + average), 100 sources
    k1 = 100
    p1 = Peeler(cad.uvw(), cad.freqs(), n_iter=args.n_iter, precision="mixed", max_sources=k1,
                sources_per_pass=1)
    d_j1 = torch.empty((k1, cad.n_ant, 4), dtype=torch.complex64, device="cuda")
    p1.cadence(d_vis, src[:k1], resid=d_resid, jones=d_j1, status=False)
    _abi.rts_peel_timing(p1.h, 1)
    a, b = ev(), ev()
    a.record()
    p1.cadence(d_vis, src[:k1], resid=d_resid, jones=d_j1, status=False)
    b.record()
    torch.cuda.synchronize()
    kt1 = _abi.rts_peel_timing_read(p1.h)
    ms_k3, n_k3, _ = kt1["sub_average"]
    k3_gbs = cad.n_vis * BYTES_PER_UPDATE / (ms_k3 / n_k3 / 1e3) / 1e9
    peaks = json.load(open(MEASURED_PEAKS)) if os.path.exists(MEASURED_PEAKS) else {}
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    out["one_source_per_pass"] = {
        "sources": k1, "ms": a.elapsed_time(b), "updates_per_s": k1 * cad.n_vis / (a.elapsed_time(b) / 1e3),
        "roofline": {"bound": "hbm", "kernel": "k_stream_mixed<SUB,ACC>", "achieved": k3_gbs, "peak": hbm_peak,
                     "unit": "GB/s", "frac": k3_gbs / hbm_peak,
                     "traffic": ncu_traffic("k_stream_mixed<true,true>"),
                     "algorithmic_bytes_per_launch": cad.n_vis * BYTES_PER_UPDATE}}
    # gains Taylor-expanded in frequency (Section 3.1), one pass per source, same cube
    _abi.rts_peel_timing(p1.h, 0)
    _abi.rts_peel_timing(p1.h, 1)
    p1.cadence_taylor(d_vis, src[:k1], resid=d_resid, status=False)
    _abi.rts_peel_timing(p1.h, 0)
    _abi.rts_peel_timing(p1.h, 1)
    a, b = ev(), ev()
    a.record()
    _, _, _, st_t = p1.cadence_taylor(d_vis, src[:k1], resid=d_resid, status=True)
    b.record()
    torch.cuda.synchronize()
    ktt = _abi.rts_peel_timing_read(p1.h)
    ms_tp, n_tp, _ = ktt["sub_average"]
    ms_ts, n_ts, _ = ktt["solve"]
    tp_gbs = cad.n_vis * BYTES_PER_UPDATE / (ms_tp / n_tp / 1e3) / 1e9
    out["taylor_gains_one_pass_per_source"] = {
        "workload": "512 ant x 768 ch x 8 t, 100 sources, one pass per source; gains G + x_c H",
        "sources": k1, "ms": a.elapsed_time(b), "updates_per_s": k1 * cad.n_vis / (a.elapsed_time(b) / 1e3),
        "ms_per_pass": ms_tp / n_tp, "ms_per_solve": ms_ts / n_ts,
        "not_converged": int(np.sum(st_t == 1)),
        "roofline": {"bound": "hbm", "kernel": "k_stream_taylor<SUB,ACC>", "achieved": tp_gbs, "peak": hbm_peak,
                     "unit": "GB/s", "frac": tp_gbs / hbm_peak, "traffic": ncu_traffic("k_stream_taylor<true,true>"),
                     "algorithmic_bytes_per_launch": cad.n_vis * BYTES_PER_UPDATE}}
    # the blocked Taylor schedule (21 sources per tcgen05 pass) on the headline
    # handle, all K sources of the cadence
    kt = len(src)
    p.cadence_taylor(d_vis, src[:min(kt, 63)], resid=d_resid, status=False)      # warm-up: three blocks
    torch.cuda.synchronize()
    _abi.rts_peel_timing(p.h, 0)
    _abi.rts_peel_timing(p.h, 1)
    a, b = ev(), ev()
    a.record()
    _, _, _, st_b = p.cadence_taylor(d_vis, src, resid=d_resid, status=True)
    b.record()
    torch.cuda.synchronize()
    ktb = _abi.rts_peel_timing_read(p.h)
    _abi.rts_peel_timing(p.h, 0)
    rel_b = p.rel(kt)
    ms_bp, n_bp, _ = ktb["block_pass"]
    ms_bs, n_bs, _ = ktb["solve"]
    ms_bf, _, _ = ktb["block_fix"]
    tay_flops = 2 * kt * cad.n_vis * 3 * FLOPS_PER_UPDATE          # three model terms and three moments
    tay_tflops = tay_flops / (ms_bp / 1e3) / 1e12
    bf16 = peaks.get("bf16_tflops_sustained") or 1700.0
    tf32_peak = bf16 * 1.1 / 2.25
    ms_b = a.elapsed_time(b)
    # the same cadence with 60 sweeps per source (the statuses settle by then)
    p60 = Peeler(cad.uvw(), cad.freqs(), n_iter=60, precision="mixed", max_sources=kt)
    p60.cadence_taylor(d_vis, src[:min(kt, 63)], resid=d_resid, status=False)
    torch.cuda.synchronize()
    a60, b60 = ev(), ev()
    a60.record()
    _, _, _, st_60 = p60.cadence_taylor(d_vis, src, resid=d_resid, status=True)
    b60.record()
    torch.cuda.synchronize()
    rel_60 = p60.rel(kt)
    p60.close()
    out["taylor_gains"] = {
        "workload": f"512 ant x 768 ch x 8 t, {kt} sources, blocked: 21 sources per pass; gains G + x_c H",
        "sources": kt, "ms": ms_b, "updates_per_s": kt * cad.n_vis / (ms_b / 1e3),
        "passes": n_bp, "ms_per_pass": ms_bp / n_bp, "ms_per_solve": ms_bs / n_bs,
        "ms_corrections_and_models": ms_bf,
        "ms_per_source": ms_b / kt,
        "one_pass_per_source_ms_per_source": out["taylor_gains_one_pass_per_source"]["ms"] / k1,
        "not_converged": int(np.sum(st_b == 1)),
        "last_relative_change": {"min": float(np.min(rel_b)), "median": float(np.median(rel_b)),
                                 "max": float(np.max(rel_b))},
        "not_converged_note": ("the status compares the last sweep's relative change of X = [G H] with 1e-6; "
                               "each sweep is followed by a Newton step along the common slope rotation "
                               "H_p -> H_p + i G_p K, which the Jacobi sweeps alone barely move; the remaining "
                               "rate is the sweeps' own (about 0.65 per sweep), see sweeps_60"),
        "sweeps_60": {"ms": a60.elapsed_time(b60), "not_converged": int(np.sum(st_60 == 1)),
                      "last_relative_change_median": float(np.median(rel_60)),
                      "last_relative_change_max": float(np.max(rel_60))},
        "roofline": {"bound": "tensor", "kernel": "k_block_pass_tc05<SUB,ACC,TAY> (tcgen05.mma kind::tf32)",
                     "achieved": tay_tflops, "peak": tf32_peak, "unit": "TFLOP/s", "frac": tay_tflops / tf32_peak,
                     "traffic": ncu_traffic("k_block_pass_tc05<true,true,true>"),
                     "algorithmic_flops_per_update": 3 * FLOPS_PER_UPDATE,
                     "algorithmic_bytes_per_launch": cad.n_vis * BYTES_PER_UPDATE,
                     "avg_launch_ms": ms_bp / n_bp,
                     "peak_source": (f"MEASURED_PEAKS.json bf16_tflops_sustained {bf16:.0f} x nominal TF32/BF16 "
                                     "ratio 1.1/2.25 (of measured)")}}
    p1.close()
    del d_j1

    # plain FP64 GPU path on the same input, first k64 sources, vs the mixed path on the same sources
    k64 = 4
    d_jm = torch.empty((k64, cad.n_ant, 4), dtype=torch.complex64, device="cuda")
    p.cadence(d_vis, src[:k64], resid=d_resid, jones=d_jm, status=False)
    torch.cuda.synchronize()
    R_mixed_sample = d_resid[:, :64].cpu().numpy()
    J_mixed = d_jm.cpu().numpy()
    p64 = Peeler(cad.uvw(), cad.freqs(), n_iter=args.n_iter, precision="fp64", max_sources=k64)
    d_j64 = torch.empty((k64, cad.n_ant, 4), dtype=torch.complex128, device="cuda")
    v64 = d_vis.to(torch.complex128)
    p64.cadence(v64, src[:1], resid=v64, jones=d_j64[:1], status=False)     # warm (in place)
    v64.copy_(d_vis)
    r64 = v64
    a, b = ev(), ev()
    a.record()
    p64.cadence(v64, src[:k64], resid=r64, jones=d_j64, status=False)
    b.record()
    torch.cuda.synchronize()
    ms_64 = a.elapsed_time(b)
    R64 = r64[:, :64].cpu().numpy()
    J64 = d_j64.cpu().numpy()
    rms = float(torch.sqrt(torch.mean(d_vis.view(torch.float32).double() ** 2)).item())
    rate64 = k64 * cad.n_vis / (ms_64 / 1e3)
    out["fp64_path"] = {
        "sources": k64, "ms_fp64": ms_64, "updates_per_s_fp64": rate64,
        "speedup_mixed_vs_fp64": mixed_rate / rate64,
        "speedup_basis": "updates/s of the timed mixed cadence (1000 sources) over updates/s of the FP64 path "
                         "(one pass per source, so its rate does not depend on the source count)",
        "mixed_vs_fp64_max_resid_err_x_rms": float(np.abs(R_mixed_sample - R64).max() / rms),
        "mixed_vs_fp64_jones_rel": float(max(np.linalg.norm(J_mixed[k] - J64[k]) / np.linalg.norm(J64[k])
                                             for k in range(k64))),
        "note": "same input cube; residual error sampled on the first 64 baselines",
    }
    # FP64 roofline: the complex arithmetic of the subtraction and the average (4 complex
    # multiply-adds each = 64 flop per update) against the measured FP64 FMA rate; the two FP64
    # sincospi per visibility are not counted, so the fraction is a lower bound
    fp64_peak = _abi.rts_fp64_rate()
    fp64_achieved = 64 * rate64 / 1e12
    out["fp64_path"]["roofline"] = {"bound": "alu", "kernel": "k_stream_fp64<SUB,ACC>", "achieved": fp64_achieved,
                                    "peak": fp64_peak, "unit": "TFLOP/s", "frac": fp64_achieved / fp64_peak,
                                    "peak_source": "measured FP64 FMA rate (rts_fp64_rate), not in MEASURED_PEAKS.json",
                                    "algorithmic_flops_per_update": 64, "traffic": None}
    del v64, r64
    p64.close()
    p.close()                      # release the pipeline cubes before the adjoint leg
    torch.cuda.empty_cache()
    torch.cuda.empty_cache()

    # adjoint step at the config-5 shape (300 sources, positions perturbed by 1 arcmin)
    c5 = config(5)
    pa = Peeler(c5.uvw(), c5.freqs(), n_iter=args.n_iter, precision="mixed", max_sources=c5.n_src)
    Jt = torch.from_numpy(c5.jones().astype(np.complex64)).cuda()
    pa.predict(c5.sources(), Jt, out=d_resid)
    s_fit = torch.from_numpy(c5.perturbed_sources()).cuda()
    J_fit = Jt.clone()
    for _ in range(2):
        pa.grad(d_resid, J_fit, s_fit)
    torch.cuda.synchronize()
    steps = max(args.steps, 3)
    a, b = ev(), ev()
    a.record()
    for _ in range(steps):
        loss, gJ, gs = pa.grad(d_resid, J_fit, s_fit)
    b.record()
    torch.cuda.synchronize()
    ms_adj = a.elapsed_time(b) / steps
    # the FP64 adjoint on a bounded number of sources, per source x visibility
    k_adj64 = 8
    pa64 = Peeler(c5.uvw(), c5.freqs(), n_iter=args.n_iter, precision="fp64", max_sources=k_adj64)
    v64 = d_resid.to(torch.complex128)
    J64 = Jt[:k_adj64].to(torch.complex128)
    pa64.grad(v64, J64, s_fit[:k_adj64])
    a, b = ev(), ev()
    a.record()
    pa64.grad(v64, J64, s_fit[:k_adj64])
    b.record()
    torch.cuda.synchronize()
    ms_adj64 = a.elapsed_time(b)
    per_upd_mixed = ms_adj / (c5.n_src * c5.n_vis)
    per_upd_64 = ms_adj64 / (k_adj64 * c5.n_vis)
    adj_tflops = ADJ_FLOPS_PER_UPDATE * c5.n_src * c5.n_vis / (ms_adj / 1e3) / 1e12
    adj_peak = fp32_peak_tflops(sm_mhz)
    out["adjoint"] = {
        "workload": "512 ant x 768 ch x 8 t, 300 sources, positions perturbed N(0, 1 arcmin^2); loss + dL/d(J,l,m,S)",
        "ms_per_step": ms_adj, "loss": float(loss.item()),
        "roofline": {"bound": "alu", "kernel": "k_grad_sweep_fac<false> (factorised phasor tables; + reductions, in the step time)",
                     "achieved": adj_tflops, "peak": adj_peak, "unit": "TFLOP/s", "frac": adj_tflops / adj_peak,
                     "algorithmic_flops_per_update": ADJ_FLOPS_PER_UPDATE,
                     "traffic": ncu_traffic("k_grad_sweep_fac<false>"),
                     "algorithmic_bytes_per_launch": c5.n_vis * 32 + c5.n_src * c5.n_bl * (64 + 24)},
        "fp64_ms_per_step_at_300_sources_extrapolated": per_upd_64 * c5.n_src * c5.n_vis,
        "fp64_sources_timed": k_adj64, "speedup_mixed_vs_fp64": per_upd_64 / per_upd_mixed,
    }
    del v64
    pa64.close()
    out["refinement"] = refine_leg(pa, c5, d_resid, Jt, ms_adj, ev)

    # visibility integrator (Section 3's first stage) on one 8 s cadence of 0.5 s samples
    out["integrator"] = integrator_leg(cad, d_vis, ev)

    # gridder (Section 6) at the paper's benchmark shape: 1125 x 1125 pixels, a 24 x 24 pixel
    # convolution function (r_max = 12) in 24 x 24 bins, 12 channels of one visibility per
    # baseline (130 816) at the cadence's middle time, 4 polarisations, 21.4 deg field of view
    out["gridder"] = gridder_leg(cad, d_resid, ev)

    # ionospheric position offsets at the same shape (Section 3, 3.1): refraction law
    # alpha = 2, the adjoint sweep with frequency-law weights + FP64 normal equations + 2x2 solves
    nu_ref = float(np.mean(c5.freqs()))
    pa.offsets(d_resid, J_fit, s_fit, alpha=2.0, nu_ref_hz=nu_ref)
    torch.cuda.synchronize()
    a, b = ev(), ev()
    a.record()
    for _ in range(steps):
        six, off = pa.offsets(d_resid, J_fit, s_fit, alpha=2.0, nu_ref_hz=nu_ref)
    b.record()
    torch.cuda.synchronize()
    ms_off = a.elapsed_time(b) / steps
    off_arcsec = off.abs().max(dim=1).values.cpu().numpy() * 180 / math.pi * 3600
    out["offsets"] = {
        "workload": "512 ant x 768 ch x 8 t, 300 sources, positions perturbed N(0, 1 arcmin^2); six numbers "
                    "per source + (dl, dm) under the refraction law (nu_ref/nu)^2",
        "ms_per_step": ms_off, "updates_per_s": c5.n_src * c5.n_vis / (ms_off / 1e3),
        "nu_ref_hz": nu_ref, "median_max_abs_offset_arcsec": float(np.median(off_arcsec)),
    }
    pa.close()

    # CPU oracle baseline on a bounded sample (rank 0, N = 1)
    if rank == 0 and int(os.environ.get("WORLD_SIZE", "1")) == 1:
        import oracle
        oc, V = oracle_sample(n_chan=64, n_src=10)          # about 10 s of 16-core work
        val, dt = time_oracle(oc, V)
        out["cpu_baseline"] = {"value": val, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                               "sample": (f"512 ant, 8 t, first {oc.n_chan} of 768 channels, {oc.n_src} "
                                          f"sources, FP64 C oracle, {dt:.1f} s")}
        # one core on a smaller sample of the same workload
        n_all = oracle.num_threads()
        oracle.set_num_threads(1)
        oc1, V1 = oracle_sample(n_chan=8, n_src=2)
        val1, dt1 = time_oracle(oc1, V1)
        oracle.set_num_threads(n_all)
        out["cpu_baseline"]["single_core"] = {
            "value": val1, "unit": UNIT, "cores": 1,
            "sample": f"512 ant, 8 t, first 8 of 768 channels, 2 sources, {dt1:.1f} s"}
    return out


if __name__ == "__main__":
    sys.exit(main())
