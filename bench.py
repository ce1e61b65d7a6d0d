#!/usr/bin/env python3
"""Throughput benchmark of the mixed-radix gate-apply engine.

Workload (one GPU): 14 qutrits (3^14 = 4,782,969 amplitudes), a seeded
500-gate circuit (40% Haar single-qutrit, 30% F_3, 30% controlled-X_3 on random
pairs and control levels), per-gate kernels.  One step = reset the register to
|0...0>, run the circuit, write the FP64 probabilities of all amplitudes to a
device buffer.  The headline runs the complex64 (FP32) path; the complex128
(FP64) path is measured in the same run for comparison.

Prints one JSON line (see the repository's design notes for every key).
  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank runs an independent replica on its own GPU; rank 0
prints the line with the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "gates/s & amplitude updates/s vs HBM roofline, fused FP32 vs plain FP64, fid>=1-1e-6"
UNIT = "gates/s"
WORKLOAD = "14 qutrits (3^14 = 4,782,969 amplitudes), 500-gate random circuit (40% Haar-1, 30% F_3, 30% CX_3), per-gate kernels"
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-sample-gates", type=int, default=0, help="gates in the CPU-baseline sample (0: auto)")
    ap.add_argument("--c2-ququarts", type=int, default=12,
                    help="ququarts of the c2 register (12: the full 2^32-amplitude case; fewer for profiling)")
    ap.add_argument("--c3-circuits", type=int, default=256,
                    help="circuits of the c3 batch (256: the full workload; fewer for profiling)")
    ap.add_argument("--workload", default="c2", choices=["c1", "c2", "c3", "c4", "strides", "blocks"],
                    help="c2 (default): 8 qubits + 12 ququarts (2^32 amplitudes), Haar layer + d=4 QFT + Toffoli "
                         "ladder, fused complex64 plan (learned cost model) vs the FP64 per-gate path; "
                         "c1: 14 qutrits, 500 gates, per-gate kernels; "
                         "c3: 256 independent circuits (6-12 qudits, dims 2..5, 200 gates each) in one persistent "
                         "graph-captured launch vs one graph-captured plan per circuit; "
                         "c4: 18 qutrits + 4 qubits (6.2e9 amplitudes), 1,000-gate circuit, fusion planned with "
                         "the learned cost model vs the greedy and exhaustive analytic plans and per-gate kernels; "
                         "strides: per-gate kernels on every target position of the c4 register (per-stride table); "
                         "blocks: fused blocks of D 6..64 on the tensor cores and on the CUDA-core dense kernels")
    ap.add_argument("--blocks-small", action="store_true",
                    help="blocks workload on a 2^26-amplitude register (8 qubits + 9 ququarts) only: the profiling size")
    ap.add_argument("--strides-register", default="c4", choices=["c4", "c2"],
                    help="register of the per-stride table (c4: 3^18 * 2^4; c2: 2^8 * 4^12)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Replicas:
    """One process per GPU, each running an independent replica of the
    workload (the path has no exchange step): a process group only for the
    barrier around the timed region and for the maximum of the ranks' times.
    NCCL with a device, gloo without (the CPU tests)."""

    def __init__(self, world: int, device=None):
        self.world = world
        self.dist = None
        self.device = device
        if world > 1:
            import torch.distributed as dist
            if device is not None and device.type == "cuda":
                dist.init_process_group("nccl", device_id=device)
            else:
                dist.init_process_group("gloo")
            self.dist = dist

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()
        if self.device is not None and self.device.type == "cuda":
            import torch
            torch.cuda.synchronize(self.device)

    def max(self, x: float) -> float:
        """Maximum over ranks (the slowest replica's time)."""
        if self.dist is None:
            return float(x)
        import torch
        on_gpu = self.device is not None and self.device.type == "cuda"
        t = torch.tensor([float(x)], dtype=torch.float64, device=self.device if on_gpu else "cpu")
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.dist is not None:
            self.dist.barrier()
            self.dist.destroy_process_group()
            self.dist = None


def aggregate_rate(units_per_rank: float, world: int, max_ms: float) -> float:
    """Whole-job throughput: the units every rank processed over the slowest
    rank's time."""
    return world * units_per_rank / (max_ms * 1e-3)


# ------------------------------------------------------------------ helpers

def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        import tempfile
        self.path = os.path.join(tempfile.gettempdir(), f"qudit_bench_clocks_{os.getpid()}_{gpu_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


KERNEL_SOURCES = ("qd_apply.cuh", "qd_common.cuh", "qd_plan.h")
BATCH_SOURCES = ("qd_batch.cu", "qd_batch.h", "qd_common.cuh")
TC_SOURCES = ("qd_tc.cu", "qd_tc.h", "qd_common.cuh")


def kernel_source_sha(files=KERNEL_SOURCES):
    """Hash of a kernel's sources (a committed ncu figure is used only while
    the sources it was taken on are unchanged)."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2211_07918_gb300", "csrc")
    for f in files:
        with open(os.path.join(d, f), "rb") as fh:
            h.update(f.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def _profile_fields(kname: str, files):
    pdir = os.path.join(ROOT, "profiles")
    if not os.path.isdir(pdir):
        return None
    sha = kernel_source_sha(files)
    for f in sorted(os.listdir(pdir)):
        if not f.endswith(".md"):
            continue
        with open(os.path.join(pdir, f)) as fh:
            txt = fh.read()
        fields = dict(re.findall(r"^(traffic_[a-z_]+|source_sha):\s*(\S+)", txt, re.M))
        if fields.get("traffic_kernel_class") == kname and fields.get("source_sha") == sha:
            return fields
    return None


def profiled_traffic(kname: str):
    """dram bytes per launch for kernel class ``kname`` from a committed ncu
    summary in profiles/, or None if absent or taken on different sources."""
    f = _profile_fields(kname, KERNEL_SOURCES)
    return float(f["traffic_bytes_per_launch"]) if f and "traffic_bytes_per_launch" in f else None


def profiled_traffic_scaled(kname: str, alg_bytes: float, files=BATCH_SOURCES):
    """dram bytes of a full launch from a capture of a smaller case of the
    same kernel: the captured dram bytes per algorithmic byte times this
    launch's algorithmic bytes (the kernel's traffic grows with the work)."""
    f = _profile_fields(kname, files)
    return float(f["traffic_per_alg_byte"]) * alg_bytes if f and "traffic_per_alg_byte" in f else None


# ------------------------------------------------------------- CPU baseline

def cpu_sample(dims, gates, ngates_sample):
    """Time the FP64 C oracle (index loop, OpenMP over all host cores) on the
    first ``ngates_sample`` gates of the circuit on the full register."""
    from oracle import fast as qf
    from oracle import qudit_oracle as qo
    qf.build()
    psi = qo.basis_state(dims)
    sub = gates[:ngates_sample]
    t0 = time.perf_counter()
    for g in sub:
        qf.apply(psi, dims, g)
    dt = time.perf_counter() - t0
    return len(sub) / dt, qf.max_threads(), dt


def cpu_baseline_obj(dims, gates, ngates, min_seconds=10.0, max_reps=20):
    """Repeat the sample until it has run ``min_seconds`` of CPU work."""
    n = ngates or len(gates)
    done, secs, cores = 0, 0.0, 1
    while secs < min_seconds and done < max_reps * n:
        rate, cores, dt = cpu_sample(dims, gates, n)
        done += n
        secs += dt
    return {"value": done / secs, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{done // n} x the first {n} of {len(gates)} gates on the full 3^14 register, "
                      f"FP64 C index loop (OpenMP), {secs:.1f} s"}


# --------------------------------------------------------------- reference

def run_reference(args, rank, world):
    """The reference arm: the FP64 C oracle on the host cores, on this bench's
    workload (the 2^32-amplitude QFT + Toffoli-ladder circuit), each step a
    bounded sample: the sample gates applied to a same-shaped 2^24-amplitude
    register, the amplitude-update rate scaled to gates/s of the full
    register.  Under torchrun only rank 0 runs it."""
    if rank != 0:
        return 0
    from oracle import fast as qf
    from oracle import qudit_oracle as qo
    from paper_2211_07918_gb300 import workloads as wl
    dims, gates = wl.circuit_c2()
    small = [2] * 8 + [4] * 8
    sub = c2_cpu_sample(gates, len(small))
    qf.build()
    psi = qo.basis_state(small)
    for _ in range(args.warmup):
        qf.apply(psi, small, sub[0])
    secs = 0.0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        for g in sub:
            qf.apply(psi, small, g)
        secs += time.perf_counter() - t0
    upd = args.steps * len(sub) * int(np.prod(small)) / secs
    value = upd / int(np.prod(dims))
    sample = (f"per step the {len(sub)} sample gates of the circuit (every gate acting below qudit 16, evenly "
              f"spread) on a 2^8 * 4^8 register (2^24 amplitudes), FP64 C index loop (OpenMP); "
              f"{upd:.3g} amplitude updates/s extrapolated to 2^32")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOAD_C2 + "; each step times a bounded sample of the circuit",
                       "amplitudes": int(np.prod(dims)), "gates": len(gates), "sample_gates_per_step": len(sub)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": qf.max_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def c2_cpu_sample(gates, nq_small, count=10):
    """``count`` gates spread evenly over the circuit among those acting only
    on qudits below nq_small (so that they apply to the smaller register)."""
    ok = [g for g in gates if max(tuple(g.targets) + tuple(g.controls or ())) < nq_small]
    idx = np.linspace(0, len(ok) - 1, min(count, len(ok))).round().astype(int)
    return [ok[i] for i in idx]


# -------------------------------------------------------------------- ours

WORKLOAD_C2 = ("8 qubits + 12 ququarts (2^8 * 4^12 = 2^32 amplitudes, 34.4 GB complex64), Haar layer (20) + "
               "d=4 QFT on the ququarts (12 F_4 + 66 controlled phases) + 7 qutrit-style Toffoli rungs (21 CX), "
               "fused complex64 plan chosen with the learned cost model (tcgen05 exact-BF16-slice blocks, "
               "CUDA-core blocks, diagonal-run tables) vs per-gate complex128")


def cpu_baseline_c2(dims, gates, min_seconds=10.0, prefix=10):
    """The FP64 C oracle (index loop, OpenMP over the host cores) on
    ``prefix`` gates spread over the circuit, on a register of the same shape
    with 8 ququarts instead of 12 (2^24 amplitudes; the full state would need
    68.7 GB in complex128), repeated until ``min_seconds`` have run.  The
    measured amplitude-update rate is scaled to gates/s of the full 2^32
    register."""
    from oracle import fast as qf
    from oracle import qudit_oracle as qo
    qf.build()
    small = [2] * 8 + [4] * 8
    sub = c2_cpu_sample(gates, len(small), prefix)
    psi = qo.basis_state(small)
    secs, done = 0.0, 0
    while secs < min_seconds:
        t0 = time.perf_counter()
        for g in sub:
            qf.apply(psi, small, g)
        secs += time.perf_counter() - t0
        done += len(sub)
    n_small = int(np.prod(small))
    upd_per_s = done * n_small / secs
    return {"value": upd_per_s / int(np.prod(dims)), "unit": UNIT, "cores": qf.max_threads(), "kind": "oracle",
            "sample": f"{done // len(sub)} x {len(sub)} gates spread over the circuit on a 2^8 * 4^8 register "
                      f"(same shape, 2^24 amplitudes), FP64 C index loop (OpenMP), {secs:.1f} s; "
                      f"{upd_per_s:.3g} amplitude updates/s extrapolated to the 2^32 register",
            "amp_updates_per_s": upd_per_s, "extrapolated": True}


def c1_summary(L, stream, steps: int):
    """The 14-qutrit per-gate workload (4.78e6 amplitudes, L2-resident) in
    complex64 and complex128, graph replay, for the compare block."""
    import torch
    from paper_2211_07918_gb300 import workloads as wl
    dims, gates = wl.circuit_c1()
    out = {}
    for name, prec in (("complex64", L.QD_C64), ("complex128", L.QD_C128)):
        reg = L.qd_create(dims, None, prec, 0, 0, stream.cuda_stream)
        plan = L.qd_plan_create(reg, gates, L.QD_PLAN_NONE)
        for _ in range(3):
            L.qd_reset(reg)
            L.qd_plan_run(plan)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for a, b in ev:
            a.record(stream)
            L.qd_reset(reg)
            L.qd_plan_run(plan)
            b.record(stream)
        stream.synchronize()
        ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
        out[name] = {"ms_per_step": ms, "gates_per_s": len(gates) / (ms * 1e-3)}
        L.qd_plan_destroy(plan)
        L.qd_destroy(reg)
    out["workload"] = "14 qutrits (3^14 amplitudes, L2-resident), 500 gates, per-gate kernels, reset + circuit"
    return out


def run_c2(args, rank, world, local):
    """Precision and fusion at scale (the metric's configuration): the fused
    complex64 path, planned with the learned cost model, against the plain
    per-gate complex128 path on the same GPU; fidelity through qd_overlap on
    the device; end to end through the C ABI with host buffers."""
    import torch

    from paper_2211_07918_gb300 import costmodel as cm
    from paper_2211_07918_gb300 import qudit as L
    from paper_2211_07918_gb300 import workloads as wl
    from paper_2211_07918_gb300.build import build

    build()
    L.load()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dims, gates = wl.circuit_c2(n_ququarts=args.c2_ququarts)
    N = int(np.prod(dims))
    ngates = len(gates)
    full = args.c2_ququarts == 12
    stream = torch.cuda.Stream(device=dev)
    rep = Replicas(world, dev)

    def timed(reg, plan, steps, warmup):
        """Per-step CUDA events on the register's stream: reset + plan."""
        for _ in range(warmup):
            L.qd_reset(reg)
            L.qd_plan_run(plan)
        stream.synchronize()
        rep.barrier()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for a, b in ev:
            a.record(stream)
            L.qd_reset(reg)
            L.qd_plan_run(plan)
            b.record(stream)
        stream.synchronize()
        rep.barrier()
        return rep.max(float(np.mean([a.elapsed_time(b) for a, b in ev])))

    reg64 = L.qd_create(dims, None, L.QD_C64, 0, 0, stream.cuda_stream)
    model = cm.load()
    L.qd_set_cost_model(reg64, model)
    plans, res = {}, {}
    for name, kind in (("learned", L.QD_PLAN_LEARNED), ("exhaustive_analytic", L.QD_PLAN_EXHAUSTIVE),
                       ("greedy_analytic", L.QD_PLAN_GREEDY), ("per_gate", L.QD_PLAN_NONE)):
        t0 = time.perf_counter()
        plans[name] = L.qd_plan_create(reg64, gates, kind)
        res[name] = {"plan_s": time.perf_counter() - t0}
    sampler = ClockSampler(local)
    sampler.start()
    ms = timed(reg64, plans["learned"], args.steps, args.warmup)
    clocks = sampler.stop()
    res["learned"].update({"ms_per_step": ms, "gates_per_s": ngates / (ms * 1e-3)})
    for name in ("exhaustive_analytic", "greedy_analytic", "per_gate"):
        t = timed(reg64, plans[name], max(2, args.steps // 4), 2)
        res[name].update({"ms_per_step": t, "gates_per_s": ngates / (t * 1e-3)})
    for name, p_ in plans.items():
        info = L.qd_plan_info(p_)
        res[name].update({"launches": info["launches"], "blocks": info["blocks"]})
    # per-kernel times of the headline plan (per-launch events, direct launches)
    L.qd_plan_profile(plans["learned"], True)
    kern, launch_list = {}, []
    for _ in range(2):
        L.qd_reset(reg64)
        L.qd_plan_run(plans["learned"])
        ms_l, ab_l, kc_l = L.qd_plan_timings(plans["learned"])
    for t, b_, c in zip(ms_l, ab_l, kc_l):
        k = kern.setdefault(L.kclass_name(int(c)), [0.0, 0.0, 0])
        k[0] += float(t)
        k[1] += float(b_)
        k[2] += 1
        launch_list.append([L.kclass_name(int(c)), round(float(t), 3), round(float(b_) / (float(t) * 1e6), 1)])
    L.qd_plan_profile(plans["learned"], False)
    alg_bytes_step = float(np.sum(ab_l))
    # fused complex64 state vs the plain per-gate complex128 state
    L.qd_reset(reg64)
    L.qd_plan_run(plans["learned"])
    reg128 = L.qd_create(dims, None, L.QD_C128, 0, 0, stream.cuda_stream)
    plan128 = L.qd_plan_create(reg128, gates, L.QD_PLAN_NONE)
    ms128 = timed(reg128, plan128, max(1, args.steps // 10), 1)
    L.qd_reset(reg128)
    L.qd_plan_run(plan128)
    ov = L.qd_overlap(reg128, reg64)
    n64, n128 = L.qd_norm(reg64), L.qd_norm(reg128)
    L.qd_plan_destroy(plan128)
    L.qd_destroy(reg128)
    for name in ("exhaustive_analytic", "greedy_analytic", "per_gate"):
        L.qd_plan_destroy(plans[name])

    # e2e: a user's call sequence with host buffers, every step: the initial
    # state in from pinned host memory, the planned circuit, all FP64
    # probabilities out to pinned host memory
    e2e = None
    if full or args.c2_ququarts >= 6:
        host_in = torch.zeros(N, dtype=torch.complex64).pin_memory()
        host_in[0] = 1.0
        host_out = torch.empty(N, dtype=torch.float64).pin_memory()
        hin, hout = host_in.numpy(), host_out.numpy()

        def e2e_step():
            L.qd_set_amplitudes(reg64, hin)
            L.qd_plan_run(plans["learned"])
            L.qd_probabilities(reg64, hout)
        e2e_step()
        rep.barrier()
        e2e_steps = max(2, args.steps // 8)
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            e2e_step()
        stream.synchronize()
        e2e_s = rep.max((time.perf_counter() - t0) / e2e_steps)
        e2e = {"value": world * ngates / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(N * 8),
               "d2h_bytes_per_step": int(N * 8), "ms_per_step": e2e_s * 1e3,
               "path": "qd_set_amplitudes(pinned host, complex64) + qd_plan_run + qd_probabilities(pinned host, FP64)",
               "p_sum_last_step": float(np.sum(hout, dtype=np.float64))}
        del host_in, host_out
    L.qd_plan_destroy(plans["learned"])
    L.qd_destroy(reg64)
    L.qd_model_destroy(model)

    c1 = c1_summary(L, stream, max(5, args.steps // 2)) if full else None
    kname, kdata = max(kern.items(), key=lambda kv: kv[1][0])
    peak, peak_src = measured_peaks()
    achieved = kdata[1] / (kdata[0] * 1e-3) / 1e9
    value = aggregate_rate(ngates, world, ms)
    tc_files = TC_SOURCES if kname.startswith("tensor_block") else KERNEL_SOURCES
    traffic = profiled_traffic_scaled(kname, kdata[1] / kdata[2], tc_files)
    cpu = cpu_baseline_c2(dims, gates) if (rank == 0 and world == 1 and full) else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD_C2 if full else f"c2 shape with {args.c2_ququarts} ququarts (profiling size)",
                   "amplitudes": N, "gates": ngates, "precision": "complex64 (FP32 arithmetic)",
                   "plan": "fusion planned with the learned cost model",
                   "l2": "inputs (34.4 GB) larger than L2; no flush needed",
                   "step": "reset to |0...0> + fused circuit (graph replay)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "amp_updates_per_s": value * N,
        "compare": {"fused_learned": res["learned"], "fused_exhaustive_analytic": res["exhaustive_analytic"],
                    "fused_greedy_analytic": res["greedy_analytic"], "per_gate_complex64": res["per_gate"],
                    "per_gate_complex128": {"ms_per_step": ms128, "gates_per_s": ngates / (ms128 * 1e-3)},
                    "fused_fp32_over_plain_fp64": ms128 / ms,
                    "fused_over_per_gate_complex64": res["per_gate"]["ms_per_step"] / ms,
                    "fidelity_fused_c64_vs_c128": abs(ov) ** 2, "norm2_c64": n64, "norm2_c128": n128,
                    "c1_per_gate_14_qutrits": c1},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "kernel": kname, "peak_source": peak_src,
                     "share_of_gate_time": kdata[0] / sum(v[0] for v in kern.values()), "launches": kdata[2],
                     "alg_bytes_per_step": alg_bytes_step,
                     "step_alg_GB_s": alg_bytes_step / (ms * 1e-3) / 1e9,
                     "note": "per-launch CUDA events over profiled direct launches; the step's algorithmic "
                             "bytes over the graph-timed step stay below the copy peak"},
        "kernels": {k: {"ms": v[0], "launches": v[2], "GB_s": v[1] / (v[0] * 1e-3) / 1e9} for k, v in kern.items()},
        "launch_list": launch_list,
        "clocks": clocks,
        "e2e": e2e,
        "gpu_launches": int(args.steps * (res["learned"]["launches"] + 1)),
        "cpu_baseline": cpu,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    rep.close()
    return 0


WORKLOAD_C3 = ("256 independent random circuits, 6-12 qudits each with dims uniform in {2,3,4,5} "
               "(2.44e8 amplitudes in total), 200 gates each (X, Z, F_d, CX_d, Haar-1, Haar-2), complex64, "
               "one persistent graph-captured launch, FP64 probabilities of every register")


def cpu_baseline_c3(circuits, min_seconds=10.0):
    """The C oracle on whole circuits of the batch, in batch order, until
    ``min_seconds`` have run; scaled to the whole batch by amplitude updates."""
    from oracle import fast as qf
    qf.build()
    work_all = sum(int(np.prod(d)) * len(g) for d, g in circuits)
    gates_all = sum(len(g) for _, g in circuits)
    secs, work, ncirc = 0.0, 0, 0
    for d, g in circuits:
        t0 = time.perf_counter()
        qf.run_circuit(d, g)
        secs += time.perf_counter() - t0
        work += int(np.prod(d)) * len(g)
        ncirc += 1
        if secs >= min_seconds:
            break
    est = secs * work_all / work
    return {"value": gates_all / est, "unit": UNIT, "cores": qf.max_threads(), "kind": "oracle",
            "sample": f"the first {ncirc} of {len(circuits)} circuits, whole, FP64 C index loop (OpenMP), "
                      f"{secs:.1f} s, scaled to the batch by amplitude updates ({work:.3g} of {work_all:.3g})"}


def run_c3(args, rank, world, local):
    """Batched execution: all 256 circuits in one persistent kernel launch
    (graph replay), against one captured plan per circuit."""
    import torch

    from paper_2211_07918_gb300 import qudit as L
    from paper_2211_07918_gb300 import workloads as wl
    from paper_2211_07918_gb300.build import build

    build()
    L.load()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    circuits = wl.batch_c3()[: args.c3_circuits]
    regs = [d for d, _ in circuits]
    Ns = [int(np.prod(d)) for d in regs]
    total = sum(Ns)
    ngates = sum(len(g) for _, g in circuits)
    amp_updates = sum(n * len(g) for n, (_, g) in zip(Ns, circuits))
    stream = torch.cuda.Stream(device=dev)
    rep = Replicas(world, dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    b = L.qd_batch_create(regs, stream.cuda_stream)
    for c, (_, g) in enumerate(circuits):
        L.qd_batch_set_circuit(b, c, g)
    tuned = L.qd_batch_autotune(b, 1)  # launch shape, chosen before the timed region

    def timed(run, steps, warmup):
        for _ in range(warmup):
            run()
        stream.synchronize()
        rep.barrier()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for i in range(steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            ev[i][0].record(stream)
            run()
            ev[i][1].record(stream)
        stream.synchronize()
        rep.barrier()
        return [rep.max(float(np.mean([a.elapsed_time(b_) for a, b_ in ev])))]

    sampler = ClockSampler(local)
    sampler.start()
    ms = timed(lambda: L.qd_batch_run(b), args.steps, args.warmup)
    clocks = sampler.stop()
    info = L.qd_batch_info(b, with_error=True)
    # persistent-kernel time with events around it (direct launches)
    L.qd_batch_profile(b, True)
    kms = []
    for _ in range(max(3, args.steps // 4)):
        with torch.cuda.stream(stream):
            flush.zero_()
        L.qd_batch_run(b)
        kms.append(L.qd_batch_timings(b)[0])
    alg_bytes = L.qd_batch_timings(b, with_time=False)[1]
    L.qd_batch_profile(b, False)
    err = L.qd_batch_info(b, with_error=True)["device_error"]
    # every 17th register's probabilities sum to 1 (parity itself is in the tests)
    sums = [float(np.sum(L.qd_batch_probabilities(b, c, Ns[c]))) for c in range(0, len(circuits), 17)]

    # e2e: a user's call sequence with host buffers: upload every circuit's
    # gates, run, read every register's FP64 probabilities to pinned host memory
    host = torch.empty(max(Ns), dtype=torch.float64).pin_memory().numpy()
    d2h = 8 * total
    h2d = sum(L.GateArray(g).matrix_bytes() for _, g in circuits)

    def e2e_step():
        for c, (_, g) in enumerate(circuits):
            L.qd_batch_set_circuit(b, c, g)
        L.qd_batch_run(b)
        for c in range(len(circuits)):
            L.qd_batch_probabilities(b, c, Ns[c], host)
    e2e_step()
    stream.synchronize()
    e2e_steps = max(2, args.steps // 4)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    stream.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    L.qd_batch_destroy(b)

    # comparison: one register and one captured plan per circuit, run in turn
    per = []
    for (d, g) in circuits:
        r = L.qd_create(d, None, L.QD_C64, 0, 0, stream.cuda_stream)
        per.append((r, L.qd_plan_create(r, g, L.QD_PLAN_NONE)))
    probs = torch.empty(max(Ns), dtype=torch.float64, device=dev)

    def per_circuit():
        for r, p in per:
            L.qd_reset(r)
            L.qd_plan_run(p)
            L.qd_probabilities(r, where=L.QD_DEVICE, dev_ptr=probs.data_ptr())
    ms_per = timed(per_circuit, max(2, args.steps // 2), 2)
    for r, p in per:
        L.qd_plan_destroy(p)
        L.qd_destroy(r)

    ms_step = float(np.mean(ms))
    value = aggregate_rate(ngates, world, ms_step)
    peak, peak_src = measured_peaks()
    kmean = float(np.mean(kms))
    achieved = alg_bytes / (kmean * 1e-3) / 1e9
    cpu = cpu_baseline_c3(circuits) if rank == 0 and world == 1 else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD_C3 if len(circuits) == 256 else
                   f"the first {len(circuits)} circuits of the c3 batch (profiling size)",
                   "circuits": len(circuits), "amplitudes": total, "gates": ngates,
                   "precision": "complex64", "l2": "flushed (256 MiB write) before every timed step; "
                   "states (1.95 GB) larger than L2",
                   "step": "reset all registers + all circuits + FP64 probabilities of every register"},
        "amp_updates_per_s": world * amp_updates / (ms_step * 1e-3),
        "batch": {"items": info["items"], "device_error": max(info["device_error"], err), "autotuned": tuned,
                  "prob_sums_sampled": sums, "kernel_ms": kmean, "kernel_share": kmean / ms_step},
        "compare": {"per_circuit_plans_ms_per_step": float(np.mean(ms_per)),
                    "per_circuit_plans_gates_per_s": world * ngates / (float(np.mean(ms_per)) * 1e-3),
                    "batch_over_per_circuit": float(np.mean(ms_per)) / ms_step},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": profiled_traffic_scaled("k_batch", alg_bytes), "kernel": "k_batch",
                     "peak_source": peak_src,
                     "alg_bytes_per_launch": alg_bytes,
                     "note": "large circuits run in groups whose states stay in L2; achieved can exceed HBM peak"},
        "clocks": clocks,
        "e2e": {"value": world * ngates / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_s * 1e3,
                "path": "qd_batch_set_circuit x256 (host gates) + qd_batch_run + qd_batch_probabilities x256 (host)"},
        "gpu_launches": int(args.steps * info["launches"]),
        "cpu_baseline": cpu,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    rep.close()
    return 0


WORKLOAD_C4 = ("18 qutrits + 4 qubits (3^18 * 2^4 = 6,198,727,824 amplitudes, 49.6 GB complex64), "
               "1,000-gate random circuit (X, Z, F_d, CX_d, Haar-1, Haar-2), fusion planned with the learned "
               "MLP cost model (weights trained on GB300 launch timings)")


def run_c4(args, rank, world, local):
    """Learned fusion planning at scale: the plan chosen with the learned
    cost model against the greedy and exhaustive plans of the analytic model
    and against per-gate kernels, on the same complex64 register; fidelity of
    the learned plan's state against the per-gate state through qd_overlap."""
    import torch

    from paper_2211_07918_gb300 import costmodel as cm
    from paper_2211_07918_gb300 import qudit as L
    from paper_2211_07918_gb300 import workloads as wl
    from paper_2211_07918_gb300.build import build

    build()
    L.load()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dims, gates = wl.circuit_c4()
    N = int(np.prod(dims))
    ngates = len(gates)
    stream = torch.cuda.Stream(device=dev)
    rep = Replicas(world, dev)
    model = cm.load()
    reg = L.qd_create(dims, None, L.QD_C64, 0, 0, stream.cuda_stream)
    L.qd_set_cost_model(reg, model)

    def timed(plan, steps, warmup):
        for _ in range(warmup):
            L.qd_reset(reg)
            L.qd_plan_run(plan)
        stream.synchronize()
        rep.barrier()
        ts = []
        for _ in range(steps):
            L.qd_reset(reg)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            L.qd_plan_run(plan)
            b.record(stream)
            stream.synchronize()
            ts.append(a.elapsed_time(b))
        rep.barrier()
        return [rep.max(float(np.mean(ts)))]

    res, plans = {}, {}
    for name, kind in (("learned", L.QD_PLAN_LEARNED), ("greedy", L.QD_PLAN_GREEDY),
                       ("exhaustive_analytic", L.QD_PLAN_EXHAUSTIVE), ("per_gate", L.QD_PLAN_NONE)):
        t0 = time.perf_counter()
        plans[name] = L.qd_plan_create(reg, gates, kind)
        res[name] = {"plan_s": time.perf_counter() - t0}
    sampler = ClockSampler(local)
    sampler.start()
    for name in plans:
        steps = args.steps if name == "learned" else max(1, args.steps // 2)
        ts = timed(plans[name], steps, 1)
        info = L.qd_plan_info(plans[name])
        res[name].update({"ms_per_step": float(np.mean(ts)), "gates_per_s": ngates / (float(np.mean(ts)) * 1e-3),
                          "launches": info["launches"], "blocks": info["blocks"]})
    clocks = sampler.stop()
    # per-kernel times of the learned plan (per-launch events)
    L.qd_plan_profile(plans["learned"], True)
    L.qd_reset(reg)
    L.qd_plan_run(plans["learned"])
    ms, ab, kc = L.qd_plan_timings(plans["learned"])
    kern = {}
    for t, b_, c in zip(ms, ab, kc):
        k = kern.setdefault(L.kclass_name(int(c)), [0.0, 0.0, 0])
        k[0] += float(t)
        k[1] += float(b_)
        k[2] += 1
    # fidelity: learned plan (fused) vs per-gate kernels, both complex64
    L.qd_reset(reg)
    L.qd_plan_run(plans["learned"])
    ref = L.qd_create(dims, None, L.QD_C64, 0, 0, stream.cuda_stream)
    plan_ref = L.qd_plan_create(ref, gates, L.QD_PLAN_NONE)
    L.qd_plan_run(plan_ref)
    ov = L.qd_overlap(ref, reg)
    n_fused, n_ref = L.qd_norm(reg), L.qd_norm(ref)
    for p_ in plans.values():
        L.qd_plan_destroy(p_)
    L.qd_plan_destroy(plan_ref)
    L.qd_destroy(ref)
    L.qd_destroy(reg)
    L.qd_model_destroy(model)
    kname, kdata = max(kern.items(), key=lambda kv: kv[1][0])
    peak, peak_src = measured_peaks()
    achieved = kdata[1] / (kdata[0] * 1e-3) / 1e9
    value = aggregate_rate(ngates, world, res["learned"]["ms_per_step"])
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": 1,
        "ms_per_step": res["learned"]["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD_C4, "amplitudes": N, "gates": ngates, "precision": "complex64",
                   "l2": "inputs (49.6 GB) larger than L2", "step": "reset + planned circuit"},
        "amp_updates_per_s": value * N,
        "compare": {**{k: v for k, v in res.items()},
                    "learned_over_greedy": res["greedy"]["ms_per_step"] / res["learned"]["ms_per_step"],
                    "learned_over_per_gate": res["per_gate"]["ms_per_step"] / res["learned"]["ms_per_step"],
                    "fidelity_learned_vs_per_gate_c64": abs(ov) ** 2, "norm2_learned": n_fused, "norm2_per_gate": n_ref},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None, "kernel": kname, "peak_source": peak_src,
                     "share_of_gate_time": kdata[0] / sum(v[0] for v in kern.values()), "launches": kdata[2]},
        "kernels": {k: {"ms": v[0], "launches": v[2], "GB_s": v[1] / (v[0] * 1e-3) / 1e9} for k, v in kern.items()},
        "clocks": clocks,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    rep.close()
    return 0

def run_strides(args, rank, world, local):
    """Per-gate kernels, one target position at a time, on an HBM-resident
    register: a Haar single-qudit gate (dense), X_{+1} (permutation), Z
    (diagonal), a controlled X_{+1} whose control is the next qudit up (or
    down, for the top qudit), and a Haar two-qudit gate on (q, q+1).  Each
    launch is timed with CUDA events (median of the repetitions) and reported
    as algorithmic GB/s and as a fraction of the measured copy peak."""
    import torch

    from paper_2211_07918_gb300 import qudit as L
    from paper_2211_07918_gb300 import workloads as wl
    from paper_2211_07918_gb300.build import build

    build()
    L.load()
    torch.cuda.set_device(local)
    dims = [3] * 18 + [2] * 4 if args.strides_register == "c4" else [2] * 8 + [4] * 12
    n = len(dims)
    N = int(np.prod(dims))
    stream = torch.cuda.Stream(device=torch.device("cuda", local))
    reg = L.qd_create(dims, None, L.QD_C64, 0, 0, stream.cuda_stream)
    peak, peak_src = measured_peaks()
    rng = np.random.default_rng(11)
    reps = max(3, args.steps)
    rows = []
    sampler = ClockSampler(local)
    sampler.start()
    for q in range(n):
        c = q + 1 if q + 1 < n else q - 1
        cases = [("dense", wl.Gate("U", (q,), matrix=wl.haar_unitary(dims[q], rng))),
                 ("perm", wl.Gate("X", (q,), param=1)),
                 ("diag", wl.Gate("Z", (q,), param=1)),
                 ("ctrl_perm", wl.Gate("X", (q,), (c,), (dims[c] - 1,), 1)),
                 ("dense2", wl.Gate("U", (q, c), matrix=wl.haar_unitary(dims[q] * dims[c], rng)))]
        row = {"q": q, "d": dims[q], "stride": int(np.prod(dims[:q])), "control": c}
        for name, g in cases:
            plan = L.qd_plan_create(reg, [g], L.QD_PLAN_NONE)
            L.qd_plan_profile(plan, True)
            ts, ab, kc = [], 0.0, 0
            for _ in range(reps + 1):
                L.qd_plan_run(plan)
                ms, b_, k_ = L.qd_plan_timings(plan)
                ts.append(float(ms[0]))
                ab, kc = float(b_[0]), int(k_[0])
            L.qd_plan_destroy(plan)
            t = float(np.median(ts[1:]))
            gbs = ab / (t * 1e-3) / 1e9
            row[name] = {"kernel": L.kclass_name(kc), "us": t * 1e3, "GB_s": gbs, "frac": gbs / peak}
        rows.append(row)
    clocks = sampler.stop()
    L.qd_destroy(reg)
    line = {"metric": "per-gate kernel bandwidth by target stride", "unit": "GB/s", "register": dims,
            "amplitudes": N, "precision": "complex64", "peak": peak, "peak_source": peak_src,
            "repetitions": reps, "rows": rows, "clocks": clocks}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0

def run_blocks(args, rank, world, local):
    """Fused dense blocks (two Haar gates whose union spans 2-3 qudits) on the
    2^32 and 6.2e9-amplitude registers, each timed on the tensor-core kernel
    (QD_TUNE_TC_MIN_D = 9) and, for D <= 32, on the CUDA-core dense kernel
    (QD_TUNE_TC_MIN_D = 65): CUDA-event time per launch (median), algorithmic
    GB/s and fraction of the measured copy peak."""
    import torch

    from paper_2211_07918_gb300 import qudit as L
    from paper_2211_07918_gb300 import workloads as wl
    from paper_2211_07918_gb300.build import build

    build()
    L.load()
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream(device=torch.device("cuda", local))
    peak, peak_src = measured_peaks()
    rng = np.random.default_rng(12)
    reps = max(3, args.steps)
    cases = {
        "c2": ([2] * 8 + [4] * 12, [(6, 7, 8), (5, 6, 7), (8, 9), (18, 19), (7, 8, 9), (8, 9, 10), (12, 13, 14),
                                     (17, 18, 19)]),
        "c4": ([3] * 18 + [2] * 4, [(0, 1), (8, 9), (17, 18), (19, 20, 21), (16, 17, 18), (17, 18, 19), (0, 1, 2),
                                     (8, 9, 10), (15, 16, 17)]),
    }
    if args.blocks_small:
        cases = {"c2_small": ([2] * 8 + [4] * 9, [(8, 9, 10), (6, 7, 8)])}
    out = {}
    sampler = ClockSampler(local)
    sampler.start()
    for name, (dims, sets) in cases.items():
        reg = L.qd_create(dims, None, L.QD_C64, 0, 0, stream.cuda_stream)
        rows = []
        for qs in sets:
            if len(qs) == 2:
                gates = [wl.Gate("U", (qs[0],), matrix=wl.haar_unitary(dims[qs[0]], rng)),
                         wl.Gate("U", (qs[1],), matrix=wl.haar_unitary(dims[qs[1]], rng))]
            else:
                a, b, c = qs
                gates = [wl.Gate("U", (a, b), matrix=wl.haar_unitary(dims[a] * dims[b], rng)),
                         wl.Gate("U", (b, c), matrix=wl.haar_unitary(dims[b] * dims[c], rng))]
            D = int(np.prod([dims[q] for q in qs]))
            row = {"qudits": list(qs), "D": D, "lowest_stride": int(np.prod(dims[:min(qs)]))}
            for route, tc in (("tensor", 9), ("cuda_core", 65)):
                if route == "cuda_core" and D > 32:
                    continue
                L.qd_set_tuning(reg, L.QD_TUNE_TC_MIN_D, tc)
                plan = L.qd_plan_create_segmented(reg, gates, [(0, len(gates) - 1)])
                L.qd_plan_profile(plan, True)
                ts, ab, kc = [], 0.0, 0
                for _ in range(reps + 1):
                    L.qd_plan_run(plan)
                    ms, b_, k_ = L.qd_plan_timings(plan)
                    ts.append(float(ms[0]))
                    ab, kc = float(b_[0]), int(k_[0])
                err = L.qd_sync(reg)
                L.qd_plan_destroy(plan)
                t = float(np.median(ts[1:]))
                gbs = ab / (t * 1e-3) / 1e9
                row[route] = {"kernel": L.kclass_name(kc), "ms": t, "GB_s": gbs, "frac": gbs / peak,
                              "device_error": err}
            rows.append(row)
        L.qd_destroy(reg)
        out[name] = {"register": dims, "amplitudes": int(np.prod(dims)), "rows": rows}
    clocks = sampler.stop()
    line = {"metric": "fused block bandwidth, tensor cores vs CUDA cores", "unit": "GB/s", "peak": peak,
            "peak_source": peak_src, "repetitions": reps, "precision": "complex64", "registers": out,
            "clocks": clocks}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_ours(args, rank, world, local):
    import torch

    from paper_2211_07918_gb300 import qudit as L
    from paper_2211_07918_gb300 import workloads as wl
    from paper_2211_07918_gb300.build import build

    build()
    L.load()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    rep = Replicas(world, dev)
    barrier = rep.barrier

    dims, gates = wl.circuit_c1()
    N = int(np.prod(dims))
    ngates = len(gates)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    probs = torch.empty(N, dtype=torch.float64, device=dev)

    def measure(prec, steps, warmup, profile_steps, plan_kind=L.QD_PLAN_NONE):
        """K timed steps with the plan replayed as a CUDA graph (the headline),
        then ``profile_steps`` steps with per-launch events (kernel times)."""
        reg = L.qd_create(dims, None, prec, 0, 0, stream.cuda_stream)
        plan = L.qd_plan_create(reg, gates, plan_kind)
        launches = L.qd_plan_info(plan)["launches"]

        def step():
            L.qd_reset(reg)
            L.qd_plan_run(plan)
            L.qd_probabilities(reg, where=L.QD_DEVICE, dev_ptr=probs.data_ptr())

        for _ in range(warmup):
            step()
        barrier()
        stream.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for i in range(steps):
            with torch.cuda.stream(stream):
                flush.zero_()  # L2 flush outside the timed interval
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
        stream.synchronize()
        barrier()
        per_step = [a.elapsed_time(b) for a, b in ev]
        kern = {}
        if profile_steps:
            L.qd_plan_profile(plan, True)
            for i in range(profile_steps):
                with torch.cuda.stream(stream):
                    flush.zero_()
                L.qd_reset(reg)
                L.qd_plan_run(plan)
                ms, ab, kc = L.qd_plan_timings(plan)
                for t, b, c in zip(ms, ab, kc):
                    k = kern.setdefault(int(c), [0.0, 0.0, 0])
                    k[0] += float(t)
                    k[1] += float(b)
                    k[2] += 1
            kern["_steps"] = profile_steps
        L.qd_plan_destroy(plan)
        L.qd_destroy(reg)
        return per_step, kern, launches

    sampler = ClockSampler(local)
    sampler.start()
    t_wall = time.perf_counter()
    ms64, kern64, launches = measure(L.QD_C64, args.steps, args.warmup, max(3, args.steps // 4))
    wall = time.perf_counter() - t_wall
    clocks = sampler.stop()
    ms128, _, _ = measure(L.QD_C128, max(3, args.steps // 4), args.warmup, 0)
    fused = {}
    for name, kind in (("greedy", L.QD_PLAN_GREEDY), ("exhaustive", L.QD_PLAN_EXHAUSTIVE)):
        msf, _, nlaunch = measure(L.QD_C64, max(3, args.steps // 2), args.warmup, 0, kind)
        fused[name] = {"gates_per_s": world * ngates / (float(np.mean(msf)) * 1e-3),
                       "ms_per_step": float(np.mean(msf)), "launches": nlaunch}
    prof_steps = kern64.pop("_steps")

    total_ms = rep.max(float(sum(ms64)))
    ms_step = total_ms / args.steps
    value = aggregate_rate(ngates, world, ms_step)
    ms_step128 = float(np.mean(ms128))

    # dominant kernel class of the c64 path, measured with per-launch events
    kname, kdata = None, None
    for c, v in kern64.items():
        if kdata is None or v[0] > kdata[0]:
            kname, kdata = L.kclass_name(c), v
    peak, peak_src = measured_peaks()
    achieved = (kdata[1] / (kdata[0] * 1e-3)) / 1e9 if kdata else None
    total_kernel_ms = sum(v[0] for v in kern64.values())
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None,
                "traffic": profiled_traffic(kname),
                "kernel": kname, "peak_source": peak_src,
                "share_of_gate_time": kdata[0] / total_kernel_ms if kdata else None,
                "launches": kdata[2] if kdata else 0,
                "note": "state (38 MB c64) is L2-resident across the gates of a step; achieved can exceed HBM peak"}
    all_bytes = sum(v[1] for v in kern64.values()) / prof_steps
    roofline["profiled_gate_ms_per_step"] = total_kernel_ms / prof_steps

    # e2e: host buffers through the public API: every step copies the initial
    # state in from pinned host memory, replays the prepared circuit and reads
    # all FP64 probabilities back to pinned host memory
    host_in = torch.zeros(N, dtype=torch.complex64).pin_memory()
    host_in[0] = 1.0
    host_out = torch.empty(N, dtype=torch.float64).pin_memory()
    hin = host_in.numpy()
    hout = host_out.numpy()
    reg = L.qd_create(dims, None, L.QD_C64, 0, 0, stream.cuda_stream)
    plan = L.qd_plan_create(reg, gates, L.QD_PLAN_NONE)
    for _ in range(2):
        L.qd_set_amplitudes(reg, hin)
        L.qd_plan_run(plan)
        L.qd_probabilities(reg, hout)
    e2e_steps = max(3, args.steps // 4)
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        L.qd_set_amplitudes(reg, hin)
        L.qd_plan_run(plan)
        L.qd_probabilities(reg, hout)
    stream.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    L.qd_plan_destroy(plan)
    L.qd_destroy(reg)
    e2e = {"value": world * ngates / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(N * 8),
           "d2h_bytes_per_step": int(N * 8), "ms_per_step": e2e_s * 1e3,
           "path": "qd_set_amplitudes(host) + qd_plan_run + qd_probabilities(host)"}

    # fidelity of the timed c64 path against the c128 path on this GPU
    regA = L.qd_create(dims, None, L.QD_C64, 0, 0, stream.cuda_stream)
    regB = L.qd_create(dims, None, L.QD_C128, 0, 0, stream.cuda_stream)
    L.qd_run_circuit(regA, gates)
    L.qd_run_circuit(regB, gates)
    a = L.qd_get_amplitudes(regA).astype(np.complex128)
    b = L.qd_get_amplitudes(regB)
    L.qd_destroy(regA)
    L.qd_destroy(regB)
    fid = float(abs(np.vdot(b, a)) ** 2)
    maxabs = float(np.max(np.abs(a - b)))

    cpu = None
    if rank == 0 and world == 1:
        cpu = cpu_baseline_obj(dims, gates, args.cpu_sample_gates)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "amplitudes": N, "gates": ngates, "precision": "complex64",
                       "step": "reset + 500 gates + FP64 probabilities to device",
                       "l2": "flushed (256 MiB write) before every timed step; inputs smaller than L2",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "amp_updates_per_s": value * N,
            "alg_bytes_per_step": all_bytes,
            "compare": {"complex128_gates_per_s": world * ngates / (ms_step128 * 1e-3),
                        "complex128_ms_per_step": ms_step128,
                        "c64_over_c128": ms_step128 / ms_step,
                        "c64_fidelity_vs_c128": fid, "c64_maxabs_vs_c128": maxabs,
                        "fused_complex64": fused,
                        "fused_greedy_over_c128": fused["greedy"]["gates_per_s"] / (world * ngates / (ms_step128 * 1e-3))},
            "roofline": roofline,
            "clocks": clocks,
            "e2e": e2e,
            "gpu_launches": int(args.steps * (launches + 2)),
            "cpu_baseline": cpu,
            "wall_s_timed_c64": wall,
        }
        print(json.dumps(line), flush=True)
    rep.close()
    return 0


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload == "c1":
        return run_ours(args, rank, world, local)
    if args.workload == "c3":
        return run_c3(args, rank, world, local)
    if args.workload == "c4":
        return run_c4(args, rank, world, local)
    if args.workload == "strides":
        return run_strides(args, rank, world, local)
    if args.workload == "blocks":
        return run_blocks(args, rank, world, local)
    return run_c2(args, rank, world, local)


if __name__ == "__main__":
    sys.exit(main())
