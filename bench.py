"""Throughput benchmark of the time step on GB300.

Workload: the precision configuration, 4096 x 4096 periodic, 512 seeded
droplets (radii uniform in [8, 40], W = 4, rho_A/rho_B = 100, sigma = 1e-3,
M = 0.05, tau_f = tau_g = 0.8).  A "step" is one full time step of both
populations over the whole grid (one kernel launch).  MLUPS = cells x
steps / seconds.

Our arm (default): FP32 form timed with CUDA events on the simulation's
stream; the populations (2.4 GB per time level) exceed L2, so no flush is
needed between steps.  Also reported: the 16-bit storage forms and the FP64
form with their errors against the FP64 path, the roofline of the step
kernel, an end-to-end number through the C ABI with host buffers, and the
FP64 CPU oracle on a bounded sample (cpu_baseline).

--impl reference: the reference arm is the FP64 CPU oracle timed on the
host cores on a bounded sample of the same workload.

Multi-GPU (torchrun): each rank advances its own replica of the domain
(weak scaling, no collective on the data path); the step time is the
maximum over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# populations read once and written once per cell-update; the deviation
# forms also move their two 16-bit reference words (P, A) each way
BYTES_PER_CELL = {"f64": 288, "f32": 144, "f16s": 76, "bf16s": 76, "f16d": 84, "bf16d": 84}
WORKLOAD = "precision-4096x4096-512-droplets-rho100"
CPU_SAMPLE_N, CPU_SAMPLE_DROPS, CPU_SAMPLE_STEPS = 1024, 32, 20


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# Sources that define the step kernels (k_strip, k_step, k_strip_batch) and
# their launch, with the batch work list and the slab launches.
STEP_SOURCES = ("lbm_internal.h", "lbm_kernels.cuh", "lbm_strip.cuh", "lbm_strip_lag.cuh",
                "lbm_ops.cuh", "lbm_f64.cu", "lbm_f32.cu", "lbm_f16.cu", "lbm_f16d.cu",
                "lbm_batch.cu", "lbm_slabs.cu")


# Sources of the D3Q19 step kernels and their launch.
STEP3_SOURCES = ("lbm3_kernels.cuh", "lbm3.cu")


def _kernel_hash(sources=STEP_SOURCES) -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1507_03521_gb300", "csrc")
    for name in sources:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def _traffic(dtype: str, sources=STEP_SOURCES, full_size=True):
    """DRAM bytes per launch of the step kernel from a committed ncu
    summary, if it was taken on the current kernel sources and the run is
    on the workload it was taken on (full_size)."""
    if not full_size:
        return None
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        e = d.get(dtype)
        if e and e.get("kernel_hash") == _kernel_hash(sources):
            return float(e["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


def _alu(dtype: str):
    """Per cell-update arithmetic of the step kernel (ncu counts) from the
    committed record, if it was taken on the current kernel sources."""
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_alu.json")) as f:
            d = json.load(f)
        if d.get("kernel_hash") == _kernel_hash():
            return d.get(dtype)
    except Exception:
        pass
    return None


def alu_peaks(lbm):
    """Measured FMA operations per second of this GPU (lbm_alu_peak), in G/s."""
    try:
        return {k: round(lbm.alu_peak(k) / 1e9, 1) for k in ("f32", "f32x2", "f64")}
    except Exception as e:  # reported, not fatal: the peaks are context
        return {"error": str(e)}


class Clocks:
    """nvidia-smi sampling during the timed region: a reader thread stamps
    each sample; entering waits until sampling is live, and only samples
    stamped inside the region count."""

    def __init__(self, index: int, interval_ms: int = 20):
        self.index = index
        self.interval_ms = interval_ms
        self.proc = None
        self.lines = []  # (time, line)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line))

    def __enter__(self):
        import threading
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                 "--format=csv,noheader,nounits", "-lms", str(self.interval_ms)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.reader = threading.Thread(target=self._read, daemon=True)
            self.reader.start()
            t_end = time.perf_counter() + 3.0
            while not self.lines and time.perf_counter() < t_end and self.proc.poll() is None:
                time.sleep(0.005)
        except Exception:
            self.proc = None
        self.t0 = time.perf_counter()
        return self

    def __exit__(self, *a):
        self.t1 = time.perf_counter()
        self.out = ""
        if self.proc is not None:
            time.sleep(self.interval_ms / 1000.0)  # the sample in flight at the end
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
                self.reader.join(timeout=5)
            except Exception:
                self.proc.kill()
            end = self.t1 + self.interval_ms / 1000.0
            self.out = "".join(l for t, l in self.lines if self.t0 <= t <= end)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(x: float, dist, device) -> float:
    """The job's time is the slowest rank's: all-reduce MAX (a no-op
    without a process group)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def time_steps(sim, steps, warmup):
    """Per-launch CUDA-event timing of `steps` steps on the sim's stream."""
    import torch
    sim.step(warmup)
    st = sim.stream
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    torch.cuda.synchronize()
    ev[0].record(st)
    for i in range(steps):
        sim.step(1)
        ev[i + 1].record(st)
    torch.cuda.synchronize()
    per = [ev[i].elapsed_time(ev[i + 1]) for i in range(steps)]
    return ev[0].elapsed_time(ev[-1]), per


def _oracle_omp():
    """The oracle's OpenMP build over this process's cores: (lib path,
    threads), or (None, 1) when the toolchain has no OpenMP."""
    import oracle
    try:
        path = oracle.build_omp()
    except Exception:
        return None, 1
    return path, oracle.set_threads(len(os.sched_getaffinity(0)), path)


def cpu_baseline():
    """FP64 oracle on a bounded sample of the workload: 1024 x 1024 with 32
    droplets (the workload's droplet density and parameters).  The OpenMP
    build of the same source over all host cores (bit-identical to the
    serial build) gives the value; the serial build, single thread, is
    reported beside it."""
    import oracle
    from paper_1507_03521_gb300 import workloads as W
    p, phi = W.precision(n=CPU_SAMPLE_N, n_drops=CPU_SAMPLE_DROPS, seed=1507035)
    cells = CPU_SAMPLE_N * CPU_SAMPLE_N

    def run(lib, steps):
        o = oracle.Oracle(p, lib=lib)
        o.init_phi(phi)
        t0 = time.perf_counter()
        o.step(steps)
        dt = time.perf_counter() - t0
        o.close()
        return cells * steps / dt / 1e6, dt

    single, dts = run(None, CPU_SAMPLE_STEPS)
    sample = f"{CPU_SAMPLE_N}x{CPU_SAMPLE_N}, {CPU_SAMPLE_DROPS} droplets, same parameters"
    out = {"value": round(single, 4), "unit": "MLUPS", "cores": 1, "kind": "oracle",
           "sample": f"{sample}, {CPU_SAMPLE_STEPS} steps, {dts:.1f} s, FP64, serial build"}
    lib, threads = _oracle_omp()
    if lib is not None and threads > 1:
        steps = CPU_SAMPLE_STEPS * 12
        par, dtp = run(lib, steps)
        out = {"value": round(par, 4), "unit": "MLUPS", "cores": threads, "kind": "oracle",
               "sample": f"{sample}, {steps} steps, {dtp:.1f} s, FP64, OpenMP build "
                         f"({threads} threads, bit-identical to the serial build)",
               "single_thread": {"value": round(single, 4), "cores": 1,
                                 "sample": f"{CPU_SAMPLE_STEPS} steps, {dts:.1f} s"}}
    return out


def run_reference(args, rank, world):
    """Reference arm: the FP64 oracle as it stands, one oracle step per
    benchmark step, on a 512 x 512 sample of the workload (8 droplets: the
    workload's droplet density, same parameters)."""
    if rank != 0:
        return 0
    import oracle
    from paper_1507_03521_gb300 import workloads as W
    n, nd = 512, 8
    p, phi = W.precision(n=n, n_drops=nd, seed=1507035)
    lib, threads = _oracle_omp()
    o = oracle.Oracle(p, lib=lib)
    o.init_phi(phi)
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    v = round(n * n * args.steps / dt / 1e6, 4)
    how = f"OpenMP build, {threads} threads" if lib is not None else "serial build, 1 thread"
    sample = f"{n}x{n}, {nd} droplets, same parameters, FP64 {how}, {args.steps} steps"
    line = {"impl": "reference", "metric": "MLUPS", "value": v, "unit": "MLUPS",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dt / max(args.steps, 1) * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def measure_batch(lbm, W, args, peak, dist):
    """Batched workload: 1024 periodic domains, sides uniform in
    {64, 96, ..., 512}, droplet or layer, rho ratio log-uniform in [1, 100],
    sigma U[1e-4, 1e-2], M U[0.01, 0.2]; FP32, one persistent launch of
    the 128-column strip kernel per step over every (domain, strip,
    segment) item, replayed from a CUDA graph, segment height autotuned."""
    import torch
    nd = args.batch_domains
    doms = W.batch_domains(nd, seed=1507036)
    b = lbm.Batch([p for p, _ in doms], "f32", graph=True)
    phis = [phi for _, phi in doms]
    b.init_phi(phis)
    seg, _ = b.autotune(steps=3)
    b.init_phi(phis)
    b.step(args.warmup)
    st = b.stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    e0.record(st)
    b.step(args.steps)
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    ms = max_over_ranks(ms, dist, "cuda")
    cells = b.cells
    world = dist.get_world_size() if dist is not None else 1
    gbs = BYTES_PER_CELL["f32"] * cells / (ms / args.steps * 1e-3) / 1e9
    wide, narrow = b.work_items()
    b.close()
    return {"workload": f"batch-{nd}-domains-64to512", "domains": nd, "cells": cells,
            "mlups": round(cells * args.steps * world / (ms * 1e-3) / 1e6, 2),
            "ms_per_step": round(ms / args.steps, 5), "hbm_gbs": round(gbs, 1),
            "frac": round(gbs / peak, 4), "seg_h": seg, "graph": True,
            "launches_per_step": 1, "items_per_step": [wide, narrow],
            "kernel": "k_strip_batch<float, 128 columns> (one launch per step over all items)",
            "traffic": _traffic("batch_f32") if nd == 1024 else None, "bytes_alg": BYTES_PER_CELL["f32"] * cells}


def measure_slabs(lbm, p, phi, args, mlups_single, dist, n_slabs=4):
    """The same FP32 workload as the headline, decomposed into n_slabs
    y-slabs stepped separately with device-to-device ghost exchange (the
    domain decomposition of the step, run on this one GPU): the cost of
    the exchange against the whole-domain step."""
    import torch
    sim = lbm.Sim(p, "f32")
    sim.init_phi(phi)
    s0, _ = sim.get_state()
    sim.close()
    sl = lbm.Slabs(p, "f32", n_slabs=n_slabs)
    sl.scatter(s0, 0)
    sl.step(args.warmup)
    st = sl.stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    e0.record(st)
    sl.step(args.steps)
    e1.record(st)
    torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1), dist, "cuda")
    world = dist.get_world_size() if dist is not None else 1
    cells = p["nx"] * p["ny"]
    mlups = cells * args.steps * world / (ms * 1e-3) / 1e6
    # bytes the exchange moves per step (read once, written once): per slab
    # edge 12 crossing slot-rows and 2 x 18 slots x 3 halo rows, 4 B a value
    exch = n_slabs * (12 + 2 * 18 * 3) * p["nx"] * 4 * 2
    sl.close()
    return {"n_slabs": n_slabs, "mlups": round(mlups, 2), "ms_per_step": round(ms / args.steps, 5),
            "vs_whole_domain": round(mlups / mlups_single, 4),
            "launches_per_step": n_slabs + 2, "exchange_bytes_per_step": exch,
            "slab_kernel_traffic": _traffic("slab_f32", full_size=args.n == 4096)}


def measure_lagged(lbm, p, phi, args, peak, mlups_sync, dist):
    """The lagged-grad-p variant (grad p in G_i from the previous step's
    pressure; not the paper's scheme) on the same FP32 workload: its speed
    against the synchronous step, its roofline (144 B of populations plus
    4 B of stored pressure read and 4 B written per cell), and how far it
    drifts from the synchronous step over the run (max-abs phi, u, p)."""
    import torch
    q = dict(p, gradp_lag=1)
    sim = lbm.Sim(q, "f32")
    sim.init_phi(phi)
    if dist is not None:
        torch.cuda.synchronize()
        dist.barrier()
    total, per = time_steps(sim, args.steps, args.warmup)
    total = max_over_ranks(total, dist, "cuda")
    world = dist.get_world_size() if dist is not None else 1
    cells = p["nx"] * p["ny"]
    mlups = cells * args.steps * world / (total * 1e-3) / 1e6
    bpc = BYTES_PER_CELL["f32"] + 8
    gbs = bpc * cells / (statistics.mean(per) * 1e-3) / 1e9
    lag_fields = sim.fields(("phi", "ux", "uy", "p"))
    sim.close()
    ref = lbm.Sim(p, "f32")
    ref.init_phi(phi)
    ref.step(args.steps + args.warmup)
    sync_fields = ref.fields(("phi", "ux", "uy", "p"))
    ref.close()
    diff = {k: float((lag_fields[k].double() - sync_fields[k].double()).abs().max().item())
            for k in lag_fields}
    return {"mlups": round(mlups, 2), "ms_per_step": round(total / args.steps, 5),
            "vs_synchronous": round(mlups / mlups_sync, 4), "bytes_per_cell": bpc,
            "hbm_gbs": round(gbs, 1), "frac": round(gbs / peak, 4),
            "traffic": _traffic("lag_f32", full_size=args.n == 4096), "kernel": "k_strip_lag_tma<float> (interior strips' g and f rows by TMA tensor tiles)",
            "max_abs_diff_vs_synchronous": diff, "steps_for_diff": args.steps + args.warmup}


def measure_3d(lbm, W, args, peak, dist):
    """The D3Q19 step on the 3-D analogue of the precision workload: 256^3
    periodic, 64 spherical droplets (the same volume fraction at --n3),
    rho ratio 100, FP32; four launches per step.  Algorithmic bytes: 19 + 19
    FP32 populations read and written, 304 B per cell."""
    import torch
    n3 = args.n3
    drops = max(1, round(64 * (n3 / 256) ** 3))
    p, phi, nz = W.precision3d(n=n3, n_drops=drops)
    sim = lbm.Sim3(p, nz, "f32")
    sim.init_phi(phi)
    sim.step(args.warmup)
    st = sim.stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    e0.record(st)
    sim.step(args.steps)
    e1.record(st)
    torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1), dist, "cuda")
    world = dist.get_world_size() if dist is not None else 1
    cells = p["nx"] * p["ny"] * nz
    mlups = cells * args.steps * world / (ms * 1e-3) / 1e6
    gbs = 304 * cells / (ms / args.steps * 1e-3) / 1e9
    m0 = sim.mass()
    sim.close()
    return {"workload": f"precision3d-{n3}^3-{drops}-droplets-rho100", "dtype": "f32",
            "mlups": round(mlups, 2), "ms_per_step": round(ms / args.steps, 5),
            "bytes_per_cell": 304, "hbm_gbs": round(gbs, 1), "frac": round(gbs / peak, 4),
            "launches_per_step": 4, "traffic_per_step": _traffic("d3q19_f32", STEP3_SOURCES) if n3 == 256 else None,
            "finite": bool(np.isfinite(m0[0]))}


def measure_adjoint(W, peak):
    """Adjoint workload: droplet in shear, 512 x 512, R = 64, walls at
    +-0.01, rho ratio 10, FP32, 4000 steps, checkpoints every 200 steps;
    loss = sum (phi_T - phi_target)^2 with phi_target from a run at
    (1.05 M, 0.95 sigma).  Times the forward (with checkpoints) and the
    backward (recompute + hand-written adjoint + initial-state adjoint)."""
    import torch
    from paper_1507_03521_gb300 import lbm
    from paper_1507_03521_gb300.adjoint import rollout_loss
    steps, K = 4000, 200
    p, phi = W.shear_droplet(512, 64.0)
    s = lbm.Sim(dict(p, M=1.05 * p["M"], sigma=0.95 * p["sigma"]), "f32")
    s.init_phi(phi)
    s.step(steps)
    target = s.fields(("phi",))["phi"].double().cpu()
    s.close()
    ph = torch.from_numpy(phi).clone().requires_grad_(True)
    M = torch.tensor(p["M"], dtype=torch.float64, requires_grad=True)
    sg = torch.tensor(p["sigma"], dtype=torch.float64, requires_grad=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    loss = rollout_loss(ph, M, sg, p, steps, target, K=K, dtype="f32")
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    loss.backward()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    cells = 512 * 512
    return {"workload": "shear-droplet-512x512-4000steps", "dtype": "f32", "checkpoint_every": K,
            "loss": loss.item(), "dL_dM": M.grad.item(), "dL_dsigma": sg.grad.item(),
            "dL_dphi0_norm": float(ph.grad.norm()),
            "forward_s": round(t1 - t0, 4), "backward_s": round(t2 - t1, 4),
            "backward_mlups": round(cells * steps / (t2 - t1) / 1e6, 2),
            # 216 B per reverse cell-update: lambda_{t+1} read and lambda_t
            # written (144 B) and the recomputed state read once (72 B); the
            # 512^2 working set sits in L2, so latency, not HBM, bounds it
            "bytes_per_cell": 216,
            "hbm_gbs": round(216 * cells * steps / (t2 - t1) / 1e9, 1),
            "frac": round(216 * cells * steps / (t2 - t1) / 1e9 / peak, 4),
            "bound": "latency (L2-resident working set)",
            "note": "wall-clock incl. host loop; backward = recompute + adjoint steps"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=4096, help="grid side (default: the workload's)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the f16s/bf16s/f64 forms")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched workload")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint workload")
    ap.add_argument("--no-slabs", action="store_true", help="skip the y-slab decomposition")
    ap.add_argument("--no-lagged", action="store_true", help="skip the lagged-grad-p variant")
    ap.add_argument("--no-3d", action="store_true", help="skip the D3Q19 workload")
    ap.add_argument("--n3", type=int, default=256, help="side of the D3Q19 workload")
    ap.add_argument("--batch-domains", type=int, default=1024,
                    help="domains of the batched workload (the first n of its 1024; smaller for ncu captures)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_1507_03521_gb300 import build, lbm, workloads as W
    if rank == 0:
        build.build()
    if dist is not None:
        dist.barrier()
    n = args.n
    n_drops = 512 if n == 4096 else max(1, int(512 * (n / 4096) ** 2))
    p, phi = W.precision(n=n, n_drops=n_drops)
    cells = n * n
    peak, peak_kind = _peaks()

    def measure(dtype, steps, warmup, clocks=False):
        sim = lbm.Sim(p, dtype)
        sim.init_phi(phi)
        if dist is not None:
            torch.cuda.synchronize()
            dist.barrier()
        if clocks:
            with Clocks(torch.cuda.current_device()) as ck:
                total, per = time_steps(sim, steps, warmup)
            ckinfo = ck.summary()
        else:
            total, per = time_steps(sim, steps, warmup)
            ckinfo = None
        if dist is not None:
            total = max_over_ranks(total, dist, "cuda")
            torch.cuda.synchronize()
            dist.barrier()
        return sim, total, per, ckinfo

    sim, total_ms, per, ck = measure("f32", args.steps, args.warmup, clocks=True)
    ms = total_ms / args.steps
    mlups = cells * args.steps * world / (total_ms * 1e-3) / 1e6
    avg_launch_ms = statistics.mean(per)
    alg = BYTES_PER_CELL["f32"] * cells
    achieved = alg / (avg_launch_ms * 1e-3) / 1e9
    sim.close()

    line = {"metric": "MLUPS", "value": round(mlups, 2), "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 5),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "nx": n, "ny": n, "droplets": n_drops,
                       "rho_ratio": 100, "storage": "f32", "parallelism": f"replicas{world}",
                       "l2": "no flush: populations 2.4 GB per time level > 129 MB L2"},
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                         "unit": "GB/s", "frac": round(achieved / peak, 4),
                         "traffic": _traffic("f32", full_size=args.n == 4096), "peak_kind": peak_kind,
                         "bytes_per_cell": BYTES_PER_CELL["f32"],
                         "kernel": ("k_strip_tma<float> (rows of interior strips by TMA tensor tiles)"
                                    if n % 8 == 0 else "k_step<float>"),
                         "launch_ms": {"mean": round(avg_launch_ms, 5), "min": round(min(per), 5),
                                       "max": round(max(per), 5)}},
            "gpu_launches": args.steps, "clocks": ck}
    # ALU side of the roofline: measured FMA rates and the FP32 lane
    # operations per cell-update (ncu counts) at the measured speed
    peaks = alu_peaks(lbm)
    line["alu_peaks_gfma_s"] = peaks
    a32 = _alu("f32")
    if a32 and "f32" in peaks:
        got = a32["fp32_lane_ops"] * mlups / 1e3 / world
        line["alu"] = {"fp32_flops_per_cell": a32["fp32_flops"], "fp32_lane_ops_per_cell": a32["fp32_lane_ops"],
                       "achieved_gops": round(got, 1), "peak_gfma": peaks["f32"],
                       "frac": round(got / peaks["f32"], 4),
                       "flop_per_byte": round(a32["fp32_flops"] / BYTES_PER_CELL["f32"], 2)}

    if not args.no_forms:
        forms = {}
        ref = None
        for dtype in ("f64", "f16s", "bf16s", "f16d", "bf16d"):
            ksteps = args.steps if dtype != "f64" else max(10, args.steps // 10)
            s2, tot, per2, _ = measure(dtype, ksteps, args.warmup)
            m2 = cells * ksteps * world / (tot * 1e-3) / 1e6
            ach2 = BYTES_PER_CELL[dtype] * cells / (statistics.mean(per2) * 1e-3) / 1e9
            forms[dtype] = {"mlups": round(m2, 2), "ms_per_step": round(tot / ksteps, 5),
                            "hbm_gbs": round(ach2, 1), "frac": round(ach2 / peak, 4),
                            "bytes_per_cell": BYTES_PER_CELL[dtype],
                            "traffic": _traffic(dtype, full_size=args.n == 4096)}
            a64 = _alu("f64") if dtype == "f64" else None
            if a64 and "f64" in peaks:
                # FP64 add, multiply and FMA each take one FP64 pipe slot
                got = a64["fp64_ops"] * m2 / 1e3 / world
                forms[dtype]["roofline"] = {"bound": "alu", "achieved": round(got, 1),
                                            "peak": peaks["f64"], "unit": "G FP64 ops/s",
                                            "frac": round(got / peaks["f64"], 4),
                                            "ops_per_cell": a64["fp64_ops"], "peak_kind": "measured (lbm_alu_peak)"}
            s2.close()
        # errors after the same number of steps, against the FP64 path
        errs = {}
        K = args.warmup + args.steps
        s64 = lbm.Sim(p, "f64")
        s64.init_phi(phi)
        s64.step(K)
        ref = s64.fields(("phi", "ux", "uy", "p"))
        s64.close()
        for dtype in ("f32", "f16s", "bf16s", "f16d", "bf16d"):
            s3 = lbm.Sim(p, dtype)
            s3.init_phi(phi)
            s3.step(K)
            f3 = s3.fields(("phi", "ux", "uy", "p"))
            s3.close()
            errs[dtype] = {k: float((f3[k].double() - ref[k]).abs().max().item()) for k in f3}
        for dtype in ("f16s", "bf16s", "f16d", "bf16d"):
            forms[dtype]["gain_vs_f32"] = round(forms[dtype]["mlups"] / mlups, 3)
            forms[dtype]["max_abs_err_vs_f64"] = errs[dtype]
            forms[dtype]["steps_for_err"] = K
        forms["f32"] = {"max_abs_err_vs_f64": errs["f32"], "steps_for_err": K}
        line["forms"] = forms

    if not args.no_batch:
        line["batched"] = measure_batch(lbm, W, args, peak, dist)
    if not args.no_slabs:
        line["slabs"] = measure_slabs(lbm, p, phi, args, mlups, dist)
    if not args.no_lagged:
        line["gradp_lag"] = measure_lagged(lbm, p, phi, args, peak, mlups, dist)
    if not args.no_3d:
        line["d3q19"] = measure_3d(lbm, W, args, peak, dist)
    if not args.no_adjoint:
        line["adjoint"] = measure_adjoint(W, peak)

    # End to end through the C ABI with host buffers: phi0 in, K steps,
    # phi/u/p out and the mass diagnostic, all inside the timed region.
    npdt = np.float32
    phi_h = torch.from_numpy(phi.astype(npdt)).pin_memory().numpy()
    outs = {k: torch.empty((n, n), dtype=torch.float32).pin_memory().numpy()
            for k in ("phi", "ux", "uy", "p")}
    sim = lbm.Sim(p, "f32")
    sim.init_phi_host(phi_h)
    sim.step(args.warmup)
    sim.fields_host(out=outs)
    # the whole job three times, the median reported (a ~0.1 s region with
    # host transfers varies by several per cent from run to run)
    times = []
    for _ in range(3):
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        t0 = time.perf_counter()
        sim.init_phi_host(phi_h)
        sim.step(args.steps)
        sim.fields_host(out=outs)
        sim.mass()
        times.append(time.perf_counter() - t0)
    sim.close()
    t_e2e = max_over_ranks(sorted(times)[1], dist, "cuda")
    h2d = phi_h.nbytes
    d2h = sum(v.nbytes for v in outs.values()) + 16
    line["e2e"] = {"value": round(cells * args.steps * world / t_e2e / 1e6, 2), "unit": "MLUPS",
                   "h2d_bytes_per_step": round(h2d / args.steps, 1),
                   "d2h_bytes_per_step": round(d2h / args.steps, 1),
                   "note": "one C-ABI job: phi0 from pinned host memory, init, steps, "
                           "4 fields + mass back to host; median of 3 jobs; bytes are per step of the job"}

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
