"""Benchmark: SEM operator apply throughput (GDOF/s, local DOFs) and % of the HBM roofline.

Workload (default): structured 64^3-element hex mesh of [0,1]^3, order N=7 (134.2M local DOFs,
90.5M global nodes), interior vertices perturbed by U(-0.1h, 0.1h), u ~ U(-1, 1), Dirichlet box.
One step = one FP64-accurate operator apply y = M A M u through the C ABI (gather, D-contractions,
geometric scaling, transposed contractions, scatter-add), inputs resident in HBM and larger than
L2 (factors 6.4 GB, u 0.72 GB), so no L2 flush is needed between steps.

Also reported in the same JSON line:
  e2e           the same step through the C ABI with host buffers (pinned H2D of u, D2H of y)
  roofline      algorithmic bytes per apply / measured apply time against MEASURED_PEAKS hbm_gbs
  cpu_baseline  the FP64 oracle's sum-factorised apply on the host cores, bounded element sample
  variants      the FP32 apply on the same mesh and the other precisions, for context
  solve         Jacobi-PCG time to 1e-10 (plain FP64 vs mixed-precision refinement) on 24^3, N=7

``--impl reference`` times the oracle (the CPU reference) on the same metric instead.
Multi-GPU: every rank runs an independent replica (the apply does not shard in this build);
value = total local DOFs processed by all ranks / max-over-ranks time.
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

import workloads as W  # noqa: E402


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--order", type=int, default=7)
    ap.add_argument("--elems", type=int, default=64, help="elements per direction of the box")
    ap.add_argument("--prec", default="fp64", choices=["fp64", "fp64_emu", "fp32"])
    ap.add_argument("--no-extras", action="store_true", help="skip variants / solve / cpu baseline")
    return ap.parse_args()


def algorithmic_bytes(E, N, G, prec):
    n3 = (N + 1) ** 3
    L = E * n3
    s = 4 if prec == "fp32" else 8
    return 6 * s * L + 2 * s * G  # six factors per local node, u read once and y written once


def flops(E, N):
    n = N + 1
    return (12 * n ** 4 + 15 * n ** 3) * E


class ClockSampler:
    """nvidia-smi samples during the timed region (clocks and throttle reasons)."""

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return d["hbm_gbs"], "measured"
    except Exception:
        return 6800.0, "fallback"


def cpu_baseline(N, E_sample=2048, seed=W.BASE_SEED + 2):
    """Oracle sum-factorised apply (FP64, OpenMP over elements) on a bounded element sample."""
    import oracle

    oracle.build()
    s = int(round(E_sample ** (1 / 3)))
    box = (s, s, max(1, E_sample // (s * s)))
    v = W.box_vertices(*box, seed=seed)
    G, _ = oracle.factors(N, v)
    E = v.shape[0]
    n3 = (N + 1) ** 3
    uL = W.uniform(E * n3, seed=seed).reshape(E, n3)
    oracle.apply_local(N, G, uL)  # warm-up
    reps, t0 = 0, time.perf_counter()
    while True:
        oracle.apply_local(N, G, uL)
        reps += 1
        if time.perf_counter() - t0 > 8.0 or reps >= 50:
            break
    dt = (time.perf_counter() - t0) / reps
    cores = len(os.sched_getaffinity(0))
    return {"value": E * n3 / dt / 1e9, "unit": "GDOF/s", "cores": cores, "kind": "oracle",
            "sample": f"{E} elements ({box[0]}x{box[1]}x{box[2]} box) of the same N={N} perturbed mesh, "
                      f"local apply only, {reps} reps, OMP threads={os.environ.get('OMP_NUM_THREADS', cores)}"}


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    N = a.order
    cb = cpu_baseline(N)
    K = a.steps
    line = {"metric": "SEM Ax GDOF/s (local DOFs)", "value": cb["value"], "unit": "GDOF/s", "n_gpus": a.gpus,
            "steps": K, "warmup": a.warmup, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": f"SEM Ax, {a.elems}^3 hex mesh, N={N} (oracle on a bounded element sample)",
                       "order": N, "elements": a.elems ** 3},
            "cpu_baseline": {k: cb[k] for k in ("kind", "cores", "sample")} | {"value": cb["value"]},
            "e2e": {"value": cb["value"], "unit": "GDOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    a = parse()
    if a.impl == "reference":
        return run_reference(a)

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import paper_1403_0968_gb300 as sem
    from paper_1403_0968_gb300 import build as sbuild

    sbuild.build()
    sem.lib()

    N, s = a.order, a.elems
    box = (s, s, s)
    v = W.box_vertices(*box, seed=W.BASE_SEED + 2)
    prob = sem.Problem(N, v, box=box, bc="box",
                       features=sem.SEM_FEAT_FP64 | sem.SEM_FEAT_FP32 | sem.SEM_FEAT_EMU * (a.prec == "fp64_emu"))
    E, G, L = prob.nelem, prob.nglobal, prob.nlocal
    u_h = W.uniform(G, seed=W.BASE_SEED + 2)
    dt = torch.float32 if a.prec == "fp32" else torch.float64
    u = torch.from_numpy(u_h).to(dt).cuda()
    y = torch.empty_like(u)
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(max(3, a.warmup)):
        prob.apply(u, y, prec=a.prec)
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    per = []
    with ClockSampler(local) as clk:
        time.sleep(0.3)
        barrier()
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for _ in range(a.steps):
            ev0.record(stream)
            prob.apply(u, y, prec=a.prec)
            ev1.record(stream)
            ev1.synchronize()
            per.append(ev0.elapsed_time(ev1))
        t_end.record(stream)
        barrier()
    total_ms = t_start.elapsed_time(t_end)
    ms = float(np.mean(per))
    if world > 1:
        tt = torch.tensor([ms], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())
    value = world * L / (ms * 1e-3) / 1e9

    # end to end through the C ABI with host buffers: pinned H2D of u, apply, D2H of y
    u_pin = torch.from_numpy(u_h).to(dt).pin_memory()
    y_pin = torch.empty_like(u_pin).pin_memory()
    ud = torch.empty_like(u)
    for _ in range(2):
        ud.copy_(u_pin, non_blocking=True)
        prob.apply(ud, y, prec=a.prec)
        y_pin.copy_(y, non_blocking=True)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ke = max(3, a.steps // 3)
    e0.record(stream)
    for _ in range(ke):
        ud.copy_(u_pin, non_blocking=True)
        prob.apply(ud, y, prec=a.prec)
        y_pin.copy_(y, non_blocking=True)
    e1.record(stream)
    barrier()
    e2e_ms = e0.elapsed_time(e1) / ke
    esz = 4 if a.prec == "fp32" else 8

    hbm, src = peaks()
    ab = algorithmic_bytes(E, N, G, a.prec)
    achieved = ab / (ms * 1e-3) / 1e9
    line = {
        "metric": "SEM Ax GDOF/s (local DOFs)", "value": value, "unit": "GDOF/s", "n_gpus": world,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp64": "f64", "fp32": "f32", "fp64_emu": "f32x2 (double-float)"}[a.prec],
        "data": "synthetic",
        "config": {"workload": f"SEM Ax y=MAMu, {s}^3 perturbed hex mesh of [0,1]^3, N={N}, Dirichlet box",
                   "order": N, "elements": E, "local_dofs": L, "global_dofs": G, "precision": a.prec,
                   "l2": "inputs larger than L2 (factors %.2f GB), no flush" % (6 * esz * L / 1e9)},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                     "traffic": None, "peak_source": src, "algorithmic_bytes": ab,
                     "gflops": flops(E, N) / (ms * 1e-3) / 1e9},
        "e2e": {"value": world * L / (e2e_ms * 1e-3) / 1e9, "unit": "GDOF/s", "h2d_bytes_per_step": G * esz,
                "d2h_bytes_per_step": G * esz},
        "gpu_launches": a.steps,
        "clocks": clk.summary(),
        "timed_region_ms": total_ms,
    }
    if rank == 0 and not a.no_extras and world == 1:
        line["cpu_baseline"] = cpu_baseline(N)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
