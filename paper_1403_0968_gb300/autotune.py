"""Tile-shape autotuner for the apply kernels, with a persisted table.

For a problem (``Problem``) or a batch (``Batch``) it times every kernel variant the library
offers for the order and precision at hand (CUDA events, after warm-up), selects the fastest and
records it in a JSON table keyed by (kind, precision, order, size bucket), so that later problems
of the same shape reuse the choice without timing.  The table lives in the file named by the
environment variable SEM_AUTOTUNE_TABLE, else in the package's build folder.
"""
from __future__ import annotations

import json
import math
import os
import threading

from . import build as _build

_lock = threading.Lock()


def table_path() -> str:
    return os.environ.get("SEM_AUTOTUNE_TABLE", os.path.join(_build.BUILD, "autotune.json"))


def _load() -> dict:
    try:
        with open(table_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(tab: dict) -> None:
    path = table_path()
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(tab, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _key(kind: str, prec: str, N: int, nlocal: int) -> str:
    return f"{kind}/{prec}/N{N}/2^{int(math.log2(max(1, nlocal)))}"


def _time(fn, reps: int) -> float:
    import torch

    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def tune_problem(prob, prec: str = "fp32", reps: int = 5, use_table: bool = True) -> int:
    """Pick the fastest apply variant for ``prob`` in precision ``prec``; returns it."""
    import torch

    key = _key("problem", prec, prob.N, prob.nlocal)
    with _lock:
        tab = _load() if use_table else {}
    if key in tab:
        prob.set_apply_variant(tab[key]["variant"])
        return tab[key]["variant"]
    dt = torch.float32 if prec in ("fp32", "bf16", "fp32_otf") else torch.float64
    u = torch.rand(prob.nglobal, dtype=dt, device="cuda")
    y = torch.empty_like(u)
    variants = [0, 1] if prec == "fp64_emu" else [0, 1, 2, 3]
    times = {}
    for v in variants:
        prob.set_apply_variant(v)
        times[v] = _time(lambda: prob.apply(u, y, prec=prec), reps)
    best = min(times, key=times.get)
    prob.set_apply_variant(best)
    with _lock:
        tab = _load()
        tab[key] = {"variant": best, "ms": times}
        _store(tab)
    return best


def tune_batch(batch, reps: int = 5, use_table: bool = True) -> dict:
    """Pick the fastest batched FP32 apply variant per order group; returns {N: variant}."""
    import torch

    u = torch.rand(batch.nglobal, dtype=torch.float32, device="cuda")
    y = torch.empty_like(u)
    chosen = {}
    total = sum(batch.nlocal)
    with _lock:
        tab = _load() if use_table else {}
    for N in batch.orders:
        key = _key("batch", "fp32", N, total)
        if key in tab:
            batch.set_variant(N, tab[key]["variant"])
            chosen[N] = tab[key]["variant"]
            continue
        times = {}
        for v in (1, 2):
            batch.set_variant(N, v)
            # the batched apply covers every order group; differences come from group N only
            times[v] = _time(lambda: batch.apply(u, y, prec="fp32"), reps)
        best = min(times, key=times.get)
        batch.set_variant(N, best)
        chosen[N] = best
        with _lock:
            t2 = _load()
            t2[key] = {"variant": best, "ms": times}
            _store(t2)
    if batch.fused_state()[0]:
        chosen["fused"] = _tune_batch_step(batch, tab, total)
    return chosen


def _tune_batch_step(batch, tab, total, steps: int = 128) -> bool:
    """Fused step kernel or per-order-group launches for the inner steps of batch.pcg: both run
    `steps` inner steps on a random right-hand side; the faster is kept."""
    import torch

    key = _key("batch", "step", "-".join(str(n) for n in batch.orders), total)
    if key in tab:
        batch.set_fused(tab[key]["fused"])
        return tab[key]["fused"]
    b = torch.rand(batch.nglobal, dtype=torch.float64, device="cuda")
    times = {}
    for fused in (True, False):
        batch.set_fused(fused)
        times[fused] = _time(lambda: batch.pcg(b, max_it=steps, rtol=1e-300, check_every=16), 2)
    best = min(times, key=times.get)
    batch.set_fused(best)
    with _lock:
        t2 = _load()
        t2[key] = {"fused": best, "ms": {"fused": times[True], "multi_launch": times[False]}}
        _store(t2)
    return best
