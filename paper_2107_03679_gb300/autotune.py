"""Autotuner for the solver's free parameters on a given problem.

Two stages, both cached in a JSON file keyed by grid, batch, precision, level count and k h:

* Method parameters.  The sweep counts nu1 = nu2 of the multigrid cycle and the GMRES restart
  length trade per-step cost against the number of steps, and the best pair depends on the grid,
  the wavenumber and the contrast.  Every candidate pair is timed on complete forward solves of a
  spread-out sample of the illumination angles (CUDA events on the solver's stream); the pair with
  the least time per solve wins.
* Launch shapes of the FP32 level kernels (mgh_set_kernel_shape): the wavefront segment length,
  warps per block and ring depth, and the first level and cluster size of the one-kernel coarse tail.  They do not
  change results, only speed, so each candidate is timed on a fixed number of Arnoldi steps of the
  full batch (the launch configuration that will run), one axis at a time from the built-in choice,
  keeping a change only when it gains more than 2 %.

All computation runs in the CUDA library; this module only drives and times it.
"""
from __future__ import annotations

import json
import os
from typing import Dict, Iterable, Optional, Tuple

import torch

from .solver import Solver

CACHE = os.environ.get("MGH_AUTOTUNE_CACHE",
                       os.path.join(os.path.expanduser("~"), ".cache", "mgh_autotune.json"))


def _key(nx: int, ny: int, B: int, precision: str, levels: int, k: float, what: str = "") -> str:
    return f"{nx}x{ny}:B{B}:{precision}:L{levels}:kh{k:.6f}" + (f":{what}" if what else "")


def _load() -> Dict[str, dict]:
    try:
        with open(CACHE) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _store(data: Dict[str, dict]) -> None:
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(data, fh, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


def tune(w, f_d: torch.Tensor, theta: torch.Tensor, device: torch.device, precision: Optional[str] = None,
         sample: int = 8, nus: Iterable[int] = (1, 2, 3), restarts: Iterable[int] = (5, 8, 12),
         use_cache: bool = True, **solver_kw) -> Tuple[dict, list]:
    """Best (nu, restart) for workload geometry `w` with contrast f_d and angles theta.

    Returns (choice, trials); choice = {"nu": .., "restart": .., "ms_per_solve": ..}."""
    precision = precision or w.precision
    B = theta.numel()
    key = _key(w.nx, w.ny, B, precision, w.levels, w.k * w.h)
    cache = _load() if use_cache else {}
    if key in cache:
        return cache[key], []
    idx = torch.linspace(0, B - 1, min(sample, B)).round().long()
    th = theta.to(device)[idx.to(device)]
    trials = []
    for nu in nus:
        for m in restarts:
            try:
                s = Solver.from_workload(w, batch_max=th.numel(), precision=precision, device=device, nu1=nu,
                                         nu2=nu, restart=m, maxit=20000, **solver_kw)
            except Exception:          # a pair this precision or engine does not support
                continue
            s.set_contrast(f_d)
            s.forward(th)                      # warm-up (kernel attributes, clocks)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s.stream)
            _, infos = s.forward(th)
            e1.record(s.stream)
            torch.cuda.synchronize(device)
            ms = e0.elapsed_time(e1) / th.numel()
            ok = all(i["converged"] for i in infos)
            trials.append({"nu": nu, "restart": m, "ms_per_solve": ms, "converged": ok,
                           "iterations": sum(i["iterations"] for i in infos) / len(infos)})
            s.close()
    good = [t for t in trials if t["converged"]] or trials
    best = min(good, key=lambda t: t["ms_per_solve"])
    choice = {"nu": best["nu"], "restart": best["restart"], "ms_per_solve": best["ms_per_solve"],
              "iterations": best["iterations"], "sample_angles": int(th.numel())}
    if use_cache:
        cache[key] = choice
        _store(cache)
    return choice, trials


def _time_steps(solver: Solver, theta: torch.Tensor, reps: int = 3) -> float:
    """Milliseconds per Arnoldi step of the whole batch: forward solves capped at the handle's maxit
    (every right-hand side runs the same number of steps), best of `reps` after one warm-up."""
    solver.forward(theta)
    best = None
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(solver.stream)
        _, infos = solver.forward(theta)
        e1.record(solver.stream)
        torch.cuda.synchronize(solver.device)
        steps = max(1, max(i["iterations"] for i in infos))
        ms = e0.elapsed_time(e1) / steps
        best = ms if best is None else min(best, ms)
    return best


def tune_shapes(w, f_d: torch.Tensor, theta: torch.Tensor, device: torch.device, precision: Optional[str] = None,
                steps: int = 48, use_cache: bool = True, **solver_kw) -> Tuple[dict, list]:
    """Launch shapes of the level kernels for workload w's full batch theta, one axis at a time:
    wavefront segment length (0 = the built-in model), warps per block, ring depth, first tail level,
    blocks per right-hand side of the tail.  Each candidate is timed on `steps` Arnoldi steps of forward solves (maxit = steps).  Returns
    (shape, trials); shape also holds the time per step of the built-in choice and of the winner."""
    precision = precision or w.precision
    B = theta.numel()
    key = _key(w.nx, w.ny, B, precision, w.levels, w.k * w.h, "shape")
    cache = _load() if use_cache else {}
    if key in cache:
        return cache[key], []
    s = Solver.from_workload(w, batch_max=B, precision=precision, device=device, maxit=steps, **solver_kw)
    s.set_contrast(f_d)
    th = theta.to(device)
    base = s.kernel_shape()
    auto_tail = base["tail_level"]
    best, best_ms = dict(base), _time_steps(s, th)
    trials = [dict(best, ms_per_step=best_ms)]
    # levels run by the level kernels: 0 .. tail-1 (all but the coarsest without a tail)
    top = auto_tail if auto_tail > 0 else w.levels - 1

    def with_seg(shape, l, v):
        segs = list(shape["wave_seg"])
        segs[l] = v
        return dict(shape, wave_seg=segs)

    axes = [(f"wave_seg[{l}]", [(lambda sh, v=v, l=l: with_seg(sh, l, v)) for v in (8, 16, 32, 64, 128)])
            for l in range(top)]
    axes += [("wave_warps", [(lambda sh, v=v: dict(sh, wave_warps=v)) for v in (2, 4)]),
             ("wave_ring", [(lambda sh, v=v: dict(sh, wave_ring=v)) for v in (1, 2)]),
             ("tail_level", [(lambda sh, v=v: dict(sh, tail_level=v)) for v in (0, auto_tail, auto_tail + 1)]),
             ("tail_cluster", [(lambda sh, v=v: dict(sh, tail_cluster=v)) for v in (1, 2, 4)])]
    for _, moves in axes:
        for move in moves:
            cand = move(best)
            if cand == best:
                continue
            try:
                s.set_kernel_shape(**cand)
            except Exception:          # not available for this handle (e.g. FP16 storage, tail too big)
                continue
            ms = _time_steps(s, th)
            trials.append(dict(cand, ms_per_step=ms))
            if ms < best_ms * 0.98:    # keep a change only for a clear gain (timing noise is ~1 %)
                best, best_ms = cand, ms
        s.set_kernel_shape(**best)
    s.close()
    shape = dict(best, ms_per_step=best_ms, builtin_ms_per_step=trials[0]["ms_per_step"], steps_timed=steps)
    if use_cache:
        cache[key] = shape
        _store(cache)
    return shape, trials
