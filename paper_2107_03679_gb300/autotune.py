"""Autotuner for the solver's free parameters on a given problem.

The sweep counts nu1 = nu2 of the multigrid cycle and the GMRES restart length trade per-step cost
against the number of steps, and the best pair depends on the grid, the wavenumber and the
contrast.  The tuner times complete forward solves of a spread-out sample of the illumination
angles for every candidate pair (CUDA events on the solver's stream), picks the pair with the
least time per solve, and caches it in a JSON file keyed by grid, batch, precision and level
count.  All computation runs in the CUDA library; this module only drives and times it.
"""
from __future__ import annotations

import json
import os
from typing import Dict, Iterable, Optional, Tuple

import torch

from .solver import Solver

CACHE = os.environ.get("MGH_AUTOTUNE_CACHE",
                       os.path.join(os.path.expanduser("~"), ".cache", "mgh_autotune.json"))


def _key(nx: int, ny: int, B: int, precision: str, levels: int, k: float) -> str:
    return f"{nx}x{ny}:B{B}:{precision}:L{levels}:kh{k:.6f}"


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
         use_cache: bool = True) -> Tuple[dict, list]:
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
            s = Solver.from_workload(w, batch_max=th.numel(), precision=precision, device=device, nu1=nu, nu2=nu,
                                     restart=m, maxit=20000)
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
