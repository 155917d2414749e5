#!/usr/bin/env python
"""Benchmark of the batched multigrid-preconditioned Helmholtz solver.

Metric: Helmholtz solves per second to relative residual 1e-6 (batched angles), with the
achieved HBM bandwidth of the dominant kernel against the measured peak.

One step is one pass over every stage of the hot path for one batch of illuminations of the
batched-forward workload (512^2 interior + 32-cell absorbing layer, 60 plane waves, contrast
from 6 seeded ellipses, FP32 V-cycle with 6 levels, FP64 FGMRES(20), tol 1e-6):
  set the contrast and rebuild the hierarchy; form the 60 right-hand sides and solve them;
  crop to the interior and sample the receivers; evaluate the data misfit; solve the 60
  adjoint systems and form the gradient in the contrast.  A step therefore completes 120
  Helmholtz solves, every one of them to true relative residual <= 1e-6.

Under torchrun each rank runs its own batch (independent problems, weak scaling, no
collective on the data path); the timing is the maximum over ranks.
`--impl reference` times the FP64 CPU oracle on the host cores instead (bounded sample).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Helmholtz solves/s to rel-res 1e-6 (batched angles); V-cycle HBM GB/s vs peak"
UNIT = "solves/s"
ITER_FIXTURE = os.path.join(ROOT, "tests", "golden", "oracle_iterations.json")


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["mgh", "reference"], default="mgh")
    ap.add_argument("--workload", default="ellipses576")
    ap.add_argument("--precision", choices=["mixed32", "mixed16", "fp64"], default=None,
                    help="mixed16: FP16 storage of the level-0 iterate and the preconditioned vectors")
    ap.add_argument("--split", type=int, default=1,
                    help="split the angles over this many handles on concurrent streams (coarse levels of one "
                         "part overlap the fine levels of another)")
    ap.add_argument("--angles", type=int, default=None,
                    help="use only the first N illumination angles (smaller case for profiling)")
    ap.add_argument("--restart", type=int, default=None, help="GMRES restart length (default: the workload's)")
    ap.add_argument("--nu", type=int, default=None, help="pre- and post-smoothing sweeps (default: the workload's)")
    ap.add_argument("--levels", type=int, default=None, help="multigrid levels (default: the workload's)")
    ap.add_argument("--shift-im", type=float, default=None,
                    help="imaginary part of the multigrid shift kappa (default: the workload's)")
    ap.add_argument("--maxit", type=int, default=20000, help="Arnoldi steps per solve before giving up")
    ap.add_argument("--arnoldi", choices=["auto", "df", "fp64", "sstep"], default="auto",
                    help="mixed-precision Krylov engine: s-step cycles (Gram/Cholesky), double-float Arnoldi, "
                         "native-FP64 Arnoldi; auto = s-step when the restart length is at most 8")
    ap.add_argument("--cycle", choices=["v", "w"], default="v",
                    help="multigrid cycle of the preconditioner (CycleType of Alg. 2)")
    ap.add_argument("--krylov", choices=["fgmres", "bicgstab", "idrs"], default=None,
                    help="outer Krylov method: flexible GMRES, the paper's Bi-CGSTAB (Alg. 3) or IDR(s) with "
                         "biorthogonalisation; default: the workload's")
    ap.add_argument("--idr-s", type=int, default=4,
                    help="shadow-space dimension s of --krylov idrs (1..8; the restart length is raised to 2 s + 2 "
                         "to hold its vectors)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="skip the autotuner (nu, restart length and level-kernel launch shapes, chosen by timing "
                         "before the timed region and cached)")
    ap.add_argument("--descent", type=int, default=0,
                    help="instead of the throughput line: N projected gradient-descent steps from f = 0")
    ap.add_argument("--fbs", type=int, default=0,
                    help="instead of the throughput line: N accelerated FBS iterations with TV (Alg. 4) from f = 0")
    ap.add_argument("--subset", type=int, default=6,
                    help="angles per FBS iteration, drawn at random each iteration (0: all angles)")
    ap.add_argument("--tv-lam", type=float, default=5e-4, help="TV weight of the backward step, gamma * tau")
    ap.add_argument("--prox-iters", type=int, default=100, help="dual FGP iterations per backward step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-sample", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--sample-steps", type=int, default=60, help=argparse.SUPPRESS)
    ap.add_argument("--sample-angle", type=int, default=0, help=argparse.SUPPRESS)
    ap.add_argument("--no-fp64-compare", action="store_true",
                    help="skip the plain-FP64 run of the same step (speed-up at the same accuracy)")
    ap.add_argument("--no-fp16-compare", action="store_true",
                    help="skip the run of the same step with FP16 storage on the fine level (mixed16)")
    return ap.parse_args(argv)


# --------------------------------------------------------------------------- inputs
def make_inputs(w):
    """Seeded synthetic inputs: ground truth phantom, the iterate the step is evaluated at,
    angles and receivers (the data are produced on the device from the ground truth)."""
    import numpy as np
    import workloads as W
    f_gt = W.phantom(w)
    f_step = 0.9 * f_gt
    th = W.angles(w)
    rec = W.receivers(w, f_gt)
    return f_gt, f_step, th, rec


# DRAM bytes of one launch of a kernel class, from ncu captures of 24-angle launches of the current
# kernels on the 576^2 workload (6 levels, nu = 2, restart 8, FP32 cycle): (bytes of the capture,
# bytes read once per launch whatever the batch); see profiles/vcycle_post_l0_ellipses576.md and
# profiles/gram_sstep_ellipses576.md.  Traffic grows with the right-hand sides (independent sweeps).
NCU_TRAFFIC_24 = {"vcycle_post_l0": (263.8e6, 5.3e6), "gs_update": (577.4e6, 0.0)}
POST_CAPTURE_FUSED = True   # whether the captured level-0 post kernel formed the s-step product itself


def captured_traffic(cls: str, w, precision: str, B: int, shape=None, fused=True):
    """Scaled capture for this launch, or None when no capture matches (another workload, launch
    shapes other than the captured built-in ones: 4 warps per block, ring of one period, or a
    level-0 post kernel with or without the fused operator product unlike the captured one)."""
    if (w.nx, w.levels, w.nu1, w.nu2, w.restart, precision) != (576, 6, 2, 2, 8, "mixed32") or cls not in NCU_TRAFFIC_24:
        return None
    if cls == "vcycle_post_l0" and fused != POST_CAPTURE_FUSED:
        return None
    if shape and (shape.get("wave_warps", 4) != 4 or shape.get("wave_ring", 1) != 1 or any(shape.get("wave_seg", []))):
        return None
    cap, once = NCU_TRAFFIC_24[cls]
    return round((cap - once) * B / 24 + once)


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of the SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 6:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[2:6]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------------- algorithmic bytes
def coarse_fraction(nx: int, ny: int, levels: int, gamma: int = 1) -> float:
    """Points of the levels 1 .. L-2 (the coarser smoothing levels) per fine point, each level
    counted once per visit in a cycle of CycleType gamma (gamma^(l-1) visits of level l)."""
    tot, cx, cy = 0, nx, ny
    for l in range(1, levels - 1):
        cx, cy = (cx - 1) // 2 + 1, (cy - 1) // 2 + 1
        tot += gamma ** (l - 1) * cx * cy
    return tot / (nx * ny)


def algorithmic_bytes(prof: dict, N: int, cs: int, launches: dict, engine: str, cfrac: float = 0.0,
                      zs: int = None, idr_s: int = 4) -> dict:
    """Minimal bytes of each kernel class from the engine counters (fields read once, per-grid
    coefficient arrays counted once per launch).  N = fine points, cs = bytes of one complex
    number of the multigrid precision, zs = bytes of one stored level-0 iterate / preconditioned
    vector entry (cs, or 4 with FP16 storage); engine = "df", "sstep", "fp64", "bicgstab" or
    "idrs" (with idr_s its s); cfrac = points of the coarser smoothing levels per fine point (their
    fields fit in L2, so this class is not bound by DRAM alone)."""
    zs = cs if zs is None else zs
    steps = prof["arnoldi_steps"]
    c16 = 16
    if engine == "bicgstab":
        # per cycle (two per iteration): A y and its dot (read y 8 + w 16, write 16); per iteration
        # the p, s and r updates read/write 72 + 96 + 104 B; counters count cycles
        return {
            "vcycle_pre_l0": steps * N * (8 + cs + cs / 4) + launches["vcycle_pre_l0"] * 2 * cs * N,
            "vcycle_post_l0": steps * N * (8 + 2 * cs + cs / 4) + launches["vcycle_post_l0"] * cs * N,
            "vcycle_coarse": steps * N * cfrac * cs * (3.25 + 3.25),
            "matvec_dots": steps * N * (cs + 2 * c16) + launches["matvec_dots"] * c16 * N,
            "gs_update": steps / 2 * N * (72 + 96 + 104),
            "true_residual": prof["residuals"] * N * 3 * c16,
        }
    if engine == "idrs":
        # IDR(s), per outer step of s + 1 cycles (counters count cycles).  Intermediate step k: v reads
        # r and G_k..G_{s-1}, writes the cycle input (cs); U_k reads U_k..U_{s-1} and the cycle output
        # (cs), writes U_k; G_k = A U_k reads U_k, writes G_k; the projection update reads G_k, U_k,
        # G_0..G_{k-1}, U_0..U_{k-1}, r, x and writes G_k, U_k, r, x.  Dimension reduction: t = A y reads
        # y (cs) and r, writes t; the update reads y (cs), x, r, t and writes x, r.
        s = idr_s
        outer = steps / (s + 1)
        upd = sum((16 + 16 * (s - k) + cs) + (16 * (s - k) + cs + 16) + (8 + 2 * k) * c16 for k in range(s))
        upd += cs + 80
        return {
            "vcycle_pre_l0": steps * N * (8 + cs + cs / 4) + launches["vcycle_pre_l0"] * 2 * cs * N,
            "vcycle_post_l0": steps * N * (8 + 2 * cs + cs / 4) + launches["vcycle_post_l0"] * cs * N,
            "vcycle_coarse": steps * N * cfrac * cs * (3.25 + 3.25),
            "matvec_dots": outer * N * (2 * c16 * s + cs + 2 * c16) + launches["matvec_dots"] * c16 * N,
            "gs_update": outer * N * upd,
            "true_residual": prof["residuals"] * N * 3 * c16,
        }
    if engine == "sstep":
        # s-step cycles: every step of a cycle runs (cycle_steps), one Gram sweep per cycle
        run = prof["cycle_steps"]
        out = {
            # levels 1 .. L-2: pre reads b, writes v and the restricted residual; post reads b, v and
            # the coarse correction, writes the result
            "vcycle_coarse": run * N * cfrac * cs * (3.25 + 3.25),
            "vcycle_pre_l0": run * N * (8 + zs + cs / 4) + launches["vcycle_pre_l0"] * 2 * cs * N,
            "vcycle_post_l0": run * N * (8 + 2 * zs + cs / 4) + launches["vcycle_post_l0"] * cs * N,
            # Gram sweep: read the m + 1 FP32 basis vectors
            "gs_update": prof["gram_reads"] * N * cs,
            "true_residual": prof["residuals"] * N * 3 * c16,
            "x_update": prof["updates"] * N * 2 * c16 + prof["update_reads"] * N * zs,
        }
        if launches.get("matvec_dots", 0) > 0:
            # v_{k+1} = A z_k in FP32: read z_k, write v_{k+1}; D_A (FP32) per launch
            out["matvec_dots"] = run * N * (zs + cs) + launches["matvec_dots"] * cs * N
        else:
            # the product fused into the post kernel: it also writes v_{k+1}; D_A per launch
            out["vcycle_post_l0"] += run * N * cs + launches["vcycle_post_l0"] * cs * N
        return out
    if engine == "df":
        # double-float Arnoldi (mixed path): the V-cycle reads the 8-byte hi plane of u_j
        return {
            "vcycle_pre_l0": steps * N * (8 + cs + cs / 4) + launches["vcycle_pre_l0"] * 2 * cs * N,
            "vcycle_post_l0": steps * N * (8 + 2 * cs + cs / 4) + launches["vcycle_post_l0"] * cs * N,
            # pass 1: read z_j (FP32) and u_j, write w, read the j final basis vectors; D_A planes per launch
            "matvec_dots": steps * N * (cs + 2 * c16) + prof["basis_reads"] * N * c16
            + launches["matvec_dots"] * c16 * N,
            # pass 2: read u_j and w, write q_j and u_{j+1}, read the j final basis vectors
            "gs_update": steps * N * 4 * c16 + prof["basis_reads"] * N * c16,
            # cycle tail: read u_m and the m basis vectors
            "gs_reorth": prof["reorth_reads"] * N * c16 + prof["updates"] * N * c16,
            # double-float residual: read x and b, write u_0 (FP64 acceptance checks are rare)
            "true_residual": prof["residuals"] * N * 3 * c16,
            # double-float iterate update: read and write x, read jend preconditioned vectors
            "x_update": prof["updates"] * N * 2 * c16 + prof["update_reads"] * N * cs,
        }
    out = {
        # level-0 pre-smoothing + residual + restriction: read b (FP64), write v (cs), write the
        # restricted residual (cs/4 per fine point); D and w/D once per launch
        "vcycle_pre_l0": steps * N * (c16 + cs + cs / 4) + launches["vcycle_pre_l0"] * 2 * cs * N,
        # level-0 prolongation + correction + post-smoothing: read b (FP64), v (cs), coarse e
        # (cs/4), write z (cs); w/D once per launch
        "vcycle_post_l0": steps * N * (c16 + 2 * cs + cs / 4) + launches["vcycle_post_l0"] * cs * N,
        # fused w = A z_j + dots: read z (cs) and j+1 basis vectors (FP64), write w (FP64); D_A per launch
        "matvec_dots": steps * N * (cs + c16) + prof["basis_reads"] * N * c16 + launches["matvec_dots"] * c16 * N,
        # update: read w and j+1 basis vectors, write v_{j+1}
        "gs_update": steps * N * 2 * c16 + prof["basis_reads"] * N * c16,
        "true_residual": prof["residuals"] * N * 3 * c16,
        "x_update": prof["updates"] * N * 2 * c16 + prof["update_reads"] * N * cs,
    }
    return out


# --------------------------------------------------------------------------- CPU oracle sample
def cpu_sample_main(args):
    """Run in a subprocess with one BLAS thread: time `sample_steps` FGMRES steps of the FP64
    oracle on one angle of the workload (--sample-angle) and print seconds per Arnoldi step."""
    import numpy as np
    import oracle as O
    import workloads as W
    w = W.WORKLOADS[args.workload]
    _, f_step, th, _ = make_inputs(w)
    p = O.Problem.from_workload(w)
    t0 = time.perf_counter()
    s = O.MGHSolver(p, f_step, w.levels, w.nu1, w.nu2, w.omega, complex(w.shift_re, w.shift_im), w.restart,
                    w.tol, maxit=args.sample_steps)
    t_setup = time.perf_counter() - t0
    b = O.rhs(p, f_step, float(th[args.sample_angle % len(th)]))
    t0 = time.perf_counter()
    _, info = s.solve(b)
    t = time.perf_counter() - t0
    print(json.dumps({"sec_per_step": t / max(info.iterations, 1), "steps": info.iterations, "setup_s": t_setup,
                      "solve_s": t}))


def oracle_iterations_per_solve(workload: str):
    if not os.path.exists(ITER_FIXTURE):
        return None
    with open(ITER_FIXTURE) as fh:
        d = json.load(fh)
    e = d.get(workload)
    if not e:
        return None
    return 0.5 * (e["forward_iterations"] + e["adjoint_iterations"])


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def cpu_model() -> str:
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith(("model name", "cpu part", "hardware")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def run_cpu_samples(workload: str, sample_steps: int, workers: int):
    """`workers` concurrent oracle processes (one BLAS thread each), worker i on angle i: each
    times `sample_steps` FGMRES steps of its own solve.  Returns the per-worker records and the
    host wall clock around all of them."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    env["CUDA_VISIBLE_DEVICES"] = ""
    t0 = time.perf_counter()
    procs = [subprocess.Popen([sys.executable, os.path.abspath(__file__), "--cpu-sample", "--workload", workload,
                               "--sample-steps", str(sample_steps), "--sample-angle", str(i)],
                              stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env)
             for i in range(workers)]
    out = []
    for pr in procs:
        so, se = pr.communicate(timeout=900)
        if pr.returncode != 0:
            raise RuntimeError(f"cpu sample failed: {se[-2000:]}")
        out.append(json.loads(so.strip().splitlines()[-1]))
    return out, time.perf_counter() - t0


def cpu_rate(samples, its: float) -> float:
    """Aggregate oracle solves/s: every worker's Arnoldi steps per second of its own solve,
    summed over workers, divided by the oracle's steps per solve."""
    return sum(s["steps"] / s["solve_s"] for s in samples) / its


def cpu_baseline_record(workload: str, sample_steps: int):
    its = oracle_iterations_per_solve(workload)
    if its is None:
        return None
    cores = host_cores()
    multi, wall = run_cpu_samples(workload, sample_steps, cores)
    one, _ = run_cpu_samples(workload, max(sample_steps // 2, 1), 1)
    return {"value": cpu_rate(multi, its), "unit": UNIT, "cores": cores, "kind": "oracle",
            "cpu": cpu_model(), "single_core_value": cpu_rate(one, its),
            "sample": (f"FP64 numpy oracle, one process per host core ({cores} x 1 BLAS thread), process i on "
                       f"angle i: {sample_steps} FGMRES steps each ({wall:.1f} s wall for all), steps/s summed and "
                       f"divided by the oracle's own {its:.0f} steps per solve (forward/adjoint mean, "
                       f"{os.path.relpath(ITER_FIXTURE, ROOT)}); single_core_value: the same with one process")}


# --------------------------------------------------------------------------- reference arm
def reference_main(args, rank, world):
    if rank != 0:
        return
    import workloads as W
    w = W.WORKLOADS[args.workload]
    its = oracle_iterations_per_solve(args.workload)
    if its is None:
        print(json.dumps({"impl": "reference", "unavailable": f"no oracle iteration fixture for {args.workload}"}))
        return
    sample_steps = 16
    cores = host_cores()
    for _ in range(args.warmup):
        run_cpu_samples(args.workload, sample_steps, cores)
    rates, walls = [], []
    for _ in range(args.steps):
        smp, wall = run_cpu_samples(args.workload, sample_steps, cores)
        rates.append(cpu_rate(smp, its))
        walls.append(wall)
    value = sum(rates) / len(rates)
    sample = (f"FP64 numpy oracle, one process per host core ({cores} x 1 BLAS thread), process i on angle i: "
              f"{sample_steps} FGMRES steps each per step, steps/s summed and divided by {its:.0f} oracle steps "
              f"per solve")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(walls) / len(walls),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "grid": f"{w.nx}x{w.ny}", "angles": w.n_angles},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu": cpu_model(),
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# --------------------------------------------------------------------------- GPU arm
def gpu_main(args, rank, world, local_rank):
    import numpy as np
    import torch
    import workloads as W
    from paper_2107_03679_gb300 import Solver

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    w = W.WORKLOADS[args.workload]
    if args.restart:
        w.restart = args.restart
    if args.nu is not None:
        w.nu1 = w.nu2 = args.nu
    if args.levels:
        w.levels = args.levels
    if args.shift_im is not None:
        w.shift_im = args.shift_im
    if args.krylov is None:
        args.krylov = getattr(w, "krylov", "fgmres")
    if args.krylov == "idrs":       # r, G, U, v and t live in the restart + 1 basis slots
        w.restart = max(w.restart, 2 * args.idr_s + 2)
    precision = args.precision or w.precision
    f_gt, f_step, th, rec = make_inputs(w)
    if args.angles:
        th = th[:args.angles]
    B = len(th)
    tuned = None
    autotune = not args.no_autotune and args.krylov == "fgmres" and args.nu is None and args.restart is None
    if autotune:
        from paper_2107_03679_gb300.autotune import tune
        tuned, _ = tune(w, torch.from_numpy(f_step).to(dev), torch.from_numpy(th), dev, precision=precision,
                        restarts=(5, 8), arnoldi=args.arnoldi, cycle_type=args.cycle)
        w.nu1 = w.nu2 = tuned["nu"]
        w.restart = tuned["restart"]
    solver = Solver.from_workload(w, batch_max=B, precision=precision, device=dev, maxit=args.maxit, arnoldi=args.arnoldi,
                                  krylov=args.krylov, cycle_type=args.cycle, idr_s=args.idr_s)
    stream = solver.stream
    d_th = torch.from_numpy(th).to(dev)
    d_rec = torch.from_numpy(rec).to(dev)
    d_fgt = torch.from_numpy(f_gt).to(dev)
    d_f = torch.from_numpy(f_step).to(dev)
    # synthetic measurements: receiver samples of the ground-truth phantom's fields
    forward_only = bool(w.extra.get("forward_only"))
    if forward_only:        # a forward problem: no data term, no end-to-end data path
        args.no_e2e = True
        d_y = None
    else:
        solver.set_contrast(d_fgt)
        u_gt, _ = solver.forward(d_th)
        d_y = solver.sample(u_gt, d_rec)
        del u_gt
    u = solver.field(B)
    runner = solver          # what the timed steps drive: one handle, or the angles split over several
    if args.split > 1:
        from paper_2107_03679_gb300.multi import SplitBatch
        solver.close()
        runner = SplitBatch.from_workload(w, batch_max=B, parts=args.split, precision=precision, device=dev,
                                          maxit=args.maxit, arnoldi=args.arnoldi, krylov=args.krylov,
                                          cycle_type=args.cycle, idr_s=args.idr_s)
        solver = runner.solvers[0]
        stream = torch.cuda.current_stream(dev)
        u_crop = torch.empty((B, w.ny_int, w.nx_int), dtype=torch.complex128, device=dev)

    if autotune:   # launch shapes of the level kernels, tuned on each handle's own batch
        from paper_2107_03679_gb300.autotune import tune_shapes
        handles = runner.solvers if args.split > 1 else [solver]
        nb = -(-B // args.split) if args.split > 1 else B
        shape, _ = tune_shapes(w, d_f, d_th[:nb], dev, precision=precision, arnoldi=args.arnoldi,
                               krylov=args.krylov, cycle_type=args.cycle)
        for hnd in handles:
            hnd.set_kernel_shape(**{k: shape[k] for k in ("wave_seg", "wave_warps", "wave_ring", "tail_level")})
        tuned = dict(tuned or {}, shape=shape)

    def sample_all(uu):
        if args.split == 1:
            return solver.sample(uu, d_rec)
        return torch.cat([s.sample(uu[a:b], d_rec) for s, (a, b) in zip(runner.solvers, runner.ranges(B))])

    def step(f_dev, y_dev):
        if forward_only:      # a forward problem (no data term): contrast, right-hand sides, solves, crop
            solver.set_contrast(f_dev)
            _, inf_f = solver.forward(d_th, out=u)
            return None, 0.0, inf_f, [], solver.crop(u)
        if args.split > 1:   # every stage below, per part, parts on concurrent streams
            loss, g, inf_f, inf_a = runner.data_term_gradient(f_dev, d_th, d_rec, y_dev, u, crop_out=u_crop)
            return g, loss, inf_f, inf_a, u_crop
        solver.set_contrast(f_dev)                               # contrast, hierarchy, coarsest inverse
        _, inf_f = solver.forward(d_th, out=u)                   # right-hand sides + forward solves
        u_int = solver.crop(u)                                   # truncation to the interior
        _, G, loss = solver.misfit(u, y_dev, d_rec)              # receiver sampling, residual, loss
        g, inf_a = solver.gradient(d_th, u, G)                   # adjoint solves + gradient
        return g, loss, inf_f, inf_a, u_int

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    infos = []
    for _ in range(args.warmup):
        _, _, a, b, _ = step(d_f, d_y)
        infos += a + b
    torch.cuda.synchronize()

    # ---- device-timed region: inputs resident in HBM
    clocks = ClockSampler(int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local_rank)).split(",")[0] or 0)
                          if os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[0].isdigit() else local_rank)
    l0 = runner.launch_count()
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    timed_infos = []
    for _ in range(args.steps):
        _, loss, a, b, _ = step(d_f, d_y)
        timed_infos += a + b
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier()
    launches = runner.launch_count() - l0
    # ---- kernel classes: the same K steps once more, every launch bracketed by CUDA events on
    # the solver's stream (kept out of the timed region above, whose time they would inflate)
    runner.profile_enable(True)
    for _ in range(args.steps):
        step(d_f, d_y)
    prof = runner.profile_read()
    runner.profile_enable(False)
    ms = ev0.elapsed_time(ev1)
    ms_max = ms
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_max = float(t.item())
    solves_rank = (1 if forward_only else 2) * B * args.steps
    value = world * solves_rank / (ms_max / 1e3)
    conv = all(i["converged"] for i in timed_infos)
    worst = max(i["rel_residual"] for i in timed_infos)
    its = [i["iterations"] for i in timed_infos]

    # ---- end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e and args.split == 1:
        # one C-ABI call per step on host buffers: contrast, angles, receivers and data in; loss,
        # gradient and receiver residuals out (mgh_data_term_gradient_host)
        h_f = torch.from_numpy(f_step).pin_memory()
        h_th = torch.from_numpy(th).pin_memory()
        h_rec = torch.from_numpy(rec).pin_memory()
        h_y = d_y.cpu().pin_memory()
        h_g = torch.empty((w.ny_int, w.nx_int), dtype=torch.float64).pin_memory()
        h_r = torch.empty((B, rec.size), dtype=torch.complex128).pin_memory()
        solver.data_term_gradient_host(h_f, h_th, h_rec, h_y, grad_out=h_g, r_out=h_r)   # staging allocated here
        h2d = h_f.numel() * 8 + h_th.numel() * 8 + h_rec.numel() * 8 + h_y.numel() * 16
        d2h = h_g.numel() * 8 + h_r.numel() * 16 + 8
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record(stream)
        for _ in range(args.steps):
            solver.data_term_gradient_host(h_f, h_th, h_rec, h_y, grad_out=h_g, r_out=h_r)
        e1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        barrier()
        ems = e0.elapsed_time(e1)
        if world > 1:
            import torch.distributed as dist
            t = torch.tensor([ems], device=dev, dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ems = float(t.item())
        e2e = {"value": world * solves_rank / (ems / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "api": "mgh_data_term_gradient_host (C ABI, host buffers)",
               "host_wall_value": round(world * solves_rank / wall, 3)}
    elif not args.no_e2e:
        h_f = torch.from_numpy(f_step).pin_memory()
        h_y = d_y.cpu().pin_memory()
        h_g = torch.empty((w.ny_int, w.nx_int), dtype=torch.float64).pin_memory()
        h_s = torch.empty((B, rec.size), dtype=torch.complex128).pin_memory()
        h2d = h_f.numel() * 8 + h_y.numel() * 16
        d2h = h_g.numel() * 8 + h_s.numel() * 16 + 8
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            f_dev = h_f.to(dev, non_blocking=True)
            y_dev = h_y.to(dev, non_blocking=True)
            g, loss, _, _, _ = step(f_dev, y_dev)
            h_g.copy_(g, non_blocking=True)
            h_s.copy_(sample_all(u), non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ems = e0.elapsed_time(e1)
        if world > 1:
            import torch.distributed as dist
            t = torch.tensor([ems], device=dev, dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ems = float(t.item())
        e2e = {"value": world * solves_rank / (ems / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}

    # ---- the plain FP64 form of the same step at the same accuracy (FP64 cycle, native-FP64 Arnoldi,
    # the same acceptance test): one warm-up and at most two timed steps, CUDA events on its stream
    fp64 = None
    if not args.no_fp64_compare and precision != "fp64" and args.krylov == "fgmres":
        s64 = Solver.from_workload(w, batch_max=B, precision="fp64", device=dev, maxit=args.maxit,
                                   cycle_type=args.cycle)
        u64 = s64.field(B)

        def step64():
            s64.set_contrast(d_f)
            _, a_ = s64.forward(d_th, out=u64)
            _, G_, _ = s64.misfit(u64, d_y, d_rec)
            _, b_ = s64.gradient(d_th, u64, G_)
            return a_ + b_

        step64()
        k64 = min(args.steps, 2)
        barrier()
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(s64.stream)
        inf64 = []
        for _ in range(k64):
            inf64 += step64()
        f1.record(s64.stream)
        torch.cuda.synchronize()
        barrier()
        ms64 = f0.elapsed_time(f1)
        if world > 1:
            import torch.distributed as dist
            t = torch.tensor([ms64], device=dev, dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms64 = float(t.item())
        v64 = world * 2 * B * k64 / (ms64 / 1e3)
        fp64 = {"value": round(v64, 3), "unit": UNIT, "steps": k64, "warmup": 1,
                "ms_per_step": round(ms64 / k64, 2), "speedup_of_mixed": round(value / v64, 2),
                "converged": all(i["converged"] for i in inf64),
                "worst_rel_residual": max(i["rel_residual"] for i in inf64),
                "iterations_mean": round(sum(i["iterations"] for i in inf64) / len(inf64), 1),
                "what": "plain FP64 form of the same step: FP64 multigrid cycle, native-FP64 Arnoldi FGMRES, "
                        "same restart, levels, sweeps and FP64 acceptance test"}
        s64.close()

    # ---- the same step with FP16 storage of the level-0 iterate and the preconditioned vectors
    # (MGH_PREC_MIXED16): one warm-up and at most three timed steps
    fp16 = None
    if not args.no_fp16_compare and precision == "mixed32" and args.krylov == "fgmres" and solver.arnoldi == "sstep":
        s16 = Solver.from_workload(w, batch_max=B, precision="mixed16", device=dev, maxit=args.maxit,
                                   cycle_type=args.cycle)
        u16 = s16.field(B)

        def step16():
            s16.set_contrast(d_f)
            _, a_ = s16.forward(d_th, out=u16)
            _, G_, _ = s16.misfit(u16, d_y, d_rec)
            _, b_ = s16.gradient(d_th, u16, G_)
            return a_ + b_

        step16()
        k16 = min(args.steps, 3)
        barrier()
        torch.cuda.synchronize()
        h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        h0.record(s16.stream)
        inf16 = []
        for _ in range(k16):
            inf16 += step16()
        h1.record(s16.stream)
        torch.cuda.synchronize()
        barrier()
        ms16 = h0.elapsed_time(h1)
        if world > 1:
            import torch.distributed as dist
            t = torch.tensor([ms16], device=dev, dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms16 = float(t.item())
        fp16 = {"value": round(world * 2 * B * k16 / (ms16 / 1e3), 3), "unit": UNIT, "steps": k16, "warmup": 1,
                "ms_per_step": round(ms16 / k16, 2), "converged": all(i["converged"] for i in inf16),
                "worst_rel_residual": max(i["rel_residual"] for i in inf16),
                "iterations_mean": round(sum(i["iterations"] for i in inf16) / len(inf16), 1),
                "what": "the same step with the level-0 iterate and the preconditioned vectors stored in FP16 "
                        "(MGH_PREC_MIXED16), FP32 arithmetic"}
        s16.close()

    if rank != 0:
        return

    # ---- roofline of the dominant kernel class (CUDA events over the timed region)
    cs = 16 if precision == "fp64" else 8
    N = solver.N
    engine = args.krylov if args.krylov in ("bicgstab", "idrs") else (solver.arnoldi if precision != "fp64" else "fp64")
    alg = algorithmic_bytes(prof, N, cs, prof["launches"], engine,
                            coarse_fraction(w.nx, w.ny, w.levels, 2 if args.cycle == "w" else 1),
                            zs=4 if precision == "mixed16" else cs, idr_s=args.idr_s)
    ms_cls = prof["ms"]
    # the dominant kernel: the class with the most time among those that are one kernel each (the
    # coarser multigrid levels and the per-RHS reductions are many small kernels)
    single = [k for k in ("vcycle_pre_l0", "vcycle_post_l0", "matvec_dots", "gs_update", "true_residual",
                          "x_update") if ms_cls.get(k, 0) > 0]
    dom = max(single, key=lambda k: ms_cls[k])
    peak, peak_kind = load_peaks()
    kernels = {}
    for k, v in ms_cls.items():
        if v <= 0:
            continue
        e = {"ms": round(v, 3), "share": round(v / sum(ms_cls.values()), 4), "launches": prof["launches"][k]}
        if k in alg:
            e["GBps"] = round(alg[k] / (v / 1e3) / 1e9, 1)
        kernels[k] = e
    vc_bytes = alg["vcycle_pre_l0"] + alg["vcycle_post_l0"]
    vc_ms = ms_cls["vcycle_pre_l0"] + ms_cls["vcycle_post_l0"]
    n_l = max(prof["launches"][dom], 1)
    if dom in alg:
        # every class is reported against its algorithmic bytes (fields read or written once per
        # launch) and the measured copy bandwidth
        achieved = alg[dom] / (ms_cls[dom] / 1e3) / 1e9
        roof = {"kernel": dom, "bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4),
                "traffic": captured_traffic(dom, w, precision, B, (tuned or {}).get("shape"),
                                            fused=prof["launches"].get("matvec_dots", 0) == 0),
                "peak_kind": peak_kind, "bytes_per_launch": round(alg[dom] / n_l)}
    else:
        roof = {"kernel": dom, "bound": "hbm", "achieved": None, "peak": peak, "unit": "GB/s", "frac": None,
                "traffic": None, "peak_kind": peak_kind}
    if dom == "gs_update" and engine == "sstep":
        # the method's arithmetic of the Gram sweep: 45 complex multiply-adds (8 flops each) per point and
        # cycle for m = 8, against the measured FP32 FMA rate (69.7 TFLOP/s on this GPU)
        nv = w.restart + 1
        flops = 8 * (nv * (nv + 1) // 2) * N * prof["gram_reads"] / nv
        roof["method_tflops"] = round(flops / (ms_cls[dom] / 1e3) / 1e12, 2)
    roof["vcycle_fine_GBps"] = round(vc_bytes / (vc_ms / 1e3) / 1e9, 1) if vc_ms > 0 else None
    roof["vcycle_fine_frac"] = round(vc_bytes / (vc_ms / 1e3) / 1e9 / peak, 4) if vc_ms > 0 else None
    vt_bytes = vc_bytes + alg.get("vcycle_coarse", 0.0)
    vt_ms = vc_ms + ms_cls.get("vcycle_coarse", 0.0)
    roof["vcycle_total_GBps"] = round(vt_bytes / (vt_ms / 1e3) / 1e9, 1) if vt_ms > 0 else None
    roof["vcycle_total_frac"] = round(vt_bytes / (vt_ms / 1e3) / 1e9 / peak, 4) if vt_ms > 0 else None
    step_bytes = sum(alg.values())
    roof["step_algorithmic_GBps"] = round(step_bytes / (sum(ms_cls.values()) / 1e3) / 1e9, 1)

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        try:
            cpu = cpu_baseline_record(args.workload, sample_steps=200)
        except Exception as ex:  # the baseline is reported, never required
            cpu = {"error": str(ex)[:200]}

    line = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 2), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"mixed32": "f32+f64", "mixed16": "f16-stored f32+f64"}.get(precision, "f64"), "data": "synthetic",
        "config": {"workload": args.workload, "grid": f"{w.nx}x{w.ny} ({w.nx_int}^2 + {w.abl}-cell layer)",
                   "angles_per_gpu": B, "angles_total": B * world, "precision": precision, "levels": w.levels, "nu": [w.nu1, w.nu2],
                   "restart": w.restart, "tol": w.tol, "krylov": args.krylov if args.krylov != "idrs" else f"idrs(s={args.idr_s})", "cycle": args.cycle.upper(), "arnoldi": solver.arnoldi if precision != "fp64" else "fp64", "shift": [w.shift_re, w.shift_im],
                   "step": (f"set_contrast + {B} forward solves + crop" if forward_only else
                            f"set_contrast + {B} forward + crop/sample/misfit + {B} adjoint solves + gradient"),
                   "solves_per_step": (1 if forward_only else 2) * B, "l2": "inputs larger than L2 (Krylov basis "
                   f"{B * (w.restart + 1) * N * 16 / 1e9:.1f} GB per GPU)", "parallelism": f"replicas x{world}",
                   "split": (f"{B} angles as {args.split} handles of about {-(-B // args.split)} on concurrent streams"
                             if args.split > 1 else None)},
        "roofline": roof,
        "kernels": kernels,
        "iterations": {"mean": round(sum(its) / len(its), 1), "min": min(its), "max": max(its)},
        "converged": conv, "worst_rel_residual": worst,
        "gpu_launches": int(launches),
        "fp64_same_accuracy": fp64,
        "fp16_storage": fp16,
        "autotuned": tuned,
        "clocks": clk,
        "e2e": e2e,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line))


# --------------------------------------------------------------------------- gradient descent
def descent_main(args, rank, world, local_rank):
    """Projected gradient descent f <- max(0, f - gamma g) on the data term, from f = 0, with the
    gradient of every step from the forward and adjoint solves of all angles (Prop. 1).  The
    step gamma is fixed after the first gradient so that the first update moves f by at most
    0.02 (the nonnegativity constraint of the MAP problem in Sec. V)."""
    import torch
    import workloads as W
    from paper_2107_03679_gb300 import Solver

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    w = W.WORKLOADS[args.workload]
    precision = args.precision or w.precision
    f_gt, _, th, rec = make_inputs(w)
    B = len(th)
    s = Solver.from_workload(w, batch_max=B, precision=precision, device=dev, maxit=20000, arnoldi=args.arnoldi)
    d_th = torch.from_numpy(th).to(dev)
    d_rec = torch.from_numpy(rec).to(dev)
    s.set_contrast(torch.from_numpy(f_gt).to(dev))
    u, _ = s.forward(d_th)
    y_clean = s.sample(u, d_rec)
    import workloads as Wm
    sigma = 0.01 * float(torch.sqrt((y_clean.abs() ** 2).mean()))
    y = y_clean + torch.from_numpy(Wm.complex_noise(tuple(y_clean.shape), sigma, 44)).to(dev)
    f = torch.zeros_like(torch.from_numpy(f_gt)).to(dev)
    losses, errs, its = [], [], []
    gamma = None
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for it in range(args.descent + 1):
        s.set_contrast(f)
        u, inf_f = s.forward(d_th, out=u)
        _, G, loss = s.misfit(u, y, d_rec)
        losses.append(loss)
        errs.append(float(torch.linalg.norm(f - torch.from_numpy(f_gt).to(dev)) / torch.linalg.norm(torch.from_numpy(f_gt).to(dev))))
        if it == args.descent:
            break
        g, inf_a = s.gradient(d_th, u, G)
        its.append(sum(i["iterations"] for i in inf_f + inf_a) / (2 * B))
        if gamma is None:
            gamma = 0.02 / float(g.abs().max())
        f = torch.clamp(f - gamma * g, min=0.0)
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    if rank == 0:
        print(json.dumps({"metric": "projected gradient descent on the data term", "workload": args.workload,
                          "precision": precision, "steps": args.descent, "gamma": gamma, "loss": losses,
                          "relative_error_to_ground_truth": errs, "mean_iterations_per_solve": its,
                          "seconds": round(sec, 2), "noise": "1% complex Gaussian (seed 44)"}))
    s.close()


# --------------------------------------------------------------------------- FBS reconstruction
def fbs_main(args, rank, world, local_rank):
    """Accelerated forward-backward splitting with nonnegativity + TV (Alg. 4) from f = 0 on the
    differentiation workload: each iteration draws `--subset` angles at random, runs their forward
    and adjoint solves for the data-term gradient, the TV proximal step (FGP on the dual) and the
    momentum step, all on the GPU.  The step gamma is fixed from the gradient of the first subset
    at f = 0 so that the first move changes f by at most 0.02; the TV weight is gamma tau =
    --tv-lam.  Reports the SNR of the refractive index n/n_b = sqrt(1 + f) per iteration."""
    import numpy as np
    import torch
    import workloads as W
    from paper_2107_03679_gb300 import Solver
    from paper_2107_03679_gb300.reconstruct import fbs, snr_db

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    w = W.WORKLOADS[args.workload if args.workload != "ellipses576" else "grad576"]
    precision = args.precision or w.precision
    f_gt, _, th, rec = make_inputs(w)
    Q = len(th)
    subsets = W.angle_subsets(Q, args.subset, args.fbs, seed=1000 + rank)
    B = max(len(sb) for sb in subsets)
    s = Solver.from_workload(w, batch_max=Q, precision=precision, device=dev, maxit=20000, arnoldi=args.arnoldi)
    d_th = torch.from_numpy(th).to(dev)
    d_rec = torch.from_numpy(rec).to(dev)
    d_gt = torch.from_numpy(f_gt).to(dev)
    s.set_contrast(d_gt)
    u, _ = s.forward(d_th)
    y_clean = s.sample(u, d_rec)
    sigma = 0.01 * float(torch.sqrt((y_clean.abs() ** 2).mean()))
    y = y_clean + torch.from_numpy(W.complex_noise(tuple(y_clean.shape), sigma, 44)).to(dev)
    f0 = torch.zeros_like(d_gt)
    # step from the first subset's gradient at f0 (not part of the timed loop)
    idx0 = torch.from_numpy(np.asarray(subsets[0])).to(dev)
    s.set_contrast(f0)
    u0, _ = s.forward(d_th.index_select(0, idx0))
    _, G0, _ = s.misfit(u0, y.index_select(0, idx0), d_rec)
    g0, _ = s.gradient(d_th.index_select(0, idx0), u0, G0)
    gamma = 0.02 / float(g0.abs().max())
    tau = args.tv_lam / gamma
    eta_gt = torch.sqrt(1.0 + d_gt)
    snr_db(torch.sqrt(1.0 + f0), eta_gt)   # first use of these torch kernels outside the timed loop
    snrs = []
    times = []
    ev = [torch.cuda.Event(enable_timing=True)]

    def cb(it, f, loss):
        e = torch.cuda.Event(enable_timing=True)
        e.record()
        ev.append(e)
        snrs.append(round(snr_db(torch.sqrt(1.0 + f), eta_gt), 3))

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ev[0].record()
    f, losses, infos = fbs(s, d_th, d_rec, y, f0, subsets, gamma, tau, prox_iters=args.prox_iters, callback=cb)
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    times = [ev[i].elapsed_time(ev[i + 1]) for i in range(len(ev) - 1)]
    # the backward step alone, timed on the solver's stream after the loop
    st = s.stream
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    buf = torch.empty_like(f)
    a.record(st)
    s.tv_prox(f, g0, gamma, args.tv_lam, args.prox_iters, out=buf)
    b.record(st)
    torch.cuda.synchronize()
    prox_ms = a.elapsed_time(b)
    n_int = w.nx_int * w.ny_int
    # w = fbar - gamma d (2 reads, 1 write), dual fields zeroed (5 writes), per iteration one pass
    # that reads w, the momentum point (p, q) and the last dual iterate (p, q) and writes the next
    # momentum point and dual iterate (5 + 4), and the final primal point (w, p, q read, 1 written)
    prox_bytes = 8.0 * n_int * (3 + 5 + args.prox_iters * 9 + 4)
    its = [sum(i["iterations"] for i in fw + adj) / max(1, len(fw) + len(adj)) for fw, adj in infos]
    if rank == 0:
        print(json.dumps({
            "metric": "accelerated FBS with TV (Alg. 4) on the data term", "workload": w.name,
            "precision": precision, "iterations": args.fbs, "angles": Q, "subset": args.subset,
            "gamma": gamma, "tau": tau, "tv_lam": args.tv_lam, "prox_iters": args.prox_iters,
            "loss": [round(x, 6) for x in losses], "snr_db": snrs,
            "ms_per_iteration": [round(t, 1) for t in times],
            "mean_iterations_per_solve": [round(x, 1) for x in its],
            "seconds": round(sec, 2),
            "tv_prox": {"ms": round(prox_ms, 3), "algorithmic_bytes": prox_bytes,
                        "GB_per_s": round(prox_bytes / prox_ms / 1e6, 1)},
            "noise": "1% complex Gaussian (seed 44)", "data": "synthetic"}))
    s.close()


# --------------------------------------------------------------------------- uneven batch
def uneven_main(args, rank, world, local_rank):
    """Four grids of different sizes solved together: one solver handle and one CUDA stream per
    grid, driven from one host thread each so that their kernels overlap on the GPU (multi.UnevenBatch);
    a step is set_contrast + forward + misfit + adjoint + gradient on every grid.  Timed with CUDA
    events on the caller's stream, which every grid's stream joins; the same step is then timed on
    the plain FP64 path."""
    import torch
    import workloads as W
    from paper_2107_03679_gb300.multi import UnevenBatch

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    precision = args.precision or "mixed32"
    ws = W.uneven_workloads()
    data = []
    for w in ws:
        f_gt, f_step, thetas, rec = make_inputs(w)
        data.append(dict(f_gt=torch.from_numpy(f_gt).to(dev), f=torch.from_numpy(f_step).to(dev),
                         th=torch.from_numpy(thetas).to(dev), rec=torch.from_numpy(rec).to(dev)))

    def measure(prec, steps, warmup):
        ub = UnevenBatch.from_workloads(ws, device=dev, precision=prec, maxit=50000, arnoldi=args.arnoldi)
        res = ub.forward([d["f_gt"] for d in data], [d["th"] for d in data])
        ys = [ub.solvers[i].sample(u, data[i]["rec"]) for i, (u, _) in enumerate(res)]
        outs = [s.field(d["th"].numel()) for s, d in zip(ub.solvers, data)]

        def step():
            return ub.data_term_gradient([d["f"] for d in data], [d["th"] for d in data], [d["rec"] for d in data],
                                         ys, outs)

        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        cur = torch.cuda.current_stream(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = ub.launch_count()
        e0.record(cur)
        per = None
        for _ in range(steps):
            per = step()
        e1.record(cur)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        launches = ub.launch_count() - l0
        ub.close()
        return ms, per, launches

    ms, per, launches = measure(precision, args.steps, args.warmup)
    solves = sum(2 * d["th"].numel() for d in data) * args.steps
    fp64 = None
    if not args.no_fp64_compare and precision != "fp64":
        k64 = 1   # one step without warm-up: the FP64 path takes minutes on the 864^2 and 2304^2 grids
        ms64, per64, _ = measure("fp64", k64, 0)
        v64 = sum(2 * d["th"].numel() for d in data) * k64 / (ms64 / 1e3)
        fp64 = {"value": round(v64, 3), "unit": UNIT, "steps": k64, "warmup": 0, "ms_per_step": round(ms64 / k64, 1),
                "speedup_of_mixed": round(solves / (ms / 1e3) / v64, 2),
                "per_grid_iterations_mean": [round(sum(i["iterations"] for i in fw + ad) / len(fw + ad), 1)
                                             for _, _, fw, ad in per64],
                "converged": all(i["converged"] for _, _, fw, ad in per64 for i in fw + ad)}
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": round(solves / (ms / 1e3), 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if precision == "mixed32" else precision,
        "data": "synthetic",
        "config": {"workload": "uneven", "grids": [f"{w.nx}x{w.ny}:{d['th'].numel()}" for w, d in zip(ws, data)],
                   "levels": [w.levels for w in ws], "precision": precision,
                   "step": "set_contrast + forward + misfit + adjoint + gradient on every grid",
                   "schedule": "one handle, stream and host thread per grid; each replays its restart cycles "
                               "from captured CUDA graphs",
                   "timing": "CUDA events on the caller's stream, which every grid's stream joins"},
        "gpu_launches": int(launches),
        "per_grid": [{"grid": f"{w.nx}x{w.ny}", "angles": d["th"].numel(),
                      "iterations_mean": round(sum(i["iterations"] for i in fw + ad) / len(fw + ad), 1),
                      "converged": all(i["converged"] for i in fw + ad)}
                     for w, d, (_, _, fw, ad) in zip(ws, data, per)],
        "fp64_same_accuracy": fp64,
    }
    print(json.dumps(line))


# --------------------------------------------------------------------------- multi-frequency batch
def multifreq_main(args, rank, world, local_rank):
    """One contrast at four illumination frequencies (3, 5, 6, 8 GHz scaled so that the highest has
    the workload's 10 points per wavelength) on the 512^2 + 32 grid, 60 angles each: one handle and
    stream per frequency, driven concurrently.  A step is the data term and its gradient summed
    over frequencies (set_contrast, forward, misfit, adjoint, gradient for every frequency and
    angle).  The same steps are also run one frequency after another for comparison."""
    import torch
    import workloads as W
    from paper_2107_03679_gb300.multi import MultiFrequency

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    base = W.WORKLOADS["ellipses576"]
    ws = W.multifrequency_workloads(base)
    precision = args.precision or base.precision
    f_gt, f_step, th, rec = make_inputs(base)
    B = len(th) if args.angles is None else args.angles
    th = th[:B]
    mf = MultiFrequency.from_workloads(ws, batch_max=B, device=dev, precision=precision, maxit=args.maxit,
                                       arnoldi=args.arnoldi, cycle_type=args.cycle)
    d_th = torch.from_numpy(th).to(dev)
    d_rec = torch.from_numpy(rec).to(dev)
    mf.set_contrast(torch.from_numpy(f_gt).to(dev))
    ys = [s.sample(u, d_rec) for s, (u, _) in zip(mf.solvers, mf.forward(d_th))]
    d_f = torch.from_numpy(f_step).to(dev)
    outs = [s.field(B) for s in mf.solvers]

    def concurrent_step():
        return mf.data_term_gradient(d_f, d_th, d_rec, ys, outs)

    def sequential_step():
        res = []
        for i, s in enumerate(mf.solvers):
            one = MultiFrequency([s]).data_term_gradient(d_f, d_th, d_rec, ys[i:i + 1], outs[i:i + 1])
            res.append(one)
        return res

    for _ in range(args.warmup):
        concurrent_step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        loss, grad, infos = concurrent_step()
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        sequential_step()
    torch.cuda.synchronize()
    sec_seq = time.perf_counter() - t0
    solves = 2 * B * len(ws) * args.steps
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": round(solves / sec, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(sec / args.steps * 1e3, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": {"mixed32": "f32+f64", "mixed16": "f16-stored f32+f64"}.get(precision, "f64"),
            "data": "synthetic",
            "config": {"workload": "multifreq576", "grid": f"{base.nx}x{base.ny}", "frequencies_GHz": [3, 5, 6, 8],
                       "points_per_wavelength": [round(w.ppw, 2) for w in ws], "angles": B,
                       "sweeps_per_level": [list(s.nu_levels) for s in mf.solvers],
                       "precision": precision, "cycle": args.cycle.upper(),
                       "step": "data term + gradient summed over frequencies (forward + adjoint solves)",
                       "timing": "host wall clock around all streams"},
            "sequential_value": round(solves / sec_seq, 3),
            "per_frequency": [{"ppw": round(w.ppw, 2),
                               "iterations_mean": round(sum(i["iterations"] for i in fw + ad) / len(fw + ad), 1),
                               "converged": all(i["converged"] for i in fw + ad)}
                              for w, (fw, ad) in zip(ws, infos)],
            "loss": loss}))
    mf.close()


def main(argv=None):
    args = parse_args(argv)
    if args.cpu_sample:
        cpu_sample_main(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if args.impl == "reference":
            dist.init_process_group("gloo")
        else:
            torch.cuda.set_device(local_rank)
            dist.init_process_group("nccl")
    try:
        if args.impl == "reference":
            reference_main(args, rank, world)
        elif args.workload == "uneven":
            uneven_main(args, rank, world, local_rank)
        elif args.workload == "multifreq576":
            multifreq_main(args, rank, world, local_rank)
        elif args.descent:
            descent_main(args, rank, world, local_rank)
        elif args.fbs:
            fbs_main(args, rank, world, local_rank)
        else:
            gpu_main(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
