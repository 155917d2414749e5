"""Several solver handles at once on one GPU: grids of different sizes (an uneven batch) or one
contrast at several illumination frequencies (Sec. VI-C reconstructs from four).

Each handle has its own CUDA stream and is driven from its own host thread (the C calls release
the GIL), so that the kernels of different handles overlap on the GPU: the coarse levels of one
handle, which cannot fill the GPU alone, run beside the fine levels of another.  This module only
orders library calls; all arithmetic is in the CUDA library.
"""
from __future__ import annotations

import threading
from typing import Callable, List, Optional, Sequence

import torch

from .solver import Solver
from .sweeps import smoothing_sweeps


def run_concurrently(solvers: Sequence[Solver], fn: Callable[[int, Solver], object]) -> list:
    """fn(i, solver) for every solver, each in its own host thread with the solver's stream as the
    current stream; returns the results in order and re-raises the first exception.  Every solver's
    stream first waits for the caller's current stream (whose work made the inputs), and on return
    the caller's current stream waits for every solver's stream.  Objects without a CUDA stream
    (stream None) are run in threads with no stream ordering."""
    cuda = all(getattr(s, "stream", None) is not None for s in solvers)
    if cuda:
        cur = torch.cuda.current_stream()
        for s in solvers:
            s.stream.wait_stream(cur)
    results: list = [None] * len(solvers)
    errors: list = [None] * len(solvers)

    def body(i: int, s):
        try:
            if cuda:
                with torch.cuda.device(s.device), torch.cuda.stream(s.stream):
                    results[i] = fn(i, s)
            else:
                results[i] = fn(i, s)
        except BaseException as e:  # re-raised in the caller's thread
            errors[i] = e

    threads = [threading.Thread(target=body, args=(i, s)) for i, s in enumerate(solvers)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    for e in errors:
        if e is not None:
            raise e
    if cuda:
        for s in solvers:
            cur.wait_stream(s.stream)
    return results


class MultiFrequency:
    """One contrast f_d on one grid, illuminated at several wavenumbers k_1..k_F: one handle per
    frequency (A and the multigrid hierarchy depend on k), all with the same angles and receivers.
    The data term is the sum over frequencies of 1/2 sum_q ||S u_sc,q - y_q||^2 and its gradient in
    f_d the sum of the per-frequency gradients (Prop. 1 for each k)."""

    def __init__(self, solvers: Sequence[Solver]):
        if not solvers:
            raise ValueError("at least one frequency")
        shapes = {(s.nx_int, s.ny_int, s.abl) for s in solvers}
        if len(shapes) != 1:
            raise ValueError("every frequency must use the same grid")
        self.solvers = list(solvers)

    @classmethod
    def from_workloads(cls, workloads, batch_max: int, device: Optional[torch.device] = None,
                       lfa_sweeps: bool = True, **kw):
        """One Solver per workload (see workloads.multifrequency_workloads), each on a new stream.
        With lfa_sweeps, each frequency's per-level sweep counts come from smoothing_sweeps (the
        same hierarchy meets a different k h on every level at every frequency)."""
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        out = []
        for w in workloads:
            stream = torch.cuda.Stream(dev)
            args = dict(kw)
            if lfa_sweeps:
                shift = complex(w.shift_re, w.shift_im)
                args.setdefault("nu1", smoothing_sweeps(w.k, w.h, w.levels, w.nu1, w.omega, shift))
                args.setdefault("nu2", smoothing_sweeps(w.k, w.h, w.levels, w.nu2, w.omega, shift))
            out.append(Solver.from_workload(w, batch_max=batch_max, device=dev, stream=stream, **args))
        return cls(out)

    @property
    def ks(self) -> List[float]:
        return [s.k for s in self.solvers]

    def close(self):
        for s in self.solvers:
            s.close()

    def set_contrast(self, f_d: torch.Tensor) -> None:
        run_concurrently(self.solvers, lambda i, s: s.set_contrast(f_d))

    def forward(self, theta: torch.Tensor, outs: Optional[List[torch.Tensor]] = None):
        """Scattered fields of every frequency: a list of ([B][ny][nx], infos)."""
        res = run_concurrently(self.solvers, lambda i, s: s.forward(theta, out=None if outs is None else outs[i]))
        cur = torch.cuda.current_stream()
        for u, _ in res:       # made on a solver's stream, used on the caller's
            u.record_stream(cur)
        return res

    def data_term_gradient(self, f_d: torch.Tensor, theta: torch.Tensor, rec: torch.Tensor, ys: Sequence[torch.Tensor],
                           outs: Optional[List[torch.Tensor]] = None):
        """Set the contrast, solve the forward and adjoint problems of every frequency and angle, and
        return (loss summed over frequencies, gradient summed over frequencies, per-frequency
        (forward infos, adjoint infos)).  ys[i]: [B][M] measurements of frequency i."""

        def one(i, s):
            s.set_contrast(f_d)
            u, inf_f = s.forward(theta, out=None if outs is None else outs[i])
            _, G, loss = s.misfit(u, ys[i], rec)
            g, inf_a = s.gradient(theta, u, G)
            return loss, g, (inf_f, inf_a)

        res = run_concurrently(self.solvers, one)
        cur = torch.cuda.current_stream()
        for _, g, _ in res:    # made on a solver's stream, used on the caller's
            g.record_stream(cur)
        grad = res[0][1]
        for _, g, _ in res[1:]:
            grad = grad + g
        return sum(r[0] for r in res), grad, [r[2] for r in res]


class SplitBatch:
    """One contrast at one frequency with the batch of illumination angles split over several
    handles of the same configuration, each with its own CUDA stream and host thread.  The angles
    are independent problems, so the results are those of one handle over all angles; what changes
    is the schedule: while one part runs the coarse levels of its multigrid cycle (short kernels
    that cannot fill the GPU), another part's fine-level kernels run beside them.  The data term
    and its gradient are sums over the parts (Prop. 1 sums over illuminations)."""

    def __init__(self, solvers: Sequence[Solver]):
        if not solvers:
            raise ValueError("at least one part")
        self.solvers = list(solvers)

    @classmethod
    def from_workload(cls, w, batch_max: int, parts: int = 2, device: Optional[torch.device] = None, **kw):
        """`parts` handles of w's configuration, each for at most ceil(batch_max / parts) angles and
        on a new stream."""
        if parts < 1 or parts > batch_max:
            raise ValueError("parts must be in [1, batch_max]")
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        per = -(-batch_max // parts)
        return cls([Solver.from_workload(w, batch_max=per, device=dev, stream=torch.cuda.Stream(dev), **kw)
                    for _ in range(parts)])

    @property
    def arnoldi(self) -> str:
        return self.solvers[0].arnoldi

    def close(self):
        for s in self.solvers:
            s.close()

    def launch_count(self) -> int:
        return sum(s.launch_count() for s in self.solvers)

    def ranges(self, n: int):
        """[start, stop) of every part's share of n angles (sizes differ by at most one)."""
        from .distributed import shard
        return [shard(n, i, len(self.solvers)) for i in range(len(self.solvers))]

    def data_term_gradient(self, f_d: torch.Tensor, theta: torch.Tensor, rec: torch.Tensor, y: torch.Tensor,
                           u_out: torch.Tensor, crop_out: Optional[torch.Tensor] = None):
        """Set the contrast, solve every angle's forward problem into u_out ([B][ny][nx]; cropped to
        the interior into crop_out when given), form the receiver misfit against y ([B][M]) and solve
        the adjoint problems; returns (loss, gradient in f_d, forward infos, adjoint infos), each over
        all B angles in order."""
        rs = self.ranges(theta.numel())

        def one(i, s):
            a, b = rs[i]
            s.set_contrast(f_d)
            u, inf_f = s.forward(theta[a:b], out=u_out[a:b])
            if crop_out is not None:
                crop_out[a:b].copy_(s.crop(u))
            _, G, loss = s.misfit(u, y[a:b], rec)
            g, inf_a = s.gradient(theta[a:b], u, G)
            return loss, g, inf_f, inf_a

        res = run_concurrently(self.solvers, one)
        if res[0][1].is_cuda:
            cur = torch.cuda.current_stream()
            for _, g, _, _ in res:   # made on a part's stream, used on the caller's
                g.record_stream(cur)
        grad = res[0][1]
        for _, g, _, _ in res[1:]:
            grad = grad + g
        return (sum(r[0] for r in res), grad, [i for r in res for i in r[2]], [i for r in res for i in r[3]])

    def profile_enable(self, enable: bool = True) -> None:
        for s in self.solvers:
            s.profile_enable(enable)

    def profile_read(self) -> dict:
        """The parts' profiles summed (class times add up across concurrent streams)."""
        out = None
        for s in self.solvers:
            p = s.profile_read()
            if out is None:
                out = {k: (dict(v) if isinstance(v, dict) else v) for k, v in p.items()}
                continue
            for k, v in p.items():
                if isinstance(v, dict):
                    for c, x in v.items():
                        out[k][c] = out[k].get(c, 0) + x
                else:
                    out[k] = out[k] + v
        return out


class UnevenBatch:
    """Grids of different sizes solved together (an uneven batch): one handle per grid, each with
    its own contrast, angles, stream and host thread, so that the kernels of all grids overlap on
    the GPU (each handle replays its own restart cycles from captured graphs).  The grids are
    independent problems; this class only orders library calls."""

    def __init__(self, solvers: Sequence[Solver]):
        if not solvers:
            raise ValueError("at least one grid")
        self.solvers = list(solvers)

    @classmethod
    def from_workloads(cls, workloads, device: Optional[torch.device] = None, precision: Optional[str] = None,
                       **kw):
        """One handle per workload (batch = its angle count), each on a new stream."""
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        return cls([Solver.from_workload(w, batch_max=w.n_angles, device=dev, stream=torch.cuda.Stream(dev),
                                         precision=precision or w.precision, **kw) for w in workloads])

    def close(self):
        for s in self.solvers:
            s.close()

    def launch_count(self) -> int:
        return sum(s.launch_count() for s in self.solvers)

    def forward(self, contrasts: Sequence[torch.Tensor], thetas: Sequence[torch.Tensor],
                outs: Optional[Sequence[torch.Tensor]] = None):
        """Set every grid's contrast and solve its forward problems: a list of (u, infos)."""
        def one(i, s):
            s.set_contrast(contrasts[i])
            return s.forward(thetas[i], out=None if outs is None else outs[i])

        res = run_concurrently(self.solvers, one)
        cur = torch.cuda.current_stream()
        for u, _ in res:       # made on a grid's stream, used on the caller's
            u.record_stream(cur)
        return res

    def data_term_gradient(self, contrasts: Sequence[torch.Tensor], thetas: Sequence[torch.Tensor],
                           recs: Sequence[torch.Tensor], ys: Sequence[torch.Tensor],
                           outs: Sequence[torch.Tensor]):
        """Per grid: set the contrast, forward solves into outs[i], misfit against ys[i], adjoint
        solves and the gradient; a list of (loss, gradient, forward infos, adjoint infos)."""
        def one(i, s):
            s.set_contrast(contrasts[i])
            u, inf_f = s.forward(thetas[i], out=outs[i])
            _, G, loss = s.misfit(u, ys[i], recs[i])
            g, inf_a = s.gradient(thetas[i], u, G)
            return loss, g, inf_f, inf_a

        res = run_concurrently(self.solvers, one)
        cur = torch.cuda.current_stream()
        for _, g, _, _ in res:
            g.record_stream(cur)
        return res
