"""Torch-facing wrapper of the C ABI: owns one solver handle and passes tensors to it.

Tensors are plumbing only (device memory and the CUDA stream); every operation is one C call
into libmgh.so.  Complex fields are torch.complex128 tensors (interleaved re/im doubles, the
layout of mgh_cdouble), shaped [B, ny, nx] on the extended grid.
"""
from __future__ import annotations

import numbers
from typing import Optional

import torch

from . import capi


def resolve_arnoldi(arnoldi: str, precision: str, restart: int, deflate: int = 0) -> str:
    """"auto": s-step cycles on the mixed path when the restart length allows them (m <= 8),
    otherwise the double-float Arnoldi; FP16 storage (mixed16) runs only with s-step cycles;
    deflated restarting runs on the native FP64 Gram-Schmidt; the FP64 path always runs native
    FP64 Gram-Schmidt."""
    if arnoldi != "auto":
        return arnoldi
    if precision == "mixed16":
        return "sstep"
    if precision != "mixed32":
        return "df"
    if deflate > 0:
        return "fp64"
    return "sstep" if restart <= 8 else "df"


def make_params(nx_int: int, ny_int: int, abl: int, h: float, k: float, beta: float = 0.15, shift=(1.0, 0.5),
                levels: int = 4, nu1=1, nu2=1, omega: float = 0.8, restart: int = 20, maxit: int = 5000,
                tol: float = 1e-6, precision: str = "mixed32", batch_max: int = 1, arnoldi: str = "auto",
                krylov: str = "fgmres", cycle_type=1, deflate: int = 0, idr_s: int = 4):
    """The mgh_params of a solver (host only) and the resolved Arnoldi engine.  nu1 / nu2: one
    count for every level, or one per level above the coarsest (per-level fields of mgh_params);
    deflate: harmonic Ritz vectors kept across FGMRES restarts (0 = plain restarts); idr_s: shadow
    dimension of krylov="idrs" (its workspace needs restart >= 2 idr_s + 2)."""
    p = capi.mgh_params()
    p.nx_int, p.ny_int, p.abl = nx_int, ny_int, abl
    p.h, p.k, p.beta = h, k, beta
    p.shift_re, p.shift_im = float(shift[0]), float(shift[1])
    p.levels, p.omega = levels, omega
    scalar = lambda v: isinstance(v, numbers.Integral)
    if scalar(nu1) and scalar(nu2):
        p.nu1, p.nu2 = int(nu1), int(nu2)
    else:
        n1 = [int(nu1)] * levels if scalar(nu1) else [int(v) for v in nu1]
        n2 = [int(nu2)] * levels if scalar(nu2) else [int(v) for v in nu2]
        if len(n1) < levels - 1 or len(n2) < levels - 1 or max(len(n1), len(n2)) > capi.MGH_MAX_LEVELS:
            raise ValueError("per-level sweeps need one count per level above the coarsest")
        p.nu1, p.nu2, p.nu_per_level = n1[0], n2[0], 1
        for l, v in enumerate(n1):
            p.nu1_level[l] = v
        for l, v in enumerate(n2):
            p.nu2_level[l] = v
    p.cycle_type = capi.CYCLES[cycle_type] if isinstance(cycle_type, str) else int(cycle_type)
    p.restart, p.maxit, p.tol = restart, maxit, tol
    p.precision = capi.PRECISIONS[precision]
    p.batch_max = batch_max
    resolved = resolve_arnoldi(arnoldi, precision, restart, deflate)
    p.arnoldi = capi.ARNOLDI[resolved]
    p.krylov = capi.KRYLOV[krylov]
    p.deflate = int(deflate)
    p.idr_s = int(idr_s)
    return p, resolved


class Solver:
    """Batched MG-preconditioned FGMRES solver for one discretised Helmholtz problem (Sec. IV)."""

    def __init__(self, nx_int: int, ny_int: int, abl: int, h: float, k: float, beta: float = 0.15,
                 shift=(1.0, 0.5), levels: int = 4, nu1: int = 1, nu2: int = 1, omega: float = 0.8,
                 restart: int = 20, maxit: int = 5000, tol: float = 1e-6, precision: str = "mixed32",
                 batch_max: int = 1, arnoldi: str = "auto", krylov: str = "fgmres", cycle_type: int = 1,
                 device: Optional[torch.device] = None, stream=None, deflate: int = 0, idr_s: int = 4):
        """nu1 / nu2: sweeps on every level, or a sequence with one count per level (the coarsest's
        is ignored); cycle_type: CycleType of Alg. 2 (1 = V, 2 = W, 3; or "v" / "w"); deflate:
        harmonic Ritz vectors kept across FGMRES restarts (GMRES-DR; 0 = plain restarts); idr_s:
        shadow dimension of krylov="idrs" (IDR(s); restart >= 2 idr_s + 2 sizes its workspace)."""
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        p, self.arnoldi = make_params(nx_int, ny_int, abl, h, k, beta, shift, levels, nu1, nu2, omega, restart, maxit,
                                      tol, precision, batch_max, arnoldi, krylov, cycle_type, deflate, idr_s)
        # (pre, post) sweeps of every level above the coarsest
        self.nu_levels = [(p.nu1_level[l], p.nu2_level[l]) if p.nu_per_level else (p.nu1, p.nu2)
                          for l in range(levels - 1)]
        self.krylov = krylov
        self.params = p
        self.precision = precision
        self.nx_int, self.ny_int, self.abl = nx_int, ny_int, abl
        self.nx, self.ny = nx_int + 2 * abl, ny_int + 2 * abl
        self.N = self.nx * self.ny
        self.h, self.k = h, k
        self.batch_max = batch_max
        with torch.cuda.device(self.device):
            self._h = capi.mgh_create(p, self.stream.cuda_stream)
        self._f_d = None

    @classmethod
    def from_workload(cls, w, batch_max: Optional[int] = None, precision: Optional[str] = None, **kw):
        args = dict(nx_int=w.nx_int, ny_int=w.ny_int, abl=w.abl, h=w.h, k=w.k, beta=w.beta,
                    shift=(w.shift_re, w.shift_im), levels=w.levels, nu1=w.nu1, nu2=w.nu2, omega=w.omega,
                    restart=w.restart, tol=w.tol, precision=precision or w.precision,
                    batch_max=batch_max or w.n_angles, krylov=getattr(w, "krylov", "fgmres"),
                    deflate=getattr(w, "deflate", 0), idr_s=getattr(w, "idr_s", 4))
        args.update(kw)
        return cls(**args)

    # ------------------------------------------------------------------ helpers
    def close(self):
        if getattr(self, "_h", None):
            capi.mgh_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def field(self, B: int) -> torch.Tensor:
        return torch.empty((B, self.ny, self.nx), dtype=torch.complex128, device=self.device)

    def _dev(self, t: torch.Tensor, dtype) -> torch.Tensor:
        t = t.to(device=self.device, dtype=dtype)
        return t.contiguous()

    def _B(self, t: torch.Tensor) -> int:
        B = t.shape[0] if t.dim() >= 1 else 1
        if B < 1 or B > self.batch_max:
            raise ValueError(f"batch {B} outside [1, {self.batch_max}]")
        return B

    # ------------------------------------------------------------------ operations
    def set_contrast(self, f_d: torch.Tensor) -> None:
        f = self._dev(f_d, torch.float64)
        if tuple(f.shape) != (self.ny_int, self.nx_int):
            raise ValueError(f"f_d must be [{self.ny_int}, {self.nx_int}]")
        capi.mgh_set_contrast(self._h, capi._ptr(f))
        self._f_d = f

    def incident_field(self, theta: torch.Tensor) -> torch.Tensor:
        th = self._dev(theta, torch.float64).reshape(-1)
        out = self.field(th.numel())
        capi.mgh_incident_field(self._h, capi._ptr(th), self._B(th), capi._ptr(out))
        return out

    def rhs(self, theta: torch.Tensor) -> torch.Tensor:
        th = self._dev(theta, torch.float64).reshape(-1)
        out = self.field(th.numel())
        capi.mgh_rhs(self._h, capi._ptr(th), self._B(th), capi._ptr(out))
        return out

    def apply(self, x: torch.Tensor) -> torch.Tensor:
        x = self._dev(x, torch.complex128)
        y = torch.empty_like(x)
        capi.mgh_apply(self._h, capi._ptr(x, numel=self.N), self._B(x), capi._ptr(y))
        return y

    def precondition(self, b: torch.Tensor) -> torch.Tensor:
        b = self._dev(b, torch.complex128)
        z = torch.empty_like(b)
        capi.mgh_precondition(self._h, capi._ptr(b, numel=self.N), self._B(b), capi._ptr(z))
        return z

    def level_shape(self, level: int):
        return capi.mgh_level_shape(self._h, level)

    def level_coefficient(self, level: int) -> torch.Tensor:
        nx, ny, _ = self.level_shape(level)
        c = torch.empty((ny, nx), dtype=torch.float64, device=self.device)
        capi.mgh_level_coefficient(self._h, level, capi._ptr(c))
        return c

    def coarse_solve(self, b: torch.Tensor) -> torch.Tensor:
        b = self._dev(b, torch.complex128)
        x = torch.empty_like(b)
        capi.mgh_coarse_solve(self._h, capi._ptr(b), self._B(b), capi._ptr(x))
        return x

    def solve(self, b: torch.Tensor, x0: Optional[torch.Tensor] = None):
        b = self._dev(b, torch.complex128)
        x = torch.zeros_like(b) if x0 is None else self._dev(x0, torch.complex128).clone()
        infos = capi.mgh_solve(self._h, capi._ptr(b, numel=self.N), self._B(b), capi._ptr(x))
        return x, infos

    def forward(self, theta: torch.Tensor, out: Optional[torch.Tensor] = None):
        th = self._dev(theta, torch.float64).reshape(-1)
        u = self.field(th.numel()) if out is None else out
        infos = capi.mgh_forward(self._h, capi._ptr(th), self._B(th), capi._ptr(u, torch.complex128))
        return u, infos

    def crop(self, u: torch.Tensor) -> torch.Tensor:
        u = self._dev(u, torch.complex128)
        B = self._B(u)
        out = torch.empty((B, self.ny_int, self.nx_int), dtype=torch.complex128, device=self.device)
        capi.mgh_crop(self._h, capi._ptr(u), B, capi._ptr(out))
        return out

    def sample(self, u: torch.Tensor, rec: torch.Tensor) -> torch.Tensor:
        u = self._dev(u, torch.complex128)
        rec = self._dev(rec, torch.int64)
        B = self._B(u)
        out = torch.empty((B, rec.numel()), dtype=torch.complex128, device=self.device)
        capi.mgh_sample(self._h, capi._ptr(u), B, capi._ptr(rec), rec.numel(), capi._ptr(out))
        return out

    def scatter(self, vals: torch.Tensor, rec: torch.Tensor) -> torch.Tensor:
        vals = self._dev(vals, torch.complex128)
        rec = self._dev(rec, torch.int64)
        B = self._B(vals)
        G = self.field(B)
        capi.mgh_scatter(self._h, capi._ptr(vals), B, capi._ptr(rec), rec.numel(), capi._ptr(G))
        return G

    def misfit(self, u: torch.Tensor, y: torch.Tensor, rec: torch.Tensor):
        """r = S u - y, G = S^T r, loss = 1/2 sum |r|^2 (Sec. V)."""
        u = self._dev(u, torch.complex128)
        y = self._dev(y, torch.complex128)
        rec = self._dev(rec, torch.int64)
        B = self._B(u)
        r = torch.empty((B, rec.numel()), dtype=torch.complex128, device=self.device)
        G = self.field(B)
        loss = capi.mgh_misfit(self._h, capi._ptr(u), capi._ptr(y), B, capi._ptr(rec), rec.numel(),
                               capi._ptr(r), capi._ptr(G))
        return r, G, loss

    def gradient(self, theta: torch.Tensor, u_sc: torch.Tensor, G: torch.Tensor):
        """grad f_d of a real loss with dL/du_sc = G (PyTorch convention), via one adjoint solve per angle."""
        th = self._dev(theta, torch.float64).reshape(-1)
        u_sc = self._dev(u_sc, torch.complex128)
        G = self._dev(G, torch.complex128)
        grad = torch.empty((self.ny_int, self.nx_int), dtype=torch.float64, device=self.device)
        infos = capi.mgh_gradient(self._h, capi._ptr(th), capi._ptr(u_sc), capi._ptr(G), self._B(th),
                                  capi._ptr(grad))
        return grad, infos

    def _interior(self, t: torch.Tensor, name: str, exact: bool = False) -> torch.Tensor:
        """A [ny_int][nx_int] float64 field on this device; `exact` (output buffers) refuses a copy."""
        if exact and (t.dtype != torch.float64 or t.device != self.device or not t.is_contiguous()):
            raise ValueError(f"{name} must be a contiguous float64 tensor on {self.device}")
        t = self._dev(t, torch.float64)
        if tuple(t.shape) != (self.ny_int, self.nx_int):
            raise ValueError(f"{name} must be [{self.ny_int}, {self.nx_int}]")
        return t

    def data_term_gradient_host(self, f_d: torch.Tensor, theta: torch.Tensor, rec: torch.Tensor, y: torch.Tensor,
                                grad_out: Optional[torch.Tensor] = None, r_out: Optional[torch.Tensor] = None,
                                want_infos: bool = False):
        """The data term and its gradient in one library call on HOST tensors (mgh_data_term_gradient_host):
        f_d [ny_int, nx_int] float64, theta [B] float64, rec [M] int64, y [B, M] complex128, all on the
        CPU (pinned memory makes the copies asynchronous).  Returns (loss, gradient [ny_int, nx_int]
        on the CPU, residuals S u - y [B, M] on the CPU, forward infos, adjoint infos)."""
        B, M = theta.numel(), rec.numel()
        self._B(theta.reshape(-1))
        nint = self.nx_int * self.ny_int
        grad = grad_out if grad_out is not None else torch.empty((self.ny_int, self.nx_int), dtype=torch.float64)
        r = r_out if r_out is not None else torch.empty((B, M), dtype=torch.complex128)
        loss, inf_f, inf_a = capi.mgh_data_term_gradient_host(
            self._h, capi._hptr(f_d, torch.float64, nint, "f_d"), capi._hptr(theta, torch.float64, B, "theta"), B,
            capi._hptr(rec, torch.int64, M, "rec"), M, capi._hptr(y, torch.complex128, B * M, "y"),
            capi._hptr(grad, torch.float64, nint, "grad"), capi._hptr(r, torch.complex128, B * M, "r"),
            want_infos=want_infos)
        return loss, grad, r, inf_f, inf_a

    def tv_prox(self, fbar: torch.Tensor, d: Optional[torch.Tensor], gamma: float, lam: float, iters: int,
                out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """argmin_{x >= 0} 1/2 ||x - (fbar - gamma d)||^2 + lam TV(x) by `iters` dual FGP iterations
        (the backward step of Alg. 4, Sec. V); d = None means w = fbar."""
        fbar = self._interior(fbar, "fbar")
        d = self._interior(d, "d") if d is not None else None
        out = torch.empty_like(fbar) if out is None else self._interior(out, "out", exact=True)
        capi.mgh_tv_prox(self._h, capi._ptr(fbar), capi._ptr(d) if d is not None else None, gamma, lam, iters,
                         capi._ptr(out))
        return out

    def fbs_momentum(self, f: torch.Tensor, f_prev: torch.Tensor, c: float,
                     out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """fbar = f + c (f - f_prev) (the momentum step of Alg. 4)."""
        f = self._interior(f, "f")
        f_prev = self._interior(f_prev, "f_prev")
        out = torch.empty_like(f) if out is None else self._interior(out, "out", exact=True)
        capi.mgh_fbs_momentum(self._h, capi._ptr(f), capi._ptr(f_prev), c, capi._ptr(out))
        return out

    def profile_enable(self, enable: bool = True) -> None:
        capi.mgh_profile_enable(self._h, enable)

    def profile_read(self) -> dict:
        return capi.mgh_profile_read(self._h)

    def launch_count(self, reset: bool = False) -> int:
        return capi.mgh_launch_count(self._h, reset)

    def kernel_shape(self) -> dict:
        """Launch shapes of the FP32 level kernels (wave_seg, wave_warps, wave_ring, tail_level,
        tail_cluster)."""
        return capi.mgh_get_kernel_shape(self._h)

    def set_kernel_shape(self, **shape) -> None:
        """Change launch shapes (speed only; see mgh_set_kernel_shape); unnamed fields keep their
        current values."""
        cur = self.kernel_shape()
        cur.update(shape)
        capi.mgh_set_kernel_shape(self._h, **cur)


class ScatteredField(torch.autograd.Function):
    """u_rec = S A(f_d)^{-1} (k^2 f_d u_in(theta)): receiver samples of the scattered fields.

    backward takes G_rec = dL/du_rec in PyTorch's complex convention, scatters it onto the grid
    (S^T), and returns dL/df_d from one adjoint solve per angle (Prop. 1), all in the CUDA library.
    """

    @staticmethod
    def forward(ctx, f_d: torch.Tensor, solver: Solver, theta: torch.Tensor, rec: torch.Tensor):
        solver.set_contrast(f_d.detach())
        u_sc, infos = solver.forward(theta)
        u_rec = solver.sample(u_sc, rec)
        ctx.solver = solver
        ctx.infos = infos
        ctx.save_for_backward(f_d.detach(), theta, u_sc, rec)
        return u_rec

    @staticmethod
    def backward(ctx, g_rec: torch.Tensor):
        f_d, theta, u_sc, rec = ctx.saved_tensors
        solver: Solver = ctx.solver
        solver.set_contrast(f_d)
        G = solver.scatter(g_rec.contiguous(), rec)
        grad, _ = solver.gradient(theta, u_sc, G)
        return grad.to(f_d.dtype), None, None, None


def scattered_field(f_d: torch.Tensor, solver: Solver, theta: torch.Tensor, rec: torch.Tensor) -> torch.Tensor:
    return ScatteredField.apply(f_d, solver, theta, rec)
