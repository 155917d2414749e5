"""ctypes binding of the C ABI in include/mgh.h (argument marshalling only).

Every function here has the name of the C entry point it calls and forwards device pointers
taken from torch tensors; all arithmetic happens in the CUDA library.  Importing this module
loads libmgh.so and raises if it is missing: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmgh.so")

MGH_OK, MGH_INVALID_ARG, MGH_NOT_CONVERGED, MGH_CUDA_ERROR, MGH_OUT_OF_MEMORY, MGH_TIMEOUT, MGH_NOT_SUPPORTED = range(7)
MGH_PREC_FP64, MGH_PREC_MIXED32, MGH_PREC_MIXED16 = 0, 1, 2
PRECISIONS = {"fp64": MGH_PREC_FP64, "mixed32": MGH_PREC_MIXED32, "mixed16": MGH_PREC_MIXED16}
MGH_ARNOLDI_DF, MGH_ARNOLDI_FP64, MGH_ARNOLDI_SSTEP = 0, 1, 2
ARNOLDI = {"df": MGH_ARNOLDI_DF, "fp64": MGH_ARNOLDI_FP64, "sstep": MGH_ARNOLDI_SSTEP}
MGH_KRYLOV_FGMRES, MGH_KRYLOV_BICGSTAB, MGH_KRYLOV_IDRS = 0, 1, 2
KRYLOV = {"fgmres": MGH_KRYLOV_FGMRES, "bicgstab": MGH_KRYLOV_BICGSTAB, "idrs": MGH_KRYLOV_IDRS}
MGH_MAX_LEVELS = 12
CYCLES = {"v": 1, "w": 2}


class mgh_params(ctypes.Structure):
    _fields_ = [
        ("nx_int", ctypes.c_int), ("ny_int", ctypes.c_int), ("abl", ctypes.c_int),
        ("h", ctypes.c_double), ("k", ctypes.c_double), ("beta", ctypes.c_double),
        ("shift_re", ctypes.c_double), ("shift_im", ctypes.c_double),
        ("levels", ctypes.c_int), ("nu1", ctypes.c_int), ("nu2", ctypes.c_int),
        ("omega", ctypes.c_double),
        ("restart", ctypes.c_int), ("maxit", ctypes.c_int), ("tol", ctypes.c_double),
        ("precision", ctypes.c_int), ("batch_max", ctypes.c_int), ("arnoldi", ctypes.c_int),
        ("krylov", ctypes.c_int), ("cycle_type", ctypes.c_int), ("nu_per_level", ctypes.c_int),
        ("nu1_level", ctypes.c_int * MGH_MAX_LEVELS), ("nu2_level", ctypes.c_int * MGH_MAX_LEVELS),
        ("deflate", ctypes.c_int), ("idr_s", ctypes.c_int),
    ]


class mgh_solve_info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("restarts", ctypes.c_int), ("converged", ctypes.c_int),
                ("rel_residual", ctypes.c_double)]


MGH_PROFILE_CLASSES = 10
PROFILE_CLASS_NAMES = ["vcycle_pre_l0", "vcycle_post_l0", "vcycle_coarse", "matvec_dots", "gs_update",
                       "gs_reorth", "reduce_givens", "true_residual", "x_update", "other"]


class mgh_profile(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * MGH_PROFILE_CLASSES), ("launches", ctypes.c_uint64 * MGH_PROFILE_CLASSES),
                ("arnoldi_steps", ctypes.c_uint64), ("basis_reads", ctypes.c_uint64),
                ("reorth_reads", ctypes.c_uint64), ("residuals", ctypes.c_uint64),
                ("updates", ctypes.c_uint64), ("update_reads", ctypes.c_uint64),
                ("cycle_steps", ctypes.c_uint64), ("gram_reads", ctypes.c_uint64)]


class mgh_kernel_shape(ctypes.Structure):
    _fields_ = [("wave_seg", ctypes.c_int * MGH_MAX_LEVELS), ("wave_warps", ctypes.c_int), ("wave_ring", ctypes.c_int),
                ("tail_level", ctypes.c_int), ("tail_cluster", ctypes.c_int)]


class MGHError(RuntimeError):
    def __init__(self, fn: str, status: int):
        msg = _lib.mgh_status_string(status).decode()
        extra = _lib.mgh_last_error().decode()
        super().__init__(f"{fn}: {msg}" + (f" [{extra}]" if extra and status == MGH_CUDA_ERROR else ""))
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build the CUDA library first "
            "(python -c 'import __graft_entry__ as g; g.build()'). There is no CPU fallback.")
    lib = ctypes.CDLL(LIB_PATH)
    P, I, D, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int
    pp = ctypes.POINTER(mgh_params)
    info_p = ctypes.POINTER(mgh_solve_info)
    sig = {
        "mgh_default_params": (None, [pp]),
        "mgh_workspace_bytes": (S, [pp, ctypes.POINTER(ctypes.c_size_t)]),
        "mgh_create": (S, [pp, P, ctypes.POINTER(P)]),
        "mgh_destroy": (None, [P]),
        "mgh_set_contrast": (S, [P, P]),
        "mgh_incident_field": (S, [P, P, I, P]),
        "mgh_rhs": (S, [P, P, I, P]),
        "mgh_apply": (S, [P, P, I, P]),
        "mgh_precondition": (S, [P, P, I, P]),
        "mgh_coarse_solve": (S, [P, P, I, P]),
        "mgh_level_shape": (S, [P, I, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(D)]),
        "mgh_level_coefficient": (S, [P, I, P]),
        "mgh_solve": (S, [P, P, I, P, info_p]),
        "mgh_forward": (S, [P, P, I, P, info_p]),
        "mgh_crop": (S, [P, P, I, P]),
        "mgh_sample": (S, [P, P, I, P, I, P]),
        "mgh_scatter": (S, [P, P, I, P, I, P]),
        "mgh_misfit": (S, [P, P, P, I, P, I, P, P, ctypes.POINTER(D)]),
        "mgh_misfit_noalloc": (S, [I, I, P, P, I, P, I, P, P, P, P]),
        "mgh_gradient": (S, [P, P, P, P, I, P, info_p]),
        "mgh_data_term_gradient_host": (S, [P, P, P, I, P, I, P, P, ctypes.POINTER(D), P, info_p, info_p]),
        "mgh_tv_prox": (S, [P, P, P, D, D, I, P]),
        "mgh_fbs_momentum": (S, [P, P, P, D, P]),
        "mgh_profile_enable": (S, [P, I]),
        "mgh_profile_read": (S, [P, ctypes.POINTER(mgh_profile)]),
        "mgh_debug_inject_timeout": (S, [P]),
        "mgh_debug_deflate": (S, [I, I, P, P, P, P, P, P, P]),
        "mgh_get_kernel_shape": (S, [P, ctypes.POINTER(mgh_kernel_shape)]),
        "mgh_set_kernel_shape": (S, [P, ctypes.POINTER(mgh_kernel_shape)]),
        "mgh_launch_count": (ctypes.c_uint64, [P, I]),
        "mgh_status_string": (ctypes.c_char_p, [S]),
        "mgh_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()

# names of the C entry points declared in include/mgh.h
EXPORTED = [
    "mgh_default_params", "mgh_workspace_bytes", "mgh_create", "mgh_destroy", "mgh_set_contrast",
    "mgh_incident_field", "mgh_rhs", "mgh_apply", "mgh_precondition", "mgh_coarse_solve",
    "mgh_level_shape", "mgh_level_coefficient", "mgh_solve", "mgh_forward", "mgh_crop", "mgh_sample",
    "mgh_scatter", "mgh_misfit", "mgh_misfit_noalloc", "mgh_gradient", "mgh_data_term_gradient_host", "mgh_tv_prox", "mgh_fbs_momentum", "mgh_profile_enable", "mgh_profile_read", "mgh_get_kernel_shape", "mgh_set_kernel_shape", "mgh_debug_inject_timeout", "mgh_debug_deflate", "mgh_launch_count", "mgh_status_string",
    "mgh_last_error",
]


def _check(fn: str, status: int, allow=(MGH_OK,)):
    if status not in allow:
        raise MGHError(fn, status)
    return status


def _ptr(t, dtype=None, numel=None, name="tensor"):
    """Device pointer of a contiguous CUDA tensor (checked dtype and size)."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor (device memory)")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if numel is not None and t.numel() < numel:
        raise ValueError(f"{name} has {t.numel()} elements, {numel} needed")
    return ctypes.c_void_p(t.data_ptr())


def _hptr(t, dtype, numel, name="tensor"):
    """Host pointer of a contiguous CPU tensor (checked dtype and size)."""
    import torch
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise ValueError(f"{name} must be a CPU torch.Tensor (host memory)")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if t.numel() < numel:
        raise ValueError(f"{name} has {t.numel()} elements, {numel} needed")
    return ctypes.c_void_p(t.data_ptr())


def mgh_default_params() -> mgh_params:
    p = mgh_params()
    _lib.mgh_default_params(ctypes.byref(p))
    return p


def mgh_workspace_bytes(p: mgh_params) -> int:
    n = ctypes.c_size_t(0)
    _check("mgh_workspace_bytes", _lib.mgh_workspace_bytes(ctypes.byref(p), ctypes.byref(n)))
    return int(n.value)


def mgh_create(p: mgh_params, stream) -> ctypes.c_void_p:
    h = ctypes.c_void_p(0)
    _check("mgh_create", _lib.mgh_create(ctypes.byref(p), ctypes.c_void_p(stream), ctypes.byref(h)))
    return h


def mgh_destroy(h) -> None:
    _lib.mgh_destroy(h)


def _infos(B):
    return (mgh_solve_info * B)()


def _infos_to_list(arr):
    return [dict(iterations=a.iterations, restarts=a.restarts, converged=bool(a.converged),
                 rel_residual=a.rel_residual) for a in arr]


def mgh_set_contrast(h, f_d):
    _check("mgh_set_contrast", _lib.mgh_set_contrast(h, f_d))


def mgh_incident_field(h, theta, B, u_in):
    _check("mgh_incident_field", _lib.mgh_incident_field(h, theta, B, u_in))


def mgh_rhs(h, theta, B, b):
    _check("mgh_rhs", _lib.mgh_rhs(h, theta, B, b))


def mgh_apply(h, x, B, y):
    _check("mgh_apply", _lib.mgh_apply(h, x, B, y))


def mgh_precondition(h, b, B, z):
    _check("mgh_precondition", _lib.mgh_precondition(h, b, B, z))


def mgh_coarse_solve(h, b, B, x):
    _check("mgh_coarse_solve", _lib.mgh_coarse_solve(h, b, B, x))


def mgh_level_shape(h, level):
    nx, ny, hl = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_double(0)
    _check("mgh_level_shape", _lib.mgh_level_shape(h, level, ctypes.byref(nx), ctypes.byref(ny), ctypes.byref(hl)))
    return nx.value, ny.value, hl.value


def mgh_level_coefficient(h, level, c):
    _check("mgh_level_coefficient", _lib.mgh_level_coefficient(h, level, c))


def mgh_solve(h, b, B, x, allow_not_converged=True):
    info = _infos(B)
    st = _lib.mgh_solve(h, b, B, x, info)
    _check("mgh_solve", st, (MGH_OK, MGH_NOT_CONVERGED) if allow_not_converged else (MGH_OK,))
    return _infos_to_list(info)


def mgh_forward(h, theta, B, u_sc, allow_not_converged=True):
    info = _infos(B)
    st = _lib.mgh_forward(h, theta, B, u_sc, info)
    _check("mgh_forward", st, (MGH_OK, MGH_NOT_CONVERGED) if allow_not_converged else (MGH_OK,))
    return _infos_to_list(info)


def mgh_crop(h, u, B, u_int):
    _check("mgh_crop", _lib.mgh_crop(h, u, B, u_int))


def mgh_sample(h, u, B, rec, M, out):
    _check("mgh_sample", _lib.mgh_sample(h, u, B, rec, M, out))


def mgh_scatter(h, vals, B, rec, M, G):
    _check("mgh_scatter", _lib.mgh_scatter(h, vals, B, rec, M, G))


def mgh_misfit(h, u, y, B, rec, M, r, G, want_loss=True):
    loss = ctypes.c_double(0.0)
    _check("mgh_misfit", _lib.mgh_misfit(h, u, y, B, rec, M, r, G, ctypes.byref(loss) if want_loss else None))
    return loss.value


def mgh_misfit_noalloc(nx, ny, u, y, B, rec, M, r, G, loss_dev, stream):
    _check("mgh_misfit_noalloc", _lib.mgh_misfit_noalloc(nx, ny, u, y, B, rec, M, r, G, loss_dev,
                                                         ctypes.c_void_p(stream)))


def mgh_gradient(h, theta, u_sc, G, B, grad, allow_not_converged=True):
    info = _infos(B)
    st = _lib.mgh_gradient(h, theta, u_sc, G, B, grad, info)
    _check("mgh_gradient", st, (MGH_OK, MGH_NOT_CONVERGED) if allow_not_converged else (MGH_OK,))
    return _infos_to_list(info)


def mgh_data_term_gradient_host(h, f_d, theta, B, rec, M, y, grad, r=None, want_infos=False,
                                allow_not_converged=True):
    """Host-buffer data term + gradient (pointers to host memory); returns (loss, infos_fwd, infos_adj)."""
    loss = ctypes.c_double(0.0)
    inf_f, inf_a = (_infos(B), _infos(B)) if want_infos else (None, None)
    st = _lib.mgh_data_term_gradient_host(h, f_d, theta, B, rec, M, y, grad, ctypes.byref(loss), r, inf_f, inf_a)
    _check("mgh_data_term_gradient_host", st, (MGH_OK, MGH_NOT_CONVERGED) if allow_not_converged else (MGH_OK,))
    return loss.value, (_infos_to_list(inf_f) if want_infos else None), (_infos_to_list(inf_a) if want_infos else None)


def mgh_tv_prox(h, fbar, d, gamma, lam, iters, out):
    _check("mgh_tv_prox", _lib.mgh_tv_prox(h, fbar, d, float(gamma), float(lam), int(iters), out))


def mgh_fbs_momentum(h, f, f_prev, c, fbar):
    _check("mgh_fbs_momentum", _lib.mgh_fbs_momentum(h, f, f_prev, float(c), fbar))


def mgh_profile_enable(h, enable=True):
    _check("mgh_profile_enable", _lib.mgh_profile_enable(h, 1 if enable else 0))


def mgh_profile_read(h) -> dict:
    p = mgh_profile()
    _check("mgh_profile_read", _lib.mgh_profile_read(h, ctypes.byref(p)))
    return dict(ms={n: p.ms[i] for i, n in enumerate(PROFILE_CLASS_NAMES)},
                launches={n: int(p.launches[i]) for i, n in enumerate(PROFILE_CLASS_NAMES)},
                arnoldi_steps=int(p.arnoldi_steps), basis_reads=int(p.basis_reads),
                reorth_reads=int(p.reorth_reads), residuals=int(p.residuals), updates=int(p.updates),
                update_reads=int(p.update_reads), cycle_steps=int(p.cycle_steps), gram_reads=int(p.gram_reads))


def mgh_get_kernel_shape(h) -> dict:
    """wave_seg: list of MGH_MAX_LEVELS per-level segment lengths (0 = the built-in model)."""
    out = mgh_kernel_shape()
    _check("mgh_get_kernel_shape", _lib.mgh_get_kernel_shape(h, ctypes.byref(out)))
    return {"wave_seg": list(out.wave_seg), "wave_warps": out.wave_warps, "wave_ring": out.wave_ring,
            "tail_level": out.tail_level, "tail_cluster": out.tail_cluster}


def mgh_set_kernel_shape(h, wave_seg=0, wave_warps: int = 4, wave_ring: int = 1, tail_level: int = -1,
                         tail_cluster: int = 0) -> None:
    """wave_seg: one length for every level, or a sequence of per-level lengths (0 = model)."""
    segs = [int(wave_seg)] * MGH_MAX_LEVELS if isinstance(wave_seg, int) else list(wave_seg)
    segs = (segs + [0] * MGH_MAX_LEVELS)[:MGH_MAX_LEVELS]
    s = mgh_kernel_shape((ctypes.c_int * MGH_MAX_LEVELS)(*segs), wave_warps, wave_ring, tail_level, tail_cluster)
    _check("mgh_set_kernel_shape", _lib.mgh_set_kernel_shape(h, ctypes.byref(s)))


def mgh_debug_inject_timeout(h) -> None:
    _check("mgh_debug_inject_timeout", _lib.mgh_debug_inject_timeout(h))


def mgh_debug_deflate(Hbar, c, k):
    """Restart data of one deflated restart from an (m+1) x m Arnoldi matrix and the residual
    coefficients c (host numpy arrays): returns (C m x k, Hh (k+1) x k, R k x k, cs k, sn k), the
    solver's host routine (see mgh_debug_deflate in include/mgh.h)."""
    import numpy as np
    Hb = np.ascontiguousarray(Hbar, dtype=np.complex128)
    cc = np.ascontiguousarray(c, dtype=np.complex128)
    m = Hb.shape[1]
    if Hb.shape != (m + 1, m) or cc.shape != (m + 1,):
        raise ValueError("Hbar must be (m+1) x m and c of length m+1")
    C = np.zeros((m, k), np.complex128)
    Hh = np.zeros((k + 1, k), np.complex128)
    R = np.zeros((k, k), np.complex128)
    cs = np.zeros(k, np.float64)
    sn = np.zeros(k, np.complex128)
    _check("mgh_debug_deflate", _lib.mgh_debug_deflate(m, k, Hb.ctypes.data, cc.ctypes.data, C.ctypes.data,
                                                       Hh.ctypes.data, R.ctypes.data, cs.ctypes.data,
                                                       sn.ctypes.data))
    return C, Hh, R, cs, sn


def mgh_launch_count(h, reset=False) -> int:
    return int(_lib.mgh_launch_count(h, 1 if reset else 0))


def mgh_status_string(s: int) -> str:
    return _lib.mgh_status_string(s).decode()


def mgh_last_error() -> str:
    return _lib.mgh_last_error().decode()
