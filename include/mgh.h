/*
 * mgh.h -- C ABI of the GB300 multigrid-preconditioned Helmholtz solver.
 *
 * The library solves, for a batch of incident plane waves that share one contrast, the
 * discretised scattered-field Helmholtz equation of the paper (Sec. II-A, Sec. IV-A)
 *
 *     A u_sc = b,   A = -lap_h - alpha * k^2 (1 + f_d),   b = k^2 f_d u_in,
 *
 * on the extended grid Omega_e = Omega + absorbing layer, with the five-point Laplacian and a
 * first-order Sommerfeld closure on the outer edge.  The solver is right-preconditioned
 * flexible GMRES(m) whose preconditioner is one multigrid cycle (Alg. 2) on the shifted
 * Laplacian K_kappa = -lap_h - kappa * alpha * k^2 (1 + f_d) (Sec. IV-B/C): damped Jacobi
 * smoothing (eq. dampedJ), full-weighting restriction, bilinear prolongation, re-discretised
 * coarse levels and an exact coarsest solve.  The gradient of the quadratic data term of
 * Sec. V in the contrast is obtained through one adjoint solve per illumination (Prop. 1).
 *
 * Conventions shared by every entry point
 *   - Complex numbers are interleaved (re, im) pairs of double (mgh_cdouble).
 *   - Every field is stored row-major [B][ny][nx] on the extended grid (nx = nx_int + 2*abl,
 *     ny = ny_int + 2*abl), x fastest: the unknown u_{m,n} is element n*nx + m (Sec. IV-A);
 *     interior-only arrays are [ny_int][nx_int] (or [B][ny_int][nx_int]).
 *   - Unless stated otherwise every data pointer is DEVICE memory owned by the caller; the
 *     library never frees it and never keeps it after the call returns.
 *   - Calls are asynchronous on the handle's CUDA stream (given at mgh_create), except that
 *     an entry point that returns host values (mgh_solve_info, a loss) synchronises that
 *     stream before returning.
 *   - Errors are reported by the return code only; nothing is thrown across the ABI.  On
 *     MGH_INVALID_ARG nothing was launched.  On MGH_CUDA_ERROR the handle should be destroyed.
 *   - A handle is not thread-safe: one host thread at a time per handle.
 *   - A handle belongs to the CUDA device that was current when mgh_create ran; every later call
 *     on it must be made with that device current (MGH_INVALID_ARG otherwise).  Handles on
 *     different devices may be used by one process.
 */
#ifndef MGH_H
#define MGH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { double re, im; } mgh_cdouble;

typedef enum {
  MGH_OK = 0,
  MGH_INVALID_ARG = 1,      /* bad size, null pointer, batch above batch_max, call order */
  MGH_NOT_CONVERGED = 2,    /* maxit reached for at least one right-hand side; best iterate kept */
  MGH_CUDA_ERROR = 3,       /* a CUDA call failed; the message is in mgh_last_error() */
  MGH_OUT_OF_MEMORY = 4,    /* device allocation failed at create */
  MGH_TIMEOUT = 5,          /* a kernel's bounded device-side wait (an mbarrier of a bulk-copy ring)
                               gave up and set the handle's device error word; the solve stops at
                               the next restart and the handle stays usable */
  MGH_NOT_SUPPORTED = 6     /* option not built into this library */
} mgh_status;

typedef enum {
  MGH_PREC_FP64 = 0,        /* everything in complex FP64 (the plain form) */
  MGH_PREC_MIXED32 = 1,     /* multigrid cycle in complex FP32 storage and arithmetic; the iterate,
                               right-hand side and restart residual in double-float (FP64-class),
                               every accepted iterate checked by the native-FP64 true residual; the
                               Krylov basis per `arnoldi` (double-float, native FP64, or FP32 for
                               the s-step cycles) */
  MGH_PREC_MIXED16 = 2      /* MGH_PREC_MIXED32 with FP16 storage on the fine level: the level-0
                               iterate between pre- and post-smoothing and the preconditioned
                               vectors Z are stored as complex FP16 (arithmetic stays FP32; the
                               level-0 cycle input is scaled by a power of two near sqrt(N)/16 so
                               that the stored values sit well inside FP16's normal range).  Needs
                               arnoldi = MGH_ARNOLDI_SSTEP, krylov = MGH_KRYLOV_FGMRES, an even
                               extended-grid width and at least one sweep before and after the
                               level-0 correction (MGH_NOT_SUPPORTED otherwise).  mgh_precondition
                               applies the FP32 cycle; FP16 storage is used inside solves */
} mgh_precision;

typedef enum {
  MGH_ARNOLDI_DF = 0,       /* mixed precision: Arnoldi vectors and Gram-Schmidt arithmetic in
                               double-float (pairs of FP32, ~48-bit significand) on the FP32 pipes */
  MGH_ARNOLDI_FP64 = 1,     /* native FP64 Gram-Schmidt (always used when precision is FP64) */
  MGH_ARNOLDI_SSTEP = 2     /* mixed precision, restart <= 8: each cycle builds the monomial basis
                               v_{k+1} = A M^{-1} v_k, stored and formed in FP32, orthogonalises it
                               at once by a Cholesky factor of its Gram matrix (FP32 running sums
                               of 32 products promoted to double-float, FP64 factor), and solves
                               the cycle's least-squares problem on that factor; one sweep over
                               the basis per cycle instead of two per step */
} mgh_arnoldi;

typedef enum {
  MGH_KRYLOV_FGMRES = 0,    /* right-preconditioned flexible GMRES(restart) (the target's method) */
  MGH_KRYLOV_BICGSTAB = 1,  /* right-preconditioned Bi-CGSTAB of Alg. 3 (the paper's method): two
                               multigrid cycles per iteration, FP64 vectors and inner products, the
                               cycle in the handle's precision; uses the GMRES workspace, so it needs
                               restart >= 5; `arnoldi` is ignored; iterations count cycles (2 per
                               Bi-CGSTAB iteration) */
  MGH_KRYLOV_IDRS = 2       /* right-preconditioned IDR(s) with biorthogonalisation (Sonneveld & van
                               Gijzen 2008; van Gijzen & Sonneveld 2011), s = idr_s: a short-
                               recurrence alternative to Bi-CGSTAB (s = 1 with the shadow vector r_0
                               is Bi-CGSTAB) whose step count grows less with the grid and does not
                               grow with an FP32 cycle on strongly scattering media.  One cycle and
                               one operator product per step; FP64 vectors and inner products, the
                               cycle in the handle's precision (FP64 or MIXED32; MIXED16 is
                               MGH_NOT_SUPPORTED); shadow space of random signs +-1 +-j from
                               MurmurHash3's 32-bit finaliser of the point index; omega raised to
                               keep |cos(A M^{-1} r, r)| >= 0.7.  Uses the GMRES workspace, so it
                               needs restart >= 2 idr_s + 2; `arnoldi` is ignored; iterations count
                               cycles, restarts count outer steps (s + 1 cycles each) */
} mgh_krylov;

#define MGH_MAX_LEVELS 12

/* Solver parameters.  Lengths are in the same unit as h (grid cells when h = 1). */
typedef struct {
  int nx_int, ny_int;       /* interior Omega size in grid points */
  int abl;                  /* absorbing-layer width L in cells, per side (Sec. IV-A) */
  double h;                 /* grid spacing */
  double k;                 /* background wavenumber k = k0 * eta_b */
  double beta;              /* layer strength: alpha = 1 + j*beta*(d/L)^2, d = distance to Omega in cells */
  double shift_re, shift_im;/* kappa of K_kappa (Sec. IV-B); (1, 0) is the unshifted operator */
  int levels;               /* multigrid levels including the finest, 2..12 (Alg. 2); the coarsest
                               level may hold at most 8192 unknowns (its dense inverse is kept) */
  int nu1, nu2;             /* pre- and post-relaxation sweeps, 0..4 (Alg. 2) */
  double omega;             /* damped-Jacobi weight omega_S in (0, 1] (eq. dampedJ) */
  int restart;              /* GMRES restart length m, 1..32 (1..20 with MGH_ARNOLDI_DF, 1..8 with
                               MGH_ARNOLDI_SSTEP) */
  int maxit;                /* maximum Arnoldi steps per right-hand side */
  double tol;               /* stop when ||b - A x||_2 <= tol * ||b||_2 (true FP64 residual) */
  int precision;            /* mgh_precision */
  int batch_max;            /* largest batch B any later call may use; sizes the workspace */
  int arnoldi;              /* mgh_arnoldi, used when precision is MGH_PREC_MIXED32 */
  int krylov;               /* mgh_krylov (default MGH_KRYLOV_FGMRES) */
  int cycle_type;           /* CycleType of Alg. 2: each level l < levels-1 runs cycle_type cycles of
                               level l+1 on its restricted residual, from a zero guess: 1 = V-cycle
                               (0 is read as 1), 2 = W-cycle, 3.  The coarsest solve is exact, so
                               it runs once per visit of the level above it */
  int nu_per_level;         /* 0: nu1 / nu2 on every level; 1: level l uses nu1_level[l] and
                               nu2_level[l] (0..4 each; Sec. III notes that the counts may differ
                               by level); entries from levels-1 on are ignored */
  int nu1_level[MGH_MAX_LEVELS];
  int nu2_level[MGH_MAX_LEVELS];
  int deflate;              /* FGMRES with deflated restarting (GMRES-DR, Morgan 2002; flexible form of
                               Giraud et al. 2010): k harmonic Ritz vectors of smallest modulus kept
                               across restarts, 0 = plain restarts (default), 1..min(restart-1, 16)
                               otherwise.  A cycle that ran its `restart` steps without converging
                               keeps V Q1 and Z P_k (P_k the harmonic Ritz vectors, Hbar P_k = Q1 R)
                               and continues Arnoldi at column k from the true residual
                               orthogonalised against them.  Needs krylov MGH_KRYLOV_FGMRES with the
                               native-FP64 Arnoldi: precision MGH_PREC_FP64, or MGH_PREC_MIXED32 with
                               arnoldi MGH_ARNOLDI_FP64 (MGH_NOT_SUPPORTED otherwise) */
  int idr_s;                /* shadow-space dimension s of MGH_KRYLOV_IDRS, 1..8 (default 4; read only
                               with that krylov) */
} mgh_params;

typedef struct {
  int iterations;           /* preconditioner applications: Arnoldi steps (FGMRES), cycles (Bi-CGSTAB, IDR(s)) */
  int restarts;             /* completed GMRES cycles; IDR(s): completed outer steps of s + 1 cycles */
  int converged;            /* 1 if the true relative residual reached tol */
  double rel_residual;      /* final true ||b - A x|| / ||b|| (0 when b = 0); a Bi-CGSTAB or IDR(s) solve stopped
                               by maxit between two true-residual checks reports its recursive residual */
} mgh_solve_info;

typedef struct mgh_handle mgh_handle;

/* Fill *p with the defaults (disk workload of 128^2 + 16, FP64, GMRES(20), 4 levels, 2+2 sweeps). */
void mgh_default_params(mgh_params* p);

/* Bytes of device memory mgh_create would allocate for these parameters. */
mgh_status mgh_workspace_bytes(const mgh_params* p, size_t* bytes);

/* Create a solver: validates p, allocates the hierarchy and Krylov workspace for p->batch_max
 * right-hand sides, and binds the handle to `cuda_stream` (a cudaStream_t; NULL = legacy
 * default stream).  The contrast starts at f_d = 0. */
mgh_status mgh_create(const mgh_params* p, void* cuda_stream, mgh_handle** out);

/* Free everything the handle owns.  NULL is ignored. */
void mgh_destroy(mgh_handle* h);

/* Set the contrast f_d = (n/n_b)^2 - 1 on Omega ([ny_int][nx_int] doubles, device) and rebuild
 * the operator and the multigrid hierarchy on the device (Sec. IV-A, Sec. IV-C): the fine
 * coefficient k^2 (1 + f_d) (k^2 in the layer), the coarse coefficients by full weighting with
 * the outer ring reset to k^2, the diagonals of A and of every K_kappa level, and the inverse
 * of the coarsest K_kappa (LU with partial pivoting). */
mgh_status mgh_set_contrast(mgh_handle* h, const double* f_d);

/* Incident plane waves u_in = exp(j k (x cos(theta) + y sin(theta))), x = m h, y = n h
 * (Sec. II-A); theta: B angles in radians (device); u_in: [B][ny][nx] (device). */
mgh_status mgh_incident_field(mgh_handle* h, const double* theta, int B, mgh_cdouble* u_in);

/* Right-hand sides b = k^2 f_d u_in for B angles (Sec. II-A, eq. HelmScatterRightIncident):
 * b: [B][ny][nx] (device), zero in the layer. */
mgh_status mgh_rhs(mgh_handle* h, const double* theta, int B, mgh_cdouble* b);

/* y = A x for B fields (Sec. IV-A five-point row with the Sommerfeld closure), FP64.
 * x, y: [B][ny][nx] (device), must not overlap. */
mgh_status mgh_apply(mgh_handle* h, const mgh_cdouble* x, int B, mgh_cdouble* y);

/* z = K_MG^{-1} b: one multigrid cycle with zero initial guess on K_kappa (Alg. 2, V-cycle),
 * computed in the handle's precision; b, z: [B][ny][nx] (device), FP64 in and out. */
mgh_status mgh_precondition(mgh_handle* h, const mgh_cdouble* b, int B, mgh_cdouble* z);

/* Exact solve with the coarsest-level operator (the last level of Alg. 2):
 * b, x: [B][ny_c][nx_c] (device), FP64; nx_c, ny_c from mgh_level_shape(levels-1). */
mgh_status mgh_coarse_solve(mgh_handle* h, const mgh_cdouble* b, int B, mgh_cdouble* x);

/* Shape and spacing of multigrid level `level` (0 = finest).  Host outputs; any may be NULL. */
mgh_status mgh_level_shape(const mgh_handle* h, int level, int* nx, int* ny, double* h_level);

/* Copy level `level`'s real coefficient k0^2 eta^2 ([ny_l][nx_l] doubles) to `c` (device). */
mgh_status mgh_level_coefficient(mgh_handle* h, int level, double* c);

/* Solve A x = b for B right-hand sides with FGMRES(m) + one multigrid cycle per step.
 * b: [B][ny][nx] (device); x: [B][ny][nx] (device), read as the initial guess and overwritten
 * with the solution; info: B host records or NULL.  Every right-hand side stops on its own
 * true FP64 residual.  A zero right-hand side gives x = 0 with 0 iterations.
 * Returns MGH_NOT_CONVERGED if any right-hand side hit maxit (x holds its last iterate). */
mgh_status mgh_solve(mgh_handle* h, const mgh_cdouble* b, int B, mgh_cdouble* x,
                     mgh_solve_info* info);

/* Forward model for B angles: u_sc = A^{-1} (k^2 f_d u_in(theta)) on Omega_e (Sec. II-A,
 * Sec. IV-A).  theta: B angles (device); u_sc: [B][ny][nx] (device, overwritten; the initial
 * guess is 0); info: B host records or NULL. */
mgh_status mgh_forward(mgh_handle* h, const double* theta, int B, mgh_cdouble* u_sc,
                       mgh_solve_info* info);

/* Truncate B fields from Omega_e to Omega (Sec. IV-A): u [B][ny][nx] -> u_int [B][ny_int][nx_int]. */
mgh_status mgh_crop(mgh_handle* h, const mgh_cdouble* u, int B, mgh_cdouble* u_int);

/* Receiver sampling S u: out[q][r] = u[q][rec[r]] for M receivers given as flat extended-grid
 * indices n*nx + m (device int64, each in [0, nx*ny)); out: [B][M] (device). */
mgh_status mgh_sample(mgh_handle* h, const mgh_cdouble* u, int B, const int64_t* rec, int M,
                      mgh_cdouble* out);

/* Adjoint of mgh_sample: G = S^T vals, i.e. G[q] = 0 except G[q][rec[r]] = vals[q][r]
 * (receivers must be distinct); vals: [B][M] (device), G: [B][ny][nx] (device, overwritten). */
mgh_status mgh_scatter(mgh_handle* h, const mgh_cdouble* vals, int B, const int64_t* rec, int M,
                       mgh_cdouble* G);

/* Data-term residual and adjoint source for L = 1/2 sum_q ||S u_q - y_q||^2 (Sec. V):
 * r = S u - y ([B][M], device), G = S^T r scattered on Omega_e ([B][ny][nx], device, zero
 * elsewhere; receivers must be distinct), and the loss L written to *loss_host (host, may be
 * NULL; when non-NULL the call synchronises the stream).  G is the gradient of L with respect
 * to u in PyTorch's complex convention (2 dL/d conj(u)). */
mgh_status mgh_misfit(mgh_handle* h, const mgh_cdouble* u, const mgh_cdouble* y, int B,
                      const int64_t* rec, int M, mgh_cdouble* r, mgh_cdouble* G, double* loss_host);

/* Gradient of a real loss L(u_sc) in the contrast f_d (Prop. 1): given G = 2 dL/d conj(u_sc)
 * on Omega_e ([B][ny][nx], device) for the B angles theta (device) and their scattered fields
 * u_sc ([B][ny][nx], device), solves A z_q = conj(G_q) with the same FGMRES engine (A is
 * complex symmetric) and writes grad[n][m] = k^2 sum_q Re(z_q u_q) on Omega, u_q = u_in,q +
 * u_sc,q ([ny_int][nx_int] doubles, device, overwritten).  info: B host records or NULL. */
mgh_status mgh_gradient(mgh_handle* h, const double* theta, const mgh_cdouble* u_sc,
                        const mgh_cdouble* G, int B, double* grad, mgh_solve_info* info);

/* The data term and its gradient in one call with HOST buffers (Sec. V, Prop. 1): for the contrast
 * f_d, the B angles theta and the receiver data y, set the contrast, solve the B forward problems,
 * form L = 1/2 sum_q ||S u_q - y_q||^2 and the residuals r = S u - y, solve the B adjoint problems and
 * write the gradient of L in f_d.  Every pointer argument is HOST memory (pinned memory makes the
 * copies asynchronous):
 *   f_d, grad   [ny_int][nx_int] doubles (in / out)
 *   theta       B angles; rec: M distinct receiver indices n*nx + m (int64); y: [B][M] complex (in)
 *   loss        one double (out); r: [B][M] complex (out, may be NULL)
 *   info_fwd, info_adj   B records each, or NULL
 * The work is the device-pointer sequence mgh_set_contrast, mgh_forward, mgh_misfit, mgh_gradient,
 * on device staging that the handle allocates on the first call (two fields of batch_max x N
 * complex values, and receiver buffers that grow with M) and keeps until mgh_destroy.  The call
 * returns when the results are on the host; MGH_NOT_CONVERGED if a forward or adjoint solve hit
 * maxit (the results are then those of the last iterates). */
mgh_status mgh_data_term_gradient_host(mgh_handle* h, const double* f_d, const double* theta, int B,
                                       const int64_t* rec, int M, const mgh_cdouble* y, double* grad, double* loss,
                                       mgh_cdouble* r, mgh_solve_info* info_fwd, mgh_solve_info* info_adj);

/* Backward step of the accelerated forward-backward splitting (Sec. V, Alg. 4): the proximal
 * operator of the nonnegativity constraint plus isotropic total variation with weight lam,
 *   out = argmin_{x >= 0} 1/2 ||x - w||^2 + lam TV(x),   w = fbar - gamma d,
 * TV(x) = sum_ij sqrt((x_ij - x_i+1,j)^2 + (x_ij - x_i,j+1)^2) with differences that are 0 across
 * the last row / column, computed by `iters` iterations of fast gradient projection on the dual
 * (Beck & Teboulle 2009; dual step 1/(8 lam), Nesterov momentum, the primal point of the last
 * dual iterate).  In Alg. 4, lam = gamma tau.
 *   fbar, d, out   [ny_int][nx_int] doubles (device); d may be NULL (w = fbar); out may alias
 *                  fbar or d (w is formed in the handle's workspace first)
 *   gamma          step of the gradient move (finite); lam >= 0 (lam = 0: out = max(w, 0))
 *   iters          >= 1 dual iterations
 * Queued on the handle's stream; no synchronisation, no allocation (the workspace of seven
 * interior fields is allocated by mgh_create). */
mgh_status mgh_tv_prox(mgh_handle* h, const double* fbar, const double* d, double gamma, double lam,
                       int iters, double* out);

/* Momentum step of Alg. 4: fbar = f + c (f - f_prev), c = (alpha_k - 1) / alpha_k+1 computed by the
 * caller.  f, f_prev, fbar: [ny_int][nx_int] doubles (device); fbar may alias f or f_prev. */
mgh_status mgh_fbs_momentum(mgh_handle* h, const double* f, const double* f_prev, double c, double* fbar);

/* Device-time profile of a handle.  Kernel classes (index into ms/launches):
 *   0 level-0 pre-smoothing + residual + restriction   5 second Gram-Schmidt pass
 *   1 level-0 prolongation + correction + smoothing    6 per-RHS reductions and Givens updates
 *   2 coarser levels and the coarsest solve            7 true residuals
 *   3 fused A z_j + Gram-Schmidt dots                   8 iterate updates x += Z y
 *   4 Gram-Schmidt update + re-orthogonalisation dots   9 everything else (set-up, right-hand sides, ...)
 * Counters let a caller turn times into bytes: every Arnoldi step runs one multigrid cycle, a
 * Gram-Schmidt pass at step j reads j+1 basis vectors. */
#define MGH_PROFILE_CLASSES 10
typedef struct {
  double ms[MGH_PROFILE_CLASSES];          /* summed device time, CUDA events on the handle's stream */
  uint64_t launches[MGH_PROFILE_CLASSES];  /* kernel launches per class */
  uint64_t arnoldi_steps;                  /* Arnoldi steps summed over right-hand sides */
  uint64_t basis_reads;                    /* sum over steps of j+1 (first pass) */
  uint64_t reorth_reads;                   /* sum over second passes of j+1 */
  uint64_t residuals;                      /* true residual evaluations, summed over right-hand sides */
  uint64_t updates;                        /* iterate updates, summed over right-hand sides */
  uint64_t update_reads;                   /* preconditioned vectors read by iterate updates */
  uint64_t cycle_steps;                    /* multigrid cycles + matvecs run, summed over right-hand sides
                                              (MGH_ARNOLDI_SSTEP runs every step of a cycle, also past
                                              the step that met the tolerance) */
  uint64_t gram_reads;                     /* basis vectors read by Gram sweeps (MGH_ARNOLDI_SSTEP) */
} mgh_profile;

/* Start (enable != 0) or stop recording; starting clears the profile.  While on, every launch
 * is bracketed by two CUDA events on the handle's stream. */
mgh_status mgh_profile_enable(mgh_handle* h, int enable);

/* Synchronise the handle's stream and return the profile accumulated since it was enabled. */
mgh_status mgh_profile_read(mgh_handle* h, mgh_profile* out);

/* Allocation-free variant of mgh_misfit (the paper has no counterpart: it is a service of this
 * library).  For callers that cannot allocate device memory: for example code whose device
 * memory is all handed out by a pool it does not own, or that must not call cudaMalloc because
 * cudaMalloc may synchronise the device.  No handle is needed and nothing is allocated: the
 * per-RHS partial losses live in a static device array of this library (32 KiB per GPU, held
 * until the process exits).
 *   nx, ny       extended grid size of the fields (u and G are [B][ny][nx])
 *   u, y, rec, M, r, G   as in mgh_misfit (device; r and G may be NULL; receivers distinct)
 *   B            1..4096 right-hand sides; larger B returns MGH_INVALID_ARG
 *   loss_dev     device double receiving 1/2 sum_q ||S u_q - y_q||^2
 *   cuda_stream  cudaStream_t the work is queued on (NULL = legacy default stream)
 * The first call on a device looks up the static array's device address (cudaGetSymbolAddress);
 * make that first call before any stream capture (a first call made while cuda_stream is being
 * captured returns MGH_INVALID_ARG and changes nothing).  All calls share the array: calls that
 * overlap on the GPU (different streams, no ordering between them) race on it. */
mgh_status mgh_misfit_noalloc(int nx, int ny, const mgh_cdouble* u, const mgh_cdouble* y, int B,
                              const int64_t* rec, int M, mgh_cdouble* r, mgh_cdouble* G,
                              double* loss_dev, void* cuda_stream);

/* Launch shapes of the FP32 multigrid level kernels (the paper has no counterpart: these are
 * choices of this implementation, for the autotuner).  They change only speed, never results. */
typedef struct {
  int wave_seg[MGH_MAX_LEVELS]; /* rows per warp segment of level l's wavefront kernels (rounded to
                               an even count the kernel's unroll period allows); 0 = the built-in
                               waves x steps model picks it for the level and batch */
  int wave_warps;           /* warps per block of the wavefront kernels: 2 or 4 */
  int wave_ring;            /* shared-memory row ring of the wavefront kernels in unroll periods:
                               1 or 2 */
  int tail_level;           /* first level of the one-kernel coarse tail; 0 = no tail (every level
                               by level kernels); -1 = the automatic choice (the finest level whose
                               fields fit one block's shared memory); a level whose fields do not
                               fit returns MGH_INVALID_ARG */
  int tail_cluster;         /* blocks per right-hand side of the coarse tail: 1 (one block), 2 or 4
                               (a thread-block cluster over bands of rows, halo rows exchanged
                               through distributed shared memory); 0 = automatic (the default): per
                               launch of B right-hand sides, 4 or else 2 when B such clusters fit on
                               the GPU at once, else 1; a count whose layout does not fit returns
                               MGH_INVALID_ARG */
} mgh_kernel_shape;

/* Current launch shapes of a handle (tail_level reports the level in use, 0 if none). */
mgh_status mgh_get_kernel_shape(const mgh_handle* h, mgh_kernel_shape* out);

/* Set the launch shapes for later calls; synchronises the handle's stream first.  MGH_PREC_MIXED16
 * handles need wave_warps = 4 and wave_ring = 1 (MGH_NOT_SUPPORTED otherwise). */
mgh_status mgh_set_kernel_shape(mgh_handle* h, const mgh_kernel_shape* s);

/* Test hook for the failure path of the bounded device-side waits (the paper has no counterpart).
 * The next mgh_solve / mgh_forward / mgh_gradient solve of this handle starts with the handle's
 * device error word set, exactly as a kernel whose bounded mbarrier wait gave up would leave it;
 * that solve returns MGH_TIMEOUT without running a cycle, and later calls work normally.  This
 * lets a test check the error-word -> MGH_TIMEOUT path without making any wait run out.  Only
 * handles whose solver polls the word: precision MGH_PREC_MIXED32, krylov MGH_KRYLOV_FGMRES,
 * arnoldi MGH_ARNOLDI_DF or MGH_ARNOLDI_SSTEP (MGH_NOT_SUPPORTED otherwise). */
mgh_status mgh_debug_inject_timeout(mgh_handle* h);

/* Host-side restart data of one deflated restart, exposed for tests (no device work; the solver
 * calls the same routine).  Inputs: Hbar, the (m+1) x m Arnoldi matrix of a cycle (row-major,
 * A Z = V Hbar), and c (m+1), the coefficients of the cycle's residual in V.  With g_1..g_k the
 * harmonic Ritz vectors of smallest harmonic Ritz value modulus -- eigenvectors of
 * H_m + |h_{m+1,m}|^2 f e_m^T with H_m^H f = e_m (Morgan 2002) -- and P = [[g_1..g_k; 0], c]
 * orthonormalised, the restart keeps V [C; 0] and Z C with C = P_k W (m x k, row-major), W a
 * k x k unitary chosen so that Hh = blockdiag(W, 1)^H P^H Hbar P_k W ((k+1) x k, row-major) is
 * upper Hessenberg; R (k x k, row-major, upper triangular), cs (k, real) and sn (k) are the Givens
 * QR of Hh (rotation i on rows i, i+1: [[cs_i, sn_i], [-conj(sn_i), cs_i]]).  2 <= m <= 32,
 * 1 <= k < m; all pointers host memory owned by the caller.  MGH_NOT_CONVERGED when the eigenvalue
 * iteration fails or a vector vanishes (the solver then restarts plainly). */
mgh_status mgh_debug_deflate(int m, int k, const mgh_cdouble* Hbar, const mgh_cdouble* c, mgh_cdouble* C,
                             mgh_cdouble* Hh, mgh_cdouble* R, double* cs, mgh_cdouble* sn);

/* Kernel launches issued by this handle since creation (or since the last reset). */
uint64_t mgh_launch_count(const mgh_handle* h, int reset);

/* Static description of a status code. */
const char* mgh_status_string(mgh_status s);

/* Message of the last failing CUDA call in this process ("" if none). */
const char* mgh_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* MGH_H */
