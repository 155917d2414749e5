// Internal host-side interface of the solver engine (not part of the C ABI).
#pragma once

#include <cuda.h>            // CUtensorMap (type only; the encoder is fetched at run time)
#include <cuda_runtime.h>
#include <cstddef>
#include <complex>
#include <cstdint>
#include <vector>

#include "mgh.h"
#include "mgh_common.cuh"

namespace mgh {

constexpr int kMaxLevels = 12;
constexpr int kMaxRestart = 32;
constexpr int kMaxRestartDf = 20;  // restart limit of the double-float Arnoldi (register budget)
constexpr int kMaxRestartSs = 8;   // restart limit of the s-step engine (Gram sums held in registers)
constexpr int kMaxDeflate = 16;    // harmonic Ritz vectors kept by a deflated restart
constexpr int kMaxIdrS = 8;        // shadow-space dimension limit of the IDR(s) engine

// Complex slots per block in the partial-sum buffer: two Gram-Schmidt regions of m + 2, or the
// (m + 1)(m + 2) / 2 entries of an s-step Gram matrix.
inline int partial_stride(int m) {
  const int a = 2 * m + 4, b = (m + 1) * (m + 2) / 2;
  return a > b ? a : b;
}
constexpr int kMaxSweeps = 4;
constexpr int kMaxCycleType = 3;   // CycleType of Alg. 2 (launches per cycle grow as CycleType^levels)
constexpr int kMaxCoarse = 8192;   // unknowns on the coarsest level (dense inverse kept on device: 1 GB in FP64)

// Device arrays of one multigrid level.  Coefficient and diagonals are shared by every
// right-hand side; the field buffers hold batch_max right-hand sides.
struct Level {
  int nx = 0, ny = 0, scale = 1;
  double h = 1.0;
  double* c = nullptr;       // real k0^2 eta^2 on this level (FP64 master copy)
  void* D = nullptr;         // complex diagonal of K_kappa, in the cycle precision
  void* wDinv = nullptr;     // omega / D, in the cycle precision
  void* b = nullptr;         // right-hand side of this level (levels >= 1)
  void* vpre = nullptr;      // iterate after pre-smoothing
  void* vfin = nullptr;      // iterate after post-smoothing (levels >= 1)
  void* wacc = nullptr;      // sum of the earlier cycles' corrections (CycleType >= 2, levels 1..L-2)
  size_t n() const { return (size_t)nx * ny; }
};

// Tensor maps of one FP32 multigrid level for the TMA level kernels (valid when *_ok).
struct LevelTma {
  bool pre_ok = false, post_ok = false;
  CUtensorMap pre_b, pre_w, pre_d;          // pre_b for levels >= 1
  CUtensorMap post_b, post_w, post_v, post_e;
};

struct Handle {
  mgh_params p{};
  cudaStream_t stream = nullptr;
  int device = -1;           // CUDA device current at mgh_create; every later call must run with it current
  int num_sms = 1;           // multiprocessors of the handle's device
  bool inject_timeout = false;  // test hook: the next double-float solve starts with the error word set
  int nx = 0, ny = 0;
  size_t N = 0;              // points of the extended grid
  size_t Np = 0;             // plane stride of double-float fields: N rounded up to 64 points
  int L = 0;                 // levels
  bool fp64 = true;          // cycle precision: double (true) or float (false)
  bool half = false;         // MGH_PREC_MIXED16: level-0 v_pre and the preconditioned vectors Z in FP16
  float zmul = 1.f;          // power-of-two scale of the level-0 cycle input when `half` (keeps the
                             // FP16 values near 1/16 in RMS: sqrt(N)/16, rounded to a power of two)
  bool vc_wave = true;       // FP32 levels: wavefront kernels (else shared-memory tiles)
  int wave_seg = 0;          // rows per warp segment of the wavefront kernels (0: automatic)
  int wave_seg_level[kMaxLevels] = {};  // per-level override of wave_seg (0: wave_seg's rule)
  int wave_min_nx = 0;       // levels narrower than this use the tiled kernels
  int wave_pf = 1;           // rows of loads in flight per warp (1 or 2; 16-byte path only)
  int wave_warps = 4;        // warps per block of the wavefront kernels (2 or 4)
  int wave_ring = 1;         // shared-memory row ring of the wavefront kernels, in unroll periods
                             // (1 or 2; 0: loads prefetched into registers)
  bool wave_lane_ring = true;  // rings filled per lane by cp.async (else by bulk copies)
  bool use_graphs = true;    // replay each restart cycle's launches from a captured CUDA graph
  int tail_l0 = 0;           // first level of the one-kernel coarse tail (0: every level by level kernels)
  int tail_cluster = 0;      // blocks per right-hand side of the tail (1, 2 or 4: a thread-block cluster;
                             // 0: per launch, the largest cluster whose launch fits the GPU at once)
  int tail_cap_l0 = -1;      // tail level tail_cap was queried for
  int tail_cap[5] = {};      // [2], [4]: clusters of that size the GPU holds at once
  // operator product of the s-step basis fused into the level-0 post kernel: the engine sets
  // fuse_v around one cycle; the post kernel launcher fuses when it can and reports its strips
  cf* fuse_v = nullptr;      // FP32 basis slot k+1 (hi plane) of right-hand side 0
  size_t fuse_vstride = 0;   // elements between right-hand sides
  int fuse_nstrips = 0;      // strips of the fused launch (0: not fused)
  bool fuse_ok = true;       // fusion allowed (MGH_FUSE_MATVEC=0 turns it off)
  bool gram8 = true;         // s-step Gram sweep by eight one-warp groups (MGH_GRAM8=0: four groups of 64)
  float* npart = nullptr;    // [Bmax][ny][strips] norm partials of the fused product
  cudaStream_t gstream = nullptr;  // non-blocking stream the cycle graphs are captured and replayed on
  cudaEvent_t gev_in = nullptr, gev_out = nullptr;  // order gstream after / before `stream`
  size_t csize = 16;         // bytes per complex of the cycle precision
  Level lev[kMaxLevels];
  bool contrast_set = false;

  // fine operator A (FP64)
  double* f_d = nullptr;     // [ny_int][nx_int] contrast (device copy)
  cd* DA = nullptr;          // diagonal of A
  float2* DAdf = nullptr;    // the same as double-float planes [2][Np] (hi, lo) for the mixed path
  float2* xdf = nullptr;     // [Bmax][2][Np] iterate of the mixed path in double-float
  float2* bdf = nullptr;     // [Bmax][2][Np] right-hand side of the mixed path in double-float

  // coarsest level: dense inverse, stored transposed (column c of K^{-1} contiguous)
  int nc = 0;
  cd* band = nullptr;        // banded LU workspace (FP64)
  int* piv = nullptr;
  cd* kinv64 = nullptr;      // [nc][nc] FP64 inverse, transposed (column c contiguous)
  cd* kinv64r = nullptr;     // [nc][nc] FP64 inverse, row-major
  cf* kinv32 = nullptr;      // [nc][nc] FP32 inverse, row-major (mixed precision)
  int* lu_info = nullptr;    // device status of the factorisation

  // Krylov workspace
  int m = 20;
  int Bmax = 1;
  cd* V = nullptr;           // [Bmax][m+1][N] Arnoldi basis (unnormalised; see vscale)
  void* Z = nullptr;         // [Bmax][m][N] preconditioned vectors, cycle precision
  cd* W = nullptr;           // [Bmax][N] A z_j
  cd* T1 = nullptr;          // [Bmax][N] scratch field (right-hand sides built by forward/gradient)
  cd* T2 = nullptr;          // [Bmax][N] scratch field
  cd* H = nullptr;           // [Bmax][m+1][m] Hessenberg matrix (column-major per RHS: H[j*(m+1)+i])
  cd* hcol = nullptr;        // [Bmax][m+1] dots of the current step
  cd* h2col = nullptr;       // [Bmax][m+1] re-orthogonalisation dots
  double* cs = nullptr;      // [Bmax][m] Givens cosines
  cd* sn = nullptr;          // [Bmax][m] Givens sines
  cd* g = nullptr;           // [Bmax][m+1] rotated right-hand side
  cd* y = nullptr;           // [Bmax][m] least-squares solution
  double* vscale = nullptr;  // [Bmax][m+1] multiplier that normalises V[b][i]
  RhsState* st = nullptr;    // [Bmax]
  RhsState* st_host = nullptr;  // pinned host mirror
  cd* hpend = nullptr;       // [Bmax][m+1] column j of H before its delayed correction (mixed path)
  cd* coef = nullptr;        // [Bmax][2m] Gram-Schmidt coefficients of the current step (mixed path)
  cd* partial = nullptr;     // [nblk*B][2m+4] block partial sums
  int nblk = 1;              // reduction blocks per right-hand side
  double* dscratch = nullptr;   // small FP64 scratch (loss)
  // device staging of the host-buffer entry point (allocated on its first call, grown with M)
  double* hs_f = nullptr;       // [ny_int][nx_int] contrast, then the gradient
  double* hs_theta = nullptr;   // [Bmax] angles
  cd* hs_u = nullptr;           // [Bmax][N] scattered fields
  cd* hs_G = nullptr;           // [Bmax][N] adjoint sources
  int64_t* hs_rec = nullptr;    // [hs_M] receivers
  cd* hs_y = nullptr;           // [Bmax][hs_M] data
  cd* hs_r = nullptr;           // [Bmax][hs_M] residuals at the receivers
  int hs_M = 0;
  // deflated restarting (p.deflate = k > 0): raw Arnoldi columns and the host's restart data
  cd* Hraw = nullptr;           // [Bmax][m][m+1] Hessenberg columns before the Givens rotations
  cd* drbuf = nullptr;          // [Bmax][dr_stride(m, k)] C, Hh, R, cs, sn of each right-hand side
  cd* g0 = nullptr;             // [Bmax][m+1] right-hand side of the cycle's least-squares problem
  int* dr_mode = nullptr;       // [Bmax] 0 none, 1 deflated restart, 2 plain restart from W
  cd* dr_hraw_host = nullptr;   // pinned host copies of Hraw, g0, y, drbuf and dr_mode
  cd* dr_g0_host = nullptr;
  cd* dr_y_host = nullptr;
  cd* dr_host = nullptr;
  int* dr_mode_host = nullptr;
  bool dr_force_plain = false;  // test hook (MGH_DEFLATE_FORCE_PLAIN=1): every deflated restart takes the
                                // plain-restart fallback, as when the host routine gives up
  double* tvbuf = nullptr;      // [7][ny_int][nx_int] TV proximal operator: w, the dual momentum
                                // point (p twice, q twice: ping-pong) and the last dual iterate (p, q)
  int* dev_err = nullptr;       // device error word written by kernels with bounded waits

  uint64_t launches = 0;

  // TMA tensor maps of the FP32 cycle (built at create when the encoder is available)
  LevelTma* tma = nullptr;        // [kMaxLevels]
  CUtensorMap* tma_in = nullptr;  // [2*m]: level-0 input (hi plane of basis slot j) for pre [j], post [m+j]
  bool tma_in_ok = false;

  // profiling (mgh_profile_enable): event pairs around launches, resolved at read time
  bool prof = false;
  std::vector<cudaEvent_t> ev;     // pool, two per recorded launch
  std::vector<int> ev_cls;         // class of each recorded pair
  size_t ev_used = 0;
  mgh_profile acc{};
};

// Sweeps of level l, the CycleType of Alg. 2 (0 is read as 1).
inline int nu_pre(const Handle& h, int l) { return h.p.nu_per_level ? h.p.nu1_level[l] : h.p.nu1; }
inline int nu_post(const Handle& h, int l) { return h.p.nu_per_level ? h.p.nu2_level[l] : h.p.nu2; }
inline int cycle_gamma(const Handle& h) { return h.p.cycle_type < 1 ? 1 : h.p.cycle_type; }

enum ProfClass { P_PRE0 = 0, P_POST0, P_COARSE, P_MATVEC_DOTS, P_UPDATE, P_REORTH, P_REDUCE, P_RESIDUAL,
                 P_XUPDATE, P_OTHER };

// Brackets the launches issued during its lifetime with CUDA events when profiling is on.
struct ProfScope {
  Handle& h;
  int slot = -1;
  ProfScope(Handle& hh, int cls);
  ~ProfScope();
};

// mgh_setup.cu
mgh_status setup_contrast(Handle& h, const double* f_d);
mgh_status launch_incident(Handle& h, const double* theta, int B, cd* out, bool times_contrast);
mgh_status launch_apply_A(Handle& h, const cd* x, int B, cd* y);
mgh_status launch_crop(Handle& h, const cd* u, int B, cd* out);
mgh_status launch_sample(Handle& h, const cd* u, int B, const int64_t* rec, int M, cd* out);
mgh_status launch_scatter(Handle& h, const cd* vals, int B, const int64_t* rec, int M, cd* G);
mgh_status launch_misfit(Handle& h, const cd* u, const cd* y, int B, const int64_t* rec, int M,
                         cd* r, cd* G, double* loss_dev);
mgh_status launch_conj(Handle& h, const cd* in, int B, cd* out);
mgh_status launch_gradient(Handle& h, const double* theta, const cd* u_sc, const cd* z, int B,
                           double* grad);
mgh_status launch_coarse_apply(Handle& h, const void* b, size_t b_stride, void* x,
                               size_t x_stride, int B, const RhsState* st, bool fp64_io);

// mgh_mg.cu: one multigrid cycle on B right-hand sides.
//   in      FP64 fine right-hand sides, rhs i at in + i*in_stride, each multiplied by
//           in_scale[i*scale_stride] when in_scale != nullptr
//   out     fine result, rhs i at out + i*out_stride, complex FP64 when out_fp64, otherwise
//           in the cycle precision
//   st      per-RHS state (a right-hand side with st[i].active == 0 is skipped) or nullptr
mgh_status vcycle(Handle& h, const cd* in, size_t in_stride, const double* in_scale,
                  size_t scale_stride, void* out, size_t out_stride, bool out_fp64, int B,
                  const RhsState* st);

// mgh_capi.cu: resolve the recorded event pairs of a synchronised stream into h.acc
mgh_status prof_flush(Handle& h);

// FP32 multigrid cycle whose level-0 input is an FP32 field (the hi plane of a double-float
// basis vector) scaled per RHS; output in FP32.
mgh_status vcycle_f32in(Handle& h, const cf* in, size_t in_stride, const double* in_scale,
                        size_t scale_stride, cf* out, size_t out_stride, int B, const RhsState* st,
                        int in_slot);
// Build the tensor maps of the FP32 level kernels (no-op when tensor maps are unavailable).
mgh_status build_vcycle_tma(Handle& h);

// mgh_krylov_df.cu: mixed-precision engine with double-float Arnoldi
mgh_status fgmres_df(Handle& h, const cd* b, int B, cd* x, mgh_solve_info* info);
mgh_status fgmres_ss(Handle& h, const cd* b, int B, cd* x, mgh_solve_info* info);
// device flag set by a kernel whose bounded wait gave up (0 = none)
constexpr int kErrTimeout = 1;

// mgh_tail.cu: every cycle of levels tail_l0 .. L-1 in one kernel, one block per right-hand side
// (input lev[tail_l0].b, output lev[tail_l0].vfin; reps cycles of level tail_l0, the first from 0)
int choose_tail_level(const Handle& h);
bool tail_level_fits(const Handle& h, int l);   // level l's tail fields fit one block's shared memory
bool tail_cluster_fits(const Handle& h, int l, int cl);   // the same for a tail over a cluster of cl blocks
mgh_status launch_tail(Handle& h, int reps, int B, const RhsState* st, bool fp64);

// mgh_inverse.cu: backward and momentum steps of the reconstruction loop (arguments checked by the caller)
mgh_status tv_prox(Handle& h, const double* fbar, const double* d, double gamma, double lam, int iters,
                   double* out);
mgh_status fbs_momentum(Handle& h, const double* f, const double* f_prev, double c, double* fbar);

// mgh_deflate.cu: restart data of one right-hand side for a deflated restart (row-major arrays:
// Hbar (m+1) x m and c (m+1) in; C m x k, Hh (k+1) x k, R k x k, cs k, sn k out); false when it
// cannot be formed
bool deflate_restart(int m, int k, const std::complex<double>* Hbar, const std::complex<double>* c,
                     std::complex<double>* C, std::complex<double>* Hh, std::complex<double>* R, double* cs,
                     std::complex<double>* sn);

// mgh_krylov.cu
mgh_status fgmres_solve(Handle& h, const cd* b, int B, cd* x, mgh_solve_info* info);
mgh_status bicgstab_solve(Handle& h, const cd* b, int B, cd* x, mgh_solve_info* info);
// mgh_idrs.cu: batched IDR(s) with biorthogonalisation (krylov MGH_KRYLOV_IDRS)
mgh_status idrs_solve(Handle& h, const cd* b, int B, cd* x, mgh_solve_info* info);

}  // namespace mgh
