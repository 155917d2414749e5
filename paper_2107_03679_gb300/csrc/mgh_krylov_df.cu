// Mixed-precision FGMRES engine: Arnoldi in double-float arithmetic on the FP32 pipes, with
// classical Gram-Schmidt whose second pass is delayed by one step (low-synchronisation GMRES;
// Swirydowicz et al. 2020, Bielich et al. 2022), so that each Arnoldi step reads the basis twice.
//
//   step j holds q_0..q_{j-1} (final, orthonormal), u_j (the candidate left by step j-1,
//   orthogonalised once) and, from the pass that wrote u_j, s = Q^H u_j and alpha = ||u_j||^2.
//   z_j = M^{-1}(u_j / ||u_j||), w = A z_j.
//   pass 1   one sweep: w = A z_j, t = Q^H w, beta = u_j^H w
//   scalars  nu = sqrt(alpha - ||s||^2); q_j = (u_j - Q s)/nu; h_{:,j} = (t, (beta - s^H t)/nu);
//            column j-1 is finalised with the correction s and h_{j,j-1} = nu, then rotated
//   pass 2   one sweep writes q_j over u_j and u_{j+1} = w - Q t - h_jj q_j, and accumulates
//            the next step's s' = [Q q_j]^H u_{j+1} and alpha' = ||u_{j+1}||^2
//
// The relation A z_j = sum_{i<=j+1} h_ij q_i holds exactly for the stored z_j, which is what
// flexible GMRES needs; the least-squares problem and the stopping estimate lag one step behind
// the preconditioner application.  At the end of a cycle the last column is finalised from the
// last pass 2's dots, with no extra sweep.
//
// Each block streams its contiguous chunk of points through a ring of shared-memory stages
// filled by bulk copies (TMA, cp.async.bulk) that complete on mbarriers, so loads of later tiles
// are in flight while the FP32 pipes work on the current one.  Double-float fields (basis
// vectors, w, the operator diagonal) are pairs of float2 planes (hi, lo) with plane stride Np.
#include <cuda_fp16.h>

#include <cmath>
#include <utility>

#include "mgh_df.cuh"
#include "mgh_krylov_common.cuh"
#include "mgh_tma.cuh"

namespace mgh {

namespace {

constexpr int kDfThreads = kTile;      // one point per thread per tile
constexpr int kMaxStages = 4;
constexpr int kMaxPlanes = 2 * kMaxRestartDf + 4;
constexpr int kSmemHeader = 512;      // mbarriers + plane pointer table, before the stage buffers
constexpr size_t kStageBudget = 96 * 1024;   // two blocks of 256 threads fit on one SM

// ---------------------------------------------------------------- double-float reductions
__device__ __forceinline__ df df_add(df a, df b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  df r;
  two_sum(s, e, r.hi, r.lo);
  return r;
}

__device__ __forceinline__ df warp_sum_df(df v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    df w;
    w.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
    w.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
    v = df_add(v, w);
  }
  return v;
}

// Stage buffer and pipeline bookkeeping of one block.
struct Pipe {
  uint64_t* bar;
  const float2** src;
  float2* buf;
  int S, P, ntiles;
  size_t p0, p1;

  __device__ __forceinline__ float2* plane(int slot, int p) const {
    return buf + ((size_t)slot * P + p) * kTile;
  }

  // Thread 0: queue the bulk copies of tile k into its slot.
  __device__ __forceinline__ void issue(int k) const {
    const int slot = k % S;
    const size_t start = p0 + (size_t)k * kTile;
    const int n = (int)((p1 - start) < (size_t)kTile ? (p1 - start) : (size_t)kTile);
    const uint32_t bytes = (uint32_t)(((n + 1) & ~1) * sizeof(float2));
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(&bar[slot], bytes * (uint32_t)P);
    for (int p = 0; p < P; ++p) bulk_load(plane(slot, p), src[p] + start, bytes, &bar[slot]);
  }
};

// Set up barriers and the first S tiles; returns the pipeline view of shared memory.
__device__ __forceinline__ Pipe pipe_begin(unsigned char* smem, int S, int P, size_t p0, size_t p1) {
  Pipe pp;
  pp.bar = reinterpret_cast<uint64_t*>(smem);
  pp.src = reinterpret_cast<const float2**>(smem + 64);
  pp.buf = reinterpret_cast<float2*>(smem + kSmemHeader);
  pp.S = S;
  pp.P = P;
  pp.p0 = p0;
  pp.p1 = p1;
  pp.ntiles = p1 > p0 ? (int)((p1 - p0 + kTile - 1) / kTile) : 0;
  return pp;
}

__device__ __forceinline__ void pipe_start(const Pipe& pp, int* fail) {
  if (threadIdx.x == 0) {
    for (int s = 0; s < pp.S; ++s) mbar_init(&pp.bar[s], 1);
    fence_mbar_init();
    *fail = 0;
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int k = 0; k < pp.S && k < pp.ntiles; ++k) pp.issue(k);
}

// Wait for tile k (each thread on its own, bounded).  A thread that gives up raises the block's
// failure flag; the flag is read by every thread after the next barrier (pipe_release).
__device__ __forceinline__ bool pipe_wait(const Pipe& pp, int k, int* fail) {
  const bool ok = mbar_wait(&pp.bar[k % pp.S], (uint32_t)((k / pp.S) & 1), kWaitLimitNs);
  if (!ok) *fail = 1;
  return ok;
}

// After all threads finished with tile k: refill its slot with tile k + S.  Returns false (for
// every thread together) if some thread's wait gave up: the block then drains the copies it
// still has in flight (bounded), raises the error word and must return.
__device__ __forceinline__ bool pipe_release(const Pipe& pp, int k, const int* fail, int* err) {
  __syncthreads();
  if (*fail) {
    if (threadIdx.x == 0) {
      atomicExch(err, kErrTimeout);
      for (int kk = k; kk < k + pp.S && kk < pp.ntiles; ++kk)
        mbar_wait(&pp.bar[kk % pp.S], (uint32_t)((kk / pp.S) & 1), kWaitLimitNs);
    }
    __syncthreads();
    return false;
  }
  if (threadIdx.x == 0 && k + pp.S < pp.ntiles) pp.issue(k + pp.S);
  return true;
}

// The same after all threads finished with tiles k and k + 1 (one barrier for both): refill their
// slots with tiles k + S and k + 1 + S.
__device__ __forceinline__ bool pipe_release2(const Pipe& pp, int k, const int* fail, int* err) {
  __syncthreads();
  if (*fail) {
    if (threadIdx.x == 0) {
      atomicExch(err, kErrTimeout);
      for (int kk = k; kk < k + pp.S && kk < pp.ntiles; ++kk)
        mbar_wait(&pp.bar[kk % pp.S], (uint32_t)((kk / pp.S) & 1), kWaitLimitNs);
    }
    __syncthreads();
    return false;
  }
  if (threadIdx.x == 0) {
    if (k + pp.S < pp.ntiles) pp.issue(k + pp.S);
    if (k + 1 + pp.S < pp.ntiles) pp.issue(k + 1 + pp.S);
  }
  return true;
}

__device__ __forceinline__ const float2* vplane(const float2* V, const KArgs& a, int rhs, int i, int h) {
  return V + (((size_t)rhs * (a.m + 1) + i) * 2 + h) * a.Np;
}

// Reduce `nv` df values per thread (vals[0..nv)) over the block and write them, converted to
// FP64, to out[dst(c)] for c < nv.  Static shared scratch of kMaxVals per warp.
constexpr int kMaxVals = 4 * kMaxRestartDf + 4;

template <typename Dst>
__device__ __forceinline__ void block_reduce_df(const df* vals, int nv, Dst dst) {
  __shared__ float2 sh[kDfThreads / 32][kMaxVals];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int c = 0; c < nv; ++c) {
    const df v = warp_sum_df(vals[c]);
    if (lane == 0) sh[warp][c] = make_float2(v.hi, v.lo);
  }
  __syncthreads();
  for (int c = threadIdx.x; c < nv; c += kDfThreads) {
    df acc = {sh[0][c].x, sh[0][c].y};
    for (int w = 1; w < kDfThreads / 32; ++w) acc = df_add(acc, df{sh[w][c].x, sh[w][c].y});
    *dst(c) = df_to_double(acc);
  }
}

// Partial-sum slots (per block, stride pstride = 2m+4):
//   region A (pass 1):  t = Q_j^H w at [0, j), beta = u_j^H w at j
//   region B (pass 2):  s = Q_{j+1}^H u_{j+1} at kB + [0, j+1), alpha = ||u_{j+1}||^2 at kB + j + 1
__host__ __device__ __forceinline__ int region_b(int m) { return m + 2; }

// ---------------------------------------------------------------- pass 1
// Planes: u_j (hi, lo), D_A (hi, lo), q_0 .. q_{j-1} (hi, lo each).
template <int NV>
__global__ void __launch_bounds__(kDfThreads)
k_df_pass1(KArgs a, int j, int S, const cf* __restrict__ Z, const float2* __restrict__ DAdf,
           const float2* __restrict__ V, float2* __restrict__ W, cd* __restrict__ partial,
           const RhsState* __restrict__ st, int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int rhs = blockIdx.y, blk = blockIdx.x;
  if (!st[rhs].active) return;
  const size_t p0 = (size_t)blk * a.chunk, p1 = (p0 + a.chunk < a.N) ? p0 + a.chunk : a.N;
  const int P = 4 + 2 * j;
  Pipe pp = pipe_begin(smem, S, P, p0, p1);
  if (threadIdx.x == 0) {
    pp.src[0] = vplane(V, a, rhs, j, 0);
    pp.src[1] = vplane(V, a, rhs, j, 1);
    pp.src[2] = DAdf;
    pp.src[3] = DAdf + a.Np;
    for (int i = 0; i < j; ++i) {
      pp.src[4 + 2 * i] = vplane(V, a, rhs, i, 0);
      pp.src[5 + 2 * i] = vplane(V, a, rhs, i, 1);
    }
  }
  int* fail = reinterpret_cast<int*>(smem + kSmemHeader - 16);
  pipe_start(pp, fail);
  const cf* z = Z + ((size_t)rhs * a.m + j) * a.N;
  float2* wh = W + (size_t)rhs * 2 * a.Np;
  float2* wl = wh + a.Np;
  const df ih = df_from_double(a.inv_h2);
  cdf t[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) t[i] = cdf_zero();
  cdf beta = cdf_zero();
  // the five stencil values of z for this thread's point of a tile (0 for missing neighbours,
  // which adds nothing to the neighbour sum); loaded one tile ahead of their use
  struct Stencil { cf c, w, e, s, n; };
  auto load_stencil = [&](int k, int m, int n) {
    Stencil v;
    v.c = v.w = v.e = v.s = v.n = mk<float>(0.f, 0.f);
    const size_t q = p0 + (size_t)k * kTile + threadIdx.x;
    if (k < pp.ntiles && q < p1) {
      v.c = z[q];
      if (m > 0) v.w = z[q - 1];
      if (m < a.nx - 1) v.e = z[q + 1];
      if (n > 0) v.s = z[q - a.nx];
      if (n < a.ny - 1) v.n = z[q + a.nx];
    }
    return v;
  };
  const unsigned q0 = (unsigned)(p0 + threadIdx.x);
  int n = (int)(q0 / (unsigned)a.nx);
  int m = (int)(q0 - (unsigned)n * (unsigned)a.nx);
  Stencil zs = load_stencil(0, m, n);
  for (int k = 0; k < pp.ntiles; ++k) {
    int mn = m + kTile, nn = n;
    while (mn >= a.nx) { mn -= a.nx; ++nn; }
    const Stencil zn = load_stencil(k + 1, mn, nn);
    const bool ready = pipe_wait(pp, k, fail);
    const int slot = k % S;
    const size_t q = p0 + (size_t)k * kTile + threadIdx.x;
    if (ready && q < p1) {
      df sr = {0.f, 0.f}, si = {0.f, 0.f};
      df_add1(sr, zs.w.re); df_add1(si, zs.w.im);
      df_add1(sr, zs.e.re); df_add1(si, zs.e.im);
      df_add1(sr, zs.s.re); df_add1(si, zs.s.im);
      df_add1(sr, zs.n.re); df_add1(si, zs.n.im);
      const cf zc = zs.c;
      const float2 dh = pp.plane(slot, 2)[threadIdx.x], dl = pp.plane(slot, 3)[threadIdx.x];
      cdf w = cdf_zero();
      // w = D z - (1/h^2) (sum of neighbours)
      df_fma1(w.re, dh.x, dl.x, zc.re);
      df_fma1(w.re, -dh.y, -dl.y, zc.im);
      df_fma1(w.im, dh.x, dl.x, zc.im);
      df_fma1(w.im, dh.y, dl.y, zc.re);
      df_fma(w.re, -ih.hi, -ih.lo, sr.hi, sr.lo);
      df_fma(w.im, -ih.hi, -ih.lo, si.hi, si.lo);
      w.re = df_norm(w.re);
      w.im = df_norm(w.im);
      wh[q] = make_float2(w.re.hi, w.im.hi);
      wl[q] = make_float2(w.re.lo, w.im.lo);
      const float2 uh = pp.plane(slot, 0)[threadIdx.x], ul = pp.plane(slot, 1)[threadIdx.x];
      cdf u;
      u.re.hi = uh.x; u.im.hi = uh.y; u.re.lo = ul.x; u.im.lo = ul.y;
      cdf_dot_acc(beta, u, w);
#pragma unroll
      for (int i = 0; i < NV; ++i) {
        if (i < j) {
          const float2 qh = pp.plane(slot, 4 + 2 * i)[threadIdx.x], ql = pp.plane(slot, 5 + 2 * i)[threadIdx.x];
          cdf qi;
          qi.re.hi = qh.x; qi.im.hi = qh.y; qi.re.lo = ql.x; qi.im.lo = ql.y;
          cdf_dot_acc(t[i], qi, w);
        }
      }
    }
    if (!pipe_release(pp, k, fail, err)) return;
    zs = zn;
    m = mn;
    n = nn;
  }
  df vals[2 * NV + 2];
#pragma unroll
  for (int i = 0; i < NV; ++i) { vals[2 * i] = t[i].re; vals[2 * i + 1] = t[i].im; }
  vals[2 * j] = beta.re;
  vals[2 * j + 1] = beta.im;
  cd* out = partial + ((size_t)rhs * a.nblk + blk) * a.pstride;
  block_reduce_df(vals, 2 * j + 2, [&](int c) -> double* { return reinterpret_cast<double*>(out + (c >> 1)) + (c & 1); });
}

// ---------------------------------------------------------------- scalars (one block per RHS)
// Delayed correction and Givens rotation of column j-1, stopping test, pass-2 coefficients.
// tail != 0 (j = m): only column m-1 is finalised, from the last pass 2's region B.
__global__ void k_df_scalars(KArgs a, int j, int tail, const cd* __restrict__ partial, cd* __restrict__ H,
                             double* __restrict__ cs, cd* __restrict__ sn, cd* __restrict__ g, cd* __restrict__ hpend,
                             cd* __restrict__ coef, RhsState* __restrict__ st, double tol, int maxit) {
  __shared__ cd shA[kMaxRestart + 2], shB[kMaxRestart + 2];
  const int rhs = blockIdx.x;
  if (!st[rhs].active) return;
  const int kB = region_b(a.m);
  const int nA = tail ? 0 : j + 1;      // t, beta
  const int nB = j >= 1 ? j + 1 : 0;    // s, alpha (from the previous pass 2)
  for (int c = threadIdx.x; c < nA + nB; c += blockDim.x) {
    const int slot = c < nA ? c : kB + (c - nA);
    cd acc = czero<double>();
    for (int b = 0; b < a.nblk; ++b) acc = acc + partial[((size_t)rhs * a.nblk + b) * a.pstride + slot];
    if (c < nA) shA[c] = acc; else shB[c - nA] = acc;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  const int m = a.m;
  RhsState& S = st[rhs];
  const cd* t = shA;
  const cd beta = tail ? czero<double>() : shA[j];
  const cd* s = shB;
  const double alpha = j >= 1 ? shB[j].re : S.rnorm * S.rnorm;
  double ss = 0.0;
  for (int i = 0; i < j; ++i) ss += cabs2(s[i]);
  const double nu2 = alpha - ss;
  const bool breakdown = !(nu2 > 1e-28 * alpha);
  const double nu = breakdown ? 0.0 : sqrt(nu2);
  if (j >= 1) {
    cd col[kMaxRestart + 1];
    const cd* pend = hpend + (size_t)rhs * (m + 1);
    for (int i = 0; i < j; ++i) col[i] = pend[i] + s[i];
    col[j] = mk<double>(nu, 0.0);
    const int c = j - 1;
    double* c_ = cs + (size_t)rhs * m;
    cd* s_ = sn + (size_t)rhs * m;
    for (int i = 0; i < c; ++i) {
      const cd tt = c_[i] * col[i] + s_[i] * col[i + 1];
      col[i + 1] = (-1.0 * cconj(s_[i])) * col[i] + c_[i] * col[i + 1];
      col[i] = tt;
    }
    const cd aa = col[c], bb = col[c + 1];
    double cc;
    cd sv;
    if (bb.re == 0.0 && bb.im == 0.0) { cc = 1.0; sv = czero<double>(); }
    else if (aa.re == 0.0 && aa.im == 0.0) { cc = 0.0; sv = mk<double>(1.0, 0.0); }
    else {
      const double na = sqrt(cabs2(aa)), rho = sqrt(cabs2(aa) + cabs2(bb));
      cc = na / rho;
      sv = (1.0 / (na * rho)) * (aa * cconj(bb));
    }
    col[c] = cc * col[c] + sv * col[c + 1];
    c_[c] = cc;
    s_[c] = sv;
    cd* gg = g + (size_t)rhs * (m + 1);
    gg[c + 1] = (-1.0 * cconj(sv)) * gg[c];
    gg[c] = cc * gg[c];
    cd* Hc = H + ((size_t)rhs * m + c) * (m + 1);
    for (int i = 0; i <= c; ++i) Hc[i] = col[i];
    S.iterations += 1;
    S.jend = j;
    const double est = sqrt(cabs2(gg[c + 1])) / S.bnorm;
    if (tail || !(est > tol) || S.iterations >= maxit || breakdown) { S.active = 0; return; }
  } else if (breakdown) {
    S.active = 0;
    S.jend = 0;
    return;
  }
  cd hjj = beta;
  for (int i = 0; i < j; ++i) hjj = hjj - cconj(s[i]) * t[i];
  hjj = (1.0 / nu) * hjj;
  cd* pend = hpend + (size_t)rhs * (m + 1);
  cd* cf_ = coef + (size_t)rhs * 2 * m;
  for (int i = 0; i < j; ++i) { pend[i] = t[i]; cf_[i] = s[i]; cf_[m + i] = t[i]; }
  pend[j] = hjj;
  S.inv_nu = 1.0 / nu;
  S.hjj_re = hjj.re;
  S.hjj_im = hjj.im;
  S.vsum += j;
}

// ---------------------------------------------------------------- pass 2
// Planes: u_j (hi, lo), w (hi, lo), q_0 .. q_{j-1}.  Writes q_j over u_j and u_{j+1} into slot
// j+1, and accumulates the next step's second-pass dots s' = Q_{j+1}^H u_{j+1} (q_j included)
// and alpha' = ||u_{j+1}||^2 into region B.
template <int NV>
__global__ void __launch_bounds__(kDfThreads)
k_df_pass2(KArgs a, int j, int S, const cd* __restrict__ coef, float2* __restrict__ V, const float2* __restrict__ W,
           cd* __restrict__ partial, const RhsState* __restrict__ st, int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int rhs = blockIdx.y, blk = blockIdx.x;
  const RhsState& SS = st[rhs];
  if (!SS.active) return;
  const size_t p0 = (size_t)blk * a.chunk, p1 = (p0 + a.chunk < a.N) ? p0 + a.chunk : a.N;
  const int P = 4 + 2 * j;
  Pipe pp = pipe_begin(smem, S, P, p0, p1);
  __shared__ cdf cs_[NV], ct_[NV];
  if (threadIdx.x == 0) {
    pp.src[0] = vplane(V, a, rhs, j, 0);
    pp.src[1] = vplane(V, a, rhs, j, 1);
    pp.src[2] = W + (size_t)rhs * 2 * a.Np;
    pp.src[3] = W + ((size_t)rhs * 2 + 1) * a.Np;
    for (int i = 0; i < j; ++i) {
      pp.src[4 + 2 * i] = vplane(V, a, rhs, i, 0);
      pp.src[5 + 2 * i] = vplane(V, a, rhs, i, 1);
    }
  }
  const cd* cf_ = coef + (size_t)rhs * 2 * a.m;
  for (int i = threadIdx.x; i < j; i += kDfThreads) {
    cs_[i] = cdf_from(cf_[i]);
    ct_[i] = cdf_from(cf_[a.m + i]);
  }
  int* fail = reinterpret_cast<int*>(smem + kSmemHeader - 16);
  pipe_start(pp, fail);   // its __syncthreads also publishes cs_/ct_
  const df inv_nu = df_from_double(SS.inv_nu);
  cdf hjj;
  hjj.re = df_from_double(SS.hjj_re);
  hjj.im = df_from_double(SS.hjj_im);
  float2* uh_g = V + (((size_t)rhs * (a.m + 1) + j) * 2) * a.Np;
  float2* ul_g = uh_g + a.Np;
  float2* nh_g = V + (((size_t)rhs * (a.m + 1) + j + 1) * 2) * a.Np;
  float2* nl_g = nh_g + a.Np;
  cdf sd[NV + 1];
#pragma unroll
  for (int i = 0; i <= NV; ++i) sd[i] = cdf_zero();
  df nrm = {0.f, 0.f};
  for (int k = 0; k < pp.ntiles; ++k) {
    const bool ready = pipe_wait(pp, k, fail);
    const int slot = k % S;
    const size_t q = p0 + (size_t)k * kTile + threadIdx.x;
    if (ready && q < p1) {
      const float2 a0 = pp.plane(slot, 0)[threadIdx.x], a1 = pp.plane(slot, 1)[threadIdx.x];
      const float2 b0 = pp.plane(slot, 2)[threadIdx.x], b1 = pp.plane(slot, 3)[threadIdx.x];
      cdf u, w;
      u.re.hi = a0.x; u.im.hi = a0.y; u.re.lo = a1.x; u.im.lo = a1.y;
      w.re.hi = b0.x; w.im.hi = b0.y; w.re.lo = b1.x; w.im.lo = b1.y;
#pragma unroll
      for (int i = 0; i < NV; ++i) {
        if (i < j) {
          const float2 qh = pp.plane(slot, 4 + 2 * i)[threadIdx.x], ql = pp.plane(slot, 5 + 2 * i)[threadIdx.x];
          cdf qi;
          qi.re.hi = qh.x; qi.im.hi = qh.y; qi.re.lo = ql.x; qi.im.lo = ql.y;
          cdf_sub_mul(u, cs_[i], qi);
          cdf_sub_mul(w, ct_[i], qi);
        }
      }
      u.re = df_norm(u.re);
      u.im = df_norm(u.im);
      cdf qj = cdf_zero();
      df_fma(qj.re, u.re.hi, u.re.lo, inv_nu.hi, inv_nu.lo);
      df_fma(qj.im, u.im.hi, u.im.lo, inv_nu.hi, inv_nu.lo);
      qj.re = df_norm(qj.re);
      qj.im = df_norm(qj.im);
      uh_g[q] = make_float2(qj.re.hi, qj.im.hi);
      ul_g[q] = make_float2(qj.re.lo, qj.im.lo);
      cdf_sub_mul(w, hjj, qj);
      w.re = df_norm(w.re);
      w.im = df_norm(w.im);
      nh_g[q] = make_float2(w.re.hi, w.im.hi);
      nl_g[q] = make_float2(w.re.lo, w.im.lo);
      cdf_abs2_acc(nrm, w);
      // second-pass dots of the new candidate against q_0 .. q_j
#pragma unroll
      for (int i = 0; i < NV; ++i) {
        if (i < j) {
          const float2 qh = pp.plane(slot, 4 + 2 * i)[threadIdx.x], ql = pp.plane(slot, 5 + 2 * i)[threadIdx.x];
          cdf qi;
          qi.re.hi = qh.x; qi.im.hi = qh.y; qi.re.lo = ql.x; qi.im.lo = ql.y;
          cdf_dot_acc(sd[i], qi, w);
        }
      }
      cdf_dot_acc(sd[NV], qj, w);
    }
    if (!pipe_release(pp, k, fail, err)) return;
  }
  df vals[2 * NV + 3];
#pragma unroll
  for (int i = 0; i < NV; ++i) { vals[2 * i] = sd[i].re; vals[2 * i + 1] = sd[i].im; }
  // compact: dots with q_0..q_{j-1}, then q_j, then alpha'
  vals[2 * j] = sd[NV].re;
  vals[2 * j + 1] = sd[NV].im;
  vals[2 * j + 2] = nrm;
  cd* out = partial + ((size_t)rhs * a.nblk + blk) * a.pstride + region_b(a.m);
  block_reduce_df(vals, 2 * j + 3, [&](int c) -> double* {
    if (c == 2 * j + 2) { out[j + 1].im = 0.0; return reinterpret_cast<double*>(out + j + 1); }
    return reinterpret_cast<double*>(out + (c >> 1)) + (c & 1);
  });
}

// 1/||u_{j+1}|| for the next preconditioner input (alpha' of region B).
__global__ void k_df_unorm(KArgs a, int j, const cd* __restrict__ partial, double* __restrict__ vscale,
                           const RhsState* __restrict__ st) {
  const int rhs = blockIdx.x;
  if (!st[rhs].active || threadIdx.x != 0) return;
  double n2 = 0.0;
  const int slot = region_b(a.m) + j + 1;
  for (int b = 0; b < a.nblk; ++b) n2 += partial[((size_t)rhs * a.nblk + b) * a.pstride + slot].re;
  vscale[(size_t)rhs * (a.m + 1) + j + 1] = n2 > 0.0 ? 1.0 / sqrt(n2) : 1.0;
}

// FP64 fields [B][N] -> double-float planes [B][2][Np].
__global__ void k_df_split(const cd* __restrict__ a, float2* __restrict__ out, size_t N, size_t Np) {
  const size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (q >= N) return;
  const int rhs = blockIdx.y;
  const cdf v = cdf_from(a[rhs * N + q]);
  float2* h = out + (size_t)rhs * 2 * Np;
  h[q] = make_float2(v.re.hi, v.im.hi);
  h[q + Np] = make_float2(v.re.lo, v.im.lo);
}

// Double-float planes -> FP64 x (every RHS when all != 0, else those awaiting verification).
__global__ void k_df_join(const float2* __restrict__ xdf, cd* __restrict__ x, size_t N, size_t Np,
                          const RhsState* __restrict__ st, int all) {
  const size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  const int rhs = blockIdx.y;
  if (q >= N || (!all && !st[rhs].verify)) return;
  if (st[rhs].bnorm == 0.0) { x[rhs * N + q] = czero<double>(); return; }   // b = 0 gives x = 0
  const float2* h = xdf + (size_t)rhs * 2 * Np;
  const float2 a = h[q], b = h[q + Np];
  x[rhs * N + q] = mk<double>((double)a.x + (double)b.x, (double)a.y + (double)b.y);
}

__device__ __forceinline__ cdf load_df(const float2* __restrict__ h, size_t Np, size_t q) {
  const float2 a = h[q], b = h[q + Np];
  cdf r;
  r.re.hi = a.x; r.im.hi = a.y; r.re.lo = b.x; r.im.lo = b.y;
  return r;
}

// r = b - A x in double-float (x, b double-float planes), written as the candidate u_0 in basis
// slot 0 (its lo plane only when `write_lo`: the s-step engine reads the FP32 hi plane); partial
// ||r||^2 (slot 0) and, on the first cycle, ||b||^2 (slot 1, double-float: it sets the acceptance
// threshold).  ||r||^2 is summed in FP32 per thread (FP64 across threads): it only scales the
// first basis vector and decides when the FP64 true residual, which decides acceptance, is checked.
__global__ void __launch_bounds__(kKThreads)
k_df_residual(KArgs a, const float2* __restrict__ bdf, const float2* __restrict__ xdf, const float2* __restrict__ DAdf,
              float2* __restrict__ V, cd* __restrict__ partial, const RhsState* __restrict__ st, int first,
              int write_lo) {
  const int rhs = blockIdx.y, blk = blockIdx.x;
  if (st[rhs].done) return;
  const float2* xb = xdf + (size_t)rhs * 2 * a.Np;
  const float2* bb = bdf + (size_t)rhs * 2 * a.Np;
  float2* rh = V + ((size_t)rhs * (a.m + 1) * 2) * a.Np;
  float2* rl = rh + a.Np;
  const df ih = df_from_double(a.inv_h2);
  float rn = 0.f;
  df bn = {0.f, 0.f};   // ||b||^2 sets the acceptance threshold: double-float, first cycle only
  const size_t p0 = blk * a.chunk, p1 = (p0 + a.chunk < a.N) ? p0 + a.chunk : a.N;
  int n = (int)((unsigned)(p0 + threadIdx.x) / (unsigned)a.nx);
  int m = (int)((unsigned)(p0 + threadIdx.x) - (unsigned)n * (unsigned)a.nx);
  for (size_t q = p0 + threadIdx.x; q < p1; q += kKThreads, m += kKThreads) {
    while (m >= a.nx) { m -= a.nx; ++n; }
    const cdf z = cdf_zero();
    const cdf vw = m > 0 ? load_df(xb, a.Np, q - 1) : z;
    const cdf ve = m < a.nx - 1 ? load_df(xb, a.Np, q + 1) : z;
    const cdf vs = n > 0 ? load_df(xb, a.Np, q - a.nx) : z;
    const cdf vn = n < a.ny - 1 ? load_df(xb, a.Np, q + a.nx) : z;
    const cdf xc = load_df(xb, a.Np, q);
    const cdf D = load_df(DAdf, a.Np, q);
    cdf r = load_df(bb, a.Np, q);
    if (first) cdf_abs2_acc(bn, r);
    cdf sum;
    sum.re = df_add(df_add(vw.re, ve.re), df_add(vs.re, vn.re));
    sum.im = df_add(df_add(vw.im, ve.im), df_add(vs.im, vn.im));
    // r = b - D x + (1/h^2) sum
    cdf_sub_mul(r, D, xc);
    df_fma(r.re, ih.hi, ih.lo, sum.re.hi, sum.re.lo);
    df_fma(r.im, ih.hi, ih.lo, sum.im.hi, sum.im.lo);
    r.re = df_norm(r.re);
    r.im = df_norm(r.im);
    rh[q] = make_float2(r.re.hi, r.im.hi);
    if (write_lo) rl[q] = make_float2(r.re.lo, r.im.lo);
    rn = fmaf(r.re.hi, r.re.hi, fmaf(r.im.hi, r.im.hi, rn));
  }
  cd acc[1] = {mk<double>((double)rn, 0.0)};
  block_reduce_store<1>(acc, 1, df_to_double(bn), 1, partial + ((size_t)rhs * a.nblk + blk) * a.pstride);
}

// The same for rows of even width: two adjacent points per thread and step (the pair never
// straddles a row), 16-byte loads of the x, b and D_A pairs and of the rows above and below, one
// 16-byte store per plane; each point is computed with k_df_residual's operations.
__device__ __forceinline__ void load_df2(const float2* __restrict__ h, size_t Np, size_t q, cdf& u0, cdf& u1) {
  const float4 a = *reinterpret_cast<const float4*>(h + q), b = *reinterpret_cast<const float4*>(h + q + Np);
  u0.re.hi = a.x; u0.im.hi = a.y; u0.re.lo = b.x; u0.im.lo = b.y;
  u1.re.hi = a.z; u1.im.hi = a.w; u1.re.lo = b.z; u1.im.lo = b.w;
}

__device__ __forceinline__ cdf df_residual_pt(cdf r, const cdf& D, const cdf& xc, const cdf& vw, const cdf& ve,
                                              const cdf& vs, const cdf& vn, const df& ih) {
  cdf sum;
  sum.re = df_add(df_add(vw.re, ve.re), df_add(vs.re, vn.re));
  sum.im = df_add(df_add(vw.im, ve.im), df_add(vs.im, vn.im));
  cdf_sub_mul(r, D, xc);
  df_fma(r.re, ih.hi, ih.lo, sum.re.hi, sum.re.lo);
  df_fma(r.im, ih.hi, ih.lo, sum.im.hi, sum.im.lo);
  r.re = df_norm(r.re);
  r.im = df_norm(r.im);
  return r;
}

__global__ void __launch_bounds__(kKThreads)
k_df_residual2(KArgs a, const float2* __restrict__ bdf, const float2* __restrict__ xdf, const float2* __restrict__ DAdf,
               float2* __restrict__ V, cd* __restrict__ partial, const RhsState* __restrict__ st, int first,
               int write_lo) {
  const int rhs = blockIdx.y, blk = blockIdx.x;
  if (st[rhs].done) return;
  const float2* xb = xdf + (size_t)rhs * 2 * a.Np;
  const float2* bb = bdf + (size_t)rhs * 2 * a.Np;
  float2* rh = V + ((size_t)rhs * (a.m + 1) * 2) * a.Np;
  float2* rl = rh + a.Np;
  const df ih = df_from_double(a.inv_h2);
  float rn = 0.f;
  df bn = {0.f, 0.f};
  const size_t p0 = blk * a.chunk, p1 = (p0 + a.chunk < a.N) ? p0 + a.chunk : a.N;   // both even
  size_t q = p0 + 2 * threadIdx.x;
  int n = (int)((unsigned)q / (unsigned)a.nx);
  int m = (int)((unsigned)q - (unsigned)n * (unsigned)a.nx);
  for (; q < p1; q += 2 * kKThreads, m += 2 * kKThreads) {
    while (m >= a.nx) { m -= a.nx; ++n; }
    const cdf z = cdf_zero();
    cdf x0, x1, b0, b1, d0, d1, s0 = z, s1 = z, n0 = z, n1 = z;
    load_df2(xb, a.Np, q, x0, x1);
    load_df2(bb, a.Np, q, b0, b1);
    load_df2(DAdf, a.Np, q, d0, d1);
    if (n > 0) load_df2(xb, a.Np, q - a.nx, s0, s1);
    if (n < a.ny - 1) load_df2(xb, a.Np, q + a.nx, n0, n1);
    const cdf wl = m > 0 ? load_df(xb, a.Np, q - 1) : z;
    const cdf er = m + 2 < a.nx ? load_df(xb, a.Np, q + 2) : z;
    if (first) {
      cdf_abs2_acc(bn, b0);
      cdf_abs2_acc(bn, b1);
    }
    const cdf r0 = df_residual_pt(b0, d0, x0, wl, x1, s0, n0, ih);
    const cdf r1 = df_residual_pt(b1, d1, x1, x0, er, s1, n1, ih);
    *reinterpret_cast<float4*>(rh + q) = make_float4(r0.re.hi, r0.im.hi, r1.re.hi, r1.im.hi);
    if (write_lo) *reinterpret_cast<float4*>(rl + q) = make_float4(r0.re.lo, r0.im.lo, r1.re.lo, r1.im.lo);
    rn = fmaf(r0.re.hi, r0.re.hi, fmaf(r0.im.hi, r0.im.hi, rn));
    rn = fmaf(r1.re.hi, r1.re.hi, fmaf(r1.im.hi, r1.im.hi, rn));
  }
  cd acc[1] = {mk<double>((double)rn, 0.0)};
  block_reduce_store<1>(acc, 1, df_to_double(bn), 1, partial + ((size_t)rhs * a.nblk + blk) * a.pstride);
}

// Cycle start from the double-float residual: a right-hand side whose residual meets its target
// waits for the FP64 verification instead of starting a cycle.
__global__ void k_df_cycle_start(KArgs a, const cd* __restrict__ partial, double* __restrict__ vscale,
                                 cd* __restrict__ g, RhsState* __restrict__ st, double tol, int maxit, int first) {
  __shared__ cd sh[2];
  const int rhs = blockIdx.x;
  if (st[rhs].done) return;
  sum_partials(a, partial, rhs, 2, sh);
  if (threadIdx.x != 0) return;
  RhsState& S = st[rhs];
  S.nres += 1;
  if (first) {
    S.bnorm = sqrt(sh[1].re);
    S.iterations = 0;
    S.restarts = 0;
    S.tol_scale = 1.0;
  } else {
    S.restarts += 1;
  }
  const double rn = sqrt(sh[0].re);
  S.rnorm = rn;
  S.jend = 0;
  S.active = 0;
  S.verify = 0;
  if (S.bnorm == 0.0) { S.done = 1; S.converged = 1; return; }
  if (rn <= tol * S.tol_scale * S.bnorm) { S.verify = 1; return; }
  if (S.iterations >= maxit || !(rn == rn)) { S.done = 1; S.converged = 0; return; }
  S.active = 1;
  vscale[(size_t)rhs * (a.m + 1)] = 1.0 / rn;
  cd* gg = g + (size_t)rhs * (a.m + 1);
  gg[0] = mk<double>(rn, 0.0);
  for (int i = 1; i <= a.m; ++i) gg[i] = czero<double>();
}

// FP64 true residual ||b - A x||^2 of the right-hand sides awaiting verification (slot 0).
__global__ void __launch_bounds__(kKThreads)
k_verify_residual(KArgs a, const cd* __restrict__ b, const cd* __restrict__ x, const cd* __restrict__ DA,
                  cd* __restrict__ partial, const RhsState* __restrict__ st) {
  const int rhs = blockIdx.y, blk = blockIdx.x;
  if (!st[rhs].verify) return;
  const cd* xb = x + (size_t)rhs * a.N;
  const cd* bb = b + (size_t)rhs * a.N;
  cd acc[1] = {czero<double>()};
  const size_t p0 = blk * a.chunk, p1 = (p0 + a.chunk < a.N) ? p0 + a.chunk : a.N;
  int n = (int)((unsigned)(p0 + threadIdx.x) / (unsigned)a.nx);
  int m = (int)((unsigned)(p0 + threadIdx.x) - (unsigned)n * (unsigned)a.nx);
  for (size_t q = p0 + threadIdx.x; q < p1; q += kKThreads, m += kKThreads) {
    while (m >= a.nx) { m -= a.nx; ++n; }
    cd s = czero<double>();
    if (m > 0) s = s + xb[q - 1];
    if (m < a.nx - 1) s = s + xb[q + 1];
    if (n > 0) s = s + xb[q - a.nx];
    if (n < a.ny - 1) s = s + xb[q + a.nx];
    const cd rv = bb[q] - (DA[q] * xb[q] - a.inv_h2 * s);
    acc[0].re += cabs2(rv);
  }
  block_reduce_store<1>(acc, 1, 0.0, 1, partial + ((size_t)rhs * a.nblk + blk) * a.pstride);
}

// Accept on the FP64 residual, or tighten the double-float target and start another cycle.
__global__ void k_verify_decide(KArgs a, const cd* __restrict__ partial, double* __restrict__ vscale,
                                cd* __restrict__ g, RhsState* __restrict__ st, double tol, int maxit) {
  __shared__ cd sh[1];
  const int rhs = blockIdx.x;
  if (!st[rhs].verify) return;
  sum_partials(a, partial, rhs, 1, sh);
  if (threadIdx.x != 0) return;
  RhsState& S = st[rhs];
  S.verify = 0;
  S.nverify += 1;
  const double r64 = sqrt(sh[0].re);
  if (r64 <= tol * S.bnorm) { S.done = 1; S.converged = 1; S.rnorm = r64; return; }
  S.tol_scale *= 0.1;
  if (S.iterations >= maxit || !(r64 == r64)) { S.done = 1; S.converged = 0; S.rnorm = r64; return; }
  // continue from the double-float residual already in basis slot 0
  S.active = 1;
  vscale[(size_t)rhs * (a.m + 1)] = 1.0 / S.rnorm;
  cd* gg = g + (size_t)rhs * (a.m + 1);
  gg[0] = mk<double>(S.rnorm, 0.0);
  for (int i = 1; i <= a.m; ++i) gg[i] = czero<double>();
}

// The preconditioned vector z_i at point q from its storage (complex FP32, or complex FP16 under
// MGH_PREC_MIXED16).
__device__ __forceinline__ cf zload(const cf* Z, size_t i) { return Z[i]; }
__device__ __forceinline__ cf zload(const __half2* Z, size_t i) {
  const float2 f = __half22float2(Z[i]);
  return mk<float>(f.x, f.y);
}

// Two adjacent points of z (q even) as (re0, im0, re1, im1): one 16-byte load of FP32 storage or
// one 8-byte load of FP16 storage.
__device__ __forceinline__ float4 zpair(const cf* z, size_t q) { return reinterpret_cast<const float4*>(z)[q / 2]; }
__device__ __forceinline__ float4 zpair(const __half2* z, size_t q) {
  const uint2 u = reinterpret_cast<const uint2*>(z)[q / 2];
  const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&u.x));
  const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&u.y));
  return make_float4(a.x, a.y, b.x, b.y);
}

// x += sum_{i < jend} y_i z_i, all in double-float (x planes, z FP32 or FP16, y split to double-float).
template <int NV, typename ZT = cf>
__global__ void __launch_bounds__(kKThreads)
k_df_xupdate(KArgs a, const ZT* __restrict__ Z, const cd* __restrict__ y, float2* __restrict__ xdf,
             const RhsState* __restrict__ st) {
  const int rhs = blockIdx.y;
  if (st[rhs].done || st[rhs].jend == 0) return;
  const int je = st[rhs].jend;
  __shared__ cdf ys[NV];
  if (threadIdx.x < NV && (int)threadIdx.x < je) ys[threadIdx.x] = cdf_from(y[(size_t)rhs * a.m + threadIdx.x]);
  __syncthreads();
  const ZT* Zb = Z + (size_t)rhs * a.m * a.N;
  float2* xh = xdf + (size_t)rhs * 2 * a.Np;
  float2* xl = xh + a.Np;
  const size_t p0 = blockIdx.x * a.chunk, p1 = (p0 + a.chunk < a.N) ? p0 + a.chunk : a.N;
  // two points per thread and iteration, every load issued before the arithmetic
  for (size_t q = p0 + threadIdx.x; q < p1; q += 2 * kKThreads) {
    const size_t q2 = q + kKThreads;
    const bool two = q2 < p1;
    cf z1[NV], z2[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      z1[i] = i < je ? zload(Zb, (size_t)i * a.N + q) : mk<float>(0.f, 0.f);
      z2[i] = (i < je && two) ? zload(Zb, (size_t)i * a.N + q2) : mk<float>(0.f, 0.f);
    }
    cdf v[2] = {load_df(xh, a.Np, q), two ? load_df(xh, a.Np, q2) : cdf_zero()};
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      if (i < je) {
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const cf z = u == 0 ? z1[i] : z2[i];
          df_fma1(v[u].re, ys[i].re.hi, ys[i].re.lo, z.re);
          df_fma1(v[u].re, -ys[i].im.hi, -ys[i].im.lo, z.im);
          df_fma1(v[u].im, ys[i].re.hi, ys[i].re.lo, z.im);
          df_fma1(v[u].im, ys[i].im.hi, ys[i].im.lo, z.re);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      if (u == 1 && !two) break;
      const size_t qq = u == 0 ? q : q2;
      v[u].re = df_norm(v[u].re);
      v[u].im = df_norm(v[u].im);
      xh[qq] = make_float2(v[u].re.hi, v[u].im.hi);
      xl[qq] = make_float2(v[u].re.lo, v[u].im.lo);
    }
  }
}

// The same for FP16 z (MGH_PREC_MIXED16, even N): two adjacent points per thread and step, one
// 8-byte load per z_i and 16-byte loads and stores of the x planes, so that a thread keeps as many
// bytes in flight as the FP32 variant does.
template <int NV>
__global__ void __launch_bounds__(kKThreads)
k_df_xupdate_h2(KArgs a, const __half2* __restrict__ Z, const cd* __restrict__ y, float2* __restrict__ xdf,
                const RhsState* __restrict__ st) {
  const int rhs = blockIdx.y;
  if (st[rhs].done || st[rhs].jend == 0) return;
  const int je = st[rhs].jend;
  __shared__ cdf ys[NV];
  if (threadIdx.x < NV && (int)threadIdx.x < je) ys[threadIdx.x] = cdf_from(y[(size_t)rhs * a.m + threadIdx.x]);
  __syncthreads();
  const __half2* Zb = Z + (size_t)rhs * a.m * a.N;
  float4* xh = reinterpret_cast<float4*>(xdf + (size_t)rhs * 2 * a.Np);
  float4* xl = reinterpret_cast<float4*>(xdf + (size_t)rhs * 2 * a.Np + a.Np);
  const size_t p0 = blockIdx.x * a.chunk, p1 = (p0 + a.chunk < a.N) ? p0 + a.chunk : a.N;   // both even
  for (size_t q = p0 + 2 * threadIdx.x; q < p1; q += 2 * kKThreads) {
    float4 z[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) z[i] = i < je ? zpair(Zb + (size_t)i * a.N, q) : make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 h = xh[q / 2], l = xl[q / 2];
    cdf v[2];
    v[0].re = df{h.x, l.x}; v[0].im = df{h.y, l.y};
    v[1].re = df{h.z, l.z}; v[1].im = df{h.w, l.w};
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      if (i < je) {
        const cf zz[2] = {mk<float>(z[i].x, z[i].y), mk<float>(z[i].z, z[i].w)};
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          df_fma1(v[u].re, ys[i].re.hi, ys[i].re.lo, zz[u].re);
          df_fma1(v[u].re, -ys[i].im.hi, -ys[i].im.lo, zz[u].im);
          df_fma1(v[u].im, ys[i].re.hi, ys[i].re.lo, zz[u].im);
          df_fma1(v[u].im, ys[i].im.hi, ys[i].im.lo, zz[u].re);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      v[u].re = df_norm(v[u].re);
      v[u].im = df_norm(v[u].im);
    }
    xh[q / 2] = make_float4(v[0].re.hi, v[0].im.hi, v[1].re.hi, v[1].im.hi);
    xl[q / 2] = make_float4(v[0].re.lo, v[0].im.lo, v[1].re.lo, v[1].im.lo);
  }
}


// ---------------------------------------------------------------- s-step cycle (MGH_ARNOLDI_SSTEP)
// One restart cycle of flexible GMRES(m) in s-step form (Chronopoulos & Gear 1989; Hoemmen 2010),
// with the Krylov basis orthogonalised at the end of the cycle by a Cholesky factor of its Gram
// matrix:
//   v_0 = r (double-float), and for k < m:  z_k = M^{-1}(v_k / ||v_k||),  v_{k+1} = A z_k
//   G = V^H V over v_0 .. v_m (one sweep),  G = R^H R (FP64, equilibrated)
//   r - A Z y = V (e_0 - [0; y]),  so  ||r - A Z y|| = ||R[:,0] - R[:,1:] y||
// The small least-squares problem is the GMRES one with the upper-Hessenberg matrix R[:,1:] and
// right-hand side R_00 e_0; Givens rotations give the residual of every prefix, and the cycle
// keeps the shortest prefix that meets the tolerance.  In exact arithmetic this is the same
// iterate as Arnoldi-based FGMRES(m) on the same z_k; a Cholesky pivot that vanishes ends the
// usable basis there.
//
// The basis is stored in FP32 (the hi planes of the basis slots) and v_{k+1} = A z_k is formed
// in FP32: the cycle only has to find a near-optimal correction, and the relation
// A Z = V_{1:m+1} then holds to FP32 rounding, which perturbs the residual reduction of a cycle by
// about eps32 * cond(V) (1e-4 for cond(V) ~ 1e3).  The Gram entries are summed by FP32 FMAs in
// runs of 32 products per thread, and the runs are added into double-float totals: an entry
// carries an error of a few eps32 * sum_p |v_i[p]| |v_j[p]|, a normwise perturbation of G of
// the size FP32 storage of the basis already makes.  On the 576^2 ellipse workload (cond of the
// equilibrated factor 1.1e3 to 1.5e3) a solve then takes the same 584 steps as with the exact
// Gram of the stored basis, also for runs of 4, 16 and 64 products.  The iterate and the restart
// residual stay double-float and every accepted iterate is checked by the FP64 true residual, so
// the attainable accuracy is that of the outer iteration (iterative refinement with an FP32 inner
// cycle).

template <int NV>
struct GramPairs {
  static constexpr int NP = NV * (NV + 1) / 2;   // pairs i <= j, row by row
  static constexpr int PG = (NP + 3) / 4;        // most pairs of one group of 64 threads (4 groups)
  // group g sums pairs [first(g), first(g + 1)): contiguous shares that differ by at most one
  __host__ __device__ static constexpr int first(int g) { return (g * NP + 2) / 4; }
  __host__ __device__ static constexpr int row(int p) {
    int i = 0;
    while (p >= NV - i) { p -= NV - i; ++i; }
    return i;
  }
  __host__ __device__ static constexpr int col(int p) {
    int i = 0;
    while (p >= NV - i) { p -= NV - i; ++i; }
    return i + p;
  }
};

template <typename F, int... I>
__device__ __forceinline__ void unroll_seq(F&& f, std::integer_sequence<int, I...>) {
  (f(std::integral_constant<int, I>{}), ...);
}
template <int N, typename F>
__device__ __forceinline__ void unroll(F&& f) {
  unroll_seq(f, std::make_integer_sequence<int, N>{});
}

// v_{k+1} = A z_k in FP32, written to the hi plane of basis slot k + 1, and its partial
// ||v_{k+1}||^2 (slot 0 of the partial buffer; FP32 sums: the norm only scales the next
// multigrid input, the Gram matrix holds the exact one).
__global__ void __launch_bounds__(kKThreads)
k_ss_matvec(KArgs a, int k, const cf* __restrict__ Z, const float2* __restrict__ D32, float2* __restrict__ V,
            cd* __restrict__ partial, const RhsState* __restrict__ st) {
  const int rhs = blockIdx.y, blk = blockIdx.x;
  if (!st[rhs].active) return;
  const cf* z = Z + ((size_t)rhs * a.m + k) * a.N;
  float2* vh = V + (((size_t)rhs * (a.m + 1) + k + 1) * 2) * a.Np;
  const float ih = (float)a.inv_h2;
  float nrm = 0.f;
  const size_t p0 = (size_t)blk * a.chunk, p1 = (p0 + a.chunk < a.N) ? p0 + a.chunk : a.N;
  int n = (int)((unsigned)(p0 + threadIdx.x) / (unsigned)a.nx);
  int m = (int)((unsigned)(p0 + threadIdx.x) - (unsigned)n * (unsigned)a.nx);
#pragma unroll 4
  for (size_t q = p0 + threadIdx.x; q < p1; q += kKThreads, m += kKThreads) {
    while (m >= a.nx) { m -= a.nx; ++n; }
    const cf zc = z[q];
    const cf zw = m > 0 ? z[q - 1] : mk<float>(0.f, 0.f);
    const cf ze = m < a.nx - 1 ? z[q + 1] : mk<float>(0.f, 0.f);
    const cf zs = n > 0 ? z[q - a.nx] : mk<float>(0.f, 0.f);
    const cf zn = n < a.ny - 1 ? z[q + a.nx] : mk<float>(0.f, 0.f);
    const float2 d = D32[q];
    const float sr = (zw.re + ze.re) + (zs.re + zn.re), si = (zw.im + ze.im) + (zs.im + zn.im);
    const float wr = fmaf(d.x, zc.re, fmaf(-d.y, zc.im, -ih * sr));
    const float wi = fmaf(d.x, zc.im, fmaf(d.y, zc.re, -ih * si));
    vh[q] = make_float2(wr, wi);
    nrm = fmaf(wr, wr, fmaf(wi, wi, nrm));
  }
  df vals[1] = {{nrm, 0.f}};
  cd* out = partial + ((size_t)rhs * a.nblk + blk) * a.pstride;
  block_reduce_df(vals, 1, [&](int) -> double* { out->im = 0.0; return &out->re; });
}

// The same for rows of even width: two adjacent points per thread and step (the pair never
// straddles a row), 16-byte loads of z (8-byte for FP16 storage), D and the rows above and below,
// one 16-byte store.
template <typename ZT = cf>
__global__ void __launch_bounds__(kKThreads)
k_ss_matvec2(KArgs a, int k, const ZT* __restrict__ Z, const float2* __restrict__ D32, float2* __restrict__ V,
             cd* __restrict__ partial, const RhsState* __restrict__ st) {
  const int rhs = blockIdx.y, blk = blockIdx.x;
  if (!st[rhs].active) return;
  const ZT* z = Z + ((size_t)rhs * a.m + k) * a.N;
  float2* vh = V + (((size_t)rhs * (a.m + 1) + k + 1) * 2) * a.Np;
  const float ih = (float)a.inv_h2;
  float nrm = 0.f;
  const size_t p0 = (size_t)blk * a.chunk, p1 = (p0 + a.chunk < a.N) ? p0 + a.chunk : a.N;   // both even
  const float4* d4 = reinterpret_cast<const float4*>(D32);
  float4* v4 = reinterpret_cast<float4*>(vh);
  size_t q = p0 + 2 * threadIdx.x;
  int n = (int)((unsigned)q / (unsigned)a.nx);
  int m = (int)((unsigned)q - (unsigned)n * (unsigned)a.nx);
#pragma unroll 2
  for (; q < p1; q += 2 * kKThreads, m += 2 * kKThreads) {
    while (m >= a.nx) { m -= a.nx; ++n; }
    const size_t h = q / 2;
    const float4 c = zpair(z, q);
    const float4 up = n > 0 ? zpair(z, q - a.nx) : make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 dn = n < a.ny - 1 ? zpair(z, q + a.nx) : make_float4(0.f, 0.f, 0.f, 0.f);
    const cf zl = m > 0 ? zload(z, q - 1) : mk<float>(0.f, 0.f);
    const cf zr = m + 2 < a.nx ? zload(z, q + 2) : mk<float>(0.f, 0.f);
    const float4 d = d4[h];
    // point q: neighbours zl, (c.z, c.w), up.xy, dn.xy; point q+1: (c.x, c.y), zr, up.zw, dn.zw
    const float s0r = (zl.re + c.z) + (up.x + dn.x), s0i = (zl.im + c.w) + (up.y + dn.y);
    const float s1r = (c.x + zr.re) + (up.z + dn.z), s1i = (c.y + zr.im) + (up.w + dn.w);
    const float w0r = fmaf(d.x, c.x, fmaf(-d.y, c.y, -ih * s0r));
    const float w0i = fmaf(d.x, c.y, fmaf(d.y, c.x, -ih * s0i));
    const float w1r = fmaf(d.z, c.z, fmaf(-d.w, c.w, -ih * s1r));
    const float w1i = fmaf(d.z, c.w, fmaf(d.w, c.z, -ih * s1i));
    v4[h] = make_float4(w0r, w0i, w1r, w1i);
    nrm = fmaf(w0r, w0r, fmaf(w0i, w0i, fmaf(w1r, w1r, fmaf(w1i, w1i, nrm))));
  }
  df vals[1] = {{nrm, 0.f}};
  cd* out = partial + ((size_t)rhs * a.nblk + blk) * a.pstride;
  block_reduce_df(vals, 1, [&](int) -> double* { out->im = 0.0; return &out->re; });
}

// 1 / ||v_{k+1}|| for the next multigrid input.
__global__ void k_ss_norm(KArgs a, int k, const cd* __restrict__ partial, double* __restrict__ vscale,
                          const RhsState* __restrict__ st) {
  // one warp per right-hand side: lanes load the block sums in parallel, a butterfly adds them
  const int rhs = blockIdx.x;
  if (!st[rhs].active) return;
  double n2 = 0.0;
  for (int b = threadIdx.x; b < a.nblk; b += 32) n2 += partial[((size_t)rhs * a.nblk + b) * a.pstride].re;
  n2 = warp_sum(n2);
  if (threadIdx.x == 0) vscale[(size_t)rhs * (a.m + 1) + k + 1] = n2 > 0.0 ? 1.0 / sqrt(n2) : 1.0;
}

// ||v_{k+1}||^2 from the per-(row pair, strip) partials of the level-0 post kernel that formed
// v_{k+1} = A z_k itself: one block per right-hand side, FP64 sums in a fixed order.
__global__ void __launch_bounds__(1024) k_ss_norm_rows(KArgs a, int k, const float* __restrict__ npart, int per_rhs,
                                                      double* __restrict__ vscale, const RhsState* __restrict__ st) {
  const int rhs = blockIdx.x;
  if (!st[rhs].active) return;
  const float* p = npart + (size_t)rhs * per_rhs;
  double n2 = 0.0;
#pragma unroll 4
  for (int t = threadIdx.x; t < per_rhs; t += 1024) n2 += (double)p[t];
  n2 = warp_sum(n2);
  __shared__ double sh[32];
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = n2;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < 32; ++w) s += sh[w];
    vscale[(size_t)rhs * (a.m + 1) + k + 1] = s > 0.0 ? 1.0 / sqrt(s) : 1.0;
  }
}

// The Gram sums of one tile's points for the pairs of thread group G, accumulated by FP32 FMAs
// into the thread's running sums `run` (re, im per pair); k_ss_gram adds the running sums into
// double-float totals every kGramRunTiles tiles.
template <int NV, int G>
__device__ __forceinline__ void gram_tile(const Pipe& pp, int slot, size_t q0, size_t p1, int l64, float2* run) {
  using PR = GramPairs<NV>;
  constexpr int P0 = PR::first(G);
  constexpr int P1 = PR::first(G + 1);
  static_assert(P1 - P0 <= PR::PG, "group share above its accumulators");
  if constexpr (P1 > P0) {
    constexpr int IMIN = PR::row(P0);
#pragma unroll 1
    for (int r = 0; r < kTile / 64; ++r) {
      const int t = l64 + 64 * r;
      if (q0 + t >= p1) break;
      float2 v[NV];
#pragma unroll
      for (int i = IMIN; i < NV; ++i) v[i] = pp.plane(slot, i)[t];
      unroll<P1 - P0>([&](auto PC) {
        constexpr int p = P0 + decltype(PC)::value;
        constexpr int i = PR::row(p), j = PR::col(p);
        float2& c = run[p - P0];
        if constexpr (i == j) {
          c.x = __fmaf_rn(v[i].x, v[i].x, __fmaf_rn(v[i].y, v[i].y, c.x));
        } else {   // conj(v_i) v_j
          c.x = __fmaf_rn(v[i].x, v[j].x, __fmaf_rn(v[i].y, v[j].y, c.x));
          c.y = __fmaf_rn(v[i].x, v[j].y, __fmaf_rn(-v[i].y, v[j].x, c.y));
        }
      });
    }
  }
}

// Tiles between two promotions of the FP32 running sums into the double-float totals: a thread
// sums 4 points of a tile, so a running sum holds 4 * kGramRunTiles products.
constexpr int kGramRunTiles = 8;

// G_ij = v_i^H v_j (i <= j) over the stored v_0 .. v_{NV-1}: one sweep of the basis through the TMA ring;
// four groups of 64 threads share the pairs, each thread sums 4 points of every tile.  Group g
// is warps g and g + 4, which run on the same SM sub-partition, so that each sub-partition's
// instruction cache holds the code of one group.
template <int NV>
__global__ void __launch_bounds__(kDfThreads)
k_ss_gram(KArgs a, int S, const float2* __restrict__ V, cd* __restrict__ partial, const RhsState* __restrict__ st,
          int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char smem[];
  using PR = GramPairs<NV>;
  static_assert(kDfThreads == 256, "four groups of 64 threads");
  const int rhs = blockIdx.y, blk = blockIdx.x;
  if (!st[rhs].active) return;
  const size_t p0 = (size_t)blk * a.chunk, p1 = (p0 + a.chunk < a.N) ? p0 + a.chunk : a.N;
  Pipe pp = pipe_begin(smem, S, NV, p0, p1);   // the FP32 (hi) planes of the basis
  if (threadIdx.x == 0)
    for (int i = 0; i < NV; ++i) pp.src[i] = vplane(V, a, rhs, i, 0);
  int* fail = reinterpret_cast<int*>(smem + kSmemHeader - 16);
  pipe_start(pp, fail);
  const int grp = (threadIdx.x >> 5) & 3, l64 = (threadIdx.x & 31) + 32 * (threadIdx.x >> 7);
  cdf acc[PR::PG];
  float2 run[PR::PG];
#pragma unroll
  for (int c = 0; c < PR::PG; ++c) {
    acc[c] = cdf_zero();
    run[c] = make_float2(0.f, 0.f);
  }
  // two tiles per barrier: wait for k and k + 1, sum both, release both
  for (int k = 0; k < pp.ntiles; k += 2) {
    const bool two = k + 1 < pp.ntiles;
    const bool ready = pipe_wait(pp, k, fail) && (!two || pipe_wait(pp, k + 1, fail));
    if (ready) {
      for (int u = 0; u < (two ? 2 : 1); ++u) {
        const int slot = (k + u) % S;
        const size_t q0 = p0 + (size_t)(k + u) * kTile;
        switch (grp) {
          case 0: gram_tile<NV, 0>(pp, slot, q0, p1, l64, run); break;
          case 1: gram_tile<NV, 1>(pp, slot, q0, p1, l64, run); break;
          case 2: gram_tile<NV, 2>(pp, slot, q0, p1, l64, run); break;
          default: gram_tile<NV, 3>(pp, slot, q0, p1, l64, run); break;
        }
      }
    }
    if (!pipe_release2(pp, k, fail, err)) return;
    if ((k + 2) % kGramRunTiles == 0 || k + 2 >= pp.ntiles) {
#pragma unroll
      for (int c = 0; c < PR::PG; ++c) {
        df_add1(acc[c].re, run[c].x);
        df_add1(acc[c].im, run[c].y);
        run[c] = make_float2(0.f, 0.f);
      }
    }
  }
  __shared__ float4 sh[kDfThreads / 32][PR::PG];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int c = 0; c < PR::PG; ++c) {
    const df re = warp_sum_df(acc[c].re), im = warp_sum_df(acc[c].im);
    if (lane == 0) sh[warp][c] = make_float4(re.hi, re.lo, im.hi, im.lo);
  }
  __syncthreads();
  cd* out = partial + ((size_t)rhs * a.nblk + blk) * a.pstride;
  for (int t = threadIdx.x; t < PR::NP; t += kDfThreads) {
    int g = 0;
    while (t >= PR::first(g + 1)) ++g;
    const int c = t - PR::first(g);
    const float4 x0 = sh[g][c], x1 = sh[g + 4][c];
    const df re = df_add(df{x0.x, x0.y}, df{x1.x, x1.y}), im = df_add(df{x0.z, x0.w}, df{x1.z, x1.w});
    out[t] = mk<double>(df_to_double(re), df_to_double(im));
  }
}

// ---- eight thread groups of one warp each: half the pairs per thread of k_ss_gram, so that the
// kernel holds half the accumulators and three blocks fit on an SM
template <int NV>
struct GramPairs8 {
  static constexpr int NP = NV * (NV + 1) / 2;
  static constexpr int PG = (NP + 7) / 8;   // most pairs of one group
  __host__ __device__ static constexpr int first(int g) { return (g * NP + 4) / 8; }
};

// Tiles between promotions of the running sums in k_ss_gram8: a thread sums 8 points of a tile,
// so a running sum again holds 32 products.
constexpr int kGramRunTiles8 = 4;

template <int NV, int G>
__device__ __forceinline__ void gram_tile8(const Pipe& pp, int slot, size_t q0, size_t p1, int lane, float2* run) {
  using PR = GramPairs<NV>;
  using P8 = GramPairs8<NV>;
  constexpr int P0 = P8::first(G);
  constexpr int P1 = P8::first(G + 1);
  static_assert(P1 - P0 <= P8::PG, "group share above its accumulators");
  if constexpr (P1 > P0) {
    constexpr int IMIN = PR::row(P0);
#pragma unroll 1
    for (int r = 0; r < kTile / 32; ++r) {
      const int t = lane + 32 * r;
      if (q0 + t >= p1) break;
      float2 v[NV];
#pragma unroll
      for (int i = IMIN; i < NV; ++i) v[i] = pp.plane(slot, i)[t];
      unroll<P1 - P0>([&](auto PC) {
        constexpr int p = P0 + decltype(PC)::value;
        constexpr int i = PR::row(p), j = PR::col(p);
        float2& c = run[p - P0];
        if constexpr (i == j) {
          c.x = __fmaf_rn(v[i].x, v[i].x, __fmaf_rn(v[i].y, v[i].y, c.x));
        } else {   // conj(v_i) v_j
          c.x = __fmaf_rn(v[i].x, v[j].x, __fmaf_rn(v[i].y, v[j].y, c.x));
          c.y = __fmaf_rn(v[i].x, v[j].y, __fmaf_rn(-v[i].y, v[j].x, c.y));
        }
      });
    }
  }
}

// k_ss_gram with warp w summing the pairs of group w (eight groups) over all 256 points of a tile.
template <int NV>
__global__ void __launch_bounds__(kDfThreads, 3)
k_ss_gram8(KArgs a, int S, const float2* __restrict__ V, cd* __restrict__ partial, const RhsState* __restrict__ st,
           int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char smem[];
  using P8 = GramPairs8<NV>;
  static_assert(kDfThreads == 256, "eight warps, one group each");
  const int rhs = blockIdx.y, blk = blockIdx.x;
  if (!st[rhs].active) return;
  const size_t p0 = (size_t)blk * a.chunk, p1 = (p0 + a.chunk < a.N) ? p0 + a.chunk : a.N;
  Pipe pp = pipe_begin(smem, S, NV, p0, p1);   // the FP32 (hi) planes of the basis
  if (threadIdx.x == 0)
    for (int i = 0; i < NV; ++i) pp.src[i] = vplane(V, a, rhs, i, 0);
  int* fail = reinterpret_cast<int*>(smem + kSmemHeader - 16);
  pipe_start(pp, fail);
  const int grp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  cdf acc[P8::PG];
  float2 run[P8::PG];
#pragma unroll
  for (int c = 0; c < P8::PG; ++c) {
    acc[c] = cdf_zero();
    run[c] = make_float2(0.f, 0.f);
  }
  for (int k = 0; k < pp.ntiles; k += 2) {
    const bool two = k + 1 < pp.ntiles;
    const bool ready = pipe_wait(pp, k, fail) && (!two || pipe_wait(pp, k + 1, fail));
    if (ready) {
      for (int u = 0; u < (two ? 2 : 1); ++u) {
        const int slot = (k + u) % S;
        const size_t q0 = p0 + (size_t)(k + u) * kTile;
        switch (grp) {
          case 0: gram_tile8<NV, 0>(pp, slot, q0, p1, lane, run); break;
          case 1: gram_tile8<NV, 1>(pp, slot, q0, p1, lane, run); break;
          case 2: gram_tile8<NV, 2>(pp, slot, q0, p1, lane, run); break;
          case 3: gram_tile8<NV, 3>(pp, slot, q0, p1, lane, run); break;
          case 4: gram_tile8<NV, 4>(pp, slot, q0, p1, lane, run); break;
          case 5: gram_tile8<NV, 5>(pp, slot, q0, p1, lane, run); break;
          case 6: gram_tile8<NV, 6>(pp, slot, q0, p1, lane, run); break;
          default: gram_tile8<NV, 7>(pp, slot, q0, p1, lane, run); break;
        }
      }
    }
    if (!pipe_release2(pp, k, fail, err)) return;
    if ((k + 2) % kGramRunTiles8 == 0 || k + 2 >= pp.ntiles) {
#pragma unroll
      for (int c = 0; c < P8::PG; ++c) {
        df_add1(acc[c].re, run[c].x);
        df_add1(acc[c].im, run[c].y);
        run[c] = make_float2(0.f, 0.f);
      }
    }
  }
  cd* out = partial + ((size_t)rhs * a.nblk + blk) * a.pstride;
  const int f0 = P8::first(grp), f1 = P8::first(grp + 1);
#pragma unroll
  for (int c = 0; c < P8::PG; ++c) {
    const df re = warp_sum_df(acc[c].re), im = warp_sum_df(acc[c].im);
    if (lane == 0 && f0 + c < f1) out[f0 + c] = mk<double>(df_to_double(re), df_to_double(im));
  }
}

// Per right-hand side: the Gram matrix from the block sums, its equilibrated Cholesky factor,
// the cycle's least-squares problem by Givens rotations, the prefix to keep and its y.  One warp
// per right-hand side (launched with 32 threads): the Gram entries are summed by lanes, row j of
// the factor is formed with lane k computing entry (j, k), and lane c carries column c of the
// least-squares matrix through the rotations; every entry is formed with the same operations in
// the same order as by a single thread.
template <int NV>
__global__ void __launch_bounds__(32) k_ss_lsq(KArgs a, const cd* __restrict__ partial, cd* __restrict__ y,
                                               RhsState* __restrict__ st, double tol, int maxit) {
  using PR = GramPairs<NV>;
  constexpr int M = NV - 1;
  static_assert(NV <= 32, "one lane per column");
  __shared__ cd Gs[PR::NP];
  __shared__ cd R[NV][NV];
  __shared__ cd Hs[NV][NV];
  __shared__ double dsc[NV];
  const int rhs = blockIdx.x;
  if (!st[rhs].active) return;
  const int lane = threadIdx.x;
  {
    // the block sums of this right-hand side are contiguous rows of pstride entries: stage
    // kLsqRows rows at a time with coalesced loads, then add each entry's rows in block order
    constexpr int kLsqRows = 8;
    __shared__ cd stage[kLsqRows * PR::NP];
    constexpr int NT = (PR::NP + 31) / 32;
    cd acc[NT];
#pragma unroll
    for (int u = 0; u < NT; ++u) acc[u] = czero<double>();
    const cd* base = partial + (size_t)rhs * a.nblk * a.pstride;
    for (int b0 = 0; b0 < a.nblk; b0 += kLsqRows) {
      const int nb = a.nblk - b0 < kLsqRows ? a.nblk - b0 : kLsqRows;
      for (int e = lane; e < nb * PR::NP; e += 32) {
        const int r = e / PR::NP, t = e - r * PR::NP;
        stage[e] = base[(size_t)(b0 + r) * a.pstride + t];
      }
      __syncwarp();
#pragma unroll
      for (int u = 0; u < NT; ++u) {
        const int t = lane + 32 * u;
        if (t < PR::NP)
          for (int r = 0; r < nb; ++r) acc[u] = acc[u] + stage[r * PR::NP + t];
      }
      __syncwarp();
    }
#pragma unroll
    for (int u = 0; u < NT; ++u)
      if (lane + 32 * u < PR::NP) Gs[lane + 32 * u] = acc[u];
  }
  __syncwarp();
  RhsState& S = st[rhs];
  auto G = [&](int i, int j) -> cd { return Gs[i * NV - i * (i - 1) / 2 + (j - i)]; };   // i <= j
  // equilibrated factor: G~ = D G D with D = diag(1 / sqrt(G_ii)), G~ = Rt^H Rt, R = Rt D^{-1}
  int nv = NV;   // basis vectors whose pivots are usable (the same value in every lane)
  for (int i = 0; i < NV; ++i)
    if (nv == NV && !(G(i, i).re > 0.0)) nv = i;
  if (lane < nv) dsc[lane] = 1.0 / sqrt(G(lane, lane).re);
  __syncwarp();
  for (int j = 0; j < nv; ++j) {
    double s = 1.0;
    for (int i = 0; i < j; ++i) s -= cabs2(R[i][j]);
    if (!(s > 1e-12)) {   // v_j (numerically) in the span of v_0 .. v_{j-1}
      if (lane == 0) R[j][j] = czero<double>();
      nv = j + 1;
      break;
    }
    const double rjj = sqrt(s);
    const int k = lane;
    if (k > j && k < nv) {
      cd t = (dsc[j] * dsc[k]) * G(j, k);
      for (int i = 0; i < j; ++i) t = t - cconj(R[i][j]) * R[i][k];
      R[j][k] = (1.0 / rjj) * t;
    }
    if (lane == 0) R[j][j] = mk<double>(rjj, 0.0);
    __syncwarp();
  }
  __syncwarp();
  for (int t = lane; t < nv * nv; t += 32) {
    const int jj = t / nv, ii = t - jj * nv;
    if (ii <= jj) R[ii][jj] = (1.0 / dsc[jj]) * R[ii][jj];
  }
  __syncwarp();
  int kmax = nv - 1;   // usable steps: columns 1 .. kmax of R
  if (kmax > maxit - S.iterations) kmax = maxit - S.iterations;
  __syncwarp();
  if (kmax < 1) {   // no usable direction: stop this right-hand side
    if (lane == 0) {
      S.active = 0;
      S.csteps += M;
      S.gsum += NV;
      S.done = 1;
      S.converged = 0;
      S.jend = 0;
    }
    return;
  }
  // Givens on the (kmax+1) x kmax upper-Hessenberg matrix H[i][c] = R[i][c+1], rhs g = R_00 e_0;
  // lane c holds column c and applies each rotation as soon as it is known
  const double thr = tol * S.tol_scale * S.bnorm;
  cd col[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) col[i] = (lane < kmax && i <= lane + 1) ? R[i][lane + 1] : czero<double>();
  cd g0 = R[0][0], g1 = czero<double>();   // g[c], g[c+1] of the current rotation (every lane)
  cd gsv[NV];
  int jend = kmax;
#pragma unroll
  for (int c = 0; c < M; ++c) {
    if (c < jend) {
      // lane c forms rotation c from its rotated column; every lane receives it
      double cc = 1.0;
      cd sv = czero<double>();
      if (lane == c) {
        const cd aa = col[c], bb = col[c + 1];
        if (bb.re == 0.0 && bb.im == 0.0) { cc = 1.0; sv = czero<double>(); }
        else if (aa.re == 0.0 && aa.im == 0.0) { cc = 0.0; sv = mk<double>(1.0, 0.0); }
        else {
          const double na = sqrt(cabs2(aa)), rho = sqrt(cabs2(aa) + cabs2(bb));
          cc = na / rho;
          sv = (1.0 / (na * rho)) * (aa * cconj(bb));
        }
        col[c] = cc * col[c] + sv * col[c + 1];
      }
      cc = __shfl_sync(0xffffffffu, cc, c);
      sv.re = __shfl_sync(0xffffffffu, sv.re, c);
      sv.im = __shfl_sync(0xffffffffu, sv.im, c);
      if (lane > c && lane < kmax) {
        const cd t = cc * col[c] + sv * col[c + 1];
        col[c + 1] = (-1.0 * cconj(sv)) * col[c] + cc * col[c + 1];
        col[c] = t;
      }
      g1 = (-1.0 * cconj(sv)) * g0;
      gsv[c] = cc * g0;
      g0 = g1;
      if (!(sqrt(cabs2(g1)) > thr)) jend = c + 1;   // the same decision in every lane
    }
  }
  if (lane < jend) {
#pragma unroll
    for (int i = 0; i < NV; ++i)
      if (i <= lane) Hs[i][lane] = col[i];
  }
  __syncwarp();
  if (lane != 0) return;
  S.active = 0;
  S.csteps += M;
  S.gsum += NV;
  cd* yy = y + (size_t)rhs * a.m;
  for (int i = jend - 1; i >= 0; --i) {
    cd t = gsv[i];
    for (int k = i + 1; k < jend; ++k) t = t - Hs[i][k] * yy[k];
    const cd d = Hs[i][i];
    const double den = cabs2(d);
    yy[i] = den > 0.0 ? t * mk<double>(d.re / den, -d.im / den) : czero<double>();
  }
  S.jend = jend;
  S.iterations += jend;
  S.nupd += 1;
  S.zsum += jend;
}

// ---------------------------------------------------------------- host side
// Stages of the shared-memory ring for P planes and the dynamic shared memory they need.
int stages_for(int P) {
  const size_t stage = (size_t)P * kTile * sizeof(float2);
  int S = (int)(kStageBudget / stage);
  return S < 2 ? 2 : (S > kMaxStages ? kMaxStages : S);
}
size_t smem_for(int P, int S) { return kSmemHeader + (size_t)S * P * kTile * sizeof(float2); }

template <typename K>
mgh_status set_smem(K kern) {
  MGH_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem_for(kMaxPlanes, 2) + 1024));
  return MGH_OK;
}

template <int NV>
mgh_status df_step_nv(Handle& h, const KArgs& a, int j, int B) {
  MGH_ONCE(MGH_TRY(set_smem(k_df_pass1<NV>)); MGH_TRY(set_smem(k_df_pass2<NV>)););
  const dim3 grid(a.nblk, B);
  float2* V = reinterpret_cast<float2*>(h.V);
  float2* W = reinterpret_cast<float2*>(h.W);
  {
    const int P = 4 + 2 * j, S = stages_for(P);
    ProfScope ps(h, P_MATVEC_DOTS);
    k_df_pass1<NV><<<grid, kDfThreads, smem_for(P, S), h.stream>>>(a, j, S, (const cf*)h.Z, h.DAdf, V, W,
                                                                    h.partial, h.st, h.dev_err);
    MGH_CHECK_LAUNCH(); h.launches++;
  }
  {
    ProfScope ps(h, P_REDUCE);
    k_df_scalars<<<B, 64, 0, h.stream>>>(a, j, 0, h.partial, h.H, h.cs, h.sn, h.g, h.hpend, h.coef, h.st,
                                         h.p.tol, h.p.maxit);
    MGH_CHECK_LAUNCH(); h.launches++;
  }
  {
    const int P = 4 + 2 * j, S = stages_for(P);
    ProfScope ps(h, P_UPDATE);
    k_df_pass2<NV><<<grid, kDfThreads, smem_for(P, S), h.stream>>>(a, j, S, h.coef, V, W, h.partial, h.st,
                                                                    h.dev_err);
    MGH_CHECK_LAUNCH(); h.launches++;
  }
  {
    ProfScope ps(h, P_REDUCE);
    k_df_unorm<<<B, 32, 0, h.stream>>>(a, j, h.partial, h.vscale, h.st);
    MGH_CHECK_LAUNCH(); h.launches++;
  }
  return MGH_OK;
}

mgh_status df_arnoldi_step(Handle& h, const KArgs& a, int j, int B) {
  // z_j = M^{-1}(u_j / ||u_j||), reading only the hi plane of u_j
  const cf* uhi = reinterpret_cast<const cf*>(reinterpret_cast<const float2*>(h.V) + (size_t)j * 2 * a.Np);
  MGH_TRY(vcycle_f32in(h, uhi, (size_t)(a.m + 1) * 2 * a.Np, h.vscale + j, (size_t)(a.m + 1),
                       (cf*)h.Z + (size_t)j * a.N, (size_t)a.m * a.N, B, h.st, j));
  if (j <= 4) return df_step_nv<4>(h, a, j, B);
  if (j <= 8) return df_step_nv<8>(h, a, j, B);
  if (j <= 12) return df_step_nv<12>(h, a, j, B);
  if (j <= 16) return df_step_nv<16>(h, a, j, B);
  return df_step_nv<kMaxRestartDf>(h, a, j, B);
}

// End of a cycle: finalise the last column from the second-pass dots of the last pass 2.
mgh_status df_tail(Handle& h, const KArgs& a, int B) {
  ProfScope ps(h, P_REDUCE);
  k_df_scalars<<<B, 64, 0, h.stream>>>(a, a.m, 1, h.partial, h.H, h.cs, h.sn, h.g, h.hpend, h.coef, h.st,
                                       h.p.tol, h.p.maxit);
  MGH_CHECK_LAUNCH(); h.launches++;
  return MGH_OK;
}

mgh_status df_xupdate(Handle& h, const KArgs& a, int B) {
  const dim3 grid(a.nblk, B);
  ProfScope ps(h, P_XUPDATE);
  const int m = a.m;
  float2* x = h.xdf;
  if (h.half) {   // FP16 preconditioned vectors (s-step engine, m <= 8)
    const __half2* Zh = reinterpret_cast<const __half2*>(h.Z);
    if (m <= 4) k_df_xupdate_h2<4><<<grid, kKThreads, 0, h.stream>>>(a, Zh, h.y, x, h.st);
    else k_df_xupdate_h2<8><<<grid, kKThreads, 0, h.stream>>>(a, Zh, h.y, x, h.st);
    MGH_CHECK_LAUNCH(); h.launches++;
    return MGH_OK;
  }
  if (m <= 4) k_df_xupdate<4><<<grid, kKThreads, 0, h.stream>>>(a, (const cf*)h.Z, h.y, x, h.st);
  else if (m <= 8) k_df_xupdate<8><<<grid, kKThreads, 0, h.stream>>>(a, (const cf*)h.Z, h.y, x, h.st);
  else if (m <= 12) k_df_xupdate<12><<<grid, kKThreads, 0, h.stream>>>(a, (const cf*)h.Z, h.y, x, h.st);
  else if (m <= 16) k_df_xupdate<16><<<grid, kKThreads, 0, h.stream>>>(a, (const cf*)h.Z, h.y, x, h.st);
  else k_df_xupdate<kMaxRestartDf><<<grid, kKThreads, 0, h.stream>>>(a, (const cf*)h.Z, h.y, x, h.st);
  MGH_CHECK_LAUNCH(); h.launches++;
  return MGH_OK;
}

}  // namespace

namespace {

// Restarted flexible GMRES with a double-float iterate: the start, the FP64-verified restarts
// and the exit are shared; `cycle` runs one restart cycle (its steps and the iterate update).
template <typename Cycle>
mgh_status df_driver(Handle& h, const cd* b, int B, cd* x, mgh_solve_info* info, bool write_lo, Cycle&& cycle) {
  KArgs a = make_kargs(h, B);
  const dim3 grid(a.nblk, B);
  const dim3 pgrid((unsigned)((a.N + 255) / 256), B);
  float2* V = reinterpret_cast<float2*>(h.V);
  MGH_CUDA(cudaMemsetAsync(h.dev_err, 0, sizeof(int), h.stream));
  if (h.inject_timeout) {   // test hook: the word a kernel whose bounded wait gave up would leave
    h.inject_timeout = false;
    MGH_CUDA(cudaMemsetAsync(h.dev_err, 1, sizeof(int), h.stream));
  }
  // start: state, double-float copies of b and x0, first residual in double-float
  auto residual_and_start = [&](int first) -> mgh_status {
    {
      ProfScope ps(h, P_RESIDUAL);
      if (a.nx % 2 == 0)
        k_df_residual2<<<grid, kKThreads, 0, h.stream>>>(a, h.bdf, h.xdf, h.DAdf, V, h.partial, h.st, first,
                                                         write_lo ? 1 : 0);
      else
        k_df_residual<<<grid, kKThreads, 0, h.stream>>>(a, h.bdf, h.xdf, h.DAdf, V, h.partial, h.st, first,
                                                        write_lo ? 1 : 0);
      MGH_CHECK_LAUNCH(); h.launches++;
    }
    {
      ProfScope ps(h, P_REDUCE);
      k_df_cycle_start<<<B, 32, 0, h.stream>>>(a, h.partial, h.vscale, h.g, h.st, h.p.tol, h.p.maxit, first);
      MGH_CHECK_LAUNCH(); h.launches++;
    }
    {
      // FP64 acceptance test of the right-hand sides whose double-float residual met the target
      ProfScope ps(h, P_RESIDUAL);
      k_df_join<<<pgrid, 256, 0, h.stream>>>(h.xdf, x, a.N, a.Np, h.st, 0);
      MGH_CHECK_LAUNCH(); h.launches++;
      k_verify_residual<<<grid, kKThreads, 0, h.stream>>>(a, b, x, h.DA, h.partial, h.st);
      MGH_CHECK_LAUNCH(); h.launches++;
    }
    {
      ProfScope ps(h, P_REDUCE);
      k_verify_decide<<<B, 32, 0, h.stream>>>(a, h.partial, h.vscale, h.g, h.st, h.p.tol, h.p.maxit);
      MGH_CHECK_LAUNCH(); h.launches++;
    }
    return MGH_OK;
  };
  {
    ProfScope ps(h, P_REDUCE);
    k_state_reset<<<(B + 63) / 64, 64, 0, h.stream>>>(h.st, B);
    MGH_CHECK_LAUNCH(); h.launches++;
  }
  {
    ProfScope ps(h, P_OTHER);
    k_df_split<<<pgrid, 256, 0, h.stream>>>(b, h.bdf, a.N, a.Np);
    MGH_CHECK_LAUNCH(); h.launches++;
    k_df_split<<<pgrid, 256, 0, h.stream>>>(x, h.xdf, a.N, a.Np);
    MGH_CHECK_LAUNCH(); h.launches++;
  }
  MGH_TRY(residual_and_start(1));
  // the body of a restart cycle (its steps with every multigrid level, and the restart) is
  // replayed from a captured graph after the first cycle
  CycleGraph graph;
  auto body = [&]() -> mgh_status {
    MGH_TRY(cycle(a));
    return residual_and_start(0);
  };
  int err_host = 0;
  for (int ncycle = 0;; ++ncycle) {
    MGH_CUDA(cudaMemcpyAsync(h.st_host, h.st, sizeof(RhsState) * B, cudaMemcpyDeviceToHost, h.stream));
    MGH_CUDA(cudaMemcpyAsync(&err_host, h.dev_err, sizeof(int), cudaMemcpyDeviceToHost, h.stream));
    MGH_CUDA(cudaStreamSynchronize(h.stream));
    MGH_TRY(prof_flush(h));
    if (err_host) return MGH_TIMEOUT;
    bool any = false;
    for (int i = 0; i < B; ++i) any |= (h.st_host[i].done == 0);
    if (!any) break;
    if (!h.use_graphs || h.prof || ncycle == 0) MGH_TRY(body());
    else MGH_TRY(graph.run(h, body));
  }
  {
    // every RHS leaves with its double-float iterate rounded to FP64
    ProfScope ps(h, P_OTHER);
    k_df_join<<<pgrid, 256, 0, h.stream>>>(h.xdf, x, a.N, a.Np, h.st, 1);
    MGH_CHECK_LAUNCH(); h.launches++;
  }
  MGH_CUDA(cudaStreamSynchronize(h.stream));
  return finish_solve(h, B, info);
}

}  // namespace

mgh_status fgmres_df(Handle& h, const cd* b, int B, cd* x, mgh_solve_info* info) {
  return df_driver(h, b, B, x, info, true, [&](const KArgs& a) -> mgh_status {
    for (int j = 0; j < a.m; ++j) MGH_TRY(df_arnoldi_step(h, a, j, B));
    MGH_TRY(df_tail(h, a, B));
    {
      ProfScope ps(h, P_REDUCE);
      k_lsq<<<(B + 63) / 64, 64, 0, h.stream>>>(a, h.H, h.g, h.y, h.st, B);
      MGH_CHECK_LAUNCH(); h.launches++;
    }
    return df_xupdate(h, a, B);
  });
}

namespace {

template <int NV>
mgh_status ss_cycle(Handle& h, const KArgs& a, int B) {
  MGH_ONCE(MGH_TRY(set_smem(k_ss_gram<NV>)); MGH_TRY(set_smem(k_ss_gram8<NV>)););
  const dim3 grid(a.nblk, B);
  float2* V = reinterpret_cast<float2*>(h.V);
  for (int k = 0; k < a.m; ++k) {
    // z_k = M^{-1}(v_k / ||v_k||), reading only the hi plane of v_k
    const cf* vhi = reinterpret_cast<const cf*>(V + (size_t)k * 2 * a.Np);
    // slot k of Z: complex FP32, or complex FP16 (half the bytes per slot) under MGH_PREC_MIXED16,
    // where it holds zmul * M^{-1}(v_k / ||v_k||): any fixed scale of z_k leaves the cycle's
    // iterate unchanged, since v_{k+1} = A z_k is formed from the stored z_k
    __half2* zh = reinterpret_cast<__half2*>(h.Z) + (size_t)k * a.N;
    cf* zk = h.half ? reinterpret_cast<cf*>(zh) : (cf*)h.Z + (size_t)k * a.N;
    // v_{k+1} = A z_k: fused into the level-0 post kernel when its launch path allows it
    h.fuse_v = reinterpret_cast<cf*>(V + (size_t)(k + 1) * 2 * a.Np);
    h.fuse_vstride = (size_t)(a.m + 1) * 2 * a.Np;
    h.fuse_nstrips = 0;
    const mgh_status vs = vcycle_f32in(h, vhi, (size_t)(a.m + 1) * 2 * a.Np, h.vscale + k, (size_t)(a.m + 1), zk,
                                       (size_t)a.m * a.N, B, h.st, k);
    const int fused = h.fuse_nstrips;
    h.fuse_v = nullptr;
    h.fuse_nstrips = 0;
    MGH_TRY(vs);
    if (fused > 0) {
      if (k + 1 < a.m) {
        ProfScope ps(h, P_REDUCE);
        k_ss_norm_rows<<<B, 1024, 0, h.stream>>>(a, k, h.npart, ((a.ny + 1) / 2) * fused, h.vscale, h.st);
        MGH_CHECK_LAUNCH(); h.launches++;
      }
      continue;
    }
    {
      ProfScope ps(h, P_MATVEC_DOTS);
      if (h.half)
        k_ss_matvec2<__half2><<<grid, kKThreads, 0, h.stream>>>(a, k, reinterpret_cast<const __half2*>(h.Z), h.DAdf,
                                                                V, h.partial, h.st);
      else if (a.nx % 2 == 0)
        k_ss_matvec2<<<grid, kKThreads, 0, h.stream>>>(a, k, (const cf*)h.Z, h.DAdf, V, h.partial, h.st);
      else
        k_ss_matvec<<<grid, kKThreads, 0, h.stream>>>(a, k, (const cf*)h.Z, h.DAdf, V, h.partial, h.st);
      MGH_CHECK_LAUNCH(); h.launches++;
    }
    if (k + 1 < a.m) {
      ProfScope ps(h, P_REDUCE);
      k_ss_norm<<<B, 32, 0, h.stream>>>(a, k, h.partial, h.vscale, h.st);
      MGH_CHECK_LAUNCH(); h.launches++;
    }
  }
  {
    ProfScope ps(h, P_UPDATE);
    if (h.gram8) {   // three blocks per SM: a ring of at most 3 stages
      const int S = std::min(3, stages_for(NV));
      k_ss_gram8<NV><<<grid, kDfThreads, smem_for(NV, S), h.stream>>>(a, S, V, h.partial, h.st, h.dev_err);
    } else {
      const int S = stages_for(NV);
      k_ss_gram<NV><<<grid, kDfThreads, smem_for(NV, S), h.stream>>>(a, S, V, h.partial, h.st, h.dev_err);
    }
    MGH_CHECK_LAUNCH(); h.launches++;
  }
  {
    ProfScope ps(h, P_REDUCE);
    k_ss_lsq<NV><<<B, 32, 0, h.stream>>>(a, h.partial, h.y, h.st, h.p.tol, h.p.maxit);
    MGH_CHECK_LAUNCH(); h.launches++;
  }
  return df_xupdate(h, a, B);
}

}  // namespace

mgh_status fgmres_ss(Handle& h, const cd* b, int B, cd* x, mgh_solve_info* info) {
  return df_driver(h, b, B, x, info, false, [&](const KArgs& a) -> mgh_status {
    switch (a.m + 1) {
      case 2: return ss_cycle<2>(h, a, B);
      case 3: return ss_cycle<3>(h, a, B);
      case 4: return ss_cycle<4>(h, a, B);
      case 5: return ss_cycle<5>(h, a, B);
      case 6: return ss_cycle<6>(h, a, B);
      case 7: return ss_cycle<7>(h, a, B);
      case 8: return ss_cycle<8>(h, a, B);
      case 9: return ss_cycle<9>(h, a, B);
    }
    return MGH_INVALID_ARG;
  });
}

}  // namespace mgh
