// Batched right-preconditioned flexible GMRES(m) in FP64 (Saad & Schultz 1986; Saad 1993),
// with one multigrid cycle as the preconditioner (Alg. 3's role: the Krylov outer loop of
// Sec. IV-C; BJ's GMRES replaces the paper's Bi-CGSTAB).
//
// All right-hand sides share the operator and advance in lock step, one Arnoldi step at a
// time; each keeps its own Hessenberg matrix, Givens rotations and stopping decision on the
// device, so the host only reads the per-RHS state once per restart cycle.
//
// Orthogonalisation is classical Gram-Schmidt with a conditional second pass (the
// Daniel-Gragg-Kaufman-Stewart criterion ||w'|| < ||w||/sqrt(2)): a fused kernel computes
// w = A z_j together with all dots <v_i, w>; a second kernel subtracts the projections, writes
// the new basis vector and already accumulates the dots needed by a second pass.  Basis
// vectors are stored unnormalised, each with a per-RHS multiplier (vscale) applied by its
// readers, so no separate normalisation pass over the vector is needed.
//
// Every iterate is accepted on the true FP64 residual ||b - A x|| <= tol ||b|| computed at the
// end of each cycle (the relative stopping rule of Sec. VI); the Givens estimate only ends a
// cycle early.
#include <algorithm>
#include <cmath>
#include <vector>

#include "mgh_df.cuh"
#include "mgh_engine.h"

namespace mgh {

namespace {

constexpr int kKThreads = 256;
constexpr int kTargetBlocks = 152 * 8;

struct KArgs {
  int nx, ny;
  size_t N;
  int m;                 // restart length
  int nblk;              // reduction blocks per RHS
  size_t chunk;          // points per block
  double inv_h2;
  int pstride;           // complex slots per block in the partial-sum buffer
};

// Block reduction of NV complex accumulators (plus one real) into partial[(rhs*nblk+blk)*(m+2) + i].
template <int NV>
__device__ __forceinline__ void block_reduce_store(cd (&acc)[NV], int nv_used, double extra, int extra_slot,
                                                   cd* __restrict__ out) {
  __shared__ double sh[kKThreads / 32][2 * NV + 1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    if (i < nv_used) {
      const double re = warp_sum(acc[i].re);
      const double im = warp_sum(acc[i].im);
      if (lane == 0) { sh[warp][2 * i] = re; sh[warp][2 * i + 1] = im; }
    }
  }
  const double ex = warp_sum(extra);
  if (lane == 0) sh[warp][2 * NV] = ex;
  __syncthreads();
  const int nw = kKThreads / 32;
  for (int t = threadIdx.x; t < 2 * nv_used; t += kKThreads) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += sh[w][t];
    double* o = reinterpret_cast<double*>(out + (t >> 1));
    o[t & 1] = s;
  }
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += sh[w][2 * NV];
    out[extra_slot] = mk<double>(s, 0.0);
  }
}

template <typename TZ>
__device__ __forceinline__ cd load_z(const Cx<TZ>* z, size_t q) { return ccast<double>(z[q]); }

// w = A z_j (FP64), W <- w, partial dots <v_i, w> (i <= j) and ||w||^2.
template <typename TZ, int NV>
__global__ void __launch_bounds__(kKThreads)
k_matvec_dots(KArgs a, int j, const Cx<TZ>* __restrict__ Z, const cd* __restrict__ DA, const cd* __restrict__ V,
              cd* __restrict__ W, cd* __restrict__ partial, const RhsState* __restrict__ st) {
  const int rhs = blockIdx.y, blk = blockIdx.x;
  if (!st[rhs].active) return;
  const Cx<TZ>* z = Z + ((size_t)rhs * a.m + j) * a.N;
  const cd* Vb = V + (size_t)rhs * (a.m + 1) * a.N;
  cd* Wb = W + (size_t)rhs * a.N;
  cd acc[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) acc[i] = czero<double>();
  double nrm = 0.0;
  const size_t p0 = blk * a.chunk, p1 = (p0 + a.chunk < a.N) ? p0 + a.chunk : a.N;
  int n = (int)((unsigned)(p0 + threadIdx.x) / (unsigned)a.nx);
  int m = (int)((unsigned)(p0 + threadIdx.x) - (unsigned)n * (unsigned)a.nx);
  for (size_t q = p0 + threadIdx.x; q < p1; q += kKThreads, m += kKThreads) {
    while (m >= a.nx) { m -= a.nx; ++n; }
    cd s = czero<double>();
    if (m > 0) s = s + load_z(z, q - 1);
    if (m < a.nx - 1) s = s + load_z(z, q + 1);
    if (n > 0) s = s + load_z(z, q - a.nx);
    if (n < a.ny - 1) s = s + load_z(z, q + a.nx);
    const cd w = DA[q] * load_z(z, q) - a.inv_h2 * s;
    Wb[q] = w;
    nrm += cabs2(w);
#pragma unroll
    for (int i = 0; i < NV; ++i)
      if (i <= j) cdot_acc(acc[i], Vb[(size_t)i * a.N + q], w);
  }
  block_reduce_store<NV>(acc, j + 1, nrm, j + 1, partial + ((size_t)rhs * a.nblk + blk) * a.pstride);
}

// w' = w - sum_i h_i v_i written as basis vector j+1; partial dots <v_i, w'> and ||w'||^2.
template <int NV>
__global__ void __launch_bounds__(kKThreads)
k_update(KArgs a, int j, const cd* __restrict__ hcol, const double* __restrict__ vscale, cd* __restrict__ V,
         const cd* __restrict__ W, cd* __restrict__ partial, const RhsState* __restrict__ st) {
  const int rhs = blockIdx.y, blk = blockIdx.x;
  if (!st[rhs].active) return;
  __shared__ cd hs[NV];
  if (threadIdx.x < NV && (int)threadIdx.x <= j) {
    const double sc = vscale[(size_t)rhs * (a.m + 1) + threadIdx.x];
    hs[threadIdx.x] = sc * hcol[(size_t)rhs * (a.m + 1) + threadIdx.x];
  }
  __syncthreads();
  cd* Vb = V + (size_t)rhs * (a.m + 1) * a.N;
  const cd* Wb = W + (size_t)rhs * a.N;
  cd acc[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) acc[i] = czero<double>();
  double nrm = 0.0;
  const size_t p0 = blk * a.chunk, p1 = (p0 + a.chunk < a.N) ? p0 + a.chunk : a.N;
  for (size_t q = p0 + threadIdx.x; q < p1; q += kKThreads) {
    cd w = Wb[q];
#pragma unroll
    for (int i = 0; i < NV; ++i)
      if (i <= j) caxpy_neg(w, hs[i], Vb[(size_t)i * a.N + q]);
    Vb[(size_t)(j + 1) * a.N + q] = w;
    nrm += cabs2(w);
#pragma unroll
    for (int i = 0; i < NV; ++i)
      if (i <= j) cdot_acc(acc[i], Vb[(size_t)i * a.N + q], w);
  }
  block_reduce_store<NV>(acc, j + 1, nrm, j + 1, partial + ((size_t)rhs * a.nblk + blk) * a.pstride);
}

// Second Gram-Schmidt pass for the right-hand sides that need it: w'' = w' - sum_i h2_i v_i.
template <int NV>
__global__ void __launch_bounds__(kKThreads)
k_reorth(KArgs a, int j, const cd* __restrict__ h2col, const double* __restrict__ vscale, cd* __restrict__ V,
         cd* __restrict__ partial, const RhsState* __restrict__ st) {
  const int rhs = blockIdx.y, blk = blockIdx.x;
  if (!st[rhs].active || !st[rhs].reorth) return;
  __shared__ cd hs[NV];
  if (threadIdx.x < NV && (int)threadIdx.x <= j) {
    const double sc = vscale[(size_t)rhs * (a.m + 1) + threadIdx.x];
    hs[threadIdx.x] = sc * h2col[(size_t)rhs * (a.m + 1) + threadIdx.x];
  }
  __syncthreads();
  cd* Vb = V + (size_t)rhs * (a.m + 1) * a.N;
  double nrm = 0.0;
  const size_t p0 = blk * a.chunk, p1 = (p0 + a.chunk < a.N) ? p0 + a.chunk : a.N;
  for (size_t q = p0 + threadIdx.x; q < p1; q += kKThreads) {
    cd w = Vb[(size_t)(j + 1) * a.N + q];
#pragma unroll
    for (int i = 0; i < NV; ++i)
      if (i <= j) caxpy_neg(w, hs[i], Vb[(size_t)i * a.N + q]);
    Vb[(size_t)(j + 1) * a.N + q] = w;
    nrm += cabs2(w);
  }
  cd none[1] = {czero<double>()};
  block_reduce_store<1>(none, 0, nrm, j + 1, partial + ((size_t)rhs * a.nblk + blk) * a.pstride);
}

// Sum the block partials of slots [0, nslots) for one right-hand side (one block per RHS).
__device__ __forceinline__ void sum_partials(const KArgs& a, const cd* __restrict__ partial, int rhs, int nslots,
                                             cd* __restrict__ out_sh) {
  for (int s = threadIdx.x; s < nslots; s += blockDim.x) {
    cd acc = czero<double>();
    for (int b = 0; b < a.nblk; ++b) acc = acc + partial[((size_t)rhs * a.nblk + b) * a.pstride + s];
    out_sh[s] = acc;
  }
  __syncthreads();
}

// After k_matvec_dots: h_i = vscale_i * <V_i, w>; ||w||^2.
__global__ void k_fin_dots(KArgs a, int j, const cd* __restrict__ partial, const double* __restrict__ vscale,
                           cd* __restrict__ hcol, RhsState* __restrict__ st) {
  __shared__ cd sh[kMaxRestart + 2];
  const int rhs = blockIdx.x;
  if (!st[rhs].active) return;
  sum_partials(a, partial, rhs, j + 2, sh);
  for (int i = threadIdx.x; i <= j; i += blockDim.x)
    hcol[(size_t)rhs * (a.m + 1) + i] = vscale[(size_t)rhs * (a.m + 1) + i] * sh[i];
  if (threadIdx.x == 0) st[rhs].wnorm2 = sh[j + 1].re;
}

// After k_update: re-orthogonalisation dots, ||w'||^2, and the second-pass decision.
__global__ void k_fin_update(KArgs a, int j, const cd* __restrict__ partial, const double* __restrict__ vscale,
                             cd* __restrict__ h2col, RhsState* __restrict__ st) {
  __shared__ cd sh[kMaxRestart + 2];
  const int rhs = blockIdx.x;
  if (!st[rhs].active) return;
  sum_partials(a, partial, rhs, j + 2, sh);
  for (int i = threadIdx.x; i <= j; i += blockDim.x)
    h2col[(size_t)rhs * (a.m + 1) + i] = vscale[(size_t)rhs * (a.m + 1) + i] * sh[i];
  if (threadIdx.x == 0) {
    const double n2 = sh[j + 1].re;
    st[rhs].norm2 = n2;
    st[rhs].reorth = (n2 > 0.0 && n2 < 0.5 * st[rhs].wnorm2) ? 1 : 0;
  }
}

__global__ void k_fin_reorth(KArgs a, int j, const cd* __restrict__ partial, const cd* __restrict__ h2col,
                             cd* __restrict__ hcol, RhsState* __restrict__ st) {
  __shared__ cd sh[kMaxRestart + 2];
  const int rhs = blockIdx.x;
  if (!st[rhs].active || !st[rhs].reorth) return;
  sum_partials(a, partial, rhs, j + 2, sh);
  for (int i = threadIdx.x; i <= j; i += blockDim.x)
    hcol[(size_t)rhs * (a.m + 1) + i] = hcol[(size_t)rhs * (a.m + 1) + i] + h2col[(size_t)rhs * (a.m + 1) + i];
  if (threadIdx.x == 0) {
    st[rhs].norm2 = sh[j + 1].re;
    st[rhs].rsum += j + 1;
  }
}

// Givens update of column j of the Hessenberg matrix and of the rotated right-hand side g;
// one thread per right-hand side.  Rotation [[c, s], [-conj(s), c]] with c real.
__global__ void k_givens(KArgs a, int j, const cd* __restrict__ hcol, cd* __restrict__ H, double* __restrict__ cs,
                         cd* __restrict__ sn, cd* __restrict__ g, double* __restrict__ vscale,
                         RhsState* __restrict__ st, int B, double tol, int maxit) {
  const int rhs = blockIdx.x * blockDim.x + threadIdx.x;
  if (rhs >= B || !st[rhs].active) return;
  const int m = a.m;
  cd col[kMaxRestart + 1];
  for (int i = 0; i <= j; ++i) col[i] = hcol[(size_t)rhs * (m + 1) + i];
  const double hn = sqrt(fmax(st[rhs].norm2, 0.0));
  col[j + 1] = mk<double>(hn, 0.0);
  double* c_ = cs + (size_t)rhs * m;
  cd* s_ = sn + (size_t)rhs * m;
  for (int i = 0; i < j; ++i) {
    const cd t = c_[i] * col[i] + s_[i] * col[i + 1];
    col[i + 1] = (-1.0 * cconj(s_[i])) * col[i] + c_[i] * col[i + 1];
    col[i] = t;
  }
  const cd aa = col[j], bb = col[j + 1];
  double c;
  cd s;
  if (bb.re == 0.0 && bb.im == 0.0) { c = 1.0; s = czero<double>(); }
  else if (aa.re == 0.0 && aa.im == 0.0) { c = 0.0; s = mk<double>(1.0, 0.0); }
  else {
    const double na = sqrt(cabs2(aa)), rho = sqrt(cabs2(aa) + cabs2(bb));
    c = na / rho;
    s = (1.0 / (na * rho)) * (aa * cconj(bb));
  }
  col[j] = c * col[j] + s * col[j + 1];
  c_[j] = c;
  s_[j] = s;
  cd* gg = g + (size_t)rhs * (m + 1);
  gg[j + 1] = (-1.0 * cconj(s)) * gg[j];
  gg[j] = c * gg[j];
  cd* Hc = H + ((size_t)rhs * m + j) * (m + 1);
  for (int i = 0; i <= j; ++i) Hc[i] = col[i];
  RhsState& S = st[rhs];
  S.iterations += 1;
  S.vsum += j + 1;
  S.jend = j + 1;
  const double est = sqrt(cabs2(gg[j + 1])) / S.bnorm;
  if (hn > 0.0) vscale[(size_t)rhs * (m + 1) + j + 1] = 1.0 / hn;
  if (!(est > tol) || S.iterations >= maxit || !(hn > 0.0) || j + 1 >= m) S.active = 0;
}

// Back substitution H(0:jend,0:jend) y = g(0:jend); one thread per right-hand side.
__global__ void k_lsq(KArgs a, const cd* __restrict__ H, const cd* __restrict__ g, cd* __restrict__ y,
                      RhsState* __restrict__ st, int B) {
  const int rhs = blockIdx.x * blockDim.x + threadIdx.x;
  if (rhs >= B || st[rhs].done || st[rhs].jend == 0) return;
  const int m = a.m, je = st[rhs].jend;
  st[rhs].nupd += 1;
  st[rhs].zsum += je;
  const cd* Hb = H + (size_t)rhs * m * (m + 1);
  const cd* gg = g + (size_t)rhs * (m + 1);
  cd* yy = y + (size_t)rhs * m;
  for (int i = je - 1; i >= 0; --i) {
    cd t = gg[i];
    for (int k = i + 1; k < je; ++k) t = t - Hb[(size_t)k * (m + 1) + i] * yy[k];
    const cd d = Hb[(size_t)i * (m + 1) + i];
    const double den = cabs2(d);
    yy[i] = t * mk<double>(d.re / den, -d.im / den);
  }
}

// x += sum_{i < jend} y_i z_i (FGMRES update with the stored preconditioned vectors).
template <typename TZ, int NV>
__global__ void __launch_bounds__(kKThreads)
k_xupdate(KArgs a, const Cx<TZ>* __restrict__ Z, const cd* __restrict__ y, cd* __restrict__ x,
          const RhsState* __restrict__ st) {
  const int rhs = blockIdx.y;
  if (st[rhs].done || st[rhs].jend == 0) return;
  const int je = st[rhs].jend;
  __shared__ cd ys[NV];
  if (threadIdx.x < NV && (int)threadIdx.x < je) ys[threadIdx.x] = y[(size_t)rhs * a.m + threadIdx.x];
  __syncthreads();
  const Cx<TZ>* Zb = Z + (size_t)rhs * a.m * a.N;
  cd* xb = x + (size_t)rhs * a.N;
  const size_t p0 = blockIdx.x * a.chunk, p1 = (p0 + a.chunk < a.N) ? p0 + a.chunk : a.N;
  for (size_t q = p0 + threadIdx.x; q < p1; q += kKThreads) {
    cd v = xb[q];
#pragma unroll
    for (int i = 0; i < NV; ++i)
      if (i < je) v = v + ys[i] * load_z(Zb, (size_t)i * a.N + q);
    xb[q] = v;
  }
}

// r = b - A x into basis slot 0; partial ||r||^2 (slot 0) and ||b||^2 (slot 1).
__global__ void __launch_bounds__(kKThreads)
k_residual(KArgs a, const cd* __restrict__ b, const cd* __restrict__ x, const cd* __restrict__ DA,
           cd* __restrict__ V, cd* __restrict__ partial, const RhsState* __restrict__ st) {
  const int rhs = blockIdx.y, blk = blockIdx.x;
  if (st[rhs].done) return;
  const cd* xb = x + (size_t)rhs * a.N;
  const cd* bb = b + (size_t)rhs * a.N;
  cd* r = V + (size_t)rhs * (a.m + 1) * a.N;
  cd acc[1] = {czero<double>()};
  double bn = 0.0;
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
    const cd bv = bb[q];
    const cd rv = bv - (DA[q] * xb[q] - a.inv_h2 * s);
    r[q] = rv;
    acc[0].re += cabs2(rv);
    bn += cabs2(bv);
  }
  block_reduce_store<1>(acc, 1, bn, 1, partial + ((size_t)rhs * a.nblk + blk) * a.pstride);
}

// Start (or end) a cycle from the true residual: converged / maxit / next cycle.
__global__ void k_cycle_start(KArgs a, const cd* __restrict__ partial, double* __restrict__ vscale,
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
  } else {
    S.restarts += 1;
  }
  const double rn = sqrt(sh[0].re);
  S.rnorm = rn;
  S.jend = 0;
  S.active = 0;
  S.reorth = 0;
  if (S.bnorm == 0.0) { S.done = 1; S.converged = 1; return; }
  if (rn <= tol * S.bnorm) { S.done = 1; S.converged = 1; return; }
  if (S.iterations >= maxit || !(rn == rn)) { S.done = 1; S.converged = 0; return; }
  S.active = 1;
  vscale[(size_t)rhs * (a.m + 1)] = 1.0 / rn;
  cd* gg = g + (size_t)rhs * (a.m + 1);
  gg[0] = mk<double>(rn, 0.0);
  for (int i = 1; i <= a.m; ++i) gg[i] = czero<double>();
}

// x = 0 for right-hand sides with b = 0 (set done at the first cycle start).
__global__ void k_zero_if_b_zero(KArgs a, cd* __restrict__ x, const RhsState* __restrict__ st) {
  const int rhs = blockIdx.y;
  if (st[rhs].bnorm != 0.0) return;
  const size_t p0 = blockIdx.x * a.chunk, p1 = (p0 + a.chunk < a.N) ? p0 + a.chunk : a.N;
  for (size_t q = p0 + threadIdx.x; q < p1; q += kKThreads) x[(size_t)rhs * a.N + q] = czero<double>();
}

__global__ void k_state_reset(RhsState* st, int B) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < B) { RhsState z = {}; st[i] = z; }
}

// ---------------------------------------------------------------- host-side dispatch on NV
template <typename TZ, int NV>
mgh_status step_nv(Handle& h, const KArgs& a, int j, int B) {
  const dim3 grid(a.nblk, B);
  {
    ProfScope ps(h, P_MATVEC_DOTS);
    k_matvec_dots<TZ, NV><<<grid, kKThreads, 0, h.stream>>>(a, j, (const Cx<TZ>*)h.Z, h.DA, h.V, h.W, h.partial,
                                                            h.st);
    MGH_CHECK_LAUNCH(); h.launches++;
  }
  {
    ProfScope ps(h, P_REDUCE);
    k_fin_dots<<<B, 64, 0, h.stream>>>(a, j, h.partial, h.vscale, h.hcol, h.st);
    MGH_CHECK_LAUNCH(); h.launches++;
  }
  {
    ProfScope ps(h, P_UPDATE);
    k_update<NV><<<grid, kKThreads, 0, h.stream>>>(a, j, h.hcol, h.vscale, h.V, h.W, h.partial, h.st);
    MGH_CHECK_LAUNCH(); h.launches++;
  }
  {
    ProfScope ps(h, P_REDUCE);
    k_fin_update<<<B, 64, 0, h.stream>>>(a, j, h.partial, h.vscale, h.h2col, h.st);
    MGH_CHECK_LAUNCH(); h.launches++;
  }
  {
    ProfScope ps(h, P_REORTH);
    k_reorth<NV><<<grid, kKThreads, 0, h.stream>>>(a, j, h.h2col, h.vscale, h.V, h.partial, h.st);
    MGH_CHECK_LAUNCH(); h.launches++;
  }
  {
    ProfScope ps(h, P_REDUCE);
    k_fin_reorth<<<B, 64, 0, h.stream>>>(a, j, h.partial, h.h2col, h.hcol, h.st);
    MGH_CHECK_LAUNCH(); h.launches++;
  }
  {
    ProfScope ps(h, P_REDUCE);
    k_givens<<<(B + 63) / 64, 64, 0, h.stream>>>(a, j, h.hcol, h.H, h.cs, h.sn, h.g, h.vscale, h.st, B, h.p.tol,
                                                 h.p.maxit);
    MGH_CHECK_LAUNCH(); h.launches++;
  }
  return MGH_OK;
}

template <typename TZ>
mgh_status arnoldi_step(Handle& h, const KArgs& a, int j, int B) {
  // z_j = M^{-1} v_j (one multigrid cycle), read with v_j's multiplier
  MGH_TRY(vcycle(h, h.V + (size_t)j * a.N, (size_t)(a.m + 1) * a.N, h.vscale + j, (size_t)(a.m + 1),
                 (Cx<TZ>*)h.Z + (size_t)j * a.N, (size_t)a.m * a.N, false, B, h.st));
  const int nv = j + 1;
  if (nv <= 4) return step_nv<TZ, 4>(h, a, j, B);
  if (nv <= 8) return step_nv<TZ, 8>(h, a, j, B);
  if (nv <= 16) return step_nv<TZ, 16>(h, a, j, B);
  if (nv <= 24) return step_nv<TZ, 24>(h, a, j, B);
  return step_nv<TZ, 32>(h, a, j, B);
}

template <typename TZ>
mgh_status xupdate(Handle& h, const KArgs& a, int B, cd* x) {
  dim3 grid(a.nblk, B);
  const int m = a.m;
  ProfScope ps(h, P_XUPDATE);
  if (m <= 4) k_xupdate<TZ, 4><<<grid, kKThreads, 0, h.stream>>>(a, (const Cx<TZ>*)h.Z, h.y, x, h.st);
  else if (m <= 8) k_xupdate<TZ, 8><<<grid, kKThreads, 0, h.stream>>>(a, (const Cx<TZ>*)h.Z, h.y, x, h.st);
  else if (m <= 16) k_xupdate<TZ, 16><<<grid, kKThreads, 0, h.stream>>>(a, (const Cx<TZ>*)h.Z, h.y, x, h.st);
  else if (m <= 24) k_xupdate<TZ, 24><<<grid, kKThreads, 0, h.stream>>>(a, (const Cx<TZ>*)h.Z, h.y, x, h.st);
  else k_xupdate<TZ, 32><<<grid, kKThreads, 0, h.stream>>>(a, (const Cx<TZ>*)h.Z, h.y, x, h.st);
  MGH_CHECK_LAUNCH(); h.launches++;
  return MGH_OK;
}

KArgs make_kargs(const Handle& h, int B) {
  KArgs a;
  a.nx = h.nx; a.ny = h.ny; a.N = h.N; a.m = h.m;
  a.nblk = std::max(1, std::min<int>((kTargetBlocks + B - 1) / B, (int)((h.N + 1023) / 1024)));
  a.chunk = (h.N + a.nblk - 1) / a.nblk;
  a.inv_h2 = 1.0 / (h.p.h * h.p.h);
  a.pstride = 2 * h.m + 4;
  return a;
}

// Per-RHS results of a finished solve (host mirror already synchronised) and profile counters.
mgh_status finish_solve(Handle& h, int B, mgh_solve_info* info) {
  bool all_conv = true;
  for (int i = 0; i < B; ++i) {
    const RhsState& S = h.st_host[i];
    all_conv &= (S.converged != 0);
    h.acc.arnoldi_steps += S.iterations;
    h.acc.basis_reads += S.vsum;
    h.acc.reorth_reads += S.rsum;
    h.acc.residuals += S.nres;
    h.acc.updates += S.nupd;
    h.acc.update_reads += S.zsum;
    if (info) {
      info[i].iterations = S.iterations;
      info[i].restarts = S.restarts;
      info[i].converged = S.converged;
      info[i].rel_residual = S.bnorm > 0.0 ? S.rnorm / S.bnorm : 0.0;
    }
  }
  return all_conv ? MGH_OK : MGH_NOT_CONVERGED;
}

template <typename TZ>
mgh_status fgmres_t(Handle& h, const cd* b, int B, cd* x, mgh_solve_info* info) {
  KArgs a = make_kargs(h, B);
  const dim3 grid(a.nblk, B);
  {
    ProfScope ps(h, P_REDUCE);
    k_state_reset<<<(B + 63) / 64, 64, 0, h.stream>>>(h.st, B);
    MGH_CHECK_LAUNCH(); h.launches++;
  }
  {
    ProfScope ps(h, P_RESIDUAL);
    k_residual<<<grid, kKThreads, 0, h.stream>>>(a, b, x, h.DA, h.V, h.partial, h.st);
    MGH_CHECK_LAUNCH(); h.launches++;
  }
  {
    ProfScope ps(h, P_REDUCE);
    k_cycle_start<<<B, 32, 0, h.stream>>>(a, h.partial, h.vscale, h.g, h.st, h.p.tol, h.p.maxit, 1);
    MGH_CHECK_LAUNCH(); h.launches++;
  }
  {
    ProfScope ps(h, P_OTHER);
    k_zero_if_b_zero<<<grid, kKThreads, 0, h.stream>>>(a, x, h.st);
    MGH_CHECK_LAUNCH(); h.launches++;
  }
  for (;;) {
    MGH_CUDA(cudaMemcpyAsync(h.st_host, h.st, sizeof(RhsState) * B, cudaMemcpyDeviceToHost, h.stream));
    MGH_CUDA(cudaStreamSynchronize(h.stream));
    MGH_TRY(prof_flush(h));
    bool any = false;
    for (int i = 0; i < B; ++i) any |= (h.st_host[i].done == 0);
    if (!any) break;
    for (int j = 0; j < a.m; ++j) MGH_TRY(arnoldi_step<TZ>(h, a, j, B));
    {
      ProfScope ps(h, P_REDUCE);
      k_lsq<<<(B + 63) / 64, 64, 0, h.stream>>>(a, h.H, h.g, h.y, h.st, B);
      MGH_CHECK_LAUNCH(); h.launches++;
    }
    MGH_TRY(xupdate<TZ>(h, a, B, x));
    {
      ProfScope ps(h, P_RESIDUAL);
      k_residual<<<grid, kKThreads, 0, h.stream>>>(a, b, x, h.DA, h.V, h.partial, h.st);
      MGH_CHECK_LAUNCH(); h.launches++;
    }
    {
      ProfScope ps(h, P_REDUCE);
      k_cycle_start<<<B, 32, 0, h.stream>>>(a, h.partial, h.vscale, h.g, h.st, h.p.tol, h.p.maxit, 0);
      MGH_CHECK_LAUNCH(); h.launches++;
    }
  }
  return finish_solve(h, B, info);
}

// ============================================================================ mixed path
// Arnoldi in double-float arithmetic on the FP32 pipes with classical Gram-Schmidt whose second
// pass is delayed by one step (one read of the basis per pass, two passes per step):
//
//   step j holds q_0..q_{j-1} (final, orthonormal) and u_j, the candidate left by step j-1
//   (orthogonalised once).  z_j = M^{-1}(u_j/||u_j||), w = A z_j.
//   pass 1   one sweep computes s = Q^H u_j, t = Q^H w, alpha = ||u_j||^2, beta = u_j^H w
//   scalars  nu = sqrt(alpha - ||s||^2); q_j = (u_j - Q s)/nu; h_{:,j} = (t, (beta - s^H t)/nu);
//            column j-1 is finalised with the correction s and h_{j,j-1} = nu, then rotated
//   pass 2   one sweep writes q_j and u_{j+1} = w - Q t - h_jj q_j
//
// The exact relation A z_j = sum_{i<=j+1} h_ij q_i holds for the stored z_j, which is all that
// flexible GMRES needs; the least-squares problem and the stopping estimate therefore lag one
// step behind the preconditioner application.

constexpr int kDfThreads = 256;

__device__ __forceinline__ const float2* vhi(const float2* V, const KArgs& a, int rhs, int i) {
  return V + (((size_t)rhs * (a.m + 1) + i) * 2) * a.N;
}

// Pass 1: w = A z_j in df (W planes), dots of q_0..q_{j-1} with u_j and w, ||u_j||^2, u_j^H w.
// Partial slots: s at [0, j), t at [j, 2j), alpha at 2j, beta at 2j+1.
template <int NV>
__global__ void __launch_bounds__(kDfThreads)
k_df_pass1(KArgs a, int j, const cf* __restrict__ Z, const float2* __restrict__ DAdf, const float2* __restrict__ V,
           float2* __restrict__ W, cd* __restrict__ partial, const RhsState* __restrict__ st) {
  const int rhs = blockIdx.y, blk = blockIdx.x;
  if (!st[rhs].active) return;
  const cf* z = Z + ((size_t)rhs * a.m + j) * a.N;
  const float2* uh = vhi(V, a, rhs, j);
  const float2* ul = uh + a.N;
  float2* wh = W + (size_t)rhs * 2 * a.N;
  float2* wl = wh + a.N;
  const float2* Dh = DAdf;
  const float2* Dl = DAdf + a.N;
  const df ih = df_from_double(a.inv_h2);
  cdf s[NV], t[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) { s[i] = cdf_zero(); t[i] = cdf_zero(); }
  df alpha = {0.f, 0.f};
  cdf beta = cdf_zero();
  const size_t p0 = blk * a.chunk, p1 = (p0 + a.chunk < a.N) ? p0 + a.chunk : a.N;
  int n = (int)((unsigned)(p0 + threadIdx.x) / (unsigned)a.nx);
  int m = (int)((unsigned)(p0 + threadIdx.x) - (unsigned)n * (unsigned)a.nx);
  for (size_t q = p0 + threadIdx.x; q < p1; q += kDfThreads, m += kDfThreads) {
    while (m >= a.nx) { m -= a.nx; ++n; }
    // neighbour sum of the FP32 z, exactly in df
    df sr = {0.f, 0.f}, si = {0.f, 0.f};
    if (m > 0) { const cf v = z[q - 1]; df_add1(sr, v.re); df_add1(si, v.im); }
    if (m < a.nx - 1) { const cf v = z[q + 1]; df_add1(sr, v.re); df_add1(si, v.im); }
    if (n > 0) { const cf v = z[q - a.nx]; df_add1(sr, v.re); df_add1(si, v.im); }
    if (n < a.ny - 1) { const cf v = z[q + a.nx]; df_add1(sr, v.re); df_add1(si, v.im); }
    const cf zc = z[q];
    const float2 dh = Dh[q], dl = Dl[q];
    cdf w;
    w.re.hi = w.re.lo = w.im.hi = w.im.lo = 0.f;
    // w = D z - (1/h^2) sum
    df_fma1(w.re, dh.x, dl.x, zc.re);
    df_fma1(w.re, -dh.y, -dl.y, zc.im);
    df_fma1(w.im, dh.x, dl.x, zc.im);
    df_fma1(w.im, dh.y, dl.y, zc.re);
    df_fma(w.re, -ih.hi, -ih.lo, sr.hi, sr.lo);
    df_fma(w.im, -ih.hi, -ih.lo, si.hi, si.lo);
    w.re = df_norm(w.re);
    w.im = df_norm(w.im);
    cdf_store(wh, wl, q, w);
    const cdf u = cdf_load(uh, ul, q);
    cdf_abs2_acc(alpha, u);
    cdf_dot_acc(beta, u, w);
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      if (i < j) {
        const float2* qh = vhi(V, a, rhs, i);
        const cdf qi = cdf_load(qh, qh + a.N, q);
        cdf_dot_acc(s[i], qi, u);
        cdf_dot_acc(t[i], qi, w);
      }
    }
  }
  // block reduction in FP64 of the df partial sums
  __shared__ double sh[kDfThreads / 32][4 * NV + 3];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    if (i < j) {
      const double v0 = warp_sum(df_to_double(s[i].re)), v1 = warp_sum(df_to_double(s[i].im));
      const double v2 = warp_sum(df_to_double(t[i].re)), v3 = warp_sum(df_to_double(t[i].im));
      if (lane == 0) { sh[warp][4 * i] = v0; sh[warp][4 * i + 1] = v1; sh[warp][4 * i + 2] = v2; sh[warp][4 * i + 3] = v3; }
    }
  }
  {
    const double v0 = warp_sum(df_to_double(alpha));
    const double v1 = warp_sum(df_to_double(beta.re)), v2 = warp_sum(df_to_double(beta.im));
    if (lane == 0) { sh[warp][4 * NV] = v0; sh[warp][4 * NV + 1] = v1; sh[warp][4 * NV + 2] = v2; }
  }
  __syncthreads();
  cd* out = partial + ((size_t)rhs * a.nblk + blk) * a.pstride;
  const int nw = kDfThreads / 32;
  for (int c = threadIdx.x; c < 4 * j + 3; c += kDfThreads) {
    const int src = c < 4 * j ? c : 4 * NV + (c - 4 * j);
    double v = 0.0;
    for (int w2 = 0; w2 < nw; ++w2) v += sh[w2][src];
    double* o;
    if (c < 4 * j) {
      const int i = c >> 2, part = c & 3;          // 0: s.re 1: s.im 2: t.re 3: t.im
      o = reinterpret_cast<double*>(out + (part < 2 ? i : j + i)) + (part & 1);
    } else if (c == 4 * j) {
      o = reinterpret_cast<double*>(out + 2 * j);
      out[2 * j].im = 0.0;
    } else {
      o = reinterpret_cast<double*>(out + 2 * j + 1) + (c - 4 * j - 1);
    }
    *o = v;
  }
}

// Tail pass at the end of a cycle: s = Q_m^H u_m and alpha = ||u_m||^2 (slots as in pass 1, t = beta = 0).
template <int NV>
__global__ void __launch_bounds__(kDfThreads)
k_df_tail(KArgs a, int j, const float2* __restrict__ V, cd* __restrict__ partial, const RhsState* __restrict__ st) {
  const int rhs = blockIdx.y, blk = blockIdx.x;
  if (!st[rhs].active) return;
  const float2* uh = vhi(V, a, rhs, j);
  const float2* ul = uh + a.N;
  cdf s[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) s[i] = cdf_zero();
  df alpha = {0.f, 0.f};
  const size_t p0 = blk * a.chunk, p1 = (p0 + a.chunk < a.N) ? p0 + a.chunk : a.N;
  for (size_t q = p0 + threadIdx.x; q < p1; q += kDfThreads) {
    const cdf u = cdf_load(uh, ul, q);
    cdf_abs2_acc(alpha, u);
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      if (i < j) {
        const float2* qh = vhi(V, a, rhs, i);
        cdf_dot_acc(s[i], cdf_load(qh, qh + a.N, q), u);
      }
    }
  }
  __shared__ double sh[kDfThreads / 32][2 * NV + 1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    if (i < j) {
      const double v0 = warp_sum(df_to_double(s[i].re)), v1 = warp_sum(df_to_double(s[i].im));
      if (lane == 0) { sh[warp][2 * i] = v0; sh[warp][2 * i + 1] = v1; }
    }
  }
  {
    const double v0 = warp_sum(df_to_double(alpha));
    if (lane == 0) sh[warp][2 * NV] = v0;
  }
  __syncthreads();
  cd* out = partial + ((size_t)rhs * a.nblk + blk) * a.pstride;
  const int nw = kDfThreads / 32;
  for (int c = threadIdx.x; c < 2 * j + 1; c += kDfThreads) {
    const int src = c < 2 * j ? c : 2 * NV;
    double v = 0.0;
    for (int w2 = 0; w2 < nw; ++w2) v += sh[w2][src];
    if (c < 2 * j) reinterpret_cast<double*>(out + (c >> 1))[c & 1] = v;
    else out[2 * j] = mk<double>(v, 0.0);
  }
  if (threadIdx.x < j) out[j + threadIdx.x] = czero<double>();
  if (threadIdx.x == 0) out[2 * j + 1] = czero<double>();
}

// Per-RHS scalar work after pass 1 (or the tail pass, tail != 0): delayed correction and
// Givens rotation of column j-1, stopping test, and the coefficients of pass 2.
__global__ void k_df_scalars(KArgs a, int j, int tail, const cd* __restrict__ partial, cd* __restrict__ H,
                             double* __restrict__ cs, cd* __restrict__ sn, cd* __restrict__ g, cd* __restrict__ hpend,
                             cd* __restrict__ coef, double* __restrict__ vscale, RhsState* __restrict__ st,
                             double tol, int maxit) {
  __shared__ cd sh[2 * kMaxRestart + 4];
  const int rhs = blockIdx.x;
  if (!st[rhs].active) return;
  for (int c = threadIdx.x; c < 2 * j + 2; c += blockDim.x) {
    cd acc = czero<double>();
    for (int b = 0; b < a.nblk; ++b) acc = acc + partial[((size_t)rhs * a.nblk + b) * a.pstride + c];
    sh[c] = acc;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  const int m = a.m;
  RhsState& S = st[rhs];
  if (tail) S.rsum += j;
  const cd* s = sh;
  const cd* t = sh + j;
  const double alpha = sh[2 * j].re;
  const cd beta = sh[2 * j + 1];
  double ss = 0.0;
  for (int i = 0; i < j; ++i) ss += cabs2(s[i]);
  const double nu2 = alpha - ss;
  const bool breakdown = !(nu2 > 1e-28 * alpha);
  const double nu = breakdown ? 0.0 : sqrt(nu2);
  if (j >= 1) {
    // finalise column j-1: pending entries + delayed correction, sub-diagonal nu
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
  // column j before its delayed correction, and the pass-2 coefficients
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
  (void)vscale;
}

// Pass 2: q_j = (u_j - Q s)/nu written over u_j, u_{j+1} = w - Q t - h_jj q_j written to slot
// j+1, partial ||u_{j+1}||^2 in slot 0.
template <int NV>
__global__ void __launch_bounds__(kDfThreads)
k_df_pass2(KArgs a, int j, const cd* __restrict__ coef, float2* __restrict__ V, const float2* __restrict__ W,
           cd* __restrict__ partial, const RhsState* __restrict__ st) {
  const int rhs = blockIdx.y, blk = blockIdx.x;
  const RhsState& S = st[rhs];
  if (!S.active) return;
  __shared__ cdf cs_[NV], ct_[NV];
  const cd* cf_ = coef + (size_t)rhs * 2 * a.m;
  for (int i = threadIdx.x; i < j; i += kDfThreads) {
    cs_[i] = cdf_from(cf_[i]);
    ct_[i] = cdf_from(cf_[a.m + i]);
  }
  __syncthreads();
  const df inv_nu = df_from_double(S.inv_nu);
  cdf hjj;
  hjj.re = df_from_double(S.hjj_re);
  hjj.im = df_from_double(S.hjj_im);
  float2* uh = const_cast<float2*>(vhi(V, a, rhs, j));
  float2* ul = uh + a.N;
  float2* nh = const_cast<float2*>(vhi(V, a, rhs, j + 1));
  float2* nl = nh + a.N;
  const float2* wh = W + (size_t)rhs * 2 * a.N;
  const float2* wl = wh + a.N;
  df nrm = {0.f, 0.f};
  const size_t p0 = blk * a.chunk, p1 = (p0 + a.chunk < a.N) ? p0 + a.chunk : a.N;
  for (size_t q = p0 + threadIdx.x; q < p1; q += kDfThreads) {
    cdf u = cdf_load(uh, ul, q);
    cdf w = cdf_load(wh, wl, q);
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      if (i < j) {
        const float2* qh = vhi(V, a, rhs, i);
        const cdf qi = cdf_load(qh, qh + a.N, q);
        cdf_sub_mul(u, cs_[i], qi);
        cdf_sub_mul(w, ct_[i], qi);
      }
    }
    cdf qj;
    qj.re.hi = qj.re.lo = qj.im.hi = qj.im.lo = 0.f;
    u.re = df_norm(u.re);
    u.im = df_norm(u.im);
    df_fma(qj.re, u.re.hi, u.re.lo, inv_nu.hi, inv_nu.lo);
    df_fma(qj.im, u.im.hi, u.im.lo, inv_nu.hi, inv_nu.lo);
    qj.re = df_norm(qj.re);
    qj.im = df_norm(qj.im);
    cdf_store(uh, ul, q, qj);
    cdf_sub_mul(w, hjj, qj);
    w.re = df_norm(w.re);
    w.im = df_norm(w.im);
    cdf_store(nh, nl, q, w);
    cdf_abs2_acc(nrm, w);
  }
  cd none[1] = {czero<double>()};
  block_reduce_store<1>(none, 0, df_to_double(nrm), 0, partial + ((size_t)rhs * a.nblk + blk) * a.pstride);
}

// 1/||u_{j+1}|| for the next preconditioner input.
__global__ void k_df_unorm(KArgs a, int j, const cd* __restrict__ partial, double* __restrict__ vscale,
                           const RhsState* __restrict__ st) {
  __shared__ cd sh[1];
  const int rhs = blockIdx.x;
  if (!st[rhs].active) return;
  sum_partials(a, partial, rhs, 1, sh);
  if (threadIdx.x == 0) {
    const double n2 = sh[0].re;
    vscale[(size_t)rhs * (a.m + 1) + j + 1] = n2 > 0.0 ? 1.0 / sqrt(n2) : 1.0;
  }
}

// r = b - A x in FP64, stored as the double-float candidate u_0 in basis slot 0;
// partial ||r||^2 (slot 0) and ||b||^2 (slot 1).
__global__ void __launch_bounds__(kKThreads)
k_df_residual(KArgs a, const cd* __restrict__ b, const cd* __restrict__ x, const cd* __restrict__ DA,
              float2* __restrict__ V, cd* __restrict__ partial, const RhsState* __restrict__ st) {
  const int rhs = blockIdx.y, blk = blockIdx.x;
  if (st[rhs].done) return;
  const cd* xb = x + (size_t)rhs * a.N;
  const cd* bb = b + (size_t)rhs * a.N;
  float2* rh = const_cast<float2*>(vhi(V, a, rhs, 0));
  float2* rl = rh + a.N;
  cd acc[1] = {czero<double>()};
  double bn = 0.0;
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
    const cd bv = bb[q];
    const cd rv = bv - (DA[q] * xb[q] - a.inv_h2 * s);
    const cdf r = cdf_from(rv);
    rh[q] = make_float2(r.re.hi, r.im.hi);
    rl[q] = make_float2(r.re.lo, r.im.lo);
    acc[0].re += cabs2(rv);
    bn += cabs2(bv);
  }
  block_reduce_store<1>(acc, 1, bn, 1, partial + ((size_t)rhs * a.nblk + blk) * a.pstride);
}

// x += sum_{i < jend} y_i z_i with the sum formed in double-float (z_i FP32), added to FP64 x.
template <int NV>
__global__ void __launch_bounds__(kKThreads)
k_df_xupdate(KArgs a, const cf* __restrict__ Z, const cd* __restrict__ y, cd* __restrict__ x,
             const RhsState* __restrict__ st) {
  const int rhs = blockIdx.y;
  if (st[rhs].done || st[rhs].jend == 0) return;
  const int je = st[rhs].jend;
  __shared__ cdf ys[NV];
  if (threadIdx.x < NV && (int)threadIdx.x < je) ys[threadIdx.x] = cdf_from(y[(size_t)rhs * a.m + threadIdx.x]);
  __syncthreads();
  const cf* Zb = Z + (size_t)rhs * a.m * a.N;
  cd* xb = x + (size_t)rhs * a.N;
  const size_t p0 = blockIdx.x * a.chunk, p1 = (p0 + a.chunk < a.N) ? p0 + a.chunk : a.N;
  for (size_t q = p0 + threadIdx.x; q < p1; q += kKThreads) {
    df sr = {0.f, 0.f}, si = {0.f, 0.f};
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      if (i < je) {
        const cf z = Zb[(size_t)i * a.N + q];
        df_fma1(sr, ys[i].re.hi, ys[i].re.lo, z.re);
        df_fma1(sr, -ys[i].im.hi, -ys[i].im.lo, z.im);
        df_fma1(si, ys[i].re.hi, ys[i].re.lo, z.im);
        df_fma1(si, ys[i].im.hi, ys[i].im.lo, z.re);
      }
    }
    cd v = xb[q];
    v.re += df_to_double(sr);
    v.im += df_to_double(si);
    xb[q] = v;
  }
}

template <int NV>
mgh_status df_step_nv(Handle& h, const KArgs& a, int j, int B) {
  const dim3 grid(a.nblk, B);
  const float2* Vd = reinterpret_cast<const float2*>(h.V);
  float2* Wd = reinterpret_cast<float2*>(h.W);
  {
    ProfScope ps(h, P_MATVEC_DOTS);
    k_df_pass1<NV><<<grid, kDfThreads, 0, h.stream>>>(a, j, (const cf*)h.Z, h.DAdf, Vd, Wd, h.partial, h.st);
    MGH_CHECK_LAUNCH(); h.launches++;
  }
  {
    ProfScope ps(h, P_REDUCE);
    k_df_scalars<<<B, 64, 0, h.stream>>>(a, j, 0, h.partial, h.H, h.cs, h.sn, h.g, h.hpend, h.coef, h.vscale,
                                         h.st, h.p.tol, h.p.maxit);
    MGH_CHECK_LAUNCH(); h.launches++;
  }
  {
    ProfScope ps(h, P_UPDATE);
    k_df_pass2<NV><<<grid, kDfThreads, 0, h.stream>>>(a, j, h.coef, reinterpret_cast<float2*>(h.V), Wd, h.partial,
                                                      h.st);
    MGH_CHECK_LAUNCH(); h.launches++;
  }
  {
    ProfScope ps(h, P_REDUCE);
    k_df_unorm<<<B, 32, 0, h.stream>>>(a, j, h.partial, h.vscale, h.st);
    MGH_CHECK_LAUNCH(); h.launches++;
  }
  return MGH_OK;
}

template <int NV>
mgh_status df_tail_nv(Handle& h, const KArgs& a, int j, int B) {
  const dim3 grid(a.nblk, B);
  {
    ProfScope ps(h, P_REORTH);
    k_df_tail<NV><<<grid, kDfThreads, 0, h.stream>>>(a, j, reinterpret_cast<const float2*>(h.V), h.partial, h.st);
    MGH_CHECK_LAUNCH(); h.launches++;
  }
  {
    ProfScope ps(h, P_REDUCE);
    k_df_scalars<<<B, 64, 0, h.stream>>>(a, j, 1, h.partial, h.H, h.cs, h.sn, h.g, h.hpend, h.coef, h.vscale,
                                         h.st, h.p.tol, h.p.maxit);
    MGH_CHECK_LAUNCH(); h.launches++;
  }
  return MGH_OK;
}

mgh_status df_arnoldi_step(Handle& h, const KArgs& a, int j, int B) {
  // z_j = M^{-1}(u_j / ||u_j||), reading only the hi plane of u_j
  const cf* uhi = reinterpret_cast<const cf*>(reinterpret_cast<const float2*>(h.V) + (size_t)j * 2 * a.N);
  MGH_TRY(vcycle_f32in(h, uhi, (size_t)(a.m + 1) * 2 * a.N, h.vscale + j, (size_t)(a.m + 1),
                       (cf*)h.Z + (size_t)j * a.N, (size_t)a.m * a.N, B, h.st));
  if (j <= 4) return df_step_nv<4>(h, a, j, B);
  if (j <= 8) return df_step_nv<8>(h, a, j, B);
  if (j <= 12) return df_step_nv<12>(h, a, j, B);
  if (j <= 16) return df_step_nv<16>(h, a, j, B);
  return df_step_nv<kMaxRestartDf>(h, a, j, B);
}

mgh_status df_tail(Handle& h, const KArgs& a, int j, int B) {
  if (j <= 4) return df_tail_nv<4>(h, a, j, B);
  if (j <= 8) return df_tail_nv<8>(h, a, j, B);
  if (j <= 12) return df_tail_nv<12>(h, a, j, B);
  if (j <= 16) return df_tail_nv<16>(h, a, j, B);
  return df_tail_nv<kMaxRestartDf>(h, a, j, B);
}

mgh_status fgmres_df(Handle& h, const cd* b, int B, cd* x, mgh_solve_info* info) {
  KArgs a = make_kargs(h, B);
  const dim3 grid(a.nblk, B);
  float2* Vd = reinterpret_cast<float2*>(h.V);
  {
    ProfScope ps(h, P_REDUCE);
    k_state_reset<<<(B + 63) / 64, 64, 0, h.stream>>>(h.st, B);
    MGH_CHECK_LAUNCH(); h.launches++;
  }
  {
    ProfScope ps(h, P_RESIDUAL);
    k_df_residual<<<grid, kKThreads, 0, h.stream>>>(a, b, x, h.DA, Vd, h.partial, h.st);
    MGH_CHECK_LAUNCH(); h.launches++;
  }
  {
    ProfScope ps(h, P_REDUCE);
    k_cycle_start<<<B, 32, 0, h.stream>>>(a, h.partial, h.vscale, h.g, h.st, h.p.tol, h.p.maxit, 1);
    MGH_CHECK_LAUNCH(); h.launches++;
  }
  {
    ProfScope ps(h, P_OTHER);
    k_zero_if_b_zero<<<grid, kKThreads, 0, h.stream>>>(a, x, h.st);
    MGH_CHECK_LAUNCH(); h.launches++;
  }
  for (;;) {
    MGH_CUDA(cudaMemcpyAsync(h.st_host, h.st, sizeof(RhsState) * B, cudaMemcpyDeviceToHost, h.stream));
    MGH_CUDA(cudaStreamSynchronize(h.stream));
    MGH_TRY(prof_flush(h));
    bool any = false;
    for (int i = 0; i < B; ++i) any |= (h.st_host[i].done == 0);
    if (!any) break;
    for (int j = 0; j < a.m; ++j) MGH_TRY(df_arnoldi_step(h, a, j, B));
    MGH_TRY(df_tail(h, a, a.m, B));
    {
      ProfScope ps(h, P_REDUCE);
      k_lsq<<<(B + 63) / 64, 64, 0, h.stream>>>(a, h.H, h.g, h.y, h.st, B);
      MGH_CHECK_LAUNCH(); h.launches++;
    }
    {
      ProfScope ps(h, P_XUPDATE);
      const int m = a.m;
      if (m <= 4) k_df_xupdate<4><<<grid, kKThreads, 0, h.stream>>>(a, (const cf*)h.Z, h.y, x, h.st);
      else if (m <= 8) k_df_xupdate<8><<<grid, kKThreads, 0, h.stream>>>(a, (const cf*)h.Z, h.y, x, h.st);
      else if (m <= 12) k_df_xupdate<12><<<grid, kKThreads, 0, h.stream>>>(a, (const cf*)h.Z, h.y, x, h.st);
      else if (m <= 16) k_df_xupdate<16><<<grid, kKThreads, 0, h.stream>>>(a, (const cf*)h.Z, h.y, x, h.st);
      else k_df_xupdate<kMaxRestartDf><<<grid, kKThreads, 0, h.stream>>>(a, (const cf*)h.Z, h.y, x, h.st);
      MGH_CHECK_LAUNCH(); h.launches++;
    }
    {
      ProfScope ps(h, P_RESIDUAL);
      k_df_residual<<<grid, kKThreads, 0, h.stream>>>(a, b, x, h.DA, Vd, h.partial, h.st);
      MGH_CHECK_LAUNCH(); h.launches++;
    }
    {
      ProfScope ps(h, P_REDUCE);
      k_cycle_start<<<B, 32, 0, h.stream>>>(a, h.partial, h.vscale, h.g, h.st, h.p.tol, h.p.maxit, 0);
      MGH_CHECK_LAUNCH(); h.launches++;
    }
  }
  return finish_solve(h, B, info);
}

}  // namespace

mgh_status fgmres_solve(Handle& h, const cd* b, int B, cd* x, mgh_solve_info* info) {
  if (h.fp64) return fgmres_t<double>(h, b, B, x, info);
  if (h.p.arnoldi == MGH_ARNOLDI_FP64) return fgmres_t<float>(h, b, B, x, info);
  return fgmres_df(h, b, B, x, info);
}

}  // namespace mgh
