// Batched right-preconditioned flexible GMRES(m) with native FP64 Arnoldi (Saad & Schultz 1986;
// Saad 1993): the engine of the FP64 path, and of the mixed path when MGH_ARNOLDI_FP64 is chosen
// (the default mixed-precision engine, double-float Arnoldi, is in mgh_krylov_df.cu),
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
#include <complex>
#include <thread>
#include <vector>

#include "mgh_krylov_common.cuh"

namespace mgh {

namespace {


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
                         RhsState* __restrict__ st, int B, double tol, int maxit, cd* __restrict__ Hraw) {
  const int rhs = blockIdx.x * blockDim.x + threadIdx.x;
  if (rhs >= B || !st[rhs].active) return;
  const int m = a.m;
  cd col[kMaxRestart + 1];
  for (int i = 0; i <= j; ++i) col[i] = hcol[(size_t)rhs * (m + 1) + i];
  const double hn = sqrt(fmax(st[rhs].norm2, 0.0));
  col[j + 1] = mk<double>(hn, 0.0);
  if (Hraw) {   // the column before rotation, kept for a deflated restart
    cd* hr = Hraw + ((size_t)rhs * m + j) * (m + 1);
    for (int i = 0; i <= j + 1; ++i) hr[i] = col[i];
  }
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

// r = b - A x into basis slot 0 (into W when the cycle restarts deflated: kdefl > 0 and the cycle
// ran its m steps); partial ||r||^2 (slot 0) and ||b||^2 (slot 1).
__global__ void __launch_bounds__(kKThreads)
k_residual(KArgs a, const cd* __restrict__ b, const cd* __restrict__ x, const cd* __restrict__ DA,
           cd* __restrict__ V, cd* __restrict__ W, cd* __restrict__ partial, const RhsState* __restrict__ st,
           int kdefl) {
  const int rhs = blockIdx.y, blk = blockIdx.x;
  if (st[rhs].done) return;
  const cd* xb = x + (size_t)rhs * a.N;
  const cd* bb = b + (size_t)rhs * a.N;
  cd* r = (kdefl > 0 && st[rhs].jend == a.m) ? W + (size_t)rhs * a.N : V + (size_t)rhs * (a.m + 1) * a.N;
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




// ---------------------------------------------------------------- deflated restart (GMRES-DR)
// After a full-length cycle whose iterate has not converged, the host computes per right-hand
// side the restart data of the k harmonic Ritz vectors (row-major at drbuf + rhs * dr_stride:
// C m x k, Hh (k+1) x k upper Hessenberg, R k x k, k Givens cosines (real parts) and sines) and a
// mode: 0 no restart work, 1 deflated restart, 2 plain restart from the true residual held in W
// (the host routine gave up).  The device then
//   V'_j = sum_{i<m} v_i C_ij,  Z'_j = sum_{i<m} z_i C_ij  (j < k, in place per point),
//   v'_k = the true residual orthogonalised against V'_0..V'_{k-1} (two classical passes),
// and starts the next cycle at column k with Hessenberg columns 0..k-1 = Hh (raw) and R (rotated),
// the host's rotations, and g = the rotated [V'^H r; ||r_perp||].  Taking v'_k from the true
// residual keeps rounding in the stored vectors (Z' in the cycle precision) from accumulating in
// the residual the least-squares problem sees.
__host__ __device__ inline size_t dr_stride(int m, int k) {
  return (size_t)m * k + (size_t)(k + 1) * k + (size_t)k * k + 2 * (size_t)k;
}

template <typename TZ, int KC>
__global__ void __launch_bounds__(kKThreads)
k_dr_combine(KArgs a, int k, const cd* __restrict__ drbuf, const int* __restrict__ mode,
             const double* __restrict__ vscale, cd* __restrict__ V, Cx<TZ>* __restrict__ Z,
             const cd* __restrict__ W) {
  const int rhs = blockIdx.y;
  const int md = mode[rhs];
  if (md == 0) return;
  const int m = a.m;
  cd* Vb = V + (size_t)rhs * (m + 1) * a.N;
  const size_t p0 = blockIdx.x * a.chunk, p1 = (p0 + a.chunk < a.N) ? p0 + a.chunk : a.N;
  if (md == 2) {   // plain restart: the residual becomes basis slot 0
    const cd* Wb = W + (size_t)rhs * a.N;
    for (size_t q = p0 + threadIdx.x; q < p1; q += kKThreads) Vb[q] = Wb[q];
    return;
  }
  __shared__ cd cv[kMaxRestart * KC];   // C with each row scaled by the multiplier of v_i
  __shared__ cd cz[kMaxRestart * KC];
  const cd* d = drbuf + (size_t)rhs * dr_stride(m, k);
  for (int t = threadIdx.x; t < m * k; t += kKThreads) {
    const int i = t / k, jj = t - i * k;
    cv[i * KC + jj] = vscale[(size_t)rhs * (m + 1) + i] * d[t];
    cz[i * KC + jj] = d[t];
  }
  __syncthreads();
  Cx<TZ>* Zb = Z + (size_t)rhs * m * a.N;
  for (size_t q = p0 + threadIdx.x; q < p1; q += kKThreads) {
    cd acc[KC];
#pragma unroll
    for (int jj = 0; jj < KC; ++jj) acc[jj] = czero<double>();
    for (int i = 0; i < m; ++i) {
      const cd v = Vb[(size_t)i * a.N + q];
#pragma unroll
      for (int jj = 0; jj < KC; ++jj)
        if (jj < k) acc[jj] = acc[jj] + cv[i * KC + jj] * v;
    }
#pragma unroll
    for (int jj = 0; jj < KC; ++jj)
      if (jj < k) Vb[(size_t)jj * a.N + q] = acc[jj];
#pragma unroll
    for (int jj = 0; jj < KC; ++jj) acc[jj] = czero<double>();
    for (int i = 0; i < m; ++i) {
      const cd z = load_z(Zb, (size_t)i * a.N + q);
#pragma unroll
      for (int jj = 0; jj < KC; ++jj)
        if (jj < k) acc[jj] = acc[jj] + cz[i * KC + jj] * z;
    }
#pragma unroll
    for (int jj = 0; jj < KC; ++jj)
      if (jj < k) Zb[(size_t)jj * a.N + q] = ccast<TZ>(acc[jj]);
  }
}

// Gram-Schmidt of the true residual against V'_0..V'_{k-1} (normalised, multiplier 1):
//   pass 0: partial <- <V'_i, r> and ||r||^2 (src = W, no write)
//   pass 1: v_k = r - sum_i c_i V'_i (c = hcol); partial <- <V'_i, v_k> and ||v_k||^2
//   pass 2: v_k -= sum_i c2_i V'_i (c2 = h2col); partial slot k <- ||v_k||^2
template <int KC>
__global__ void __launch_bounds__(kKThreads)
k_dr_orth(KArgs a, int k, int pass, const int* __restrict__ mode, const cd* __restrict__ coef,
          cd* __restrict__ V, const cd* __restrict__ W, cd* __restrict__ partial) {
  const int rhs = blockIdx.y, blk = blockIdx.x;
  if (mode[rhs] != 1) return;
  const int m = a.m;
  __shared__ cd cs_[KC];
  if (pass > 0 && threadIdx.x < k) cs_[threadIdx.x] = coef[(size_t)rhs * (m + 1) + threadIdx.x];
  __syncthreads();
  cd* Vb = V + (size_t)rhs * (m + 1) * a.N;
  const cd* Wb = W + (size_t)rhs * a.N;
  cd acc[KC];
#pragma unroll
  for (int i = 0; i < KC; ++i) acc[i] = czero<double>();
  double nrm = 0.0;
  const size_t p0 = blk * a.chunk, p1 = (p0 + a.chunk < a.N) ? p0 + a.chunk : a.N;
  for (size_t q = p0 + threadIdx.x; q < p1; q += kKThreads) {
    cd w = pass == 2 ? Vb[(size_t)k * a.N + q] : Wb[q];
    if (pass > 0) {
#pragma unroll
      for (int i = 0; i < KC; ++i)
        if (i < k) caxpy_neg(w, cs_[i], Vb[(size_t)i * a.N + q]);
      Vb[(size_t)k * a.N + q] = w;
    }
    nrm += cabs2(w);
    if (pass < 2) {
#pragma unroll
      for (int i = 0; i < KC; ++i)
        if (i < k) cdot_acc(acc[i], Vb[(size_t)i * a.N + q], w);
    }
  }
  block_reduce_store<KC>(acc, pass < 2 ? k : 0, nrm, k, partial + ((size_t)rhs * a.nblk + blk) * a.pstride);
}

// Sums of k_dr_orth's partials (one block per RHS): pass 0 -> hcol; pass 1 -> h2col, hcol += h2col.
__global__ void k_dr_fin(KArgs a, int k, int pass, const int* __restrict__ mode, const cd* __restrict__ partial,
                         cd* __restrict__ hcol, cd* __restrict__ h2col) {
  __shared__ cd sh[kMaxRestart + 2];
  const int rhs = blockIdx.x;
  if (mode[rhs] != 1) return;
  sum_partials(a, partial, rhs, k + 1, sh);
  const size_t o = (size_t)rhs * (a.m + 1);
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    if (pass == 0) {
      hcol[o + i] = sh[i];
    } else {
      h2col[o + i] = sh[i];
      hcol[o + i] = hcol[o + i] + sh[i];
    }
  }
}

// Start of the next cycle (one block per RHS).  Mode 1: g0 = [hcol_0..hcol_{k-1}, ||v_k||, 0..]
// (kept unrotated for the next restart) and g = g0 rotated by the host's k rotations; multipliers
// 1 for V'_0..V'_{k-1} and 1/||v_k|| for v_k; Hessenberg columns 0..k-1 = Hh (raw) and [R; 0]
// (rotated); first new column k (activated when the step loop reaches it).  Mode 2: the plain
// start from the residual norm.
__global__ void k_dr_finish(KArgs a, int k, const int* __restrict__ mode, const cd* __restrict__ drbuf,
                            const cd* __restrict__ partial, const cd* __restrict__ hcol, double* __restrict__ vscale,
                            cd* __restrict__ g, cd* __restrict__ g0, cd* __restrict__ H, cd* __restrict__ Hraw,
                            double* __restrict__ cs, cd* __restrict__ sn, RhsState* __restrict__ st) {
  __shared__ cd sh[kMaxRestart + 2];
  const int rhs = blockIdx.x;
  const int md = mode[rhs];
  if (md == 0) return;
  const int m = a.m;
  RhsState& S = st[rhs];
  cd* gg = g + (size_t)rhs * (m + 1);
  cd* g0b = g0 + (size_t)rhs * (m + 1);
  double* vs = vscale + (size_t)rhs * (m + 1);
  if (md == 2) {
    if (threadIdx.x == 0) {
      const double rn = S.rnorm;
      vs[0] = 1.0 / rn;
      for (int i = 0; i <= m; ++i) gg[i] = g0b[i] = i == 0 ? mk<double>(rn, 0.0) : czero<double>();
      S.deflate = 0;
      S.jstart = 0;
      S.active = 1;
    }
    return;
  }
  sum_partials(a, partial, rhs, k + 1, sh);
  const double nk = sqrt(fmax(sh[k].re, 0.0));
  const cd* d = drbuf + (size_t)rhs * dr_stride(m, k);
  const cd* Hh = d + (size_t)m * k;
  const cd* R = Hh + (size_t)(k + 1) * k;
  const cd* rc = R + (size_t)k * k;
  const cd* rs = rc + k;
  for (int t = threadIdx.x; t < k * (m + 1); t += blockDim.x) {   // columns 0..k-1 of H and Hraw
    const int jc = t / (m + 1), i = t - jc * (m + 1);
    H[((size_t)rhs * m + jc) * (m + 1) + i] = i < k ? R[(size_t)i * k + jc] : czero<double>();
    Hraw[((size_t)rhs * m + jc) * (m + 1) + i] = i <= k ? Hh[(size_t)i * k + jc] : czero<double>();
  }
  for (int i = threadIdx.x; i <= m; i += blockDim.x) {
    g0b[i] = i < k ? hcol[(size_t)rhs * (m + 1) + i] : (i == k ? mk<double>(nk, 0.0) : czero<double>());
    if (i < k) vs[i] = 1.0;
  }
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    cs[(size_t)rhs * m + i] = rc[i].re;
    sn[(size_t)rhs * m + i] = rs[i];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 0; i <= m; ++i) gg[i] = g0b[i];
    for (int i = 0; i < k; ++i) {
      const double c = rc[i].re;
      const cd s = rs[i];
      const cd t = c * gg[i] + s * gg[i + 1];
      gg[i + 1] = (-1.0 * cconj(s)) * gg[i] + c * gg[i + 1];
      gg[i] = t;
    }
    vs[k] = nk > 0.0 ? 1.0 / nk : 0.0;
    S.deflate = 0;
    S.jstart = k;
    S.jend = k;
    S.active = 0;
    if (!(nk > 0.0)) { S.done = 1; S.converged = 0; }
  }
}

// Right-hand sides whose cycle starts at column j join the step loop there.
__global__ void k_dr_activate(RhsState* st, int B, int j) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < B && !st[i].done && st[i].jstart == j && j > 0) st[i].active = 1;
}

// Cycle start of the deflated engine: k_cycle_start's decisions, but a right-hand side whose
// cycle ran all m steps (its residual is in W) is marked for the host's deflated restart instead
// of restarting from basis slot 0.
__global__ void k_cycle_start_dr(KArgs a, const cd* __restrict__ partial, double* __restrict__ vscale,
                                 cd* __restrict__ g, cd* __restrict__ g0, RhsState* __restrict__ st, double tol,
                                 int maxit, int first, int kdefl) {
  __shared__ cd sh[2];
  const int rhs = blockIdx.x;
  if (st[rhs].done) return;
  sum_partials(a, partial, rhs, 2, sh);
  if (threadIdx.x != 0) return;
  RhsState& S = st[rhs];
  const bool defl = !first && kdefl > 0 && S.jend == a.m;
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
  S.deflate = 0;
  S.jstart = 0;
  if (S.bnorm == 0.0) { S.done = 1; S.converged = 1; return; }
  if (rn <= tol * S.bnorm) { S.done = 1; S.converged = 1; return; }
  if (S.iterations >= maxit || !(rn == rn)) { S.done = 1; S.converged = 0; return; }
  if (defl) { S.deflate = 1; return; }
  S.active = 1;
  vscale[(size_t)rhs * (a.m + 1)] = 1.0 / rn;
  cd* gg = g + (size_t)rhs * (a.m + 1);
  cd* g0b = g0 + (size_t)rhs * (a.m + 1);
  for (int i = 0; i <= a.m; ++i) gg[i] = g0b[i] = i == 0 ? mk<double>(rn, 0.0) : czero<double>();
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
                                                 h.p.maxit, h.p.deflate > 0 ? h.Hraw : nullptr);
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
    k_residual<<<grid, kKThreads, 0, h.stream>>>(a, b, x, h.DA, h.V, h.W, h.partial, h.st, h.p.deflate);
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
  // a restart cycle: every launch is gated by the per-RHS state, so after the first cycle its
  // launches are replayed from a captured graph
  CycleGraph graph;
  auto body = [&]() -> mgh_status {
    for (int j = 0; j < a.m; ++j) MGH_TRY(arnoldi_step<TZ>(h, a, j, B));
    {
      ProfScope ps(h, P_REDUCE);
      k_lsq<<<(B + 63) / 64, 64, 0, h.stream>>>(a, h.H, h.g, h.y, h.st, B);
      MGH_CHECK_LAUNCH(); h.launches++;
    }
    MGH_TRY(xupdate<TZ>(h, a, B, x));
    {
      ProfScope ps(h, P_RESIDUAL);
      k_residual<<<grid, kKThreads, 0, h.stream>>>(a, b, x, h.DA, h.V, h.W, h.partial, h.st, h.p.deflate);
      MGH_CHECK_LAUNCH(); h.launches++;
    }
    {
      ProfScope ps(h, P_REDUCE);
      k_cycle_start<<<B, 32, 0, h.stream>>>(a, h.partial, h.vscale, h.g, h.st, h.p.tol, h.p.maxit, 0);
      MGH_CHECK_LAUNCH(); h.launches++;
    }
    return MGH_OK;
  };
  for (int ncycle = 0;; ++ncycle) {
    MGH_CUDA(cudaMemcpyAsync(h.st_host, h.st, sizeof(RhsState) * B, cudaMemcpyDeviceToHost, h.stream));
    MGH_CUDA(cudaStreamSynchronize(h.stream));
    MGH_TRY(prof_flush(h));
    bool any = false;
    for (int i = 0; i < B; ++i) any |= (h.st_host[i].done == 0);
    if (!any) break;
    if (!h.use_graphs || h.prof || ncycle == 0) MGH_TRY(body());
    else MGH_TRY(graph.run(h, body));
  }
  return finish_solve(h, B, info);
}


template <typename TZ, int KC>
mgh_status dr_restart_kc(Handle& h, const KArgs& a, int B, int k) {
  const dim3 grid(a.nblk, B);
  {
    ProfScope ps(h, P_UPDATE);
    k_dr_combine<TZ, KC><<<grid, kKThreads, 0, h.stream>>>(a, k, h.drbuf, h.dr_mode, h.vscale, h.V,
                                                          (Cx<TZ>*)h.Z, h.W);
    MGH_CHECK_LAUNCH(); h.launches++;
  }
  for (int pass = 0; pass < 3; ++pass) {
    {
      ProfScope ps(h, pass == 0 ? P_MATVEC_DOTS : (pass == 1 ? P_UPDATE : P_REORTH));
      k_dr_orth<KC><<<grid, kKThreads, 0, h.stream>>>(a, k, pass, h.dr_mode, pass == 1 ? h.hcol : h.h2col, h.V,
                                                      h.W, h.partial);
      MGH_CHECK_LAUNCH(); h.launches++;
    }
    if (pass < 2) {
      ProfScope ps(h, P_REDUCE);
      k_dr_fin<<<B, 64, 0, h.stream>>>(a, k, pass, h.dr_mode, h.partial, h.hcol, h.h2col);
      MGH_CHECK_LAUNCH(); h.launches++;
    }
  }
  {
    ProfScope ps(h, P_REDUCE);
    k_dr_finish<<<B, 64, 0, h.stream>>>(a, k, h.dr_mode, h.drbuf, h.partial, h.hcol, h.vscale, h.g, h.g0, h.H,
                                        h.Hraw, h.cs, h.sn, h.st);
    MGH_CHECK_LAUNCH(); h.launches++;
  }
  return MGH_OK;
}

// Host part of the deflated restarts of one cycle end: restart data of every right-hand side the
// device marked (in parallel threads when there are several), then the device restart.  Returns
// in *j0 the first column the next cycle's step loop must visit and in *any_defl whether some
// right-hand side starts at column k.
template <typename TZ>
mgh_status dr_restart(Handle& h, const KArgs& a, int B, int* j0, bool* any_defl) {
  const int m = a.m, k = h.p.deflate;
  const size_t stride = dr_stride(m, k);
  std::vector<int> idx;
  *j0 = m;
  *any_defl = false;
  for (int i = 0; i < B; ++i) {
    const RhsState& S = h.st_host[i];
    h.dr_mode_host[i] = 0;
    if (S.done) continue;
    if (S.deflate) idx.push_back(i); else *j0 = 0;
  }
  if (idx.empty()) return MGH_OK;
  auto work = [&](size_t lo, size_t hi) {
    using cplx = std::complex<double>;
    std::vector<cplx> Hb((size_t)(m + 1) * m), c(m + 1);
    std::vector<double> rc(k);
    for (size_t t = lo; t < hi; ++t) {
      const int rhs = idx[t];
      const cd* hr = h.dr_hraw_host + (size_t)rhs * m * (m + 1);
      const cd* g0 = h.dr_g0_host + (size_t)rhs * (m + 1);
      const cd* y = h.dr_y_host + (size_t)rhs * m;
      for (int i = 0; i <= m; ++i)
        for (int j = 0; j < m; ++j) {
          const cd v = hr[(size_t)j * (m + 1) + i];
          Hb[(size_t)i * m + j] = cplx(v.re, v.im);
        }
      for (int i = 0; i <= m; ++i) {   // c = g0 - Hbar y: the residual's coefficients in V
        cplx s(g0[i].re, g0[i].im);
        for (int j = 0; j < m; ++j) s -= Hb[(size_t)i * m + j] * cplx(y[j].re, y[j].im);
        c[i] = s;
      }
      cplx* out = reinterpret_cast<cplx*>(h.dr_host + (size_t)rhs * stride);
      cplx* C = out;
      cplx* Hh = C + (size_t)m * k;
      cplx* R = Hh + (size_t)(k + 1) * k;
      cplx* cs = R + (size_t)k * k;
      cplx* sn = cs + k;
      const bool ok = !h.dr_force_plain && deflate_restart(m, k, Hb.data(), c.data(), C, Hh, R, rc.data(), sn);
      for (int i = 0; i < k; ++i) cs[i] = cplx(rc[i], 0.0);
      h.dr_mode_host[rhs] = ok ? 1 : 2;
    }
  };
  const size_t n = idx.size();
  const unsigned hc = std::max(1u, std::thread::hardware_concurrency());
  const size_t nt = std::min<size_t>({n / 2 + 1, (size_t)hc, (size_t)16});
  if (nt <= 1) {
    work(0, n);
  } else {
    std::vector<std::thread> th;
    const size_t per = (n + nt - 1) / nt;
    for (size_t t = 0; t < nt; ++t) {
      const size_t lo = t * per, hi = std::min(n, lo + per);
      if (lo < hi) th.emplace_back(work, lo, hi);
    }
    for (std::thread& t : th) t.join();
  }
  for (int rhs : idx) {
    if (h.dr_mode_host[rhs] == 1) *any_defl = true; else *j0 = 0;
  }
  if (*any_defl) *j0 = std::min(*j0, k);
  MGH_CUDA(cudaMemcpyAsync(h.dr_mode, h.dr_mode_host, sizeof(int) * B, cudaMemcpyHostToDevice, h.stream));
  MGH_CUDA(cudaMemcpyAsync(h.drbuf, h.dr_host, sizeof(cd) * stride * B, cudaMemcpyHostToDevice, h.stream));
  if (k <= 4) return dr_restart_kc<TZ, 4>(h, a, B, k);
  if (k <= 8) return dr_restart_kc<TZ, 8>(h, a, B, k);
  return dr_restart_kc<TZ, 16>(h, a, B, k);
}

// FGMRES(m) with deflated restarting (the deflate parameter k >= 1): the plain engine's cycle, with
// each full-length cycle that has not converged followed by the deflated restart above; a cycle
// that ends early (its Givens estimate met the target, maxit, breakdown) restarts plainly.
template <typename TZ>
mgh_status fgmres_dr_t(Handle& h, const cd* b, int B, cd* x, mgh_solve_info* info) {
  KArgs a = make_kargs(h, B);
  const dim3 grid(a.nblk, B);
  const int k = h.p.deflate;
  {
    ProfScope ps(h, P_REDUCE);
    k_state_reset<<<(B + 63) / 64, 64, 0, h.stream>>>(h.st, B);
    MGH_CHECK_LAUNCH(); h.launches++;
  }
  {
    ProfScope ps(h, P_RESIDUAL);
    k_residual<<<grid, kKThreads, 0, h.stream>>>(a, b, x, h.DA, h.V, h.W, h.partial, h.st, k);
    MGH_CHECK_LAUNCH(); h.launches++;
  }
  {
    ProfScope ps(h, P_REDUCE);
    k_cycle_start_dr<<<B, 32, 0, h.stream>>>(a, h.partial, h.vscale, h.g, h.g0, h.st, h.p.tol, h.p.maxit, 1, k);
    MGH_CHECK_LAUNCH(); h.launches++;
  }
  {
    ProfScope ps(h, P_OTHER);
    k_zero_if_b_zero<<<grid, kKThreads, 0, h.stream>>>(a, x, h.st);
    MGH_CHECK_LAUNCH(); h.launches++;
  }
  for (;;) {
    MGH_CUDA(cudaMemcpyAsync(h.st_host, h.st, sizeof(RhsState) * B, cudaMemcpyDeviceToHost, h.stream));
    MGH_CUDA(cudaMemcpyAsync(h.dr_hraw_host, h.Hraw, sizeof(cd) * (size_t)B * a.m * (a.m + 1),
                             cudaMemcpyDeviceToHost, h.stream));
    MGH_CUDA(cudaMemcpyAsync(h.dr_g0_host, h.g0, sizeof(cd) * (size_t)B * (a.m + 1), cudaMemcpyDeviceToHost,
                             h.stream));
    MGH_CUDA(cudaMemcpyAsync(h.dr_y_host, h.y, sizeof(cd) * (size_t)B * a.m, cudaMemcpyDeviceToHost, h.stream));
    MGH_CUDA(cudaStreamSynchronize(h.stream));
    MGH_TRY(prof_flush(h));
    bool any = false;
    for (int i = 0; i < B; ++i) any |= (h.st_host[i].done == 0);
    if (!any) break;
    int j0 = 0;
    bool any_defl = false;
    MGH_TRY(dr_restart<TZ>(h, a, B, &j0, &any_defl));
    for (int j = j0; j < a.m; ++j) {
      if (any_defl && j == k) {
        ProfScope ps(h, P_REDUCE);
        k_dr_activate<<<(B + 63) / 64, 64, 0, h.stream>>>(h.st, B, j);
        MGH_CHECK_LAUNCH(); h.launches++;
      }
      MGH_TRY(arnoldi_step<TZ>(h, a, j, B));
    }
    {
      ProfScope ps(h, P_REDUCE);
      k_lsq<<<(B + 63) / 64, 64, 0, h.stream>>>(a, h.H, h.g, h.y, h.st, B);
      MGH_CHECK_LAUNCH(); h.launches++;
    }
    MGH_TRY(xupdate<TZ>(h, a, B, x));
    {
      ProfScope ps(h, P_RESIDUAL);
      k_residual<<<grid, kKThreads, 0, h.stream>>>(a, b, x, h.DA, h.V, h.W, h.partial, h.st, k);
      MGH_CHECK_LAUNCH(); h.launches++;
    }
    {
      ProfScope ps(h, P_REDUCE);
      k_cycle_start_dr<<<B, 32, 0, h.stream>>>(a, h.partial, h.vscale, h.g, h.g0, h.st, h.p.tol, h.p.maxit, 0, k);
      MGH_CHECK_LAUNCH(); h.launches++;
    }
  }
  return finish_solve(h, B, info);
}

}  // namespace

mgh_status fgmres_solve(Handle& h, const cd* b, int B, cd* x, mgh_solve_info* info) {
  if (h.p.krylov == MGH_KRYLOV_BICGSTAB) return bicgstab_solve(h, b, B, x, info);
  if (h.p.krylov == MGH_KRYLOV_IDRS) return idrs_solve(h, b, B, x, info);
  if (h.fp64) return h.p.deflate > 0 ? fgmres_dr_t<double>(h, b, B, x, info) : fgmres_t<double>(h, b, B, x, info);
  if (h.p.arnoldi == MGH_ARNOLDI_FP64)
    return h.p.deflate > 0 ? fgmres_dr_t<float>(h, b, B, x, info) : fgmres_t<float>(h, b, B, x, info);
  if (h.p.arnoldi == MGH_ARNOLDI_SSTEP) return fgmres_ss(h, b, B, x, info);
  return fgmres_df(h, b, B, x, info);
}

}  // namespace mgh
