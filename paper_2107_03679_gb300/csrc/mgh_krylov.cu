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

}  // namespace

mgh_status fgmres_solve(Handle& h, const cd* b, int B, cd* x, mgh_solve_info* info) {
  if (h.p.krylov == MGH_KRYLOV_BICGSTAB) return bicgstab_solve(h, b, B, x, info);
  if (h.fp64) return fgmres_t<double>(h, b, B, x, info);
  if (h.p.arnoldi == MGH_ARNOLDI_FP64) return fgmres_t<float>(h, b, B, x, info);
  if (h.p.arnoldi == MGH_ARNOLDI_SSTEP) return fgmres_ss(h, b, B, x, info);
  return fgmres_df(h, b, B, x, info);
}

}  // namespace mgh
