// Pieces shared by the short-recurrence engines (Bi-CGSTAB of Alg. 3 and IDR(s)): complex division,
// the operator row at one point, and the true-residual check that accepts a right-hand side whose
// recursive residual met tol.
#pragma once

#include "mgh_krylov_common.cuh"

namespace mgh {

namespace {

__device__ __forceinline__ cd cdiv(cd a, cd b) {
  const double d = cabs2(b);
  return mk<double>((a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d);
}

// A x at point q of one field (FP64 operator diagonal, neighbours 0 outside the grid).
template <typename T>
__device__ __forceinline__ cd apply_at(const Cx<T>* __restrict__ x, const cd* __restrict__ DA, size_t q, int m, int n,
                                       const KArgs& a) {
  cd s = czero<double>();
  if (m > 0) s = s + ccast<double>(x[q - 1]);
  if (m < a.nx - 1) s = s + ccast<double>(x[q + 1]);
  if (n > 0) s = s + ccast<double>(x[q - a.nx]);
  if (n < a.ny - 1) s = s + ccast<double>(x[q + a.nx]);
  return DA[q] * ccast<double>(x[q]) - a.inv_h2 * s;
}

// The points of reduction block blk of one right-hand side, with their grid column m and row n
// (the body first carries m past the row end into n).
#define SR_POINT_LOOP                                                                       \
  const size_t p0 = (size_t)blk * a.chunk, p1 = (p0 + a.chunk < a.N) ? p0 + a.chunk : a.N;  \
  int n = (int)((unsigned)(p0 + threadIdx.x) / (unsigned)a.nx);                            \
  int m = (int)((unsigned)(p0 + threadIdx.x) - (unsigned)n * (unsigned)a.nx);              \
  for (size_t q = p0 + threadIdx.x; q < p1; q += kKThreads, m += kKThreads)

// ||b - A x||^2 of the right-hand sides awaiting the check (slot 0).
__global__ void __launch_bounds__(kKThreads)
k_sr_true_residual(KArgs a, const cd* __restrict__ b, const cd* __restrict__ x, const cd* __restrict__ DA,
                   cd* __restrict__ partial, const RhsState* __restrict__ st) {
  const int rhs = blockIdx.y, blk = blockIdx.x;
  if (!st[rhs].active || !st[rhs].verify) return;
  const cd* bb = b + rhs * a.N;
  const cd* xb = x + rhs * a.N;
  cd acc[1] = {czero<double>()};
  SR_POINT_LOOP {
    while (m >= a.nx) { m -= a.nx; ++n; }
    acc[0].re += cabs2(bb[q] - apply_at(xb, DA, q, m, n, a));
  }
  block_reduce_store<1>(acc, 1, 0.0, 1, partial + ((size_t)rhs * a.nblk + blk) * a.pstride);
}

// Accept on the true residual, else go on from the recursive one; maxit stops.
__global__ void k_sr_decide(KArgs a, const cd* __restrict__ partial, RhsState* __restrict__ st, double tol,
                            int maxit) {
  __shared__ cd sh[1];
  const int rhs = blockIdx.x;
  if (!st[rhs].active || !st[rhs].verify) return;
  sum_partials(a, partial, rhs, 1, sh);
  if (threadIdx.x != 0) return;
  RhsState& S = st[rhs];
  S.verify = 0;
  S.nres += 1;
  const double r64 = sqrt(sh[0].re);
  if (r64 <= tol * S.bnorm) { S.done = 1; S.converged = 1; S.active = 0; S.rnorm = r64; return; }
  if (S.iterations >= maxit) { S.done = 1; S.converged = 0; S.active = 0; S.rnorm = r64; }
}

}  // namespace

}  // namespace mgh
