// Batched right-preconditioned IDR(s) with biorthogonalisation (induced dimension reduction:
// Sonneveld & van Gijzen 2008; the biorthogonal form of van Gijzen & Sonneveld 2011), a
// short-recurrence alternative to the Bi-CGSTAB of Alg. 3 with the same multigrid cycle as
// preconditioner.  Residuals are driven into shrinking spaces orthogonal to an s-dimensional
// shadow space P.  One outer step makes s intermediate residuals with update directions U
// (preconditioned) and G = A U kept biorthogonal to P (M_s = P^H G lower triangular), then one
// dimension-reduction step r <- r - omega A M^{-1} r, omega the minimal-residual choice raised to
// keep |cos(t, r)| >= kappa = 0.7.  Every step costs one cycle and one operator product; the
// iteration count is the number of cycles.  With s = 1 and P = r_0 the method is Bi-CGSTAB.
//
// Per intermediate step k (0 <= k < s) and right-hand side:
//   c = M_s[k:, k:]^{-1} f[k:]  (forward substitution)      v = r - G[:, k:] c
//   U_k = U[:, k:] c + omega M^{-1} v                         G_k = A U_k,  d = P^H G_k
//   alpha = M_s[:k, :k]^{-1} d[:k],  M_s[i, k] = d_i - M_s[i, :k] alpha  (i >= k)
//   G_k -= G[:, :k] alpha,  U_k -= U[:, :k] alpha;  beta = f_k / M_s[k, k]
//   r -= beta G_k,  x += beta U_k,  f[k+1:] -= beta M_s[k+1:, k]
// The projections of G_k onto the earlier directions come from one pass of s inner products and
// a triangular solve, instead of k sequential product-and-update passes: the same vectors in
// exact arithmetic, since P_i^H G_j = 0 for j < i.
//
// The shadow space is generated, not stored: P_i[q] = (1 - 2 b_{2i}) + j (1 - 2 b_{2i+1}) with b
// the bits of MurmurHash3's 32-bit finaliser (fmix32, Appleby) of q + 0x9E3779B9 (mod 2^32):
// random signs, a generic space for every s <= 16, read by sign flips and additions only.
//
// All right-hand sides advance in lock step with their own scalars (device resident); one that
// converged, broke down or reached maxit drops out of every kernel through its state flag.  Vectors
// are complex FP64 and every inner product is an FP64 block reduction; the cycle runs in the
// handle's precision (FP32 on FP32 copies of its inputs on the mixed path).  The vectors live in
// the GMRES workspace: r, G_0..G_{s-1}, U_0..U_{s-1}, v, t in basis slots 0..2s+2 (so
// restart >= 2s + 2), the FP32 cycle input and the cycle output in preconditioned slots 0 and 1.
// The host reads the state once per outer step; the outer step's launches are replayed from a
// captured CUDA graph after the first one.
#include "mgh_short_rec.cuh"

namespace mgh {

namespace {

constexpr double kIdrKappa = 0.7;
constexpr int kIdrNV = kMaxIdrS + 2;   // accumulators of the widest block reduction

// Launch arguments of the IDR kernels: the shadow dimension, the vector slots and the per-RHS
// scalars (kept in the Hessenberg buffer, m (m+1) complex words per right-hand side):
// M_s row-major s x s at 0, f at s^2, c at s^2 + s, alpha at s^2 + 2s, then omega, beta, ||r||^2.
struct IArgs {
  int s;
  cd* V;                // basis slots; slot i of RHS b at V + b * vs + i * Np
  size_t vs;
  cd* sc;               // scalars; RHS b at sc + b * scs
  size_t scs;
  __device__ __forceinline__ cd* slot(int rhs, int i, size_t Np) const { return V + rhs * vs + (size_t)i * Np; }
  __device__ __forceinline__ cd* Ms(int rhs) const { return sc + rhs * scs; }
  __device__ __forceinline__ cd* f(int rhs) const { return sc + rhs * scs + s * s; }
  __device__ __forceinline__ cd* c(int rhs) const { return sc + rhs * scs + s * s + s; }
  __device__ __forceinline__ cd* alpha(int rhs) const { return sc + rhs * scs + s * s + 2 * s; }
  __device__ __forceinline__ cd* misc(int rhs) const { return sc + rhs * scs + s * s + 3 * s; }  // omega, beta, ||r||^2
};

enum { sR = 0 };                                  // basis slot of r; G_j at 1 + j, U_j at 1 + s + j
__host__ __device__ __forceinline__ int slot_g(int j) { return 1 + j; }
__host__ __device__ __forceinline__ int slot_u(int s, int j) { return 1 + s + j; }
__host__ __device__ __forceinline__ int slot_v(int s) { return 2 * s + 1; }
__host__ __device__ __forceinline__ int slot_t(int s) { return 2 * s + 2; }
enum { zIn32 = 0, zY = 1 };                       // preconditioned slots

// Sign bits of the shadow space at point q.
__device__ __forceinline__ uint32_t shadow_bits(size_t q) {
  uint32_t h = (uint32_t)q + 0x9E3779B9u;
  h ^= h >> 16;
  h *= 0x85EBCA6Bu;
  h ^= h >> 13;
  h *= 0xC2B2AE35u;
  h ^= h >> 16;
  return h;
}

// acc_i += conj(P_i[q]) x for i < s: with P_i = a + j b (a, b = +-1),
// conj(P_i) x = (a x.re + b x.im) + j (a x.im - b x.re).
__device__ __forceinline__ void shadow_dots(cd* acc, int s, uint32_t bits, cd x) {
#pragma unroll
  for (int i = 0; i < kMaxIdrS; ++i) {
    if (i < s) {
      const double xr_a = (bits >> (2 * i)) & 1u ? -x.re : x.re;
      const double xi_a = (bits >> (2 * i)) & 1u ? -x.im : x.im;
      const double xr_b = (bits >> (2 * i + 1)) & 1u ? -x.re : x.re;
      const double xi_b = (bits >> (2 * i + 1)) & 1u ? -x.im : x.im;
      acc[i].re += xr_a + xi_b;
      acc[i].im += xi_a - xr_b;
    }
  }
}

#define IDR_POINTS                                                                         \
  const size_t p0 = (size_t)blk * a.chunk, p1 = (p0 + a.chunk < a.N) ? p0 + a.chunk : a.N;

__device__ __forceinline__ cd* partial_of(const KArgs& a, cd* partial, int rhs, int blk) {
  return partial + ((size_t)rhs * a.nblk + blk) * a.pstride;
}

// r = b - A x, G_j = U_j = 0; partial ||b||^2 (slot 0), ||r||^2 (slot 1), P^H r (slots 2..s+1).
__global__ void __launch_bounds__(kKThreads)
k_idr_init(KArgs a, IArgs ia, const cd* __restrict__ b, const cd* __restrict__ x, const cd* __restrict__ DA,
           cd* __restrict__ partial) {
  const int rhs = blockIdx.y, blk = blockIdx.x, s = ia.s;
  const cd* bb = b + rhs * a.N;
  const cd* xb = x + rhs * a.N;
  cd* rr = ia.slot(rhs, sR, a.Np);
  cd acc[kIdrNV];
#pragma unroll
  for (int i = 0; i < kIdrNV; ++i) acc[i] = czero<double>();
  SR_POINT_LOOP {
    while (m >= a.nx) { m -= a.nx; ++n; }
    const cd bq = bb[q];
    const cd rq = bq - apply_at(xb, DA, q, m, n, a);
    rr[q] = rq;
    for (int j = 0; j < s; ++j) {
      ia.slot(rhs, slot_g(j), a.Np)[q] = czero<double>();
      ia.slot(rhs, slot_u(s, j), a.Np)[q] = czero<double>();
    }
    acc[0].re += cabs2(bq);
    acc[1].re += cabs2(rq);
    shadow_dots(acc + 2, s, shadow_bits(q), rq);
  }
  block_reduce_store<kIdrNV>(acc, 2 + s, 0.0, 2 + s, partial_of(a, partial, rhs, blk));
}

// Start: ||b||, ||r||, f = P^H r, M_s = I, omega = 1; b = 0 or an initial guess that already meets
// tol ends here.
__global__ void k_idr_start(KArgs a, IArgs ia, const cd* __restrict__ partial, RhsState* __restrict__ st,
                            double tol) {
  __shared__ cd sh[kIdrNV];
  const int rhs = blockIdx.x, s = ia.s;
  sum_partials(a, partial, rhs, 2 + s, sh);
  if (threadIdx.x != 0) return;
  RhsState& S = st[rhs];
  S.bnorm = sqrt(sh[0].re);
  S.rnorm = sqrt(sh[1].re);
  S.nres = 1;
  cd* M = ia.Ms(rhs);
  cd* f = ia.f(rhs);
  cd* misc = ia.misc(rhs);
  for (int i = 0; i < s; ++i) {
    for (int j = 0; j < s; ++j) M[i * s + j] = mk<double>(i == j ? 1.0 : 0.0, 0.0);
    f[i] = sh[2 + i];
  }
  misc[0] = mk<double>(1.0, 0.0);
  misc[1] = czero<double>();
  misc[2] = mk<double>(sh[1].re, 0.0);
  if (S.bnorm == 0.0 || S.rnorm <= tol * S.bnorm) { S.done = 1; S.converged = 1; S.active = 0; return; }
  S.active = 1;
}

// c[k..s-1] from M_s[k:, k:] c = f[k:] (lower triangular).
__global__ void k_idr_coef(IArgs ia, const RhsState* __restrict__ st, int B, int k) {
  const int rhs = blockIdx.x * blockDim.x + threadIdx.x;
  if (rhs >= B || !st[rhs].active) return;
  const int s = ia.s;
  const cd* M = ia.Ms(rhs);
  const cd* f = ia.f(rhs);
  cd* c = ia.c(rhs);
  for (int i = k; i < s; ++i) {
    cd t = f[i];
    for (int j = k; j < i; ++j) t = t - M[i * s + j] * c[j];
    c[i] = cdiv(t, M[i * s + i]);
  }
}

// v = r - sum_{j >= k} c_j G_j, written as FP64 (v64) or as the FP32 cycle input (v32).
__global__ void __launch_bounds__(kKThreads)
k_idr_v(KArgs a, IArgs ia, const RhsState* __restrict__ st, int k, cd* __restrict__ v64, size_t v64_stride,
        cf* __restrict__ v32, size_t v32_stride) {
  const int rhs = blockIdx.y, blk = blockIdx.x, s = ia.s;
  if (!st[rhs].active) return;
  cd cc[kMaxIdrS];
  const cd* cg[kMaxIdrS];
#pragma unroll
  for (int j = 0; j < kMaxIdrS; ++j) {
    const bool use = j >= k && j < s;
    cc[j] = use ? ia.c(rhs)[j] : czero<double>();
    cg[j] = use ? ia.slot(rhs, slot_g(j), a.Np) : nullptr;
  }
  const cd* rr = ia.slot(rhs, sR, a.Np);
  cd* vo = v64 ? v64 + rhs * v64_stride : nullptr;
  cf* vo32 = v32 ? v32 + rhs * v32_stride : nullptr;
  IDR_POINTS
  for (size_t q = p0 + threadIdx.x; q < p1; q += kKThreads) {
    cd v = rr[q];
#pragma unroll
    for (int j = 0; j < kMaxIdrS; ++j)
      if (j >= k && j < s) caxpy_neg(v, cc[j], cg[j][q]);
    if (vo) vo[q] = v;
    else vo32[q] = ccast<float>(v);
  }
}

// U_k = sum_{j >= k} c_j U_j + omega y (y = M^{-1} v, the cycle output; U_k is read before it is
// overwritten at the same point).
template <typename TZ>
__global__ void __launch_bounds__(kKThreads)
k_idr_u(KArgs a, IArgs ia, const RhsState* __restrict__ st, int k, const Cx<TZ>* __restrict__ y, size_t y_stride) {
  const int rhs = blockIdx.y, blk = blockIdx.x, s = ia.s;
  if (!st[rhs].active) return;
  cd cc[kMaxIdrS];
  cd* cu[kMaxIdrS];
#pragma unroll
  for (int j = 0; j < kMaxIdrS; ++j) {
    const bool use = j >= k && j < s;
    cc[j] = use ? ia.c(rhs)[j] : czero<double>();
    cu[j] = use ? ia.slot(rhs, slot_u(s, j), a.Np) : nullptr;
  }
  const cd om = ia.misc(rhs)[0];
  const Cx<TZ>* yb = y + rhs * y_stride;
  cd* uk = ia.slot(rhs, slot_u(s, k), a.Np);
  IDR_POINTS
  for (size_t q = p0 + threadIdx.x; q < p1; q += kKThreads) {
    cd u = om * ccast<double>(yb[q]);
#pragma unroll
    for (int j = 0; j < kMaxIdrS; ++j)
      if (j >= k && j < s) u = u + cc[j] * cu[j][q];
    uk[q] = u;
  }
}

// G_k = A U_k; partial d = P^H G_k (slots 0..s-1).
__global__ void __launch_bounds__(kKThreads)
k_idr_g(KArgs a, IArgs ia, const cd* __restrict__ DA, cd* __restrict__ partial, const RhsState* __restrict__ st,
        int k) {
  const int rhs = blockIdx.y, blk = blockIdx.x, s = ia.s;
  if (!st[rhs].active) return;
  const cd* uk = ia.slot(rhs, slot_u(s, k), a.Np);
  cd* gk = ia.slot(rhs, slot_g(k), a.Np);
  cd acc[kIdrNV];
#pragma unroll
  for (int i = 0; i < kIdrNV; ++i) acc[i] = czero<double>();
  SR_POINT_LOOP {
    while (m >= a.nx) { m -= a.nx; ++n; }
    const cd g = apply_at(uk, DA, q, m, n, a);
    gk[q] = g;
    shadow_dots(acc, s, shadow_bits(q), g);
  }
  block_reduce_store<kIdrNV>(acc, s, 0.0, s, partial_of(a, partial, rhs, blk));
}

// From d = P^H G_k: alpha (the projection of G_k off G_0..G_{k-1}), column k of M_s, beta and the
// update of f.  A zero M_s[k, k] is a breakdown (the RHS stops, not converged).
__global__ void k_idr_col(KArgs a, IArgs ia, const cd* __restrict__ partial, RhsState* __restrict__ st, int k) {
  __shared__ cd sh[kIdrNV];
  const int rhs = blockIdx.x, s = ia.s;
  if (!st[rhs].active) return;
  sum_partials(a, partial, rhs, s, sh);
  if (threadIdx.x != 0) return;
  cd* M = ia.Ms(rhs);
  cd* f = ia.f(rhs);
  cd* al = ia.alpha(rhs);
  for (int i = 0; i < k; ++i) {
    cd t = sh[i];
    for (int j = 0; j < i; ++j) t = t - M[i * s + j] * al[j];
    al[i] = cdiv(t, M[i * s + i]);
  }
  for (int i = k; i < s; ++i) {
    cd t = sh[i];
    for (int j = 0; j < k; ++j) t = t - M[i * s + j] * al[j];
    M[i * s + k] = t;
  }
  const cd mkk = M[k * s + k];
  if (!(cabs2(mkk) > 0.0)) { st[rhs].done = 1; st[rhs].converged = 0; st[rhs].active = 0; return; }
  const cd beta = cdiv(f[k], mkk);
  ia.misc(rhs)[1] = beta;
  for (int i = k + 1; i < s; ++i) f[i] = f[i] - beta * M[i * s + k];
}

// G_k -= sum_{i<k} alpha_i G_i, U_k -= sum_{i<k} alpha_i U_i, r -= beta G_k, x += beta U_k;
// partial ||r||^2 (slot 0); r32 = FP32 copy of r (the next cycle's input) when given.
__global__ void __launch_bounds__(kKThreads)
k_idr_r(KArgs a, IArgs ia, cd* __restrict__ x, cd* __restrict__ partial, const RhsState* __restrict__ st, int k,
        cf* __restrict__ r32, size_t r32_stride) {
  const int rhs = blockIdx.y, blk = blockIdx.x, s = ia.s;
  if (!st[rhs].active) return;
  cd al[kMaxIdrS];
  const cd* pg[kMaxIdrS];
  const cd* pu[kMaxIdrS];
#pragma unroll
  for (int j = 0; j < kMaxIdrS; ++j) {
    const bool use = j < k;
    al[j] = use ? ia.alpha(rhs)[j] : czero<double>();
    pg[j] = use ? ia.slot(rhs, slot_g(j), a.Np) : nullptr;
    pu[j] = use ? ia.slot(rhs, slot_u(s, j), a.Np) : nullptr;
  }
  const cd beta = ia.misc(rhs)[1];
  cd* gk = ia.slot(rhs, slot_g(k), a.Np);
  cd* uk = ia.slot(rhs, slot_u(s, k), a.Np);
  cd* rr = ia.slot(rhs, sR, a.Np);
  cd* xb = x + rhs * a.N;
  cf* r3 = r32 ? r32 + rhs * r32_stride : nullptr;
  cd acc[1] = {czero<double>()};
  IDR_POINTS
  for (size_t q = p0 + threadIdx.x; q < p1; q += kKThreads) {
    cd g = gk[q], u = uk[q];
#pragma unroll
    for (int j = 0; j < kMaxIdrS; ++j)
      if (j < k) {
        caxpy_neg(g, al[j], pg[j][q]);
        caxpy_neg(u, al[j], pu[j][q]);
      }
    gk[q] = g;
    uk[q] = u;
    cd r = rr[q];
    caxpy_neg(r, beta, g);
    rr[q] = r;
    xb[q] = xb[q] + beta * u;
    if (r3) r3[q] = ccast<float>(r);
    acc[0].re += cabs2(r);
  }
  block_reduce_store<1>(acc, 1, 0.0, 1, partial_of(a, partial, rhs, blk));
}

// End of an intermediate step: one cycle counted, ||r||^2 kept for the next dimension reduction; a
// recursive residual that meets tol asks for the true one; maxit stops.
__global__ void k_idr_step_end(KArgs a, IArgs ia, const cd* __restrict__ partial, RhsState* __restrict__ st,
                               double tol, int maxit) {
  __shared__ cd sh[1];
  const int rhs = blockIdx.x;
  if (!st[rhs].active) return;
  sum_partials(a, partial, rhs, 1, sh);
  if (threadIdx.x != 0) return;
  RhsState& S = st[rhs];
  ia.misc(rhs)[2] = mk<double>(sh[0].re, 0.0);
  S.iterations += 1;
  S.rnorm = sqrt(sh[0].re);
  S.verify = (S.rnorm <= tol * S.bnorm) ? 1 : 0;
  if (!S.verify && (S.iterations >= maxit || !(S.rnorm == S.rnorm))) { S.done = 1; S.converged = 0; S.active = 0; }
}

// t = A y (y = M^{-1} r, the cycle output); partial r^H t (slot 0) and ||t||^2 (slot 1).
template <typename TZ>
__global__ void __launch_bounds__(kKThreads)
k_idr_t(KArgs a, IArgs ia, const Cx<TZ>* __restrict__ y, size_t y_stride, const cd* __restrict__ DA,
        cd* __restrict__ partial, const RhsState* __restrict__ st) {
  const int rhs = blockIdx.y, blk = blockIdx.x, s = ia.s;
  if (!st[rhs].active) return;
  const Cx<TZ>* yb = y + rhs * y_stride;
  const cd* rr = ia.slot(rhs, sR, a.Np);
  cd* tt = ia.slot(rhs, slot_t(s), a.Np);
  cd acc[2] = {czero<double>(), czero<double>()};
  SR_POINT_LOOP {
    while (m >= a.nx) { m -= a.nx; ++n; }
    const cd t = apply_at(yb, DA, q, m, n, a);
    tt[q] = t;
    cdot_acc(acc[0], rr[q], t);
    acc[1].re += cabs2(t);
  }
  block_reduce_store<2>(acc, 2, 0.0, 2, partial_of(a, partial, rhs, blk));
}

// omega = (t^H r) / (t^H t), raised to omega kappa / rho when rho = |t^H r| / (||t|| ||r||) < kappa
// (a t orthogonal to r takes |omega| = kappa ||r|| / ||t||); t = 0 is a breakdown.
__global__ void k_idr_omega(KArgs a, IArgs ia, const cd* __restrict__ partial, RhsState* __restrict__ st) {
  __shared__ cd sh[2];
  const int rhs = blockIdx.x;
  if (!st[rhs].active) return;
  sum_partials(a, partial, rhs, 2, sh);
  if (threadIdx.x != 0) return;
  const cd tr = cconj(sh[0]);
  const double t2 = sh[1].re, rn = sqrt(ia.misc(rhs)[2].re), tn = sqrt(t2);
  if (!(t2 > 0.0)) { st[rhs].done = 1; st[rhs].converged = 0; st[rhs].active = 0; return; }
  cd om = (1.0 / t2) * tr;
  const double rho = rn > 0.0 ? sqrt(cabs2(tr)) / (tn * rn) : 1.0;
  if (rho == 0.0) om = mk<double>(kIdrKappa * rn / tn, 0.0);
  else if (rho < kIdrKappa) om = (kIdrKappa / rho) * om;
  ia.misc(rhs)[0] = om;
}

// x += omega y, r -= omega t; partial ||r||^2 (slot 0) and P^H r (slots 1..s).
template <typename TZ>
__global__ void __launch_bounds__(kKThreads)
k_idr_dr(KArgs a, IArgs ia, const Cx<TZ>* __restrict__ y, size_t y_stride, cd* __restrict__ x,
         cd* __restrict__ partial, const RhsState* __restrict__ st) {
  const int rhs = blockIdx.y, blk = blockIdx.x, s = ia.s;
  if (!st[rhs].active) return;
  const cd om = ia.misc(rhs)[0];
  const Cx<TZ>* yb = y + rhs * y_stride;
  cd* rr = ia.slot(rhs, sR, a.Np);
  const cd* tt = ia.slot(rhs, slot_t(s), a.Np);
  cd* xb = x + rhs * a.N;
  cd acc[kIdrNV];
#pragma unroll
  for (int i = 0; i < kIdrNV; ++i) acc[i] = czero<double>();
  IDR_POINTS
  for (size_t q = p0 + threadIdx.x; q < p1; q += kKThreads) {
    xb[q] = xb[q] + om * ccast<double>(yb[q]);
    cd r = rr[q];
    caxpy_neg(r, om, tt[q]);
    rr[q] = r;
    acc[0].re += cabs2(r);
    shadow_dots(acc + 1, s, shadow_bits(q), r);
  }
  block_reduce_store<kIdrNV>(acc, 1 + s, 0.0, 1 + s, partial_of(a, partial, rhs, blk));
}

// End of a dimension reduction: one cycle and one outer step counted, f = P^H r for the next outer
// step; the residual test as at the end of an intermediate step.
__global__ void k_idr_dr_end(KArgs a, IArgs ia, const cd* __restrict__ partial, RhsState* __restrict__ st,
                             double tol, int maxit) {
  __shared__ cd sh[kIdrNV];
  const int rhs = blockIdx.x, s = ia.s;
  if (!st[rhs].active) return;
  sum_partials(a, partial, rhs, 1 + s, sh);
  if (threadIdx.x != 0) return;
  RhsState& S = st[rhs];
  cd* f = ia.f(rhs);
  for (int i = 0; i < s; ++i) f[i] = sh[1 + i];
  ia.misc(rhs)[2] = mk<double>(sh[0].re, 0.0);
  S.iterations += 1;
  S.restarts += 1;
  S.rnorm = sqrt(sh[0].re);
  S.verify = (S.rnorm <= tol * S.bnorm) ? 1 : 0;
  if (!S.verify && (S.iterations >= maxit || !(S.rnorm == S.rnorm))) { S.done = 1; S.converged = 0; S.active = 0; }
}

template <typename TZ>
mgh_status idrs_t(Handle& h, const cd* b, int B, cd* x, mgh_solve_info* info) {
  KArgs a = make_kargs(h, B);
  const dim3 grid(a.nblk, B);
  const int s = h.p.idr_s;
  IArgs ia;
  ia.s = s;
  ia.V = reinterpret_cast<cd*>(h.V);
  ia.vs = (size_t)(a.m + 1) * a.Np;
  ia.sc = h.H;
  ia.scs = (size_t)a.m * (a.m + 1);
  const size_t zs = (size_t)a.m * a.N;   // preconditioned-slot stride between right-hand sides
  Cx<TZ>* y = reinterpret_cast<Cx<TZ>*>(h.Z) + (size_t)zY * a.N;
  cf* in32 = h.fp64 ? nullptr : reinterpret_cast<cf*>(h.Z) + (size_t)zIn32 * a.N;
  cd* v64 = h.fp64 ? ia.V + (size_t)slot_v(s) * a.Np : nullptr;
  cd* r64 = ia.V + (size_t)sR * a.Np;
  const double tol = h.p.tol;
  const int maxit = h.p.maxit;
  const int sblocks = (B + 31) / 32;
  {
    ProfScope ps(h, P_REDUCE);
    k_state_reset<<<(B + 63) / 64, 64, 0, h.stream>>>(h.st, B);
    MGH_CHECK_LAUNCH(); h.launches++;
  }
  {
    ProfScope ps(h, P_RESIDUAL);
    k_idr_init<<<grid, kKThreads, 0, h.stream>>>(a, ia, b, x, h.DA, h.partial);
    MGH_CHECK_LAUNCH(); h.launches++;
  }
  {
    ProfScope ps(h, P_REDUCE);
    k_idr_start<<<B, 32, 0, h.stream>>>(a, ia, h.partial, h.st, tol);
    MGH_CHECK_LAUNCH(); h.launches++;
    k_zero_if_b_zero<<<grid, kKThreads, 0, h.stream>>>(a, x, h.st);
    MGH_CHECK_LAUNCH(); h.launches++;
  }
  auto check = [&]() -> mgh_status {
    {
      ProfScope ps(h, P_RESIDUAL);
      k_sr_true_residual<<<grid, kKThreads, 0, h.stream>>>(a, b, x, h.DA, h.partial, h.st);
      MGH_CHECK_LAUNCH(); h.launches++;
    }
    {
      ProfScope ps(h, P_REDUCE);
      k_sr_decide<<<B, 32, 0, h.stream>>>(a, h.partial, h.st, tol, maxit);
      MGH_CHECK_LAUNCH(); h.launches++;
    }
    return MGH_OK;
  };
  auto precondition = [&](const cd* in64, size_t in64_stride) -> mgh_status {
    if (h.fp64) return vcycle(h, in64, in64_stride, nullptr, 0, y, zs, true, B, h.st);
    return vcycle_f32in(h, in32, zs, nullptr, 0, reinterpret_cast<cf*>(y), zs, B, h.st, -1);
  };
  // one outer step: s intermediate steps, then one dimension reduction
  auto body = [&]() -> mgh_status {
    for (int k = 0; k < s; ++k) {
      {
        ProfScope ps(h, P_REDUCE);
        k_idr_coef<<<sblocks, 32, 0, h.stream>>>(ia, h.st, B, k);
        MGH_CHECK_LAUNCH(); h.launches++;
      }
      {
        ProfScope ps(h, P_UPDATE);
        k_idr_v<<<grid, kKThreads, 0, h.stream>>>(a, ia, h.st, k, v64, ia.vs, in32, zs);
        MGH_CHECK_LAUNCH(); h.launches++;
      }
      MGH_TRY(precondition(v64, ia.vs));
      {
        ProfScope ps(h, P_UPDATE);
        k_idr_u<TZ><<<grid, kKThreads, 0, h.stream>>>(a, ia, h.st, k, y, zs);
        MGH_CHECK_LAUNCH(); h.launches++;
      }
      {
        ProfScope ps(h, P_MATVEC_DOTS);
        k_idr_g<<<grid, kKThreads, 0, h.stream>>>(a, ia, h.DA, h.partial, h.st, k);
        MGH_CHECK_LAUNCH(); h.launches++;
      }
      {
        ProfScope ps(h, P_REDUCE);
        k_idr_col<<<B, 32, 0, h.stream>>>(a, ia, h.partial, h.st, k);
        MGH_CHECK_LAUNCH(); h.launches++;
      }
      {
        ProfScope ps(h, P_UPDATE);
        k_idr_r<<<grid, kKThreads, 0, h.stream>>>(a, ia, x, h.partial, h.st, k, k == s - 1 ? in32 : nullptr, zs);
        MGH_CHECK_LAUNCH(); h.launches++;
      }
      {
        ProfScope ps(h, P_REDUCE);
        k_idr_step_end<<<B, 32, 0, h.stream>>>(a, ia, h.partial, h.st, tol, maxit);
        MGH_CHECK_LAUNCH(); h.launches++;
      }
      MGH_TRY(check());
    }
    MGH_TRY(precondition(r64, ia.vs));
    {
      ProfScope ps(h, P_MATVEC_DOTS);
      k_idr_t<TZ><<<grid, kKThreads, 0, h.stream>>>(a, ia, y, zs, h.DA, h.partial, h.st);
      MGH_CHECK_LAUNCH(); h.launches++;
    }
    {
      ProfScope ps(h, P_REDUCE);
      k_idr_omega<<<B, 32, 0, h.stream>>>(a, ia, h.partial, h.st);
      MGH_CHECK_LAUNCH(); h.launches++;
    }
    {
      ProfScope ps(h, P_UPDATE);
      k_idr_dr<TZ><<<grid, kKThreads, 0, h.stream>>>(a, ia, y, zs, x, h.partial, h.st);
      MGH_CHECK_LAUNCH(); h.launches++;
    }
    {
      ProfScope ps(h, P_REDUCE);
      k_idr_dr_end<<<B, 32, 0, h.stream>>>(a, ia, h.partial, h.st, tol, maxit);
      MGH_CHECK_LAUNCH(); h.launches++;
    }
    return check();
  };
  // the outer step is replayed from a captured graph after the first one
  CycleGraph graph;
  for (int it = 0;; ++it) {
    MGH_CUDA(cudaMemcpyAsync(h.st_host, h.st, sizeof(RhsState) * B, cudaMemcpyDeviceToHost, h.stream));
    MGH_CUDA(cudaStreamSynchronize(h.stream));
    MGH_TRY(prof_flush(h));
    bool any = false;
    for (int i = 0; i < B; ++i) any |= (h.st_host[i].active != 0);
    if (!any) break;
    if (!h.use_graphs || h.prof || it == 0) MGH_TRY(body());
    else MGH_TRY(graph.run(h, body));
  }
  return finish_solve(h, B, info);
}

}  // namespace

mgh_status idrs_solve(Handle& h, const cd* b, int B, cd* x, mgh_solve_info* info) {
  if (h.fp64) return idrs_t<double>(h, b, B, x, info);
  return idrs_t<float>(h, b, B, x, info);
}

}  // namespace mgh
