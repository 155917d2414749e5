// Batched right-preconditioned Bi-CGSTAB of Alg. 3 (van der Vorst 1992), the paper's own Krylov
// method, with the multigrid cycle as preconditioner at both of its preconditioning steps:
//
//   r = b - A x,  r^ = r,  rho_prev = alpha = omega = 1,  v = p = 0
//   repeat:  rho = r^H r;  beta = (rho / rho_prev)(alpha / omega)
//            p = r + beta (p - omega v);  y = M^{-1} p;  v = A y;  alpha = rho / (r^H v)
//            s = r - alpha v;  x += alpha y;  z = M^{-1} s;  t = A z;  omega = (t^H s) / (t^H t)
//            x += omega z;  r = s - omega t
//   stop when ||r|| <= tol ||b|| and the true residual ||b - A x|| confirms it.
//
// All right-hand sides advance in lock step, each with its own scalars (device resident); one
// that converged or broke down drops out of every kernel through its state flag.  Vectors are
// complex FP64 and every inner product is an FP64 block reduction.  On the mixed path the cycle
// runs in FP32 on FP32 copies of p and s written by the update kernels; on the FP64 path it runs
// in FP64 on p and s directly.  The vectors live in the GMRES workspace: r, r^, p, v, s, t in the
// first six basis slots (so restart >= 5) and p32, y, s32, z in the first four preconditioned
// slots.  The host reads the state once per iteration; the iteration's launches are replayed from
// a captured CUDA graph after the first one.
#include "mgh_short_rec.cuh"

namespace mgh {

namespace {

enum { kR = 0, kRhat = 1, kP = 2, kV = 3, kS = 4, kT = 5 };   // FP64 vector slots
enum { kP32 = 0, kY = 1, kS32 = 2, kZ = 3 };                    // preconditioner slots
enum { cRho = 0, cRhoPrev = 1, cAlpha = 2, cOmega = 3 };        // per-RHS scalars (coef)

struct Vec {
  cd* base;
  size_t stride;
  __device__ __forceinline__ cd* at(int rhs) const { return base + rhs * stride; }
};

// r = b - A x, r^ = r, p = v = 0; partial ||b||^2 (slot 0) and ||r||^2 (slot 1).
__global__ void __launch_bounds__(kKThreads)
k_bc_init(KArgs a, const cd* __restrict__ b, const cd* __restrict__ x, const cd* __restrict__ DA, Vec r, Vec rh,
          Vec p, Vec v, cd* __restrict__ partial) {
  const int rhs = blockIdx.y, blk = blockIdx.x;
  const cd* bb = b + rhs * a.N;
  const cd* xb = x + rhs * a.N;
  cd* rr = r.at(rhs);
  cd* rhh = rh.at(rhs);
  cd* pp = p.at(rhs);
  cd* vv = v.at(rhs);
  cd acc[2] = {czero<double>(), czero<double>()};
  SR_POINT_LOOP {
    while (m >= a.nx) { m -= a.nx; ++n; }
    const cd bq = bb[q];
    const cd rq = bq - apply_at(xb, DA, q, m, n, a);
    rr[q] = rq;
    rhh[q] = rq;
    pp[q] = czero<double>();
    vv[q] = czero<double>();
    acc[0].re += cabs2(bq);
    acc[1].re += cabs2(rq);
  }
  block_reduce_store<2>(acc, 2, 0.0, 2, partial + ((size_t)rhs * a.nblk + blk) * a.pstride);
}

// Start: ||b||, the first rho = ||r||^2; b = 0 or an initial guess that already meets tol ends here.
__global__ void k_bc_start(KArgs a, const cd* __restrict__ partial, cd* __restrict__ coef, RhsState* __restrict__ st,
                           double tol) {
  __shared__ cd sh[2];
  const int rhs = blockIdx.x;
  sum_partials(a, partial, rhs, 2, sh);
  if (threadIdx.x != 0) return;
  RhsState& S = st[rhs];
  S.bnorm = sqrt(sh[0].re);
  S.rnorm = sqrt(sh[1].re);
  S.nres = 1;
  cd* c = coef + (size_t)rhs * 2 * a.m;
  c[cRho] = mk<double>(sh[1].re, 0.0);
  c[cRhoPrev] = mk<double>(1.0, 0.0);
  c[cAlpha] = mk<double>(1.0, 0.0);
  c[cOmega] = mk<double>(1.0, 0.0);
  if (S.bnorm == 0.0 || S.rnorm <= tol * S.bnorm) { S.done = 1; S.converged = 1; S.active = 0; return; }
  S.active = 1;
}

// p = r + beta (p - omega v) with beta = (rho / rho_prev)(alpha / omega); p32 = FP32 copy (mixed).
__global__ void __launch_bounds__(kKThreads)
k_bc_p(KArgs a, Vec r, Vec p, Vec v, cf* __restrict__ p32, size_t p32_stride, const cd* __restrict__ coef,
       const RhsState* __restrict__ st) {
  const int rhs = blockIdx.y, blk = blockIdx.x;
  if (!st[rhs].active) return;
  const cd* c = coef + (size_t)rhs * 2 * a.m;
  const cd beta = cdiv(c[cRho], c[cRhoPrev]) * cdiv(c[cAlpha], c[cOmega]);
  const cd om = c[cOmega];
  const cd* rr = r.at(rhs);
  cd* pp = p.at(rhs);
  const cd* vv = v.at(rhs);
  cf* p3 = p32 ? p32 + rhs * p32_stride : nullptr;
  const size_t p0 = (size_t)blk * a.chunk, p1 = (p0 + a.chunk < a.N) ? p0 + a.chunk : a.N;
  for (size_t q = p0 + threadIdx.x; q < p1; q += kKThreads) {
    const cd pq = rr[q] + beta * (pp[q] - om * vv[q]);
    pp[q] = pq;
    if (p3) p3[q] = ccast<float>(pq);
  }
}

// out = A y (y the cycle output, FP32 or FP64); partial w^H out (slot 0) and ||out||^2 (slot 1).
template <typename TZ>
__global__ void __launch_bounds__(kKThreads)
k_bc_apply_dots(KArgs a, const Cx<TZ>* __restrict__ y, size_t y_stride, const cd* __restrict__ DA, Vec out, Vec w,
                cd* __restrict__ partial, const RhsState* __restrict__ st) {
  const int rhs = blockIdx.y, blk = blockIdx.x;
  if (!st[rhs].active) return;
  const Cx<TZ>* yb = y + rhs * y_stride;
  cd* ob = out.at(rhs);
  const cd* wb = w.at(rhs);
  cd acc[2] = {czero<double>(), czero<double>()};
  SR_POINT_LOOP {
    while (m >= a.nx) { m -= a.nx; ++n; }
    const cd oq = apply_at(yb, DA, q, m, n, a);
    ob[q] = oq;
    cdot_acc(acc[0], wb[q], oq);
    acc[1].re += cabs2(oq);
  }
  block_reduce_store<2>(acc, 2, 0.0, 2, partial + ((size_t)rhs * a.nblk + blk) * a.pstride);
}

// alpha = rho / (r^H v); a zero denominator is a breakdown (the RHS stops, not converged).
__global__ void k_bc_alpha(KArgs a, const cd* __restrict__ partial, cd* __restrict__ coef, RhsState* __restrict__ st) {
  __shared__ cd sh[1];
  const int rhs = blockIdx.x;
  if (!st[rhs].active) return;
  sum_partials(a, partial, rhs, 1, sh);
  if (threadIdx.x != 0) return;
  cd* c = coef + (size_t)rhs * 2 * a.m;
  if (!(cabs2(sh[0]) > 0.0)) { st[rhs].done = 1; st[rhs].converged = 0; st[rhs].active = 0; return; }
  c[cAlpha] = cdiv(c[cRho], sh[0]);
}

// s = r - alpha v, x += alpha y; s32 = FP32 copy of s (mixed).
template <typename TZ>
__global__ void __launch_bounds__(kKThreads)
k_bc_s(KArgs a, Vec r, Vec v, Vec s, const Cx<TZ>* __restrict__ y, size_t y_stride, cd* __restrict__ x,
       cf* __restrict__ s32, size_t s32_stride, const cd* __restrict__ coef, const RhsState* __restrict__ st) {
  const int rhs = blockIdx.y, blk = blockIdx.x;
  if (!st[rhs].active) return;
  const cd al = coef[(size_t)rhs * 2 * a.m + cAlpha];
  const cd* rr = r.at(rhs);
  const cd* vv = v.at(rhs);
  cd* ss = s.at(rhs);
  const Cx<TZ>* yb = y + rhs * y_stride;
  cd* xb = x + rhs * a.N;
  cf* s3 = s32 ? s32 + rhs * s32_stride : nullptr;
  const size_t p0 = (size_t)blk * a.chunk, p1 = (p0 + a.chunk < a.N) ? p0 + a.chunk : a.N;
  for (size_t q = p0 + threadIdx.x; q < p1; q += kKThreads) {
    const cd sq = rr[q] - al * vv[q];
    ss[q] = sq;
    xb[q] = xb[q] + al * ccast<double>(yb[q]);
    if (s3) s3[q] = ccast<float>(sq);
  }
}

// omega = (t^H s) / (t^H t); the fused pass summed s^H t = conj(t^H s); t = 0 (then s = 0) gives
// omega = 0.
__global__ void k_bc_omega(KArgs a, const cd* __restrict__ partial, cd* __restrict__ coef,
                           const RhsState* __restrict__ st) {
  __shared__ cd sh[2];
  const int rhs = blockIdx.x;
  if (!st[rhs].active) return;
  sum_partials(a, partial, rhs, 2, sh);
  if (threadIdx.x != 0) return;
  cd* c = coef + (size_t)rhs * 2 * a.m;
  c[cOmega] = sh[1].re > 0.0 ? (1.0 / sh[1].re) * cconj(sh[0]) : czero<double>();
}

// x += omega z, r = s - omega t; partial r^^H r (slot 0) and ||r||^2 (slot 1).
template <typename TZ>
__global__ void __launch_bounds__(kKThreads)
k_bc_r(KArgs a, Vec s, Vec t, Vec r, Vec rh, const Cx<TZ>* __restrict__ z, size_t z_stride, cd* __restrict__ x,
       const cd* __restrict__ coef, cd* __restrict__ partial, const RhsState* __restrict__ st) {
  const int rhs = blockIdx.y, blk = blockIdx.x;
  if (!st[rhs].active) return;
  const cd om = coef[(size_t)rhs * 2 * a.m + cOmega];
  const cd* ss = s.at(rhs);
  const cd* tt = t.at(rhs);
  cd* rr = r.at(rhs);
  const cd* rhh = rh.at(rhs);
  const Cx<TZ>* zb = z + rhs * z_stride;
  cd* xb = x + rhs * a.N;
  cd acc[2] = {czero<double>(), czero<double>()};
  const size_t p0 = (size_t)blk * a.chunk, p1 = (p0 + a.chunk < a.N) ? p0 + a.chunk : a.N;
  for (size_t q = p0 + threadIdx.x; q < p1; q += kKThreads) {
    xb[q] = xb[q] + om * ccast<double>(zb[q]);
    const cd rq = ss[q] - om * tt[q];
    rr[q] = rq;
    cdot_acc(acc[0], rhh[q], rq);
    acc[1].re += cabs2(rq);
  }
  block_reduce_store<2>(acc, 2, 0.0, 2, partial + ((size_t)rhs * a.nblk + blk) * a.pstride);
}

// End of an iteration: rho_prev = rho, rho = r^^H r; two steps counted; a recursive residual that
// meets tol asks for the true one; maxit stops.
__global__ void k_bc_end(KArgs a, const cd* __restrict__ partial, cd* __restrict__ coef, RhsState* __restrict__ st,
                         double tol, int maxit) {
  __shared__ cd sh[2];
  const int rhs = blockIdx.x;
  if (!st[rhs].active) return;
  sum_partials(a, partial, rhs, 2, sh);
  if (threadIdx.x != 0) return;
  RhsState& S = st[rhs];
  cd* c = coef + (size_t)rhs * 2 * a.m;
  c[cRhoPrev] = c[cRho];
  c[cRho] = sh[0];
  S.iterations += 2;
  S.rnorm = sqrt(sh[1].re);
  S.verify = (S.rnorm <= tol * S.bnorm) ? 1 : 0;
  if (!S.verify && (S.iterations >= maxit || !(S.rnorm == S.rnorm))) { S.done = 1; S.converged = 0; S.active = 0; }
}

template <typename TZ>
mgh_status bicgstab_t(Handle& h, const cd* b, int B, cd* x, mgh_solve_info* info) {
  KArgs a = make_kargs(h, B);
  const dim3 grid(a.nblk, B);
  const size_t vs = (size_t)(a.m + 1) * a.Np;   // FP64 slot stride between right-hand sides
  cd* V = reinterpret_cast<cd*>(h.V);
  auto vec = [&](int i) { return Vec{V + (size_t)i * a.Np, vs}; };
  const Vec r = vec(kR), rh = vec(kRhat), p = vec(kP), v = vec(kV), s = vec(kS), t = vec(kT);
  Cx<TZ>* Z = reinterpret_cast<Cx<TZ>*>(h.Z);
  const size_t zs = (size_t)a.m * a.N;
  Cx<TZ>* y = Z + (size_t)kY * a.N;
  Cx<TZ>* z = Z + (size_t)kZ * a.N;
  cf* p32 = h.fp64 ? nullptr : reinterpret_cast<cf*>(h.Z) + (size_t)kP32 * a.N;
  cf* s32 = h.fp64 ? nullptr : reinterpret_cast<cf*>(h.Z) + (size_t)kS32 * a.N;
  const double tol = h.p.tol;
  const int maxit = h.p.maxit;
  {
    ProfScope ps(h, P_REDUCE);
    k_state_reset<<<(B + 63) / 64, 64, 0, h.stream>>>(h.st, B);
    MGH_CHECK_LAUNCH(); h.launches++;
  }
  {
    ProfScope ps(h, P_RESIDUAL);
    k_bc_init<<<grid, kKThreads, 0, h.stream>>>(a, b, x, h.DA, r, rh, p, v, h.partial);
    MGH_CHECK_LAUNCH(); h.launches++;
  }
  {
    ProfScope ps(h, P_REDUCE);
    k_bc_start<<<B, 32, 0, h.stream>>>(a, h.partial, h.coef, h.st, tol);
    MGH_CHECK_LAUNCH(); h.launches++;
    k_zero_if_b_zero<<<grid, kKThreads, 0, h.stream>>>(a, x, h.st);
    MGH_CHECK_LAUNCH(); h.launches++;
  }
  auto body = [&]() -> mgh_status {
    {
      ProfScope ps(h, P_UPDATE);
      k_bc_p<<<grid, kKThreads, 0, h.stream>>>(a, r, p, v, p32, zs, h.coef, h.st);
      MGH_CHECK_LAUNCH(); h.launches++;
    }
    if (h.fp64)
      MGH_TRY(vcycle(h, p.base, p.stride, nullptr, 0, y, zs, true, B, h.st));
    else
      MGH_TRY(vcycle_f32in(h, p32, zs, nullptr, 0, reinterpret_cast<cf*>(y), zs, B, h.st, -1));
    {
      ProfScope ps(h, P_MATVEC_DOTS);
      k_bc_apply_dots<TZ><<<grid, kKThreads, 0, h.stream>>>(a, y, zs, h.DA, v, rh, h.partial, h.st);
      MGH_CHECK_LAUNCH(); h.launches++;
    }
    {
      ProfScope ps(h, P_REDUCE);
      k_bc_alpha<<<B, 32, 0, h.stream>>>(a, h.partial, h.coef, h.st);
      MGH_CHECK_LAUNCH(); h.launches++;
    }
    {
      ProfScope ps(h, P_UPDATE);
      k_bc_s<TZ><<<grid, kKThreads, 0, h.stream>>>(a, r, v, s, y, zs, x, s32, zs, h.coef, h.st);
      MGH_CHECK_LAUNCH(); h.launches++;
    }
    if (h.fp64)
      MGH_TRY(vcycle(h, s.base, s.stride, nullptr, 0, z, zs, true, B, h.st));
    else
      MGH_TRY(vcycle_f32in(h, s32, zs, nullptr, 0, reinterpret_cast<cf*>(z), zs, B, h.st, -1));
    {
      ProfScope ps(h, P_MATVEC_DOTS);
      k_bc_apply_dots<TZ><<<grid, kKThreads, 0, h.stream>>>(a, z, zs, h.DA, t, s, h.partial, h.st);
      MGH_CHECK_LAUNCH(); h.launches++;
    }
    {
      ProfScope ps(h, P_REDUCE);
      k_bc_omega<<<B, 32, 0, h.stream>>>(a, h.partial, h.coef, h.st);
      MGH_CHECK_LAUNCH(); h.launches++;
    }
    {
      ProfScope ps(h, P_UPDATE);
      k_bc_r<TZ><<<grid, kKThreads, 0, h.stream>>>(a, s, t, r, rh, z, zs, x, h.coef, h.partial, h.st);
      MGH_CHECK_LAUNCH(); h.launches++;
    }
    {
      ProfScope ps(h, P_REDUCE);
      k_bc_end<<<B, 32, 0, h.stream>>>(a, h.partial, h.coef, h.st, tol, maxit);
      MGH_CHECK_LAUNCH(); h.launches++;
    }
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
  // the iteration is replayed from a captured graph after the first one
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

mgh_status bicgstab_solve(Handle& h, const cd* b, int B, cd* x, mgh_solve_info* info) {
  if (h.fp64) return bicgstab_t<double>(h, b, B, x, info);
  return bicgstab_t<float>(h, b, B, x, info);
}

}  // namespace mgh
