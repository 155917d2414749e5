// Reconstruction-loop kernels (Sec. V, Alg. 4): the proximal operator of nonnegativity + isotropic
// total variation by fast gradient projection on the dual (Beck & Teboulle 2009), and the momentum
// step of the accelerated forward-backward splitting.  Fields are real FP64 on the interior grid
// [ny_int][nx_int] (x fastest); TV uses forward differences along y (rows) and x that are 0 across
// the last row / column:
//   p_ij = x_ij - x_i+1,j,  q_ij = x_ij - x_i,j+1,  TV(x) = sum sqrt(p^2 + q^2)
//   adj(p, q)_ij = p_ij [i < ny-1] - p_i-1,j [i > 0] + q_ij [j < nx-1] - q_i,j-1 [j > 0]
// One prox iteration, with (pr, qr) the momentum point and (pp, qq) the last dual iterate:
//   x = max(w - lam adj(pr, qr), 0)
//   (pn, qn) = (pr, qr) + grad(x) / (8 lam), divided by max(1, |(pn, qn)|)
//   (pr, qr) = (pn, qn) + c ((pn, qn) - (pp, qq)),  (pp, qq) = (pn, qn),  c = (t - 1) / t'
// and the result is max(w - lam adj(pp, qq), 0).
//
// The fields are small (2 MB each on a 512^2 interior, all six held in L2), so one iteration is
// one launch: each thread forms x at its point and at the two forward neighbours from the
// momentum point (read from one buffer of a ping-pong pair, written to the other), so no pass
// over x is stored between the primal and the dual step.
#include <cmath>

#include "mgh_engine.h"

namespace mgh {

namespace {

constexpr int kTx = 32, kTy = 8;   // 2-D blocks over (x, y) of the interior
constexpr int kInvThreads = 256;

__device__ __forceinline__ double adj_at(const double* __restrict__ p, const double* __restrict__ q, int i, int j,
                                         int nx, int ny) {
  const size_t k = (size_t)i * nx + j;
  double s = 0.0;
  if (i < ny - 1) s += p[k];
  if (i > 0) s -= p[k - nx];
  if (j < nx - 1) s += q[k];
  if (j > 0) s -= q[k - 1];
  return s;
}

__device__ __forceinline__ double primal_at(const double* __restrict__ w, const double* __restrict__ p,
                                            const double* __restrict__ q, double lam, int i, int j, int nx, int ny) {
  const double v = w[(size_t)i * nx + j] - lam * adj_at(p, q, i, j, nx, ny);
  return v > 0.0 ? v : 0.0;
}

// w = fbar - gamma d (d may be null)
__global__ void k_tv_w(const double* __restrict__ fbar, const double* __restrict__ d, double gamma,
                       double* __restrict__ w, size_t n) {
  const size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (k >= n) return;
  w[k] = d ? fbar[k] - gamma * d[k] : fbar[k];
}

// x = max(w - lam adj(p, q), 0)
__global__ void k_tv_primal(const double* __restrict__ w, const double* __restrict__ p, const double* __restrict__ q,
                            double lam, double* __restrict__ x, int nx, int ny) {
  const int j = blockIdx.x * kTx + threadIdx.x, i = blockIdx.y * kTy + threadIdx.y;
  if (i >= ny || j >= nx) return;
  x[(size_t)i * nx + j] = primal_at(w, p, q, lam, i, j, nx, ny);
}

// One FGP iteration: the primal point of the momentum point (pr, qr) at (i, j), (i+1, j) and
// (i, j+1), the projected dual step, the next momentum point into (pr_out, qr_out) and the dual
// iterate into (pp, qq) (each thread owns its entries of pp, qq).
__global__ void k_tv_iter(const double* __restrict__ w, const double* __restrict__ pr, const double* __restrict__ qr,
                          double* __restrict__ pr_out, double* __restrict__ qr_out, double* __restrict__ pp,
                          double* __restrict__ qq, double lam, double step, double c, int nx, int ny) {
  const int j = blockIdx.x * kTx + threadIdx.x, i = blockIdx.y * kTy + threadIdx.y;
  if (i >= ny || j >= nx) return;
  const size_t k = (size_t)i * nx + j;
  const double x0 = primal_at(w, pr, qr, lam, i, j, nx, ny);
  const double gp = i < ny - 1 ? x0 - primal_at(w, pr, qr, lam, i + 1, j, nx, ny) : 0.0;
  const double gq = j < nx - 1 ? x0 - primal_at(w, pr, qr, lam, i, j + 1, nx, ny) : 0.0;
  double pn = pr[k] + step * gp, qn = qr[k] + step * gq;
  const double nrm = sqrt(pn * pn + qn * qn);
  if (nrm > 1.0) { pn /= nrm; qn /= nrm; }
  pr_out[k] = pn + c * (pn - pp[k]);
  qr_out[k] = qn + c * (qn - qq[k]);
  pp[k] = pn;
  qq[k] = qn;
}

__global__ void k_fbs_momentum(const double* __restrict__ f, const double* __restrict__ fp, double c,
                               double* __restrict__ fbar, size_t n) {
  const size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (k >= n) return;
  fbar[k] = f[k] + c * (f[k] - fp[k]);
}

unsigned blocks(size_t n) { return (unsigned)((n + kInvThreads - 1) / kInvThreads); }

}  // namespace

mgh_status tv_prox(Handle& h, const double* fbar, const double* d, double gamma, double lam, int iters,
                   double* out) {
  const int nx = h.p.nx_int, ny = h.p.ny_int;
  const size_t n = (size_t)nx * ny;
  double* w = h.tvbuf;
  double* pr[2] = {w + n, w + 2 * n};
  double* qr[2] = {w + 3 * n, w + 4 * n};
  double *pp = w + 5 * n, *qq = w + 6 * n;
  const dim3 blk(kTx, kTy), grd((unsigned)((nx + kTx - 1) / kTx), (unsigned)((ny + kTy - 1) / kTy));
  ProfScope ps(h, P_OTHER);
  k_tv_w<<<blocks(n), kInvThreads, 0, h.stream>>>(fbar, d, gamma, w, n);
  MGH_CHECK_LAUNCH(); h.launches++;
  if (lam == 0.0) {   // prox of the constraint alone: the clamp
    MGH_CUDA(cudaMemsetAsync(pp, 0, 2 * n * sizeof(double), h.stream));
    k_tv_primal<<<grd, blk, 0, h.stream>>>(w, pp, qq, 0.0, out, nx, ny);
    MGH_CHECK_LAUNCH(); h.launches++;
    return MGH_OK;
  }
  // pr[0], qr[0] (the first momentum point) and pp, qq start at 0; pr[1], qr[1] are written first
  MGH_CUDA(cudaMemsetAsync(pr[0], 0, n * sizeof(double), h.stream));
  MGH_CUDA(cudaMemsetAsync(qr[0], 0, 3 * n * sizeof(double), h.stream));   // qr[0], qr[1], pp: contiguous
  MGH_CUDA(cudaMemsetAsync(qq, 0, n * sizeof(double), h.stream));
  double t = 1.0;
  for (int it = 0; it < iters; ++it) {
    const double tn = (1.0 + std::sqrt(1.0 + 4.0 * t * t)) / 2.0;
    const int a = it & 1;
    k_tv_iter<<<grd, blk, 0, h.stream>>>(w, pr[a], qr[a], pr[a ^ 1], qr[a ^ 1], pp, qq, lam, 1.0 / (8.0 * lam),
                                         (t - 1.0) / tn, nx, ny);
    MGH_CHECK_LAUNCH(); h.launches++;
    t = tn;
  }
  k_tv_primal<<<grd, blk, 0, h.stream>>>(w, pp, qq, lam, out, nx, ny);
  MGH_CHECK_LAUNCH(); h.launches++;
  return MGH_OK;
}

mgh_status fbs_momentum(Handle& h, const double* f, const double* f_prev, double c, double* fbar) {
  const size_t n = (size_t)h.p.nx_int * h.p.ny_int;
  ProfScope ps(h, P_OTHER);
  k_fbs_momentum<<<blocks(n), kInvThreads, 0, h.stream>>>(f, f_prev, c, fbar, n);
  MGH_CHECK_LAUNCH(); h.launches++;
  return MGH_OK;
}

}  // namespace mgh
