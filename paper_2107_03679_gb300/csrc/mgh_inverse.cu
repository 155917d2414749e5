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
#include <cmath>

#include "mgh_engine.h"

namespace mgh {

namespace {

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
  const size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (k >= (size_t)nx * ny) return;
  const int i = (int)(k / nx), j = (int)(k - (size_t)i * nx);
  const double v = w[k] - lam * adj_at(p, q, i, j, nx, ny);
  x[k] = v > 0.0 ? v : 0.0;
}

// dual projected-gradient step from the momentum point and the next momentum point
__global__ void k_tv_dual(const double* __restrict__ x, double* __restrict__ pr, double* __restrict__ qr,
                          double* __restrict__ pp, double* __restrict__ qq, double step, double c, int nx, int ny) {
  const size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (k >= (size_t)nx * ny) return;
  const int i = (int)(k / nx), j = (int)(k - (size_t)i * nx);
  const double gp = i < ny - 1 ? x[k] - x[k + nx] : 0.0;
  const double gq = j < nx - 1 ? x[k] - x[k + 1] : 0.0;
  double pn = pr[k] + step * gp, qn = qr[k] + step * gq;
  const double nrm = sqrt(pn * pn + qn * qn);
  if (nrm > 1.0) { pn /= nrm; qn /= nrm; }
  pr[k] = pn + c * (pn - pp[k]);
  qr[k] = qn + c * (qn - qq[k]);
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
  double* x = w + n;
  double *pr = x + n, *qr = pr + n, *pp = qr + n, *qq = pp + n;
  ProfScope ps(h, P_OTHER);
  k_tv_w<<<blocks(n), kInvThreads, 0, h.stream>>>(fbar, d, gamma, w, n);
  MGH_CHECK_LAUNCH(); h.launches++;
  if (lam == 0.0) {   // prox of the constraint alone: the clamp
    MGH_CUDA(cudaMemsetAsync(pp, 0, 2 * n * sizeof(double), h.stream));
    k_tv_primal<<<blocks(n), kInvThreads, 0, h.stream>>>(w, pp, qq, 0.0, out, nx, ny);
    MGH_CHECK_LAUNCH(); h.launches++;
    return MGH_OK;
  }
  MGH_CUDA(cudaMemsetAsync(pr, 0, 4 * n * sizeof(double), h.stream));
  double t = 1.0;
  for (int it = 0; it < iters; ++it) {
    const double tn = (1.0 + std::sqrt(1.0 + 4.0 * t * t)) / 2.0;
    k_tv_primal<<<blocks(n), kInvThreads, 0, h.stream>>>(w, pr, qr, lam, x, nx, ny);
    MGH_CHECK_LAUNCH(); h.launches++;
    k_tv_dual<<<blocks(n), kInvThreads, 0, h.stream>>>(x, pr, qr, pp, qq, 1.0 / (8.0 * lam), (t - 1.0) / tn, nx, ny);
    MGH_CHECK_LAUNCH(); h.launches++;
    t = tn;
  }
  k_tv_primal<<<blocks(n), kInvThreads, 0, h.stream>>>(w, pp, qq, lam, out, nx, ny);
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
