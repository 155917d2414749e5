// Operator set-up and the pointwise kernels of the forward model:
//   * fine coefficient k0^2 eta^2 = k^2 (1 + f_d) on Omega, k^2 in the layer (Sec. II-A, IV-A)
//   * coarse coefficients by full weighting with the outer ring reset to k^2 (Sec. IV-C)
//   * diagonals of A and of K_kappa on every level: 4/h^2 - kappa*alpha*c, plus -(1 + j h k)/h^2
//     per neighbour closed by the first-order Sommerfeld ghost value (Sec. IV-A/B)
//   * exact coarsest solve: banded LU with partial pivoting, then the dense inverse (Alg. 2)
//   * plane waves and right-hand sides (Sec. II-A), y = A x, truncation to Omega (Sec. IV-A),
//     receiver sampling, the quadratic data term and the gradient of Prop. 1 (Sec. V)
#include <cmath>
#include <cstring>

#include "mgh_diag.cuh"
#include "mgh_engine.h"

namespace mgh {

namespace {

constexpr int kThreads = 256;

inline unsigned blocks_for(size_t n, int threads = kThreads) {
  size_t b = (n + threads - 1) / threads;
  return (unsigned)(b > 0 ? b : 1);
}

__global__ void k_fine_coef(const double* __restrict__ f_d, double* __restrict__ c, int nx, int ny,
                            int abl, int nx_int, int ny_int, double k2) {
  const size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (q >= (size_t)nx * ny) return;
  const int n = (int)((unsigned)q / (unsigned)nx), m = (int)((unsigned)q - (unsigned)n * (unsigned)nx);
  const int mi = m - abl, ni = n - abl;
  double v = k2;
  if (mi >= 0 && mi < nx_int && ni >= 0 && ni < ny_int) v = k2 * (1.0 + f_d[(size_t)ni * nx_int + mi]);
  c[q] = v;
}

// Full weighting of the coefficient (fine samples outside the grid count as 0), then the outer
// ring of the coarse level reset to the background value k^2.
__global__ void k_restrict_coef(const double* __restrict__ cf_, double* __restrict__ cc, int nx, int ny,
                                int nxc, int nyc, double k2) {
  const size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (q >= (size_t)nxc * nyc) return;
  const int j = (int)((unsigned)q / (unsigned)nxc), i = (int)((unsigned)q - (unsigned)j * (unsigned)nxc);
  if (i == 0 || j == 0 || i == nxc - 1 || j == nyc - 1) { cc[q] = k2; return; }
  double s = 0.0;
  for (int dn = -1; dn <= 1; ++dn)
    for (int dm = -1; dm <= 1; ++dm) {
      const int m = 2 * i + dm, n = 2 * j + dn;
      if (m < 0 || m >= nx || n < 0 || n >= ny) continue;
      const double w = (dm == 0 ? 2.0 : 1.0) * (dn == 0 ? 2.0 : 1.0);
      s += w * cf_[(size_t)n * nx + m];
    }
  cc[q] = s / 16.0;
}

template <typename T>
__global__ void k_level_diag(const double* __restrict__ c, DiagArgs<double> a, Cx<T>* __restrict__ D,
                             Cx<T>* __restrict__ wDinv) {
  const size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (q >= (size_t)a.nx * a.ny) return;
  const int j = (int)((unsigned)q / (unsigned)a.nx), i = (int)((unsigned)q - (unsigned)j * (unsigned)a.nx);
  const cd d = level_diag(a, i, j, c[q]);
  D[q] = ccast<T>(d);
  if (wDinv) {
    const double den = d.re * d.re + d.im * d.im;
    wDinv[q] = ccast<T>(mk<double>(a.omega * d.re / den, -a.omega * d.im / den));
  }
}

// ---------------------------------------------------------------- coarsest level (Alg. 2)
// Band storage: row i keeps columns c in [i-kl, i+kl+ku] at band[i*W + c - i + kl],
// W = 2*kl + ku + 1 (the extra kl columns hold the fill-in of partial pivoting).
__global__ void k_band_assemble(const cd* __restrict__ D, cd* __restrict__ band, int nx, int ny, int W,
                                double off) {
  const int n = nx * ny, kl = nx;
  const size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (q >= (size_t)n * W) return;
  const int i = (int)(q / W), o = (int)(q % W);
  const int c = i + o - kl;
  cd v = czero<double>();
  if (c >= 0 && c < n) {
    if (c == i) v = D[i];
    else {
      const int mi = i % nx, mc = c % nx;
      const bool xnb = (c == i - 1 && mi > 0) || (c == i + 1 && mi < nx - 1);
      const bool ynb = (c == i - nx) || (c == i + nx);
      if (xnb || (ynb && mc == mi)) v = mk<double>(off, 0.0);
    }
  }
  band[q] = v;
}

// LU with partial pivoting of the banded coarsest operator; one block walks the columns.
__global__ void k_band_lu(cd* __restrict__ band, int* __restrict__ piv, int n, int kl, int ku,
                          int* __restrict__ info) {
  const int W = 2 * kl + ku + 1;
  __shared__ int s_p;
  __shared__ int s_fail;
  if (threadIdx.x == 0) s_fail = 0;
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    const int last = min(n - 1, j + kl);
    if (threadIdx.x < 32) {
      double best = -1.0;
      int bi = j;
      for (int i = j + (int)threadIdx.x; i <= last; i += 32) {
        const double a = cabs2(band[(size_t)i * W + j - i + kl]);
        if (a > best) { best = a; bi = i; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (threadIdx.x == 0) {
        s_p = bi;
        piv[j] = bi;
        if (!(best > 0.0)) s_fail = j + 1;
      }
    }
    __syncthreads();
    if (s_fail) break;
    const int p = s_p;
    const int cend = min(n - 1, j + kl + ku);
    if (p != j) {
      for (int c = j + (int)threadIdx.x; c <= cend; c += blockDim.x) {
        cd* a = &band[(size_t)j * W + c - j + kl];
        cd* b = &band[(size_t)p * W + c - p + kl];
        const cd t = *a; *a = *b; *b = t;
      }
    }
    __syncthreads();
    const cd piv_v = band[(size_t)j * W + kl];
    const double den = cabs2(piv_v);
    const cd inv = mk<double>(piv_v.re / den, -piv_v.im / den);
    for (int i = j + 1 + (int)threadIdx.x; i <= last; i += blockDim.x) {
      cd* l = &band[(size_t)i * W + j - i + kl];
      *l = *l * inv;
    }
    __syncthreads();
    const int nr = last - j, ncol = cend - j;
    for (int t = threadIdx.x; t < nr * ncol; t += blockDim.x) {
      const int i = j + 1 + t / ncol, c = j + 1 + t % ncol;
      const cd l = band[(size_t)i * W + j - i + kl];
      const cd u = band[(size_t)j * W + c - j + kl];
      cd* a = &band[(size_t)i * W + c - i + kl];
      *a = *a - l * u;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *info = s_fail;
}

// Column k of K^{-1}: forward (row swaps + unit lower L) and backward (U) substitution in one
// warp; the column is written contiguously, kinvT[k*n + r] = (K^{-1})[r][k].
__global__ void k_band_inverse(const cd* __restrict__ band, const int* __restrict__ piv, int n, int kl,
                               int ku, cd* __restrict__ kinvT) {
  extern __shared__ cd y[];
  const int W = 2 * kl + ku + 1;
  const int k = blockIdx.x;
  const int lane = threadIdx.x;
  for (int r = lane; r < n; r += 32) y[r] = mk<double>(r == k ? 1.0 : 0.0, 0.0);
  __syncwarp();
  for (int j = 0; j < n; ++j) {
    const int p = piv[j];
    if (p != j && lane == 0) { const cd t = y[j]; y[j] = y[p]; y[p] = t; }
    __syncwarp();
    const cd yj = y[j];
    const int last = min(n - 1, j + kl);
    for (int i = j + 1 + lane; i <= last; i += 32) y[i] = y[i] - band[(size_t)i * W + j - i + kl] * yj;
    __syncwarp();
  }
  const int ub = kl + ku;
  for (int j = n - 1; j >= 0; --j) {
    const cd u = band[(size_t)j * W + kl];
    const double den = cabs2(u);
    const cd yj = y[j] * mk<double>(u.re / den, -u.im / den);
    __syncwarp();
    if (lane == 0) y[j] = yj;
    for (int i = max(0, j - ub) + lane; i < j; i += 32) y[i] = y[i] - band[(size_t)i * W + j - i + kl] * yj;
    __syncwarp();
  }
  for (int r = lane; r < n; r += 32) kinvT[(size_t)k * n + r] = y[r];
}

// Split a complex FP64 array into double-float planes: hi[q] = (float)v, lo[q] = (float)(v - hi).
__global__ void k_split_df(const cd* __restrict__ a, float2* __restrict__ hi, float2* __restrict__ lo, size_t n) {
  const size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (q >= n) return;
  const cd v = a[q];
  const float rh = (float)v.re, ih = (float)v.im;
  hi[q] = make_float2(rh, ih);
  lo[q] = make_float2((float)(v.re - (double)rh), (float)(v.im - (double)ih));
}


// Row-major copies of the transposed inverse: Kr[r][c] = kinvT[c][r] (FP64 and FP32).
__global__ void k_transpose_inv(const cd* __restrict__ kinvT, int n, cd* __restrict__ k64r, cf* __restrict__ k32r) {
  const size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (q >= (size_t)n * n) return;
  const int r = (int)(q / n), c = (int)(q % n);
  const cd v = kinvT[(size_t)c * n + r];
  k64r[q] = v;
  if (k32r) k32r[q] = ccast<float>(v);
}

template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// x[q][r] = sum_c K^{-1}[r][c] b[q][c]: one warp per (row, right-hand side), the lanes split the
// columns (coalesced reads of the row-major inverse and of b), two independent accumulators.
template <typename TK, typename TIO>
__global__ void k_coarse_apply_w(const Cx<TK>* __restrict__ Kr, int n, int B, const Cx<TIO>* __restrict__ b,
                                 size_t b_stride, Cx<TIO>* __restrict__ x, size_t x_stride,
                                 const RhsState* __restrict__ st) {
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= (long long)n * B) return;
  const int rhs = (int)(warp / n), r = (int)(warp - (long long)rhs * n);
  if (st && !st[rhs].active) return;
  const Cx<TIO>* bb = b + rhs * b_stride;
  const Cx<TK>* row = Kr + (size_t)r * n;
  TK a0r = 0, a0i = 0, a1r = 0, a1i = 0;
  int c = lane;
  for (; c + 32 < n; c += 64) {
    const Cx<TK> k0 = row[c], k1 = row[c + 32];
    const Cx<TK> b0 = ccast<TK>(bb[c]), b1 = ccast<TK>(bb[c + 32]);
    a0r = fma(k0.re, b0.re, fma(-k0.im, b0.im, a0r));
    a0i = fma(k0.re, b0.im, fma(k0.im, b0.re, a0i));
    a1r = fma(k1.re, b1.re, fma(-k1.im, b1.im, a1r));
    a1i = fma(k1.re, b1.im, fma(k1.im, b1.re, a1i));
  }
  if (c < n) {
    const Cx<TK> k0 = row[c];
    const Cx<TK> b0 = ccast<TK>(bb[c]);
    a0r = fma(k0.re, b0.re, fma(-k0.im, b0.im, a0r));
    a0i = fma(k0.re, b0.im, fma(k0.im, b0.re, a0i));
  }
  const TK sr = warp_sum_t<TK>(a0r + a1r), si = warp_sum_t<TK>(a0i + a1i);
  if (lane == 0) x[rhs * x_stride + r] = ccast<TIO>(mk<TK>(sr, si));
}

// ---------------------------------------------------------------- forward-model kernels
// u_in = exp(j k (x cos(theta) + y sin(theta))), x = m h, y = n h; optionally times k^2 f_d.
__global__ void k_incident(const double* __restrict__ theta, const double* __restrict__ f_d, int nx,
                           int ny, int abl, int nx_int, int ny_int, double h, double k,
                           cd* __restrict__ out) {
  const size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  const size_t N = (size_t)nx * ny;
  if (q >= N) return;
  const int rhs = blockIdx.y;
  const int n = (int)((unsigned)q / (unsigned)nx), m = (int)((unsigned)q - (unsigned)n * (unsigned)nx);
  double s = 1.0;
  if (f_d) {
    const int mi = m - abl, ni = n - abl;
    s = (mi >= 0 && mi < nx_int && ni >= 0 && ni < ny_int) ? k * k * f_d[(size_t)ni * nx_int + mi] : 0.0;
  }
  const double th = theta[rhs];
  const double ph = k * (cos(th) * (m * h) + sin(th) * (n * h));
  double sv, cv;
  sincos(ph, &sv, &cv);
  out[rhs * N + q] = mk<double>(s * cv, s * sv);
}

// y = A x: (4 x - sum of in-grid neighbours)/h^2 - alpha c x with the closure in the diagonal DA.
__global__ void k_apply_A(const cd* __restrict__ DA, const cd* __restrict__ x, cd* __restrict__ y, int nx,
                          int ny, double inv_h2) {
  const size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  const size_t N = (size_t)nx * ny;
  if (q >= N) return;
  const int n = (int)((unsigned)q / (unsigned)nx), m = (int)((unsigned)q - (unsigned)n * (unsigned)nx);
  const cd* xb = x + blockIdx.y * N;
  cd s = czero<double>();
  if (m > 0) s = s + xb[q - 1];
  if (m < nx - 1) s = s + xb[q + 1];
  if (n > 0) s = s + xb[q - nx];
  if (n < ny - 1) s = s + xb[q + nx];
  y[blockIdx.y * N + q] = DA[q] * xb[q] - inv_h2 * s;
}

__global__ void k_crop(const cd* __restrict__ u, cd* __restrict__ out, int nx, int ny, int abl, int nx_int,
                       int ny_int) {
  const size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  const size_t Ni = (size_t)nx_int * ny_int;
  if (q >= Ni) return;
  const int ni = (int)((unsigned)q / (unsigned)nx_int), mi = (int)((unsigned)q - (unsigned)ni * (unsigned)nx_int);
  out[blockIdx.y * Ni + q] = u[blockIdx.y * (size_t)nx * ny + (size_t)(ni + abl) * nx + mi + abl];
}

__global__ void k_sample(const cd* __restrict__ u, size_t N, const int64_t* __restrict__ rec, int M,
                         cd* __restrict__ out) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= M) return;
  out[(size_t)blockIdx.y * M + r] = u[blockIdx.y * N + rec[r]];
}

__global__ void k_scatter(const cd* __restrict__ vals, size_t N, const int64_t* __restrict__ rec, int M,
                          cd* __restrict__ G) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= M) return;
  G[blockIdx.y * N + rec[r]] = vals[(size_t)blockIdx.y * M + r];
}

// r = S u - y; G (pre-zeroed) gets S^T r; per-RHS partial loss sums.
__global__ void k_misfit(const cd* __restrict__ u, const cd* __restrict__ y, size_t N,
                         const int64_t* __restrict__ rec, int M, cd* __restrict__ r, cd* __restrict__ G,
                         double* __restrict__ loss_part) {
  __shared__ double sh[32];
  const int rhs = blockIdx.x;
  double acc = 0.0;
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    const cd d = u[rhs * N + rec[i]] - y[(size_t)rhs * M + i];
    if (r) r[(size_t)rhs * M + i] = d;
    if (G) G[rhs * N + rec[i]] = d;
    acc += cabs2(d);
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) loss_part[rhs] = 0.5 * v;
  }
}

__global__ void k_sum_small(const double* __restrict__ a, int n, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += a[i];
    *out = s;
  }
}

__global__ void k_conj(const cd* __restrict__ in, cd* __restrict__ out, size_t n) {
  const size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (q < n) out[q] = cconj(in[q]);
}

// grad[ni][mi] = k^2 sum_q Re(z_q (u_sc,q + u_in,q)) on Omega (Prop. 1).
__global__ void k_gradient(const double* __restrict__ theta, const cd* __restrict__ u_sc,
                           const cd* __restrict__ z, int B, int nx, int ny, int abl, int nx_int,
                           int ny_int, double h, double k, double* __restrict__ grad) {
  const size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (q >= (size_t)nx_int * ny_int) return;
  const int ni = (int)((unsigned)q / (unsigned)nx_int), mi = (int)((unsigned)q - (unsigned)ni * (unsigned)nx_int);
  const int m = mi + abl, n = ni + abl;
  const size_t N = (size_t)nx * ny, p = (size_t)n * nx + m;
  double acc = 0.0;
  for (int b = 0; b < B; ++b) {
    const double th = theta[b];
    double sv, cv;
    sincos(k * (cos(th) * (m * h) + sin(th) * (n * h)), &sv, &cv);
    const cd u = u_sc[b * N + p] + mk<double>(cv, sv);
    const cd zz = z[b * N + p];
    acc += zz.re * u.re - zz.im * u.im;
  }
  grad[q] = k * k * acc;
}

}  // namespace

// ------------------------------------------------------------------------------- host side
mgh_status setup_contrast(Handle& h, const double* f_d) {
  const mgh_params& p = h.p;
  cudaStream_t s = h.stream;
  MGH_CUDA(cudaMemcpyAsync(h.f_d, f_d, sizeof(double) * p.nx_int * p.ny_int, cudaMemcpyDeviceToDevice, s));
  const double k2 = p.k * p.k;
  k_fine_coef<<<blocks_for(h.N), kThreads, 0, s>>>(h.f_d, h.lev[0].c, h.nx, h.ny, p.abl, p.nx_int,
                                                   p.ny_int, k2);
  MGH_CHECK_LAUNCH(); h.launches++;
  for (int l = 0; l + 1 < h.L; ++l) {
    const Level& a = h.lev[l];
    Level& b = h.lev[l + 1];
    k_restrict_coef<<<blocks_for(b.n()), kThreads, 0, s>>>(a.c, b.c, a.nx, a.ny, b.nx, b.ny, k2);
    MGH_CHECK_LAUNCH(); h.launches++;
  }
  DiagArgs<double> da;
  da.x0 = p.abl; da.x1 = p.abl + p.nx_int - 1;
  da.y0 = p.abl; da.y1 = p.abl + p.ny_int - 1;
  da.inv_L2 = p.abl > 0 ? 1.0 / ((double)p.abl * p.abl) : 0.0;
  da.beta = p.beta; da.omega = p.omega;
  // fine operator A (unshifted)
  da.nx = h.nx; da.ny = h.ny; da.scale = 1; diag_set_spacing(da, p.h, p.k); da.kap_re = 1.0; da.kap_im = 0.0;
  k_level_diag<double><<<blocks_for(h.N), kThreads, 0, s>>>(h.lev[0].c, da, h.DA, nullptr);
  MGH_CHECK_LAUNCH(); h.launches++;
  k_split_df<<<blocks_for(h.N), kThreads, 0, s>>>(h.DA, h.DAdf, h.DAdf + h.Np, h.N);
  MGH_CHECK_LAUNCH(); h.launches++;
  // K_kappa on every level
  da.kap_re = p.shift_re; da.kap_im = p.shift_im;
  for (int l = 0; l < h.L; ++l) {
    Level& lv = h.lev[l];
    da.nx = lv.nx; da.ny = lv.ny; da.scale = lv.scale; diag_set_spacing(da, lv.h, p.k);
    if (h.fp64)
      k_level_diag<double><<<blocks_for(lv.n()), kThreads, 0, s>>>(lv.c, da, (cd*)lv.D, (cd*)lv.wDinv);
    else
      k_level_diag<float><<<blocks_for(lv.n()), kThreads, 0, s>>>(lv.c, da, (cf*)lv.D, (cf*)lv.wDinv);
    MGH_CHECK_LAUNCH(); h.launches++;
  }
  // coarsest: FP64 diagonal (recomputed in FP64 whatever the cycle precision), banded LU, inverse
  const Level& cl = h.lev[h.L - 1];
  const int n = h.nc, kl = cl.nx, ku = cl.nx, W = 2 * kl + ku + 1;
  da.nx = cl.nx; da.ny = cl.ny; da.scale = cl.scale; diag_set_spacing(da, cl.h, p.k);
  cd* Dc = h.kinv64;  // borrow the inverse buffer (n*n >= n) for the FP64 diagonal
  k_level_diag<double><<<blocks_for(cl.n()), kThreads, 0, s>>>(cl.c, da, Dc, nullptr);
  MGH_CHECK_LAUNCH(); h.launches++;
  k_band_assemble<<<blocks_for((size_t)n * W), kThreads, 0, s>>>(Dc, h.band, cl.nx, cl.ny, W,
                                                                 -1.0 / (cl.h * cl.h));
  MGH_CHECK_LAUNCH(); h.launches++;
  k_band_lu<<<1, 256, 0, s>>>(h.band, h.piv, n, kl, ku, h.lu_info);
  MGH_CHECK_LAUNCH(); h.launches++;
  MGH_CUDA(cudaFuncSetAttribute(k_band_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(sizeof(cd) * n)));
  k_band_inverse<<<n, 32, sizeof(cd) * n, s>>>(h.band, h.piv, n, kl, ku, h.kinv64);
  MGH_CHECK_LAUNCH(); h.launches++;
  k_transpose_inv<<<blocks_for((size_t)n * n), kThreads, 0, s>>>(h.kinv64, n, h.kinv64r, h.fp64 ? nullptr : h.kinv32);
  MGH_CHECK_LAUNCH(); h.launches++;
  int info = 0;
  MGH_CUDA(cudaMemcpyAsync(&info, h.lu_info, sizeof(int), cudaMemcpyDeviceToHost, s));
  MGH_CUDA(cudaStreamSynchronize(s));
  MGH_TRY(prof_flush(h));
  if (info != 0) return MGH_INVALID_ARG;   // singular coarsest operator
  h.contrast_set = true;
  return MGH_OK;
}

mgh_status launch_coarse_apply(Handle& h, const void* b, size_t b_stride, void* x, size_t x_stride, int B,
                               const RhsState* st, bool fp64_io) {
  const int n = h.nc;
  const long long warps = (long long)n * B;
  const unsigned grid = (unsigned)((warps * 32 + 255) / 256);
  ProfScope ps(h, st ? P_COARSE : P_OTHER);
  if (fp64_io) {
    k_coarse_apply_w<double, double><<<grid, 256, 0, h.stream>>>(h.kinv64r, n, B, (const cd*)b, b_stride, (cd*)x,
                                                                 x_stride, st);
  } else {
    k_coarse_apply_w<float, float><<<grid, 256, 0, h.stream>>>(h.kinv32, n, B, (const cf*)b, b_stride, (cf*)x,
                                                               x_stride, st);
  }
  MGH_CHECK_LAUNCH(); h.launches++;
  return MGH_OK;
}

mgh_status launch_incident(Handle& h, const double* theta, int B, cd* out, bool times_contrast) {
  const mgh_params& p = h.p;
  dim3 grid(blocks_for(h.N), B);
  k_incident<<<grid, kThreads, 0, h.stream>>>(theta, times_contrast ? h.f_d : nullptr, h.nx, h.ny, p.abl,
                                              p.nx_int, p.ny_int, p.h, p.k, out);
  MGH_CHECK_LAUNCH(); h.launches++;
  return MGH_OK;
}

mgh_status launch_apply_A(Handle& h, const cd* x, int B, cd* y) {
  dim3 grid(blocks_for(h.N), B);
  k_apply_A<<<grid, kThreads, 0, h.stream>>>(h.DA, x, y, h.nx, h.ny, 1.0 / (h.p.h * h.p.h));
  MGH_CHECK_LAUNCH(); h.launches++;
  return MGH_OK;
}

mgh_status launch_crop(Handle& h, const cd* u, int B, cd* out) {
  const mgh_params& p = h.p;
  dim3 grid(blocks_for((size_t)p.nx_int * p.ny_int), B);
  k_crop<<<grid, kThreads, 0, h.stream>>>(u, out, h.nx, h.ny, p.abl, p.nx_int, p.ny_int);
  MGH_CHECK_LAUNCH(); h.launches++;
  return MGH_OK;
}

mgh_status launch_sample(Handle& h, const cd* u, int B, const int64_t* rec, int M, cd* out) {
  dim3 grid((M + 127) / 128, B);
  k_sample<<<grid, 128, 0, h.stream>>>(u, h.N, rec, M, out);
  MGH_CHECK_LAUNCH(); h.launches++;
  return MGH_OK;
}

mgh_status launch_scatter(Handle& h, const cd* vals, int B, const int64_t* rec, int M, cd* G) {
  MGH_CUDA(cudaMemsetAsync(G, 0, sizeof(cd) * h.N * B, h.stream));
  dim3 grid((M + 127) / 128, B);
  k_scatter<<<grid, 128, 0, h.stream>>>(vals, h.N, rec, M, G);
  MGH_CHECK_LAUNCH(); h.launches++;
  return MGH_OK;
}

mgh_status launch_misfit(Handle& h, const cd* u, const cd* y, int B, const int64_t* rec, int M, cd* r,
                         cd* G, double* loss_dev) {
  if (G) MGH_CUDA(cudaMemsetAsync(G, 0, sizeof(cd) * h.N * B, h.stream));
  k_misfit<<<B, 256, 0, h.stream>>>(u, y, h.N, rec, M, r, G, h.dscratch);
  MGH_CHECK_LAUNCH(); h.launches++;
  k_sum_small<<<1, 32, 0, h.stream>>>(h.dscratch, B, loss_dev);
  MGH_CHECK_LAUNCH(); h.launches++;
  return MGH_OK;
}

mgh_status launch_conj(Handle& h, const cd* in, int B, cd* out) {
  const size_t n = h.N * B;
  k_conj<<<blocks_for(n), kThreads, 0, h.stream>>>(in, out, n);
  MGH_CHECK_LAUNCH(); h.launches++;
  return MGH_OK;
}

mgh_status launch_gradient(Handle& h, const double* theta, const cd* u_sc, const cd* z, int B,
                           double* grad) {
  const mgh_params& p = h.p;
  k_gradient<<<blocks_for((size_t)p.nx_int * p.ny_int), kThreads, 0, h.stream>>>(
      theta, u_sc, z, B, h.nx, h.ny, p.abl, p.nx_int, p.ny_int, p.h, p.k, grad);
  MGH_CHECK_LAUNCH(); h.launches++;
  return MGH_OK;
}

}  // namespace mgh
