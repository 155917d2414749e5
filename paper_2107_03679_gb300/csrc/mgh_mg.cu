// One multigrid cycle (Alg. 2, zero initial guess; V-cycle, or CycleType >= 2 such as the W-cycle)
// on the shifted-Laplacian operator K_kappa for a batch of right-hand sides, in complex FP32 or
// FP64, with nu1 / nu2 sweeps that may differ by level.
//
// Each level other than the coarsest runs two fused, shared-memory tiled kernels:
//   k_pre   nu1 damped-Jacobi sweeps from v = 0 (eq. dampedJ), the residual r = b - K v and
//           its full-weighting restriction to the next level's right-hand side (Sec. IV-C);
//           all sweeps are done on one tile with a halo of nu1 + 1 points (temporal blocking)
//   k_post  bilinear prolongation of the coarse correction, v += P e (Sec. IV-C), then nu2
//           damped-Jacobi sweeps on a tile with a halo of nu2 points
// and the coarsest level applies the dense inverse of its operator (exact solve).
//
// Damped Jacobi is written v <- (1 - w) v + (w / D)(b + (sum of neighbours)/h^2), which is
// v - w D^{-1}(K v - b) for K v = D v - (sum of neighbours)/h^2; w/D is precomputed per level.
// Points outside the grid hold 0 in every tile buffer: the Sommerfeld closure already sits in D,
// and the restriction counts out-of-grid fine samples as 0.
#include <cudaTypedefs.h>
#include <algorithm>
#include <new>
#include <type_traits>

#include "mgh_engine.h"
#include "mgh_tma.cuh"
#include "mgh_wave.cuh"

namespace mgh {

namespace {

constexpr int kVThreads = 256;
constexpr int kVcThreadsTma = 512;   // threads of the TMA level kernels (one tile per block)

// Right-hand side of a level: complex TIn (FP64 input, FP32 hi plane of a double-float
// basis vector, or the level's own precision) times a per-RHS scale, converted to T.
template <typename T, typename TIn>
__device__ __forceinline__ Cx<T> load_rhs(const void* __restrict__ b, size_t off, double sc) {
  const Cx<TIn> v = reinterpret_cast<const Cx<TIn>*>(b)[off];
  if constexpr (sizeof(TIn) == 8) {
    return mk<T>(static_cast<T>(v.re * sc), static_cast<T>(v.im * sc));
  } else {
    const T s = static_cast<T>(sc);
    return mk<T>(static_cast<T>(v.re) * s, static_cast<T>(v.im) * s);
  }
}

template <typename T>
__device__ __forceinline__ Cx<T> jacobi_point(const Cx<T>* v, int idx, int SW, Cx<T> b, Cx<T> wd,
                                              T inv_h2, T om1) {
  const Cx<T> s = v[idx - 1] + v[idx + 1] + v[idx - SW] + v[idx + SW];
  const Cx<T> t = mk<T>(b.re + inv_h2 * s.re, b.im + inv_h2 * s.im);
  const Cx<T> c = v[idx];
  return mk<T>(om1 * c.re + wd.re * t.re - wd.im * t.im, om1 * c.im + wd.re * t.im + wd.im * t.re);
}

// Pre-smoothing + residual + full-weighting restriction on one TX x TY tile of level l.
template <typename T, int NU, int TX, int TY, typename TIn>
__global__ void __launch_bounds__(kVThreads)
k_pre(const void* __restrict__ bin, size_t b_stride, const double* __restrict__ bscale, size_t scale_stride,
      const Cx<T>* __restrict__ D, const Cx<T>* __restrict__ wDinv, Cx<T>* __restrict__ vpre,
      size_t v_stride, Cx<T>* __restrict__ bc, size_t bc_stride, int nx, int ny, int nxc, int nyc,
      T inv_h2, T om1, const RhsState* __restrict__ st) {
  constexpr int H = NU + 1;
  constexpr int SW = TX + 2 * H, SH = TY + 2 * H, S = SW * SH;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  Cx<T>* sb = reinterpret_cast<Cx<T>*>(smem_raw);
  Cx<T>* sw = sb + S;
  Cx<T>* sd = sw + S;
  Cx<T>* va = sd + S;
  Cx<T>* vb = va + S;

  const int rhs = blockIdx.z;
  if (st && !st[rhs].active) return;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const double sc = bscale ? bscale[rhs * scale_stride] : 1.0;
  const size_t boff = rhs * b_stride;

  // tile load: every global load of this thread is issued before the first shared store
  constexpr int NL = (S + kVThreads - 1) / kVThreads;
  {
    Cx<T> rb[NL], rw[NL], rd[NL];
#pragma unroll
    for (int r = 0; r < NL; ++r) {
      const int idx = threadIdx.x + r * kVThreads;
      rb[r] = czero<T>(); rw[r] = czero<T>(); rd[r] = czero<T>();
      const int ly = idx / SW, lx = idx - ly * SW;
      const int gx = x0 - H + lx, gy = y0 - H + ly;
      if (idx < S && gx >= 0 && gx < nx && gy >= 0 && gy < ny) {
        const size_t q = (size_t)gy * nx + gx;
        rb[r] = load_rhs<T, TIn>(bin, boff + q, sc);
        rw[r] = wDinv[q];
        rd[r] = D[q];
      }
    }
#pragma unroll
    for (int r = 0; r < NL; ++r) {
      const int idx = threadIdx.x + r * kVThreads;
      if (idx < S) {
        sb[idx] = rb[r]; sw[idx] = rw[r]; sd[idx] = rd[r];
        if constexpr (NU >= 1) va[idx] = rw[r] * rb[r];     // first sweep from v = 0
      }
    }
  }
  __syncthreads();

  Cx<T>* vcur = va;
  Cx<T>* vnxt = vb;
#pragma unroll
  for (int s = 2; s <= NU; ++s) {
    const int lo = s - 1, W = SW - 2 * lo, Hh = SH - 2 * lo;
    for (int t = threadIdx.x; t < W * Hh; t += kVThreads) {
      const int ly = lo + t / W, lx = lo + t % W;
      const int idx = ly * SW + lx;
      vnxt[idx] = jacobi_point(vcur, idx, SW, sb[idx], sw[idx], inv_h2, om1);
    }
    __syncthreads();
    Cx<T>* tmp = vcur; vcur = vnxt; vnxt = tmp;
  }

  // residual r = b - K v on fine [x0-1, x0+TX-1] x [y0-1, y0+TY-1] (local offset NU)
  Cx<T>* r = vnxt;
  {
    constexpr int W = TX + 1, Hh = TY + 1;
    for (int t = threadIdx.x; t < W * Hh; t += kVThreads) {
      const int ly = NU + t / W, lx = NU + t % W;
      const int idx = ly * SW + lx;
      const int gx = x0 - H + lx, gy = y0 - H + ly;
      Cx<T> rv = czero<T>();
      if (gx >= 0 && gx < nx && gy >= 0 && gy < ny) {
        if constexpr (NU >= 1) {
          const Cx<T> s = vcur[idx - 1] + vcur[idx + 1] + vcur[idx - SW] + vcur[idx + SW];
          const Cx<T> kv = sd[idx] * vcur[idx] - inv_h2 * s;
          rv = sb[idx] - kv;
        } else {
          rv = sb[idx];
        }
      }
      r[idx] = rv;
    }
  }
  __syncthreads();

  // restriction to the coarse points (2ci, 2cj) owned by this tile, and v on the owned points
  {
    constexpr int CW = TX / 2, CH = TY / 2;
    const int ci0 = x0 / 2, cj0 = y0 / 2;
    Cx<T>* bco = bc + rhs * bc_stride;
    for (int t = threadIdx.x; t < CW * CH; t += kVThreads) {
      const int ci = ci0 + t % CW, cj = cj0 + t / CW;
      if (ci >= nxc || cj >= nyc) continue;
      const int lx = 2 * ci - x0 + H, ly = 2 * cj - y0 + H;
      const int idx = ly * SW + lx;
      const Cx<T> e = r[idx - 1] + r[idx + 1] + r[idx - SW] + r[idx + SW];
      const Cx<T> c = r[idx - SW - 1] + r[idx - SW + 1] + r[idx + SW - 1] + r[idx + SW + 1];
      const T q16 = T(1) / T(16);
      bco[(size_t)cj * nxc + ci] = mk<T>(q16 * (T(4) * r[idx].re + T(2) * e.re + c.re),
                                         q16 * (T(4) * r[idx].im + T(2) * e.im + c.im));
    }
    Cx<T>* vo = vpre + rhs * v_stride;
    for (int t = threadIdx.x; t < TX * TY; t += kVThreads) {
      const int lx = H + t % TX, ly = H + t / TX;
      const int gx = x0 + t % TX, gy = y0 + t / TX;
      if (gx < nx && gy < ny) {
        Cx<T> v = czero<T>();
        if constexpr (NU >= 1) v = vcur[ly * SW + lx];
        vo[(size_t)gy * nx + gx] = v;
      }
    }
  }
}

__device__ __forceinline__ int floor_half(int a) { return a >= 0 ? a / 2 : -((1 - a) / 2); }

// Prolongation + correction + post-smoothing on one TX x TY tile of level l.
template <typename T, int NU, int TX, int TY, typename TIn, typename TOut>
__global__ void __launch_bounds__(kVThreads)
k_post(const void* __restrict__ bin, size_t b_stride, const double* __restrict__ bscale, size_t scale_stride,
       const Cx<T>* __restrict__ wDinv, const Cx<T>* __restrict__ vpre, size_t v_stride,
       const Cx<T>* __restrict__ ec, size_t ec_stride, int nxc, int nyc, Cx<TOut>* __restrict__ out,
       size_t out_stride, int nx, int ny, T inv_h2, T om1, const RhsState* __restrict__ st) {
  constexpr int H = NU;
  constexpr int SW = TX + 2 * H, SH = TY + 2 * H, S = SW * SH;
  constexpr int CW = TX / 2 + H + 2, CH = TY / 2 + H + 2, CS = CW * CH;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  Cx<T>* sb = reinterpret_cast<Cx<T>*>(smem_raw);
  Cx<T>* sw = sb + S;
  Cx<T>* va = sw + S;
  Cx<T>* vb = va + S;
  Cx<T>* se = vb + S;

  const int rhs = blockIdx.z;
  if (st && !st[rhs].active) return;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int cx0 = floor_half(x0 - H - 1), cy0 = floor_half(y0 - H - 1);
  const double sc = bscale ? bscale[rhs * scale_stride] : 1.0;
  const size_t boff = rhs * b_stride;
  const Cx<T>* vp = vpre + rhs * v_stride;
  const Cx<T>* eco = ec + rhs * ec_stride;

  // tile load: every global load of this thread is issued before the first shared store
  constexpr int NC = (CS + kVThreads - 1) / kVThreads;
  constexpr int NL = (S + kVThreads - 1) / kVThreads;
  {
    Cx<T> re[NC], rb[NL], rw[NL], rv[NL];
#pragma unroll
    for (int r = 0; r < NC; ++r) {
      const int t = threadIdx.x + r * kVThreads;
      const int cj = cy0 + t / CW, ci = cx0 + t % CW;
      re[r] = czero<T>();
      if (t < CS && ci >= 0 && ci < nxc && cj >= 0 && cj < nyc) re[r] = eco[(size_t)cj * nxc + ci];
    }
#pragma unroll
    for (int r = 0; r < NL; ++r) {
      const int idx = threadIdx.x + r * kVThreads;
      rb[r] = czero<T>(); rw[r] = czero<T>(); rv[r] = czero<T>();
      const int ly = idx / SW, lx = idx - ly * SW;
      const int gx = x0 - H + lx, gy = y0 - H + ly;
      if (idx < S && gx >= 0 && gx < nx && gy >= 0 && gy < ny) {
        const size_t q = (size_t)gy * nx + gx;
        if constexpr (NU >= 1) {
          rb[r] = load_rhs<T, TIn>(bin, boff + q, sc);
          rw[r] = wDinv[q];
        }
        rv[r] = vp[q];
      }
    }
#pragma unroll
    for (int r = 0; r < NC; ++r) {
      const int t = threadIdx.x + r * kVThreads;
      if (t < CS) se[t] = re[r];
    }
#pragma unroll
    for (int r = 0; r < NL; ++r) {
      const int idx = threadIdx.x + r * kVThreads;
      if (idx < S) { sb[idx] = rb[r]; sw[idx] = rw[r]; vb[idx] = rv[r]; }
    }
  }
  __syncthreads();

  // v = v_pre + P e on every in-grid point of the tile (bilinear weights per fine parity)
  for (int idx = threadIdx.x; idx < S; idx += kVThreads) {
    const int ly = idx / SW, lx = idx - ly * SW;
    const int gx = x0 - H + lx, gy = y0 - H + ly;
    Cx<T> v = czero<T>();
    if (gx >= 0 && gx < nx && gy >= 0 && gy < ny) {
      const int ia = (gx >> 1) - cx0, ja = (gy >> 1) - cy0;
      Cx<T> p;
      const bool ox = gx & 1, oy = gy & 1;
      if (!ox && !oy) {
        p = se[ja * CW + ia];
      } else if (ox && !oy) {
        const Cx<T> s = se[ja * CW + ia] + se[ja * CW + ia + 1];
        p = T(0.5) * s;
      } else if (!ox && oy) {
        const Cx<T> s = se[ja * CW + ia] + se[(ja + 1) * CW + ia];
        p = T(0.5) * s;
      } else {
        const Cx<T> s = se[ja * CW + ia] + se[ja * CW + ia + 1] + se[(ja + 1) * CW + ia] + se[(ja + 1) * CW + ia + 1];
        p = T(0.25) * s;
      }
      v = vb[idx] + p;
    }
    va[idx] = v;
  }
  __syncthreads();

  Cx<T>* vcur = va;
  Cx<T>* vnxt = vb;
#pragma unroll
  for (int s = 1; s <= NU; ++s) {
    const int lo = s, W = SW - 2 * lo, Hh = SH - 2 * lo;
    for (int t = threadIdx.x; t < W * Hh; t += kVThreads) {
      const int ly = lo + t / W, lx = lo + t % W;
      const int idx = ly * SW + lx;
      vnxt[idx] = jacobi_point(vcur, idx, SW, sb[idx], sw[idx], inv_h2, om1);
    }
    __syncthreads();
    Cx<T>* tmp = vcur; vcur = vnxt; vnxt = tmp;
  }

  Cx<TOut>* o = out + rhs * out_stride;
  for (int t = threadIdx.x; t < TX * TY; t += kVThreads) {
    const int gx = x0 + t % TX, gy = y0 + t / TX;
    if (gx < nx && gy < ny) o[(size_t)gy * nx + gx] = ccast<TOut>(vcur[(H + t / TX) * SW + H + t % TX]);
  }
}

// ---------------------------------------------------------------- streaming FP32 level kernels
// Persistent variants of k_pre / k_post for FP32 levels (inputs already FP32): each block walks
// tiles blockIdx.x, blockIdx.x + gridDim.x, ... (RHS-major, then y, then x) and copies the next
// tile's inputs into the other half of a double buffer with cp.async (zero-filled outside the
// grid) while it computes the current tile, so the tile loads no longer stall the block.

__device__ __forceinline__ void cp_async8(void* dst, const void* src, bool valid) {
  const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(valid ? 8u : 0u) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

struct TileWalk {
  int ntx, nty, per_rhs, total;
  const RhsState* st;
  __device__ __forceinline__ int next(int t, int step) const {
    while (t < total && st && !st[t / per_rhs].active) t += step;
    return t;
  }
};

template <int NU, int TX, int TY>
__global__ void __launch_bounds__(kVThreads)
k_pre_s(const cf* __restrict__ bin, size_t b_stride, const double* __restrict__ bscale, size_t scale_stride,
        const cf* __restrict__ D, const cf* __restrict__ wDinv, cf* __restrict__ vpre, size_t v_stride,
        cf* __restrict__ bc, size_t bc_stride, int nx, int ny, int nxc, int nyc, float inv_h2, float om1,
        TileWalk tw) {
  constexpr int H = NU + 1;
  constexpr int SW = TX + 2 * H, SH = TY + 2 * H, S = SW * SH;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  cf* in = reinterpret_cast<cf*>(smem_raw);          // [2][3][S]: b, w/D, D
  cf* va = in + 6 * S;
  cf* vb = va + S;
  const int step = gridDim.x;

  auto issue = [&](int t, int buf) {
    const int rhs = t / tw.per_rhs, r = t - rhs * tw.per_rhs;
    const int y0 = (r / tw.ntx) * TY, x0 = (r % tw.ntx) * TX;
    const cf* bb = bin + rhs * b_stride;
    cf* sb = in + (2 * buf * 3 + 0) * S;
    for (int idx = threadIdx.x; idx < S; idx += kVThreads) {
      const int ly = idx / SW, lx = idx - ly * SW;
      const int gx = x0 - H + lx, gy = y0 - H + ly;
      const bool ok = gx >= 0 && gx < nx && gy >= 0 && gy < ny;
      const size_t q = ok ? (size_t)gy * nx + gx : 0;
      cp_async8(sb + idx, bb + q, ok);
      cp_async8(sb + S + idx, wDinv + q, ok);
      cp_async8(sb + 2 * S + idx, D + q, ok);
    }
  };
  int t = tw.next(blockIdx.x, step);
  if (t < tw.total) issue(t, 0);
  cp_async_commit();
  int buf = 0;
  while (t < tw.total) {
    const int tn = tw.next(t + step, step);
    if (tn < tw.total) issue(tn, buf ^ 1);
    cp_async_commit();
    cp_async_wait1();
    __syncthreads();
    const cf* sb = in + (2 * buf * 3 + 0) * S;
    const cf* sw = sb + S;
    const cf* sd = sb + 2 * S;
    const int rhs = t / tw.per_rhs, r = t - rhs * tw.per_rhs;
    const int y0 = (r / tw.ntx) * TY, x0 = (r % tw.ntx) * TX;
    const float sc = bscale ? (float)bscale[rhs * scale_stride] : 1.f;
    cf* vcur = va;
    cf* vnxt = vb;
    if constexpr (NU >= 1) {
      for (int idx = threadIdx.x; idx < S; idx += kVThreads) va[idx] = sw[idx] * (sc * sb[idx]);   // first sweep from 0
      __syncthreads();
    }
#pragma unroll
    for (int sw_i = 2; sw_i <= NU; ++sw_i) {
      const int lo = sw_i - 1, W = SW - 2 * lo, Hh = SH - 2 * lo;
      for (int u = threadIdx.x; u < W * Hh; u += kVThreads) {
        const int ly = lo + u / W, lx = lo + u % W;
        const int idx = ly * SW + lx;
        vnxt[idx] = jacobi_point(vcur, idx, SW, sc * sb[idx], sw[idx], inv_h2, om1);
      }
      __syncthreads();
      cf* tmp = vcur; vcur = vnxt; vnxt = tmp;
    }
    cf* rr = vnxt;
    {
      constexpr int W = TX + 1, Hh = TY + 1;
      for (int u = threadIdx.x; u < W * Hh; u += kVThreads) {
        const int ly = NU + u / W, lx = NU + u % W;
        const int idx = ly * SW + lx;
        const int gx = x0 - H + lx, gy = y0 - H + ly;
        cf rv = czero<float>();
        if (gx >= 0 && gx < nx && gy >= 0 && gy < ny) {
          if constexpr (NU >= 1) {
            const cf s4 = vcur[idx - 1] + vcur[idx + 1] + vcur[idx - SW] + vcur[idx + SW];
            const cf kv = sd[idx] * vcur[idx] - inv_h2 * s4;
            rv = sc * sb[idx] - kv;
          } else {
            rv = sc * sb[idx];
          }
        }
        rr[idx] = rv;
      }
    }
    __syncthreads();
    {
      constexpr int CW = TX / 2, CH = TY / 2;
      const int ci0 = x0 / 2, cj0 = y0 / 2;
      cf* bco = bc + rhs * bc_stride;
      for (int u = threadIdx.x; u < CW * CH; u += kVThreads) {
        const int ci = ci0 + u % CW, cj = cj0 + u / CW;
        if (ci >= nxc || cj >= nyc) continue;
        const int idx = (2 * cj - y0 + H) * SW + 2 * ci - x0 + H;
        const cf e = rr[idx - 1] + rr[idx + 1] + rr[idx - SW] + rr[idx + SW];
        const cf c = rr[idx - SW - 1] + rr[idx - SW + 1] + rr[idx + SW - 1] + rr[idx + SW + 1];
        bco[(size_t)cj * nxc + ci] = mk<float>(0.0625f * (4.f * rr[idx].re + 2.f * e.re + c.re),
                                               0.0625f * (4.f * rr[idx].im + 2.f * e.im + c.im));
      }
      cf* vo = vpre + rhs * v_stride;
      for (int u = threadIdx.x; u < TX * TY; u += kVThreads) {
        const int gx = x0 + u % TX, gy = y0 + u / TX;
        if (gx < nx && gy < ny) {
          cf v = czero<float>();
          if constexpr (NU >= 1) v = vcur[(H + u / TX) * SW + H + u % TX];
          vo[(size_t)gy * nx + gx] = v;
        }
      }
    }
    __syncthreads();
    t = tn;
    buf ^= 1;
  }
}

template <int NU, int TX, int TY>
__global__ void __launch_bounds__(kVThreads)
k_post_s(const cf* __restrict__ bin, size_t b_stride, const double* __restrict__ bscale, size_t scale_stride,
         const cf* __restrict__ wDinv, const cf* __restrict__ vpre, size_t v_stride, const cf* __restrict__ ec,
         size_t ec_stride, int nxc, int nyc, cf* __restrict__ out, size_t out_stride, int nx, int ny,
         float inv_h2, float om1, TileWalk tw) {
  constexpr int H = NU;
  constexpr int SW = TX + 2 * H, SH = TY + 2 * H, S = SW * SH;
  constexpr int CW = TX / 2 + H + 2, CH = TY / 2 + H + 2, CS = CW * CH;
  constexpr int STAGE = 3 * S + CS;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  cf* in = reinterpret_cast<cf*>(smem_raw);          // [2][STAGE]: v_pre, b, w/D, coarse e
  cf* va = in + 2 * STAGE;
  cf* vb = va + S;
  const int step = gridDim.x;

  auto issue = [&](int t, int buf) {
    const int rhs = t / tw.per_rhs, r = t - rhs * tw.per_rhs;
    const int y0 = (r / tw.ntx) * TY, x0 = (r % tw.ntx) * TX;
    const int cx0 = floor_half(x0 - H - 1), cy0 = floor_half(y0 - H - 1);
    cf* base = in + buf * STAGE;
    const cf* vp = vpre + rhs * v_stride;
    const cf* bb = bin + rhs * b_stride;
    for (int idx = threadIdx.x; idx < S; idx += kVThreads) {
      const int ly = idx / SW, lx = idx - ly * SW;
      const int gx = x0 - H + lx, gy = y0 - H + ly;
      const bool ok = gx >= 0 && gx < nx && gy >= 0 && gy < ny;
      const size_t q = ok ? (size_t)gy * nx + gx : 0;
      cp_async8(base + idx, vp + q, ok);
      if constexpr (NU >= 1) {
        cp_async8(base + S + idx, bb + q, ok);
        cp_async8(base + 2 * S + idx, wDinv + q, ok);
      }
    }
    const cf* eco = ec + rhs * ec_stride;
    for (int u = threadIdx.x; u < CS; u += kVThreads) {
      const int cj = cy0 + u / CW, ci = cx0 + u % CW;
      const bool ok = ci >= 0 && ci < nxc && cj >= 0 && cj < nyc;
      cp_async8(base + 3 * S + u, eco + (ok ? (size_t)cj * nxc + ci : 0), ok);
    }
  };
  int t = tw.next(blockIdx.x, step);
  if (t < tw.total) issue(t, 0);
  cp_async_commit();
  int buf = 0;
  while (t < tw.total) {
    const int tn = tw.next(t + step, step);
    if (tn < tw.total) issue(tn, buf ^ 1);
    cp_async_commit();
    cp_async_wait1();
    __syncthreads();
    const cf* svp = in + buf * STAGE;
    const cf* sb = svp + S;
    const cf* sw = svp + 2 * S;
    const cf* se = svp + 3 * S;
    const int rhs = t / tw.per_rhs, r = t - rhs * tw.per_rhs;
    const int y0 = (r / tw.ntx) * TY, x0 = (r % tw.ntx) * TX;
    const int cx0 = floor_half(x0 - H - 1), cy0 = floor_half(y0 - H - 1);
    const float sc = bscale ? (float)bscale[rhs * scale_stride] : 1.f;
    // v = v_pre + P e
    for (int idx = threadIdx.x; idx < S; idx += kVThreads) {
      const int ly = idx / SW, lx = idx - ly * SW;
      const int gx = x0 - H + lx, gy = y0 - H + ly;
      cf v = czero<float>();
      if (gx >= 0 && gx < nx && gy >= 0 && gy < ny) {
        const int ia = (gx >> 1) - cx0, ja = (gy >> 1) - cy0;
        const bool ox = gx & 1, oy = gy & 1;
        cf p;
        if (!ox && !oy) p = se[ja * CW + ia];
        else if (ox && !oy) p = 0.5f * (se[ja * CW + ia] + se[ja * CW + ia + 1]);
        else if (!ox && oy) p = 0.5f * (se[ja * CW + ia] + se[(ja + 1) * CW + ia]);
        else p = 0.25f * (se[ja * CW + ia] + se[ja * CW + ia + 1] + se[(ja + 1) * CW + ia] + se[(ja + 1) * CW + ia + 1]);
        v = svp[idx] + p;
      }
      va[idx] = v;
    }
    __syncthreads();
    cf* vcur = va;
    cf* vnxt = vb;
#pragma unroll
    for (int s_i = 1; s_i <= NU; ++s_i) {
      const int lo = s_i, W = SW - 2 * lo, Hh = SH - 2 * lo;
      for (int u = threadIdx.x; u < W * Hh; u += kVThreads) {
        const int ly = lo + u / W, lx = lo + u % W;
        const int idx = ly * SW + lx;
        vnxt[idx] = jacobi_point(vcur, idx, SW, sc * sb[idx], sw[idx], inv_h2, om1);
      }
      __syncthreads();
      cf* tmp = vcur; vcur = vnxt; vnxt = tmp;
    }
    cf* o = out + rhs * out_stride;
    for (int u = threadIdx.x; u < TX * TY; u += kVThreads) {
      const int gx = x0 + u % TX, gy = y0 + u / TX;
      if (gx < nx && gy < ny) o[(size_t)gy * nx + gx] = vcur[(H + u / TX) * SW + H + u % TX];
    }
    __syncthreads();
    t = tn;
    buf ^= 1;
  }
}

// ---------------------------------------------------------------- TMA tensor-tile level kernels
// The same persistent double-buffered scheme with the tile inputs fetched by the tensor-memory
// accelerator: one thread issues a 2-D or 3-D tensor copy per input array and stage, points
// outside the grid arrive as zeros, and the copies complete on an mbarrier per stage.  A box
// must start at an even x (8-byte elements, 16-byte rule), so the x halo is rounded up to an
// even width.  Used for FP32 levels of even width; odd widths use the cp.async kernels.

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

// Shared arrays start on 128-byte boundaries (16 complex FP32 values).
__host__ __device__ constexpr int pad16(int n) { return (n + 15) & ~15; }

template <int NU, int TX, int TY>
struct PreGeom {
  static constexpr int H = NU + 1, HX = (H + 1) & ~1;
  static constexpr int SW = TX + 2 * HX, SH = TY + 2 * H, S = SW * SH, SP = pad16(S);
  static constexpr size_t smem() { return 128 + sizeof(cf) * (2 * 3 * SP + 2 * SP); }
};

template <int NU, int TX, int TY, int NT>
__global__ void __launch_bounds__(NT)
k_pre_t(const __grid_constant__ CUtensorMap tm_b, const __grid_constant__ CUtensorMap tm_w,
        const __grid_constant__ CUtensorMap tm_d, const double* __restrict__ bscale, size_t scale_stride,
        cf* __restrict__ vpre, size_t v_stride, cf* __restrict__ bc, size_t bc_stride, int nx, int ny, int nxc,
        int nyc, float inv_h2, float om1, TileWalk tw, int* __restrict__ err) {
  using G = PreGeom<NU, TX, TY>;
  constexpr int H = G::H, HX = G::HX, SW = G::SW, SH = G::SH, S = G::S, SP = G::SP;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  __shared__ int fail;
  cf* in = reinterpret_cast<cf*>(smem_raw + 128);  // [2][3][SP]: b, w/D, D
  cf* va = in + 6 * SP;
  cf* vb = va + SP;
  const int step = gridDim.x;
  constexpr uint32_t kBytes = 3u * S * sizeof(cf);
  auto issue = [&](int t, int buf) {
    const int rhs = t / tw.per_rhs, r = t - rhs * tw.per_rhs;
    const int y0 = (r / tw.ntx) * TY, x0 = (r % tw.ntx) * TX;
    cf* base = in + buf * 3 * SP;
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(&bar[buf], kBytes);
    tma_load_3d(base, &tm_b, x0 - HX, y0 - H, rhs, &bar[buf]);
    tma_load_2d(base + SP, &tm_w, x0 - HX, y0 - H, &bar[buf]);
    tma_load_2d(base + 2 * SP, &tm_d, x0 - HX, y0 - H, &bar[buf]);
  };
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
    fail = 0;
  }
  __syncthreads();
  int t = tw.next(blockIdx.x, step);
  if (threadIdx.x == 0 && t < tw.total) issue(t, 0);
  int buf = 0, k = 0;
  uint32_t phase[2] = {0u, 0u};
  while (t < tw.total) {
    const int tn = tw.next(t + step, step);
    if (threadIdx.x == 0 && tn < tw.total) issue(tn, buf ^ 1);
    if (!mbar_wait(&bar[buf], phase[buf], kWaitLimitNs)) fail = 1;
    phase[buf] ^= 1u;
    __syncthreads();
    if (fail) {
      if (threadIdx.x == 0) {
        atomicExch(err, kErrTimeout);
        if (tn < tw.total) mbar_wait(&bar[buf ^ 1], phase[buf ^ 1], kWaitLimitNs);
      }
      __syncthreads();
      return;
    }
    const cf* sb = in + buf * 3 * SP;
    const cf* sw = sb + SP;
    const cf* sd = sb + 2 * SP;
    const int rhs = t / tw.per_rhs, r = t - rhs * tw.per_rhs;
    const int y0 = (r / tw.ntx) * TY, x0 = (r % tw.ntx) * TX;
    const float sc = bscale ? (float)bscale[rhs * scale_stride] : 1.f;
    cf* vcur = va;
    cf* vnxt = vb;
    if constexpr (NU >= 1) {
      for (int idx = threadIdx.x; idx < S; idx += NT) va[idx] = sw[idx] * (sc * sb[idx]);
      __syncthreads();
    }
#pragma unroll
    for (int s_i = 2; s_i <= NU; ++s_i) {
      const int lo = s_i - 1, W = SW - 2 * lo, Hh = SH - 2 * lo;
      for (int u = threadIdx.x; u < W * Hh; u += NT) {
        const int ly = lo + u / W, lx = lo + u % W;
        const int idx = ly * SW + lx;
        vnxt[idx] = jacobi_point(vcur, idx, SW, sc * sb[idx], sw[idx], inv_h2, om1);
      }
      __syncthreads();
      cf* tmp = vcur; vcur = vnxt; vnxt = tmp;
    }
    cf* rr = vnxt;
    {
      constexpr int W = TX + 1, Hh = TY + 1;
      for (int u = threadIdx.x; u < W * Hh; u += NT) {
        const int ly = H - 1 + u / W, lx = HX - 1 + u % W;
        const int idx = ly * SW + lx;
        const int gx = x0 - HX + lx, gy = y0 - H + ly;
        cf rv = czero<float>();
        if (gx >= 0 && gx < nx && gy >= 0 && gy < ny) {
          if constexpr (NU >= 1) {
            const cf s4 = vcur[idx - 1] + vcur[idx + 1] + vcur[idx - SW] + vcur[idx + SW];
            const cf kv = sd[idx] * vcur[idx] - inv_h2 * s4;
            rv = sc * sb[idx] - kv;
          } else {
            rv = sc * sb[idx];
          }
        }
        rr[idx] = rv;
      }
    }
    __syncthreads();
    {
      constexpr int CW = TX / 2, CH = TY / 2;
      const int ci0 = x0 / 2, cj0 = y0 / 2;
      cf* bco = bc + rhs * bc_stride;
      for (int u = threadIdx.x; u < CW * CH; u += NT) {
        const int ci = ci0 + u % CW, cj = cj0 + u / CW;
        if (ci >= nxc || cj >= nyc) continue;
        const int idx = (2 * cj - y0 + H) * SW + 2 * ci - x0 + HX;
        const cf e = rr[idx - 1] + rr[idx + 1] + rr[idx - SW] + rr[idx + SW];
        const cf c = rr[idx - SW - 1] + rr[idx - SW + 1] + rr[idx + SW - 1] + rr[idx + SW + 1];
        bco[(size_t)cj * nxc + ci] = mk<float>(0.0625f * (4.f * rr[idx].re + 2.f * e.re + c.re),
                                               0.0625f * (4.f * rr[idx].im + 2.f * e.im + c.im));
      }
      cf* vo = vpre + rhs * v_stride;
      for (int u = threadIdx.x; u < TX * TY; u += NT) {
        const int gx = x0 + u % TX, gy = y0 + u / TX;
        if (gx < nx && gy < ny) {
          cf v = czero<float>();
          if constexpr (NU >= 1) v = vcur[(H + u / TX) * SW + HX + u % TX];
          vo[(size_t)gy * nx + gx] = v;
        }
      }
    }
    __syncthreads();
    t = tn;
    buf ^= 1;
    ++k;
  }
}

template <int NU, int TX, int TY>
struct PostGeom {
  static constexpr int H = NU, HX = (NU + 1) & ~1;
  static constexpr int SW = TX + 2 * HX, SH = TY + 2 * H, S = SW * SH, SP = pad16(S);
  static constexpr int CW = ((TX / 2 + HX + 3) + 1) & ~1, CH = TY / 2 + H + 2, CS = CW * CH, CSP = pad16(CS);
  static constexpr int STAGE = 3 * SP + CSP;
  static constexpr size_t smem() { return 128 + sizeof(cf) * (2 * STAGE + 2 * SP); }
};

template <int NU, int TX, int TY, int NT>
__global__ void __launch_bounds__(NT)
k_post_t(const __grid_constant__ CUtensorMap tm_v, const __grid_constant__ CUtensorMap tm_b,
         const __grid_constant__ CUtensorMap tm_w, const __grid_constant__ CUtensorMap tm_e,
         const double* __restrict__ bscale, size_t scale_stride, cf* __restrict__ out, size_t out_stride, int nx,
         int ny, float inv_h2, float om1, TileWalk tw, int* __restrict__ err) {
  using G = PostGeom<NU, TX, TY>;
  constexpr int H = G::H, HX = G::HX, SW = G::SW, SH = G::SH, S = G::S, SP = G::SP, CW = G::CW, CS = G::CS,
                STAGE = G::STAGE;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  __shared__ int fail;
  cf* in = reinterpret_cast<cf*>(smem_raw + 128);  // [2][STAGE]: v_pre, b, w/D, coarse e
  cf* va = in + 2 * STAGE;
  cf* vb = va + SP;
  const int step = gridDim.x;
  constexpr uint32_t kBytes = (uint32_t)((NU >= 1 ? 3 * S : S) + CS) * sizeof(cf);
  auto coarse_origin = [&](int x0, int y0, int& cx0, int& cy0) {
    cx0 = floor_half(x0 - H - 1);
    cx0 -= (cx0 & 1);            // even start for the 16-byte rule
    cy0 = floor_half(y0 - H - 1);
  };
  auto issue = [&](int t, int buf) {
    const int rhs = t / tw.per_rhs, r = t - rhs * tw.per_rhs;
    const int y0 = (r / tw.ntx) * TY, x0 = (r % tw.ntx) * TX;
    int cx0, cy0;
    coarse_origin(x0, y0, cx0, cy0);
    cf* base = in + buf * STAGE;
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(&bar[buf], kBytes);
    tma_load_3d(base, &tm_v, x0 - HX, y0 - H, rhs, &bar[buf]);
    if constexpr (NU >= 1) {
      tma_load_3d(base + SP, &tm_b, x0 - HX, y0 - H, rhs, &bar[buf]);
      tma_load_2d(base + 2 * SP, &tm_w, x0 - HX, y0 - H, &bar[buf]);
    }
    tma_load_3d(base + 3 * SP, &tm_e, cx0, cy0, rhs, &bar[buf]);
  };
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
    fail = 0;
  }
  __syncthreads();
  int t = tw.next(blockIdx.x, step);
  if (threadIdx.x == 0 && t < tw.total) issue(t, 0);
  int buf = 0;
  uint32_t phase[2] = {0u, 0u};
  while (t < tw.total) {
    const int tn = tw.next(t + step, step);
    if (threadIdx.x == 0 && tn < tw.total) issue(tn, buf ^ 1);
    if (!mbar_wait(&bar[buf], phase[buf], kWaitLimitNs)) fail = 1;
    phase[buf] ^= 1u;
    __syncthreads();
    if (fail) {
      if (threadIdx.x == 0) {
        atomicExch(err, kErrTimeout);
        if (tn < tw.total) mbar_wait(&bar[buf ^ 1], phase[buf ^ 1], kWaitLimitNs);
      }
      __syncthreads();
      return;
    }
    const cf* svp = in + buf * STAGE;
    const cf* sb = svp + SP;
    const cf* sw = svp + 2 * SP;
    const cf* se = svp + 3 * SP;
    const int rhs = t / tw.per_rhs, r = t - rhs * tw.per_rhs;
    const int y0 = (r / tw.ntx) * TY, x0 = (r % tw.ntx) * TX;
    int cx0, cy0;
    coarse_origin(x0, y0, cx0, cy0);
    const float sc = bscale ? (float)bscale[rhs * scale_stride] : 1.f;
    for (int idx = threadIdx.x; idx < S; idx += NT) {
      const int ly = idx / SW, lx = idx - ly * SW;
      const int gx = x0 - HX + lx, gy = y0 - H + ly;
      cf v = czero<float>();
      if (gx >= 0 && gx < nx && gy >= 0 && gy < ny) {
        const int ia = (gx >> 1) - cx0, ja = (gy >> 1) - cy0;
        const bool ox = gx & 1, oy = gy & 1;
        cf p;
        if (!ox && !oy) p = se[ja * CW + ia];
        else if (ox && !oy) p = 0.5f * (se[ja * CW + ia] + se[ja * CW + ia + 1]);
        else if (!ox && oy) p = 0.5f * (se[ja * CW + ia] + se[(ja + 1) * CW + ia]);
        else p = 0.25f * (se[ja * CW + ia] + se[ja * CW + ia + 1] + se[(ja + 1) * CW + ia] + se[(ja + 1) * CW + ia + 1]);
        v = svp[idx] + p;
      }
      va[idx] = v;
    }
    __syncthreads();
    cf* vcur = va;
    cf* vnxt = vb;
#pragma unroll
    for (int s_i = 1; s_i <= NU; ++s_i) {
      const int lo = s_i, W = SW - 2 * lo, Hh = SH - 2 * lo;
      for (int u = threadIdx.x; u < W * Hh; u += NT) {
        const int ly = lo + u / W, lx = lo + u % W;
        const int idx = ly * SW + lx;
        vnxt[idx] = jacobi_point(vcur, idx, SW, sc * sb[idx], sw[idx], inv_h2, om1);
      }
      __syncthreads();
      cf* tmp = vcur; vcur = vnxt; vnxt = tmp;
    }
    cf* o = out + rhs * out_stride;
    for (int u = threadIdx.x; u < TX * TY; u += NT) {
      const int gx = x0 + u % TX, gy = y0 + u / TX;
      if (gx < nx && gy < ny) o[(size_t)gy * nx + gx] = vcur[(H + u / TX) * SW + HX + u % TX];
    }
    __syncthreads();
    t = tn;
    buf ^= 1;
  }
}

template <int NU>
size_t pre_s_smem() {
  constexpr int H = NU + 1, SW = 64 + 2 * H, SH = 16 + 2 * H;
  return sizeof(cf) * 8 * SW * SH;
}
template <int NU>
size_t post_s_smem() {
  constexpr int H = NU, SW = 64 + 2 * H, SH = 16 + 2 * H;
  constexpr int CW = 32 + H + 2, CH = 8 + H + 2;
  return sizeof(cf) * (2 * (3 * SW * SH + CW * CH) + 2 * SW * SH);
}

template <typename T> struct Tile;
template <> struct Tile<float> { static constexpr int X = 64, Y = 16; };
template <> struct Tile<double> { static constexpr int X = 32, Y = 16; };

template <typename T, int NU>
size_t pre_smem() {
  constexpr int H = NU + 1, SW = Tile<T>::X + 2 * H, SH = Tile<T>::Y + 2 * H;
  return 5 * sizeof(Cx<T>) * SW * SH;
}
template <typename T, int NU>
size_t post_smem() {
  constexpr int H = NU, SW = Tile<T>::X + 2 * H, SH = Tile<T>::Y + 2 * H;
  constexpr int CW = Tile<T>::X / 2 + H + 2, CH = Tile<T>::Y / 2 + H + 2;
  return sizeof(Cx<T>) * (4 * SW * SH + CW * CH);
}

// Persistent grid size of a streaming kernel: resident blocks per SM times SMs, at most `tiles`.
template <typename K>
int persistent_blocks(Handle& h, K kern, size_t smem, int tiles, int threads = kVThreads) {
  int per_sm = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  const int n = per_sm * h.num_sms;
  return n < tiles ? n : tiles;
}

// ---------------------------------------------------------------- wavefront level kernels (host side)
bool a16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }
bool a8(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 7) == 0; }

// Rows per warp segment.  All warps of a launch run the same number of steps K (rows + halo
// rows, rounded up to the unroll period P), so a launch takes about K times the number of
// waves of resident warps; the even segment length from 4 to 128 with the least
// K * ceil(warps / resident) is taken (long segments repeat fewer halo rows, short ones fill
// the GPU on small levels).
int wave_seg(const Handle& h, int l, int ny, int nstrips, int B, int extra, int P, long resident) {
  const int fixed = h.wave_seg_level[l] > 0 ? h.wave_seg_level[l] : h.wave_seg;
  if (fixed > 0) {
    const int seg = (fixed + 1) & ~1;
    for (int s = seg; s >= 4; s -= 2)
      if ((P - (s + extra) % P) % P <= 1) return s;
    return seg;
  }
  if (resident < 1) resident = 1;
  long best = -1;
  int bs = 4;
  for (int s = 4; s <= 128; s += 2) {
    const long K = (s + extra + P - 1) / P * P;
    const long warps = (long)nstrips * ((ny + s - 1) / s) * B;
    const long t = K * ((warps + resident - 1) / resident);
    if (best < 0 || t < best) { best = t; bs = s; }
    if ((ny + s - 1) / s == 1) break;   // one segment covers the level
  }
  return bs;
}

// Warps of a wavefront kernel resident on the whole GPU (occupancy of the default variant).
template <typename K>
long resident_warps(const Handle& h, K kern, int threads, size_t smem) {
  int blocks = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kern, threads, smem) != cudaSuccess || blocks < 1)
    return -1;
  return (long)blocks * (threads / 32) * h.num_sms;
}

// resident_warps cached per device (the figure depends on the device's SM count and limits); a
// failed occupancy query is not cached and counts as one block per SM.
template <typename K>
long resident_cached(std::atomic<long>* cache, const Handle& h, K kern, int threads, size_t smem) {
  const bool slot = h.device >= 0 && h.device < 64;
  long v = slot ? cache[h.device].load(std::memory_order_acquire) : 0;
  if (v > 0) return v;
  v = resident_warps(h, kern, threads, smem);
  if (v <= 0) return (long)(threads / 32) * h.num_sms;
  if (slot) cache[h.device].store(v, std::memory_order_release);
  return v;
}

bool use_wave(const Handle& h, int l) { return h.vc_wave && h.lev[l].nx >= h.wave_min_nx; }

template <int NU, bool V4, int PF, int NW>
void pre_wave_go(Handle& h, int l, const cf* bin, size_t b_stride, const double* bscale, size_t scale_stride, int B,
                 const RhsState* st, int nstrips, int nwarps, int seg) {
  const Level& lv = h.lev[l];
  const Level& cl = h.lev[l + 1];
  const dim3 grid((nwarps + NW - 1) / NW, 1, B);
  wave::k_pre_w<NU, V4, PF, NW><<<grid, 32 * NW, 0, h.stream>>>(
      bin, b_stride, bscale, scale_stride, (const cf*)lv.D, (const cf*)lv.wDinv, (cf*)lv.vpre, lv.n(), (cf*)cl.b,
      cl.n(), lv.nx, lv.ny, cl.nx, (float)(1.0 / (lv.h * lv.h)), (float)(1.0 - h.p.omega), nstrips, nwarps, seg, st);
}

template <int NU, bool V4, int PF, int NW>
void post_wave_go(Handle& h, int l, const cf* bin, size_t b_stride, const double* bscale, size_t scale_stride,
                  cf* out, size_t out_stride, int B, const RhsState* st, int nstrips, int nwarps, int seg) {
  const Level& lv = h.lev[l];
  const Level& cl = h.lev[l + 1];
  const dim3 grid((nwarps + NW - 1) / NW, 1, B);
  wave::k_post_w<NU, V4, PF, NW><<<grid, 32 * NW, 0, h.stream>>>(
      bin, b_stride, bscale, scale_stride, (const cf*)lv.wDinv, (const cf*)lv.vpre, lv.n(), (const cf*)cl.vfin,
      cl.n(), cl.nx, cl.ny, out, out_stride, lv.nx, lv.ny, (float)(1.0 / (lv.h * lv.h)), (float)(1.0 - h.p.omega),
      nstrips, nwarps, seg, st);
}

template <int NU, int NW, int MS>
mgh_status pre_ring_go(Handle& h, int l, const cf* bin, size_t b_stride, const double* bscale, size_t scale_stride,
                       int B, const RhsState* st, int nstrips, int nwarps, int seg) {
  const Level& lv = h.lev[l];
  const Level& cl = h.lev[l + 1];
  auto kern = wave::k_pre_wt<NU, NW, MS>;
  constexpr int S = wave::RingLen<wave::PreW<NU, 1>::P, NU, MS>::S;
  constexpr size_t smem = wave::RingSmem<NW, S>::bytes();
  MGH_ONCE(MGH_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)););
  const dim3 grid((nwarps + NW - 1) / NW, 1, B);
  kern<<<grid, 32 * NW, smem, h.stream>>>(bin, b_stride, bscale, scale_stride, (const cf*)lv.D, (const cf*)lv.wDinv,
                                          (cf*)lv.vpre, lv.n(), (cf*)cl.b, cl.n(), lv.nx, lv.ny, cl.nx,
                                          (float)(1.0 / (lv.h * lv.h)), (float)(1.0 - h.p.omega), nstrips, nwarps,
                                          seg, st, h.dev_err);
  return MGH_OK;
}

template <int NU, int NW, int MS>
mgh_status post_ring_go(Handle& h, int l, const cf* bin, size_t b_stride, const double* bscale,
                        size_t scale_stride, cf* out, size_t out_stride, int B, const RhsState* st, int nstrips,
                        int nwarps, int seg) {
  const Level& lv = h.lev[l];
  const Level& cl = h.lev[l + 1];
  auto kern = wave::k_post_wt<NU, NW, MS>;
  constexpr int S = wave::RingLen<wave::PostW<NU, 1>::P, NU, MS>::S;
  constexpr size_t smem = wave::RingSmem<NW, S>::bytes();
  MGH_ONCE(MGH_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)););
  const dim3 grid((nwarps + NW - 1) / NW, 1, B);
  kern<<<grid, 32 * NW, smem, h.stream>>>(bin, b_stride, bscale, scale_stride, (const cf*)lv.wDinv,
                                          (const cf*)lv.vpre, lv.n(), (const cf*)cl.vfin, cl.n(), cl.nx, cl.ny, out,
                                          out_stride, lv.nx, lv.ny, (float)(1.0 / (lv.h * lv.h)),
                                          (float)(1.0 - h.p.omega), nstrips, nwarps, seg, st, h.dev_err);
  return MGH_OK;
}

// VT / OT: storage of the level's v_pre and of the result; FP16 only on level 0 of an
// MGH_PREC_MIXED16 handle, whose cycle input is scaled by h.zmul (an exact power of two).
template <int NU, int NW, int MS, typename VT = cf>
mgh_status pre_lane_go(Handle& h, int l, const cf* bin, size_t b_stride, const double* bscale, size_t scale_stride,
                       int B, const RhsState* st, int nstrips, int nwarps, int seg) {
  const Level& lv = h.lev[l];
  const Level& cl = h.lev[l + 1];
  auto kern = wave::k_pre_wa<NU, NW, MS, VT>;
  constexpr int S = wave::RingLen<wave::PreW<NU, 1>::P, NU, MS>::S;
  constexpr size_t smem = wave::LaneRingSmem<NW, S>::bytes();
  MGH_ONCE(MGH_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)););
  const dim3 grid((nwarps + NW - 1) / NW, 1, B);
  const float smul = std::is_same<VT, cf>::value ? 1.f : h.zmul;
  kern<<<grid, 32 * NW, smem, h.stream>>>(bin, b_stride, bscale, scale_stride, (const cf*)lv.D, (const cf*)lv.wDinv,
                                          (VT*)lv.vpre, lv.n(), (cf*)cl.b, cl.n(), lv.nx, lv.ny, cl.nx,
                                          (float)(1.0 / (lv.h * lv.h)), (float)(1.0 - h.p.omega), nstrips, nwarps,
                                          seg, st, smul);
  return MGH_OK;
}

template <int NU, int NW, int MS, typename VT = cf>
mgh_status post_lane_go(Handle& h, int l, const cf* bin, size_t b_stride, const double* bscale,
                        size_t scale_stride, cf* out, size_t out_stride, int B, const RhsState* st, int nstrips,
                        int nwarps, int seg) {
  const Level& lv = h.lev[l];
  const Level& cl = h.lev[l + 1];
  auto kern = wave::k_post_wa<NU, NW, MS, VT, VT>;
  constexpr int S = wave::RingLen<wave::PostW<NU, 1>::P, NU, MS>::S;
  constexpr size_t smem = wave::LaneRingSmem<NW, S>::bytes();
  MGH_ONCE(MGH_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)););
  const dim3 grid((nwarps + NW - 1) / NW, 1, B);
  const float smul = std::is_same<VT, cf>::value ? 1.f : h.zmul;
  // an FP16 result goes to the FP16 slot whose address the caller passed as `out`
  kern<<<grid, 32 * NW, smem, h.stream>>>(bin, b_stride, bscale, scale_stride, (const cf*)lv.wDinv,
                                          (const VT*)lv.vpre, lv.n(), (const cf*)cl.vfin, cl.n(), cl.nx, cl.ny,
                                          reinterpret_cast<VT*>(out), out_stride, lv.nx, lv.ny,
                                          (float)(1.0 / (lv.h * lv.h)), (float)(1.0 - h.p.omega), nstrips, nwarps,
                                          seg, st, smul);
  return MGH_OK;
}

// Level-0 post kernel with the s-step operator product fused (k_post_waf): v_{k+1} = A z_k into
// h.fuse_v and per-(row, strip) norm partials into h.npart.
template <int NU, int NW, int MS, typename VT = cf>
mgh_status post_lane_fgo(Handle& h, int l, const cf* bin, size_t b_stride, const double* bscale,
                         size_t scale_stride, cf* out, size_t out_stride, int B, const RhsState* st, int nstrips,
                         int nwarps, int seg) {
  const Level& lv = h.lev[l];
  const Level& cl = h.lev[l + 1];
  auto kern = wave::k_post_waf<NU, NW, MS, VT, VT>;
  constexpr int S = wave::RingLen<wave::PostWF<NU, 1>::P, NU, MS>::S;
  constexpr size_t smem = wave::LaneRingSmem<NW, S>::bytes();
  MGH_ONCE(MGH_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)););
  const dim3 grid((nwarps + NW - 1) / NW, 1, B);
  const float smul = std::is_same<VT, cf>::value ? 1.f : h.zmul;
  const float ih = (float)(1.0 / (lv.h * lv.h));
  kern<<<grid, 32 * NW, smem, h.stream>>>(bin, b_stride, bscale, scale_stride, (const cf*)lv.wDinv,
                                          (const VT*)lv.vpre, lv.n(), (const cf*)cl.vfin, cl.n(), cl.nx, cl.ny,
                                          reinterpret_cast<VT*>(out), out_stride, lv.nx, lv.ny, ih,
                                          (float)(1.0 - h.p.omega), nstrips, nwarps, seg, st, smul,
                                          reinterpret_cast<const cf*>(h.DAdf), ih, h.fuse_v, h.fuse_vstride,
                                          h.npart);
  return MGH_OK;
}

// Ring variants: ring length multiplier (1 or 2 unroll periods) and warps per block.
#define MGH_RING_DISPATCH(GO, NU, MS, NW, ...)                                                   \
  ((MS) >= 2 ? ((NW) == 2 ? GO<NU, 2, 2>(__VA_ARGS__) : GO<NU, 4, 2>(__VA_ARGS__))            \
             : ((NW) == 2 ? GO<NU, 2, 1>(__VA_ARGS__) : GO<NU, 4, 1>(__VA_ARGS__)))

// Variant dispatch: 16-byte vector accesses or not, prefetch depth 1 or 2, 2 or 4 warps per block.
#define MGH_WAVE_DISPATCH(GO, NU, V4, PF, NW, ...)                         \
  do {                                                                     \
    if (V4) {                                                              \
      if (PF == 2) {                                                       \
        if (NW == 2) GO<NU, true, 2, 2>(__VA_ARGS__); else GO<NU, true, 2, 4>(__VA_ARGS__);    \
      } else {                                                             \
        if (NW == 2) GO<NU, true, 1, 2>(__VA_ARGS__); else GO<NU, true, 1, 4>(__VA_ARGS__);    \
      }                                                                    \
    } else {                                                               \
      if (NW == 2) GO<NU, false, 1, 2>(__VA_ARGS__); else GO<NU, false, 1, 4>(__VA_ARGS__);    \
    }                                                                      \
  } while (0)

template <int NU>
mgh_status launch_pre_wave(Handle& h, int l, const cf* bin, size_t b_stride, const double* bscale,
                           size_t scale_stride, int B, const RhsState* st) {
  const Level& lv = h.lev[l];
  using G = wave::PreW<NU, 2>;   // period of the PF = 2 variant (a multiple of the PF = 1 one)
  const bool hv = l == 0 && h.half;   // v_pre in FP16: 8-byte pairs
  const bool v4 = lv.nx % 2 == 0 && b_stride % 2 == 0 && lv.n() % 2 == 0 && a16(bin) && a16(lv.D) &&
                  a16(lv.wDinv) && (hv ? a8(lv.vpre) : a16(lv.vpre));
  const bool ring = v4 && h.wave_ring > 0;
  const int period = !ring ? G::P
                           : (h.wave_ring >= 2 ? wave::RingLen<wave::PreW<NU, 1>::P, NU, 2>::S
                                               : wave::RingLen<wave::PreW<NU, 1>::P, NU, 1>::S);
  const int nstrips = (lv.nx + G::XO - 1) / G::XO;
  constexpr int S1 = wave::RingLen<wave::PreW<NU, 1>::P, NU, 1>::S;
  constexpr size_t smem1 = wave::LaneRingSmem<4, S1>::bytes();
  MGH_ONCE(MGH_CUDA(cudaFuncSetAttribute(wave::k_pre_wa<NU, 4, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem1)););
  static std::atomic<long> resident_by_dev[64];
  const long resident = resident_cached(resident_by_dev, h, wave::k_pre_wa<NU, 4, 1>, 128, smem1);
  const int seg = wave_seg(h, l, lv.ny, nstrips, B, 2 * G::H - 1, period, resident);
  const int nwarps = nstrips * ((lv.ny + seg - 1) / seg);
  ProfScope ps(h, l == 0 ? P_PRE0 : P_COARSE);
  if (l == 0 && h.half) {   // FP16 storage: lane rings, 4 warps, one unroll period (checked at create)
    if (!ring) return MGH_NOT_SUPPORTED;
    MGH_TRY((pre_lane_go<NU, 4, 1, __half2>(h, l, bin, b_stride, bscale, scale_stride, B, st, nstrips, nwarps, seg)));
    MGH_CHECK_LAUNCH(); h.launches++;
    return MGH_OK;
  }
  if (ring) {
    if (h.wave_lane_ring)
      MGH_TRY(MGH_RING_DISPATCH(pre_lane_go, NU, h.wave_ring, h.wave_warps, h, l, bin, b_stride, bscale,
                                scale_stride, B, st, nstrips, nwarps, seg));
    else
      MGH_TRY(MGH_RING_DISPATCH(pre_ring_go, NU, h.wave_ring, h.wave_warps, h, l, bin, b_stride, bscale,
                                scale_stride, B, st, nstrips, nwarps, seg));
    MGH_CHECK_LAUNCH(); h.launches++;
    return MGH_OK;
  }
  MGH_WAVE_DISPATCH(pre_wave_go, NU, v4, h.wave_pf, h.wave_warps, h, l, bin, b_stride, bscale, scale_stride, B, st,
                    nstrips, nwarps, seg);
  MGH_CHECK_LAUNCH(); h.launches++;
  return MGH_OK;
}

template <int NU>
mgh_status launch_post_wave(Handle& h, int l, const cf* bin, size_t b_stride, const double* bscale,
                            size_t scale_stride, cf* out, size_t out_stride, int B, const RhsState* st) {
  const Level& lv = h.lev[l];
  using G = wave::PostW<NU, 2>;
  const bool hv = l == 0 && h.half;   // v_pre and the result in FP16: 8-byte pairs
  const bool v4 = lv.nx % 2 == 0 && b_stride % 2 == 0 && out_stride % 2 == 0 && lv.n() % 2 == 0 && a16(bin) &&
                  (hv ? a8(out) && a8(lv.vpre) : a16(out) && a16(lv.vpre)) && a16(lv.wDinv);
  const bool ring = v4 && h.wave_ring > 0;
  const int period = !ring ? G::P
                           : (h.wave_ring >= 2 ? wave::RingLen<wave::PostW<NU, 1>::P, NU, 2>::S
                                               : wave::RingLen<wave::PostW<NU, 1>::P, NU, 1>::S);
  const int nstrips = (lv.nx + G::XO - 1) / G::XO;
  constexpr int S1 = wave::RingLen<wave::PostW<NU, 1>::P, NU, 1>::S;
  constexpr size_t smem1 = wave::LaneRingSmem<4, S1>::bytes();
  MGH_ONCE(MGH_CUDA(cudaFuncSetAttribute(wave::k_post_wa<NU, 4, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem1)););
  static std::atomic<long> resident_by_dev[64];
  const long resident = resident_cached(resident_by_dev, h, wave::k_post_wa<NU, 4, 1>, 128, smem1);
  if (l == 0 && h.fuse_v && h.fuse_ok && !h.half && ring && h.wave_lane_ring && a16(h.DAdf) && a16(h.fuse_v) &&
      h.fuse_vstride % 2 == 0) {
    // the s-step operator product fused in: one more halo column per side and row above and below
    // (FP32 storage only: with FP16 storage the fused kernel needs 111 registers and the product
    // in its own kernel is faster)
    using GF = wave::PostWF<NU, 1>;
    const int nstrips_f = (lv.nx + GF::XO - 1) / GF::XO;
    constexpr int SF = wave::RingLen<GF::P, NU, 1>::S;
    constexpr size_t smemf = wave::LaneRingSmem<4, SF>::bytes();
    MGH_ONCE(MGH_CUDA(cudaFuncSetAttribute(wave::k_post_waf<NU, 4, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smemf)););
    static std::atomic<long> resident_f_by_dev[64];
    const long resident_f = resident_cached(resident_f_by_dev, h, wave::k_post_waf<NU, 4, 1>, 128, smemf);
    const int periodf = h.wave_ring >= 2 ? wave::RingLen<GF::P, NU, 2>::S : SF;
    const int segf = wave_seg(h, l, lv.ny, nstrips_f, B, 2 * NU + 2, periodf, resident_f);
    const int nwarps_f = nstrips_f * ((lv.ny + segf - 1) / segf);
    ProfScope ps(h, P_POST0);
    MGH_TRY(MGH_RING_DISPATCH(post_lane_fgo, NU, h.wave_ring, h.wave_warps, h, l, bin, b_stride, bscale,
                              scale_stride, out, out_stride, B, st, nstrips_f, nwarps_f, segf));
    MGH_CHECK_LAUNCH(); h.launches++;
    h.fuse_nstrips = nstrips_f;
    return MGH_OK;
  }
  const int seg = wave_seg(h, l, lv.ny, nstrips, B, 2 * NU, period, resident);
  const int nwarps = nstrips * ((lv.ny + seg - 1) / seg);
  ProfScope ps(h, l == 0 ? P_POST0 : P_COARSE);
  if (l == 0 && h.half) {
    if (!ring) return MGH_NOT_SUPPORTED;
    MGH_TRY((post_lane_go<NU, 4, 1, __half2>(h, l, bin, b_stride, bscale, scale_stride, out, out_stride, B, st,
                                             nstrips, nwarps, seg)));
    MGH_CHECK_LAUNCH(); h.launches++;
    return MGH_OK;
  }
  if (ring) {
    if (h.wave_lane_ring)
      MGH_TRY(MGH_RING_DISPATCH(post_lane_go, NU, h.wave_ring, h.wave_warps, h, l, bin, b_stride, bscale,
                                scale_stride, out, out_stride, B, st, nstrips, nwarps, seg));
    else
      MGH_TRY(MGH_RING_DISPATCH(post_ring_go, NU, h.wave_ring, h.wave_warps, h, l, bin, b_stride, bscale,
                                scale_stride, out, out_stride, B, st, nstrips, nwarps, seg));
    MGH_CHECK_LAUNCH(); h.launches++;
    return MGH_OK;
  }
  MGH_WAVE_DISPATCH(post_wave_go, NU, v4, h.wave_pf, h.wave_warps, h, l, bin, b_stride, bscale, scale_stride, out,
                    out_stride, B, st, nstrips, nwarps, seg);
  MGH_CHECK_LAUNCH(); h.launches++;
  return MGH_OK;
}

template <typename T, int NU, typename TIn>
mgh_status launch_pre_nu(Handle& h, int l, const void* bin, size_t b_stride, const double* bscale,
                         size_t scale_stride, int B, const RhsState* st, int in_slot) {
  const Level& lv = h.lev[l];
  const Level& cl = h.lev[l + 1];
  if constexpr (std::is_same<T, float>::value && std::is_same<TIn, float>::value) {
    if constexpr (NU >= 1) {
      if (use_wave(h, l))
        return launch_pre_wave<NU>(h, l, (const cf*)bin, b_stride, bscale, scale_stride, B, st);
    }
    const bool tma = h.tma && h.tma[l].pre_ok && (l > 0 || (in_slot >= 0 && h.tma_in_ok));
    if (tma) {
      using G = PreGeom<NU, 64, 16>;
      auto kern = k_pre_t<NU, 64, 16, kVcThreadsTma>;
      MGH_ONCE(MGH_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::smem())););
      TileWalk tw;
      tw.ntx = (lv.nx + 63) / 64; tw.nty = (lv.ny + 15) / 16; tw.per_rhs = tw.ntx * tw.nty; tw.total = tw.per_rhs * B;
      tw.st = st;
      const int grid = persistent_blocks(h, kern, G::smem(), tw.total, kVcThreadsTma);
      const CUtensorMap& mb = l == 0 ? h.tma_in[in_slot] : h.tma[l].pre_b;
      ProfScope ps(h, l == 0 ? P_PRE0 : P_COARSE);
      kern<<<grid, kVcThreadsTma, G::smem(), h.stream>>>(mb, h.tma[l].pre_w, h.tma[l].pre_d, bscale, scale_stride,
                                                     (cf*)lv.vpre, lv.n(), (cf*)cl.b, cl.n(), lv.nx, lv.ny, cl.nx,
                                                     cl.ny, (float)(1.0 / (lv.h * lv.h)), (float)(1.0 - h.p.omega),
                                                     tw, h.dev_err);
      MGH_CHECK_LAUNCH(); h.launches++;
      return MGH_OK;
    }
    const size_t smem = pre_s_smem<NU>();
    auto kern = k_pre_s<NU, 64, 16>;
    MGH_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    TileWalk tw;
    tw.ntx = (lv.nx + 63) / 64; tw.nty = (lv.ny + 15) / 16; tw.per_rhs = tw.ntx * tw.nty; tw.total = tw.per_rhs * B;
    tw.st = st;
    const int grid = persistent_blocks(h, kern, smem, tw.total);
    ProfScope ps(h, l == 0 ? P_PRE0 : P_COARSE);
    kern<<<grid, kVThreads, smem, h.stream>>>((const cf*)bin, b_stride, bscale, scale_stride, (const cf*)lv.D,
                                              (const cf*)lv.wDinv, (cf*)lv.vpre, lv.n(), (cf*)cl.b, cl.n(), lv.nx,
                                              lv.ny, cl.nx, cl.ny, (float)(1.0 / (lv.h * lv.h)),
                                              (float)(1.0 - h.p.omega), tw);
    MGH_CHECK_LAUNCH(); h.launches++;
    return MGH_OK;
  }
  constexpr int TX = Tile<T>::X, TY = Tile<T>::Y;
  const size_t smem = pre_smem<T, NU>();
  auto kern = k_pre<T, NU, TX, TY, TIn>;
  MGH_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  dim3 grid((lv.nx + TX - 1) / TX, (lv.ny + TY - 1) / TY, B);
  const T ih2 = static_cast<T>(1.0 / (lv.h * lv.h));
  const T om1 = static_cast<T>(1.0 - h.p.omega);
  ProfScope ps(h, l == 0 ? P_PRE0 : P_COARSE);
  kern<<<grid, kVThreads, smem, h.stream>>>(bin, b_stride, bscale, scale_stride, (const Cx<T>*)lv.D,
                                            (const Cx<T>*)lv.wDinv, (Cx<T>*)lv.vpre, lv.n(),
                                            (Cx<T>*)cl.b, cl.n(), lv.nx, lv.ny, cl.nx, cl.ny, ih2, om1, st);
  MGH_CHECK_LAUNCH(); h.launches++;
  return MGH_OK;
}

template <typename T, int NU, typename TIn, typename TOut>
mgh_status launch_post_nu(Handle& h, int l, const void* bin, size_t b_stride, const double* bscale,
                          size_t scale_stride, Cx<TOut>* out, size_t out_stride, int B, const RhsState* st,
                          int in_slot) {
  const Level& lv = h.lev[l];
  const Level& cl = h.lev[l + 1];
  if constexpr (std::is_same<T, float>::value && std::is_same<TIn, float>::value &&
                std::is_same<TOut, float>::value) {
    if constexpr (NU >= 1) {
      if (use_wave(h, l))
        return launch_post_wave<NU>(h, l, (const cf*)bin, b_stride, bscale, scale_stride, out, out_stride, B, st);
    }
    const bool tma = h.tma && h.tma[l].post_ok && (l > 0 || (in_slot >= 0 && h.tma_in_ok));
    if (tma) {
      using G = PostGeom<NU, 64, 16>;
      auto kern = k_post_t<NU, 64, 16, kVcThreadsTma>;
      MGH_ONCE(MGH_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::smem())););
      TileWalk tw;
      tw.ntx = (lv.nx + 63) / 64; tw.nty = (lv.ny + 15) / 16; tw.per_rhs = tw.ntx * tw.nty; tw.total = tw.per_rhs * B;
      tw.st = st;
      const int grid = persistent_blocks(h, kern, G::smem(), tw.total, kVcThreadsTma);
      const CUtensorMap& mb = l == 0 ? h.tma_in[h.m + in_slot] : h.tma[l].post_b;
      ProfScope ps(h, l == 0 ? P_POST0 : P_COARSE);
      kern<<<grid, kVcThreadsTma, G::smem(), h.stream>>>(h.tma[l].post_v, mb, h.tma[l].post_w, h.tma[l].post_e, bscale,
                                                     scale_stride, (cf*)out, out_stride, lv.nx, lv.ny,
                                                     (float)(1.0 / (lv.h * lv.h)), (float)(1.0 - h.p.omega), tw,
                                                     h.dev_err);
      MGH_CHECK_LAUNCH(); h.launches++;
      return MGH_OK;
    }
    const size_t smem = post_s_smem<NU>();
    auto kern = k_post_s<NU, 64, 16>;
    MGH_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    TileWalk tw;
    tw.ntx = (lv.nx + 63) / 64; tw.nty = (lv.ny + 15) / 16; tw.per_rhs = tw.ntx * tw.nty; tw.total = tw.per_rhs * B;
    tw.st = st;
    const int grid = persistent_blocks(h, kern, smem, tw.total);
    ProfScope ps(h, l == 0 ? P_POST0 : P_COARSE);
    kern<<<grid, kVThreads, smem, h.stream>>>((const cf*)bin, b_stride, bscale, scale_stride, (const cf*)lv.wDinv,
                                              (const cf*)lv.vpre, lv.n(), (const cf*)cl.vfin, cl.n(), cl.nx, cl.ny,
                                              (cf*)out, out_stride, lv.nx, lv.ny, (float)(1.0 / (lv.h * lv.h)),
                                              (float)(1.0 - h.p.omega), tw);
    MGH_CHECK_LAUNCH(); h.launches++;
    return MGH_OK;
  }
  constexpr int TX = Tile<T>::X, TY = Tile<T>::Y;
  const size_t smem = post_smem<T, NU>();
  auto kern = k_post<T, NU, TX, TY, TIn, TOut>;
  MGH_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  dim3 grid((lv.nx + TX - 1) / TX, (lv.ny + TY - 1) / TY, B);
  const T ih2 = static_cast<T>(1.0 / (lv.h * lv.h));
  const T om1 = static_cast<T>(1.0 - h.p.omega);
  ProfScope ps(h, l == 0 ? P_POST0 : P_COARSE);
  kern<<<grid, kVThreads, smem, h.stream>>>(bin, b_stride, bscale, scale_stride, (const Cx<T>*)lv.wDinv,
                                            (const Cx<T>*)lv.vpre, lv.n(), (const Cx<T>*)cl.vfin, cl.n(),
                                            cl.nx, cl.ny, out, out_stride, lv.nx, lv.ny, ih2, om1, st);
  MGH_CHECK_LAUNCH(); h.launches++;
  return MGH_OK;
}

template <typename T, typename TIn>
mgh_status launch_pre(Handle& h, int l, const void* bin, size_t b_stride, const double* bscale,
                      size_t scale_stride, int B, const RhsState* st, int in_slot = -1) {
  switch (nu_pre(h, l)) {
    case 0: return launch_pre_nu<T, 0, TIn>(h, l, bin, b_stride, bscale, scale_stride, B, st, in_slot);
    case 1: return launch_pre_nu<T, 1, TIn>(h, l, bin, b_stride, bscale, scale_stride, B, st, in_slot);
    case 2: return launch_pre_nu<T, 2, TIn>(h, l, bin, b_stride, bscale, scale_stride, B, st, in_slot);
    case 3: return launch_pre_nu<T, 3, TIn>(h, l, bin, b_stride, bscale, scale_stride, B, st, in_slot);
    case 4: return launch_pre_nu<T, 4, TIn>(h, l, bin, b_stride, bscale, scale_stride, B, st, in_slot);
  }
  return MGH_INVALID_ARG;
}

template <typename T, typename TIn, typename TOut>
mgh_status launch_post(Handle& h, int l, const void* bin, size_t b_stride, const double* bscale,
                       size_t scale_stride, Cx<TOut>* out, size_t out_stride, int B, const RhsState* st,
                       int in_slot = -1) {
  switch (nu_post(h, l)) {
    case 0: return launch_post_nu<T, 0, TIn, TOut>(h, l, bin, b_stride, bscale, scale_stride, out, out_stride, B, st, in_slot);
    case 1: return launch_post_nu<T, 1, TIn, TOut>(h, l, bin, b_stride, bscale, scale_stride, out, out_stride, B, st, in_slot);
    case 2: return launch_post_nu<T, 2, TIn, TOut>(h, l, bin, b_stride, bscale, scale_stride, out, out_stride, B, st, in_slot);
    case 3: return launch_post_nu<T, 3, TIn, TOut>(h, l, bin, b_stride, bscale, scale_stride, out, out_stride, B, st, in_slot);
    case 4: return launch_post_nu<T, 4, TIn, TOut>(h, l, bin, b_stride, bscale, scale_stride, out, out_stride, B, st, in_slot);
  }
  return MGH_INVALID_ARG;
}

// CycleType >= 2 (Alg. 2): before the next cycle of level l, whose last cycle left its result v in
// vfin, the right-hand side b becomes the residual b - K v and v joins the sum of the earlier
// corrections, so that the next cycle (from a zero guess) computes the correction to that sum:
// a cycle is affine in its initial guess, MG(b, v) = v + MG(b - K v, 0).
template <typename T>
__global__ void k_wc_residual(const Cx<T>* __restrict__ D, Cx<T>* __restrict__ b, const Cx<T>* __restrict__ v,
                              Cx<T>* __restrict__ acc, int first, int nx, int ny, T inv_h2,
                              const RhsState* __restrict__ st) {
  const int rhs = blockIdx.y;
  if (st && !st[rhs].active) return;
  const int n = nx * ny;
  const size_t off = (size_t)rhs * n;
  const Cx<T>* vr = v + off;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const int i = k / nx, j = k - i * nx;
    Cx<T> s = czero<T>();
    if (j > 0) s = s + vr[k - 1];
    if (j + 1 < nx) s = s + vr[k + 1];
    if (i > 0) s = s + vr[k - nx];
    if (i + 1 < ny) s = s + vr[k + nx];
    const Cx<T> vk = vr[k];
    const Cx<T> kv = D[k] * vk - inv_h2 * s;
    b[off + k] = b[off + k] - kv;
    acc[off + k] = first ? vk : acc[off + k] + vk;
  }
}

// vfin += the sum of the earlier corrections, after the last cycle of level l.
template <typename T>
__global__ void k_wc_add(Cx<T>* __restrict__ v, const Cx<T>* __restrict__ acc, int n, const RhsState* __restrict__ st) {
  const int rhs = blockIdx.y;
  if (st && !st[rhs].active) return;
  const size_t off = (size_t)rhs * n;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
    v[off + k] = v[off + k] + acc[off + k];
}

unsigned wc_blocks(int n) { return (unsigned)std::min(4096, (n + kVThreads - 1) / kVThreads); }

template <typename T>
mgh_status level_cycles(Handle& h, int l, int B, const RhsState* st);

// One cycle of level l >= 1 from a zero guess: right-hand side lev[l].b, result in lev[l].vfin.
template <typename T>
mgh_status level_cycle(Handle& h, int l, int B, const RhsState* st) {
  const Level& lv = h.lev[l];
  if (l == h.L - 1)   // coarsest: exact solve
    return launch_coarse_apply(h, lv.b, lv.n(), lv.vfin, lv.n(), B, st, sizeof(T) == 8);
  MGH_TRY((launch_pre<T, T>(h, l, lv.b, lv.n(), nullptr, 0, B, st)));
  MGH_TRY(level_cycles<T>(h, l + 1, B, st));
  return launch_post<T, T, T>(h, l, lv.b, lv.n(), nullptr, 0, (Cx<T>*)lv.vfin, lv.n(), B, st);
}

// The CycleType cycles that level l - 1 runs on level l (Alg. 2); the coarsest level's exact solve
// gives the same result every time, so it runs once.
template <typename T>
mgh_status level_cycles(Handle& h, int l, int B, const RhsState* st) {
  if (h.tail_l0 > 0 && l == h.tail_l0) return launch_tail(h, cycle_gamma(h), B, st, sizeof(T) == 8);
  MGH_TRY(level_cycle<T>(h, l, B, st));
  const int gamma = cycle_gamma(h);
  if (gamma == 1 || l == h.L - 1) return MGH_OK;
  Level& lv = h.lev[l];
  const int n = (int)lv.n();
  const dim3 grid(wc_blocks(n), B);
  for (int c = 1; c < gamma; ++c) {
    {
      ProfScope ps(h, P_COARSE);
      k_wc_residual<T><<<grid, kVThreads, 0, h.stream>>>((const Cx<T>*)lv.D, (Cx<T>*)lv.b, (const Cx<T>*)lv.vfin,
                                                         (Cx<T>*)lv.wacc, c == 1, lv.nx, lv.ny,
                                                         static_cast<T>(1.0 / (lv.h * lv.h)), st);
      MGH_CHECK_LAUNCH(); h.launches++;
    }
    MGH_TRY(level_cycle<T>(h, l, B, st));
  }
  ProfScope ps(h, P_COARSE);
  k_wc_add<T><<<grid, kVThreads, 0, h.stream>>>((Cx<T>*)lv.vfin, (const Cx<T>*)lv.wacc, n, st);
  MGH_CHECK_LAUNCH(); h.launches++;
  return MGH_OK;
}

// One cycle of Alg. 2 from a zero guess on the fine input: pre-smoothing and restriction of level
// 0, CycleType cycles of level 1 (recursively), prolongation and post-smoothing of level 0.
template <typename T, typename TIn>
mgh_status vcycle_t(Handle& h, const void* in, size_t in_stride, const double* in_scale, size_t scale_stride,
                    void* out, size_t out_stride, bool out_fp64, int B, const RhsState* st, int in_slot = -1) {
  MGH_TRY((launch_pre<T, TIn>(h, 0, in, in_stride, in_scale, scale_stride, B, st, in_slot)));
  MGH_TRY(level_cycles<T>(h, 1, B, st));
  if (out_fp64)
    return launch_post<T, TIn, double>(h, 0, in, in_stride, in_scale, scale_stride, (cd*)out, out_stride, B, st);
  return launch_post<T, TIn, T>(h, 0, in, in_stride, in_scale, scale_stride, (Cx<T>*)out, out_stride, B, st,
                                in_slot);
}

}  // namespace

mgh_status vcycle(Handle& h, const cd* in, size_t in_stride, const double* in_scale, size_t scale_stride,
                  void* out, size_t out_stride, bool out_fp64, int B, const RhsState* st) {
  if (h.fp64)
    return vcycle_t<double, double>(h, in, in_stride, in_scale, scale_stride, out, out_stride, out_fp64, B, st);
  return vcycle_t<float, double>(h, in, in_stride, in_scale, scale_stride, out, out_stride, out_fp64, B, st);
}

mgh_status vcycle_f32in(Handle& h, const cf* in, size_t in_stride, const double* in_scale, size_t scale_stride,
                        cf* out, size_t out_stride, int B, const RhsState* st, int in_slot) {
  return vcycle_t<float, float>(h, in, in_stride, in_scale, scale_stride, out, out_stride, false, B, st, in_slot);
}

// ---------------------------------------------------------------- tensor maps
namespace {

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    return nullptr;
  }();
  return fn;
}

// Tensor map over complex FP32 data (8-byte elements): dims (nx, ny[, nz]), byte strides of
// rows and planes, box (bx, by[, 1]).  False if the 16-byte rules of the encoder are not met.
bool encode_map(CUtensorMap* map, const void* base, int rank, uint64_t nx, uint64_t ny, uint64_t nz,
                uint64_t row_bytes, uint64_t plane_bytes, uint32_t bx, uint32_t by) {
  auto enc = tensor_map_encoder();
  if (!enc) return false;
  if ((reinterpret_cast<uintptr_t>(base) & 15) || (row_bytes & 15) || (rank == 3 && (plane_bytes & 15))) return false;
  if ((bx * 8) % 16 || bx > 256 || by > 256) return false;
  cuuint64_t dims[3] = {nx, ny, nz};
  cuuint64_t strides[2] = {row_bytes, plane_bytes};
  cuuint32_t box[3] = {bx, by, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, (cuuint32_t)rank, const_cast<void*>(base), dims, strides,
                         box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// Box geometry of the TMA level kernels for nu sweeps (mirrors PreGeom / PostGeom).
struct BoxDims { int sw, sh, cw, ch; };
BoxDims pre_box(int nu) {
  const int H = nu + 1, HX = (H + 1) & ~1;
  return {64 + 2 * HX, 16 + 2 * H, 0, 0};
}
BoxDims post_box(int nu) {
  const int H = nu, HX = (nu + 1) & ~1;
  return {64 + 2 * HX, 16 + 2 * H, ((32 + HX + 3) + 1) & ~1, 8 + H + 2};
}

}  // namespace

mgh_status build_vcycle_tma(Handle& h) {
  if (h.fp64 || !tensor_map_encoder()) return MGH_OK;
  h.tma = new (std::nothrow) LevelTma[kMaxLevels];
  h.tma_in = new (std::nothrow) CUtensorMap[2 * h.m];
  if (!h.tma || !h.tma_in) return MGH_OUT_OF_MEMORY;
  const uint64_t B = h.Bmax;
  for (int l = 0; l + 1 < h.L; ++l) {
    const BoxDims bp = pre_box(nu_pre(h, l)), bq = post_box(nu_post(h, l));
    const Level& lv = h.lev[l];
    const Level& cl = h.lev[l + 1];
    LevelTma& t = h.tma[l];
    const uint64_t row = (uint64_t)lv.nx * 8, plane = (uint64_t)lv.n() * 8;
    bool ok = (lv.nx % 2 == 0);
    ok = ok && encode_map(&t.pre_w, lv.wDinv, 2, lv.nx, lv.ny, 1, row, 0, bp.sw, bp.sh);
    ok = ok && encode_map(&t.pre_d, lv.D, 2, lv.nx, lv.ny, 1, row, 0, bp.sw, bp.sh);
    if (l >= 1) ok = ok && encode_map(&t.pre_b, lv.b, 3, lv.nx, lv.ny, B, row, plane, bp.sw, bp.sh);
    t.pre_ok = ok;
    bool okp = (lv.nx % 2 == 0) && (cl.nx % 2 == 0);
    okp = okp && encode_map(&t.post_w, lv.wDinv, 2, lv.nx, lv.ny, 1, row, 0, bq.sw, bq.sh);
    okp = okp && encode_map(&t.post_v, lv.vpre, 3, lv.nx, lv.ny, B, row, plane, bq.sw, bq.sh);
    if (l >= 1) okp = okp && encode_map(&t.post_b, lv.b, 3, lv.nx, lv.ny, B, row, plane, bq.sw, bq.sh);
    okp = okp && encode_map(&t.post_e, cl.vfin, 3, cl.nx, cl.ny, B, (uint64_t)cl.nx * 8, (uint64_t)cl.n() * 8,
                            bq.cw, bq.ch);
    t.post_ok = okp;
  }
  // level-0 inputs: the hi plane of basis slot j of every right-hand side
  const BoxDims bp = pre_box(nu_pre(h, 0)), bq = post_box(nu_post(h, 0));
  bool ok = (h.nx % 2 == 0);
  const float2* V = reinterpret_cast<const float2*>(h.V);
  const uint64_t rhs_bytes = (uint64_t)(h.m + 1) * 2 * h.Np * 8;
  for (int j = 0; j < h.m && ok; ++j) {
    const float2* base = V + (size_t)j * 2 * h.Np;
    ok = encode_map(&h.tma_in[j], base, 3, h.nx, h.ny, B, (uint64_t)h.nx * 8, rhs_bytes, bp.sw, bp.sh) &&
         encode_map(&h.tma_in[h.m + j], base, 3, h.nx, h.ny, B, (uint64_t)h.nx * 8, rhs_bytes, bq.sw, bq.sh);
  }
  h.tma_in_ok = ok;
  return MGH_OK;
}

}  // namespace mgh
