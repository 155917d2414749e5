// Register-streaming ("wavefront") level kernels of the complex FP32 V-cycle (Alg. 2).
//
// A warp owns a strip of 64 columns of one right-hand side (two adjacent columns per lane) and a
// segment of its rows, and walks the rows once from top to bottom.  Each stage of the fused level
// kernel runs a fixed number of rows behind the stage before it, so that all damped-Jacobi sweeps,
// the residual and the full-weighting restriction advance together through the strip (temporal
// blocking along y):
//
//   pre   row i: v1 = (w/D) b;  sweep s (2..nu1) on row i-(s-1);  r = b - K v on row i-nu1;
//         restriction on fine row i-nu1-1 when it is even
//   post  row i: v0 = v_pre + P e;  sweep s (1..nu2) on row i-s, the last one stored
//
// The rows a stage still needs sit in small register rings whose slots are fixed at compile time
// (the row loop is unrolled over the ring period); the left and right neighbours of a point come
// from the adjacent lanes by warp shuffles.  Nothing is staged in shared memory and no barrier is
// taken.  The strip overlaps its neighbours by HX columns per side, one column for each stencil
// stage that reads across the strip edge, and each segment starts its wavefront a few rows above
// its first row.  Points outside the grid are 0 in every stage, as in the tiled kernels: the
// Sommerfeld closure sits in D, so w/D = 0 there keeps the iterate at 0, and the residual is
// masked before it is restricted.
#pragma once

#include <cuda_fp16.h>

#include <cstddef>
#include <type_traits>
#include <utility>

#include "mgh_common.cuh"
#include "mgh_engine.h"
#include "mgh_tma.cuh"

namespace mgh {
namespace wave {

constexpr unsigned kFull = 0xffffffffu;

// The values of a lane's two columns g0 (a) and g0 + 1 (b), g0 even.
struct C2 {
  cf a, b;
};

__device__ __forceinline__ C2 c2zero() {
  C2 r;
  r.a = czero<float>();
  r.b = czero<float>();
  return r;
}

__device__ __forceinline__ cf shfl_up1(cf v) {
  return mk<float>(__shfl_up_sync(kFull, v.re, 1), __shfl_up_sync(kFull, v.im, 1));
}
__device__ __forceinline__ cf shfl_dn1(cf v) {
  return mk<float>(__shfl_down_sync(kFull, v.re, 1), __shfl_down_sync(kFull, v.im, 1));
}

// The lane's two points of one row.  Load columns are clamped into the grid so that every address
// is valid (the caller masks what was read outside); V4: one 16-byte load at the even column c0
// (rows of even width, 16-byte aligned base), else two 8-byte loads at c0 and c1.
template <bool V4>
__device__ __forceinline__ C2 ld2(const cf* __restrict__ row, int c0, int c1) {
  C2 r;
  if constexpr (V4) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(row + c0));
    r.a = mk<float>(v.x, v.y);
    r.b = mk<float>(v.z, v.w);
  } else {
    r.a = row[c0];
    r.b = row[c1];
  }
  return r;
}

__device__ __forceinline__ cf sel(bool ok, cf v) { return ok ? v : czero<float>(); }

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

template <bool V4>
__device__ __forceinline__ void st2(cf* __restrict__ p, ptrdiff_t off, bool ok0, bool ok1, const C2& v) {
  if constexpr (V4) {
    if (ok0) *reinterpret_cast<float4*>(p + off) = make_float4(v.a.re, v.a.im, v.b.re, v.b.im);
  } else {
    if (ok0) p[off] = v.a;
    if (ok1) p[off + 1] = v.b;
  }
}

// Complex FP16 storage (MGH_PREC_MIXED16): one __half2 per point, x = re, y = im.  Arithmetic
// stays FP32; values are rounded to nearest on store.
__device__ __forceinline__ __half2 to_h2(cf v) { return __floats2half2_rn(v.re, v.im); }
__device__ __forceinline__ cf from_h2(__half2 v) {
  const float2 f = __half22float2(v);
  return mk<float>(f.x, f.y);
}

// The lane's two points (8 bytes, g0 even so the pair is 8-byte aligned) as FP16.
__device__ __forceinline__ void st2h(__half2* __restrict__ p, ptrdiff_t off, bool ok0, const C2& v) {
  if (ok0) {
    __half2 h[2] = {to_h2(v.a), to_h2(v.b)};
    *reinterpret_cast<uint2*>(p + off) = *reinterpret_cast<const uint2*>(h);
  }
}

// Store of the lane's two points in the storage type VT (cf or __half2).
template <typename VT>
__device__ __forceinline__ void st2v(VT* __restrict__ p, ptrdiff_t off, bool ok0, bool ok1, const C2& v) {
  if constexpr (std::is_same<VT, __half2>::value) st2h(p, off, ok0, v);
  else st2<true>(p, off, ok0, ok1, v);
}

// Damped Jacobi at one point: (1 - omega) c + (omega/D) (sb + (l + r + u + d) / h^2).
__device__ __forceinline__ cf jac_pt(cf c, cf l, cf r, cf u, cf d, cf sb, cf wd, float ih, float om1) {
  const float sr = (l.re + r.re) + (u.re + d.re), si = (l.im + r.im) + (u.im + d.im);
  const float tr = fmaf(ih, sr, sb.re), ti = fmaf(ih, si, sb.im);
  return mk<float>(fmaf(wd.re, tr, fmaf(-wd.im, ti, om1 * c.re)), fmaf(wd.re, ti, fmaf(wd.im, tr, om1 * c.im)));
}

// Residual at one point: sb - D c + (l + r + u + d) / h^2.
__device__ __forceinline__ cf res_pt(cf c, cf l, cf r, cf u, cf d, cf sb, cf dd, float ih) {
  const float sr = (l.re + r.re) + (u.re + d.re), si = (l.im + r.im) + (u.im + d.im);
  const float tr = fmaf(ih, sr, sb.re), ti = fmaf(ih, si, sb.im);
  return mk<float>(fmaf(-dd.re, c.re, fmaf(dd.im, c.im, tr)), fmaf(-dd.re, c.im, fmaf(-dd.im, c.re, ti)));
}

// One sweep on the lane's two points of a row, from the rows above (up), at (mid) and below (dn).
__device__ __forceinline__ C2 jac_row(const C2& up, const C2& mid, const C2& dn, const C2& sb, const C2& wd, float ih,
                                      float om1) {
  const cf left = shfl_up1(mid.b), right = shfl_dn1(mid.a);
  C2 o;
  o.a = jac_pt(mid.a, left, mid.b, up.a, dn.a, sb.a, wd.a, ih, om1);
  o.b = jac_pt(mid.b, mid.a, right, up.b, dn.b, sb.b, wd.b, ih, om1);
  return o;
}

__device__ __forceinline__ C2 scale2(float s, const C2& v) {
  C2 o;
  o.a = s * v.a;
  o.b = s * v.b;
  return o;
}

// Ring slot of the row d rows above the newest one, at unrolled step Kc of a ring of R rows.
__host__ __device__ constexpr int slot(int Kc, int d, int R) { return ((Kc - d) % R + R) % R; }

template <typename F, int... I>
__device__ __forceinline__ void unroll_seq(F&& f, std::integer_sequence<int, I...>) {
  (f(std::integral_constant<int, I>{}), ...);
}
template <int N, typename F>
__device__ __forceinline__ void unroll(F&& f) {
  unroll_seq(f, std::make_integer_sequence<int, N>{});
}

__host__ __device__ constexpr int gcd_c(int a, int b) { return b == 0 ? a : gcd_c(b, a % b); }
__host__ __device__ constexpr int lcm_c(int a, int b) { return a / gcd_c(a, b) * b; }

// Geometry of the fused level kernels for nu sweeps: halo columns HX (even, so that a lane's
// column pair is 16-byte aligned), owned columns XO per strip, ring length R, unroll period P (a
// multiple of R, of 2 for the row parity of the restriction and prolongation, and of PF, the rows
// of input loads kept in flight ahead of the row being computed).
template <int NU, int PF>
struct PreW {
  static constexpr int H = NU + 1, HX = (H + 1) & ~1, XO = 64 - 2 * HX;
  static constexpr int R = NU + 1 > 3 ? NU + 1 : 3;
  static constexpr int P = lcm_c(lcm_c(R, 2), PF);
};

template <int NU, int PF>
struct PostW {
  static constexpr int H = NU, HX = (NU + 1) & ~1, XO = 64 - 2 * HX;
  static constexpr int R = NU + 1 > 3 ? NU + 1 : 3;
  static constexpr int P = lcm_c(lcm_c(R, 2), PF);
};

// nu1 >= 1 damped-Jacobi sweeps from v = 0, the residual and its full-weighting restriction.
// b of right-hand side q is bin[q * b_stride + ...] times bscale[q * scale_stride] (1 if null).
// Writes v to vpre and the restricted residual to bc (coarse grid nxc x nyc).
template <int NU, bool V4, int PF, int NW>
__global__ void __launch_bounds__(32 * NW)
k_pre_w(const cf* __restrict__ bin, size_t b_stride, const double* __restrict__ bscale, size_t scale_stride,
        const cf* __restrict__ D, const cf* __restrict__ wD, cf* __restrict__ vpre, size_t v_stride,
        cf* __restrict__ bc, size_t bc_stride, int nx, int ny, int nxc, float ih, float om1, int nstrips,
        int nwarps, int seg, const RhsState* __restrict__ st) {
  static_assert(NU >= 1, "the wavefront pre kernel starts with one pointwise sweep");
  using G = PreW<NU, PF>;
  constexpr int H = G::H, HX = G::HX, XO = G::XO, R = G::R, P = G::P;
  const int rhs = blockIdx.z;
  if (st && !st[rhs].active) return;
  const int w = blockIdx.x * NW + (threadIdx.x >> 5);
  if (w >= nwarps) return;
  const int lane = threadIdx.x & 31;
  const int xs = (w % nstrips) * XO, ys = (w / nstrips) * seg;
  const int g0 = xs - HX + 2 * lane;
  const bool in0 = g0 >= 0 && g0 < nx, in1 = g0 + 1 >= 0 && g0 + 1 < nx;
  const bool own = lane >= HX / 2 && lane < HX / 2 + XO / 2;
  const int ci = g0 >> 1;
  const bool own_c = own && g0 >= 0 && ci < nxc;
  const float sc = bscale ? (float)bscale[rhs * scale_stride] : 1.f;
  const cf* __restrict__ bb = bin + rhs * b_stride;
  cf* __restrict__ vo = vpre + rhs * v_stride;
  cf* __restrict__ co = bc + rhs * bc_stride;
  const int i0 = ys - H;                                  // first input row of the wavefront
  int rows = ny - ys < seg ? ny - ys : seg;
  rows = (rows + 1) & ~1;                                 // the last even fine row needs its row below
  // steps: rows + 2H - 1, rounded up to whole unrolled periods (the extra steps only read rows
  // and store nothing), so that the unrolled period has no exit and the rings need no moves
  const int K = (rows + 2 * H - 1 + P - 1) / P * P;

  C2 v[NU][R], sbr[R], wdr[R];
  cf hr[R];   // r(g0 - 1) + 2 r(g0) + r(g0 + 1) per row
#pragma unroll
  for (int i = 0; i < R; ++i) {
#pragma unroll
    for (int s = 0; s < NU; ++s) v[s][i] = c2zero();
    sbr[i] = c2zero();
    wdr[i] = c2zero();
    hr[i] = czero<float>();
  }
  struct In {
    C2 b, w, d;
  };
  const int c0 = V4 ? clampi(g0, 0, nx - 2) : clampi(g0, 0, nx - 1), c1 = clampi(g0 + 1, 0, nx - 1);
  // b and D unmasked (b only meets w/D or the masked residual); w/D is 0 outside the grid
  auto load = [&](int k) {
    In t;
    const int y = i0 + k, yd = y - NU;
    if (y >= 0 && y < ny) {
      const ptrdiff_t off = (ptrdiff_t)y * nx;
      t.b = ld2<V4>(bb + off, c0, c1);
      t.w = ld2<V4>(wD + off, c0, c1);
      t.w.a = sel(in0, t.w.a);
      t.w.b = sel(in1, t.w.b);
    } else {
      t.b = t.w = c2zero();
    }
    if (yd >= 0 && yd < ny) t.d = ld2<V4>(D + (ptrdiff_t)yd * nx, c0, c1);
    else t.d = c2zero();
    return t;
  };
  In nxt[PF];
#pragma unroll
  for (int i = 0; i < PF; ++i) nxt[i] = load(i);
  for (int kb = 0; kb < K; kb += P) {
    unroll<P>([&](auto KC) {
      constexpr int Kc = decltype(KC)::value;
      const int k = kb + Kc;
      const In cur = nxt[Kc % PF];
      nxt[Kc % PF] = load(k + PF);
      // row k: scaled right-hand side, omega/D, first sweep from v = 0
      constexpr int s0 = slot(Kc, 0, R);
      sbr[s0] = scale2(sc, cur.b);
      wdr[s0] = cur.w;
      v[0][s0].a = cur.w.a * sbr[s0].a;
      v[0][s0].b = cur.w.b * sbr[s0].b;
      // sweep s on row k - (s - 1)
      unroll<NU - 1>([&](auto SC) {
        constexpr int s = decltype(SC)::value + 2;
        constexpr int so = slot(Kc, s - 1, R);
        v[s - 1][so] = jac_row(v[s - 2][slot(Kc, s, R)], v[s - 2][so], v[s - 2][slot(Kc, s - 2, R)], sbr[so], wdr[so],
                               ih, om1);
      });
      // residual on row k - nu1, 0 outside the grid, and its horizontal (1, 2, 1) weighting
      {
        constexpr int sr = slot(Kc, NU, R);
        const int yr = i0 + k - NU;
        const bool okr = yr >= 0 && yr < ny;
        const C2& up = v[NU - 1][slot(Kc, NU + 1, R)];
        const C2& mid = v[NU - 1][sr];
        const C2& dn = v[NU - 1][slot(Kc, NU - 1, R)];
        const cf left = shfl_up1(mid.b), right = shfl_dn1(mid.a);
        const cf r0 = sel(okr && in0, res_pt(mid.a, left, mid.b, up.a, dn.a, sbr[sr].a, cur.d.a, ih));
        const cf r1 = sel(okr && in1, res_pt(mid.b, mid.a, right, up.b, dn.b, sbr[sr].b, cur.d.b, ih));
        const cf rl = shfl_up1(r1);
        hr[sr] = mk<float>(rl.re + 2.f * r0.re + r1.re, rl.im + 2.f * r0.im + r1.im);
      }
      // full weighting at the coarse points of fine row k - nu1 - 1 (even rows only)
      if constexpr (Kc % 2 == 0) {
        const int yf = i0 + k - NU - 1;
        if (k >= 2 * H && yf < ys + rows && yf < ny && own_c) {
          const cf a = hr[slot(Kc, NU + 2, R)], m = hr[slot(Kc, NU + 1, R)], c = hr[slot(Kc, NU, R)];
          co[(size_t)(yf >> 1) * nxc + ci] =
              mk<float>(0.0625f * (a.re + 2.f * m.re + c.re), 0.0625f * (a.im + 2.f * m.im + c.im));
        }
      }
      // the finished iterate on row k - (nu1 - 1)
      {
        const int yv = i0 + k - (NU - 1);
        if (yv >= ys && yv < ys + seg && yv < ny)
          st2<V4>(vo, (ptrdiff_t)yv * nx + g0, own && in0, own && in1, v[NU - 1][slot(Kc, NU - 1, R)]);
      }
    });
  }
}

// Coarse-grid values of a lane at coarse columns ci and ci + 1 of one coarse row.
struct E2 {
  cf c0, c1;
};

// Bilinear prolongation of the coarse correction e (coarse grid nxc x nyc), v0 = v_pre + P e,
// then nu2 >= 1 damped-Jacobi sweeps; the result goes to out.
template <int NU, bool V4, int PF, int NW>
__global__ void __launch_bounds__(32 * NW)
k_post_w(const cf* __restrict__ bin, size_t b_stride, const double* __restrict__ bscale, size_t scale_stride,
         const cf* __restrict__ wD, const cf* __restrict__ vpre, size_t v_stride, const cf* __restrict__ ec,
         size_t ec_stride, int nxc, int nyc, cf* __restrict__ out, size_t out_stride, int nx, int ny, float ih,
         float om1, int nstrips, int nwarps, int seg, const RhsState* __restrict__ st) {
  static_assert(NU >= 1, "the wavefront post kernel ends with a sweep");
  using G = PostW<NU, PF>;
  constexpr int HX = G::HX, XO = G::XO, R = G::R, P = G::P;
  const int rhs = blockIdx.z;
  if (st && !st[rhs].active) return;
  const int w = blockIdx.x * NW + (threadIdx.x >> 5);
  if (w >= nwarps) return;
  const int lane = threadIdx.x & 31;
  const int xs = (w % nstrips) * XO, ys = (w / nstrips) * seg;
  const int g0 = xs - HX + 2 * lane;
  const bool in0 = g0 >= 0 && g0 < nx, in1 = g0 + 1 >= 0 && g0 + 1 < nx;
  const bool own = lane >= HX / 2 && lane < HX / 2 + XO / 2;
  const int ci = g0 >> 1;
  const bool okc0 = ci >= 0 && ci < nxc, okc1 = ci + 1 >= 0 && ci + 1 < nxc;
  const float sc = bscale ? (float)bscale[rhs * scale_stride] : 1.f;
  const cf* __restrict__ bb = bin + rhs * b_stride;
  const cf* __restrict__ vp = vpre + rhs * v_stride;
  const cf* __restrict__ eb = ec + rhs * ec_stride;
  cf* __restrict__ o = out + rhs * out_stride;
  const int i0 = ys - NU;
  const int rows = ny - ys < seg ? ny - ys : seg;
  const int K = (rows + 2 * NU + P - 1) / P * P;   // whole unrolled periods, as in k_pre_w

  C2 v[NU][R], sbr[R], wdr[R];
#pragma unroll
  for (int i = 0; i < R; ++i) {
#pragma unroll
    for (int s = 0; s < NU; ++s) v[s][i] = c2zero();
    sbr[i] = c2zero();
    wdr[i] = c2zero();
  }
  const int e0 = clampi(ci, 0, nxc - 1), e1 = clampi(ci + 1, 0, nxc - 1);
  auto load_e = [&](int c) {
    E2 e;
    if (c >= 0 && c < nyc) {
      const cf* row = eb + (size_t)c * nxc;
      e.c0 = sel(okc0, row[e0]);
      e.c1 = sel(okc1, row[e1]);
    } else {
      e.c0 = e.c1 = czero<float>();
    }
    return e;
  };
  struct In {
    C2 vp, b, w;
  };
  const int c0 = V4 ? clampi(g0, 0, nx - 2) : clampi(g0, 0, nx - 1), c1 = clampi(g0 + 1, 0, nx - 1);
  // v_pre and b unmasked (v0 is masked, b only meets w/D); w/D is 0 outside the grid
  auto load = [&](int k) {
    In t;
    const int y = i0 + k;
    if (y >= 0 && y < ny) {
      const ptrdiff_t off = (ptrdiff_t)y * nx;
      t.vp = ld2<V4>(vp + off, c0, c1);
      t.b = ld2<V4>(bb + off, c0, c1);
      t.w = ld2<V4>(wD + off, c0, c1);
      t.w.a = sel(in0, t.w.a);
      t.w.b = sel(in1, t.w.b);
    } else {
      t.vp = t.b = t.w = c2zero();
    }
    return t;
  };
  // ea: coarse row floor(y / 2) of the current fine row y; enext: the row after it, loaded one
  // fine row ahead of its first use
  E2 ea = load_e(i0 >> 1), enext = ea;
  if (i0 & 1) enext = load_e((i0 >> 1) + 1);
  In nxt[PF];
#pragma unroll
  for (int i = 0; i < PF; ++i) nxt[i] = load(i);
  for (int kb = 0; kb < K; kb += P) {
    unroll<P>([&](auto KC) {
      constexpr int Kc = decltype(KC)::value;
      constexpr bool odd = ((Kc + NU) & 1) != 0;   // parity of fine row i0 + k (ys is even)
      const int k = kb + Kc;
      const In cur = nxt[Kc % PF];
      nxt[Kc % PF] = load(k + PF);
      const int y = i0 + k;
      // v0 on row k: v_pre + P e, 0 outside the grid
      C2 pe;
      if constexpr (!odd) {
        pe.a = ea.c0;
        pe.b = 0.5f * (ea.c0 + ea.c1);
        enext = load_e((y >> 1) + 1);
      } else {
        const cf m0 = 0.5f * (ea.c0 + enext.c0), m1 = 0.5f * (ea.c1 + enext.c1);
        pe.a = m0;
        pe.b = 0.5f * (m0 + m1);
        ea = enext;
      }
      const bool oky = y >= 0 && y < ny;
      constexpr int s0 = slot(Kc, 0, R);
      v[0][s0].a = sel(oky && in0, cur.vp.a + pe.a);
      v[0][s0].b = sel(oky && in1, cur.vp.b + pe.b);
      sbr[s0] = scale2(sc, cur.b);
      wdr[s0] = cur.w;
      // sweeps 1 .. nu2-1 on rows k - s
      unroll<NU - 1>([&](auto SC) {
        constexpr int s = decltype(SC)::value + 1;
        constexpr int so = slot(Kc, s, R);
        v[s][so] = jac_row(v[s - 1][slot(Kc, s + 1, R)], v[s - 1][so], v[s - 1][slot(Kc, s - 1, R)], sbr[so], wdr[so],
                           ih, om1);
      });
      // last sweep on row k - nu2, stored on the owned points
      {
        constexpr int so = slot(Kc, NU, R);
        const C2 vn = jac_row(v[NU - 1][slot(Kc, NU + 1, R)], v[NU - 1][so], v[NU - 1][slot(Kc, NU - 1, R)], sbr[so],
                              wdr[so], ih, om1);
        const int yv = y - NU;
        if (yv >= ys && yv < ys + seg && yv < ny) st2<V4>(o, (ptrdiff_t)yv * nx + g0, own && in0, own && in1, vn);
      }
    });
  }
}


// ---------------------------------------------------------------- shared-memory row rings (TMA)
// The same wavefront, with the input rows of each warp streamed through a private ring of S
// shared-memory slots by bulk copies (cp.async.bulk, one mbarrier per slot): lane 0 keeps
// S - nu - 1 rows in flight ahead of the row being computed, and the stages that work on older
// rows read them back from the ring, so neither the loads in flight nor the delayed inputs take
// registers.  S is a multiple of the unroll period, so every slot offset is a compile-time
// constant.  A slot holds three arrays of the 64 strip columns; the columns outside the grid are
// zeroed once and never copied, and the slot of a row outside the grid is zeroed by the warp
// instead of copied, so reads need no checks and omega/D is 0 outside the grid as required.
// Every wait is bounded: after a timeout the warp issues and waits for nothing more, computes on
// stale rows (every address stays in bounds), raises the error word and, before it returns,
// waits (bounded) for its own copies in flight.  Needs rows and planes of even width and 16-byte
// aligned bases (the 16-byte rule of the bulk copy).

template <int NW, int S>
struct RingSmem {
  static constexpr int ROW = 64;            // complex values per array row of a strip
  static constexpr int SLOT = 3 * ROW;      // three arrays per slot
  __host__ __device__ static constexpr size_t bars() { return ((size_t)NW * S * 8 + 127) / 128 * 128; }
  __host__ __device__ static constexpr size_t bytes() { return bars() + (size_t)NW * S * SLOT * sizeof(cf); }
};

__device__ __forceinline__ C2 lds2(const cf* p) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  C2 r;
  r.a = mk<float>(v.x, v.y);
  r.b = mk<float>(v.z, v.w);
  return r;
}

// Per-warp ring: barriers, slots, and the geometry of the strip's copies.
struct Ring {
  uint64_t* bar;
  cf* buf;        // slot 0 of this warp
  cf* mine;       // slot 0 at this lane's two columns
  int lo, doff, i0, ny, nx;
  uint32_t rbytes;

  __device__ __forceinline__ bool row_ok(int r) const { const int y = i0 + r; return y >= 0 && y < ny; }

  // Row r into slot s: lane 0 queues the copies of the three arrays; a row outside the grid is
  // zeroed by the whole warp and its barrier phase completed by a plain arrival.
  __device__ __forceinline__ void issue(int r, int s, int lane, const cf* a0, const cf* a1, const cf* a2) const {
    uint64_t* b = &bar[s];
    if (row_ok(r)) {
      if (lane == 0) {
        const size_t off = (size_t)(i0 + r) * nx + lo;
        cf* dst = buf + s * (3 * 64) + doff;
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(b, 3u * rbytes);
        bulk_load(dst, a0 + off, rbytes, b);
        bulk_load(dst + 64, a1 + off, rbytes, b);
        bulk_load(dst + 128, a2 + off, rbytes, b);
      }
    } else {
      float4* z = reinterpret_cast<float4*>(buf + s * (3 * 64));
      const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
      z[lane] = zero;
      z[lane + 32] = zero;
      z[lane + 64] = zero;
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(b);
    }
  }
  __device__ __forceinline__ bool wait(int s, uint32_t parity) const { return mbar_wait(&bar[s], parity, kWaitLimitNs); }
  // array a of slot s at the lane's two columns
  __device__ __forceinline__ C2 get(int s, int a) const { return lds2(mine + s * (3 * 64) + a * 64); }
};

template <int NW, int S>
__device__ __forceinline__ Ring ring_begin(unsigned char* smem, int x0, int nx, int ny, int i0, int lane) {
  using M = RingSmem<NW, S>;
  const int wib = threadIdx.x >> 5;
  Ring g;
  g.bar = reinterpret_cast<uint64_t*>(smem) + wib * S;
  g.buf = reinterpret_cast<cf*>(smem + M::bars()) + (size_t)wib * S * M::SLOT;
  g.mine = g.buf + 2 * lane;
  g.lo = x0 < 0 ? 0 : x0;
  const int hi = x0 + 64 < nx ? x0 + 64 : nx;
  g.rbytes = (uint32_t)(hi - g.lo) * (uint32_t)sizeof(cf);
  g.doff = g.lo - x0;
  g.i0 = i0;
  g.ny = ny;
  g.nx = nx;
  if (lane == 0) {
    for (int s = 0; s < S; ++s) mbar_init(&g.bar[s], 1);
    fence_mbar_init();
  }
  float4* z = reinterpret_cast<float4*>(g.buf);
  for (int i = lane; i < S * M::SLOT / 2; i += 32) z[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  fence_proxy_async_smem();
  __syncwarp();
  return g;
}

// After a timeout at row `from`: raise the error word and wait (bounded) for rows [from, to).
template <int S>
__device__ __forceinline__ void ring_abort(const Ring& g, int from, int to, int lane, int* err) {
  if (lane == 0) {
    atomicExch(err, kErrTimeout);
    for (int r = from; r < to; ++r) g.wait(r % S, (uint32_t)((r / S) & 1));
  }
  __syncwarp();
}

// Ring length for nu sweeps: the smallest multiple of the unroll period with at least two rows
// in flight, times MS.
template <int P, int NU, int MS>
struct RingLen {
  static constexpr int S0 = (NU + 3 + P - 1) / P * P;
  static constexpr int S = S0 * MS;
};

template <int NU, int NW, int MS>
__global__ void __launch_bounds__(32 * NW)
k_pre_wt(const cf* __restrict__ bin, size_t b_stride, const double* __restrict__ bscale, size_t scale_stride,
         const cf* __restrict__ D, const cf* __restrict__ wD, cf* __restrict__ vpre, size_t v_stride,
         cf* __restrict__ bc, size_t bc_stride, int nx, int ny, int nxc, float ih, float om1, int nstrips,
         int nwarps, int seg, const RhsState* __restrict__ st, int* __restrict__ err) {
  static_assert(NU >= 1, "the wavefront pre kernel starts with one pointwise sweep");
  using G = PreW<NU, 1>;
  constexpr int H = G::H, HX = G::HX, XO = G::XO, R = G::R;
  constexpr int S = RingLen<G::P, NU, MS>::S;   // also the unroll period
  constexpr int PFD = S - NU - 1;                // rows in flight ahead of the current one
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int rhs = blockIdx.z;
  if (st && !st[rhs].active) return;
  const int w = blockIdx.x * NW + (threadIdx.x >> 5);
  if (w >= nwarps) return;
  const int lane = threadIdx.x & 31;
  const int xs = (w % nstrips) * XO, ys = (w / nstrips) * seg;
  const int g0 = xs - HX + 2 * lane;
  const bool in0 = g0 >= 0 && g0 < nx, in1 = g0 + 1 >= 0 && g0 + 1 < nx;
  const bool own = lane >= HX / 2 && lane < HX / 2 + XO / 2;
  const int ci = g0 >> 1;
  const bool own_c = own && g0 >= 0 && ci < nxc;
  const float sc = bscale ? (float)bscale[rhs * scale_stride] : 1.f;
  const cf* __restrict__ bb = bin + rhs * b_stride;
  cf* __restrict__ vo = vpre + rhs * v_stride;
  cf* __restrict__ co = bc + rhs * bc_stride;
  const int i0 = ys - H;
  int rows = ny - ys < seg ? ny - ys : seg;
  rows = (rows + 1) & ~1;
  const int K = (rows + 2 * H - 1 + S - 1) / S * S;
  const Ring g = ring_begin<NW, S>(smem_raw, xs - HX, nx, ny, i0, lane);
  // slot arrays: 0 = b, 1 = omega/D, 2 = D
  for (int r = 0; r < PFD && r < K; ++r) g.issue(r, r, lane, bb, wD, D);

  C2 v[NU][R];
  cf hr[R];
#pragma unroll
  for (int i = 0; i < R; ++i) {
#pragma unroll
    for (int s = 0; s < NU; ++s) v[s][i] = c2zero();
    hr[i] = czero<float>();
  }
  int fail_at = -1;
  for (int kb = 0; kb < K; kb += S) {
    const uint32_t par = (uint32_t)((kb / S) & 1);
    unroll<S>([&](auto KC) {
      constexpr int Kc = decltype(KC)::value;
      const int k = kb + Kc;
      __syncwarp();   // every lane is done with row k - nu1 - 1: its slot takes row k + PFD
      if (fail_at < 0) {
        if (k + PFD < K) g.issue(k + PFD, (Kc + PFD) % S, lane, bb, wD, D);
        if (!__all_sync(kFull, g.wait(Kc, par))) fail_at = k;
      }
      // row k: first sweep from v = 0
      constexpr int s0 = slot(Kc, 0, R);
      {
        const C2 sb = scale2(sc, g.get(Kc, 0)), wd = g.get(Kc, 1);
        v[0][s0].a = wd.a * sb.a;
        v[0][s0].b = wd.b * sb.b;
      }
      unroll<NU - 1>([&](auto SC) {
        constexpr int s = decltype(SC)::value + 2;
        constexpr int so = slot(Kc, s - 1, R);
        constexpr int gs = slot(Kc, s - 1, S);
        v[s - 1][so] = jac_row(v[s - 2][slot(Kc, s, R)], v[s - 2][so], v[s - 2][slot(Kc, s - 2, R)],
                               scale2(sc, g.get(gs, 0)), g.get(gs, 1), ih, om1);
      });
      {
        constexpr int sr = slot(Kc, NU, R);
        constexpr int gs = slot(Kc, NU, S);
        const int yr = i0 + k - NU;
        const bool okr = yr >= 0 && yr < ny;
        const C2 sb = scale2(sc, g.get(gs, 0)), dd = g.get(gs, 2);
        const C2& up = v[NU - 1][slot(Kc, NU + 1, R)];
        const C2& mid = v[NU - 1][sr];
        const C2& dn = v[NU - 1][slot(Kc, NU - 1, R)];
        const cf left = shfl_up1(mid.b), right = shfl_dn1(mid.a);
        const cf r0 = sel(okr && in0, res_pt(mid.a, left, mid.b, up.a, dn.a, sb.a, dd.a, ih));
        const cf r1 = sel(okr && in1, res_pt(mid.b, mid.a, right, up.b, dn.b, sb.b, dd.b, ih));
        const cf rl = shfl_up1(r1);
        hr[sr] = mk<float>(rl.re + 2.f * r0.re + r1.re, rl.im + 2.f * r0.im + r1.im);
      }
      if constexpr (Kc % 2 == 0) {
        const int yf = i0 + k - NU - 1;
        if (k >= 2 * H && yf < ys + rows && yf < ny && own_c) {
          const cf a = hr[slot(Kc, NU + 2, R)], m = hr[slot(Kc, NU + 1, R)], c = hr[slot(Kc, NU, R)];
          co[(size_t)(yf >> 1) * nxc + ci] =
              mk<float>(0.0625f * (a.re + 2.f * m.re + c.re), 0.0625f * (a.im + 2.f * m.im + c.im));
        }
      }
      {
        const int yv = i0 + k - (NU - 1);
        if (yv >= ys && yv < ys + seg && yv < ny)
          st2<true>(vo, (ptrdiff_t)yv * nx + g0, own && in0, own && in1, v[NU - 1][slot(Kc, NU - 1, R)]);
      }
    });
  }
  if (fail_at >= 0) ring_abort<S>(g, fail_at, fail_at + PFD + 1 < K ? fail_at + PFD + 1 : K, lane, err);
}

template <int NU, int NW, int MS>
__global__ void __launch_bounds__(32 * NW)
k_post_wt(const cf* __restrict__ bin, size_t b_stride, const double* __restrict__ bscale, size_t scale_stride,
          const cf* __restrict__ wD, const cf* __restrict__ vpre, size_t v_stride, const cf* __restrict__ ec,
          size_t ec_stride, int nxc, int nyc, cf* __restrict__ out, size_t out_stride, int nx, int ny, float ih,
          float om1, int nstrips, int nwarps, int seg, const RhsState* __restrict__ st, int* __restrict__ err) {
  static_assert(NU >= 1, "the wavefront post kernel ends with a sweep");
  using G = PostW<NU, 1>;
  constexpr int HX = G::HX, XO = G::XO, R = G::R;
  constexpr int S = RingLen<G::P, NU, MS>::S;
  constexpr int PFD = S - NU - 1;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int rhs = blockIdx.z;
  if (st && !st[rhs].active) return;
  const int w = blockIdx.x * NW + (threadIdx.x >> 5);
  if (w >= nwarps) return;
  const int lane = threadIdx.x & 31;
  const int xs = (w % nstrips) * XO, ys = (w / nstrips) * seg;
  const int g0 = xs - HX + 2 * lane;
  const bool in0 = g0 >= 0 && g0 < nx, in1 = g0 + 1 >= 0 && g0 + 1 < nx;
  const bool own = lane >= HX / 2 && lane < HX / 2 + XO / 2;
  const int ci = g0 >> 1;
  const bool okc0 = ci >= 0 && ci < nxc, okc1 = ci + 1 >= 0 && ci + 1 < nxc;
  const float sc = bscale ? (float)bscale[rhs * scale_stride] : 1.f;
  const cf* __restrict__ bb = bin + rhs * b_stride;
  const cf* __restrict__ vp = vpre + rhs * v_stride;
  const cf* __restrict__ eb = ec + rhs * ec_stride;
  cf* __restrict__ o = out + rhs * out_stride;
  const int i0 = ys - NU;
  const int rows = ny - ys < seg ? ny - ys : seg;
  const int K = (rows + 2 * NU + S - 1) / S * S;
  const Ring g = ring_begin<NW, S>(smem_raw, xs - HX, nx, ny, i0, lane);
  // slot arrays: 0 = v_pre, 1 = b, 2 = omega/D
  for (int r = 0; r < PFD && r < K; ++r) g.issue(r, r, lane, vp, bb, wD);

  const int e0 = clampi(ci, 0, nxc - 1), e1 = clampi(ci + 1, 0, nxc - 1);
  auto load_e = [&](int c) {
    E2 e;
    if (c >= 0 && c < nyc) {
      const cf* row = eb + (size_t)c * nxc;
      e.c0 = sel(okc0, row[e0]);
      e.c1 = sel(okc1, row[e1]);
    } else {
      e.c0 = e.c1 = czero<float>();
    }
    return e;
  };
  E2 ea = load_e(i0 >> 1), enext = ea;
  if (i0 & 1) enext = load_e((i0 >> 1) + 1);
  C2 v[NU][R];
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int s = 0; s < NU; ++s) v[s][i] = c2zero();
  int fail_at = -1;   // as in k_pre_wt
  for (int kb = 0; kb < K; kb += S) {
    const uint32_t par = (uint32_t)((kb / S) & 1);
    unroll<S>([&](auto KC) {
      constexpr int Kc = decltype(KC)::value;
      constexpr bool odd = ((Kc + NU) & 1) != 0;
      const int k = kb + Kc;
      __syncwarp();
      if (fail_at < 0) {
        if (k + PFD < K) g.issue(k + PFD, (Kc + PFD) % S, lane, vp, bb, wD);
        if (!__all_sync(kFull, g.wait(Kc, par))) fail_at = k;
      }
      const int y = i0 + k;
      C2 pe;
      if constexpr (!odd) {
        pe.a = ea.c0;
        pe.b = 0.5f * (ea.c0 + ea.c1);
        enext = load_e((y >> 1) + 1);
      } else {
        const cf m0 = 0.5f * (ea.c0 + enext.c0), m1 = 0.5f * (ea.c1 + enext.c1);
        pe.a = m0;
        pe.b = 0.5f * (m0 + m1);
        ea = enext;
      }
      const bool oky = y >= 0 && y < ny;
      constexpr int s0 = slot(Kc, 0, R);
      {
        const C2 vpk = g.get(Kc, 0);
        v[0][s0].a = sel(oky && in0, vpk.a + pe.a);
        v[0][s0].b = sel(oky && in1, vpk.b + pe.b);
      }
      unroll<NU - 1>([&](auto SC) {
        constexpr int s = decltype(SC)::value + 1;
        constexpr int so = slot(Kc, s, R);
        constexpr int gs = slot(Kc, s, S);
        v[s][so] = jac_row(v[s - 1][slot(Kc, s + 1, R)], v[s - 1][so], v[s - 1][slot(Kc, s - 1, R)],
                           scale2(sc, g.get(gs, 1)), g.get(gs, 2), ih, om1);
      });
      {
        constexpr int so = slot(Kc, NU, R);
        constexpr int gs = slot(Kc, NU, S);
        const C2 vn = jac_row(v[NU - 1][slot(Kc, NU + 1, R)], v[NU - 1][so], v[NU - 1][slot(Kc, NU - 1, R)],
                              scale2(sc, g.get(gs, 1)), g.get(gs, 2), ih, om1);
        const int yv = y - NU;
        if (yv >= ys && yv < ys + seg && yv < ny) st2<true>(o, (ptrdiff_t)yv * nx + g0, own && in0, own && in1, vn);
      }
    });
  }
  if (fail_at >= 0) ring_abort<S>(g, fail_at, fail_at + PFD + 1 < K ? fail_at + PFD + 1 : K, lane, err);
}

// ---------------------------------------------------------------- lane-private rings (cp.async)
// The same wavefront with a ring of S rows in shared memory that every lane fills for its own two
// columns with 16-byte cp.async copies (zero-filled for points outside the grid, so reads need no
// checks and omega/D is 0 outside the grid), one commit group per row; a lane only ever reads back
// what it copied itself, so the ring needs no barrier, and `cp.async.wait_group` keeps S - nu - 1
// rows in flight ahead of the row being computed.  S is a multiple of the unroll period (slot
// offsets are compile-time constants).  16-byte path only.

template <int NW, int S>
struct LaneRingSmem {
  __host__ __device__ static constexpr size_t bytes() { return (size_t)NW * S * 3 * 32 * 16; }
};

__device__ __forceinline__ void cp16(uint32_t dst, const void* src, uint32_t n) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp8(uint32_t dst, const void* src, uint32_t n) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

struct LaneRing {
  const cf* mine;      // this lane's 16 bytes of slot 0, array 0 (consecutive lanes consecutive)
  uint32_t base;       // its shared-space address
  int i0, ny, nx, g0;
  bool in0;

  // row r into slot s: the lane's columns of the three arrays, then one commit group; array 0 may
  // be stored in FP16 (8 bytes for the lane's two points, in the first half of its 16-byte cell)
  template <typename A0>
  __device__ __forceinline__ void issue(int r, int s, const A0* a0, const cf* a1, const cf* a2) const {
    const int y = i0 + r;
    const bool ok = in0 && y >= 0 && y < ny;
    const size_t off = ok ? (size_t)y * nx + g0 : 0;
    const uint32_t d = base + (uint32_t)(s * 3) * 512u;
    if constexpr (std::is_same<A0, __half2>::value) cp8(d, a0 + off, ok ? 8u : 0u);
    else cp16(d, a0 + off, ok ? 16u : 0u);
    cp16(d + 512u, a1 + off, ok ? 16u : 0u);
    cp16(d + 1024u, a2 + off, ok ? 16u : 0u);
    cp_commit();
  }
  __device__ __forceinline__ C2 get(int s, int a) const { return lds2(mine + (s * 3 + a) * 64); }
  // array 0 of slot s stored as FP16
  __device__ __forceinline__ C2 get_h(int s) const {
    const uint2 u = *reinterpret_cast<const uint2*>(mine + (s * 3) * 64);
    C2 r;
    r.a = from_h2(*reinterpret_cast<const __half2*>(&u.x));
    r.b = from_h2(*reinterpret_cast<const __half2*>(&u.y));
    return r;
  }
  template <typename A0>
  __device__ __forceinline__ C2 get0(int s) const {
    if constexpr (std::is_same<A0, __half2>::value) return get_h(s);
    else return get(s, 0);
  }
};

template <int NW, int S>
__device__ __forceinline__ LaneRing lane_ring_begin(unsigned char* smem, int nx, int ny, int i0, int g0, bool in0,
                                                    int lane) {
  const int wib = threadIdx.x >> 5;
  LaneRing g;
  cf* buf = reinterpret_cast<cf*>(smem) + (size_t)wib * S * 3 * 64;
  g.mine = buf + 2 * lane;
  g.base = smem_u32(g.mine);
  g.i0 = i0;
  g.ny = ny;
  g.nx = nx;
  g.g0 = g0;
  g.in0 = in0;
  // rows before the first one are read (never used for a result) before they are copied
  float4* z = reinterpret_cast<float4*>(const_cast<cf*>(g.mine));
#pragma unroll
  for (int i = 0; i < S * 3; ++i) z[i * 32] = make_float4(0.f, 0.f, 0.f, 0.f);
  return g;
}

// VT: storage of v_pre (cf, or __half2 for FP16 storage).  smul multiplies the right-hand side's
// scale: the cycle is linear, so every output (v_pre, the restricted residual and, through the
// coarser levels and the post kernel, z) is smul times the cycle of the scaled input.
template <int NU, int NW, int MS, typename VT = cf>
__global__ void __launch_bounds__(32 * NW)
k_pre_wa(const cf* __restrict__ bin, size_t b_stride, const double* __restrict__ bscale, size_t scale_stride,
         const cf* __restrict__ D, const cf* __restrict__ wD, VT* __restrict__ vpre, size_t v_stride,
         cf* __restrict__ bc, size_t bc_stride, int nx, int ny, int nxc, float ih, float om1, int nstrips,
         int nwarps, int seg, const RhsState* __restrict__ st, float smul) {
  static_assert(NU >= 1, "the wavefront pre kernel starts with one pointwise sweep");
  using G = PreW<NU, 1>;
  constexpr int H = G::H, HX = G::HX, XO = G::XO, R = G::R;
  constexpr int S = RingLen<G::P, NU, MS>::S;   // also the unroll period
  constexpr int PFD = S - NU - 1;                // rows in flight ahead of the current one
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int rhs = blockIdx.z;
  if (st && !st[rhs].active) return;
  const int w = blockIdx.x * NW + (threadIdx.x >> 5);
  if (w >= nwarps) return;
  const int lane = threadIdx.x & 31;
  const int xs = (w % nstrips) * XO, ys = (w / nstrips) * seg;
  const int g0 = xs - HX + 2 * lane;
  const bool in0 = g0 >= 0 && g0 < nx, in1 = g0 + 1 >= 0 && g0 + 1 < nx;
  const bool own = lane >= HX / 2 && lane < HX / 2 + XO / 2;
  const int ci = g0 >> 1;
  const bool own_c = own && g0 >= 0 && ci < nxc;
  const float sc = smul * (bscale ? (float)bscale[rhs * scale_stride] : 1.f);
  const float fw = 0.0625f * sc;   // full-weighting factor 1/16 times the right-hand side's scale
  const cf* __restrict__ bb = bin + rhs * b_stride;
  VT* __restrict__ vo = vpre + rhs * v_stride;
  cf* __restrict__ co = bc + rhs * bc_stride;
  const int i0 = ys - H;
  int rows = ny - ys < seg ? ny - ys : seg;
  rows = (rows + 1) & ~1;
  const int K = (rows + 2 * H - 1 + S - 1) / S * S;
  const LaneRing g = lane_ring_begin<NW, S>(smem_raw, nx, ny, i0, g0, in0, lane);
  // slot arrays: 0 = b, 1 = omega/D, 2 = D
#pragma unroll
  for (int r = 0; r < PFD; ++r) g.issue(r, r, bb, wD, D);

  C2 v[NU][R];
  cf hr[R];
#pragma unroll
  for (int i = 0; i < R; ++i) {
#pragma unroll
    for (int s = 0; s < NU; ++s) v[s][i] = c2zero();
    hr[i] = czero<float>();
  }
  for (int kb = 0; kb < K; kb += S) {
    unroll<S>([&](auto KC) {
      constexpr int Kc = decltype(KC)::value;
      const int k = kb + Kc;
      g.issue(k + PFD, (Kc + PFD) % S, bb, wD, D);   // rows past the end read as zeros
      cp_wait<PFD>();
      // the cycle is linear: the stages run on b unscaled and the two outputs are scaled by sc
      constexpr int s0 = slot(Kc, 0, R);
      {
        const C2 b0 = g.get(Kc, 0), wd = g.get(Kc, 1);
        v[0][s0].a = wd.a * b0.a;
        v[0][s0].b = wd.b * b0.b;
      }
      unroll<NU - 1>([&](auto SC) {
        constexpr int s = decltype(SC)::value + 2;
        constexpr int so = slot(Kc, s - 1, R);
        constexpr int gs = slot(Kc, s - 1, S);
        v[s - 1][so] = jac_row(v[s - 2][slot(Kc, s, R)], v[s - 2][so], v[s - 2][slot(Kc, s - 2, R)],
                               g.get(gs, 0), g.get(gs, 1), ih, om1);
      });
      {
        constexpr int sr = slot(Kc, NU, R);
        constexpr int gs = slot(Kc, NU, S);
        const int yr = i0 + k - NU;
        const bool okr = yr >= 0 && yr < ny;
        const C2 sb = g.get(gs, 0), dd = g.get(gs, 2);
        const C2& up = v[NU - 1][slot(Kc, NU + 1, R)];
        const C2& mid = v[NU - 1][sr];
        const C2& dn = v[NU - 1][slot(Kc, NU - 1, R)];
        const cf left = shfl_up1(mid.b), right = shfl_dn1(mid.a);
        const cf r0 = sel(okr && in0, res_pt(mid.a, left, mid.b, up.a, dn.a, sb.a, dd.a, ih));
        const cf r1 = sel(okr && in1, res_pt(mid.b, mid.a, right, up.b, dn.b, sb.b, dd.b, ih));
        const cf rl = shfl_up1(r1);
        hr[sr] = mk<float>(rl.re + 2.f * r0.re + r1.re, rl.im + 2.f * r0.im + r1.im);
      }
      if constexpr (Kc % 2 == 0) {
        const int yf = i0 + k - NU - 1;
        if (k >= 2 * H && yf < ys + rows && yf < ny && own_c) {
          const cf a = hr[slot(Kc, NU + 2, R)], m = hr[slot(Kc, NU + 1, R)], c = hr[slot(Kc, NU, R)];
          co[(size_t)(yf >> 1) * nxc + ci] =
              mk<float>(fw * (a.re + 2.f * m.re + c.re), fw * (a.im + 2.f * m.im + c.im));
        }
      }
      {
        const int yv = i0 + k - (NU - 1);
        if (yv >= ys && yv < ys + seg && yv < ny)
          st2v<VT>(vo, (ptrdiff_t)yv * nx + g0, own && in0, own && in1, scale2(sc, v[NU - 1][slot(Kc, NU - 1, R)]));
      }
    });
  }
  cp_wait<0>();   // the copies of rows past the end
}

// VT: storage of v_pre, OT: storage of the result (cf, or __half2 for FP16 storage); smul as in
// k_pre_wa (the same factor must reach both kernels of a cycle).
template <int NU, int NW, int MS, typename VT = cf, typename OT = cf>
__global__ void __launch_bounds__(32 * NW)
k_post_wa(const cf* __restrict__ bin, size_t b_stride, const double* __restrict__ bscale, size_t scale_stride,
          const cf* __restrict__ wD, const VT* __restrict__ vpre, size_t v_stride, const cf* __restrict__ ec,
          size_t ec_stride, int nxc, int nyc, OT* __restrict__ out, size_t out_stride, int nx, int ny, float ih,
          float om1, int nstrips, int nwarps, int seg, const RhsState* __restrict__ st, float smul) {
  static_assert(NU >= 1, "the wavefront post kernel ends with a sweep");
  using G = PostW<NU, 1>;
  constexpr int HX = G::HX, XO = G::XO, R = G::R;
  constexpr int S = RingLen<G::P, NU, MS>::S;
  constexpr int PFD = S - NU - 1;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int rhs = blockIdx.z;
  if (st && !st[rhs].active) return;
  const int w = blockIdx.x * NW + (threadIdx.x >> 5);
  if (w >= nwarps) return;
  const int lane = threadIdx.x & 31;
  const int xs = (w % nstrips) * XO, ys = (w / nstrips) * seg;
  const int g0 = xs - HX + 2 * lane;
  const bool in0 = g0 >= 0 && g0 < nx, in1 = g0 + 1 >= 0 && g0 + 1 < nx;
  const bool own = lane >= HX / 2 && lane < HX / 2 + XO / 2;
  const int ci = g0 >> 1;
  const bool okc0 = ci >= 0 && ci < nxc, okc1 = ci + 1 >= 0 && ci + 1 < nxc;
  const float sc = smul * (bscale ? (float)bscale[rhs * scale_stride] : 1.f);
  const cf* __restrict__ bb = bin + rhs * b_stride;
  const VT* __restrict__ vp = vpre + rhs * v_stride;
  const cf* __restrict__ eb = ec + rhs * ec_stride;
  OT* __restrict__ o = out + rhs * out_stride;
  const int i0 = ys - NU;
  const int rows = ny - ys < seg ? ny - ys : seg;
  const int K = (rows + 2 * NU + S - 1) / S * S;
  const LaneRing g = lane_ring_begin<NW, S>(smem_raw, nx, ny, i0, g0, in0, lane);
  // slot arrays: 0 = v_pre, 1 = b, 2 = omega/D
#pragma unroll
  for (int r = 0; r < PFD; ++r) g.issue(r, r, vp, bb, wD);

  const int e0 = clampi(ci, 0, nxc - 1), e1 = clampi(ci + 1, 0, nxc - 1);
  auto load_e = [&](int c) {
    E2 e;
    if (c >= 0 && c < nyc) {
      const cf* row = eb + (size_t)c * nxc;
      e.c0 = sel(okc0, row[e0]);
      e.c1 = sel(okc1, row[e1]);
    } else {
      e.c0 = e.c1 = czero<float>();
    }
    return e;
  };
  E2 ea = load_e(i0 >> 1), enext = ea;
  if (i0 & 1) enext = load_e((i0 >> 1) + 1);
  C2 v[NU][R];
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int s = 0; s < NU; ++s) v[s][i] = c2zero();
  for (int kb = 0; kb < K; kb += S) {
    unroll<S>([&](auto KC) {
      constexpr int Kc = decltype(KC)::value;
      constexpr bool odd = ((Kc + NU) & 1) != 0;
      const int k = kb + Kc;
      g.issue(k + PFD, (Kc + PFD) % S, vp, bb, wD);
      const int y = i0 + k;
      C2 pe;
      if constexpr (!odd) {
        pe.a = ea.c0;
        pe.b = 0.5f * (ea.c0 + ea.c1);
        enext = load_e((y >> 1) + 1);
      } else {
        const cf m0 = 0.5f * (ea.c0 + enext.c0), m1 = 0.5f * (ea.c1 + enext.c1);
        pe.a = m0;
        pe.b = 0.5f * (m0 + m1);
        ea = enext;
      }
      cp_wait<PFD>();
      const bool oky = y >= 0 && y < ny;
      constexpr int s0 = slot(Kc, 0, R);
      {
        const C2 vpk = g.template get0<VT>(Kc);
        v[0][s0].a = sel(oky && in0, vpk.a + pe.a);
        v[0][s0].b = sel(oky && in1, vpk.b + pe.b);
      }
      unroll<NU - 1>([&](auto SC) {
        constexpr int s = decltype(SC)::value + 1;
        constexpr int so = slot(Kc, s, R);
        constexpr int gs = slot(Kc, s, S);
        v[s][so] = jac_row(v[s - 1][slot(Kc, s + 1, R)], v[s - 1][so], v[s - 1][slot(Kc, s - 1, R)],
                           scale2(sc, g.get(gs, 1)), g.get(gs, 2), ih, om1);
      });
      {
        constexpr int so = slot(Kc, NU, R);
        constexpr int gs = slot(Kc, NU, S);
        const C2 vn = jac_row(v[NU - 1][slot(Kc, NU + 1, R)], v[NU - 1][so], v[NU - 1][slot(Kc, NU - 1, R)],
                              scale2(sc, g.get(gs, 1)), g.get(gs, 2), ih, om1);
        const int yv = y - NU;
        if (yv >= ys && yv < ys + seg && yv < ny) st2v<OT>(o, (ptrdiff_t)yv * nx + g0, own && in0, own && in1, vn);
      }
    });
  }
  cp_wait<0>();
}


// Geometry of the post kernel with the fused operator product (k_post_waf): the product A z is one
// more stencil stage that reads across the strip edge, and it needs z one row above and below the
// segment.
template <int NU, int PF>
struct PostWF {
  static constexpr int H = NU + 1, HX = (NU + 2) & ~1, XO = 64 - 2 * HX;
  static constexpr int R = NU + 1 > 3 ? NU + 1 : 3;
  static constexpr int P = lcm_c(lcm_c(R, 2), PF);
};

// k_post_wa followed, one row behind its last sweep, by the operator product of the s-step basis:
// w = A z on the stored z (FP32; the FP16-rounded values if OT is FP16 storage), written as the
// FP32 basis vector v_{k+1} (vout), with the same operations as k_ss_matvec2, and the sum of
// |w|^2 over the strip's owned points of each row pair (2i, 2i + 1) in
// npart[(rhs * ceil(ny / 2) + i) * nstrips + strip] (FP32; a fixed warp butterfly, so the partials
// do not depend on the segment length or warps per block).
// DA32: the FP32 diagonal of A (complex, row-major like the level).
template <int NU, int NW, int MS, typename VT = cf, typename OT = cf>
__global__ void __launch_bounds__(32 * NW)
k_post_waf(const cf* __restrict__ bin, size_t b_stride, const double* __restrict__ bscale, size_t scale_stride,
           const cf* __restrict__ wD, const VT* __restrict__ vpre, size_t v_stride, const cf* __restrict__ ec,
           size_t ec_stride, int nxc, int nyc, OT* __restrict__ out, size_t out_stride, int nx, int ny, float ih,
           float om1, int nstrips, int nwarps, int seg, const RhsState* __restrict__ st, float smul,
           const cf* __restrict__ DA32, float ih0, cf* __restrict__ vout, size_t vout_stride,
           float* __restrict__ npart) {
  static_assert(NU >= 1, "the wavefront post kernel ends with a sweep");
  using G = PostWF<NU, 1>;
  constexpr int HX = G::HX, XO = G::XO, R = G::R;
  constexpr int S = RingLen<G::P, NU, MS>::S;
  constexpr int PFD = S - NU - 1;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int rhs = blockIdx.z;
  if (st && !st[rhs].active) return;
  const int w = blockIdx.x * NW + (threadIdx.x >> 5);
  if (w >= nwarps) return;
  const int lane = threadIdx.x & 31;
  const int strip = w % nstrips;
  const int xs = strip * XO, ys = (w / nstrips) * seg;
  const int g0 = xs - HX + 2 * lane;
  const bool in0 = g0 >= 0 && g0 < nx, in1 = g0 + 1 >= 0 && g0 + 1 < nx;
  const bool own = lane >= HX / 2 && lane < HX / 2 + XO / 2;
  const int ci = g0 >> 1;
  const bool okc0 = ci >= 0 && ci < nxc, okc1 = ci + 1 >= 0 && ci + 1 < nxc;
  const float sc = smul * (bscale ? (float)bscale[rhs * scale_stride] : 1.f);
  const cf* __restrict__ bb = bin + rhs * b_stride;
  const VT* __restrict__ vp = vpre + rhs * v_stride;
  const cf* __restrict__ eb = ec + rhs * ec_stride;
  OT* __restrict__ o = out + rhs * out_stride;
  cf* __restrict__ vo = vout + rhs * vout_stride;
  float* __restrict__ np = npart + (size_t)rhs * ((ny + 1) >> 1) * nstrips + strip;
  float nrm_even = 0.f;   // |w|^2 of the even row of the current row pair
  const int i0 = ys - NU - 1;
  const int rows = ny - ys < seg ? ny - ys : seg;
  const int K = (rows + 2 * NU + 2 + S - 1) / S * S;
  const LaneRing g = lane_ring_begin<NW, S>(smem_raw, nx, ny, i0, g0, in0, lane);
  // slot arrays: 0 = v_pre, 1 = b, 2 = omega/D
#pragma unroll
  for (int r = 0; r < PFD; ++r) g.issue(r, r, vp, bb, wD);

  const int e0 = clampi(ci, 0, nxc - 1), e1 = clampi(ci + 1, 0, nxc - 1);
  auto load_e = [&](int c) {
    E2 e;
    if (c >= 0 && c < nyc) {
      const cf* row = eb + (size_t)c * nxc;
      e.c0 = sel(okc0, row[e0]);
      e.c1 = sel(okc1, row[e1]);
    } else {
      e.c0 = e.c1 = czero<float>();
    }
    return e;
  };
  E2 ea = load_e(i0 >> 1), enext = ea;
  if (i0 & 1) enext = load_e((i0 >> 1) + 1);
  C2 v[NU][R];
  C2 zr[R];   // the stored z of the last rows (0 outside the grid)
#pragma unroll
  for (int i = 0; i < R; ++i) {
#pragma unroll
    for (int s = 0; s < NU; ++s) v[s][i] = c2zero();
    zr[i] = c2zero();
  }
  for (int kb = 0; kb < K; kb += S) {
    unroll<S>([&](auto KC) {
      constexpr int Kc = decltype(KC)::value;
      constexpr bool odd = ((Kc + NU + 1) & 1) != 0;   // parity of y (ys and S are even)
      const int k = kb + Kc;
      g.issue(k + PFD, (Kc + PFD) % S, vp, bb, wD);
      const int y = i0 + k;
      // the diagonal of A on the product's row (read from L2 while the sweeps run)
      const int ya = y - NU - 1;
      const bool oka = ya >= 0 && ya < ny && in0;
      const float4 da = __ldg(reinterpret_cast<const float4*>(DA32 + (oka ? (size_t)ya * nx + g0 : 0)));
      C2 pe;
      if constexpr (!odd) {
        pe.a = ea.c0;
        pe.b = 0.5f * (ea.c0 + ea.c1);
        enext = load_e((y >> 1) + 1);
      } else {
        const cf m0 = 0.5f * (ea.c0 + enext.c0), m1 = 0.5f * (ea.c1 + enext.c1);
        pe.a = m0;
        pe.b = 0.5f * (m0 + m1);
        ea = enext;
      }
      cp_wait<PFD>();
      const bool oky = y >= 0 && y < ny;
      constexpr int s0 = slot(Kc, 0, R);
      {
        const C2 vpk = g.template get0<VT>(Kc);
        v[0][s0].a = sel(oky && in0, vpk.a + pe.a);
        v[0][s0].b = sel(oky && in1, vpk.b + pe.b);
      }
      unroll<NU - 1>([&](auto SC) {
        constexpr int s = decltype(SC)::value + 1;
        constexpr int so = slot(Kc, s, R);
        constexpr int gs = slot(Kc, s, S);
        v[s][so] = jac_row(v[s - 1][slot(Kc, s + 1, R)], v[s - 1][so], v[s - 1][slot(Kc, s - 1, R)],
                           scale2(sc, g.get(gs, 1)), g.get(gs, 2), ih, om1);
      });
      {
        constexpr int so = slot(Kc, NU, R);
        constexpr int gs = slot(Kc, NU, S);
        const C2 vn = jac_row(v[NU - 1][slot(Kc, NU + 1, R)], v[NU - 1][so], v[NU - 1][slot(Kc, NU - 1, R)],
                              scale2(sc, g.get(gs, 1)), g.get(gs, 2), ih, om1);
        const int yv = y - NU;
        if (yv >= ys && yv < ys + seg && yv < ny) st2v<OT>(o, (ptrdiff_t)yv * nx + g0, own && in0, own && in1, vn);
        if constexpr (std::is_same<OT, __half2>::value) {   // the product reads what was stored
          zr[so].a = from_h2(to_h2(vn.a));
          zr[so].b = from_h2(to_h2(vn.b));
        } else {
          zr[so] = vn;
        }
      }
      {
        // w = A z on row ya = y - nu - 1: rows ya - 1, ya, ya + 1 of z
        const C2& zu = zr[slot(Kc, NU + 2, R)];
        const C2& zm = zr[slot(Kc, NU + 1, R)];
        const C2& zd = zr[slot(Kc, NU, R)];
        const cf zl = shfl_up1(zm.b), zrt = shfl_dn1(zm.a);
        const float s0r = (zl.re + zm.b.re) + (zu.a.re + zd.a.re), s0i = (zl.im + zm.b.im) + (zu.a.im + zd.a.im);
        const float s1r = (zm.a.re + zrt.re) + (zu.b.re + zd.b.re), s1i = (zm.a.im + zrt.im) + (zu.b.im + zd.b.im);
        const float w0r = fmaf(da.x, zm.a.re, fmaf(-da.y, zm.a.im, -ih0 * s0r));
        const float w0i = fmaf(da.x, zm.a.im, fmaf(da.y, zm.a.re, -ih0 * s0i));
        const float w1r = fmaf(da.z, zm.b.re, fmaf(-da.w, zm.b.im, -ih0 * s1r));
        const float w1i = fmaf(da.z, zm.b.im, fmaf(da.w, zm.b.re, -ih0 * s1i));
        const bool rowok = ya >= ys && ya < ys + seg && ya < ny;
        const bool put = rowok && own && in0;
        if (put) *reinterpret_cast<float4*>(vo + (ptrdiff_t)ya * nx + g0) = make_float4(w0r, w0i, w1r, w1i);
        const float nrm = put ? fmaf(w0r, w0r, fmaf(w0i, w0i, fmaf(w1r, w1r, w1i * w1i))) : 0.f;
        // rows pair up as (2i, 2i + 1) (segments start on even rows and are of even length; ya has
        // the parity of Kc): the pair's sum over the strip goes to npart[(rhs ny2 + i) nstrips + strip]
        if constexpr (Kc % 2 == 0) {
          nrm_even = nrm;
        } else {
          float t = nrm_even + nrm;
#pragma unroll
          for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(kFull, t, off);
          const int y2 = ya - 1;
          if (y2 >= ys && y2 < ys + seg && y2 < ny && lane == 0) np[(size_t)(y2 >> 1) * nstrips] = t;
        }
      }
    });
  }
  cp_wait<0>();
}

}  // namespace wave
}  // namespace mgh
