// The coarse tail of the multigrid cycle in one kernel: one thread block per right-hand side runs
// every cycle of levels l0 .. L-1 (Alg. 2 with its CycleType recursion: damped-Jacobi smoothing,
// residual, full-weighting restriction, exact coarsest solve, bilinear prolongation and
// correction) with all of that right-hand side's fields in shared memory.
//
// Below some level a multigrid level is too small to fill the GPU: its kernels run for a few
// microseconds on a few blocks and the cycle is bound by launch latency (the W-cycle visits level l
// CycleType^(l-1) times per cycle).  From the first level l0 whose fields fit in a block's shared
// memory on, each right-hand side is independent and small (a 73 x 73 level holds 43 KB of complex
// FP32), so a block keeps the right-hand side and iterate of every tail level, plus one scratch
// field, on chip and synchronises with __syncthreads() between the steps of the cycle.
//
// Arithmetic is that of the level kernels: Jacobi v <- (1 - w) v + (w / D)(b + (sum of
// neighbours)/h^2) (the first sweep from v = 0 is (w / D) b), residual b - (D v - (sum)/h^2), the
// 1/16 [1 2 1; 2 4 2; 1 2 1] restriction onto coarse point (i, j) at fine (2i, 2j), prolongation by
// parity with weights 1, 1/2, 1/4, every sample outside a grid read as 0, and the coarsest solve
// as the product with the dense inverse.  A later cycle of a level starts from that level's last
// iterate (Alg. 2); the exact coarsest solve gives the same result every time, so it runs once
// per visit of the level above it.
#include <algorithm>

#include "mgh_engine.h"

namespace mgh {

namespace {

constexpr int kTailThreads = 1024;
constexpr size_t kTailSmemMax = 200 * 1024;

template <typename T>
struct TailLevel {
  const Cx<T>* D;      // diagonal of K_kappa on this level
  const Cx<T>* wd;     // omega / D
  int nx, ny, nu1, nu2;
  int pitch;           // nx + 2: fields carry a border of zeros one point wide
  int dx, dy;          // a step of kTailThreads points in row-major order: dy rows and dx columns
  int off_b, off_v;    // element offsets of the right-hand side and iterate (bordered)
  int off_t;           // scratch field (bordered; on the coarsest level a plain copy of b)
  T inv_h2;
};

template <typename T>
struct TailArgs {
  TailLevel<T> lv[kMaxLevels];  // index 0 = level l0
  int depth;                    // tail levels, the coarsest included (>= 2)
  int gamma;                    // CycleType
  int reps;                     // cycles of level l0 (the level above runs it CycleType times)
  int total;                    // elements of shared memory in use
  T om1;                        // 1 - omega
  const Cx<T>* b_in;            // right-hand sides of level l0, b_in + rhs * stride
  Cx<T>* v_out;                 // results on level l0, v_out + rhs * stride
  size_t stride;
  const Cx<T>* kinv;            // coarsest inverse, row-major [nc][nc]
  const RhsState* st;
};

// Every interior point of a level once, kTailThreads apart in row-major order: k is the plain
// index y * nx + x (of the coefficient arrays), i the bordered index (y + 1) * pitch + x + 1.
// The body runs as body(k, i, x, y).
template <typename T, typename Body>
__device__ __forceinline__ void for_points(const TailLevel<T>& L, Body&& body) {
  const int n = L.nx * L.ny;
  int y = threadIdx.x / L.nx, x = threadIdx.x - y * L.nx;
  for (int k = threadIdx.x; k < n; k += kTailThreads) {
    body(k, k + 2 * y + L.pitch + 1, x, y);
    x += L.dx;
    y += L.dy;
    if (x >= L.nx) { x -= L.nx; ++y; }
  }
}

// `sweeps` damped-Jacobi sweeps on K v = b, from v = 0 when `zero`, starting from the iterate in
// field `cur` (off_v or off_t of the level); returns the field that holds the result (a level's
// iterate lives in whichever of its two fields the last sweep wrote: no copy pass).
template <typename T>
__device__ int tail_smooth(Cx<T>* sm, const TailLevel<T>& L, int cur, int sweeps, bool zero, T om1) {
  const Cx<T>* b = sm + L.off_b;
  const int P = L.pitch;
  int s = 0;
  if (zero) {
    Cx<T>* v = sm + cur;
    for_points(L, [&](int k, int i, int, int) { v[i] = sweeps > 0 ? L.wd[k] * b[i] : czero<T>(); });
    __syncthreads();
    s = 1;
  }
  for (; s < sweeps; ++s) {
    const Cx<T>* src = sm + cur;
    const int nxt = cur == L.off_v ? L.off_t : L.off_v;
    Cx<T>* dst = sm + nxt;
    for_points(L, [&](int k, int i, int, int) {
      const Cx<T> nb = src[i - 1] + src[i + 1] + src[i - P] + src[i + P];
      const Cx<T> bk = b[i];
      const Cx<T> t = mk<T>(bk.re + L.inv_h2 * nb.re, bk.im + L.inv_h2 * nb.im);
      const Cx<T> c = src[i], w = L.wd[k];
      dst[i] = mk<T>(om1 * c.re + w.re * t.re - w.im * t.im, om1 * c.im + w.re * t.im + w.im * t.re);
    });
    __syncthreads();
    cur = nxt;
  }
  return cur;
}

// r = b - K v (v in field `cur`) into the level's other field, then its full-weighting restriction
// into the next level's b.
template <typename T>
__device__ void tail_restrict(Cx<T>* sm, const TailLevel<T>& L, int cur, const TailLevel<T>& C) {
  const Cx<T>* v = sm + cur;
  const Cx<T>* b = sm + L.off_b;
  Cx<T>* r = sm + (cur == L.off_v ? L.off_t : L.off_v);
  const int P = L.pitch;
  for_points(L, [&](int k, int i, int, int) {
    const Cx<T> s = v[i - 1] + v[i + 1] + v[i - P] + v[i + P];
    const Cx<T> kv = L.D[k] * v[i] - L.inv_h2 * s;
    r[i] = b[i] - kv;
  });
  __syncthreads();
  Cx<T>* bc = sm + C.off_b;
  const T q16 = T(1) / T(16);
  for_points(C, [&](int, int ic, int ci, int cj) {
    const int i = (2 * cj + 1) * P + 2 * ci + 1;   // fine point (2 ci, 2 cj)
    const Cx<T> e = r[i - 1] + r[i + 1] + r[i - P] + r[i + P];
    const Cx<T> c = r[i - P - 1] + r[i - P + 1] + r[i + P - 1] + r[i + P + 1];
    const Cx<T> rc = r[i];
    bc[ic] = mk<T>(q16 * (T(4) * rc.re + T(2) * e.re + c.re), q16 * (T(4) * rc.im + T(2) * e.im + c.im));
  });
  __syncthreads();
}

// v += P e, v in field `cur` of L and e in field `ccur` of C (bilinear by parity; the zero border
// supplies coarse samples outside the coarse grid).
template <typename T>
__device__ void tail_prolong(Cx<T>* sm, const TailLevel<T>& L, int cur, const TailLevel<T>& C, int ccur) {
  Cx<T>* v = sm + cur;
  const Cx<T>* e = sm + ccur;
  const int PC = C.pitch;
  for_points(L, [&](int, int i, int x, int y) {
    const int ic = ((y >> 1) + 1) * PC + (x >> 1) + 1;
    const bool ox = x & 1, oy = y & 1;
    Cx<T> p;
    if (!ox && !oy) {
      p = e[ic];
    } else if (ox && !oy) {
      p = T(0.5) * (e[ic] + e[ic + 1]);
    } else if (!ox && oy) {
      p = T(0.5) * (e[ic] + e[ic + PC]);
    } else {
      p = T(0.25) * (e[ic] + e[ic + 1] + e[ic + PC] + e[ic + PC + 1]);
    }
    v[i] = v[i] + p;
  });
  __syncthreads();
}

// Coarsest level: v = K^{-1} b, one warp per row of the inverse (read from L2), lanes over columns;
// b is first copied without its border into the level's scratch field.
template <typename T>
__device__ void tail_coarsest(Cx<T>* sm, const TailLevel<T>& L, const Cx<T>* __restrict__ kinv) {
  const Cx<T>* bb = sm + L.off_b;
  Cx<T>* b = sm + L.off_t;
  Cx<T>* v = sm + L.off_v;
  for_points(L, [&](int k, int i, int, int) { b[k] = bb[i]; });
  __syncthreads();
  const int n = L.nx * L.ny;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int r = warp; r < n; r += kTailThreads / 32) {
    const Cx<T>* row = kinv + (size_t)r * n;
    T ar = 0, ai = 0;
    for (int c = lane; c < n; c += 32) {
      const Cx<T> k = row[c], x = b[c];
      ar = fma(k.re, x.re, fma(-k.im, x.im, ar));
      ai = fma(k.re, x.im, fma(k.im, x.re, ai));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ar += __shfl_xor_sync(0xffffffffu, ar, o);
      ai += __shfl_xor_sync(0xffffffffu, ai, o);
    }
    if (lane == 0) {
      const int ry = r / L.nx, rx = r - ry * L.nx;
      v[(ry + 1) * L.pitch + rx + 1] = mk<T>(ar, ai);
    }
  }
  __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(kTailThreads, 1) k_tail(const TailArgs<T> a) {
  const int rhs = blockIdx.x;
  if (a.st && !a.st[rhs].active) return;
  extern __shared__ __align__(16) unsigned char tail_smem[];
  Cx<T>* sm = reinterpret_cast<Cx<T>*>(tail_smem);
  // zero everything once: the borders are never written afterwards
  for (int k = threadIdx.x; k < a.total; k += kTailThreads) sm[k] = czero<T>();
  __syncthreads();
  const TailLevel<T>& top = a.lv[0];
  const Cx<T>* bin = a.b_in + rhs * a.stride;
  {
    Cx<T>* b0 = sm + top.off_b;
    for_points(top, [&](int k, int i, int, int) { b0[i] = bin[k]; });
  }
  __syncthreads();

  const int last = a.depth - 1;
  int cnt[kMaxLevels];
  bool zero[kMaxLevels];
  int cur[kMaxLevels];   // field holding each level's iterate
  for (int d = 0; d < a.depth; ++d) cur[d] = a.lv[d].off_v;
  for (int rep = 0; rep < a.reps; ++rep) {
    // the state (d, down, cnt, zero, cur) is the same in every thread: all of them take every branch
    int d = 0;
    bool down = true;
    zero[0] = rep == 0;
    while (true) {
      if (down) {
        if (d == last) {                       // exact solve, once per visit of the level above
          tail_coarsest(sm, a.lv[d], a.kinv);
          cur[d] = a.lv[d].off_v;
          --d;
          down = false;
          cnt[d] = a.gamma - 1;
          continue;
        }
        cur[d] = tail_smooth(sm, a.lv[d], cur[d], a.lv[d].nu1, zero[d], a.om1);
        tail_restrict(sm, a.lv[d], cur[d], a.lv[d + 1]);
        cnt[d] = 0;
        zero[d + 1] = true;
        ++d;
        continue;
      }
      if (++cnt[d] < a.gamma) {                // next cycle of level d + 1 from its last iterate
        zero[d + 1] = false;
        ++d;
        down = true;
        continue;
      }
      tail_prolong(sm, a.lv[d], cur[d], a.lv[d + 1], cur[d + 1]);
      cur[d] = tail_smooth(sm, a.lv[d], cur[d], a.lv[d].nu2, false, a.om1);
      if (d == 0) break;
      --d;
    }
  }
  Cx<T>* vo = a.v_out + rhs * a.stride;
  const Cx<T>* v0 = sm + cur[0];
  for_points(top, [&](int k, int i, int, int) { vo[k] = v0[i]; });
}

// Shared-memory layout of a tail from level l0 (element offsets per level; returns the total):
// bordered right-hand side, iterate and scratch field on every level above the coarsest; on the
// coarsest, bordered right-hand side and iterate and a plain copy of the right-hand side.
template <typename T>
int tail_layout(const Handle& h, int l0, TailLevel<T>* lv) {
  int off = 0;
  for (int l = l0; l < h.L; ++l) {
    const Level& L = h.lev[l];
    const int ps = (L.nx + 2) * (L.ny + 2);
    TailLevel<T> t{};
    t.nx = L.nx; t.ny = L.ny; t.pitch = L.nx + 2;
    t.dx = kTailThreads % L.nx; t.dy = kTailThreads / L.nx;
    t.off_b = off; off += ps;
    t.off_v = off; off += ps;
    t.off_t = off; off += l + 1 < h.L ? ps : (int)L.n();
    if (lv) lv[l - l0] = t;
  }
  return off;
}

template <typename T>
size_t tail_smem_bytes(const Handle& h, int l0) {
  return (size_t)tail_layout<T>(h, l0, nullptr) * sizeof(Cx<T>);
}

template <typename T>
mgh_status launch_tail_t(Handle& h, int reps, int B, const RhsState* st) {
  const int l0 = h.tail_l0;
  TailArgs<T> a{};
  a.total = tail_layout<T>(h, l0, a.lv);
  for (int l = l0; l < h.L; ++l) {
    const Level& lv = h.lev[l];
    TailLevel<T>& t = a.lv[l - l0];
    t.D = (const Cx<T>*)lv.D;
    t.wd = (const Cx<T>*)lv.wDinv;
    t.nu1 = nu_pre(h, l); t.nu2 = nu_post(h, l);
    t.inv_h2 = static_cast<T>(1.0 / (lv.h * lv.h));
  }
  a.depth = h.L - l0;
  a.gamma = cycle_gamma(h);
  a.reps = reps;
  a.om1 = static_cast<T>(1.0 - h.p.omega);
  a.b_in = (const Cx<T>*)h.lev[l0].b;
  a.v_out = (Cx<T>*)h.lev[l0].vfin;
  a.stride = h.lev[l0].n();
  a.kinv = sizeof(T) == 8 ? (const Cx<T>*)(const void*)h.kinv64r : (const Cx<T>*)(const void*)h.kinv32;
  a.st = st;
  const size_t smem = (size_t)a.total * sizeof(Cx<T>);
  MGH_ONCE(MGH_CUDA(cudaFuncSetAttribute(k_tail<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTailSmemMax)););
  ProfScope ps(h, P_COARSE);
  k_tail<T><<<B, kTailThreads, smem, h.stream>>>(a);
  MGH_CHECK_LAUNCH(); h.launches++;
  return MGH_OK;
}

}  // namespace

bool tail_level_fits(const Handle& h, int l) {
  if (l < 1 || l + 2 > h.L) return false;
  const size_t bytes = h.fp64 ? tail_smem_bytes<double>(h, l) : tail_smem_bytes<float>(h, l);
  return bytes <= kTailSmemMax;
}

int choose_tail_level(const Handle& h) {
  for (int l = 1; l + 2 <= h.L; ++l) {
    const size_t bytes = h.fp64 ? tail_smem_bytes<double>(h, l) : tail_smem_bytes<float>(h, l);
    if (bytes <= kTailSmemMax) return l;
  }
  return 0;
}

mgh_status launch_tail(Handle& h, int reps, int B, const RhsState* st, bool fp64) {
  return fp64 ? launch_tail_t<double>(h, reps, B, st) : launch_tail_t<float>(h, reps, B, st);
}

}  // namespace mgh
