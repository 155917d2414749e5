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

#include <cooperative_groups.h>

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


// ---------------------------------------------------------------- the tail over a cluster
// The same cycle with each right-hand side split over a cluster of CL blocks by bands of rows:
// block r of the cluster owns rows [r band_l, (r + 1) band_l) of level l, with band_l = 2 band_{l+1}
// so that the rows a restriction or prolongation reads lie in the block's band or in the row just
// above or below it.  Each field holds the band plus one halo row on each side (and the zero
// column border); after every pass that writes a field whose vertical neighbours are read next,
// the blocks meet at a cluster barrier and copy their halo rows from the neighbouring blocks'
// shared memory.  The exact coarsest solve gathers the whole right-hand side from the cluster and
// each block forms its own rows of v = K^{-1} b (each block reads 1/CL of the inverse).  Every
// point and every row of the coarsest product is computed with the operations of k_tail, so the
// results do not depend on CL.
namespace cg = cooperative_groups;

template <typename T>
struct ClLevel {
  const Cx<T>* D;      // diagonal of K_kappa on this level
  const Cx<T>* wd;     // omega / D
  int nx, ny, nu1, nu2;
  int pitch;           // nx + 2
  int band;            // rows per block (the last blocks may own fewer, or none)
  int off_b, off_v, off_t;   // (band + 2) x pitch fields; off_t on the coarsest: the gathered b (nx * ny)
  T inv_h2;
};

template <typename T>
struct ClArgs {
  ClLevel<T> lv[kMaxLevels];
  int depth, gamma, reps, total, cl;
  T om1;
  const Cx<T>* b_in;
  Cx<T>* v_out;
  size_t stride;
  const Cx<T>* kinv;
  const RhsState* st;
};

// Rows [y0, y0 + rows) of a level owned by block `rank`.
template <typename T>
__device__ __forceinline__ void cl_rows(const ClLevel<T>& L, int rank, int& y0, int& rows) {
  y0 = rank * L.band;
  rows = L.ny - y0;
  rows = rows < 0 ? 0 : (rows > L.band ? L.band : rows);
}

// The owned points of a level, TPB apart in row-major order: body(k, i, x, y) with k the plain
// index of the level (coefficients), i the local bordered index, (x, y) the global point.
template <int TPB, typename T, typename Body>
__device__ __forceinline__ void cl_points(const ClLevel<T>& L, int y0, int rows, Body&& body) {
  const int n = rows * L.nx;
  const int dy = TPB / L.nx, dx = TPB - dy * L.nx;
  int yl = threadIdx.x / L.nx, x = threadIdx.x - yl * L.nx;
  for (int kl = threadIdx.x; kl < n; kl += TPB) {
    body((y0 + yl) * L.nx + x, (yl + 1) * L.pitch + x + 1, x, y0 + yl);
    x += dx;
    yl += dy;
    if (x >= L.nx) { x -= L.nx; ++yl; }
  }
}

// Cluster barrier, then the halo rows of field `off` from the neighbouring blocks (rows outside
// the grid stay 0), then a block barrier.
template <typename T>
__device__ void cl_halo(Cx<T>* sm, const ClLevel<T>& L, int off, int rank, int cl) {
  cg::cluster_group cluster = cg::this_cluster();
  cluster.sync();
  int y0, rows;
  cl_rows(L, rank, y0, rows);
  if (rows > 0) {
    if (rank > 0) {   // the block above owns a full band: its last row is local row band
      const Cx<T>* src = cluster.map_shared_rank(sm + off, rank - 1) + (size_t)L.band * L.pitch;
      for (int x = threadIdx.x; x < L.pitch; x += blockDim.x) sm[off + x] = src[x];
    }
    if (rank + 1 < cl && y0 + rows < L.ny) {   // first row of the block below: local row 1
      const Cx<T>* src = cluster.map_shared_rank(sm + off, rank + 1) + L.pitch;
      for (int x = threadIdx.x; x < L.pitch; x += blockDim.x) sm[off + (size_t)(rows + 1) * L.pitch + x] = src[x];
    }
  }
  __syncthreads();
}

template <int TPB, typename T>
__device__ int cl_smooth(Cx<T>* sm, const ClLevel<T>& L, int rank, int cl, int cur, int sweeps, bool zero, T om1) {
  int y0, rows;
  cl_rows(L, rank, y0, rows);
  const Cx<T>* b = sm + L.off_b;
  const Cx<T>* wd = L.wd;
  const int P = L.pitch;
  int s = 0;
  if (zero) {
    Cx<T>* v = sm + cur;
    cl_points<TPB>(L, y0, rows, [&](int k, int i, int, int) { v[i] = sweeps > 0 ? wd[k] * b[i] : czero<T>(); });
    cl_halo(sm, L, cur, rank, cl);
    s = 1;
  }
  for (; s < sweeps; ++s) {
    const Cx<T>* src = sm + cur;
    const int nxt = cur == L.off_v ? L.off_t : L.off_v;
    Cx<T>* dst = sm + nxt;
    cl_points<TPB>(L, y0, rows, [&](int k, int i, int, int) {
      const Cx<T> nb = src[i - 1] + src[i + 1] + src[i - P] + src[i + P];
      const Cx<T> bk = b[i];
      const Cx<T> t = mk<T>(bk.re + L.inv_h2 * nb.re, bk.im + L.inv_h2 * nb.im);
      const Cx<T> c = src[i], w = wd[k];
      dst[i] = mk<T>(om1 * c.re + w.re * t.re - w.im * t.im, om1 * c.im + w.re * t.im + w.im * t.re);
    });
    cl_halo(sm, L, nxt, rank, cl);
    cur = nxt;
  }
  return cur;
}

template <int TPB, typename T>
__device__ void cl_restrict(Cx<T>* sm, const ClLevel<T>& L, int rank, int cl, int cur, const ClLevel<T>& C) {
  int y0, rows, cy0, crows;
  cl_rows(L, rank, y0, rows);
  cl_rows(C, rank, cy0, crows);
  const Cx<T>* v = sm + cur;
  const Cx<T>* b = sm + L.off_b;
  const int roff = cur == L.off_v ? L.off_t : L.off_v;
  Cx<T>* r = sm + roff;
  const int P = L.pitch;
  const Cx<T>* D = L.D;
  cl_points<TPB>(L, y0, rows, [&](int k, int i, int, int) {
    const Cx<T> s = v[i - 1] + v[i + 1] + v[i - P] + v[i + P];
    const Cx<T> kv = D[k] * v[i] - L.inv_h2 * s;
    r[i] = b[i] - kv;
  });
  cl_halo(sm, L, roff, rank, cl);
  Cx<T>* bc = sm + C.off_b;
  const T q16 = T(1) / T(16);
  cl_points<TPB>(C, cy0, crows, [&](int, int ic, int ci, int cj) {
    const int i = (2 * cj - y0 + 1) * P + 2 * ci + 1;   // fine point (2 ci, 2 cj), local row 2 cj - y0
    const Cx<T> e = r[i - 1] + r[i + 1] + r[i - P] + r[i + P];
    const Cx<T> c = r[i - P - 1] + r[i - P + 1] + r[i + P - 1] + r[i + P + 1];
    const Cx<T> rc = r[i];
    bc[ic] = mk<T>(q16 * (T(4) * rc.re + T(2) * e.re + c.re), q16 * (T(4) * rc.im + T(2) * e.im + c.im));
  });
  __syncthreads();
}

template <int TPB, typename T>
__device__ void cl_prolong(Cx<T>* sm, const ClLevel<T>& L, int rank, int cl, int cur, const ClLevel<T>& C,
                           int ccur) {
  int y0, rows, cy0, crows;
  cl_rows(L, rank, y0, rows);
  cl_rows(C, rank, cy0, crows);
  Cx<T>* v = sm + cur;
  const Cx<T>* e = sm + ccur;
  const int PC = C.pitch;
  cl_points<TPB>(L, y0, rows, [&](int, int i, int x, int y) {
    const int ic = ((y >> 1) - cy0 + 1) * PC + (x >> 1) + 1;
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
  cl_halo(sm, L, cur, rank, cl);
}

// Coarsest level: gather b from every block of the cluster into a plain copy, then this block's
// rows of K^{-1} b, one warp per row (read from L2), lanes over columns, as in tail_coarsest.
template <int TPB, typename T>
__device__ void cl_coarsest(Cx<T>* sm, const ClLevel<T>& L, int rank, int cl, const Cx<T>* __restrict__ kinv) {
  cg::cluster_group cluster = cg::this_cluster();
  cluster.sync();
  Cx<T>* bfull = sm + L.off_t;
  const int n = L.nx * L.ny;
  for (int k = threadIdx.x; k < n; k += TPB) {
    const int y = k / L.nx, x = k - y * L.nx;
    const int owner = y / L.band;
    const Cx<T>* src = cluster.map_shared_rank(sm + L.off_b, owner);
    bfull[k] = src[(y - owner * L.band + 1) * L.pitch + x + 1];
  }
  __syncthreads();
  int y0, rows;
  cl_rows(L, rank, y0, rows);
  Cx<T>* v = sm + L.off_v;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int r = y0 * L.nx + warp; r < (y0 + rows) * L.nx; r += TPB / 32) {
    const Cx<T>* row = kinv + (size_t)r * n;
    T ar = 0, ai = 0;
    for (int c = lane; c < n; c += 32) {
      const Cx<T> k = row[c], x = bfull[c];
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
      v[(ry - y0 + 1) * L.pitch + rx + 1] = mk<T>(ar, ai);
    }
  }
  cl_halo(sm, L, L.off_v, rank, cl);
}

template <int TPB, typename T>
__global__ void __launch_bounds__(TPB, 1) k_tail_cl(const ClArgs<T> a) {
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int rhs = blockIdx.x / a.cl;
  // the state is read before any barrier: every block of a cluster takes the same branch
  if (a.st && !a.st[rhs].active) return;
  extern __shared__ __align__(16) unsigned char tail_smem[];
  Cx<T>* sm = reinterpret_cast<Cx<T>*>(tail_smem);
  for (int k = threadIdx.x; k < a.total; k += TPB) sm[k] = czero<T>();
  const ClLevel<T>& top = a.lv[0];
  int ty0, trows;
  cl_rows(top, rank, ty0, trows);
  __syncthreads();
  const int last = a.depth - 1;
  {
    const Cx<T>* bin = a.b_in + rhs * a.stride;
    Cx<T>* b0 = sm + top.off_b;
    cl_points<TPB>(top, ty0, trows, [&](int k, int i, int, int) { b0[i] = bin[k]; });
  }
  __syncthreads();
  int cnt[kMaxLevels];
  bool zero[kMaxLevels];
  int cur[kMaxLevels];
  for (int d = 0; d < a.depth; ++d) cur[d] = a.lv[d].off_v;
  for (int rep = 0; rep < a.reps; ++rep) {
    int d = 0;
    bool down = true;
    zero[0] = rep == 0;
    while (true) {
      if (down) {
        if (d == last) {
          cl_coarsest<TPB>(sm, a.lv[d], rank, a.cl, a.kinv);
          cur[d] = a.lv[d].off_v;
          --d;
          down = false;
          cnt[d] = a.gamma - 1;
          continue;
        }
        cur[d] = cl_smooth<TPB>(sm, a.lv[d], rank, a.cl, cur[d], a.lv[d].nu1, zero[d], a.om1);
        cl_restrict<TPB>(sm, a.lv[d], rank, a.cl, cur[d], a.lv[d + 1]);
        cnt[d] = 0;
        zero[d + 1] = true;
        ++d;
        continue;
      }
      if (++cnt[d] < a.gamma) {
        zero[d + 1] = false;
        ++d;
        down = true;
        continue;
      }
      cl_prolong<TPB>(sm, a.lv[d], rank, a.cl, cur[d], a.lv[d + 1], cur[d + 1]);
      cur[d] = cl_smooth<TPB>(sm, a.lv[d], rank, a.cl, cur[d], a.lv[d].nu2, false, a.om1);
      if (d == 0) break;
      --d;
    }
  }
  Cx<T>* vo = a.v_out + rhs * a.stride;
  const Cx<T>* v0 = sm + cur[0];
  cl_points<TPB>(top, ty0, trows, [&](int k, int i, int, int) { vo[k] = v0[i]; });
  cluster.sync();   // no block leaves while another may still read its shared memory
}

// Shared-memory layout of one block of a CL-block tail from level l0 (element offsets; returns the
// total), with band_l = 2^(L-1-l) ceil(ny_{L-1} / CL).
template <typename T>
int cl_layout(const Handle& h, int l0, int cl, ClLevel<T>* lv) {
  const int last = h.L - 1;
  const int bc = (h.lev[last].ny + cl - 1) / cl;
  int off = 0;
  for (int l = l0; l < h.L; ++l) {
    const Level& L = h.lev[l];
    ClLevel<T> t{};
    t.nx = L.nx; t.ny = L.ny; t.pitch = L.nx + 2;
    t.band = bc << (last - l);
    const int ps = (t.band + 2) * t.pitch;
    t.off_b = off; off += ps;
    t.off_v = off; off += ps;
    t.off_t = off; off += l + 1 < h.L ? ps : (int)L.n();
    if (lv) lv[l - l0] = t;
  }
  return off;
}

template <typename T>
size_t cl_smem_bytes(const Handle& h, int l0, int cl) {
  return (size_t)cl_layout<T>(h, l0, cl, nullptr) * sizeof(Cx<T>);
}

constexpr int kTpb2 = 1024, kTpb4 = 512;   // threads per block of the 2- and 4-block clusters

template <typename T>
mgh_status set_tail_cl_attrs() {
  MGH_ONCE(MGH_CUDA(cudaFuncSetAttribute(k_tail_cl<kTpb2, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kTailSmemMax));
           MGH_CUDA(cudaFuncSetAttribute(k_tail_cl<kTpb4, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kTailSmemMax)););
  return MGH_OK;
}

// Clusters of cl blocks of the tail from level tail_l0 that the GPU holds at once (0 if none).
template <typename T>
int tail_cl_capacity(Handle& h, int cl) {
  if (set_tail_cl_attrs<T>() != MGH_OK) return 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)cl, 1, 1);
  cfg.blockDim = dim3(cl == 2 ? kTpb2 : kTpb4, 1, 1);
  cfg.dynamicSmemBytes = cl_smem_bytes<T>(h, h.tail_l0, cl);
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cl;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  const cudaError_t e = cl == 2 ? cudaOccupancyMaxActiveClusters(&n, k_tail_cl<kTpb2, T>, &cfg)
                                : cudaOccupancyMaxActiveClusters(&n, k_tail_cl<kTpb4, T>, &cfg);
  if (e != cudaSuccess) { cudaGetLastError(); return 0; }
  return n;
}

template <typename T>
mgh_status launch_tail_cl(Handle& h, int reps, int B, const RhsState* st, int cl) {
  const int l0 = h.tail_l0;
  ClArgs<T> a{};
  a.total = cl_layout<T>(h, l0, cl, a.lv);
  for (int l = l0; l < h.L; ++l) {
    const Level& lv = h.lev[l];
    ClLevel<T>& t = a.lv[l - l0];
    t.D = (const Cx<T>*)lv.D;
    t.wd = (const Cx<T>*)lv.wDinv;
    t.nu1 = nu_pre(h, l); t.nu2 = nu_post(h, l);
    t.inv_h2 = static_cast<T>(1.0 / (lv.h * lv.h));
  }
  a.depth = h.L - l0;
  a.gamma = cycle_gamma(h);
  a.reps = reps;
  a.cl = cl;
  a.om1 = static_cast<T>(1.0 - h.p.omega);
  a.b_in = (const Cx<T>*)h.lev[l0].b;
  a.v_out = (Cx<T>*)h.lev[l0].vfin;
  a.stride = h.lev[l0].n();
  a.kinv = sizeof(T) == 8 ? (const Cx<T>*)(const void*)h.kinv64r : (const Cx<T>*)(const void*)h.kinv32;
  a.st = st;
  const size_t smem = (size_t)a.total * sizeof(Cx<T>);
  MGH_TRY(set_tail_cl_attrs<T>());
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(B * cl), 1, 1);
  cfg.blockDim = dim3(cl == 2 ? kTpb2 : kTpb4, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = h.stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cl;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  ProfScope ps(h, P_COARSE);
  if (cl == 2) MGH_CUDA(cudaLaunchKernelEx(&cfg, k_tail_cl<kTpb2, T>, a));
  else MGH_CUDA(cudaLaunchKernelEx(&cfg, k_tail_cl<kTpb4, T>, a));
  h.launches++;
  return MGH_OK;
}

}  // namespace

bool tail_level_fits(const Handle& h, int l) {
  if (l < 1 || l + 2 > h.L) return false;
  const size_t bytes = h.fp64 ? tail_smem_bytes<double>(h, l) : tail_smem_bytes<float>(h, l);
  return bytes <= kTailSmemMax;
}

bool tail_cluster_fits(const Handle& h, int l, int cl) {
  if (cl == 1) return tail_level_fits(h, l);
  if ((cl != 2 && cl != 4) || l < 1 || l + 2 > h.L || h.lev[h.L - 1].ny < cl) return false;
  const size_t bytes = h.fp64 ? cl_smem_bytes<double>(h, l, cl) : cl_smem_bytes<float>(h, l, cl);
  return bytes <= kTailSmemMax;
}

int choose_tail_level(const Handle& h) {
  for (int l = 1; l + 2 <= h.L; ++l) {
    const size_t bytes = h.fp64 ? tail_smem_bytes<double>(h, l) : tail_smem_bytes<float>(h, l);
    if (bytes <= kTailSmemMax) return l;
  }
  return 0;
}

// Blocks per right-hand side of a tail launch of B right-hand sides: the handle's setting, or with
// the automatic setting (0) the largest cluster (4, then 2) whose B clusters the GPU holds at once,
// else one block.  The cluster size changes no result.
int tail_cluster_for(Handle& h, int B) {
  if (h.tail_cluster > 0) return h.tail_cluster;
  if (h.tail_cap_l0 != h.tail_l0) {   // capacities of this tail level, queried once
    for (int c : {2, 4})
      h.tail_cap[c] = tail_cluster_fits(h, h.tail_l0, c)
                          ? (h.fp64 ? tail_cl_capacity<double>(h, c) : tail_cl_capacity<float>(h, c)) : 0;
    h.tail_cap_l0 = h.tail_l0;
  }
  if (B <= h.tail_cap[4]) return 4;
  if (B <= h.tail_cap[2]) return 2;
  return 1;
}

mgh_status launch_tail(Handle& h, int reps, int B, const RhsState* st, bool fp64) {
  const int cl = tail_cluster_for(h, B);
  if (cl > 1)
    return fp64 ? launch_tail_cl<double>(h, reps, B, st, cl) : launch_tail_cl<float>(h, reps, B, st, cl);
  return fp64 ? launch_tail_t<double>(h, reps, B, st) : launch_tail_t<float>(h, reps, B, st);
}

}  // namespace mgh
