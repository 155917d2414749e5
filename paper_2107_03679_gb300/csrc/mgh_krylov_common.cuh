// Pieces shared by the FP64 and the double-float FGMRES engines: launch arguments, block
// reductions into the per-block partial-sum buffer, restart-cycle bookkeeping, the
// Hessenberg back substitution and the per-solve result collection.
#pragma once

#include <algorithm>

#include "mgh_engine.h"

namespace mgh {

namespace {

constexpr int kKThreads = 256;
constexpr int kTargetBlocks = 152 * 8;

struct KArgs {
  int nx, ny;
  size_t N;
  int m;                 // restart length
  int nblk;              // reduction blocks per RHS
  size_t chunk;          // points per block
  double inv_h2;
  int pstride;           // complex slots per block in the partial-sum buffer
  size_t Np;             // plane stride of double-float fields (N rounded up to 64 points)
};

constexpr int kTile = 256;  // points per pipeline tile of the double-float kernels; chunks are multiples

// Block reduction of NV complex accumulators (plus one real) into partial[(rhs*nblk+blk)*(m+2) + i].
template <int NV>
__device__ __forceinline__ void block_reduce_store(cd (&acc)[NV], int nv_used, double extra, int extra_slot,
                                                   cd* __restrict__ out) {
  __shared__ double sh[kKThreads / 32][2 * NV + 1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    if (i < nv_used) {
      const double re = warp_sum(acc[i].re);
      const double im = warp_sum(acc[i].im);
      if (lane == 0) { sh[warp][2 * i] = re; sh[warp][2 * i + 1] = im; }
    }
  }
  const double ex = warp_sum(extra);
  if (lane == 0) sh[warp][2 * NV] = ex;
  __syncthreads();
  const int nw = kKThreads / 32;
  for (int t = threadIdx.x; t < 2 * nv_used; t += kKThreads) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += sh[w][t];
    double* o = reinterpret_cast<double*>(out + (t >> 1));
    o[t & 1] = s;
  }
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += sh[w][2 * NV];
    out[extra_slot] = mk<double>(s, 0.0);
  }
}

template <typename TZ>
__device__ __forceinline__ cd load_z(const Cx<TZ>* z, size_t q) { return ccast<double>(z[q]); }

__device__ __forceinline__ void sum_partials(const KArgs& a, const cd* __restrict__ partial, int rhs, int nslots,
                                             cd* __restrict__ out_sh) {
  for (int s = threadIdx.x; s < nslots; s += blockDim.x) {
    // the loads are independent: unrolled, they are in flight together while the adds keep
    // the block order
    cd acc = czero<double>();
#pragma unroll 8
    for (int b = 0; b < a.nblk; ++b) acc = acc + partial[((size_t)rhs * a.nblk + b) * a.pstride + s];
    out_sh[s] = acc;
  }
  __syncthreads();
}

// Back substitution H(0:jend,0:jend) y = g(0:jend); one thread per right-hand side.
__global__ void k_lsq(KArgs a, const cd* __restrict__ H, const cd* __restrict__ g, cd* __restrict__ y,
                      RhsState* __restrict__ st, int B) {
  const int rhs = blockIdx.x * blockDim.x + threadIdx.x;
  if (rhs >= B || st[rhs].done || st[rhs].jend == 0) return;
  const int m = a.m, je = st[rhs].jend;
  st[rhs].nupd += 1;
  st[rhs].zsum += je;
  const cd* Hb = H + (size_t)rhs * m * (m + 1);
  const cd* gg = g + (size_t)rhs * (m + 1);
  cd* yy = y + (size_t)rhs * m;
  for (int i = je - 1; i >= 0; --i) {
    cd t = gg[i];
    for (int k = i + 1; k < je; ++k) t = t - Hb[(size_t)k * (m + 1) + i] * yy[k];
    const cd d = Hb[(size_t)i * (m + 1) + i];
    const double den = cabs2(d);
    yy[i] = t * mk<double>(d.re / den, -d.im / den);
  }
}

// Start (or end) a cycle from the true residual: converged / maxit / next cycle.
__global__ void k_cycle_start(KArgs a, const cd* __restrict__ partial, double* __restrict__ vscale,
                              cd* __restrict__ g, RhsState* __restrict__ st, double tol, int maxit, int first) {
  __shared__ cd sh[2];
  const int rhs = blockIdx.x;
  if (st[rhs].done) return;
  sum_partials(a, partial, rhs, 2, sh);
  if (threadIdx.x != 0) return;
  RhsState& S = st[rhs];
  S.nres += 1;
  if (first) {
    S.bnorm = sqrt(sh[1].re);
    S.iterations = 0;
    S.restarts = 0;
  } else {
    S.restarts += 1;
  }
  const double rn = sqrt(sh[0].re);
  S.rnorm = rn;
  S.jend = 0;
  S.active = 0;
  S.reorth = 0;
  if (S.bnorm == 0.0) { S.done = 1; S.converged = 1; return; }
  if (rn <= tol * S.bnorm) { S.done = 1; S.converged = 1; return; }
  if (S.iterations >= maxit || !(rn == rn)) { S.done = 1; S.converged = 0; return; }
  S.active = 1;
  vscale[(size_t)rhs * (a.m + 1)] = 1.0 / rn;
  cd* gg = g + (size_t)rhs * (a.m + 1);
  gg[0] = mk<double>(rn, 0.0);
  for (int i = 1; i <= a.m; ++i) gg[i] = czero<double>();
}

// x = 0 for right-hand sides with b = 0 (set done at the first cycle start).
__global__ void k_zero_if_b_zero(KArgs a, cd* __restrict__ x, const RhsState* __restrict__ st) {
  const int rhs = blockIdx.y;
  if (st[rhs].bnorm != 0.0) return;
  const size_t p0 = blockIdx.x * a.chunk, p1 = (p0 + a.chunk < a.N) ? p0 + a.chunk : a.N;
  for (size_t q = p0 + threadIdx.x; q < p1; q += kKThreads) x[(size_t)rhs * a.N + q] = czero<double>();
}

__global__ void k_state_reset(RhsState* st, int B) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < B) { RhsState z = {}; st[i] = z; }
}

KArgs make_kargs(const Handle& h, int B) {
  KArgs a;
  a.nx = h.nx; a.ny = h.ny; a.N = h.N; a.m = h.m;
  const int want = std::max(1, std::min<int>((kTargetBlocks + B - 1) / B, (int)((h.N + 1023) / 1024)));
  a.chunk = ((h.N + want - 1) / want + kTile - 1) / kTile * kTile;
  a.nblk = (int)((h.N + a.chunk - 1) / a.chunk);
  a.Np = (h.N + 63) / 64 * 64;
  a.inv_h2 = 1.0 / (h.p.h * h.p.h);
  a.pstride = partial_stride(h.m);
  return a;
}

// A launch sequence that repeats between two host reads of the per-RHS state (a restart cycle,
// a Bi-CGSTAB iteration), every launch gated by device state, captured once into a CUDA graph and
// replayed.  Capture and replay happen on the handle's own non-blocking stream (the caller's may
// be the legacy default stream, which cannot be captured), ordered after and before the caller's
// stream by events.  The caller runs the first repetition directly, so that lazy kernel attributes
// and occupancy queries happen outside capture; graphs are off while launches are profiled.
struct CycleGraph {
  cudaGraphExec_t exec = nullptr;
  uint64_t launches = 0;   // launches of one repetition
  CycleGraph() = default;
  CycleGraph(const CycleGraph&) = delete;
  CycleGraph& operator=(const CycleGraph&) = delete;
  ~CycleGraph() { if (exec) cudaGraphExecDestroy(exec); }

  template <typename Body>
  mgh_status run(Handle& h, Body&& body) {
    if (!h.gstream) {
      MGH_CUDA(cudaStreamCreateWithFlags(&h.gstream, cudaStreamNonBlocking));
      MGH_CUDA(cudaEventCreateWithFlags(&h.gev_in, cudaEventDisableTiming));
      MGH_CUDA(cudaEventCreateWithFlags(&h.gev_out, cudaEventDisableTiming));
    }
    if (!exec) {
      const uint64_t l0 = h.launches;
      cudaStream_t user = h.stream;
      h.stream = h.gstream;
      const cudaError_t eb = cudaStreamBeginCapture(h.gstream, cudaStreamCaptureModeRelaxed);
      if (eb != cudaSuccess) { h.stream = user; MGH_CUDA(eb); }
      const mgh_status sb = body();
      cudaGraph_t g = nullptr;
      const cudaError_t ec = cudaStreamEndCapture(h.gstream, &g);
      h.stream = user;
      launches = h.launches - l0;
      h.launches = l0;
      if (sb != MGH_OK) { if (g) cudaGraphDestroy(g); return sb; }
      if (ec != cudaSuccess) { if (g) cudaGraphDestroy(g); MGH_CUDA(ec); }
      const cudaError_t ei = cudaGraphInstantiate(&exec, g, 0);
      cudaGraphDestroy(g);
      MGH_CUDA(ei);
    }
    MGH_CUDA(cudaEventRecord(h.gev_in, h.stream));
    MGH_CUDA(cudaStreamWaitEvent(h.gstream, h.gev_in, 0));
    MGH_CUDA(cudaGraphLaunch(exec, h.gstream));
    MGH_CUDA(cudaEventRecord(h.gev_out, h.gstream));
    MGH_CUDA(cudaStreamWaitEvent(h.stream, h.gev_out, 0));
    h.launches += launches;
    return MGH_OK;
  }
};

// Per-RHS results of a finished solve (host mirror already synchronised) and profile counters.
mgh_status finish_solve(Handle& h, int B, mgh_solve_info* info) {
  bool all_conv = true;
  for (int i = 0; i < B; ++i) {
    const RhsState& S = h.st_host[i];
    all_conv &= (S.converged != 0);
    h.acc.arnoldi_steps += S.iterations;
    h.acc.basis_reads += S.vsum;
    h.acc.reorth_reads += S.rsum;
    h.acc.residuals += S.nres;
    h.acc.updates += S.nupd;
    h.acc.update_reads += S.zsum;
    h.acc.cycle_steps += S.csteps > 0 ? S.csteps : S.iterations;
    h.acc.gram_reads += S.gsum;
    if (info) {
      info[i].iterations = S.iterations;
      info[i].restarts = S.restarts;
      info[i].converged = S.converged;
      info[i].rel_residual = S.bnorm > 0.0 ? S.rnorm / S.bnorm : 0.0;
    }
  }
  return all_conv ? MGH_OK : MGH_NOT_CONVERGED;
}

}  // namespace

}  // namespace mgh
