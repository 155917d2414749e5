// Allocation-free variant of the data-misfit entry point (mgh_misfit): the per-RHS partial
// losses that mgh_misfit keeps in handle-owned device memory live here in a file-scope device
// array, so the call needs neither a handle nor any device allocation.
#include <mutex>

#include "mgh_common.cuh"

namespace {

constexpr int kNoallocMaxBatch = 4096;   // right-hand sides per call (32 KiB of scratch)
constexpr int kMaxDevices = 64;

// Shared by every call on a device and kept until the process exits; each call overwrites the
// entries 0..B-1 it uses before reading them.
static __device__ __align__(256) double g_misfit_scratch[kNoallocMaxBatch];

std::mutex g_mutex;
double* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device, resolved once per device.  The
// look-up is not a stream operation: while `s` is being captured into a graph it is refused
// (MGH_INVALID_ARG, nothing changed) instead of being run inside the caller's capture.
mgh_status scratch_address(double** out, cudaStream_t s) {
  int dev = 0;
  MGH_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return MGH_NOT_SUPPORTED;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_addr[dev]) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    MGH_CUDA(cudaStreamIsCapturing(s, &cap));
    if (cap != cudaStreamCaptureStatusNone) return MGH_INVALID_ARG;
    void* p = nullptr;
    MGH_CUDA(cudaGetSymbolAddress(&p, g_misfit_scratch));
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return MGH_OK;
}

using mgh::cd;

__global__ void k_misfit_scratch(const cd* __restrict__ u, const cd* __restrict__ y, size_t N,
                                 const int64_t* __restrict__ rec, int M, cd* __restrict__ r, cd* __restrict__ G,
                                 double* __restrict__ part) {
  __shared__ double sh[32];
  const int rhs = blockIdx.x;
  double acc = 0.0;
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    const cd d = u[rhs * N + rec[i]] - y[(size_t)rhs * M + i];
    if (r) r[(size_t)rhs * M + i] = d;
    if (G) G[rhs * N + rec[i]] = d;
    acc += mgh::cabs2(d);
  }
  acc = mgh::warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    v = mgh::warp_sum(v);
    if (threadIdx.x == 0) part[rhs] = 0.5 * v;
  }
}

__global__ void k_sum_scratch(const double* __restrict__ part, int B, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < B; ++i) s += part[i];
    *out = s;
  }
}

}  // namespace

extern "C" mgh_status mgh_misfit_noalloc(int nx, int ny, const mgh_cdouble* u, const mgh_cdouble* y, int B,
                                         const int64_t* rec, int M, mgh_cdouble* r, mgh_cdouble* G,
                                         double* loss_dev, void* cuda_stream) {
  if (nx < 1 || ny < 1 || !u || !y || !rec || !loss_dev || M < 1 || B < 1) return MGH_INVALID_ARG;
  if (B > kNoallocMaxBatch) return MGH_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  double* part = nullptr;
  MGH_TRY(scratch_address(&part, s));
  const size_t N = (size_t)nx * ny;
  if (G) MGH_CUDA(cudaMemsetAsync(G, 0, sizeof(cd) * N * B, s));
  k_misfit_scratch<<<B, 256, 0, s>>>(reinterpret_cast<const cd*>(u), reinterpret_cast<const cd*>(y), N, rec, M,
                                     reinterpret_cast<cd*>(r), reinterpret_cast<cd*>(G), part);
  MGH_CHECK_LAUNCH();
  k_sum_scratch<<<1, 32, 0, s>>>(part, B, loss_dev);
  MGH_CHECK_LAUNCH();
  return MGH_OK;
}
