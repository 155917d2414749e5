// Device helpers shared by the CUDA translation units of the solver: complex arithmetic on
// interleaved (re, im) pairs, block reductions, and the launch/error bookkeeping.
#pragma once

#include <cuda_runtime.h>
#include <atomic>
#include <cstdint>
#include <cstdio>

#include "mgh.h"

namespace mgh {

// Interleaved complex number; alignment 2*sizeof(T) so that a field can be read with one
// 8-byte (float) or 16-byte (double) vector access per point.
template <typename T>
struct alignas(2 * sizeof(T)) Cx {
  T re, im;
};
using cf = Cx<float>;
using cd = Cx<double>;

template <typename T>
__host__ __device__ __forceinline__ Cx<T> mk(T re, T im) { Cx<T> r; r.re = re; r.im = im; return r; }
template <typename T>
__host__ __device__ __forceinline__ Cx<T> operator+(Cx<T> a, Cx<T> b) { return mk<T>(a.re + b.re, a.im + b.im); }
template <typename T>
__host__ __device__ __forceinline__ Cx<T> operator-(Cx<T> a, Cx<T> b) { return mk<T>(a.re - b.re, a.im - b.im); }
template <typename T>
__host__ __device__ __forceinline__ Cx<T> operator*(Cx<T> a, Cx<T> b) {
  return mk<T>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename T>
__host__ __device__ __forceinline__ Cx<T> operator*(T s, Cx<T> a) { return mk<T>(s * a.re, s * a.im); }
template <typename T>
__host__ __device__ __forceinline__ Cx<T> cconj(Cx<T> a) { return mk<T>(a.re, -a.im); }
template <typename T>
__host__ __device__ __forceinline__ T cabs2(Cx<T> a) { return a.re * a.re + a.im * a.im; }
template <typename T>
__host__ __device__ __forceinline__ Cx<T> czero() { return mk<T>(T(0), T(0)); }

// acc += conj(a) * b
template <typename T>
__device__ __forceinline__ void cdot_acc(Cx<T>& acc, Cx<T> a, Cx<T> b) {
  acc.re = fma(a.re, b.re, fma(a.im, b.im, acc.re));
  acc.im = fma(a.re, b.im, fma(-a.im, b.re, acc.im));
}
// acc -= s * a
template <typename T>
__device__ __forceinline__ void caxpy_neg(Cx<T>& acc, Cx<T> s, Cx<T> a) {
  acc.re = fma(-s.re, a.re, fma(s.im, a.im, acc.re));
  acc.im = fma(-s.re, a.im, fma(-s.im, a.re, acc.im));
}

template <typename To, typename From>
__device__ __forceinline__ Cx<To> ccast(Cx<From> a) { return mk<To>(static_cast<To>(a.re), static_cast<To>(a.im)); }

// Warp / block sums of doubles (deterministic order for a fixed launch shape).
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Per-right-hand-side state of the batched FGMRES engine (device resident).
struct RhsState {
  int active;        // 1 while this right-hand side takes Arnoldi steps in the current cycle
  int done;          // 1 once converged, hit maxit, or b = 0
  int converged;     // 1 if the true residual reached tol
  int jend;          // Arnoldi steps taken in the current cycle
  int iterations;    // total Arnoldi steps
  int restarts;      // completed cycles
  int reorth;        // 1 if the current step needs a second Gram-Schmidt pass
  int vsum;          // sum over steps of j+1 (basis vectors read per Gram-Schmidt pass)
  int rsum;          // the same for second passes
  int nres;          // true residual evaluations
  int nupd;          // iterate updates
  int zsum;          // preconditioned vectors read by iterate updates
  int verify;        // mixed path: the double-float residual met the target, FP64 check pending
  int nverify;       // FP64 verifications run
  int csteps;        // s-step engine: multigrid cycles + matvecs run (all steps of every cycle)
  int gsum;          // s-step engine: basis vectors read by the Gram sweeps
  double bnorm;      // ||b||
  double rnorm;      // last true residual norm
  double wnorm2;     // ||A z_j||^2 of the current step
  double norm2;      // ||w'||^2 after orthogonalisation
  double inv_nu;     // 1 / ||u_j - Q_j s|| of the current step (mixed path)
  double hjj_re, hjj_im;  // <q_j, w> of the current step (mixed path)
  double tol_scale;  // mixed path: factor on tol for the double-float residual (tightened if the FP64 check fails)
  int jstart;        // first Arnoldi column of the current cycle (k after a deflated restart)
  int deflate;       // 1: the cycle ended full length and restarts deflated (residual kept apart from V)
};

}  // namespace mgh

// Record a CUDA error (message kept for mgh_last_error) and return MGH_CUDA_ERROR.
namespace mgh { void set_error(const char* what, cudaError_t e, const char* file, int line); }
#define MGH_CUDA(call)                                                   \
  do {                                                                   \
    cudaError_t e_ = (call);                                             \
    if (e_ != cudaSuccess) {                                             \
      ::mgh::set_error(#call, e_, __FILE__, __LINE__);                   \
      return MGH_CUDA_ERROR;                                             \
    }                                                                    \
  } while (0)
#define MGH_CHECK_LAUNCH()                                               \
  do {                                                                   \
    cudaError_t e_ = cudaGetLastError();                                 \
    if (e_ != cudaSuccess) {                                             \
      ::mgh::set_error("kernel launch", e_, __FILE__, __LINE__);         \
      return MGH_CUDA_ERROR;                                             \
    }                                                                    \
  } while (0)
#define MGH_TRY(expr)                                                    \
  do {                                                                   \
    mgh_status s_ = (expr);                                              \
    if (s_ != MGH_OK) return s_;                                         \
  } while (0)
// A one-time set-up step (kernel attributes) run once per device: cudaFuncSetAttribute applies to
// the device that is current when it is called, so every device a process drives handles on needs
// its own call.  One bit per device (devices 0..63; others run the step on every call) records a
// step that succeeded; a step that failed is tried again by the next call.  Host threads that reach
// the step together on one device may each run it: the steps are idempotent attribute settings.
// The arguments are the statements of the step.
#define MGH_ONCE(...)                                                                          \
  do {                                                                                         \
    static std::atomic<unsigned long long> once_done_{0ull};                                   \
    int once_dev_ = -1;                                                                        \
    MGH_CUDA(cudaGetDevice(&once_dev_));                                                       \
    const unsigned long long once_bit_ =                                                       \
        (once_dev_ >= 0 && once_dev_ < 64) ? (1ull << once_dev_) : 0ull;                       \
    if (once_bit_ == 0ull || !(once_done_.load(std::memory_order_acquire) & once_bit_)) {      \
      const mgh_status once_s_ = [&]() -> mgh_status { __VA_ARGS__ return MGH_OK; }();        \
      if (once_s_ != MGH_OK) return once_s_;                                                   \
      once_done_.fetch_or(once_bit_, std::memory_order_acq_rel);                               \
    }                                                                                          \
  } while (0)
