// Diagonal of the discrete operators on one multigrid level (Sec. IV-A/B): for K_kappa,
//   D = 4/h^2 - kappa * alpha * c - nmiss * (1 + j h k) / h^2,   alpha = 1 + j beta d^2 / L^2,
// with c the level's real coefficient k0^2 eta^2, d the distance in fine cells from the point's
// fine position to Omega's index box, L the layer width, and nmiss the neighbours closed by the
// first-order Sommerfeld ghost value; A is the case kappa = 1 on the fine level.  Shared by the
// set-up kernels (FP64) and the one-kernel coarse tail, which forms D from c on the fly (FP32).
#pragma once

#include "mgh_common.cuh"

namespace mgh {

template <typename T>
struct DiagArgs {
  int nx, ny, scale;      // level size and its spacing in fine cells
  int x0, x1, y0, y1;     // Omega index box on the fine grid (inclusive)
  T inv_L2;               // 1 / abl^2 (0 without a layer)
  T beta;
  T ih2;                  // 1 / h^2 of the level
  T k_h;                  // k / h of the level
  T kap_re, kap_im;
  T omega;
};

// The level fields of DiagArgs from its spacing h and the background wavenumber k.
template <typename T>
inline void diag_set_spacing(DiagArgs<T>& a, double h, double k) {
  a.ih2 = static_cast<T>(1.0 / (h * h));
  a.k_h = static_cast<T>(k / h);
}

template <typename T>
__host__ __device__ __forceinline__ Cx<T> level_diag(const DiagArgs<T>& a, int i, int j, T c) {
  const int fx = a.scale * i, fy = a.scale * j;
  const int dx = fx < a.x0 ? a.x0 - fx : (fx > a.x1 ? fx - a.x1 : 0);
  const int dy = fy < a.y0 ? a.y0 - fy : (fy > a.y1 ? fy - a.y1 : 0);
  const T t = a.beta * ((T)dx * dx + (T)dy * dy) * a.inv_L2;
  // kappa * alpha = (kr + j ki)(1 + j t)
  const T ka_re = a.kap_re - a.kap_im * t;
  const T ka_im = a.kap_im + a.kap_re * t;
  const int nmiss = (i == 0) + (i == a.nx - 1) + (j == 0) + (j == a.ny - 1);
  Cx<T> d;
  d.re = T(4) * a.ih2 - ka_re * c - nmiss * a.ih2;
  d.im = -ka_im * c - nmiss * a.k_h;   // nmiss <= 2, so nmiss * (k / h) = (nmiss k) / h exactly
  return d;
}

// omega / D (one division)
template <typename T>
__host__ __device__ __forceinline__ Cx<T> damped_inverse(const Cx<T>& d, T omega) {
  const T s = omega / (d.re * d.re + d.im * d.im);
  return mk<T>(s * d.re, -s * d.im);
}

}  // namespace mgh
