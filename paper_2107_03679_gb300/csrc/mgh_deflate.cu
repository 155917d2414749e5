// Host-side small dense linear algebra of the deflated restart of flexible GMRES (GMRES-DR,
// Morgan 2002, in the flexible form of Giraud, Gratton, Pinel & Vasseur 2010).
//
// At the end of a cycle of m Arnoldi steps a right-hand side holds V (m+1 orthonormal columns),
// Z (m preconditioned vectors), the (m+1) x m Arnoldi matrix Hbar with A Z = V Hbar and the
// coefficients c = g0 - Hbar y of its residual in V.  The next cycle keeps the k harmonic Ritz
// vectors of smallest harmonic Ritz value modulus:
//   g_1 .. g_k   eigenvectors of T = H_m + |h_{m+1,m}|^2 f e_m^T (H_m^H f = e_m)
//   P = [[g_1 .. g_k; 0], c] orthonormalised (modified Gram-Schmidt, two passes)
//   V' = V P,  Z' = Z P_k,  Hbar' = P^H Hbar P_k ((k+1) x k),  A Z' = V' Hbar'
// (the same coefficients P_k for the kept columns of V and of Z, so that z_i = M^{-1} v_i carries
// over for a fixed preconditioner).  Hbar' is full; a unitary change W of the k kept columns
// (applied to V' and Z' alike: the device receives C = P_k W) brings it to upper Hessenberg form,
// so that its QR factorisation is k Givens rotations and the device's Arnoldi/Givens loop simply
// continues at column k.  The residual lies in span(V'), and its component orthogonal to the kept
// columns is V c~ with c~ the last column of P; the device takes that direction from the true
// residual.  Everything here is a few thousand flops on matrices of order <= 33.
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "mgh_engine.h"

namespace mgh {

namespace {

using cplx = std::complex<double>;

// Dense row-major matrix.
struct Mat {
  int r = 0, c = 0;
  std::vector<cplx> a;
  Mat(int rows, int cols) : r(rows), c(cols), a((size_t)rows * cols) {}
  cplx& operator()(int i, int j) { return a[(size_t)i * c + j]; }
  const cplx& operator()(int i, int j) const { return a[(size_t)i * c + j]; }
};

// Solve A x = b in place (n x n, LU with partial pivoting); a zero pivot is replaced by a tiny one
// (inverse iteration solves with nearly singular shifted matrices on purpose).
void lu_solve(Mat A, std::vector<cplx>& b) {
  const int n = A.r;
  double scale = 0.0;
  for (const cplx& v : A.a) scale = std::max(scale, std::abs(v));
  const double tiny = (scale > 0.0 ? scale : 1.0) * 1e-14;
  for (int col = 0; col < n; ++col) {
    int p = col;
    for (int i = col + 1; i < n; ++i)
      if (std::abs(A(i, col)) > std::abs(A(p, col))) p = i;
    if (p != col) {
      for (int j = 0; j < n; ++j) std::swap(A(col, j), A(p, j));
      std::swap(b[col], b[p]);
    }
    if (std::abs(A(col, col)) < tiny) A(col, col) = tiny;
    for (int i = col + 1; i < n; ++i) {
      const cplx l = A(i, col) / A(col, col);
      if (l == cplx(0.0)) continue;
      for (int j = col; j < n; ++j) A(i, j) -= l * A(col, j);
      b[i] -= l * b[col];
    }
  }
  for (int i = n - 1; i >= 0; --i) {
    cplx t = b[i];
    for (int j = i + 1; j < n; ++j) t -= A(i, j) * b[j];
    b[i] = t / A(i, i);
  }
}

// Rotation [[c, s], [-conj(s), c]] (c real) that maps (x, y) to (rho, 0).
void givens(const cplx& x, const cplx& y, double& c, cplx& s) {
  if (y == cplx(0.0)) { c = 1.0; s = 0.0; return; }
  if (x == cplx(0.0)) { c = 0.0; s = 1.0; return; }
  const double ax = std::abs(x), rho = std::hypot(ax, std::abs(y));
  c = ax / rho;
  s = (x / ax) * std::conj(y) / rho;
}

// Eigenvalues of an upper Hessenberg matrix by the shifted QR algorithm (Wilkinson shifts,
// deflation on negligible subdiagonal entries, an exceptional shift every tenth iteration).
// Returns false if it does not converge within 60 n iterations.
bool hessenberg_eigenvalues(Mat H, std::vector<cplx>& eig) {
  const int n = H.r;
  eig.clear();
  int hi = n - 1, iter = 0, total = 0;
  const double eps = 1e-15;
  while (hi >= 0) {
    if (hi == 0) { eig.push_back(H(0, 0)); break; }
    int l = hi;
    while (l > 0) {
      const double sub = std::abs(H(l, l - 1));
      if (sub <= eps * (std::abs(H(l, l)) + std::abs(H(l - 1, l - 1))) || sub == 0.0) break;
      --l;
    }
    if (l == hi) {
      eig.push_back(H(hi, hi));
      --hi;
      iter = 0;
      continue;
    }
    if (++total > 60 * n) return false;
    // Wilkinson shift: the eigenvalue of the trailing 2 x 2 block nearer its last diagonal entry
    const cplx a = H(hi - 1, hi - 1), b = H(hi - 1, hi), c = H(hi, hi - 1), d = H(hi, hi);
    const cplx half = 0.5 * (a - d);
    const cplx disc = std::sqrt(half * half + b * c);
    cplx mu1 = 0.5 * (a + d) + disc, mu2 = 0.5 * (a + d) - disc;
    cplx shift = std::abs(mu1 - d) < std::abs(mu2 - d) ? mu1 : mu2;
    if (++iter % 10 == 0) shift += std::abs(H(hi, hi - 1));   // exceptional shift
    for (int i = l; i <= hi; ++i) H(i, i) -= shift;
    std::vector<double> cs(hi - l);
    std::vector<cplx> sn(hi - l);
    for (int i = l; i < hi; ++i) {   // H = Q R on the active block
      double cc;
      cplx ss;
      givens(H(i, i), H(i + 1, i), cc, ss);
      cs[i - l] = cc;
      sn[i - l] = ss;
      for (int j = i; j <= hi; ++j) {
        const cplx t = cc * H(i, j) + ss * H(i + 1, j);
        H(i + 1, j) = -std::conj(ss) * H(i, j) + cc * H(i + 1, j);
        H(i, j) = t;
      }
    }
    for (int i = l; i < hi; ++i) {   // R Q
      const double cc = cs[i - l];
      const cplx ss = sn[i - l];
      for (int r = l; r <= std::min(i + 2, hi); ++r) {
        const cplx t = cc * H(r, i) + std::conj(ss) * H(r, i + 1);
        H(r, i + 1) = -ss * H(r, i) + cc * H(r, i + 1);
        H(r, i) = t;
      }
    }
    for (int i = l; i <= hi; ++i) H(i, i) += shift;
  }
  return (int)eig.size() == n;
}

// Modified Gram-Schmidt, two passes, on the columns of P in order; false if a column vanishes.
bool orthonormalise(Mat& P) {
  for (int j = 0; j < P.c; ++j) {
    double n0 = 0.0;
    for (int i = 0; i < P.r; ++i) n0 += std::norm(P(i, j));
    n0 = std::sqrt(n0);
    for (int pass = 0; pass < 2; ++pass)
      for (int q = 0; q < j; ++q) {
        cplx d = 0.0;
        for (int i = 0; i < P.r; ++i) d += std::conj(P(i, q)) * P(i, j);
        for (int i = 0; i < P.r; ++i) P(i, j) -= d * P(i, q);
      }
    double nn = 0.0;
    for (int i = 0; i < P.r; ++i) nn += std::norm(P(i, j));
    nn = std::sqrt(nn);
    if (!(nn > 1e-10 * n0) || !(nn > 0.0)) return false;
    for (int i = 0; i < P.r; ++i) P(i, j) /= nn;
  }
  return true;
}

}  // namespace

// Deflated-restart data of one right-hand side (row-major arrays).
//   in:  Hbar (m+1) x m, c (m+1)
//   out: C (m x k) = P_k W with orthonormal columns; Hh ((k+1) x k) upper Hessenberg, the Arnoldi
//        matrix of the kept columns in the basis [V C, V c~]; R (k x k) upper triangular and the k
//        Givens rotations (cs real, sn) that reduce Hh to [R; 0] (rotation i acts on rows i, i+1 as
//        [[cs, sn], [-conj(sn), cs]]).
// Returns false when the eigenvalue iteration does not converge or a column vanishes (the caller
// then restarts plainly from the residual).
bool deflate_restart(int m, int k, const cplx* Hbar, const cplx* c, cplx* C, cplx* Hh, cplx* R, double* cs,
                     cplx* sn) {
  if (k < 1 || k >= m) return false;
  Mat Hb(m + 1, m);
  for (int i = 0; i <= m; ++i)
    for (int j = 0; j < m; ++j) Hb(i, j) = Hbar[(size_t)i * m + j];
  // T = H_m + |h_{m+1,m}|^2 f e_m^T with H_m^H f = e_m
  Mat Hc(m, m);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) Hc(i, j) = std::conj(Hb(j, i));
  std::vector<cplx> f(m, 0.0);
  f[m - 1] = 1.0;
  lu_solve(Hc, f);
  Mat T(m, m);
  const double h2 = std::norm(Hb(m, m - 1));
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) T(i, j) = Hb(i, j) + (j == m - 1 ? h2 * f[i] : cplx(0.0));
  std::vector<cplx> theta;
  if (!hessenberg_eigenvalues(T, theta)) return false;
  std::sort(theta.begin(), theta.end(), [](const cplx& x, const cplx& y) { return std::abs(x) < std::abs(y); });
  // eigenvectors of the k smallest by inverse iteration on T - theta I (shift nudged off the
  // computed eigenvalue so that the factorisation stays regular), then P = [[G_k; 0], c]
  Mat P(m + 1, k + 1);
  double tn = 0.0;
  for (const cplx& v : T.a) tn = std::max(tn, std::abs(v));
  for (int q = 0; q < k; ++q) {
    Mat S = T;
    const cplx sh = theta[q] + cplx(1e-12 * tn, 1e-12 * tn);
    for (int i = 0; i < m; ++i) S(i, i) -= sh;
    std::vector<cplx> x(m);
    for (int i = 0; i < m; ++i) x[i] = cplx(1.0 + 0.1 * i, 0.05 * (q + 1));
    for (int it = 0; it < 3; ++it) {
      lu_solve(S, x);
      double nx = 0.0;
      for (const cplx& v : x) nx += std::norm(v);
      nx = std::sqrt(nx);
      if (!(nx > 0.0) || !std::isfinite(nx)) return false;
      for (cplx& v : x) v /= nx;
    }
    for (int i = 0; i < m; ++i) P(i, q) = x[i];
  }
  for (int i = 0; i <= m; ++i) P(i, k) = c[i];
  if (!orthonormalise(P)) return false;
  // Hbar' = P^H Hbar P_k
  Mat HP(m + 1, k);
  for (int i = 0; i <= m; ++i)
    for (int j = 0; j < k; ++j) {
      cplx s = 0.0;
      for (int l = 0; l < m; ++l) s += Hb(i, l) * P(l, j);
      HP(i, j) = s;
    }
  Mat G(k + 1, k);
  for (int i = 0; i <= k; ++i)
    for (int j = 0; j < k; ++j) {
      cplx s = 0.0;
      for (int l = 0; l <= m; ++l) s += std::conj(P(l, i)) * HP(l, j);
      G(i, j) = s;
    }
  // Hessenberg form by a unitary change W of the kept columns, from the bottom row up: for row r
  // (k down to 2) rotations in the column planes (col, r-1) zero G(r, col) for col < r-1; each is
  // applied to the columns of G (all rows), to rows col and r-1 of G (the same change of the kept
  // basis vectors, rows < r), and accumulated into W.
  Mat Wm(k, k);
  for (int i = 0; i < k; ++i) Wm(i, i) = 1.0;
  for (int r = k; r >= 2; --r) {
    const int piv = r - 1;
    for (int col = 0; col < piv; ++col) {
      // column rotation (col, piv): [a b] -> [0 rho]:  new_col = cc*a' ... chosen so that
      // G(r, col) becomes zero:  new_col = cc * col - s * piv,  new_piv = conj(s) * col + cc * piv
      const cplx a = G(r, col), b = G(r, piv);
      if (a == cplx(0.0)) continue;
      double cc;
      cplx ss;
      givens(b, a, cc, ss);   // maps (b, a) -> (rho, 0): rho = cc b + ss a, 0 = -conj(ss) b + cc a
      // column op: piv <- cc*piv + ss*col, col <- -conj(ss)*piv + cc*col  (a unitary 2 x 2 on columns)
      for (int i = 0; i <= k; ++i) {
        const cplx vp = G(i, piv), vc = G(i, col);
        G(i, piv) = cc * vp + ss * vc;
        G(i, col) = -std::conj(ss) * vp + cc * vc;
      }
      for (int i = 0; i < k; ++i) {
        const cplx vp = Wm(i, piv), vc = Wm(i, col);
        Wm(i, piv) = cc * vp + ss * vc;
        Wm(i, col) = -std::conj(ss) * vp + cc * vc;
      }
      // the same change of basis on the rows (conjugate transpose of the column op)
      for (int j = 0; j < k; ++j) {
        const cplx vp = G(piv, j), vc = G(col, j);
        G(piv, j) = cc * vp + std::conj(ss) * vc;
        G(col, j) = -ss * vp + cc * vc;
      }
    }
  }
  // C = P_k W
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < k; ++j) {
      cplx s = 0.0;
      for (int l = 0; l < k; ++l) s += P(i, l) * Wm(l, j);
      C[(size_t)i * k + j] = s;
    }
  for (int i = 0; i <= k; ++i)
    for (int j = 0; j < k; ++j) Hh[(size_t)i * k + j] = (i > j + 1) ? cplx(0.0) : G(i, j);
  // Givens QR of the Hessenberg block
  Mat Rr(k + 1, k);
  for (int i = 0; i <= k; ++i)
    for (int j = 0; j < k; ++j) Rr(i, j) = (i > j + 1) ? cplx(0.0) : G(i, j);
  for (int j = 0; j < k; ++j) {
    double cc;
    cplx ss;
    givens(Rr(j, j), Rr(j + 1, j), cc, ss);
    for (int col = j; col < k; ++col) {
      const cplx t = cc * Rr(j, col) + ss * Rr(j + 1, col);
      Rr(j + 1, col) = -std::conj(ss) * Rr(j, col) + cc * Rr(j + 1, col);
      Rr(j, col) = t;
    }
    cs[j] = cc;
    sn[j] = ss;
  }
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < k; ++j) R[(size_t)i * k + j] = (i <= j) ? Rr(i, j) : cplx(0.0);
  return true;
}

}  // namespace mgh

extern "C" mgh_status mgh_debug_deflate(int m, int k, const mgh_cdouble* Hbar, const mgh_cdouble* c,
                                        mgh_cdouble* C, mgh_cdouble* Hh, mgh_cdouble* R, double* cs,
                                        mgh_cdouble* sn) {
  if (m < 2 || m > mgh::kMaxRestart || k < 1 || k >= m || !Hbar || !c || !C || !Hh || !R || !cs || !sn)
    return MGH_INVALID_ARG;
  using cplx = std::complex<double>;
  const bool ok = mgh::deflate_restart(m, k, reinterpret_cast<const cplx*>(Hbar), reinterpret_cast<const cplx*>(c),
                                       reinterpret_cast<cplx*>(C), reinterpret_cast<cplx*>(Hh),
                                       reinterpret_cast<cplx*>(R), cs, reinterpret_cast<cplx*>(sn));
  return ok ? MGH_OK : MGH_NOT_CONVERGED;
}
