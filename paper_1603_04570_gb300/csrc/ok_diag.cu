// Spectral diagnostics of the preconditioned Jacobian, host side.
//
// Sec. 3: with A inverted exactly, the right-preconditioned Jacobian J P^{-1}
// has the eigenvalue 1 (multiplicity N_v) and the eigenvalues of S~^{-1} S;
// Lemma 1 makes the latter real and Lemma 2 confines them (K perturbed to be
// SPD) to [1/2 + sqrt(c) l_- / (2 eps), 1 + sqrt(c) l_+ / (2 eps)), l_-/l_+
// the clipped extremes of eig(M^{-1} M_E).  FGMRES already runs the Arnoldi
// process on J P^{-1}: J Z_k = V_{k+1} Hbar_k with Z_k = P^{-1} V_k (Saad,
// SISC 1993).  The eigenvalues of the square part H_k (Ritz values) estimate
// that spectrum at any problem size at the cost of the solve itself.
//
// The device keeps Hbar reduced to triangular form by Givens rotations (the
// least-squares update); this file restores it and computes the eigenvalues
// of a small upper Hessenberg matrix.  Both routines are plain host code and
// need no GPU.
#include <algorithm>
#include <cmath>
#include <limits>
#include <vector>

#include "ok.h"

namespace {

// a(i, j) of a dense k x k row-major array
struct Dense {
  int k;
  std::vector<double> a;
  explicit Dense(int k_) : k(k_), a((size_t)k_ * k_, 0.0) {}
  double& operator()(int i, int j) { return a[(size_t)i * k + j]; }
};

// eigenvalues of [[a, b], [c, d]]
void eig2(double a, double b, double c, double d, double* re, double* im) {
  const double p = 0.5 * (a - d);
  const double disc = p * p + b * c;
  if (disc >= 0.0) {
    const double z = p + std::copysign(std::sqrt(disc), p);   // no cancellation
    re[0] = d + z;
    re[1] = z != 0.0 ? d - (b * c) / z : d;
    im[0] = im[1] = 0.0;
  } else {
    re[0] = re[1] = d + p;
    im[0] = std::sqrt(-disc);
    im[1] = -im[0];
  }
}

// Householder reflector I - tau v v^T with v = (1, v1, v2) mapping (x, y, z)
// to a multiple of e_1; returns false when (x, y, z) = 0 (nothing to do).
bool house3(double x, double y, double z, double& v1, double& v2, double& tau) {
  const double sc = std::fabs(x) + std::fabs(y) + std::fabs(z);   // the reflector ignores scale
  if (sc == 0.0) return false;
  x /= sc;
  y /= sc;
  z /= sc;
  const double nrm = std::sqrt(x * x + y * y + z * z);
  const double alpha = -std::copysign(nrm, x);
  const double u0 = x - alpha;                      // |u0| >= |x|: no cancellation
  v1 = y / u0;
  v2 = z / u0;
  tau = (alpha - x) / alpha;                        // 2 / (v^T v)
  return true;
}

int hessenberg_qr(int k, const double* H, int ldh, double* re, double* im);

}  // namespace

extern "C" {

int ok_givens_unrotate(int k, double* H, int ldh, const double* cs, const double* sn) {
  if (k < 0 || (k > 0 && (!H || !cs || !sn)) || ldh < k + 1) return OK_ERR_INVALID_ARG;
  for (int j = 0; j < k; ++j) {
    double* h = H + (size_t)ldh * j;
    h[j + 1] = 0.0;                                 // reduced form: zero below the diagonal
    for (int i = j; i >= 0; --i) {                  // G_0^T ... G_j^T applied to column j
      const double a = h[i], b = h[i + 1];
      h[i] = cs[i] * a - sn[i] * b;
      h[i + 1] = sn[i] * a + cs[i] * b;
    }
    for (int i = j + 2; i <= k; ++i) h[i] = 0.0;
  }
  return OK_SUCCESS;
}

int ok_hessenberg_eigenvalues(int k, const double* H, int ldh, double* re, double* im) {
  if (k < 0 || k > 4096 || (k > 0 && (!H || !re || !im)) || ldh < k) return OK_ERR_INVALID_ARG;
  try {
    return hessenberg_qr(k, H, ldh, re, im);      // a dense k x k working copy
  } catch (...) {
    return OK_ERR_NOMEM;
  }
}

}  // extern "C"

namespace {

int hessenberg_qr(int k, const double* H, int ldh, double* re, double* im) {
  Dense A(k);
  double amax = 0.0;
  for (int j = 0; j < k; ++j)
    for (int i = 0; i <= j + 1 && i < k; ++i) {       // Hessenberg part only
      const double v = H[(size_t)ldh * j + i];
      if (!std::isfinite(v)) return OK_ERR_NONFINITE;
      amax = std::max(amax, std::fabs(v));
    }
  // scaled by a power of two (exact) so that the largest entry is in [1/2, 1):
  // the shift products below neither overflow nor underflow
  int e2 = 0;
  if (amax > 0.0) std::frexp(amax, &e2);
  double fro = 0.0;
  for (int j = 0; j < k; ++j)
    for (int i = 0; i <= j + 1 && i < k; ++i) {
      A(i, j) = std::ldexp(H[(size_t)ldh * j + i], -e2);
      fro += A(i, j) * A(i, j);
    }
  fro = std::sqrt(fro);
  const double eps = std::numeric_limits<double>::epsilon();
  int hi = k - 1, its = 0, total = 0;
  while (hi >= 0) {
    // l: start of the unreduced block ending at hi
    int l = hi;
    for (; l > 0; --l) {
      double s = std::fabs(A(l - 1, l - 1)) + std::fabs(A(l, l));
      if (s == 0.0) s = fro;
      if (std::fabs(A(l, l - 1)) <= eps * s) {
        A(l, l - 1) = 0.0;
        break;
      }
    }
    if (l == hi) {                                  // 1 x 1 block deflates
      re[hi] = A(hi, hi);
      im[hi] = 0.0;
      hi -= 1;
      its = 0;
      continue;
    }
    if (l == hi - 1) {                              // 2 x 2 block deflates
      eig2(A(hi - 1, hi - 1), A(hi - 1, hi), A(hi, hi - 1), A(hi, hi), re + hi - 1, im + hi - 1);
      hi -= 2;
      its = 0;
      continue;
    }
    if (++total > 40 * k) return OK_ERR_NOT_CONVERGED;
    ++its;
    // Shifts: the trailing 2 x 2 block's eigenvalues, through their sum s and
    // product t; every tenth sweep without deflation an exceptional pair from
    // the size of the last subdiagonals breaks a stalled cycle.
    double s, t;
    if (its % 10 == 0) {
      const double w = std::fabs(A(hi, hi - 1)) + std::fabs(A(hi - 1, hi - 2));
      s = 1.5 * w;
      t = w * w;
    } else {
      s = A(hi - 1, hi - 1) + A(hi, hi);
      t = A(hi - 1, hi - 1) * A(hi, hi) - A(hi - 1, hi) * A(hi, hi - 1);
    }
    // first column of (A - s1 I)(A - s2 I) = A^2 - s A + t I in the block
    double x = A(l, l) * A(l, l) + A(l, l + 1) * A(l + 1, l) - s * A(l, l) + t;
    double y = A(l + 1, l) * (A(l, l) + A(l + 1, l + 1) - s);
    double z = A(l + 1, l) * A(l + 2, l + 1);
    // chase the bulge down the block with 3 x 3 reflectors
    for (int p = l; p <= hi - 2; ++p) {
      double v1, v2, tau;
      if (house3(x, y, z, v1, v2, tau)) {
        const int c0 = p > l ? p - 1 : l;
        for (int j = c0; j <= hi; ++j) {            // rows p..p+2 from the left
          const double w = tau * (A(p, j) + v1 * A(p + 1, j) + v2 * A(p + 2, j));
          A(p, j) -= w;
          A(p + 1, j) -= w * v1;
          A(p + 2, j) -= w * v2;
        }
        if (p > l) A(p + 1, p - 1) = A(p + 2, p - 1) = 0.0;
        const int r1 = p + 3 < hi ? p + 3 : hi;
        for (int i = l; i <= r1; ++i) {             // columns p..p+2 from the right
          const double w = tau * (A(i, p) + v1 * A(i, p + 1) + v2 * A(i, p + 2));
          A(i, p) -= w;
          A(i, p + 1) -= w * v1;
          A(i, p + 2) -= w * v2;
        }
      }
      x = A(p + 1, p);
      y = A(p + 2, p);
      z = p + 3 <= hi ? A(p + 3, p) : 0.0;
    }
    // last step: a rotation on rows / columns hi-1, hi removes A(hi, hi-2)
    const double r = std::hypot(x, y);
    if (r > 0.0) {
      const double c = x / r, sg = y / r;
      const int p = hi - 1;
      for (int j = p - 1; j <= hi; ++j) {
        const double a = A(p, j), b = A(p + 1, j);
        A(p, j) = c * a + sg * b;
        A(p + 1, j) = -sg * a + c * b;
      }
      A(p + 1, p - 1) = 0.0;
      for (int i = l; i <= hi; ++i) {
        const double a = A(i, p), b = A(i, p + 1);
        A(i, p) = c * a + sg * b;
        A(i, p + 1) = -sg * a + c * b;
      }
    }
  }
  for (int i = 0; i < k; ++i) {
    re[i] = std::ldexp(re[i], e2);
    im[i] = std::ldexp(im[i], e2);
  }
  return OK_SUCCESS;
}

}  // namespace
