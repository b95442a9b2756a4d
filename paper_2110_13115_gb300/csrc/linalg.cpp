// Small dense FP64 linear algebra on the host for rb_build (l x l, l <= 1024):
// Cholesky factorisation of a Hermitian positive definite matrix, inversion of the
// lower-triangular factor, and the eigen-decomposition of a Hermitian matrix by cyclic
// Jacobi rotations (descending eigenvalues).
#include <algorithm>
#include <cmath>
#include <complex>
#include <numeric>
#include <vector>

#include "linalg.h"

namespace rb {

using cd = std::complex<double>;

// A (n x n, row-major, Hermitian PD) -> lower-triangular L with A = L L^H. Returns false when a
// pivot is not positive (A is not numerically positive definite).
bool cholesky(int n, const cd* A, cd* L) {
  std::fill(L, L + (size_t)n * n, cd(0.0));
  for (int j = 0; j < n; ++j) {
    double d = A[(size_t)j * n + j].real();
    for (int p = 0; p < j; ++p) d -= std::norm(L[(size_t)j * n + p]);
    if (!(d > 0.0) || !std::isfinite(d)) return false;
    const double ljj = std::sqrt(d);
    L[(size_t)j * n + j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      cd s = A[(size_t)i * n + j];
      for (int p = 0; p < j; ++p) s -= L[(size_t)i * n + p] * std::conj(L[(size_t)j * n + p]);
      L[(size_t)i * n + j] = s / ljj;
    }
  }
  return true;
}

// Inverse of a lower-triangular matrix by forward substitution, column by column.
void lower_inverse(int n, const cd* L, cd* Li) {
  std::fill(Li, Li + (size_t)n * n, cd(0.0));
  for (int c = 0; c < n; ++c) {
    Li[(size_t)c * n + c] = 1.0 / L[(size_t)c * n + c];
    for (int i = c + 1; i < n; ++i) {
      cd s = 0.0;
      for (int p = c; p < i; ++p) s += L[(size_t)i * n + p] * Li[(size_t)p * n + c];
      Li[(size_t)i * n + c] = -s / L[(size_t)i * n + i];
    }
  }
}

// Cyclic Jacobi for a Hermitian matrix A (row-major, destroyed). On return w holds the
// eigenvalues in descending order and column j of V (row-major n x n) the unit eigenvector of
// w[j]. Each rotation U = D P zeroes A[p][q]: D = diag(1, e^{-i phi}) makes the (p, q) entry
// real, P is the real Jacobi rotation [[c, s], [-s, c]] with t = sgn(theta)/(|theta| +
// sqrt(theta^2 + 1)), theta = (a_qq - a_pp) / (2 |a_pq|); then A <- U^H A U, V <- V U.
void herm_eig(int n, cd* A, double* w, cd* V) {
  std::fill(V, V + (size_t)n * n, cd(0.0));
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
  auto at = [&](int r, int c) -> cd& { return A[(size_t)r * n + c]; };
  double fro = 0.0;
  for (size_t i = 0; i < (size_t)n * n; ++i) fro += std::norm(A[i]);
  const double tiny = 1e-300;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += std::norm(at(p, q));
    if (off <= 1e-32 * fro || off < tiny) break;
    for (int p = 0; p < n - 1; ++p) {
      for (int q = p + 1; q < n; ++q) {
        const cd apq = at(p, q);
        const double g = std::abs(apq);
        if (g == 0.0) continue;
        const double app = at(p, p).real(), aqq = at(q, q).real();
        if (sweep > 3 && g < 1e-18 * (std::fabs(app) + std::fabs(aqq))) {
          at(p, q) = 0.0;
          at(q, p) = 0.0;
          continue;
        }
        const cd ph = apq / g;  // e^{i phi}
        const double theta = (aqq - app) / (2.0 * g);
        double t = 1.0 / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        if (theta < 0) t = -t;
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        const cd ephm = std::conj(ph);  // e^{-i phi}
        // columns: A U
        for (int r = 0; r < n; ++r) {
          const cd arp = at(r, p), arq = at(r, q);
          at(r, p) = c * arp - s * ephm * arq;
          at(r, q) = s * arp + c * ephm * arq;
        }
        // rows: U^H (A U)
        for (int r = 0; r < n; ++r) {
          const cd xpr = at(p, r), xqr = at(q, r);
          at(p, r) = c * xpr - s * ph * xqr;
          at(q, r) = s * xpr + c * ph * xqr;
        }
        at(p, q) = 0.0;
        at(q, p) = 0.0;
        at(p, p) = at(p, p).real();
        at(q, q) = at(q, q).real();
        for (int r = 0; r < n; ++r) {
          const cd vrp = V[(size_t)r * n + p], vrq = V[(size_t)r * n + q];
          V[(size_t)r * n + p] = c * vrp - s * ephm * vrq;
          V[(size_t)r * n + q] = s * vrp + c * ephm * vrq;
        }
      }
    }
  }
  std::vector<int> idx(n);
  std::iota(idx.begin(), idx.end(), 0);
  std::vector<double> d(n);
  for (int i = 0; i < n; ++i) d[i] = at(i, i).real();
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return d[a] > d[b]; });
  std::vector<cd> Vs((size_t)n * n);
  for (int j = 0; j < n; ++j) {
    w[j] = d[idx[j]];
    for (int r = 0; r < n; ++r) Vs[(size_t)r * n + j] = V[(size_t)r * n + idx[j]];
  }
  std::copy(Vs.begin(), Vs.end(), V);
}

}  // namespace rb

// Host-only hook used by the CPU tests of the eigen-solver (interleaved re/im doubles).
extern "C" int rbx_herm_eig(int n, double* a, double* w, double* v) {
  if (n < 1 || !a || !w || !v) return -1;
  rb::herm_eig(n, reinterpret_cast<std::complex<double>*>(a), w, reinterpret_cast<std::complex<double>*>(v));
  return 0;
}

extern "C" int rbx_cholesky(int n, const double* a, double* l) {
  if (n < 1 || !a || !l) return -1;
  return rb::cholesky(n, reinterpret_cast<const std::complex<double>*>(a), reinterpret_cast<std::complex<double>*>(l))
             ? 0
             : 1;
}
