// Fast-diagonalization data for the Poisson stiffness on a tensor-product mesh.
//
// On axis-aligned hexahedra the stiffness of Eq. 19 is separable:
//   K = Ax (x) By (x) Bz + Bx (x) Ay (x) Bz + Bx (x) By (x) Az      (interior nodes)
// with the 1-D assembled matrices A_d = sum_e (2/h_e) K1 and B_d = sum_e (h_e/2) Mg
// (K1 = D^T W D, Mg = B^T W B on the Gauss rule).  With the generalized eigenpairs
// A_d S_d = B_d S_d diag(lam_d), S_d^T B_d S_d = I, the inverse is
//   K^-1 = (Sx (x) Sy (x) Sz) diag(lam_x + lam_y + lam_z)^-1 (Sx (x) Sy (x) Sz)^T
// (fast diagonalization, Lynch, Rice & Thomas 1964).  Here it serves as the CG
// preconditioner; for these meshes it is the exact inverse up to rounding.
//
// Host algorithm per axis: Cholesky B = L L^T, C = L^-1 A L^-T, cyclic Jacobi
// eigenvalue iteration on C (Golub & Van Loan, Sec. 8.5), S = L^-T Q.
#include <cmath>
#include <stdexcept>
#include <vector>

#include "tdks_internal.h"

namespace {

void jacobi_eigen(std::vector<double>& C, int n, std::vector<double>& V, std::vector<double>& lam) {
  V.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
  auto at = [&](int i, int j) -> double& { return C[(size_t)i * n + j]; };
  double norm = 0.0;
  for (size_t k = 0; k < C.size(); ++k) norm += C[k] * C[k];
  norm = std::sqrt(norm);
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += at(p, q) * at(p, q);
    if (std::sqrt(2.0 * off) <= 1e-15 * norm) break;
    for (int p = 0; p < n; ++p) {
      for (int q = p + 1; q < n; ++q) {
        const double apq = at(p, q);
        if (std::fabs(apq) <= 1e-300) continue;
        const double theta = (at(q, q) - at(p, p)) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {       // columns p, q
          const double akp = at(k, p), akq = at(k, q);
          at(k, p) = c * akp - s * akq;
          at(k, q) = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {       // rows p, q
          const double apk = at(p, k), aqk = at(q, k);
          at(p, k) = c * apk - s * aqk;
          at(q, k) = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
          V[(size_t)k * n + p] = c * vkp - s * vkq;
          V[(size_t)k * n + q] = s * vkp + c * vkq;
        }
      }
    }
  }
  lam.resize(n);
  for (int i = 0; i < n; ++i) lam[i] = at(i, i);
}

}  // namespace

// S (row-major [i][mode], n x n) and lam (n) for one axis with breakpoints br (n_el + 1).
void tdks_fdm_axis(const Tables1D& t, int p, const double* br, int n_el, std::vector<double>& S,
                   std::vector<double>& lam) {
  const int P1 = p + 1;
  const int N = n_el * p + 1;    // all nodes
  const int n = N - 2;           // interior
  if (n < 1) throw std::invalid_argument("no interior node");
  std::vector<double> A((size_t)n * n, 0.0), B((size_t)n * n, 0.0);
  for (int e = 0; e < n_el; ++e) {
    const double h = br[e + 1] - br[e];
    for (int a = 0; a < P1; ++a)
      for (int b = 0; b < P1; ++b) {
        const int I = e * p + a - 1, J = e * p + b - 1;
        if (I < 0 || J < 0 || I >= n || J >= n) continue;
        A[(size_t)I * n + J] += (2.0 / h) * t.K1[a * P1 + b];
        B[(size_t)I * n + J] += (0.5 * h) * t.Mg[a * P1 + b];
      }
  }
  // Cholesky B = L L^T (lower, in place in L)
  std::vector<double> L((size_t)n * n, 0.0);
  for (int j = 0; j < n; ++j) {
    double d = B[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) d -= L[(size_t)j * n + k] * L[(size_t)j * n + k];
    if (!(d > 0)) throw std::runtime_error("1-D mass not positive definite");
    const double ljj = std::sqrt(d);
    L[(size_t)j * n + j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      double s = B[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) s -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
      L[(size_t)i * n + j] = s / ljj;
    }
  }
  // W = L^-1 A (forward substitution on every column), C = L^-1 W^T
  auto lsolve = [&](std::vector<double>& X) {   // X <- L^-1 X, X is n x n row-major
    for (int c = 0; c < n; ++c)
      for (int i = 0; i < n; ++i) {
        double s = X[(size_t)i * n + c];
        for (int k = 0; k < i; ++k) s -= L[(size_t)i * n + k] * X[(size_t)k * n + c];
        X[(size_t)i * n + c] = s / L[(size_t)i * n + i];
      }
  };
  std::vector<double> W = A;
  lsolve(W);
  std::vector<double> C((size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) C[(size_t)i * n + j] = W[(size_t)j * n + i];
  lsolve(C);
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) {
      const double s = 0.5 * (C[(size_t)i * n + j] + C[(size_t)j * n + i]);
      C[(size_t)i * n + j] = s;
      C[(size_t)j * n + i] = s;
    }
  std::vector<double> Q;
  jacobi_eigen(C, n, Q, lam);
  // S = L^-T Q (back substitution on every column)
  S = Q;
  for (int c = 0; c < n; ++c)
    for (int i = n - 1; i >= 0; --i) {
      double s = S[(size_t)i * n + c];
      for (int k = i + 1; k < n; ++k) s -= L[(size_t)k * n + i] * S[(size_t)k * n + c];
      S[(size_t)i * n + c] = s / L[(size_t)i * n + i];
    }
}

// Symmetric eigendecomposition of a small dense matrix (C is overwritten):
// columns of V are the eigenvectors, lam the eigenvalues.
void tdks_sym_eigen(std::vector<double>& C, int n, std::vector<double>& V, std::vector<double>& lam) {
  jacobi_eigen(C, n, V, lam);
}
