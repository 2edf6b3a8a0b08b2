// Host construction of the 1-D spectral-element tables in extended precision.
//
// Sec. VI.A: the element nodes are the Gauss-Lobatto-Legendre (GLL) points
// (+-1 and the roots of P_p'), the overlap is integrated with the GLL rule on
// them (diagonal M), and all other integrals use the Gauss-Legendre rule.
// Only nq = p + 1 Gauss points are used on the device.  With that choice the
// degree-p nodal interpolant is determined by its values at the Gauss points,
// so the 1-D stiffness D^T W D equals B^T (Dg^T W Dg) B with Dg the derivative
// matrix of the Lagrange basis on the Gauss points; the kinetic form can then be
// applied in Gauss-point space (see elements.cu).
#include <cmath>
#include <stdexcept>
#include <vector>

#include "tdks_internal.h"

namespace {

typedef long double ld;

// P_n(x) and P_n'(x) by the three-term recurrence; |x| < 1 for the derivative.
void legendre(int n, ld x, ld* P, ld* dP) {
  ld p0 = 1.0L, p1 = x;
  if (n == 0) {
    *P = 1.0L;
    *dP = 0.0L;
    return;
  }
  for (int k = 1; k < n; ++k) {
    ld p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1);
    p0 = p1;
    p1 = p2;
  }
  *P = p1;
  *dP = n * (p0 - x * p1) / (1.0L - x * x);
}

const ld kPi = 3.141592653589793238462643383279502884L;

void gll_nodes(int p, std::vector<ld>& x, std::vector<ld>& w) {
  x.assign(p + 1, 0.0L);
  w.assign(p + 1, 0.0L);
  x[0] = -1.0L;
  x[p] = 1.0L;
  for (int i = 1; i < p; ++i) {
    ld t = -cosl(kPi * i / p);
    for (int it = 0; it < 100; ++it) {
      ld P, dP;
      legendre(p, t, &P, &dP);
      ld d2P = (2.0L * t * dP - (ld)p * (p + 1) * P) / (1.0L - t * t);
      ld step = dP / d2P;
      t -= step;
      if (fabsl(step) < 1e-30L) break;
    }
    x[i] = t;
  }
  for (int i = 0; i <= p; ++i) {
    ld P;
    if (i == 0)
      P = (p % 2) ? -1.0L : 1.0L;
    else if (i == p)
      P = 1.0L;
    else {
      ld dP;
      legendre(p, x[i], &P, &dP);
    }
    w[i] = 2.0L / ((ld)p * (p + 1) * P * P);
  }
}

void gauss_nodes(int n, std::vector<ld>& x, std::vector<ld>& w) {
  x.assign(n, 0.0L);
  w.assign(n, 0.0L);
  for (int i = 0; i < n; ++i) {
    ld t = -cosl(kPi * (i + 0.75L) / (n + 0.5L));
    for (int it = 0; it < 100; ++it) {
      ld P, dP;
      legendre(n, t, &P, &dP);
      ld step = P / dP;
      t -= step;
      if (fabsl(step) < 1e-30L) break;
    }
    ld P, dP;
    legendre(n, t, &P, &dP);
    x[i] = t;
    w[i] = 2.0L / ((1.0L - t * t) * dP * dP);
  }
}

// Lagrange basis on nodes z evaluated (value, derivative) at point x.
void lagrange_at(const std::vector<ld>& z, ld x, std::vector<ld>& val, std::vector<ld>& der) {
  int n = (int)z.size();
  val.assign(n, 0.0L);
  der.assign(n, 0.0L);
  for (int i = 0; i < n; ++i) {
    ld v = 1.0L;
    for (int m = 0; m < n; ++m)
      if (m != i) v *= (x - z[m]) / (z[i] - z[m]);
    val[i] = v;
    ld d = 0.0L;
    for (int l = 0; l < n; ++l) {
      if (l == i) continue;
      ld t = 1.0L / (z[i] - z[l]);
      for (int m = 0; m < n; ++m)
        if (m != i && m != l) t *= (x - z[m]) / (z[i] - z[m]);
      d += t;
    }
    der[i] = d;
  }
}

}  // namespace

Tables1D tdks_build_tables(int p, int nq) {
  if (p < 1 || p > TDKS_MAX_P1 - 1) throw std::invalid_argument("p out of range");
  if (nq != p + 1) throw std::invalid_argument("nq must be p+1");
  const int P1 = p + 1;
  std::vector<ld> xi, w, eta, om;
  gll_nodes(p, xi, w);
  gauss_nodes(nq, eta, om);
  std::vector<ld> B(nq * P1), D(nq * P1), Dg(nq * nq);
  std::vector<ld> val, der;
  for (int q = 0; q < nq; ++q) {
    lagrange_at(xi, eta[q], val, der);
    for (int i = 0; i < P1; ++i) {
      B[q * P1 + i] = val[i];
      D[q * P1 + i] = der[i];
    }
    lagrange_at(eta, eta[q], val, der);
    for (int r = 0; r < nq; ++r) Dg[q * nq + r] = der[r];
  }
  Tables1D t;
  t.xi.resize(P1);
  t.w.resize(P1);
  t.eta.resize(nq);
  t.omega.resize(nq);
  for (int i = 0; i < P1; ++i) {
    t.xi[i] = (double)xi[i];
    t.w[i] = (double)w[i];
  }
  for (int q = 0; q < nq; ++q) {
    t.eta[q] = (double)eta[q];
    t.omega[q] = (double)om[q];
  }
  t.B.resize(nq * P1);
  t.D.resize(nq * P1);
  for (int k = 0; k < nq * P1; ++k) {
    t.B[k] = (double)B[k];
    t.D[k] = (double)D[k];
  }
  t.Kq.resize(nq * nq);
  for (int a = 0; a < nq; ++a)
    for (int b = 0; b < nq; ++b) {
      ld s = 0.0L;
      for (int m = 0; m < nq; ++m) s += Dg[m * nq + a] * om[m] * Dg[m * nq + b];
      t.Kq[a * nq + b] = (double)s;
    }
  t.K1.resize(P1 * P1);
  t.Mg.resize(P1 * P1);
  for (int i = 0; i < P1; ++i)
    for (int j = 0; j < P1; ++j) {
      ld sk = 0.0L, sm = 0.0L;
      for (int q = 0; q < nq; ++q) {
        sk += D[q * P1 + i] * om[q] * D[q * P1 + j];
        sm += B[q * P1 + i] * om[q] * B[q * P1 + j];
      }
      t.K1[i * P1 + j] = (double)sk;
      t.Mg[i * P1 + j] = (double)sm;
    }
  return t;
}
