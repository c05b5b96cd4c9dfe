// Host-side tables of the DSEM-SL step: solution nodes, quadrature weights, barycentric
// weights, face basis values (Sec. 3, eq. gaussquad, 3.5, quad) and the constrained-fit
// operators (Sec. 4.3, eq. matrix_a).  Computed once per context in long double.
#include <algorithm>
#include <cmath>
#include <stdexcept>

#include "sl_internal.h"

namespace sl {
namespace {

using ld = long double;
const ld PI_L = 3.141592653589793238462643383279502884L;

// Legendre P_n and its derivative at x by the three-term recurrence.
void legendre(int n, ld x, ld& p, ld& dp) {
  ld p0 = 1.0L, p1 = x;
  if (n == 0) { p = 1.0L; dp = 0.0L; return; }
  for (int k = 2; k <= n; ++k) {
    ld pk = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k;
    p0 = p1;
    p1 = pk;
  }
  p = p1;
  dp = n * (x * p1 - p0) / (x * x - 1.0L);
}

// Gauss-Legendre nodes on [-1, 1] by Newton's method from Chebyshev-like initial guesses.
void gauss_legendre(int n, std::vector<ld>& x, std::vector<ld>& w) {
  x.assign(n, 0.0L);
  w.assign(n, 0.0L);
  if (n == 1) { x[0] = 0.0L; w[0] = 2.0L; return; }
  for (int i = 0; i < n; ++i) {
    ld z = -std::cos(PI_L * (i + 0.75L) / (n + 0.5L));
    for (int it = 0; it < 100; ++it) {
      ld p, dp;
      legendre(n, z, p, dp);
      ld dz = p / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-19L) break;
    }
    ld p, dp;
    legendre(n, z, p, dp);
    x[i] = z;
    w[i] = 2.0L / ((1.0L - z * z) * dp * dp);
  }
}

// Fejer's first rule on Chebyshev-Gauss nodes, closed form (weights on [-1, 1]).
void fejer1(int n, std::vector<ld>& x, std::vector<ld>& w) {
  x.assign(n, 0.0L);
  w.assign(n, 0.0L);
  for (int i = 0; i < n; ++i) {
    ld th = (2 * i + 1) * PI_L / (2 * n);
    x[i] = std::cos(th);
    ld s = 1.0L;
    for (int j = 1; j <= n / 2; ++j) s -= 2.0L * std::cos(2 * j * th) / (4.0L * j * j - 1.0L);
    w[i] = 2.0L * s / n;
  }
}

// Symmetric eigen-decomposition by cyclic Jacobi rotations: A = V diag(e) V^T (row-major).
void jacobi_eigen(int m, std::vector<ld> A, std::vector<ld>& e, std::vector<ld>& V) {
  V.assign(m * m, 0.0L);
  for (int i = 0; i < m; ++i) V[i * m + i] = 1.0L;
  for (int sweep = 0; sweep < 100; ++sweep) {
    ld off = 0.0L, diag = 0.0L;
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) (i == j ? diag : off) += A[i * m + j] * A[i * m + j];
    if (off <= 1e-36L * diag || off == 0.0L) break;
    for (int p = 0; p < m; ++p)
      for (int q = p + 1; q < m; ++q) {
        ld apq = A[p * m + q];
        if (apq == 0.0L) continue;
        ld theta = (A[q * m + q] - A[p * m + p]) / (2.0L * apq);
        ld t = (theta >= 0 ? 1.0L : -1.0L) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0L));
        ld c = 1.0L / std::sqrt(t * t + 1.0L), s = t * c;
        for (int k = 0; k < m; ++k) {          // A <- A J
          ld akp = A[k * m + p], akq = A[k * m + q];
          A[k * m + p] = c * akp - s * akq;
          A[k * m + q] = s * akp + c * akq;
        }
        for (int k = 0; k < m; ++k) {          // A <- J^T A
          ld apk = A[p * m + k], aqk = A[q * m + k];
          A[p * m + k] = c * apk - s * aqk;
          A[q * m + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < m; ++k) {          // V <- V J
          ld vkp = V[k * m + p], vkq = V[k * m + q];
          V[k * m + p] = c * vkp - s * vkq;
          V[k * m + q] = s * vkp + c * vkq;
        }
      }
  }
  e.resize(m);
  for (int i = 0; i < m; ++i) e[i] = A[i * m + i];
}

// Inverse of a dense matrix by Gauss-Jordan elimination with partial pivoting.
std::vector<ld> invert(int n, std::vector<ld> A) {
  std::vector<ld> I(n * n, 0.0L);
  for (int i = 0; i < n; ++i) I[i * n + i] = 1.0L;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[r * n + c]) > std::fabs(A[piv * n + c])) piv = r;
    if (A[piv * n + c] == 0.0L) throw std::runtime_error("singular matrix in fit operator");
    if (piv != c)
      for (int k = 0; k < n; ++k) {
        std::swap(A[c * n + k], A[piv * n + k]);
        std::swap(I[c * n + k], I[piv * n + k]);
      }
    ld inv = 1.0L / A[c * n + c];
    for (int k = 0; k < n; ++k) { A[c * n + k] *= inv; I[c * n + k] *= inv; }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      ld f = A[r * n + c];
      if (f == 0.0L) continue;
      for (int k = 0; k < n; ++k) { A[r * n + k] -= f * A[c * n + k]; I[r * n + k] -= f * I[c * n + k]; }
    }
  }
  return I;
}

}  // namespace

Basis1D make_basis(int n, int basis) {
  std::vector<ld> x, w;
  if (basis == SL_GAUSS_LEGENDRE) gauss_legendre(n, x, w);
  else fejer1(n, x, w);
  // map [-1, 1] -> [0, 1] in increasing order
  std::vector<std::pair<ld, ld>> xw;
  for (int i = 0; i < n; ++i) xw.push_back({(1.0L + x[i]) / 2.0L, w[i] / 2.0L});
  std::sort(xw.begin(), xw.end());
  std::vector<ld> xi(n), wi(n), lam(n);
  for (int i = 0; i < n; ++i) { xi[i] = xw[i].first; wi[i] = xw[i].second; }
  for (int j = 0; j < n; ++j) {
    ld prod = 1.0L;
    for (int m = 0; m < n; ++m)
      if (m != j) prod *= (xi[j] - xi[m]);
    lam[j] = 1.0L / prod;
  }
  Basis1D b;
  b.n = n;
  for (int j = 0; j < n; ++j) {
    b.xi.push_back((double)xi[j]);
    b.w.push_back((double)wi[j]);
    b.lam.push_back((double)lam[j]);
  }
  // face values from the barycentric (first) form l_j(x) = lam_j prod_{m != j} (x - xi_m)
  for (ld face : {0.0L, 1.0L}) {
    for (int j = 0; j < n; ++j) {
      ld prod = lam[j];
      for (int m = 0; m < n; ++m)
        if (m != j) prod *= (face - xi[m]);
      (face == 0.0L ? b.l0 : b.l1).push_back((double)prod);
    }
  }
  return b;
}

void finish_fit(FitOps& f, bool soft) {
  const int m = f.m, nd = f.nd;
  if (m == 0) {                    // no linear rows: phi_L = phihat, q = a
    f.S.assign(nd * nd, 0.0);
    for (int r = 0; r < nd; ++r) f.S[r * nd + r] = 1.0;
    return;
  }
  std::vector<ld> C(f.C.begin(), f.C.end());
  if (!soft) {
    // C^+ = C^T (C C^T)^+ with the pseudo-inverse of the Gram matrix from its eigen-decomposition
    std::vector<ld> G(m * m, 0.0L);
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) {
        ld s = 0.0L;
        for (int k = 0; k < nd; ++k) s += C[i * nd + k] * C[j * nd + k];
        G[i * m + j] = s;
      }
    std::vector<ld> e, V;
    jacobi_eigen(m, G, e, V);
    ld emax = 0.0L;
    for (ld v : e) emax = std::max(emax, std::fabs(v));
    std::vector<ld> Gp(m * m, 0.0L);
    for (int k = 0; k < m; ++k) {
      if (e[k] <= 1e-14L * emax) continue;       // dependent rows (2D corners)
      ld inv = 1.0L / e[k];
      for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) Gp[i * m + j] += V[i * m + k] * inv * V[j * m + k];
    }
    f.Cpinv.assign(nd * m, 0.0);
    for (int r = 0; r < nd; ++r)
      for (int j = 0; j < m; ++j) {
        ld s = 0.0L;
        for (int i = 0; i < m; ++i) s += C[i * nd + r] * Gp[i * m + j];
        f.Cpinv[r * m + j] = (double)s;
      }
  } else {
    std::vector<ld> A(nd * nd, 0.0L);
    for (int r = 0; r < nd; ++r) A[r * nd + r] = 1.0L;
    for (int i = 0; i < m; ++i)
      for (int r = 0; r < nd; ++r)
        for (int c = 0; c < nd; ++c) A[r * nd + c] += C[i * nd + r] * C[i * nd + c];
    std::vector<ld> S = invert(nd, A);
    f.S.assign(S.begin(), S.end());
    f.SCt.assign(nd * m, 0.0);
    for (int r = 0; r < nd; ++r)
      for (int j = 0; j < m; ++j) {
        ld s = 0.0L;
        for (int k = 0; k < nd; ++k) s += S[r * nd + k] * C[j * nd + k];
        f.SCt[r * m + j] = (double)s;
      }
  }
}

FitOps make_fit_1d(const Basis1D& b, unsigned mask) {
  FitOps f;
  f.nd = b.n;
  if (mask & SL_C_BOUNDARY) {
    f.C.insert(f.C.end(), b.l0.begin(), b.l0.end());
    f.C.insert(f.C.end(), b.l1.begin(), b.l1.end());
    f.m += 2;
  }
  if (mask & SL_C_MASS) {
    f.C.insert(f.C.end(), b.w.begin(), b.w.end());
    f.m += 1;
  }
  return f;
}

FitOps make_fit_2d(const Basis1D& b, unsigned mask, bool soft) {
  FitOps f;
  const int n = b.n, nd = n * n;
  f.nd = nd;
  auto add_row = [&](const std::vector<double>& r) { f.C.insert(f.C.end(), r.begin(), r.end()); f.m++; };
  if (mask & SL_C_BOUNDARY) {
    for (int face = 0; face < 4; ++face)
      for (int q = 0; q < n; ++q) {
        std::vector<double> r(nd, 0.0);
        const std::vector<double>& L = (face == 1 || face == 3) ? b.l1 : b.l0;
        for (int k = 0; k < n; ++k) {
          if (face < 2) r[q * n + k] = L[k];   // W/E: sum_i phi[q][i] l_i(face)
          else r[k * n + q] = L[k];            // S/N: sum_j phi[j][q] l_j(face)
        }
        add_row(r);
      }
  }
  if (mask & SL_C_MASS) {
    std::vector<double> r(nd);
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) r[j * n + i] = b.w[j] * b.w[i];
    add_row(r);
  }
  finish_fit(f, soft);
  return f;
}

}  // namespace sl
