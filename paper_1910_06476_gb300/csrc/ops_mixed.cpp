// Host construction (long double) of the shared 1D step operator used by the mixed-precision
// path when every element sees the same advected geometry: uniform mesh and constant
// velocity.  Then the particles of every element move by the same reference displacement
// delta = a dt / h, so the remap (eq. 4.9), the traces (eq. remap_bnd), the upwinded boundary
// values (eq. 4.12a), the mass target (eq. remap_mass with the RK quadrature of the face flux)
// and the constrained fit (eq. matrix_a) compose into one linear map
//     phi_L = G_self phi_self + G_up phi_upwind
// applied to every element.  The energy constraint stays per element (it is quadratic); its
// flux needs the upwind and own polynomial at the characteristic feet of the outflow face.
#include <algorithm>
#include <cmath>
#include <map>

#include "sl_internal.h"

namespace sl {
namespace {
using ld = long double;

// Lagrange basis on nodes evaluated at z (product formula, long double)
std::vector<ld> basis_at(const std::vector<ld>& nodes, ld z) {
  const int n = (int)nodes.size();
  std::vector<ld> v(n, 1.0L);
  for (int j = 0; j < n; ++j)
    for (int m = 0; m < n; ++m)
      if (m != j) v[j] *= (z - nodes[m]) / (nodes[j] - nodes[m]);
  return v;
}

}  // namespace

bool build_mixed1d(const sl_ctx* c, const FitOps& fit, double a, double dt, unsigned cons, int rk, int fitmode,
                   Mixed1DParams& P, std::string& err) {
  const int n = c->n;
  const Basis1D& b = c->b;
  const double h = (c->mesh.x1 - c->mesh.x0) / c->mesh.kx;
  if (a == 0.0) { err = "the shared-operator path needs a non-zero velocity"; return false; }
  if (fitmode == SL_FIT_SOFT && (cons & SL_C_ENERGY)) {
    err = "the mixed path supports the energy constraint with the hard fit only";
    return false;
  }
  const ld delta = (ld)a * (ld)dt / (ld)h;
  std::vector<ld> xi(b.xi.begin(), b.xi.end()), w(b.w.begin(), b.w.end());
  std::vector<ld> xs(n);
  for (int i = 0; i < n; ++i) xs[i] = xi[i] + delta;
  // remap R[j][i] = h*_i(xi_j)
  std::vector<ld> R(n * n);
  for (int j = 0; j < n; ++j) {
    std::vector<ld> v = basis_at(xs, xi[j]);
    for (int i = 0; i < n; ++i) R[j * n + i] = v[i];
  }
  const bool left_up = a > 0.0;               // upwind neighbour on the left
  std::vector<ld> l0 = basis_at(xi, 0.0L), l1 = basis_at(xi, 1.0L);
  const std::vector<ld>& lout = left_up ? l1 : l0;
  std::vector<ld> rout(n, 0.0L);              // trace of the remapped polynomial at the outflow face
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) rout[i] += lout[j] * R[j * n + i];
  // distinct stage times of the RK quadrature of the face flux, feet on the outflow face
  static const double rkb[5][4] = {{}, {1.0}, {0.5, 0.5}, {1.0 / 6, 2.0 / 3, 1.0 / 6}, {1.0 / 6, 1.0 / 3, 1.0 / 3, 1.0 / 6}};
  static const double rkc[5][4] = {{}, {0.0}, {0.0, 1.0}, {0.0, 0.5, 1.0}, {0.0, 0.5, 0.5, 1.0}};
  std::map<double, ld> stages;
  for (int s = 0; s < rk; ++s) stages[rkc[rk][s]] += (ld)rkb[rk][s];
  std::vector<std::vector<ld>> feet;
  std::vector<ld> fb;
  for (auto& kv : stages) {
    const ld cs = kv.first;
    const ld z = left_up ? 1.0L - cs * delta : -cs * delta;   // foot in the element's frame
    feet.push_back(basis_at(xi, z));
    fb.push_back(kv.second);
  }
  std::vector<ld> f(n, 0.0L);
  for (size_t s = 0; s < feet.size(); ++s)
    for (int j = 0; j < n; ++j) f[j] += fb[s] * feet[s][j];
  const ld lam = std::fabs((ld)a) * (ld)dt / (ld)h;

  // constraint data d = Ds psi_self + Du psi_up, rows in the order [left, right, mass]
  const int m = fit.m;
  std::vector<ld> Ds(m * n, 0.0L), Du(m * n, 0.0L);
  int r = 0;
  if (cons & SL_C_BOUNDARY) {
    const int in_row = left_up ? 0 : 1, out_row = left_up ? 1 : 0;
    for (int i = 0; i < n; ++i) {
      Du[(r + in_row) * n + i] = rout[i];     // upwind neighbour's outflow trace
      Ds[(r + out_row) * n + i] = rout[i];    // own outflow trace
    }
    r += 2;
  }
  if (cons & SL_C_MASS) {
    for (int i = 0; i < n; ++i) {
      Ds[r * n + i] = w[i] - lam * f[i];
      Du[r * n + i] = lam * f[i];
    }
    ++r;
  }
  std::vector<ld> C(fit.C.begin(), fit.C.end());
  std::vector<ld> Gs(n * n, 0.0L), Gu(n * n, 0.0L);
  if (fitmode == SL_FIT_HARD) {
    // phi_L = R ps + C+ (Ds ps + Du pu - C R ps)
    std::vector<ld> CR(m * n, 0.0L);
    for (int k = 0; k < m; ++k)
      for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) CR[k * n + i] += C[k * n + j] * R[j * n + i];
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) {
        ld gs = R[j * n + i], gu = 0.0L;
        for (int k = 0; k < m; ++k) {
          const ld cp = fit.Cpinv[j * m + k];
          gs += cp * (Ds[k * n + i] - CR[k * n + i]);
          gu += cp * Du[k * n + i];
        }
        Gs[j * n + i] = gs;
        Gu[j * n + i] = gu;
      }
  } else {
    // phi_L = S R ps + S C^T (Ds ps + Du pu)
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) {
        ld gs = 0.0L, gu = 0.0L;
        for (int k = 0; k < n; ++k) gs += (ld)fit.S[j * n + k] * R[k * n + i];
        for (int k = 0; k < m; ++k) {
          gs += (ld)fit.SCt[j * m + k] * Ds[k * n + i];
          gu += (ld)fit.SCt[j * m + k] * Du[k * n + i];
        }
        Gs[j * n + i] = gs;
        Gu[j * n + i] = gu;
      }
  }
  P = Mixed1DParams{};
  P.n = n;
  P.K = c->mesh.kx;
  P.left_up = left_up ? 1 : 0;
  P.periodic = c->mesh.bc[0] == SL_BC_PERIODIC ? 1 : 0;
  P.ghost = c->mesh.ghost;
  P.lam = (float)lam;
  P.m = m;
  P.mass_on = (cons & SL_C_MASS) ? 1 : 0;
  P.energy_on = (cons & SL_C_ENERGY) ? 1 : 0;
  P.nst = (int)feet.size();
  for (int j = 0; j < n * n; ++j) { P.Gs[j] = (float)Gs[j]; P.Gu[j] = (float)Gu[j]; }
  for (int pr = 0; pr < n / 2; ++pr)
    for (int i = 0; i < n; ++i) {
      P.Gp[pr][i] = make_float2(P.Gs[2 * pr * n + i], P.Gs[(2 * pr + 1) * n + i]);
      P.Gp[pr][n + i] = make_float2(P.Gu[2 * pr * n + i], P.Gu[(2 * pr + 1) * n + i]);
    }
  for (int j = 0; j < n; ++j) P.w[j] = (float)w[j];
  for (int s = 0; s < P.nst; ++s) {
    P.fb[s] = (float)fb[s];
    for (int j = 0; j < n; ++j) P.E[s][j] = (float)feet[s][j];
  }
  for (int k = 0; k < m * n; ++k) P.C[k] = (float)C[k];
  if (fitmode == SL_FIT_HARD)
    for (int k = 0; k < n * m; ++k) P.Cp[k] = (float)fit.Cpinv[k];
  // the refinement moves mass along C+ e_m, which keeps the other rows only when C C+ e_m = e_m
  // (the mass row independent of the face rows: n >= 3)
  bool indep = false;
  if (fitmode == SL_FIT_HARD && (cons & SL_C_MASS)) {
    ld dev = 0.0L;
    for (int k = 0; k < m; ++k) {
      ld acc = 0.0L;
      for (int j = 0; j < n; ++j) acc += (ld)fit.C[k * n + j] * (ld)fit.Cpinv[j * m + (m - 1)];
      dev = std::max(dev, std::fabs(acc - (k == m - 1 ? 1.0L : 0.0L)));
    }
    indep = dev < 1e-9L;
  }
  P.refine = indep ? 1 : 0;
  P.lam_lo = (float)(lam - (ld)P.lam);
  float sumf = 0.0f;
  for (int j = 0; j < n; ++j) {
    P.Ff[j] = (float)f[j];
    sumf += P.Ff[j];
    P.wh[j] = (float)b.w[j];
    P.wl[j] = (float)(b.w[j] - (double)P.wh[j]);
    P.cmass[j] = P.refine ? (float)fit.Cpinv[j * m + (m - 1)] : 0.0f;
  }
  P.sumf = sumf;
  return true;
}

}  // namespace sl
