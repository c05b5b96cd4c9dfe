// Host construction (long double) of the shared 2D step operator for a uniform mesh under a
// constant velocity (a, b): every element then sees the same advected geometry (Sec. 5.3), so the
// remap (eq. 5.4, separable: A_y (x) A_x), the face traces (eq. 2dx/2dy_bnd_interpolate), the
// upwind values (eq. 4.12a), the mass target (eq. remap_mass with the RK quadrature of the face
// flux) and the constrained fit (eq. matrix_a) reduce to a few small operators applied per
// element in structured form (psi: the element's n x n values, rows j = y index):
//   psihat = R_y psi R_x^T                        (separable remap, R = A^{-1} of a uniform shift)
//   x inflow residual, row q = sum_m R_y[q][m] (psi_X[m][.] . r_ox - psi[m][.] . R_x^T l_in,x)
//   y inflow residual, col i = sum_p R_x[i][p] (r_oy . psi_Y[.][p]) - l_in,y . psihat[.][i]
//   mass residual            = K_s . psi + K_x . psi_X + K_y . psi_Y  (target minus mass of psihat)
//   phi_L = psihat + C+ r = psihat + C^T s,  s = (C C^T)^+ r over the inflow-face and mass rows
// (the outflow-face rows meet their targets exactly: they are this element's own traces).  C^T s
// is separable: face rows are l0/l1 along one index and a unit vector along the other, the mass
// row is w (x) w, so the correction costs five products per node.
#include <algorithm>
#include <cmath>
#include <map>

#include "sl_internal.h"

namespace sl {
namespace {
using ld = long double;

std::vector<ld> basis_at(const std::vector<ld>& nodes, ld z) {
  const int n = (int)nodes.size();
  std::vector<ld> v(n, 1.0L);
  for (int j = 0; j < n; ++j)
    for (int m = 0; m < n; ++m)
      if (m != j) v[j] *= (z - nodes[m]) / (nodes[j] - nodes[m]);
  return v;
}

}  // namespace

bool build_mixed2d_const(const sl_ctx* c, double a, double b, double dt, unsigned cons, int rk,
                         std::vector<float>& buf, Mixed2DConstParams& P, std::string& err) {
  const int n = c->n, nd = n * n;
  const Basis1D& B = c->b;
  const double hx = (c->mesh.x1 - c->mesh.x0) / c->mesh.kx, hy = (c->mesh.y1 - c->mesh.y0) / c->mesh.ky;
  if (a == 0.0 || b == 0.0) { err = "the 2D shared-operator path needs both velocity components non-zero"; return false; }
  if (cons & SL_C_ENERGY) { err = "energy is applied by the general 2D mixed path"; return false; }
  std::vector<ld> xi(B.xi.begin(), B.xi.end()), w(B.w.begin(), B.w.end());
  const ld dx = (ld)a * dt / hx, dy = (ld)b * dt / hy;
  // remap matrices R[l][q] = l_q(xi_l - shift)
  std::vector<ld> Rx(nd), Ry(nd);
  for (int l = 0; l < n; ++l) {
    std::vector<ld> vx = basis_at(xi, xi[l] - dx), vy = basis_at(xi, xi[l] - dy);
    for (int q = 0; q < n; ++q) { Rx[l * n + q] = vx[q]; Ry[l * n + q] = vy[q]; }
  }
  const bool xw = a > 0.0, ys = b > 0.0;       // x-upwind neighbour is W (else E); y-upwind is S (else N)
  std::vector<ld> l0 = basis_at(xi, 0.0L), l1 = basis_at(xi, 1.0L);
  const std::vector<ld>& lin_x = xw ? l0 : l1;
  const std::vector<ld>& lout_x = xw ? l1 : l0;
  const std::vector<ld>& lin_y = ys ? l0 : l1;
  const std::vector<ld>& lout_y = ys ? l1 : l0;
  std::vector<ld> r_ox(n, 0.0L), r_oy(n, 0.0L);
  for (int q = 0; q < n; ++q)
    for (int i = 0; i < n; ++i) {
      r_ox[q] += Rx[i * n + q] * lout_x[i];
      r_oy[q] += Ry[i * n + q] * lout_y[i];
    }
  // outflow-face flux functionals (mass): Kx[m][l] = |a| hy sum_s b_s sum_q w_q l_m(eta_q - c dy) l_l(xo - c dx)
  static const double rkb[5][4] = {{}, {1.0}, {0.5, 0.5}, {1.0 / 6, 2.0 / 3, 1.0 / 6}, {1.0 / 6, 1.0 / 3, 1.0 / 3, 1.0 / 6}};
  static const double rkc[5][4] = {{}, {0.0}, {0.0, 1.0}, {0.0, 0.5, 1.0}, {0.0, 0.5, 0.5, 1.0}};
  std::map<double, ld> stages;
  for (int s = 0; s < rk; ++s) stages[rkc[rk][s]] += (ld)rkb[rk][s];
  std::vector<ld> Kx(nd, 0.0L), Ky(nd, 0.0L);
  const ld xo = xw ? 1.0L : 0.0L, yo = ys ? 1.0L : 0.0L;
  for (auto& kv : stages) {
    const ld cs = kv.first, bs = kv.second;
    std::vector<ld> ex = basis_at(xi, xo - cs * dx), ey = basis_at(xi, yo - cs * dy);
    for (int q = 0; q < n; ++q) {
      std::vector<ld> ty = basis_at(xi, xi[q] - cs * dy), tx = basis_at(xi, xi[q] - cs * dx);
      for (int m = 0; m < n; ++m)
        for (int l = 0; l < n; ++l) {
          Kx[m * n + l] += std::fabs((ld)a) * hy * bs * w[q] * ty[m] * ex[l];
          Ky[m * n + l] += std::fabs((ld)b) * hx * bs * w[q] * ey[m] * tx[l];
        }
    }
  }
  const ld lam = (ld)dt / ((ld)hx * hy);
  // rows of the hard fit: W (n), E (n), S (n), N (n), mass (1) -- see make_fit_2d
  const FitOps& F = c->fit[cons & 3u][0];
  const int m = F.m;
  const bool bnd = cons & SL_C_BOUNDARY, mass = cons & SL_C_MASS;
  std::vector<int> cols;                         // residuals kept: inflow x rows, inflow y rows, mass
  if (bnd) {
    const int fx = xw ? 0 : 1, fy = ys ? 2 : 3;
    for (int q = 0; q < n; ++q) cols.push_back(fx * n + q);
    for (int q = 0; q < n; ++q) cols.push_back(fy * n + q);
  }
  if (mass) cols.push_back(bnd ? 4 * n : 0);
  const int mc = (int)cols.size();
  // (C C^T)^+ = (C+)^T C+, restricted to the kept columns: G[r][k]
  std::vector<ld> G((size_t)m * mc, 0.0L);
  for (int r = 0; r < m; ++r)
    for (int k = 0; k < mc; ++k) {
      ld acc = 0.0L;
      for (int q = 0; q < nd; ++q) acc += (ld)F.Cpinv[q * m + r] * (ld)F.Cpinv[q * m + cols[k]];
      G[(size_t)r * mc + k] = acc;
    }
  P = Mixed2DConstParams{};
  P.n = n;
  P.kx = c->mesh.kx;
  P.ky = c->mesh.ky;
  P.xw = xw ? 1 : 0;
  P.ys = ys ? 1 : 0;
  P.per_x = c->mesh.bc[0] == SL_BC_PERIODIC ? 1 : 0;
  P.per_y = c->mesh.bc[2] == SL_BC_PERIODIC ? 1 : 0;
  P.ghost = c->mesh.ghost;
  P.bnd = bnd ? 1 : 0;
  P.mass = mass ? 1 : 0;
  P.mc = mc;
  for (int l = 0; l < n; ++l)
    for (int q = 0; q < n; ++q) {
      P.Rx[l * n + q] = (float)Rx[l * n + q];
      P.Ry[l * n + q] = (float)Ry[l * n + q];
    }
  for (int q = 0; q < n / 2; ++q)
    for (int i = 0; i < n; ++i) {
      P.Rxp[q][i] = make_float2(P.Rx[2 * q * n + i], P.Rx[(2 * q + 1) * n + i]);
      P.Ryp[q][i] = make_float2(P.Ry[2 * q * n + i], P.Ry[(2 * q + 1) * n + i]);
    }
  std::vector<ld> wxr(n, 0.0L), wyr(n, 0.0L);   // R_x^T w, R_y^T w: mass of psihat is wyr^T psi wxr
  for (int p = 0; p < n; ++p) {
    ld xi_in = 0.0L;
    for (int l = 0; l < n; ++l) {
      xi_in += Rx[l * n + p] * lin_x[l];
      wxr[p] += Rx[l * n + p] * w[l];
      wyr[p] += Ry[l * n + p] * w[l];
    }
    P.xix[p] = (float)xi_in;
    P.rox[p] = (float)r_ox[p];
    P.roy[p] = (float)r_oy[p];
    P.liny[p] = (float)lin_y[p];
    P.l0[p] = (float)l0[p];
    P.l1[p] = (float)l1[p];
    P.w[p] = (float)w[p];
  }
  if (mass) {
    const int rm = bnd ? 4 * n : 0;
    for (int k = 0; k < mc; ++k) P.gm[k] = (float)G[(size_t)rm * mc + k];
  }
  buf.clear();
  auto put = [&](const std::vector<ld>& v) {
    size_t off = buf.size();
    for (ld x : v) buf.push_back((float)x);
    return (int)off;
  };
  // tables a thread reads by its own row j are stored [other index][j], so that the n threads of
  // an element read n consecutive floats
  auto transpose = [n](const std::vector<ld>& M) {
    std::vector<ld> T(M.size());
    for (int r = 0; r < n; ++r)
      for (int q = 0; q < n; ++q) T[q * n + r] = M[r * n + q];
    return T;
  };
  // mass residual functionals (reference measure): own psi, x-neighbour psi_X (row j of each) and
  // y-neighbour psi_Y (column j); the mass of psihat is folded into the own functional
  std::vector<ld> Ks(nd), Kxl(nd), Kyl(nd);
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) {
      const int k = j * n + i;
      Ks[k] = w[j] * w[i] - lam * (Kx[k] + Ky[k]) - wyr[j] * wxr[i];
      Kxl[k] = lam * Kx[k];
      Kyl[k] = lam * Ky[k];
    }
  P.o_ks = put(transpose(Ks));
  P.o_kx = put(transpose(Kxl));
  P.o_ky = put(Kyl);                             // column j of psi_Y: entry [m][j]
  P.o_RxT = put(transpose(Rx));
  P.o_RyT = put(transpose(Ry));
  // face rows of G as Gt[(f * mc + k) * n + j] = G[f n + j][k], f = W, E, S, N
  if (bnd) {
    std::vector<ld> Gt((size_t)4 * mc * n);
    for (int f = 0; f < 4; ++f)
      for (int k = 0; k < mc; ++k)
        for (int j = 0; j < n; ++j) Gt[((size_t)f * mc + k) * n + j] = G[(size_t)(f * n + j) * mc + k];
    P.o_g = put(Gt);
  }
  P.o_l0 = put(l0);
  P.o_l1 = put(l1);
  P.o_w = put(w);
  // mass refinement: each element's outflow flux through its x- and y-outflow faces is a fixed
  // float functional of its own values (lam Kx, lam Ky), evaluated alike by the element and by its
  // downstream neighbour; w (x) w in float-float; the mass column of C+
  // the refinement moves mass along C+ e_m, which keeps the face rows only when C C+ e_m = e_m
  bool indep = false;
  if (mass) {
    const int rm = bnd ? 4 * n : 0;
    ld dev = 0.0L;
    for (int k = 0; k < m; ++k) {
      ld acc = 0.0L;
      for (int q = 0; q < nd; ++q) acc += (ld)F.C[(size_t)k * nd + q] * (ld)F.Cpinv[(size_t)q * m + rm];
      dev = std::max(dev, std::fabs(acc - (k == rm ? 1.0L : 0.0L)));
    }
    indep = dev < 1e-9L;
  }
  P.refine = indep ? 1 : 0;
  if (indep) {
    std::vector<ld> fx(nd), fy(nd), wh(nd), wl(nd), cm(nd);
    float sfx = 0.0f, sfy = 0.0f;
    for (int k = 0; k < nd; ++k) {
      fx[k] = (ld)(float)(lam * Kx[k]);
      fy[k] = (ld)(float)(lam * Ky[k]);
    }
    // the sums in the order the kernel forms a row's partial sums and then adds the rows
    for (int j = 0; j < n; ++j) {
      float rx = 0.0f, ry = 0.0f;
      for (int i = 0; i < n; ++i) {
        rx += (float)fx[j * n + i];
        ry += (float)fy[j * n + i];
      }
      sfx += rx;
      sfy += ry;
    }
    P.sfx = sfx;
    P.sfy = sfy;
    const int rmass = bnd ? 4 * n : 0;
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) {
        const double v = B.w[i] * B.w[j];
        wh[j * n + i] = (ld)(float)v;
        wl[j * n + i] = (ld)(float)(v - (double)(float)v);
        cm[j * n + i] = (ld)F.Cpinv[(size_t)(j * n + i) * m + rmass];
      }
    P.o_fx = put(transpose(fx));
    P.o_fy = put(transpose(fy));
    P.o_wh = put(transpose(wh));
    P.o_wl = put(transpose(wl));
    P.o_cm = put(cm);                          // [k][j]: node (j, k) of column j at k n + j
  }
  buf.resize((buf.size() + 3) & ~size_t(3), 0.0f);
  return true;
}

}  // namespace sl
