#pragma once
// 2D DSEM-SL step in double precision for any prescribed velocity (Sec. 4, two-dimensional
// scheme), in two kernels with one CTA per element and one thread per particle / node.
//
// Phase 1 (k_p1): seed particles at the tensor Gauss nodes, integrate them with explicit RK
// (eq. 4.4a with u and v), solve the collocation system of eq. 5.4,
//     sum_{l,m} phihat_{ml} h_l(xi*_p) h_m(eta*_p) = phi*_p   for every particle p,
// take the face traces of phihat (eq. 2dx_bnd_interpolate, 2dy_bnd_interpolate) and integrate
// the outflow mass/energy flux through each face over the step (RK quadrature of the face flux,
// the face value being this element's phi^n at the backward characteristic foot).  phihat,
// traces and fluxes go to workspace in global memory.
// Phase 2 (k_p2): upwind the interface values per face point (eq. 4.12a), form the mass and
// energy targets (eq. remap_mass, remap_energy) from own and neighbour fluxes, apply the
// constrained least-squares fit (eq. matrix_a; 4n boundary rows + mass) and the energy
// iteration, and store phi^{n+1}.
//
// The collocation matrix is solved matrix-free by preconditioned iterative refinement:
// phihat <- phihat + M^{-1} (phi* - H phihat), with M = A_y (x) A_x the exact matrix of a uniform
// shift by the element's mean particle displacement, whose inverse is the 1D remap R_y (x) R_x.
// H phihat costs n^2 per particle (the advected basis values are kept in registers).
#include <cfloat>

#include "k_map2d.cuh"

namespace sl {
namespace k2d {

static __constant__ int c_rk_s[5] = {0, 1, 2, 3, 4};
static __constant__ double c_rk_a[5][4][4] = {
    {},
    {{0}},
    {{0, 0}, {1.0, 0}},
    {{0, 0, 0}, {0.5, 0, 0}, {-1.0, 2.0, 0}},
    {{0, 0, 0, 0}, {0.5, 0, 0, 0}, {0, 0.5, 0, 0}, {0, 0, 1.0, 0}}};
static __constant__ double c_rk_b[5][4] = {
    {}, {1.0}, {0.5, 0.5}, {1.0 / 6, 2.0 / 3, 1.0 / 6}, {1.0 / 6, 1.0 / 3, 1.0 / 3, 1.0 / 6}};
static __constant__ double c_rk_c[5][4] = {{}, {0.0}, {0.0, 1.0}, {0.0, 0.5, 1.0}, {0.0, 0.5, 0.5, 1.0}};

constexpr int SOLVE_CAP = 60;
constexpr double SOLVE_RTOL = 1e-15;        // target, relative to max |phi*|
constexpr double SOLVE_STALL = 1e-13;       // a residual that stops improving below this is the floor

// prescribed 2D velocity (divergence-free kinds only)
__device__ __forceinline__ void vel2d(const StepParams& P, double x, double y, double t, double& u, double& v) {
  switch (P.vel_kind) {
    case SL_VEL_ROTATION:
      u = -P.vp[0] * (y - P.vp[2]);
      v = P.vp[0] * (x - P.vp[1]);
      break;
    case SL_VEL_SWIRL: {
      const double c = cospi(t / P.vp[0]);
      const double sx = sinpi(x), sy = sinpi(y);
      u = sx * sx * sinpi(2.0 * y) * c;
      v = -sy * sy * sinpi(2.0 * x) * c;
      break;
    }
    default:
      u = P.vp[0];
      v = P.vp[1];
  }
}

// Lagrange basis on the fixed nodes at z: out_l = lam_l prod_{k != l} (z - xi_k)
template <int NN>
__device__ __forceinline__ void basis_at(const double* xi, const double* lam, double z, double* out) {
  double d[NN], pre[NN];
#pragma unroll
  for (int k = 0; k < NN; ++k) d[k] = z - xi[k];
  double acc = 1.0;
#pragma unroll
  for (int k = 0; k < NN; ++k) { pre[k] = acc; acc *= d[k]; }
  double suf = 1.0;
#pragma unroll
  for (int l = NN - 1; l >= 0; --l) {
    out[l] = lam[l] * pre[l] * suf;
    suf *= d[l];
  }
}

// Lagrange basis and its derivative at z (prefix and suffix products carry their derivatives)
template <int NN>
__device__ __forceinline__ void basis_d(const double* xi, const double* lam, double z, double* L, double* D) {
  double d[NN], pre[NN], dpre[NN];
#pragma unroll
  for (int k = 0; k < NN; ++k) d[k] = z - xi[k];
  double acc = 1.0, dacc = 0.0;
#pragma unroll
  for (int k = 0; k < NN; ++k) {
    pre[k] = acc;
    dpre[k] = dacc;
    dacc = dacc * d[k] + acc;
    acc *= d[k];
  }
  double suf = 1.0, dsuf = 0.0;
#pragma unroll
  for (int l = NN - 1; l >= 0; --l) {
    L[l] = lam[l] * pre[l] * suf;
    D[l] = lam[l] * (dpre[l] * suf + pre[l] * dsuf);
    dsuf = dsuf * d[l] + suf;
    suf *= d[l];
  }
}

// SL_VEL_NODAL along one direction: the elements (index, reference coordinate) that give the field
// at coordinate x, two when x lies on a face (the elements sharing it), else the containing one
// (the boundary element beyond a non-periodic face, wrapped across a periodic one); returns the count
__device__ __forceinline__ int nodal_locate(double x, double lo, double h, int K, bool per, int* ks, double* zs) {
  const double hi = lo + K * h;
  const double s = (x - lo) / h;
  const double r = rint(s);
  if (fabs(x - (lo + r * h)) <= FACE_RTOL * (fabs(lo) + fabs(hi))) {
    const long long ri = (long long)r;
    int cnt = 0;
    for (int side = 0; side < 2; ++side) {
      long long k = side ? ri : ri - 1;
      if (k < 0 || k >= K) {
        if (!per) continue;
        k %= K;
        if (k < 0) k += K;
      }
      ks[cnt] = (int)k;
      zs[cnt] = side ? 0.0 : 1.0;
      ++cnt;
    }
    return cnt;
  }
  const double fk = floor(s);
  long long k = (long long)fk;
  double z = s - fk;
  if (k < 0 || k >= K) {
    if (per) {
      k %= K;
      if (k < 0) k += K;
    } else {
      k = k < 0 ? 0 : K - 1;
      z = s - (double)k;
    }
  }
  ks[0] = (int)k;
  zs[0] = z;
  return 1;
}

// SL_VEL_NODAL: u, v and div u at (x, y, t) from the node velocities of the step (linear in time),
// averaged over the elements that share a face or corner the point lies on
template <int NN>
__device__ __noinline__ void nodal2d(const StepParams& P, const double* xi, const double* lam, double x, double y,
                                     double t, double& u, double& v, double& dv) {
  constexpr int ND = NN * NN;
  const double th = (t - P.t) / P.dt;
  int kxs[2], kys[2];
  double zxs[2], zys[2];
  const int nx = nodal_locate(x, P.x0, P.hx, P.kx, P.bc[0] == SL_BC_PERIODIC, kxs, zxs);
  const int ny = nodal_locate(y, P.y0, P.hy, P.ky, P.bc[2] == SL_BC_PERIODIC, kys, zys);
  const double wt = 1.0 / (nx * ny);
  u = v = dv = 0.0;
  for (int a = 0; a < ny; ++a) {
    double Ly[NN], Dy[NN];
    basis_d<NN>(xi, lam, zys[a], Ly, Dy);
    for (int b = 0; b < nx; ++b) {
      double Lx[NN], Dx[NN];
      basis_d<NN>(xi, lam, zxs[b], Lx, Dx);
      const double* U0 = P.nodal + ((size_t)kys[a] * P.kx + kxs[b]) * ND;
      const double* V0 = U0 + P.nvals;
      const double* U1 = U0 + 2 * P.nvals;
      const double* V1 = U0 + 3 * P.nvals;
      double su = 0.0, sv = 0.0, sux = 0.0, svy = 0.0;
      for (int m = 0; m < NN; ++m) {
        double ru = 0.0, rv = 0.0, rux = 0.0;
#pragma unroll
        for (int l = 0; l < NN; ++l) {
          const double uu = (1.0 - th) * U0[m * NN + l] + th * U1[m * NN + l];
          const double vv = (1.0 - th) * V0[m * NN + l] + th * V1[m * NN + l];
          ru += Lx[l] * uu;
          rv += Lx[l] * vv;
          rux += Dx[l] * uu;
        }
        su += Ly[m] * ru;
        sv += Ly[m] * rv;
        sux += Ly[m] * rux;
        svy += Dy[m] * rv;
      }
      u += wt * su;
      v += wt * sv;
      dv += wt * (sux / P.hx + svy / P.hy);
    }
  }
}

// velocity and its divergence (zero for the analytic kinds, which are divergence free); NOD: the
// kernel is the instantiation that reads nodal velocities (the others carry no nodal code)
template <int NN, bool NOD>
__device__ __forceinline__ void vel2dd(const StepParams& P, const double* xi, const double* lam, double x, double y,
                                       double t, double& u, double& v, double& dv) {
  if (NOD) {
    nodal2d<NN>(P, xi, lam, x, y, t, u, v, dv);
  } else {
    vel2d(P, x, y, t, u, v);
    dv = 0.0;
  }
}

// one explicit RK step of dx/dt = u, dy/dt = v and of the value factor dg/dt = -g div u (eq. 4.8;
// g stays 1 for divergence-free kinds), size h (h < 0 runs the characteristic back)
template <int NN, bool NOD>
__device__ __forceinline__ void rk2d(const StepParams& P, const double* xi, const double* lam, double& x, double& y,
                                     double& g, double t, double h) {
  if (P.vel_kind == SL_VEL_CONST) {
    x += h * P.vp[0];
    y += h * P.vp[1];
    return;
  }
  const int S = c_rk_s[P.rk];
  double kx[4], ky[4], kg[4];
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    if (s < S) {
      double xs = x, ys = y, gs = g;
#pragma unroll
      for (int j = 0; j < s; ++j) {
        xs += h * c_rk_a[P.rk][s][j] * kx[j];
        ys += h * c_rk_a[P.rk][s][j] * ky[j];
        gs += h * c_rk_a[P.rk][s][j] * kg[j];
      }
      double dv;
      vel2dd<NN, NOD>(P, xi, lam, xs, ys, t + c_rk_c[P.rk][s] * h, kx[s], ky[s], dv);
      kg[s] = -gs * dv;
    }
  }
  double sx = 0.0, sy = 0.0, sg = 0.0;
#pragma unroll
  for (int s = 0; s < 4; ++s)
    if (s < S) {
      sx += c_rk_b[P.rk][s] * kx[s];
      sy += c_rk_b[P.rk][s] * ky[s];
      sg += c_rk_b[P.rk][s] * kg[s];
    }
  x += h * sx;
  y += h * sy;
  if (NOD) g += h * sg;
}

// deterministic block reductions (fixed tree order); every thread gets the result
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, ln = threadIdx.x & 31;
  __syncthreads();
  if (ln == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < NT / 32; ++i) s += red[i];
  return s;
}

template <int NT>
__device__ __forceinline__ double block_max(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, ln = threadIdx.x & 31;
  __syncthreads();
  if (ln == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < NT / 32; ++i) s = fmax(s, red[i]);
  return s;
}

template <int NN>
struct Shape {
  static constexpr int ND = NN * NN;
  static constexpr int NT = ((ND > 4 * NN ? ND : 4 * NN) + 31) / 32 * 32;   // threads per CTA
};

__device__ __forceinline__ int nb_index(const StepParams& P, int ex, int ey, int face, bool& wrapped) {
  int jx = ex + (face == 0 ? -1 : face == 1 ? 1 : 0);
  int jy = ey + (face == 2 ? -1 : face == 3 ? 1 : 0);
  wrapped = false;
  if (jx >= 0 && jx < P.kx && jy >= 0 && jy < P.ky) return jy * P.kx + jx;
  if (P.bc[face] != SL_BC_PERIODIC) return -1;
  wrapped = true;
  jx = (jx + P.kx) % P.kx;
  jy = (jy + P.ky) % P.ky;
  return jy * P.kx + jx;
}

template <int NN, bool NOD>
__global__ void __launch_bounds__(Shape<NN>::NT) k_p1(StepParams P0, Tables1D tb, Map2D M,
                                                     const double* __restrict__ in, Work2D W, unsigned* status) {
  constexpr int ND = Shape<NN>::ND, NT = Shape<NN>::NT;
  __shared__ double s_xi[NN], s_lam[NN], s_w[NN], s_l0[NN], s_l1[NN];
  __shared__ double s_phi[ND], s_ph[ND], s_t[ND], s_r[ND];
  __shared__ double s_Rx[ND], s_Ry[ND];
  __shared__ double s_red[NT / 32];
  __shared__ double s_face[4][NMAX][2];
  __shared__ int s_nq[4];
  const int tid = threadIdx.x;
  StepParams P = P0;
  const Elem E = elem_of<NN>(P, M);
  const int ex = E.ex, ey = E.ey;
  const double hx = P.hx, hy = P.hy;
  const double x0 = P.x0 + ex * hx, y0 = P.y0 + ey * hy;
  if (tid < NN) {
    s_xi[tid] = tb.xi[tid]; s_lam[tid] = tb.lam[tid]; s_w[tid] = tb.w[tid];
    s_l0[tid] = tb.l0[tid]; s_l1[tid] = tb.l1[tid];
  }
  const bool part = tid < ND;
  const int i = tid % NN, j = tid / NN;
  if (part) s_phi[tid] = in[E.base + tid];
  __syncthreads();

  // (a)-(b) seed and advect the particle of node (i, j)
  double Lx[NN], Ly[NN], phs = 0.0, dxs = 0.0, dys = 0.0;
  if (part) {
    double x = x0 + hx * s_xi[i], y = y0 + hy * s_xi[j];
    double g = 1.0;                          // value factor of eq. 4.8 (1 when div u = 0)
    rk2d<NN, NOD>(P, s_xi, s_lam, x, y, g, P.t, P.dt);
    const double xs = (x - x0) / hx, ys = (y - y0) / hy;
    basis_at<NN>(s_xi, s_lam, xs, Lx);
    basis_at<NN>(s_xi, s_lam, ys, Ly);
    phs = NOD ? s_phi[tid] * g : s_phi[tid];
    dxs = xs - s_xi[i];
    dys = ys - s_xi[j];
  }
  const double mdx = block_sum<NT>(dxs, s_red) / ND;
  const double mdy = block_sum<NT>(dys, s_red) / ND;
  // 1D remap operators of the mean shift: R[l][q] = h_q(xi_l - shift)
  if (part) {
    double b[NN];
    basis_at<NN>(s_xi, s_lam, s_xi[j] - mdx, b);
    s_Rx[tid] = b[i];                        // row l = j, column q = i
    basis_at<NN>(s_xi, s_lam, s_xi[j] - mdy, b);
    s_Ry[tid] = b[i];
    s_r[tid] = phs;
  }
  __syncthreads();
  // apply M^{-1} = R_y (x) R_x to s_r, add into s_ph (init = 0 on the first call)
  auto precond_add = [&](bool first) {
    if (part) {                              // t[j][l] = sum_q Rx[l][q] r[j][q]   (thread: j, l = i)
      double acc = 0.0;
#pragma unroll
      for (int q = 0; q < NN; ++q) acc += s_Rx[i * NN + q] * s_r[j * NN + q];
      s_t[tid] = acc;
    }
    __syncthreads();
    if (part) {                              // out[m][l] = sum_q Ry[m][q] t[q][l] (thread: m = j, l = i)
      double acc = 0.0;
#pragma unroll
      for (int q = 0; q < NN; ++q) acc += s_Ry[j * NN + q] * s_t[q * NN + i];
      s_ph[tid] = first ? acc : s_ph[tid] + acc;
    }
    __syncthreads();
  };
  precond_add(true);
  const double scale = block_max<NT>(part ? fabs(phs) : 0.0, s_red);
  bool solved = false;
  double prev = INFINITY;
  for (int it = 0; it < SOLVE_CAP; ++it) {
    double r = 0.0;
    if (part) {                              // residual at the particle: phi* - sum Ly_m Lx_l phihat_ml
      double acc = 0.0;
#pragma unroll 1
      for (int mm = 0; mm < NN; ++mm) {
        double row = 0.0;
#pragma unroll
        for (int l = 0; l < NN; ++l) row += s_ph[mm * NN + l] * Lx[l];
        acc += Ly[mm] * row;
      }
      r = phs - acc;
      s_r[tid] = r;
    }
    const double rmax = block_max<NT>(fabs(r), s_red);
    // (data near the bottom of the double range carry no relative accuracy: a residual below
    // DBL_MIN / DBL_EPSILON, about 1e-292, is at the floor of the arithmetic)
    if (rmax <= SOLVE_RTOL * scale || rmax <= DBL_MIN / DBL_EPSILON) { solved = true; break; }
    // a residual that has stopped improving at the rounding floor counts as converged
    if (rmax > 0.5 * prev && rmax <= SOLVE_STALL * scale) { solved = true; break; }
    prev = rmax;
    precond_add(false);
  }
  if (!solved && tid == 0) atomicOr(status, SL_ST_SOLVE_NOCONV);
  if (part) W.phihat[E.base + tid] = s_ph[tid];

  // interface values at the face points, thread (face, q): traces of phihat (eq. 2dx/2dy_bnd_interpolate),
  // or phi^n at the backward characteristic foot of the face point from t^{n+1} (eq. 4.11)
  if (tid < 4 * NN) {
    const int f = tid / NN, q = tid % NN;
    double acc = 0.0;
    if (P.bvalue == SL_BV_BACKTRACK) {
      double fx = f == 0 ? x0 : f == 1 ? x0 + hx : x0 + hx * s_xi[q];
      double fy = f == 2 ? y0 : f == 3 ? y0 + hy : y0 + hy * s_xi[q];
      double gf = 1.0;
      rk2d<NN, NOD>(P, s_xi, s_lam, fx, fy, gf, P.t + P.dt, -P.dt);
      double bx[NN], by[NN];
      basis_at<NN>(s_xi, s_lam, (fx - x0) / hx, bx);
      basis_at<NN>(s_xi, s_lam, (fy - y0) / hy, by);
#pragma unroll 1
      for (int mm = 0; mm < NN; ++mm) {
        double row = 0.0;
#pragma unroll
        for (int l = 0; l < NN; ++l) row += s_phi[mm * NN + l] * bx[l];
        acc += by[mm] * row;
      }
      if (NOD) acc /= gf;
    } else {
      const double* L = (f == 1 || f == 3) ? s_l1 : s_l0;
#pragma unroll
      for (int k = 0; k < NN; ++k) acc += (f < 2 ? s_ph[q * NN + k] : s_ph[k * NN + q]) * L[k];
    }
    W.traces[E.g * M.tstride + tid] = acc;
  }
  // outflow fluxes: for each face point and RK stage where u.n_out > TIE, phi^n at the foot.
  // A face shared with a neighbour of another node count takes the rule of the finer side, so
  // that both elements integrate the same points (the flux telescopes).
  if (P.cons & (SL_C_MASS | SL_C_ENERGY)) {
    if (tid < 4) {
      bool wr;
      const int nb = nb_index(P, ex, ey, tid, wr);
      s_nq[tid] = nb < 0 ? NN : max(NN, order_of<NN>(M, E.gb + nb));
    }
    __syncthreads();
    for (int idx = tid; idx < 4 * NMAX; idx += NT) {
      const int f = idx / NMAX, q = idx % NMAX;
      const int nq = s_nq[f];
      if (q >= nq) continue;
      const double* rule = tb.rules + (size_t)nq * 3 * NMAX;
      double fm = 0.0, fe = 0.0;
      const double xf = f == 0 ? x0 : f == 1 ? x0 + hx : x0 + hx * rule[q];
      const double yf = f == 2 ? y0 : f == 3 ? y0 + hy : y0 + hy * rule[q];
      const double nx = f == 0 ? -1.0 : f == 1 ? 1.0 : 0.0, ny = f == 2 ? -1.0 : f == 3 ? 1.0 : 0.0;
      const double Wq = (f < 2 ? hy : hx) * rule[2 * NMAX + q];
      const int S = c_rk_s[P.rk];
      for (int s = 0; s < S; ++s) {
        const double cs = c_rk_c[P.rk][s];
        const double tau = P.t + cs * P.dt;
        double u, v, dvf;
        vel2dd<NN, NOD>(P, s_xi, s_lam, xf, yf, tau, u, v, dvf);
        const double un = u * nx + v * ny;
        if (un > TIE) {
          double fx = xf, fy = yf, gf = 1.0;
          if (cs != 0.0) rk2d<NN, NOD>(P, s_xi, s_lam, fx, fy, gf, tau, -cs * P.dt);
          double bx[NN], by[NN];
          basis_at<NN>(s_xi, s_lam, (fx - x0) / hx, bx);
          basis_at<NN>(s_xi, s_lam, (fy - y0) / hy, by);
          double val = 0.0;
#pragma unroll 1
          for (int mm = 0; mm < NN; ++mm) {
            double row = 0.0;
#pragma unroll
            for (int l = 0; l < NN; ++l) row += s_phi[mm * NN + l] * bx[l];
            val += by[mm] * row;
          }
          if (NOD) val /= gf;
          const double bw = c_rk_b[P.rk][s] * Wq * un;
          fm += bw * val;
          fe += bw * val * val;
        }
      }
      s_face[f][q][0] = fm;
      s_face[f][q][1] = fe;
    }
    __syncthreads();
    if (tid < 8) {                           // per face, sum over the points in index order
      const int f = tid >> 1, k = tid & 1;
      double acc = 0.0;
      for (int q = 0; q < s_nq[f]; ++q) acc += s_face[f][q][k];
      W.fluxes[E.g * 8 + tid] = acc;
    }
  }
}

template <int NN, bool NOD>
__global__ void __launch_bounds__(Shape<NN>::NT) k_p2(StepParams P0, Tables1D tb, Map2D M,
                                                     const double* __restrict__ in, Work2D W, double* __restrict__ out,
                                                     unsigned* status) {
  constexpr int ND = Shape<NN>::ND, NT = Shape<NN>::NT;
  constexpr int MMAX = 4 * NN + 1;
  __shared__ double s_xi[NN], s_lam[NN], s_w[NN], s_l0[NN], s_l1[NN];
  __shared__ double s_ph[ND], s_a[ND];
  __shared__ double s_r[MMAX], s_d[MMAX], s_ca[MMAX];
  __shared__ double s_red[NT / 32];
  const int tid = threadIdx.x;
  StepParams P = P0;
  const Elem E = elem_of<NN>(P, M);
  const int ex = E.ex, ey = E.ey;
  const double hx = P.hx, hy = P.hy;
  const double x0 = P.x0 + ex * hx, y0 = P.y0 + ey * hy;
  const double tn1 = P.t + P.dt;
  if (tid < NN) {
    s_xi[tid] = tb.xi[tid]; s_lam[tid] = tb.lam[tid]; s_w[tid] = tb.w[tid];
    s_l0[tid] = tb.l0[tid]; s_l1[tid] = tb.l1[tid];
  }
  const bool part = tid < ND;
  const int i = tid % NN, j = tid / NN;
  double phn = 0.0, ph = 0.0;
  if (part) {
    phn = in[E.base + tid];
    ph = W.phihat[E.base + tid];
    s_ph[tid] = ph;
  }
  __syncthreads();
  const double w2 = part ? s_w[i] * s_w[j] : 0.0;
  const bool bnd = (P.cons & SL_C_BOUNDARY) != 0;
  const int nb_rows = bnd ? 4 * NN : 0;
  // upwinded interface values (rows W, E, S, N at the tangential nodes); residual d - C phihat
  if (bnd && tid < 4 * NN) {
    const int f = tid / NN, q = tid % NN;
    bool wr;
    const int nb = nb_index(P, ex, ey, f, wr);
    const int fo = f ^ 1;                    // opposite face of the neighbour
    const double own = W.traces[E.g * M.tstride + tid];
    double other = P.ghost;
    if (nb >= 0) {                           // the neighbour's trace at this element's face points
      const int nn = order_of<NN>(M, E.gb + nb);
      const double* tr = W.traces + (E.gb + nb) * M.tstride + fo * nn;
      other = nn == NN ? tr[q] : interp_rule(tb.rules, nn, tr, s_xi[q]);
    }
    const double xf = f == 0 ? x0 : f == 1 ? x0 + hx : x0 + hx * s_xi[q];
    const double yf = f == 2 ? y0 : f == 3 ? y0 + hy : y0 + hy * s_xi[q];
    double u, v, dvf;
    vel2dd<NN, NOD>(P, s_xi, s_lam, xf, yf, tn1, u, v, dvf);
    const double un = f == 0 ? -u : f == 1 ? u : f == 2 ? -v : v;
    double val;
    if (un > TIE) val = own;
    else if (un < -TIE) val = other;
    else val = nb < 0 ? own : 0.5 * (own + other);
    // the row's value at phihat: the own trace when the interface values are traces of phihat,
    // else the trace formed here
    double trh = own;
    if (P.bvalue == SL_BV_BACKTRACK) {
      const double* L = (f == 1 || f == 3) ? s_l1 : s_l0;
      trh = 0.0;
#pragma unroll
      for (int k = 0; k < NN; ++k) trh += (f < 2 ? s_ph[q * NN + k] : s_ph[k * NN + q]) * L[k];
    }
    s_d[tid] = val;
    s_r[tid] = val - trh;
  }
  // mass and energy targets (reference measure)
  double Et = 0.0;
  const bool mass = (P.cons & SL_C_MASS) != 0, energy = (P.cons & SL_C_ENERGY) != 0;
  if (mass || energy) {
    double netm = 0.0, nete = 0.0;
    if (tid == 0) {
      for (int f = 0; f < 4; ++f) {
        bool wr;
        const int nb = nb_index(P, ex, ey, f, wr);
        netm += W.fluxes[E.g * 8 + 2 * f];
        nete += W.fluxes[E.g * 8 + 2 * f + 1];
        if (nb >= 0) {
          netm -= W.fluxes[(E.gb + nb) * 8 + 2 * (f ^ 1)];
          nete -= W.fluxes[(E.gb + nb) * 8 + 2 * (f ^ 1) + 1];
        } else {                              // inflow from the ghost value at a domain face
          for (int q = 0; q < NN; ++q) {
            const double xf = f == 0 ? x0 : f == 1 ? x0 + hx : x0 + hx * s_xi[q];
            const double yf = f == 2 ? y0 : f == 3 ? y0 + hy : y0 + hy * s_xi[q];
            const double Wq = (f < 2 ? hy : hx) * s_w[q];
            for (int s = 0; s < c_rk_s[P.rk]; ++s) {
              double u, v, dvf;
              vel2dd<NN, NOD>(P, s_xi, s_lam, xf, yf, P.t + c_rk_c[P.rk][s] * P.dt, u, v, dvf);
              const double un = f == 0 ? -u : f == 1 ? u : f == 2 ? -v : v;
              if (un < -TIE) {
                netm += c_rk_b[P.rk][s] * Wq * un * P.ghost;
                nete += c_rk_b[P.rk][s] * Wq * un * P.ghost * P.ghost;
              }
            }
          }
        }
      }
      s_a[0] = netm;
      s_a[1] = nete;
    }
    __syncthreads();
    netm = s_a[0];
    nete = s_a[1];
    __syncthreads();
    const double area = hx * hy;
    const double Mn = block_sum<NT>(w2 * phn, s_red);
    const double En = block_sum<NT>(w2 * phn * phn, s_red);
    if (mass) {
      const double Mh = block_sum<NT>(w2 * ph, s_red);
      if (tid == 0) {
        s_d[nb_rows] = Mn - P.dt / area * netm;
        s_r[nb_rows] = s_d[nb_rows] - Mh;
      }
    }
    Et = En - P.dt / area * nete;
  }
  __syncthreads();
  const int m = P.m;
  // linear constrained fit
  double phL = ph;
  if (part) {
    if (P.fit == SL_FIT_HARD) {
      double acc = ph;
      for (int k = 0; k < m; ++k) acc += tb.Cpinv[(size_t)tid * m + k] * s_r[k];
      phL = acc;
    } else {
      double acc = 0.0;
      for (int k = 0; k < ND; ++k) acc += tb.S[(size_t)tid * ND + k] * s_ph[k];
      for (int k = 0; k < m; ++k) acc += tb.SCt[(size_t)tid * m + k] * s_d[k];
      phL = acc;
    }
  }
  double cur = phL;
  bool ok = true;
  if (energy) {
    const double EL = block_sum<NT>(w2 * phL * phL, s_red);
    const double gamma = EL - Et;
    const double pmax = block_max<NT>(part ? fabs(ph) : 0.0, s_red);
    const bool apply = fabs(gamma) > ENERGY_SKIP_RTOL * fmax(fabs(Et), EL);
    if (apply) {
      const double tol = P.picard_rtol * fmax(pmax, 1e-300);
      bool conv = false, feasible = true;
      for (int it = 0; it < P.picard_cap; ++it) {
        const double a = w2 * cur;
        if (part) s_a[tid] = a;
        __syncthreads();
        double q = 0.0;
        if (P.fit == SL_FIT_HARD) {
          // C a: boundary rows (traces of a), then the mass row
          if (bnd && tid < 4 * NN) {
            const int f = tid / NN, qq = tid % NN;
            const double* L = (f == 1 || f == 3) ? s_l1 : s_l0;
            double acc = 0.0;
            for (int k = 0; k < NN; ++k) acc += (f < 2 ? s_a[qq * NN + k] : s_a[k * NN + qq]) * L[k];
            s_ca[tid] = acc;
          }
          if (mass) {
            const double cm = block_sum<NT>(w2 * a, s_red);
            if (tid == 0) s_ca[nb_rows] = cm;
          }
          __syncthreads();
          if (part) {
            double acc = a;
            for (int k = 0; k < m; ++k) acc -= tb.Cpinv[(size_t)tid * m + k] * s_ca[k];
            q = acc;
          }
          const double alpha = block_sum<NT>(w2 * phL * q, s_red);
          const double beta = block_sum<NT>(w2 * q * q, s_red);
          double s;
          if (beta <= 0.0) { s = 0.0; feasible = gamma <= 0.0; }
          else {
            const double disc = alpha * alpha - beta * gamma;
            if (disc < 0.0) { s = -alpha / beta; feasible = false; }
            else {
              const double root = sqrt(disc);
              const double den = alpha + (alpha >= 0.0 ? root : -root);
              s = den == 0.0 ? 0.0 : -gamma / den;
              feasible = true;
            }
          }
          const double nv = part ? phL + s * q : 0.0;
          const double delta = block_max<NT>(part ? fabs(nv - cur) : 0.0, s_red);
          cur = nv;
          if (delta < tol) { conv = feasible; break; }
        } else {
          if (part) {
            double acc = 0.0;
            for (int k = 0; k < ND; ++k) acc += tb.S[(size_t)tid * ND + k] * s_a[k];
            q = acc;
          }
          const double aphi = block_sum<NT>(a * phL, s_red);
          const double aq = block_sum<NT>(a * q, s_red);
          const double s = (Et - aphi) / (1.0 + aq);
          const double nv = part ? phL + s * q : 0.0;
          const double delta = block_max<NT>(part ? fabs(nv - cur) : 0.0, s_red);
          cur = nv;
          if (delta < tol) { conv = true; break; }
        }
        __syncthreads();
      }
      ok = conv;
      if (!conv) cur = phL;                   // keep the linear-constraint solution
    }
  }
  if (part) {
    out[E.base + tid] = cur;
    if (!isfinite(cur)) atomicOr(status, SL_ST_NONFINITE);
  }
  if (!ok && tid == 0) atomicOr(status, SL_ST_PICARD_NOCONV);
}

template <int NN>
void launch_n(int phase, const StepParams& p, const Tables1D& tb, const Map2D& m, int64_t count, const double* in,
              double* out, const Work2D& w, unsigned* st, cudaStream_t s) {
  if (count <= 0) return;
  const bool nod = p.vel_kind == SL_VEL_NODAL;
  if (phase == 1) {
    if (nod) k_p1<NN, true><<<(unsigned)count, Shape<NN>::NT, 0, s>>>(p, tb, m, in, w, st);
    else k_p1<NN, false><<<(unsigned)count, Shape<NN>::NT, 0, s>>>(p, tb, m, in, w, st);
  } else {
    if (nod) k_p2<NN, true><<<(unsigned)count, Shape<NN>::NT, 0, s>>>(p, tb, m, in, w, out, st);
    else k_p2<NN, false><<<(unsigned)count, Shape<NN>::NT, 0, s>>>(p, tb, m, in, w, out, st);
  }
}

}  // namespace k2d
}  // namespace sl
