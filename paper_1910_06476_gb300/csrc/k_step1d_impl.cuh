#pragma once
// 1D DSEM-SL step in double precision, one thread per element (Sec. 4, steps a-d).
//
// A CTA of BLOCK threads owns BLOCK-2 consecutive elements plus one halo element on each
// side.  Phase 1 (every thread, halo included): seed particles at the Gauss nodes, integrate
// them with explicit RK (eq. 4.4a, 4.8), remap by interpolation through the advected nodes
// (eq. 4.9), take the two face traces (eq. remap_bnd, or eq. 4.11 when backtracking), and
// integrate the outflow mass/energy flux through each face over the step.  These six numbers
// go to shared memory.  Phase 2 (core threads): upwind the interface values (eq. 4.12a),
// form the mass/energy targets (eq. remap_mass, remap_energy), apply the constrained fit
// (eq. matrix_a) and the energy iteration, and store phi^{n+1}.  Nothing but the state is
// read from or written to global memory; halo elements are recomputed (2/BLOCK overhead).
#include <cfloat>

#include "sl_internal.h"

namespace sl {
namespace k1d {

constexpr int BLOCK = 128;

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

// value at reference point z of the polynomial with nodal values v on nodes xn (barycentric
// weights lam): sum_j lam_j prod_{m != j} (z - xn_m) v_j, by prefix/suffix products
template <int NN>
__device__ __forceinline__ double eval_poly(const double* xn, const double* lam, const double* v, double z) {
  double d[NN], pre[NN];
#pragma unroll
  for (int m = 0; m < NN; ++m) d[m] = z - xn[m];
  double acc = 1.0;
#pragma unroll
  for (int m = 0; m < NN; ++m) { pre[m] = acc; acc *= d[m]; }
  double suf = 1.0, out = 0.0;
#pragma unroll
  for (int j = NN - 1; j >= 0; --j) {
    out += lam[j] * pre[j] * suf * v[j];
    suf *= d[j];
  }
  return out;
}

// the same polynomial and its derivative in z: the prefix and suffix products carry their
// derivatives along (product rule), so nodes need no special case
template <int NN>
__device__ __forceinline__ void eval_poly_d(const double* xn, const double* lam, const double* v, double z,
                                            double& val, double& der) {
  double d[NN], pre[NN], dpre[NN];
#pragma unroll
  for (int m = 0; m < NN; ++m) d[m] = z - xn[m];
  double acc = 1.0, dacc = 0.0;
#pragma unroll
  for (int m = 0; m < NN; ++m) {
    pre[m] = acc;
    dpre[m] = dacc;
    dacc = dacc * d[m] + acc;
    acc *= d[m];
  }
  double suf = 1.0, dsuf = 0.0, out = 0.0, dout = 0.0;
#pragma unroll
  for (int j = NN - 1; j >= 0; --j) {
    const double c = lam[j] * v[j];
    out += c * pre[j] * suf;
    dout += c * (dpre[j] * suf + pre[j] * dsuf);
    dsuf = dsuf * d[j] + suf;
    suf *= d[j];
  }
  val = out;
  der = dout;
}

// SL_VEL_NODAL in 1D: the node velocities of element k at time t (linear between the step's
// two arrays), evaluated with their derivative at reference point z
template <int NN>
__device__ __forceinline__ void nodal_elem1d(const StepParams& P, const double* xi, const double* lam, int k,
                                             double z, double th, double& u, double& du) {
  const double* U0 = P.nodal + (size_t)k * NN;
  const double* U1 = U0 + P.nvals;
  double v[NN];
#pragma unroll
  for (int j = 0; j < NN; ++j) v[j] = (1.0 - th) * U0[j] + th * U1[j];
  eval_poly_d<NN>(xi, lam, v, z, u, du);
}

// the nodal field at physical x: the containing element's interpolant (the boundary element's
// beyond a non-periodic face, wrapped across a periodic one); on a face the average over the
// elements that share it
template <int NN>
__device__ void nodal1d(const StepParams& P, const double* xi, const double* lam, double x, double t, double& u,
                        double& dv) {
  const double h = P.hx, x1 = P.x0 + P.K * h;
  const double th = (t - P.t) / P.dt;
  const double s = (x - P.x0) / h;
  const double r = rint(s);
  const bool perW = P.bc[0] == SL_BC_PERIODIC, perE = P.bc[1] == SL_BC_PERIODIC;
  u = 0.0;
  dv = 0.0;
  if (fabs(x - (P.x0 + r * h)) <= FACE_RTOL * (fabs(P.x0) + fabs(x1))) {
    int ks[2];
    double zs[2];
    int cnt = 0;
    const long long ri = (long long)r;
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      long long k = side ? ri : ri - 1;
      if (k < 0 || k >= P.K) {
        if (!(k < 0 ? perW : perE)) continue;
        k %= P.K;
        if (k < 0) k += P.K;
      }
      ks[cnt] = (int)k;
      zs[cnt] = side ? 0.0 : 1.0;
      ++cnt;
    }
    for (int q = 0; q < cnt; ++q) {
      double uq, dq;
      nodal_elem1d<NN>(P, xi, lam, ks[q], zs[q], th, uq, dq);
      u += uq / cnt;
      dv += dq / h / cnt;
    }
    return;
  }
  const double fk = floor(s);
  long long k = (long long)fk;
  double z = s - fk;
  if (k < 0 || k >= P.K) {
    if (k < 0 ? perW : perE) {
      k %= P.K;
      if (k < 0) k += P.K;
    } else {
      k = k < 0 ? 0 : P.K - 1;
      z = s - (double)k;
    }
  }
  double du;
  nodal_elem1d<NN>(P, xi, lam, (int)k, z, th, u, du);
  dv = du / h;
}

// velocity u(x, t) and its divergence in 1D (Sec. 5.1: constant; Sec. 5.2: u = -sin x; Sec. 4.2:
// given at the nodes)
template <int NN>
__device__ __forceinline__ void vel1d(const StepParams& P, const double* xi, const double* lam, double x, double t,
                                      double& u, double& dv) {
  if (P.vel_kind == SL_VEL_SINX) {
    double s, c;
    sincos(x, &s, &c);
    u = -s;
    dv = -c;
  } else if (P.vel_kind == SL_VEL_NODAL) {
    nodal1d<NN>(P, xi, lam, x, t, u, dv);
  } else {
    u = P.vp[0];
    dv = 0.0;
  }
}

// one explicit RK step of dx/dt = u, dphi/dt = -phi div u, size h (h < 0 runs backward)
template <int NN>
__device__ __forceinline__ void rk_step(const StepParams& P, const double* xi, const double* lam, double& x,
                                        double& ph, double t, double h) {
  if (P.vel_kind == SL_VEL_CONST) {       // exact for any scheme: sum b = 1
    x += h * P.vp[0];
    return;
  }
  const int S = c_rk_s[P.rk];
  double kx[4], kp[4];
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    if (s < S) {
      double xs = x, ps = ph;
#pragma unroll
      for (int j = 0; j < s; ++j) {
        xs += h * c_rk_a[P.rk][s][j] * kx[j];
        ps += h * c_rk_a[P.rk][s][j] * kp[j];
      }
      double u, dv;
      vel1d<NN>(P, xi, lam, xs, t + c_rk_c[P.rk][s] * h, u, dv);
      kx[s] = u;
      kp[s] = -ps * dv;
    }
  }
  double sx = 0.0, sp = 0.0;
#pragma unroll
  for (int s = 0; s < 4; ++s)
    if (s < S) {
      sx += c_rk_b[P.rk][s] * kx[s];
      sp += c_rk_b[P.rk][s] * kp[s];
    }
  x += h * sx;
  ph += h * sp;
}

struct Smem1D {
  double xi[NMAX], w[NMAX], lam[NMAX], l0[NMAX], l1[NMAX];
  double Cp[NMAX * MMAX1D];
  double SCt[NMAX * MMAX1D];
  double S[NMAX * NMAX];
  double tr[2][BLOCK];       // face traces at t^{n+1}
  double fm[2][BLOCK];       // outflow mass flux per face
  double fe[2][BLOCK];       // outflow energy flux per face
};

__device__ __forceinline__ int wrap_elem(int e, int K, bool periodic) {
  if (e >= 0 && e < K) return e;
  if (!periodic) return -1;
  e %= K;
  return e < 0 ? e + K : e;
}

template <int NN>
__global__ void __launch_bounds__(BLOCK) k_step1d_f64(StepParams P, Tables1D tb, const double* __restrict__ in,
                                                     double* __restrict__ out, unsigned* status) {
  __shared__ Smem1D sm;
  const int tid = threadIdx.x;
  const int m = P.m;
  for (int i = tid; i < NN; i += BLOCK) {
    sm.xi[i] = tb.xi[i]; sm.w[i] = tb.w[i]; sm.lam[i] = tb.lam[i];
    sm.l0[i] = tb.l0[i]; sm.l1[i] = tb.l1[i];
  }
  if (P.fit == SL_FIT_HARD) {
    for (int i = tid; i < NN * m; i += BLOCK) sm.Cp[i] = tb.Cpinv[i];
  } else {
    for (int i = tid; i < NN * m; i += BLOCK) sm.SCt[i] = tb.SCt[i];
    for (int i = tid; i < NN * NN; i += BLOCK) sm.S[i] = tb.S[i];
  }
  __syncthreads();

  const int K = P.K;
  const bool perW = P.bc[0] == SL_BC_PERIODIC, perE = P.bc[1] == SL_BC_PERIODIC;
  const int ecore0 = blockIdx.x * (BLOCK - 2);
  const int eraw = ecore0 + tid - 1;
  const int e = wrap_elem(eraw, K, eraw < 0 ? perW : perE);
  const bool core = tid >= 1 && tid <= BLOCK - 2 && eraw < K;
  const double h = P.hx;
  const double tn1 = P.t + P.dt;

  // ---------------- phase 1 --------------------------------------------------------------
  double phi[NN], ph[NN];
  if (e >= 0) {
    const double xk = P.x0 + e * h;
#pragma unroll
    for (int i = 0; i < NN; ++i) phi[i] = in[(size_t)e * NN + i];
    // (a)-(b) seed at the Gauss nodes and advect
    double xs[NN], ps[NN];
#pragma unroll
    for (int i = 0; i < NN; ++i) {
      double x = xk + h * sm.xi[i], p = phi[i];
      rk_step<NN>(P, sm.xi, sm.lam, x, p, P.t, P.dt);
      xs[i] = (x - xk) / h;
      ps[i] = p;
    }
    // (c) remap: phihat_j = sum_i phi*_i h*_i(xi_j) with barycentric weights of the advected nodes
    double lams[NN];
#pragma unroll
    for (int i = 0; i < NN; ++i) {
      double prod = 1.0;
#pragma unroll
      for (int q = 0; q < NN; ++q)
        if (q != i) prod *= (xs[i] - xs[q]);
      lams[i] = 1.0 / prod;
    }
#pragma unroll
    for (int j = 0; j < NN; ++j) ph[j] = eval_poly<NN>(xs, lams, ps, sm.xi[j]);
    // face traces at t^{n+1}
    double T0, T1;
    if (P.bvalue == SL_BV_BACKTRACK) {
      double f0 = xk, f1 = xk + h, g0 = 1.0, g1 = 1.0;
      rk_step<NN>(P, sm.xi, sm.lam, f0, g0, tn1, -P.dt);
      rk_step<NN>(P, sm.xi, sm.lam, f1, g1, tn1, -P.dt);
      T0 = eval_poly<NN>(sm.xi, sm.lam, phi, (f0 - xk) / h) / g0;
      T1 = eval_poly<NN>(sm.xi, sm.lam, phi, (f1 - xk) / h) / g1;
    } else {
      T0 = 0.0; T1 = 0.0;
#pragma unroll
      for (int j = 0; j < NN; ++j) { T0 += sm.l0[j] * ph[j]; T1 += sm.l1[j] * ph[j]; }
    }
    // outflow fluxes over the step by the RK quadrature, face value from phi^n at the foot
    double fm0 = 0.0, fm1 = 0.0, fe0 = 0.0, fe1 = 0.0;
    if (P.cons & (SL_C_MASS | SL_C_ENERGY)) {
      const int S = c_rk_s[P.rk];
      for (int s = 0; s < S; ++s) {
        const double cs = c_rk_c[P.rk][s], bs = c_rk_b[P.rk][s];
        const double tau = P.t + cs * P.dt;
#pragma unroll
        for (int side = 0; side < 2; ++side) {
          const double xf = xk + (side ? h : 0.0);
          double u, dv;
          vel1d<NN>(P, sm.xi, sm.lam, xf, tau, u, dv);
          const double un = side ? u : -u;
          if (un > TIE) {
            double fx = xf, g = 1.0;
            if (cs != 0.0) rk_step<NN>(P, sm.xi, sm.lam, fx, g, tau, -cs * P.dt);
            const double val = eval_poly<NN>(sm.xi, sm.lam, phi, (fx - xk) / h) / g;
            if (side) { fm1 += bs * un * val; fe1 += bs * un * val * val; }
            else { fm0 += bs * un * val; fe0 += bs * un * val * val; }
          }
        }
      }
    }
    sm.tr[0][tid] = T0; sm.tr[1][tid] = T1;
    sm.fm[0][tid] = fm0; sm.fm[1][tid] = fm1;
    sm.fe[0][tid] = fe0; sm.fe[1][tid] = fe1;
  }
  __syncthreads();
  if (!core) return;

  // ---------------- phase 2 --------------------------------------------------------------
  const double xk = P.x0 + e * h;
  double d[MMAX1D];
  int r = 0;
  double netm = 0.0, nete = 0.0;        // net outward flux (mass, energy) through both faces
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    const double xf = xk + (side ? h : 0.0);
    const int nbraw = side ? eraw + 1 : eraw - 1;
    const bool onbnd = nbraw < 0 || nbraw >= K;
    const bool per = side ? perE : perW;
    const bool ghostface = onbnd && !per;
    const int nbt = side ? tid + 1 : tid - 1;     // neighbour's thread in this CTA
    if (P.cons & SL_C_BOUNDARY) {
      double u, dv;
      vel1d<NN>(P, sm.xi, sm.lam, xf, tn1, u, dv);
      (void)dv;
      const double un = side ? u : -u;
      const double own = sm.tr[side][tid];
      const double other = ghostface ? (P.gtab ? P.gtab[side * 5] : P.ghost) : sm.tr[1 - side][nbt];
      double val;
      if (un > TIE) val = own;
      else if (un < -TIE) val = other;
      else val = ghostface ? own : 0.5 * (own + other);
      d[side] = val;
    }
    if (P.cons & (SL_C_MASS | SL_C_ENERGY)) {
      netm += sm.fm[side][tid];
      nete += sm.fe[side][tid];
      if (!ghostface) {
        netm -= sm.fm[1 - side][nbt];
        nete -= sm.fe[1 - side][nbt];
      } else {
        const int S = c_rk_s[P.rk];
        for (int s = 0; s < S; ++s) {
          const double tau = P.t + c_rk_c[P.rk][s] * P.dt;
          double u, dv;
          vel1d<NN>(P, sm.xi, sm.lam, xf, tau, u, dv);
          const double un = side ? u : -u;
          if (un < -TIE) {
            const double g = P.gtab ? P.gtab[side * 5 + 1 + s] : P.ghost;
            netm += c_rk_b[P.rk][s] * un * g;
            nete += c_rk_b[P.rk][s] * un * g * g;
          }
        }
      }
    }
  }
  if (P.cons & SL_C_BOUNDARY) r = 2;
  if (P.cons & SL_C_MASS) {
    double Mn = 0.0;
#pragma unroll
    for (int i = 0; i < NN; ++i) Mn += sm.w[i] * phi[i];
    d[r++] = Mn - P.dt / h * netm;      // reference-measure target (eq. remap_mass)
  }
  // linear constrained fit
  double phL[NN];
  if (P.fit == SL_FIT_HARD) {
    double res[MMAX1D];
    int q = 0;
    if (P.cons & SL_C_BOUNDARY) {
      double c0 = 0.0, c1 = 0.0;
#pragma unroll
      for (int j = 0; j < NN; ++j) { c0 += sm.l0[j] * ph[j]; c1 += sm.l1[j] * ph[j]; }
      res[q] = d[q] - c0; ++q;
      res[q] = d[q] - c1; ++q;
    }
    if (P.cons & SL_C_MASS) {
      double cm = 0.0;
#pragma unroll
      for (int j = 0; j < NN; ++j) cm += sm.w[j] * ph[j];
      res[q] = d[q] - cm; ++q;
    }
#pragma unroll
    for (int j = 0; j < NN; ++j) {
      double acc = ph[j];
      for (int k = 0; k < m; ++k) acc += sm.Cp[j * m + k] * res[k];
      phL[j] = acc;
    }
  } else {
#pragma unroll
    for (int j = 0; j < NN; ++j) {
      double acc = 0.0;
#pragma unroll
      for (int k = 0; k < NN; ++k) acc += sm.S[j * NN + k] * ph[k];
      for (int k = 0; k < m; ++k) acc += sm.SCt[j * m + k] * d[k];
      phL[j] = acc;
    }
  }
  double res_phi[NN];
#pragma unroll
  for (int j = 0; j < NN; ++j) res_phi[j] = phL[j];

  bool ok = true;
  if (P.cons & SL_C_ENERGY) {
    double En = 0.0, pmax = 0.0;
#pragma unroll
    for (int i = 0; i < NN; ++i) { En += sm.w[i] * phi[i] * phi[i]; pmax = fmax(pmax, fabs(ph[i])); }
    const double Et = En - P.dt / h * nete;
    const double tol = P.picard_rtol * fmax(pmax, 1e-300);
    double EL = 0.0;
#pragma unroll
    for (int i = 0; i < NN; ++i) EL += sm.w[i] * phL[i] * phL[i];
    const double gamma = EL - Et;
    // energy row only when the linear fit misses its target beyond rounding level
    const bool apply = fabs(gamma) > ENERGY_SKIP_RTOL * fmax(fabs(Et), EL);
    bool conv = !apply, feasible = true;
    for (int it = 0; apply && it < P.picard_cap; ++it) {
      double a[NN], qv[NN];
#pragma unroll
      for (int i = 0; i < NN; ++i) a[i] = sm.w[i] * res_phi[i];
      if (P.fit == SL_FIT_HARD) {
        double ca[MMAX1D];
        int q = 0;
        if (P.cons & SL_C_BOUNDARY) {
          double c0 = 0.0, c1 = 0.0;
#pragma unroll
          for (int j = 0; j < NN; ++j) { c0 += sm.l0[j] * a[j]; c1 += sm.l1[j] * a[j]; }
          ca[q++] = c0; ca[q++] = c1;
        }
        if (P.cons & SL_C_MASS) {
          double cm = 0.0;
#pragma unroll
          for (int j = 0; j < NN; ++j) cm += sm.w[j] * a[j];
          ca[q++] = cm;
        }
#pragma unroll
        for (int j = 0; j < NN; ++j) {
          double acc = a[j];
          for (int k = 0; k < m; ++k) acc -= sm.Cp[j * m + k] * ca[k];
          qv[j] = acc;
        }
        double alpha = 0.0, beta = 0.0;
#pragma unroll
        for (int i = 0; i < NN; ++i) { alpha += sm.w[i] * phL[i] * qv[i]; beta += sm.w[i] * qv[i] * qv[i]; }
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
        double delta = 0.0;
#pragma unroll
        for (int i = 0; i < NN; ++i) {
          const double nv = phL[i] + s * qv[i];
          delta = fmax(delta, fabs(nv - res_phi[i]));
          res_phi[i] = nv;
        }
        if (delta < tol) { conv = feasible; break; }
      } else {
#pragma unroll
        for (int j = 0; j < NN; ++j) {
          double acc = 0.0;
#pragma unroll
          for (int k = 0; k < NN; ++k) acc += sm.S[j * NN + k] * a[k];
          qv[j] = acc;
        }
        double aphi = 0.0, aq = 0.0;
#pragma unroll
        for (int i = 0; i < NN; ++i) { aphi += a[i] * phL[i]; aq += a[i] * qv[i]; }
        const double s = (Et - aphi) / (1.0 + aq);
        double delta = 0.0;
#pragma unroll
        for (int i = 0; i < NN; ++i) {
          const double nv = phL[i] + s * qv[i];
          delta = fmax(delta, fabs(nv - res_phi[i]));
          res_phi[i] = nv;
        }
        if (delta < tol) { conv = true; break; }
      }
    }
    if (!conv) {                          // keep the linear-constraint solution
      ok = false;
#pragma unroll
      for (int i = 0; i < NN; ++i) res_phi[i] = phL[i];
    }
  }
  bool finite = true;
#pragma unroll
  for (int i = 0; i < NN; ++i) {
    out[(size_t)e * NN + i] = res_phi[i];
    finite = finite && isfinite(res_phi[i]);
  }
  unsigned bits = (finite ? 0u : SL_ST_NONFINITE) | (ok ? 0u : SL_ST_PICARD_NOCONV);
  if (bits) atomicOr(status, bits);
}

template <int NN>
void launch_n(const StepParams& p, const Tables1D& tb, const double* in, double* out, unsigned* st,
              cudaStream_t s) {
  const int grid = (p.K + BLOCK - 3) / (BLOCK - 2);
  k_step1d_f64<NN><<<grid, BLOCK, 0, s>>>(p, tb, in, out, st);
}

}  // namespace k1d
}  // namespace sl
