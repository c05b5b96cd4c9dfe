#pragma once
// 2D DSEM-SL step in mixed precision for any prescribed velocity: double-float state, float
// arithmetic on increments relative to a per-element reference value (Sec. 4, two-dimensional
// scheme).  Same two phases as the FP64 kernels (k_step2d_impl.cuh):
//   phase 1: advect the particles in element-local coordinates (float), solve the collocation
//            system of eq. 5.4 for the increments psi = phi - ref by preconditioned iterative
//            refinement, take the face traces, and integrate per face over the step
//              U_out, U_in : RK/Gauss quadrature of u.n_out split by its sign,
//              Psi, Psi2   : the same of u.n psi and u.n psi^2 at the feet of the outflow points;
//   phase 2: interface values, mass and energy targets, constrained fit, energy iteration.
// Without the energy row the element reference is linear, L = r0 + gx (xi - 1/2) + gy (eta - 1/2)
// (from the corner values; evaluated in double wherever a node value is formed), and psi = phi - L
// is what the float arithmetic carries: for resolved data it is smaller than phi - r0 by about the
// element width over the data's length scale, and so is every rounding error of the remap, the
// traces and the fit.  Particles keep phi (divergence-free velocity), so the collocation data for
// psihat = phihat - L is psi_p - grad L . d_p (d_p the particle's displacement).  With the energy
// row the reference is the constant r0 (gx = gy = 0).
// Everything a target needs is assembled from increments: the net mass flux of element e is
//   ref_e (U_out + U_in)  +  sum_f (ref_nb - ref_e) U_in,f  +  sum_f (Psi_out,f - Psi'_f),
// Psi'_f being the neighbour's outflow flux through the shared face, so float rounding scales
// with the variation of the data instead of |phi|.  The result is written back exactly as
// L + psi (a double sum split into hi + lo).
// The face quadrature of phase 1 is spread over the whole CTA: one work item per (face, point,
// distinct RK stage time), partial sums added in a fixed order (deterministic).
#include "k_map2d.cuh"

namespace sl {
namespace k2m {

static __constant__ int c_rk_s[5] = {0, 1, 2, 3, 4};
static __constant__ float c_rk_a[5][4][4] = {
    {},
    {{0}},
    {{0, 0}, {1.0f, 0}},
    {{0, 0, 0}, {0.5f, 0, 0}, {-1.0f, 2.0f, 0}},
    {{0, 0, 0, 0}, {0.5f, 0, 0, 0}, {0, 0.5f, 0, 0}, {0, 0, 1.0f, 0}}};
static __constant__ float c_rk_b[5][4] = {
    {}, {1.0f}, {0.5f, 0.5f}, {1.0f / 6, 2.0f / 3, 1.0f / 6}, {1.0f / 6, 1.0f / 3, 1.0f / 3, 1.0f / 6}};
static __constant__ float c_rk_c[5][4] = {{}, {0.0f}, {0.0f, 1.0f}, {0.0f, 0.5f, 1.0f}, {0.0f, 0.5f, 0.5f, 1.0f}};
// distinct stage times of the face-flux quadrature and their summed weights (RK4's two c = 1/2
// stages see the same face velocity and the same foot)
static __constant__ int c_ds_n[5] = {0, 1, 2, 3, 3};
static __constant__ float c_ds_c[5][3] = {{}, {0.0f}, {0.0f, 1.0f}, {0.0f, 0.5f, 1.0f}, {0.0f, 0.5f, 1.0f}};
static __constant__ float c_ds_b[5][3] = {
    {}, {1.0f}, {0.5f, 0.5f}, {1.0f / 6, 2.0f / 3, 1.0f / 6}, {1.0f / 6, 1.0f / 3 + 1.0f / 3, 1.0f / 6}};

// sum_l row[l] b[l] over a row of NN values stored 16-byte aligned: the row is read with 16-byte
// loads (a broadcast when every thread reads the same row), even and odd columns accumulate in
// the two lanes of paired FMAs
template <int NN>
__device__ __forceinline__ float row_dot(const float* row, const float (&b)[NN]) {
  const float4* rowp = reinterpret_cast<const float4*>(row);
  float2 r2 = make_float2(0.0f, 0.0f);
#pragma unroll
  for (int q = 0; q < NN / 4; ++q) {
    const float4 v = rowp[q];
    r2 = __ffma2_rn(make_float2(v.x, v.y), make_float2(b[4 * q], b[4 * q + 1]), r2);
    r2 = __ffma2_rn(make_float2(v.z, v.w), make_float2(b[4 * q + 2], b[4 * q + 3]), r2);
  }
  float r = r2.x + r2.y;
  if (NN % 4 != 0) {
    const float4 v = rowp[NN / 4];
    constexpr int l0 = NN & ~3;
    r = fmaf(v.x, b[l0], r);
    if (NN % 4 > 1) r = fmaf(v.y, b[(l0 + 1) % NN], r);
    if (NN % 4 > 2) r = fmaf(v.z, b[(l0 + 2) % NN], r);
  }
  return r;
}

constexpr int SOLVE_CAP = 40;
constexpr float SOLVE_RTOL = 3e-7f;          // target, relative to max |psi*|
constexpr float SOLVE_STALL = 4e-6f;         // a residual that stops improving below this is the float floor
constexpr float SOLVE_FLOOR = 1e-4f;         // best residual accepted when the iteration stalls or diverges

// velocity divided by the element size: the time derivative of the reference coordinates
__device__ __forceinline__ void vel_ref(const StepParams& P, const Mixed2DExtra& X, float x, float y, float tT,
                                        float& u, float& v) {
  switch (P.vel_kind) {
    case SL_VEL_ROTATION:
      u = -X.om * (y - X.cy) * X.ihx;
      v = X.om * (x - X.cx) * X.ihy;
      break;
    case SL_VEL_SWIRL: {
      const float c = cospif(tT);
      const float sx = sinpif(x), sy = sinpif(y);
      u = sx * sx * sinpif(2.0f * y) * c * X.ihx;
      v = -sy * sy * sinpif(2.0f * x) * c * X.ihy;
      break;
    }
    default:
      u = X.a * X.ihx;
      v = X.b * X.ihy;
  }
}

// One RK step of the displacement (dx, dy), in reference coordinates, of the point (bx, by) of
// the element with origin (x0, y0); tT = t / T (swirl), h = step in time, hT = h / T.  The
// displacement is integrated by itself (not the position), so that its float rounding is
// relative to the displacement and not to the coordinate.
__device__ __forceinline__ void rk_disp(const StepParams& P, const Mixed2DExtra& X, float x0, float y0, float bx,
                                        float by, float& dx, float& dy, float tT, float h, float hT) {
  const int S = c_rk_s[P.rk];
  float kx[4], ky[4];
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    if (s < S) {
      float xs = dx, ys = dy;
#pragma unroll
      for (int j = 0; j < s; ++j) {
        xs = fmaf(h * c_rk_a[P.rk][s][j], kx[j], xs);
        ys = fmaf(h * c_rk_a[P.rk][s][j], ky[j], ys);
      }
      vel_ref(P, X, fmaf(X.hx, bx + xs, x0), fmaf(X.hy, by + ys, y0), fmaf(c_rk_c[P.rk][s], hT, tT), kx[s], ky[s]);
    }
  }
  float sx = 0.0f, sy = 0.0f;
#pragma unroll
  for (int s = 0; s < 4; ++s)
    if (s < S) {
      sx = fmaf(c_rk_b[P.rk][s], kx[s], sx);
      sy = fmaf(c_rk_b[P.rk][s], ky[s], sy);
    }
  dx = fmaf(h, sx, dx);
  dy = fmaf(h, sy, dy);
}

// Lagrange basis at z = z0 + dz with the differences formed as (z0 - xi_k) + dz: when z0 is a
// node, its own difference is dz exactly
template <int NN>
__device__ __forceinline__ void basis_at(const float* xi, const float* lam, float z0, float dz, float* out) {
  float d[NN], pre[NN];
#pragma unroll
  for (int k = 0; k < NN; ++k) d[k] = (z0 - xi[k]) + dz;
  float acc = 1.0f;
#pragma unroll
  for (int k = 0; k < NN; ++k) { pre[k] = acc; acc *= d[k]; }
  float suf = 1.0f;
#pragma unroll
  for (int l = NN - 1; l >= 0; --l) {
    out[l] = lam[l] * pre[l] * suf;
    suf *= d[l];
  }
}

template <int NT>
__device__ __forceinline__ float block_sum(float v, float* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, ln = threadIdx.x & 31;
  __syncthreads();
  if (ln == 0) red[w] = v;
  __syncthreads();
  float s = 0.0f;
#pragma unroll
  for (int i = 0; i < NT / 32; ++i) s += red[i];
  return s;
}

// two block sums in one pass (each component summed exactly as block_sum would); red holds
// 2 NT / 32 floats
template <int NT>
__device__ __forceinline__ float2 block_sum2(float a, float b, float* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  const int w = threadIdx.x >> 5, ln = threadIdx.x & 31;
  __syncthreads();
  if (ln == 0) {
    red[w] = a;
    red[NT / 32 + w] = b;
  }
  __syncthreads();
  float sa = 0.0f, sb = 0.0f;
#pragma unroll
  for (int i = 0; i < NT / 32; ++i) {
    sa += red[i];
    sb += red[NT / 32 + i];
  }
  return make_float2(sa, sb);
}

template <int NT>
__device__ __forceinline__ float block_max(float v, float* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_down_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, ln = threadIdx.x & 31;
  __syncthreads();
  if (ln == 0) red[w] = v;
  __syncthreads();
  float s = 0.0f;
#pragma unroll
  for (int i = 0; i < NT / 32; ++i) s = fmaxf(s, red[i]);
  return s;
}

template <int NN>
struct Shape {
  static constexpr int ND = NN * NN;
  static constexpr int NT = ((ND > 4 * NN ? ND : 4 * NN) + 31) / 32 * 32;
  // resident CTAs asked of the compiler (one element per CTA keeps the SM latency-bound): register
  // caps of 64 per thread for n <= 9 (a few bytes of spill at most), about 100 for n <= 13, 128
  // above (a tighter cap spills there and runs slower)
  static constexpr int MINB = NN <= 9 ? 65536 / (64 * NT) : NN <= 13 ? 65536 / (96 * NT)
                                                           : (65536 / (128 * NT) > 1 ? 65536 / (128 * NT) : 1);
  // phase 2 (less register demand): 64 for n <= 9, about 96 above
  static constexpr int MINB2 = NN <= 9 ? 65536 / (64 * NT) : 65536 / (96 * NT);
};

// per-problem float parameters of a batch element (the FP64 geometry is already in P)
__device__ __forceinline__ void batch_extra(const StepParams& P, const Map2D& M, Mixed2DExtra& X) {
  if (!M.geo) return;
  X.hx = (float)P.hx;
  X.hy = (float)P.hy;
  X.ihx = (float)(1.0 / P.hx);
  X.ihy = (float)(1.0 / P.hy);
  X.dt = (float)P.dt;
  X.dt_area = (float)(P.dt / (P.hx * P.hy));
  if (X.Tper != 0.0) {
    X.tT = (float)(P.t / X.Tper);
    X.dtT = (float)(P.dt / X.Tper);
  }
}

__device__ __forceinline__ int nb_index(const StepParams& P, int ex, int ey, int face) {
  int jx = ex + (face == 0 ? -1 : face == 1 ? 1 : 0);
  int jy = ey + (face == 2 ? -1 : face == 3 ? 1 : 0);
  if (jx >= 0 && jx < P.kx && jy >= 0 && jy < P.ky) return jy * P.kx + jx;
  if (P.bc[face] != SL_BC_PERIODIC) return -1;
  jx = (jx + P.kx) % P.kx;
  jy = (jy + P.ky) % P.ky;
  return jy * P.kx + jx;
}

// element reference L = r0 + gx (xi - 1/2) + gy (eta - 1/2) in double
__device__ __forceinline__ double lref(float r0, float gx, float gy, double xi, double eta) {
  return (double)r0 + (double)gx * (xi - 0.5) + (double)gy * (eta - 0.5);
}

template <int NN>
__global__ void __launch_bounds__(Shape<NN>::NT, Shape<NN>::MINB) k_p1(StepParams P0, const __grid_constant__ Mixed2DExtra X0,
                                                     Map2D M, const float* __restrict__ in, Work2M W,
                                                     unsigned* status) {
  constexpr int ND = Shape<NN>::ND, NT = Shape<NN>::NT;
  __shared__ float s_xi[NN], s_lam[NN], s_w[NN], s_l0[NN], s_l1[NN];
  constexpr int NP = (NN + 3) & ~3;                // psihat rows padded to 16 bytes
  __shared__ float s_t[ND], s_r[ND], s_Rx[ND], s_Ry[ND];
  __shared__ __align__(16) float s_psi[NN * NP];   // psi^n rows, padded like psihat
  __shared__ __align__(16) float s_ph[NN * NP];
  __shared__ float s_red[NT / 32];
  __shared__ float s_fs[4][NMAX][3][4];          // face point x distinct stage partial sums
  __shared__ int s_nq[4];
  const int tid = threadIdx.x;
  StepParams P = P0;
  const Elem E = elem_of<NN>(P, M);
  Mixed2DExtra X = X0;
  batch_extra(P, M, X);
  const int ex = E.ex, ey = E.ey;
  const float x0 = (float)(P.x0 + ex * P.hx), y0 = (float)(P.y0 + ey * P.hy);
  if (tid < NN) {
    s_xi[tid] = X.xi[tid]; s_lam[tid] = X.lam[tid]; s_w[tid] = X.w[tid];
    s_l0[tid] = X.l0[tid]; s_l1[tid] = X.l1[tid];
  }
  const bool part = tid < ND;
  const int i = tid % NN, j = tid / NN;
  // element reference: linear from the four corner values, or the first node value
  const float c00 = in[E.base], c01 = in[E.base + NN - 1], c10 = in[E.base + (NN - 1) * NN], c11 = in[E.base + ND - 1];
  float ref = c00, gx = 0.0f, gy = 0.0f;
  if (X.linref) {
    const float span = (float)(0.5 / (X.xid[NN - 1] - X.xid[0]));
    ref = 0.25f * ((c00 + c01) + (c10 + c11));
    gx = ((c01 + c11) - (c00 + c10)) * span;
    gy = ((c10 + c11) - (c00 + c01)) * span;
  }
  if (part)
    s_psi[j * NP + i] = (float)(((double)in[E.base + tid] + (double)in[X.plane + E.base + tid]) -
                         lref(ref, gx, gy, X.xid[i], X.xid[j]));
  __syncthreads();

  // advect the particle of node (i, j) in reference coordinates
  float Lx[NN], Ly[NN], ps = 0.0f, pn = 0.0f, dxs = 0.0f, dys = 0.0f;
  if (part) {
    float ddx = 0.0f, ddy = 0.0f;
    rk_disp(P, X, x0, y0, s_xi[i], s_xi[j], ddx, ddy, X.tT, X.dt, X.dtT);
    basis_at<NN>(s_xi, s_lam, s_xi[i], ddx, Lx);
    basis_at<NN>(s_xi, s_lam, s_xi[j], ddy, Ly);
    pn = s_psi[j * NP + i];
    ps = pn - fmaf(gx, ddx, gy * ddy);       // collocation data of phihat - L
    dxs = ddx;
    dys = ddy;
  }
  const float mdx = block_sum<NT>(dxs, s_red) / ND;
  const float mdy = block_sum<NT>(dys, s_red) / ND;
  if (part) {
    float b[NN];
    basis_at<NN>(s_xi, s_lam, s_xi[j], -mdx, b);
    s_Rx[tid] = b[i];
    basis_at<NN>(s_xi, s_lam, s_xi[j], -mdy, b);
    s_Ry[tid] = b[i];
    s_r[tid] = ps;
  }
  __syncthreads();
  auto precond_add = [&](bool first) {
    if (part) {
      float acc = 0.0f;
#pragma unroll
      for (int q = 0; q < NN; ++q) acc = fmaf(s_Rx[i * NN + q], s_r[j * NN + q], acc);
      s_t[tid] = acc;
    }
    __syncthreads();
    if (part) {
      float acc = 0.0f;
#pragma unroll
      for (int q = 0; q < NN; ++q) acc = fmaf(s_Ry[j * NN + q], s_t[q * NN + i], acc);
      s_ph[j * NP + i] = first ? acc : s_ph[j * NP + i] + acc;
    }
    __syncthreads();
  };
  precond_add(true);
  const float scale = block_max<NT>(part ? fabsf(ps) : 0.0f, s_red);
  // Stop at the tolerance, or once the residual has stalled at the float floor; guard against
  // divergence by keeping the best iterate.
  bool solved = false;
  float prev = INFINITY, best = INFINITY;
  __shared__ float s_best[ND];
  for (int it = 0; it < SOLVE_CAP; ++it) {
    float r = 0.0f;
    if (part) {
      // row sums: every thread reads the same psihat row
      float acc = 0.0f;
#pragma unroll 1
      for (int mm = 0; mm < NN; ++mm) {
        const float row = row_dot<NN>(s_ph + mm * NP, Lx);
        acc = fmaf(Ly[mm], row, acc);
      }
      r = ps - acc;
      s_r[tid] = r;
    }
    const float rmax = block_max<NT>(fabsf(r), s_red);
    // values below the normal float range carry no accuracy to refine
    if (rmax <= SOLVE_RTOL * scale || rmax == 0.0f || scale < 1e-30f) { solved = true; break; }
    const bool stalled = rmax > 0.5f * prev && rmax <= SOLVE_STALL * scale;   // at the float floor
    const bool diverging = !(rmax <= 4.0f * best);                             // or not finite
    if (stalled || diverging) {
      if (!(rmax <= best)) {                  // back to the best iterate
        if (part) s_ph[j * NP + i] = s_best[tid];
        __syncthreads();
      }
      solved = fminf(rmax, best) <= SOLVE_FLOOR * scale;
      break;
    }
    if (rmax < best) {
      best = rmax;
      if (part) s_best[tid] = s_ph[j * NP + i];
    }
    prev = rmax;
    precond_add(false);
  }
  if (!solved && tid == 0) atomicOr(status, SL_ST_SOLVE_NOCONV);
  if (part) W.psihat[E.base + tid] = s_ph[j * NP + i];
  // element sums of psi^n (reference measure)
  const float w2 = part ? s_w[i] * s_w[j] : 0.0f;
  const float m1 = block_sum<NT>(w2 * pn, s_red);
  const float m2 = block_sum<NT>(w2 * pn * pn, s_red);
  if (tid == 0) {
    W.elem[E.g * 8 + 0] = ref;
    W.elem[E.g * 8 + 1] = gx;
    W.elem[E.g * 8 + 2] = gy;
    W.elem[E.g * 8 + 3] = m1;
    W.elem[E.g * 8 + 4] = m2;
  }
  // traces of psihat (relative to ref)
  if (tid < 4 * NN) {
    const int f = tid / NN, q = tid % NN;
    const float* L = (f == 1 || f == 3) ? s_l1 : s_l0;
    float acc = 0.0f;
#pragma unroll
    for (int k = 0; k < NN; ++k) acc = fmaf(f < 2 ? s_ph[q * NP + k] : s_ph[k * NP + q], L[k], acc);
    W.traces[E.g * M.tstride + tid] = acc;
  }
  // face sums over the step; a face shared with a neighbour of another node count takes the rule
  // of the finer side, so that both elements integrate the same points
  if (P.cons & (SL_C_MASS | SL_C_ENERGY)) {
    if (tid < 4) {
      const int nb = nb_index(P, ex, ey, tid);
      s_nq[tid] = nb < 0 ? NN : max(NN, order_of<NN>(M, E.gb + nb));
    }
    __syncthreads();
    // one work item per (face, point, distinct stage time), partial sums kept per item and added
    // in a fixed order below
    const int S = c_ds_n[P.rk];
    for (int idx = tid; idx < 4 * NMAX * 3; idx += NT) {
      const int f = idx / (NMAX * 3), q = (idx / 3) % NMAX, s = idx % 3;
      const int nq = s_nq[f];
      if (q >= nq || s >= S) continue;
      const float* rule = X.rules + (size_t)nq * 3 * NMAX;
      const float xr = f == 0 ? 0.0f : f == 1 ? 1.0f : rule[q];
      const float yr = f == 2 ? 0.0f : f == 3 ? 1.0f : rule[q];
      const float hn = f < 2 ? X.hx : X.hy;          // velocity in reference units times this = u.n
      const float sg = (f == 0 || f == 2) ? -1.0f : 1.0f;
      const float Wq = (f < 2 ? X.hy : X.hx) * rule[2 * NMAX + q];
      float uo = 0.0f, ui = 0.0f, p1 = 0.0f, p2 = 0.0f;
      const float cs = c_ds_c[P.rk][s];
      float ur, vr;
      vel_ref(P, X, fmaf(X.hx, xr, x0), fmaf(X.hy, yr, y0), fmaf(cs, X.dtT, X.tT), ur, vr);
      const float un = sg * (f < 2 ? ur : vr) * hn;
      const float bw = c_ds_b[P.rk][s] * Wq * un;
      if (un > (float)TIE) {
        uo = bw;
        float fdx = 0.0f, fdy = 0.0f;
        if (cs != 0.0f) rk_disp(P, X, x0, y0, xr, yr, fdx, fdy, fmaf(cs, X.dtT, X.tT), -cs * X.dt, -cs * X.dtT);
        float bx[NN], by[NN];
        basis_at<NN>(s_xi, s_lam, xr, fdx, bx);
        basis_at<NN>(s_xi, s_lam, yr, fdy, by);
        float val = 0.0f;
#pragma unroll 1
        for (int mm = 0; mm < NN; ++mm) val = fmaf(by[mm], row_dot<NN>(s_psi + mm * NP, bx), val);
        val += fmaf(gx, (xr - 0.5f) + fdx, gy * ((yr - 0.5f) + fdy));   // phi - r0 = (L - r0) + psi
        p1 = bw * val;
        p2 = p1 * val;
      } else if (un < -(float)TIE) {
        ui = bw;
      }
      s_fs[f][q][s][0] = uo; s_fs[f][q][s][1] = ui; s_fs[f][q][s][2] = p1; s_fs[f][q][s][3] = p2;
    }
    __syncthreads();
    if (tid < 16) {
      const int f = tid >> 2, k = tid & 3;
      float acc = 0.0f;
      for (int q = 0; q < s_nq[f]; ++q)
        for (int s = 0; s < S; ++s) acc += s_fs[f][q][s][k];
      W.faces[E.g * 16 + tid] = acc;
    }
  }
}

template <int NN>
__global__ void __launch_bounds__(Shape<NN>::NT, Shape<NN>::MINB2) k_p2(StepParams P0, const __grid_constant__ Mixed2DExtra X0,
                                                     Map2D M, const float* __restrict__ in, Work2M W,
                                                     float* __restrict__ out, unsigned* status) {
  constexpr int ND = Shape<NN>::ND, NT = Shape<NN>::NT;
  constexpr int MMAX = 4 * NN + 1;
  __shared__ float s_xi[NN], s_w[NN], s_l0[NN], s_l1[NN];
  __shared__ float s_ph[ND], s_a[ND];
  __shared__ float s_r[MMAX], s_ca[MMAX];
  __shared__ float s_red[NT / 32];
  __shared__ float s_red2[2 * (NT / 32)];
  __shared__ float s_scal[4];
  const int tid = threadIdx.x;
  StepParams P = P0;
  const Elem E = elem_of<NN>(P, M);
  Mixed2DExtra X = X0;
  batch_extra(P, M, X);
  const int ex = E.ex, ey = E.ey;
  const float x0 = (float)(P.x0 + ex * P.hx), y0 = (float)(P.y0 + ey * P.hy);
  const float tn1T = X.tT + X.dtT;
  if (tid < NN) { s_xi[tid] = X.xi[tid]; s_w[tid] = X.w[tid]; s_l0[tid] = X.l0[tid]; s_l1[tid] = X.l1[tid]; }
  const bool part = tid < ND;
  const int i = tid % NN, j = tid / NN;
  const float ref = W.elem[E.g * 8], gx = W.elem[E.g * 8 + 1], gy = W.elem[E.g * 8 + 2];
  float ph = 0.0f;
  if (part) {
    ph = W.psihat[E.base + tid];
    s_ph[tid] = ph;
  }
  __syncthreads();
  const float w2 = part ? s_w[i] * s_w[j] : 0.0f;
  const bool bnd = (P.cons & SL_C_BOUNDARY) != 0;
  const int nb_rows = bnd ? 4 * NN : 0;
  if (bnd && tid < 4 * NN) {
    const int f = tid / NN, q = tid % NN;
    const int nb = nb_index(P, ex, ey, f);
    const float own = W.traces[E.g * M.tstride + tid];
    // neighbour's value at this element's face points, relative to this element's reference L:
    // (L_nb - L) in double (it is of the size of psi when both references fit the same data), plus
    // the neighbour's trace of its own psihat
    const double xq = X.xid[q];
    const double fx = f == 0 ? 0.0 : f == 1 ? 1.0 : xq, fy = f == 2 ? 0.0 : f == 3 ? 1.0 : xq;
    const double lown = lref(ref, gx, gy, fx, fy);
    float other = (float)(P.ghost - lown);
    if (nb >= 0) {
      const int64_t gn = E.gb + nb;
      const int nn = order_of<NN>(M, gn);
      const float* tr = W.traces + gn * M.tstride + (f ^ 1) * nn;
      const float* en = W.elem + gn * 8;
      const double lnb = lref(en[0], en[1], en[2], f == 0 ? 1.0 : f == 1 ? 0.0 : fx, f == 2 ? 1.0 : f == 3 ? 0.0 : fy);
      other = (float)(lnb - lown) + (nn == NN ? tr[q] : interp_rule(X.rules, nn, tr, s_xi[q]));
    }
    const float xr = f == 0 ? 0.0f : f == 1 ? 1.0f : s_xi[q];
    const float yr = f == 2 ? 0.0f : f == 3 ? 1.0f : s_xi[q];
    float ur, vr;
    vel_ref(P, X, fmaf(X.hx, xr, x0), fmaf(X.hy, yr, y0), tn1T, ur, vr);
    const float un = (f == 0 || f == 2 ? -1.0f : 1.0f) * (f < 2 ? ur * X.hx : vr * X.hy);
    float val;
    if (un > (float)TIE) val = own;
    else if (un < -(float)TIE) val = other;
    else val = nb < 0 ? own : 0.5f * (own + other);
    s_r[tid] = val - own;
  }
  const bool mass = (P.cons & SL_C_MASS) != 0, energy = (P.cons & SL_C_ENERGY) != 0;
  float netm = 0.0f, netd2 = 0.0f, nu = 0.0f;
  if ((mass || energy) && tid < 32) {
    // net outflow of mass (increments) and of the squared increments, plus the velocity balance:
    // lanes 0-3 of the first warp take one face each, summed in face order
    float cu = 0.0f, cm = 0.0f, cd = 0.0f;
    if (tid < 4) {
      const int f = tid;
      const float* F = W.faces + E.g * 16 + 4 * f;
      const int nb = nb_index(P, ex, ey, f);
      cu = F[0] + F[1];
      if (nb >= 0) {
        const float* G = W.faces + (E.gb + nb) * 16 + 4 * (f ^ 1);
        const float dref = W.elem[(E.gb + nb) * 8] - ref;
        // inflow part: u.n (dref + psi_nb) with the neighbour's u.n = -ours
        cm = F[2] + (dref * F[1] - G[2]);
        cd = F[3] + (dref * dref * F[1] - 2.0f * dref * G[2] - G[3]);
      } else {
        const float g = (float)(P.ghost - (double)ref);
        cm = F[2] + g * F[1];
        cd = F[3] + g * g * F[1];
      }
    }
    float su = 0.0f, sm = 0.0f, sd = 0.0f;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      su += __shfl_sync(0xffffffffu, cu, f);
      sm += __shfl_sync(0xffffffffu, cm, f);
      sd += __shfl_sync(0xffffffffu, cd, f);
    }
    if (tid == 0) {
      s_scal[0] = sm;
      s_scal[1] = sd;
      s_scal[2] = su;
    }
  }
  __syncthreads();
  netm = s_scal[0];
  netd2 = s_scal[1];
  nu = s_scal[2];
  const float lam = X.dt_area;               // dt / (hx hy)
  if (mass) {
    const float mh = block_sum<NT>(w2 * ph, s_red);
    // target (increments): sum w psi^n - lam (net increment outflow + ref * closed-surface u.n)
    // ref * (closed-surface integral of u.n) is dropped: every 2D velocity here is divergence free
    // and the face quadrature integrates it to rounding; in float it would be noise of eps |U|
    if (tid == 0) s_r[nb_rows] = (W.elem[E.g * 8 + 3] - lam * netm) - mh;
  }
  __syncthreads();
  const int m = P.m;
  float phL = ph;
  if (part) {
    float acc = ph;
    for (int k = 0; k < m; ++k) acc = fmaf(X.Cp[(size_t)k * ND + tid], s_r[k], acc);
    phL = acc;
  }
  float cur = phL;
  bool ok = true;
  if (energy) {
    // energy mismatch from increments (mass enforced): sum w (psiL - psi)(psiL + psi) + lam net(delta^2);
    // without the mass row, add 2 ref times the mass residual (closed-surface u.n taken as zero)
    const float psin = part ? (float)(((double)in[E.base + tid] + (double)in[X.plane + E.base + tid]) -
                                      lref(ref, gx, gy, X.xid[i], X.xid[j]))
                            : 0.0f;
    const float dpsi = part ? phL - psin : 0.0f;
    const float2 evml = block_sum2<NT>(w2 * dpsi * (phL + (phL - dpsi)), w2 * phL, s_red2);
    const float ev = evml.x, ml = evml.y;
    const float m1 = W.elem[E.g * 8 + 3];
    float gamma;
    if (mass) gamma = ev + lam * netd2;
    else gamma = fmaf(2.0f * ref, (ml - m1) + lam * netm, ev + lam * netd2);
    const float escale = block_sum<NT>(part ? w2 * (ref + cur) * (ref + cur) : 0.0f, s_red);
    float smax = block_max<NT>(part ? fmaxf(fabsf(phL), fabsf(ref)) : 0.0f, s_red);
    if (smax >= 1e-30f && fabsf(gamma) > (float)ENERGY_SKIP_RTOL_MIXED * escale) {
      int exn;
      frexpf(smax, &exn);
      const float sc = ldexpf(1.0f, -exn), usc = ldexpf(1.0f, exn);
      const float rf = ref * sc, gm = gamma * sc * sc;
      const float ql = phL * sc;
      float c2 = ql;
      const float tol = 2.4e-7f * 1.0f + 1e-30f;   // scaled units: values are of order one
      bool conv = false, feasible = true;
      for (int it = 0; it < P.picard_cap; ++it) {
        const float a = w2 * (mass ? c2 : rf + c2);
        if (part) s_a[tid] = a;
        __syncthreads();
        if (bnd && tid < 4 * NN) {
          const int f = tid / NN, qq = tid % NN;
          const float* L = (f == 1 || f == 3) ? s_l1 : s_l0;
          float acc = 0.0f;
          for (int k = 0; k < NN; ++k) acc = fmaf(f < 2 ? s_a[qq * NN + k] : s_a[k * NN + qq], L[k], acc);
          s_ca[tid] = acc;
        }
        if (mass) {
          const float cm = block_sum<NT>(w2 * a, s_red);
          if (tid == 0) s_ca[nb_rows] = cm;
        }
        __syncthreads();
        float q = 0.0f;
        if (part) {
          float acc = a;
          for (int k = 0; k < m; ++k) acc = fmaf(-X.Cp[(size_t)k * ND + tid], s_ca[k], acc);
          q = acc;
        }
        const float2 ab = block_sum2<NT>(w2 * ql * q, w2 * q * q, s_red2);
        float alpha = ab.x;
        if (!mass) alpha = fmaf(rf, block_sum<NT>(w2 * q, s_red), alpha);
        const float beta = ab.y;
        float s;
        if (beta <= 0.0f) { s = 0.0f; feasible = gm <= 0.0f; }
        else {
          const float disc = alpha * alpha - beta * gm;
          if (disc < 0.0f) { s = -alpha / beta; feasible = false; }
          else {
            const float root = sqrtf(disc);
            const float den = alpha + (alpha >= 0.0f ? root : -root);
            s = den == 0.0f ? 0.0f : -gm / den;
            feasible = true;
          }
        }
        const float nv = part ? fmaf(s, q, ql) : 0.0f;
        const float delta = block_max<NT>(part ? fabsf(nv - c2) : 0.0f, s_red);
        c2 = nv;
        if (delta <= tol) { conv = feasible; break; }
        __syncthreads();
      }
      if (conv) cur = c2 * usc;               // else keep the linear-constraint solution
      ok = conv;
    }
  }
  if (part) {
    const double v = lref(ref, gx, gy, X.xid[i], X.xid[j]) + (double)cur;   // L + psi, split into hi + lo
    const float s = (float)v;
    out[E.base + tid] = s;
    out[X.plane + E.base + tid] = (float)(v - (double)s);
    if (!isfinite(s)) atomicOr(status, SL_ST_NONFINITE);
  }
  if (!ok && tid == 0) atomicOr(status, SL_ST_PICARD_NOCONV);
}

template <int NN>
void launch_n(int phase, const StepParams& p, const Mixed2DExtra& x, const Map2D& m, int64_t count, const float* in,
              float* out, const Work2M& w, unsigned* st, cudaStream_t s) {
  if (count <= 0) return;
  if (phase == 1) k_p1<NN><<<(unsigned)count, Shape<NN>::NT, 0, s>>>(p, x, m, in, w, st);
  else k_p2<NN><<<(unsigned)count, Shape<NN>::NT, 0, s>>>(p, x, m, in, w, out, st);
}

}  // namespace k2m
}  // namespace sl
