#pragma once
// 2D DSEM-SL step, mixed precision, shared operator: uniform mesh and constant velocity (a, b), so
// every element sees the same advected geometry (Sec. 5.3).  Operators are built once on the host
// (ops_mixed2d.cpp) and applied here in structured form, n threads per element:
//   row phase (thread j owns row j): x-remap of the row, x inflow residual pieces, y-neighbour
//     outflow functional, mass residual pieces                      (eq. 5.4, 4.12a, remap_mass)
//   column phase (thread j owns column j): y-remap of the column, inflow residuals
//   fit: s = (C C^T)^+ r over the inflow-face and mass rows, phi_L = psihat + C^T s   (eq. matrix_a)
// C^T s is separable (face rows are l0/l1 along one index and a unit vector along the other, the
// mass row is w (x) w), so the constrained fit costs O(n) per node instead of O(n) per constraint.
// Operators applied with the same entry by every thread are read from the parameter bank.
// State is double-float (hi plane, lo plane); all arithmetic is in float on increments relative to
// the element's first hi value and the result is written back exactly (TwoSum).
//
// A CTA owns a TX x TY tile of elements.  Each staged tile row (the TX elements plus the x-upwind
// halo element) is one contiguous run of global memory; it is copied in aligned 16-byte vectors
// into a shared row buffer at the same offset modulo 16 bytes, followed by the y-upwind halo row.
// Results are written back into the own slots and stored from there with aligned vectors.
// With the mass row, the element's mass target is also formed in float-float: M^n (float-float sum of
// w (x) w (hi + lo)) minus its outflow fluxes through the x- and y-outflow faces plus its upwind
// neighbours' outflow fluxes, each flux a fixed float functional of one element's values evaluated
// alike by that element and by its downstream neighbour (so global mass telescopes); after the fit
// the float-float miss of the written element mass is moved along the mass column of the
// pseudo-inverse into the lo words.
#include "ffloat.cuh"
#include "sl_internal.h"

namespace sl {
namespace k2c {

template <int NN, int TX, int TY>
struct Tile {
  static constexpr int ND = NN * NN;
  static constexpr int NE = TX * TY;              // elements advanced by one CTA
  static constexpr int RW = TX + 1;               // slots per staged tile row (with the x halo)
  static constexpr int RS = (RW * ND + 8 + 3) & ~3;   // floats per staged row buffer (16-byte multiple)
  static constexpr int HS = (TX * ND + 8 + 3) & ~3;   // floats of the y-halo row buffer
  static constexpr int SP = TY * RS + HS;         // floats per staged plane
  static constexpr int VR = RS / 4, VH = HS / 4, VT = TY * VR + VH;   // 16-byte vectors
  static constexpr int NT = NE * NN;              // threads
  static constexpr int MAXV = (VT + NT - 1) / NT; // vectors per thread and plane
};

__device__ __forceinline__ int wrapi(int i, int n, bool per) {
  if (i >= 0 && i < n) return i;
  if (!per) return -1;
  i %= n;
  return i < 0 ? i + n : i;
}

__device__ __forceinline__ int64_t floor4(int64_t g) { return g & ~int64_t(3); }

template <int NN, int TX, int TY>
__global__ void __launch_bounds__(Tile<NN, TX, TY>::NT)
    k_step2d_shared(const __grid_constant__ Mixed2DConstParams P, const float* __restrict__ tab,
                    const float* __restrict__ in, float* __restrict__ out, unsigned* status) {
  using T = Tile<NN, TX, TY>;
  constexpr int ND = T::ND, NE = T::NE, RW = T::RW, RS = T::RS, SP = T::SP, NT = T::NT;
  constexpr int VR = T::VR, VT = T::VT, MAXV = T::MAXV;
  __shared__ __align__(16) float s_hi[SP];
  __shared__ __align__(16) float s_lo[SP];
  __shared__ float s_t[NE * ND];                  // x-remapped rows
  __shared__ float s_dx[NE][NN], s_v[NE][NN], s_p[NE][NN], s_r[NE][2 * NN], s_sw[NE][NN], s_se[NE][NN];
  __shared__ int64_t s_a0[TY + 1];                // first aligned global float of each staged row
  __shared__ int s_off[TY + 1], s_nv[TY + 1];     // row data offset in its buffer; vectors (0: gather)
  const int tid = threadIdx.x;
  // mass refinement (dynamic shared memory): per element and row, the row partials of the own and
  // upwind outflow fluxes and of M^n (slots 0-5), then per column the written mass (6, 7)
  extern __shared__ __align__(16) float s_dyn[];
  float (*s_fp)[NN][8] = reinterpret_cast<float (*)[NN][8]>(s_dyn);
  const int ex0 = blockIdx.x * TX, ey0 = blockIdx.y * TY;
  const bool perx = P.per_x != 0, pery = P.per_y != 0;
  const int xs0 = P.xw ? ex0 - 1 : ex0;           // first element of a staged tile row
  const int eyh = P.ys ? ey0 - 1 : ey0 + TY;      // element row of the y halo
  if (tid <= TY) {
    const int ey = tid < TY ? ey0 + tid : eyh;
    const int xa = tid < TY ? xs0 : ex0, cnt = tid < TY ? RW : TX;
    const int64_t g0 = ((int64_t)ey * P.kx + xa) * ND;
    const int64_t a0 = floor4(g0);
    const bool fast = ey >= 0 && ey < P.ky && xa >= 0 && xa + cnt <= P.kx;
    s_a0[tid] = a0;
    s_off[tid] = (int)(g0 - a0);
    s_nv[tid] = fast ? (int)((floor4(g0 + cnt * ND + 3) - a0) >> 2) : 0;
  }
  __syncthreads();
  // contiguous rows: every vector load first, then the shared stores
  {
    float4 vh[MAXV], vl[MAXV];
#pragma unroll
    for (int k = 0; k < MAXV; ++k) {
      const int v = tid + k * NT;
      const int r = v < TY * VR ? v / VR : TY;
      const int vv = v - r * VR;
      if (v < VT && vv < s_nv[r]) {
        const float4* src = reinterpret_cast<const float4*>(in + s_a0[r]) + vv;
        vh[k] = __ldg(src);
        vl[k] = __ldg(reinterpret_cast<const float4*>(reinterpret_cast<const float*>(src) + P.plane));
      }
    }
#pragma unroll
    for (int k = 0; k < MAXV; ++k) {
      const int v = tid + k * NT;
      const int r = v < TY * VR ? v / VR : TY;
      const int vv = v - r * VR;
      if (v < VT && vv < s_nv[r]) {
        reinterpret_cast<float4*>(s_hi + r * RS)[vv] = vh[k];
        reinterpret_cast<float4*>(s_lo + r * RS)[vv] = vl[k];
      }
    }
  }
  // rows that wrap, leave the mesh or are ragged: element by element (ghost slots hold zero)
#pragma unroll 1
  for (int r = 0; r <= TY; ++r) {
    if (s_nv[r] != 0) continue;
    const int ey = r < TY ? ey0 + r : eyh;
    const int xa = r < TY ? xs0 : ex0, cnt = r < TY ? RW : TX;
    const int wy = wrapi(ey, P.ky, pery);
    const int base = r * RS + s_off[r];
    for (int idx = tid; idx < cnt * ND; idx += NT) {
      const int sl = idx / ND, q = idx - sl * ND;
      const int wx = wrapi(xa + sl, P.kx, perx);
      const bool ok = wx >= 0 && wy >= 0;
      const size_t g = ((size_t)wy * P.kx + wx) * ND + q;
      s_hi[base + idx] = ok ? __ldg(in + g) : 0.0f;
      s_lo[base + idx] = ok ? __ldg(in + P.plane + g) : 0.0f;
    }
  }
  __syncthreads();

  const int el = tid / NN, j = tid - (tid / NN) * NN;   // element in the tile, row / column index
  const int lx = el % TX, ly = el / TX;
  const int ex = ex0 + lx, ey = ey0 + ly;
  const bool active = ex < P.kx && ey < P.ky;
  // own slot, x-upwind neighbour (same staged row), y-upwind neighbour (adjacent row or the halo)
  const int so = ly * RS + s_off[ly] + (lx + P.xw) * ND;
  const int sx = ly * RS + s_off[ly] + (P.xw ? lx : lx + 1) * ND;
  const int ry = P.ys ? ly - 1 : ly + 1;
  const int sy = (ry >= 0 && ry < TY) ? ry * RS + s_off[ry] + (lx + P.xw) * ND : TY * RS + s_off[TY] + lx * ND;
  const bool gx = wrapi(P.xw ? ex - 1 : ex + 1, P.kx, perx) < 0;
  const bool gy = wrapi(P.ys ? ey - 1 : ey + 1, P.ky, pery) < 0;
  const float ref = s_hi[so];
  const float gval = (float)(P.ghost - (double)ref);

  // ---- row phase: thread j holds row j of psi and psi_X, column j of psi_Y
  float ps[NN];
  {
    float px[NN], py[NN];
    const float2 mref = make_float2(-ref, -ref);
#pragma unroll
    for (int i = 0; i < NN; ++i) {                // own and x-neighbour node side by side
      const float2 d = __fadd2_rn(make_float2(s_hi[so + j * NN + i], s_hi[sx + j * NN + i]), mref);
      const float2 v = __fadd2_rn(d, make_float2(s_lo[so + j * NN + i], s_lo[sx + j * NN + i]));
      ps[i] = v.x;
      px[i] = gx ? gval : v.y;
      py[i] = gy ? gval : (s_hi[sy + i * NN + j] - ref) + s_lo[sy + i * NN + j];
    }
    // x inflow residual pieces: upwind outflow trace minus own inflow trace, before the y-remap
    float u = 0.0f, tau = 0.0f, v = 0.0f, pm = 0.0f;
#pragma unroll
    for (int i = 0; i < NN; ++i) {
      u = fmaf(P.rox[i], px[i], u);
      tau = fmaf(P.xix[i], ps[i], tau);
      v = fmaf(P.roy[i], py[i], v);
    }
    // mass residual pieces (target minus the mass of psihat, reference measure)
    const float* Ks = tab + P.o_ks;
    const float* Kx = tab + P.o_kx;
    const float* Ky = tab + P.o_ky;
#pragma unroll
    for (int i = 0; i < NN; ++i) {
      pm = fmaf(__ldg(Ks + i * NN + j), ps[i], pm);
      pm = fmaf(__ldg(Kx + i * NN + j), px[i], pm);
      pm = fmaf(__ldg(Ky + i * NN + j), py[i], pm);
    }
    s_dx[el][j] = (gx ? 0.0f : u) - tau;
    s_v[el][j] = gy ? 0.0f : v;
    s_p[el][j] = pm;
  }
  if (P.refine) {
    // row j of: the own outflow fluxes (x, y faces), the upwind neighbours' outflow fluxes (their
    // rows with their own references, in the same operations as they use themselves), the own mass
    const float* Fx = tab + P.o_fx;
    const float* Fy = tab + P.o_fy;
    const float* Wh = tab + P.o_wh;
    const float* Wl = tab + P.o_wl;
    float fxo = 0.0f, fyo = 0.0f, fxu = 0.0f, fyu = 0.0f;
    cdot mn;
    const float refx = s_hi[sx], refy = s_hi[sy];
#pragma unroll
    for (int i = 0; i < NN; ++i) {
      const float fxi = __ldg(Fx + i * NN + j), fyi = __ldg(Fy + i * NN + j);
      const float hi = s_hi[so + j * NN + i], lo = s_lo[so + j * NN + i];
      const float qo = __fadd_rn(__fsub_rn(hi, ref), lo);
      const float qx = __fadd_rn(__fsub_rn(s_hi[sx + j * NN + i], refx), s_lo[sx + j * NN + i]);
      const float qy = __fadd_rn(__fsub_rn(s_hi[sy + j * NN + i], refy), s_lo[sy + j * NN + i]);
      fxo = fmaf(fxi, qo, fxo);
      fyo = fmaf(fyi, qo, fyo);
      fxu = fmaf(fxi, qx, fxu);
      fyu = fmaf(fyi, qy, fyu);
      mn.add(__ldg(Wh + i * NN + j), __ldg(Wl + i * NN + j), hi, lo);
    }
    const ff mnr = mn.get();
    s_fp[el][j][0] = fxo;
    s_fp[el][j][1] = fyo;
    s_fp[el][j][2] = fxu;
    s_fp[el][j][3] = fyu;
    s_fp[el][j][4] = mnr.hi;
    s_fp[el][j][5] = mnr.lo;
  }
  // x-remap of row j: t[j][l] = sum_i R_x[l][i] psi[j][i]; rows l, l + 1 in paired FMAs (each
  // lane rounds like fmaf, in the same order)
#pragma unroll
  for (int q = 0; q < NN / 2; ++q) {
    float2 acc = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int i = 0; i < NN; ++i) acc = __ffma2_rn(P.Rxp[q][i], make_float2(ps[i], ps[i]), acc);
    s_t[el * ND + j * NN + 2 * q] = acc.x;
    s_t[el * ND + j * NN + 2 * q + 1] = acc.y;
  }
  if (NN & 1) {
    constexpr int l = NN - 1;
    float acc = 0.0f;
#pragma unroll
    for (int i = 0; i < NN; ++i) acc = fmaf(P.Rx[l * NN + i], ps[i], acc);
    s_t[el * ND + j * NN + l] = acc;
  }
  __syncthreads();

  // ---- column phase: thread j holds column j of psihat = R_y t
  float ph[NN];
  {
    float tc[NN];
#pragma unroll
    for (int m = 0; m < NN; ++m) tc[m] = s_t[el * ND + m * NN + j];
#pragma unroll
    for (int q = 0; q < NN / 2; ++q) {
      float2 acc = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int m = 0; m < NN; ++m) acc = __ffma2_rn(P.Ryp[q][m], make_float2(tc[m], tc[m]), acc);
      ph[2 * q] = acc.x;
      ph[2 * q + 1] = acc.y;
    }
    if (NN & 1) {
      constexpr int k = NN - 1;
      float acc = 0.0f;
#pragma unroll
      for (int m = 0; m < NN; ++m) acc = fmaf(P.Ry[k * NN + m], tc[m], acc);
      ph[k] = acc;
    }
  }
  float rm = 0.0f;                                // mass residual (same summation order everywhere)
#pragma unroll
  for (int q = 0; q < NN; ++q) rm += s_p[el][q];
  if (P.bnd) {
    const float* RxT = tab + P.o_RxT;
    const float* RyT = tab + P.o_RyT;
    float rx = 0.0f, vy = 0.0f, ty = 0.0f;
#pragma unroll
    for (int m = 0; m < NN; ++m) {
      rx = fmaf(__ldg(RyT + m * NN + j), s_dx[el][m], rx);
      vy = fmaf(__ldg(RxT + m * NN + j), s_v[el][m], vy);
      ty = fmaf(P.liny[m], ph[m], ty);
    }
    s_r[el][j] = rx + (gx ? gval : 0.0f);
    s_r[el][NN + j] = (vy + (gy ? gval : 0.0f)) - ty;
  }
  __syncthreads();

  // ---- fit: s = (C C^T)^+ r; thread j forms the face entries of row / column j
  float sS = 0.0f, sN = 0.0f, sm = 0.0f;
  if (P.bnd) {
    const int mc = P.mc;
    const float* G = tab + P.o_g;
    float sW = 0.0f, sE = 0.0f;
#pragma unroll
    for (int k = 0; k < 2 * NN; ++k) {
      const float rk = s_r[el][k];
      sW = fmaf(__ldg(G + (0 * mc + k) * NN + j), rk, sW);
      sE = fmaf(__ldg(G + (1 * mc + k) * NN + j), rk, sE);
      sS = fmaf(__ldg(G + (2 * mc + k) * NN + j), rk, sS);
      sN = fmaf(__ldg(G + (3 * mc + k) * NN + j), rk, sN);
      sm = fmaf(P.gm[k], rk, sm);
    }
    if (P.mass) {
      sW = fmaf(__ldg(G + (0 * mc + 2 * NN) * NN + j), rm, sW);
      sE = fmaf(__ldg(G + (1 * mc + 2 * NN) * NN + j), rm, sE);
      sS = fmaf(__ldg(G + (2 * mc + 2 * NN) * NN + j), rm, sS);
      sN = fmaf(__ldg(G + (3 * mc + 2 * NN) * NN + j), rm, sN);
      sm = fmaf(P.gm[2 * NN], rm, sm);
    }
    s_sw[el][j] = sW;
    s_se[el][j] = sE;
    __syncthreads();
  } else {
    sm = P.gm[0] * rm;
  }

  // ---- phi_L = psihat + C^T s, column j; exact write-back into the own slot
  {
    const float l0j = __ldg(tab + P.o_l0 + j), l1j = __ldg(tab + P.o_l1 + j);
    const float wj = __ldg(tab + P.o_w + j) * sm;
    bool finite = true;
    float vh[NN], vl[NN];
    // nodes k and k + 1 in paired operations, each lane in the scalar order (a - b as fma(b, -1, a))
    const float2 rr = make_float2(ref, ref), m1 = make_float2(-1.0f, -1.0f);
#pragma unroll
    for (int k = 0; k + 1 < NN; k += 2) {
      float2 acc = make_float2(ph[k], ph[k + 1]);
      acc = __ffma2_rn(make_float2(sS, sS), make_float2(P.l0[k], P.l0[k + 1]), acc);
      acc = __ffma2_rn(make_float2(sN, sN), make_float2(P.l1[k], P.l1[k + 1]), acc);
      acc = __ffma2_rn(make_float2(wj, wj), make_float2(P.w[k], P.w[k + 1]), acc);
      if (P.bnd) {
        acc = __ffma2_rn(make_float2(s_sw[el][k], s_sw[el][k + 1]), make_float2(l0j, l0j), acc);
        acc = __ffma2_rn(make_float2(s_se[el][k], s_se[el][k + 1]), make_float2(l1j, l1j), acc);
      }
      const float2 s2 = __fadd2_rn(rr, acc);
      const float2 bb = __ffma2_rn(rr, m1, s2);                         // s - ref
      const float2 t = __ffma2_rn(__ffma2_rn(bb, m1, s2), m1, rr);      // ref - (s - bb)
      const float2 e = __fadd2_rn(t, __ffma2_rn(bb, m1, acc));          // + (acc - bb)
      vh[k] = s2.x;
      vh[k + 1] = s2.y;
      vl[k] = e.x;
      vl[k + 1] = e.y;
    }
    if (NN & 1) {
      constexpr int k = NN - 1;
      float acc = ph[k];
      acc = fmaf(sS, P.l0[k], acc);
      acc = fmaf(sN, P.l1[k], acc);
      acc = fmaf(wj, P.w[k], acc);
      if (P.bnd) {
        acc = fmaf(s_sw[el][k], l0j, acc);
        acc = fmaf(s_se[el][k], l1j, acc);
      }
      const float s = ref + acc;
      const float bb = s - ref;
      vh[k] = s;
      vl[k] = (ref - (s - bb)) + (acc - bb);
    }
    if (P.refine) {
      // float-float mass of column j, summed over the columns by the element's first thread; the
      // miss against the target goes along the mass column of the pseudo-inverse into the lo words
      const float* Wh = tab + P.o_wh;
      const float* Wl = tab + P.o_wl;
      cdot mvc;
#pragma unroll
      for (int k = 0; k < NN; ++k) mvc.add(__ldg(Wh + k * NN + j), __ldg(Wl + k * NN + j), vh[k], vl[k]);
      const ff mv = mvc.get();
      s_fp[el][j][6] = mv.hi;
      s_fp[el][j][7] = mv.lo;
      __syncthreads();
      // F(element) = ref sum(f) + the row partials added in row order: own fluxes with this element's
      // reference, upwind fluxes with the neighbour's (or the ghost value); every thread of the
      // element forms the target and the miss in the same order
      float axo = 0.0f, ayo = 0.0f, axu = 0.0f, ayu = 0.0f;
      ff mn = {0.0f, 0.0f}, tot = {0.0f, 0.0f};
#pragma unroll
      for (int q = 0; q < NN; ++q) {
        axo += s_fp[el][q][0];
        ayo += s_fp[el][q][1];
        axu += s_fp[el][q][2];
        ayu += s_fp[el][q][3];
        mn = ff_add(mn, ff{s_fp[el][q][4], s_fp[el][q][5]});
        tot = ff_add(tot, ff{s_fp[el][q][6], s_fp[el][q][7]});
      }
      const float gh = (float)P.ghost;
      const float Fxo = fmaf(ref, P.sfx, axo), Fyo = fmaf(ref, P.sfy, ayo);
      const float Fxu = gx ? gh * P.sfx : fmaf(s_hi[sx], P.sfx, axu);
      const float Fyu = gy ? gh * P.sfy : fmaf(s_hi[sy], P.sfy, ayu);
      // M^{n+1} = M^n - (outflow) + (inflow), float-float
      const ff tg = ff_add(mn, ff_add(two_sum(-Fxo, -Fyo), two_sum(Fxu, Fyu)));
      const float miss = ff_to_f(ff_add(tg, ff_neg(tot)));
      const float* Cm = tab + P.o_cm;
#pragma unroll
      for (int k = 0; k < NN; ++k) {
        const ff v = fast_two_sum(vh[k], fmaf(miss, __ldg(Cm + k * NN + j), vl[k]));
        vh[k] = v.hi;
        vl[k] = v.lo;
      }
    }
#pragma unroll
    for (int k = 0; k < NN; ++k) {
      s_hi[so + k * NN + j] = vh[k];
      s_lo[so + k * NN + j] = vl[k];
      finite = finite && isfinite(vh[k]);
    }
    if (active && !finite) atomicOr(status, SL_ST_NONFINITE);
  }
  __syncthreads();

  // ---- stores: the own elements of a tile row are one contiguous run; aligned vectors inside,
  // single floats at its ends
#pragma unroll 1
  for (int r = 0; r < TY; ++r) {
    const int eyr = ey0 + r;
    if (eyr >= P.ky) break;
    const int cnt = min(TX, P.kx - ex0);
    const int64_t g0 = ((int64_t)eyr * P.kx + ex0) * ND, g1 = g0 + (int64_t)cnt * ND;
    const int64_t A = floor4(g0 + 3), B = floor4(g1);
    const int64_t a0 = s_a0[r];                   // global float G of this row is at r RS + (G - a0)
    const float* rh = s_hi + r * RS;
    const float* rl = s_lo + r * RS;
    if (A <= B) {
      const int nvec = (int)((B - A) >> 2);
      for (int v = tid; v < nvec; v += NT) {
        const int64_t G = A + 4 * (int64_t)v;
        const int q = (int)(G - a0);
        *reinterpret_cast<float4*>(out + G) = *reinterpret_cast<const float4*>(rh + q);
        *reinterpret_cast<float4*>(out + P.plane + G) = *reinterpret_cast<const float4*>(rl + q);
      }
      if (tid < A - g0) {
        const int q = (int)(g0 + tid - a0);
        out[g0 + tid] = rh[q];
        out[P.plane + g0 + tid] = rl[q];
      }
      if (tid < g1 - B) {
        const int q = (int)(B + tid - a0);
        out[B + tid] = rh[q];
        out[P.plane + B + tid] = rl[q];
      }
    } else if (tid < g1 - g0) {
      const int q = (int)(g0 + tid - a0);
      out[g0 + tid] = rh[q];
      out[P.plane + g0 + tid] = rl[q];
    }
  }
}

template <int NN, int TX, int TY>
void launch(const Mixed2DConstParams& p, const float* tab, const float* in, float* out, unsigned* st, cudaStream_t s) {
  dim3 grid((p.kx + TX - 1) / TX, (p.ky + TY - 1) / TY);
  const size_t dyn = p.refine ? (size_t)Tile<NN, TX, TY>::NE * NN * 8 * sizeof(float) : 0;
  if (dyn) allow_dynamic_smem((const void*)k_step2d_shared<NN, TX, TY>, dyn);
  k_step2d_shared<NN, TX, TY><<<grid, Tile<NN, TX, TY>::NT, dyn, s>>>(p, tab, in, out, st);
}

}  // namespace k2c
}  // namespace sl
