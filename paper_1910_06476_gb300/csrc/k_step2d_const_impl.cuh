#pragma once
// 2D DSEM-SL step, mixed precision, shared operator: uniform mesh and constant velocity (a, b), so
// every element sees the same advected geometry (Sec. 5.3).  Operators are built once on the host
// (ops_mixed2d.cpp) and applied here in structured form, n threads per element (thread j owns row
// j of the element's n x n nodes):
//   x-remap of row j, then y-remap through shared memory      psihat = R_y psi R_x^T   (eq. 5.4)
//   own traces at the inflow faces and the upwind neighbours' traces     (eq. 2dx/2dy, 4.12a)
//   mass target from the outflow-face flux functionals                   (eq. remap_mass)
//   constrained fit restricted to the inflow-face rows and the mass row  (eq. matrix_a)
// State is double-float (hi plane, lo plane); all arithmetic is in float on increments relative to
// the element's first hi value and the result is written back exactly (TwoSum).  A CTA owns a
// TX x TY tile of elements plus the x-upwind halo column and the y-upwind halo row.
#include "sl_internal.h"

namespace sl {
namespace k2c {

template <int NN, int TX, int TY>
struct Tile {
  static constexpr int ND = NN * NN;
  static constexpr int NE = TX * TY;              // elements advanced by one CTA
  static constexpr int NS = NE + TX + TY;         // staged elements (tile + halo column + halo row)
  static constexpr int NT = NE * NN;              // threads
  static constexpr int NR = 2 * NN + 1;           // residuals kept: inflow x rows, inflow y rows, mass
};

__device__ __forceinline__ int wrapi(int i, int n, bool per) {
  if (i >= 0 && i < n) return i;
  if (!per) return -1;
  i %= n;
  return i < 0 ? i + n : i;
}

template <int NN, int TX, int TY>
__global__ void __launch_bounds__(Tile<NN, TX, TY>::NT) k_step(const __grid_constant__ Mixed2DConstParams P,
                                                               const float* __restrict__ tab,
                                                               const float* __restrict__ in, float* __restrict__ out,
                                                               unsigned* status) {
  using T = Tile<NN, TX, TY>;
  constexpr int ND = T::ND, NE = T::NE, NS = T::NS, NT = T::NT, NR = T::NR;
  __shared__ float s_hi[NS * ND];
  __shared__ float s_lo[NS * ND];
  __shared__ float s_t[NE * ND];                  // x-remapped rows, then psihat
  __shared__ float s_gx[NE][NN], s_gy[NE][NN], s_p[NE][NN], s_r[NE][NR];
  __shared__ int s_ge[NS];                        // global element of each staged slot (-1: ghost)
  const int tid = threadIdx.x;
  const int ex0 = blockIdx.x * TX, ey0 = blockIdx.y * TY;
  const bool perx = P.per_x != 0, pery = P.per_y != 0;
  // slot -> global element: tile (lx, ly) at ly*TX + lx; x halo of row ly at NE + ly; y halo of
  // column lx at NE + TY + lx
  if (tid < NS) {
    int ex, ey;
    if (tid < NE) { ex = ex0 + tid % TX; ey = ey0 + tid / TX; }
    else if (tid < NE + TY) { ex = P.xw ? ex0 - 1 : ex0 + TX; ey = ey0 + (tid - NE); }
    else { ex = ex0 + (tid - NE - TY); ey = P.ys ? ey0 - 1 : ey0 + TY; }
    const int wx = wrapi(ex, P.kx, perx), wy = wrapi(ey, P.ky, pery);
    s_ge[tid] = (wx < 0 || wy < 0) ? -1 : wy * P.kx + wx;
  }
  __syncthreads();
  {
    constexpr int PER = (NS * ND + NT - 1) / NT;
    float vh[PER], vl[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {                // issue all loads, then store
      const int idx = tid + k * NT;
      vh[k] = 0.0f;
      vl[k] = 0.0f;
      if (idx < NS * ND) {
        const int slot = idx / ND, q = idx - slot * ND;
        const int g = s_ge[slot];
        if (g >= 0) {
          vh[k] = __ldg(in + (size_t)g * ND + q);
          vl[k] = __ldg(in + P.plane + (size_t)g * ND + q);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int idx = tid + k * NT;
      if (idx < NS * ND) { s_hi[idx] = vh[k]; s_lo[idx] = vl[k]; }
    }
  }
  __syncthreads();

  const int el = tid / NN, j = tid % NN;          // element slot in the tile, row
  const int lx = el % TX, ly = el / TX;
  const bool active = (ex0 + lx < P.kx) && (ey0 + ly < P.ky);
  const int sx = P.xw ? (lx > 0 ? el - 1 : NE + ly) : (lx < TX - 1 ? el + 1 : NE + ly);
  const int sy = P.ys ? (ly > 0 ? el - TX : NE + TY + lx) : (ly < TY - 1 ? el + TX : NE + TY + lx);
  const bool gx = s_ge[sx] < 0, gy = s_ge[sy] < 0;
  const float* Rx = tab + P.o_Rx;
  const float* Ry = tab + P.o_Ry;
  const float ref = s_hi[el * ND];
  const float gval = (float)(P.ghost - (double)ref);
  float ps[NN], px[NN];
#pragma unroll
  for (int i = 0; i < NN; ++i) {
    ps[i] = (s_hi[el * ND + j * NN + i] - ref) + s_lo[el * ND + j * NN + i];
    px[i] = gx ? gval : (s_hi[sx * ND + j * NN + i] - ref) + s_lo[sx * ND + j * NN + i];
  }
  // x-remap of row j
#pragma unroll
  for (int l = 0; l < NN; ++l) {
    float acc = 0.0f;
#pragma unroll
    for (int i = 0; i < NN; ++i) acc = fmaf(__ldg(Rx + l * NN + i), ps[i], acc);
    s_t[el * ND + j * NN + l] = acc;
  }
  // x-upwind neighbour: row functional for its outflow trace; y-upwind neighbour: column j functional
  {
    float u = 0.0f, v = 0.0f, pm = 0.0f;
#pragma unroll
    for (int q = 0; q < NN; ++q) {
      u = fmaf(px[q], __ldg(tab + P.o_rox + q), u);
      const float yq = gy ? gval : (s_hi[sy * ND + q * NN + j] - ref) + s_lo[sy * ND + q * NN + j];
      v = fmaf(__ldg(tab + P.o_roy + q), yq, v);
    }
    // mass target, row j: K_self . psi + K_x . psi_X + K_y . psi_Y (row j of psi_Y)
#pragma unroll
    for (int i = 0; i < NN; ++i) {
      const float yi = gy ? gval : (s_hi[sy * ND + j * NN + i] - ref) + s_lo[sy * ND + j * NN + i];
      pm = fmaf(__ldg(tab + P.o_kself + j * NN + i), ps[i], pm);
      pm = fmaf(__ldg(tab + P.o_kx + j * NN + i), px[i], pm);
      pm = fmaf(__ldg(tab + P.o_ky + j * NN + i), yi, pm);
    }
    s_gx[el][j] = u;
    s_gy[el][j] = v;
    s_p[el][j] = pm;
  }
  __syncthreads();
  // y-remap: psihat row j = sum_q R_y[j][q] t[q][.]
  float ph[NN];
#pragma unroll
  for (int l = 0; l < NN; ++l) ph[l] = 0.0f;
#pragma unroll
  for (int q = 0; q < NN; ++q) {
    const float r = __ldg(Ry + j * NN + q);
#pragma unroll
    for (int l = 0; l < NN; ++l) ph[l] = fmaf(r, s_t[el * ND + q * NN + l], ph[l]);
  }
  // x inflow face, row j: upwind value minus own trace
  float trx = 0.0f, valx = 0.0f, mh = 0.0f;
#pragma unroll
  for (int l = 0; l < NN; ++l) {
    trx = fmaf(ph[l], __ldg(tab + P.o_linx + l), trx);
    valx = fmaf(__ldg(Ry + j * NN + l), s_gx[el][l], valx);
    mh = fmaf(__ldg(tab + P.o_w2 + j * NN + l), ph[l], mh);
  }
  if (gx) valx = gval;
  __syncthreads();                                // every thread has read s_t: reuse it for psihat
#pragma unroll
  for (int l = 0; l < NN; ++l) s_t[el * ND + j * NN + l] = ph[l];
  s_r[el][j] = valx - trx;
  const float pmh = mh;
  __syncthreads();
  // y inflow face, column j: upwind value minus own trace
  {
    float tr = 0.0f, val = 0.0f;
#pragma unroll
    for (int m = 0; m < NN; ++m) {
      tr = fmaf(s_t[el * ND + m * NN + j], __ldg(tab + P.o_liny + m), tr);
      val = fmaf(__ldg(Rx + j * NN + m), s_gy[el][m], val);
    }
    if (gy) val = gval;
    s_r[el][NN + j] = val - tr;
  }
  // mass residual: target minus the mass of psihat (row sums in index order)
  s_p[el][j] -= pmh;
  __syncthreads();
  if (j == 0) {
    float acc = 0.0f;
#pragma unroll
    for (int q = 0; q < NN; ++q) acc += s_p[el][q];
    s_r[el][2 * NN] = acc;
  }
  __syncthreads();
  // constrained fit: phi_L = psihat + C+_sub r over the kept rows
  const int mc = P.mc;
  const int r0 = P.bnd ? 0 : 2 * NN;               // without boundary rows only the mass residual
  const float* Cp = tab + P.o_cp;
  float res[NN];
#pragma unroll
  for (int l = 0; l < NN; ++l) {
    float acc = ph[l];
    for (int k = 0; k < mc; ++k) acc = fmaf(__ldg(Cp + (j * NN + l) * mc + k), s_r[el][r0 + k], acc);
    res[l] = acc;
  }
  // exact write-back (TwoSum) into the staging rows of this element, then coalesced stores
  bool finite = true;
#pragma unroll
  for (int l = 0; l < NN; ++l) {
    const float s = ref + res[l];
    const float bb = s - ref;
    const float e = (ref - (s - bb)) + (res[l] - bb);
    s_hi[el * ND + j * NN + l] = s;
    s_lo[el * ND + j * NN + l] = e;
    finite = finite && isfinite(s);
  }
  if (active && !finite) atomicOr(status, SL_ST_NONFINITE);
  __syncthreads();
  // the TX elements of a tile row are consecutive in memory
  for (int idx = tid; idx < NE * ND; idx += NT) {
    const int slot = idx / ND, q = idx - slot * ND;
    const int ex = ex0 + slot % TX, ey = ey0 + slot / TX;
    if (ex < P.kx && ey < P.ky) {
      const size_t g = ((size_t)ey * P.kx + ex) * ND + q;
      out[g] = s_hi[idx];
      out[P.plane + g] = s_lo[idx];
    }
  }
}

template <int NN, int TX, int TY>
void launch(const Mixed2DConstParams& p, const float* tab, const float* in, float* out, unsigned* st, cudaStream_t s) {
  dim3 grid((p.kx + TX - 1) / TX, (p.ky + TY - 1) / TY);
  k_step<NN, TX, TY><<<grid, Tile<NN, TX, TY>::NT, 0, s>>>(p, tab, in, out, st);
}

}  // namespace k2c
}  // namespace sl
