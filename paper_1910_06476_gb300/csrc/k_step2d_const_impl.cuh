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
// the element's first hi value and the result is written back exactly (TwoSum).
//
// A CTA owns a TX x TY tile of elements.  Staging slots are laid out row by row with the x-upwind
// halo element next to its row, so each staged row is one contiguous run of global memory (moved
// with aligned 16-byte vectors), followed by the y-upwind halo row.  Tables that a thread reads by
// its own row are stored transposed, so an element's n threads read consecutive floats.
#include "sl_internal.h"

namespace sl {
namespace k2c {

template <int NN, int TX, int TY>
struct Tile {
  static constexpr int ND = NN * NN;
  static constexpr int NE = TX * TY;              // elements advanced by one CTA
  static constexpr int RW = TX + 1;               // slots per staged tile row (with the x halo)
  static constexpr int NS = TY * RW + TX;         // staged elements (+ the y halo row)
  static constexpr int NT = NE * NN;              // threads
  static constexpr int NR = 2 * NN + 1;           // residuals kept: inflow x rows, inflow y rows, mass
};

__device__ __forceinline__ int wrapi(int i, int n, bool per) {
  if (i >= 0 && i < n) return i;
  if (!per) return -1;
  i %= n;
  return i < 0 ? i + n : i;
}

// Copy cnt contiguous floats of each plane, starting at global float g0, to shared memory at s0;
// the global window is rounded out to 16-byte boundaries (the planes are 256-byte aligned and the
// state buffer ends on a 64-float boundary).
template <int NT, int MAXV>
__device__ __forceinline__ void copy_run(const float* __restrict__ in, int64_t plane, int64_t g0, int cnt, float* shi,
                                         float* slo, int s0, int tid) {
  const int64_t a0 = g0 & ~int64_t(3);
  const int nvec = (int)(((g0 + cnt + 3) & ~int64_t(3)) - a0) >> 2;
  const int off = (int)(g0 - a0);
  const float4* ih = reinterpret_cast<const float4*>(in + a0);
  const float4* il = reinterpret_cast<const float4*>(in + plane + a0);
  float4 vh[MAXV], vl[MAXV];
#pragma unroll
  for (int k = 0; k < MAXV; ++k) {
    const int v = tid + k * NT;
    if (v < nvec) { vh[k] = __ldg(ih + v); vl[k] = __ldg(il + v); }
  }
#pragma unroll
  for (int k = 0; k < MAXV; ++k) {
    const int v = tid + k * NT;
    if (v < nvec) {
      const float h4[4] = {vh[k].x, vh[k].y, vh[k].z, vh[k].w};
      const float l4[4] = {vl[k].x, vl[k].y, vl[k].z, vl[k].w};
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int q = 4 * v + c - off;           // float index within the run
        if (q >= 0 && q < cnt) { shi[s0 + q] = h4[c]; slo[s0 + q] = l4[c]; }
      }
    }
  }
}

template <int NN, int TX, int TY>
__global__ void __launch_bounds__(Tile<NN, TX, TY>::NT) k_step2d_shared(const __grid_constant__ Mixed2DConstParams P,
                                                               const float* __restrict__ tab,
                                                               const float* __restrict__ in, float* __restrict__ out,
                                                               unsigned* status) {
  using T = Tile<NN, TX, TY>;
  constexpr int ND = T::ND, NE = T::NE, RW = T::RW, NS = T::NS, NT = T::NT, NR = T::NR;
  constexpr int MAXV = ((RW * ND + 8) / 4 + NT - 1) / NT;
  __shared__ float s_hi[NS * ND];
  __shared__ float s_lo[NS * ND];
  __shared__ float s_t[NE * ND];                  // x-remapped rows, then psihat
  __shared__ float s_gx[NE][NN], s_gy[NE][NN], s_p[NE][NN], s_r[NE][NR];
  __shared__ int s_ge[NS];                        // global element of each staged slot (-1: ghost)
  const int tid = threadIdx.x;
  const int ex0 = blockIdx.x * TX, ey0 = blockIdx.y * TY;
  const bool perx = P.per_x != 0, pery = P.per_y != 0;
  const int xs0 = P.xw ? ex0 - 1 : ex0;           // first element of a staged tile row
  // slot -> global element
  if (tid < NS) {
    int ex, ey;
    if (tid < TY * RW) { ex = xs0 + tid % RW; ey = ey0 + tid / RW; }
    else { ex = ex0 + (tid - TY * RW); ey = P.ys ? ey0 - 1 : ey0 + TY; }
    const int wx = wrapi(ex, P.kx, perx), wy = wrapi(ey, P.ky, pery);
    s_ge[tid] = (wx < 0 || wy < 0) ? -1 : wy * P.kx + wx;
  }
  __syncthreads();
  // staged rows: contiguous global runs when they need no wrap, else element by element
  const int yrow = P.ys ? ey0 - 1 : ey0 + TY;
#pragma unroll
  for (int r = 0; r <= TY; ++r) {
    const int ey = r < TY ? ey0 + r : yrow;
    const int xa = r < TY ? xs0 : ex0, cntx = r < TY ? RW : TX;
    const int s0 = r < TY ? r * RW : TY * RW;
    const bool fast = ey >= 0 && ey < P.ky && xa >= 0 && xa + cntx <= P.kx;
    if (fast) {
      copy_run<NT, MAXV>(in, P.plane, ((int64_t)ey * P.kx + xa) * ND, cntx * ND, s_hi, s_lo, s0 * ND, tid);
    } else {
      for (int idx = tid; idx < cntx * ND; idx += NT) {
        const int slot = s0 + idx / ND, q = idx % ND;
        const int g = s_ge[slot];
        s_hi[slot * ND + q] = g >= 0 ? __ldg(in + (size_t)g * ND + q) : 0.0f;
        s_lo[slot * ND + q] = g >= 0 ? __ldg(in + P.plane + (size_t)g * ND + q) : 0.0f;
      }
    }
  }
  __syncthreads();

  const int el = tid / NN, j = tid % NN;          // element in the tile, row
  const int lx = el % TX, ly = el / TX;
  const bool active = (ex0 + lx < P.kx) && (ey0 + ly < P.ky);
  const int so = ly * RW + lx + P.xw;             // own slot
  const int sx = P.xw ? so - 1 : so + 1;          // x-upwind neighbour (the halo is in the row)
  const int sy = P.ys ? (ly > 0 ? so - RW : TY * RW + lx) : (ly < TY - 1 ? so + RW : TY * RW + lx);
  const bool gx = s_ge[sx] < 0, gy = s_ge[sy] < 0;
  const float* Rx = tab + P.o_Rx;
  const float* RxT = tab + P.o_RxT;
  const float* RyT = tab + P.o_RyT;
  const float ref = s_hi[so * ND];
  const float gval = (float)(P.ghost - (double)ref);
  float ps[NN], px[NN];
#pragma unroll
  for (int i = 0; i < NN; ++i) {
    ps[i] = (s_hi[so * ND + j * NN + i] - ref) + s_lo[so * ND + j * NN + i];
    px[i] = gx ? gval : (s_hi[sx * ND + j * NN + i] - ref) + s_lo[sx * ND + j * NN + i];
  }
  // x-remap of row j (every thread reads the same R_x entry: a broadcast)
#pragma unroll
  for (int l = 0; l < NN; ++l) {
    float acc = 0.0f;
#pragma unroll
    for (int i = 0; i < NN; ++i) acc = fmaf(__ldg(Rx + l * NN + i), ps[i], acc);
    s_t[el * ND + j * NN + l] = acc;
  }
  // x-upwind neighbour row functional, y-upwind neighbour column functional, mass target row j
  {
    float u = 0.0f, v = 0.0f, pm = 0.0f;
#pragma unroll
    for (int q = 0; q < NN; ++q) {
      u = fmaf(px[q], __ldg(tab + P.o_rox + q), u);
      const float yq = gy ? gval : (s_hi[sy * ND + q * NN + j] - ref) + s_lo[sy * ND + q * NN + j];
      v = fmaf(__ldg(tab + P.o_roy + q), yq, v);
    }
#pragma unroll
    for (int i = 0; i < NN; ++i) {
      const float yi = gy ? gval : (s_hi[sy * ND + j * NN + i] - ref) + s_lo[sy * ND + j * NN + i];
      pm = fmaf(__ldg(tab + P.o_kself + i * NN + j), ps[i], pm);
      pm = fmaf(__ldg(tab + P.o_kx + i * NN + j), px[i], pm);
      pm = fmaf(__ldg(tab + P.o_ky + i * NN + j), yi, pm);
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
    const float r = __ldg(RyT + q * NN + j);
#pragma unroll
    for (int l = 0; l < NN; ++l) ph[l] = fmaf(r, s_t[el * ND + q * NN + l], ph[l]);
  }
  // x inflow face, row j: upwind value minus own trace; mass of psihat row j
  float trx = 0.0f, valx = 0.0f, mh = 0.0f;
#pragma unroll
  for (int l = 0; l < NN; ++l) {
    trx = fmaf(ph[l], __ldg(tab + P.o_linx + l), trx);
    valx = fmaf(__ldg(RyT + l * NN + j), s_gx[el][l], valx);
    mh = fmaf(__ldg(tab + P.o_w2 + l * NN + j), ph[l], mh);
  }
  if (gx) valx = gval;
  __syncthreads();                                // every thread has read s_t: reuse it for psihat
#pragma unroll
  for (int l = 0; l < NN; ++l) s_t[el * ND + j * NN + l] = ph[l];
  s_r[el][j] = valx - trx;
  __syncthreads();
  // y inflow face, column j: upwind value minus own trace
  {
    float tr = 0.0f, val = 0.0f;
#pragma unroll
    for (int m = 0; m < NN; ++m) {
      tr = fmaf(s_t[el * ND + m * NN + j], __ldg(tab + P.o_liny + m), tr);
      val = fmaf(__ldg(RxT + m * NN + j), s_gy[el][m], val);
    }
    if (gy) val = gval;
    s_r[el][NN + j] = val - tr;
  }
  // mass residual: target minus the mass of psihat (row sums in index order)
  s_p[el][j] -= mh;
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
    for (int k = 0; k < mc; ++k) acc = fmaf(__ldg(Cp + (l * mc + k) * NN + j), s_r[el][r0 + k], acc);
    res[l] = acc;
  }
  // exact write-back (TwoSum) into this element's staging rows, then coalesced stores
  bool finite = true;
#pragma unroll
  for (int l = 0; l < NN; ++l) {
    const float s = ref + res[l];
    const float bb = s - ref;
    const float e = (ref - (s - bb)) + (res[l] - bb);
    s_hi[so * ND + j * NN + l] = s;
    s_lo[so * ND + j * NN + l] = e;
    finite = finite && isfinite(s);
  }
  if (active && !finite) atomicOr(status, SL_ST_NONFINITE);
  __syncthreads();
  // the TX elements of a tile row are consecutive in memory and in the staging rows
  for (int idx = tid; idx < NE * ND; idx += NT) {
    const int row = idx / (TX * ND), rem = idx - row * (TX * ND);
    const int ex = ex0 + rem / ND, ey = ey0 + row;
    if (ex < P.kx && ey < P.ky) {
      const size_t g = ((size_t)ey * P.kx + ex0) * ND + rem;
      const int sidx = (row * RW + P.xw) * ND + rem;
      out[g] = s_hi[sidx];
      out[P.plane + g] = s_lo[sidx];
    }
  }
}

template <int NN, int TX, int TY>
void launch(const Mixed2DConstParams& p, const float* tab, const float* in, float* out, unsigned* st, cudaStream_t s) {
  dim3 grid((p.kx + TX - 1) / TX, (p.ky + TY - 1) / TY);
  k_step2d_shared<NN, TX, TY><<<grid, Tile<NN, TX, TY>::NT, 0, s>>>(p, tab, in, out, st);
}

}  // namespace k2c
}  // namespace sl
