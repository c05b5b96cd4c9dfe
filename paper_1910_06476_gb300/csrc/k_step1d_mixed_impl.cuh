#pragma once
// 1D DSEM-SL step, mixed precision, shared operator (uniform mesh, constant velocity).
//
// State: double-float, a hi plane and a lo plane of floats (phi = hi + lo, about 48 bits).
// Every element of a CTA tile is advanced by one thread:
//   - its values and its upwind neighbour's are read relative to a per-element reference
//     ref = hi of its first node: psi = (hi - ref) + lo, in float.  The step operator
//     reproduces constants, so phi^{n+1} = ref + G psi and the float rounding scales with the
//     variation inside the stencil rather than with |phi|;
//   - the linear step (remap eq. 4.9, upwinded boundary values eq. 4.12a, mass target
//     eq. remap_mass, constrained fit eq. matrix_a) is one shared operator applied in float;
//   - the energy constraint (eq. remap_energy) is solved per element; its mismatch is formed
//     from increments only, so that the decision to apply it is free of float cancellation;
//   - the result is written back exactly as ref + psi by TwoSum (Knuth), hi = fl(ref + psi),
//     lo = (ref + psi) - hi.
// The tile (and its upwind halo element) is staged through shared memory with coalesced loads
// and stores; the kernel reads 8 and writes 8 bytes per node from HBM.
#include "sl_internal.h"

namespace sl {
namespace k1m {

constexpr int TILE = 256;                  // elements (threads) per CTA

__device__ __forceinline__ int wrap_elem(int e, int K, bool periodic) {
  if (e >= 0 && e < K) return e;
  if (!periodic) return -1;
  e %= K;
  return e < 0 ? e + K : e;
}

template <int NN>
__global__ void __launch_bounds__(TILE) k_step1d_mixed(const __grid_constant__ Mixed1DParams P,
                                                       const float* __restrict__ in, float* __restrict__ out,
                                                       unsigned* status) {
  constexpr int SH = 4;                     // row r of the tile lives at s[SH + r * NN + i]
  constexpr int SMEM = (TILE + 1) * NN + 16;
  __shared__ __align__(16) float shi[SMEM];
  __shared__ __align__(16) float slo[SMEM];
  const int tid = threadIdx.x;
  const int K = P.K;
  const int64_t plane = P.plane;            // float offset of the lo plane (multiple of 64)
  const int e0 = blockIdx.x * TILE;
  // tile rows: left upwind -> elements [e0-1, e0+TILE), right upwind -> [e0, e0+TILE]
  const int first = P.left_up ? e0 - 1 : e0;
  // rows whose elements lie in [0, K) are contiguous in memory: one aligned 16-byte window
  const int r_lo = max(0, -first), r_hi = min(TILE + 1, K - first);
  {
    const int64_t g0 = (int64_t)(first + r_lo) * NN, g1 = (int64_t)(first + r_hi) * NN;
    const int64_t a0 = g0 & ~int64_t(3), a1 = (g1 + 3) & ~int64_t(3);   // a1 <= plane: padded
    const int sbase = SH + r_lo * NN - (int)(g0 - a0);
    const int nvec = (int)((a1 - a0) >> 2);
    const float4* ih = reinterpret_cast<const float4*>(in + a0);
    const float4* il = reinterpret_cast<const float4*>(in + plane + a0);
    constexpr int VPT = ((TILE + 1) * NN + 8 + 4 * TILE - 1) / (4 * TILE);   // vectors per thread
    float4 vh[VPT], vl[VPT];
#pragma unroll
    for (int k = 0; k < VPT; ++k) {          // issue every load before the first shared store
      const int v = tid + k * TILE;
      if (v < nvec) { vh[k] = __ldg(ih + v); vl[k] = __ldg(il + v); }
    }
#pragma unroll
    for (int k = 0; k < VPT; ++k) {
      const int v = tid + k * TILE;
      if (v < nvec) {
        float* dh = shi + sbase + 4 * v;
        float* dl = slo + sbase + 4 * v;
        dh[0] = vh[k].x; dh[1] = vh[k].y; dh[2] = vh[k].z; dh[3] = vh[k].w;
        dl[0] = vl[k].x; dl[1] = vl[k].y; dl[2] = vl[k].z; dl[3] = vl[k].w;
      }
    }
  }
  // the one halo row that can fall outside [0, K): periodic wrap (or none at an inflow face)
  const int hrow = P.left_up ? 0 : r_hi;
  const bool hfix = P.left_up ? (r_lo == 1) : (r_hi <= TILE);
  __syncthreads();
  if (hfix && tid < NN) {
    const int eh = wrap_elem(first + hrow, K, P.periodic != 0);
    shi[SH + hrow * NN + tid] = eh >= 0 ? in[(int64_t)eh * NN + tid] : 0.0f;
    slo[SH + hrow * NN + tid] = eh >= 0 ? in[plane + (int64_t)eh * NN + tid] : 0.0f;
  }
  __syncthreads();

  const int e = e0 + tid;
  const bool active = e < K;
  const int own = SH + (P.left_up ? tid + 1 : tid) * NN;
  const int up = SH + (P.left_up ? tid : tid + 1) * NN;
  const int eup = wrap_elem(P.left_up ? e - 1 : e + 1, K, P.periodic != 0);
  float res[NN];
  float ref = 0.0f;
  bool ok = true;
  if (active) {
    ref = shi[own];
    float ps[NN], pu[NN];
#pragma unroll
    for (int i = 0; i < NN; ++i) ps[i] = (shi[own + i] - ref) + slo[own + i];
    if (eup >= 0) {
#pragma unroll
      for (int i = 0; i < NN; ++i) pu[i] = (shi[up + i] - ref) + slo[up + i];
    } else {
      const float g = (float)(P.ghost - (double)ref);   // ghost value at the inflow domain face
#pragma unroll
      for (int i = 0; i < NN; ++i) pu[i] = g;
    }
    // shared linear operator
    float pl[NN];
#pragma unroll
    for (int j = 0; j < NN; ++j) {
      float acc = 0.0f;
#pragma unroll
      for (int i = 0; i < NN; ++i) acc = fmaf(P.Gs[j * NN + i], ps[i], acc);
#pragma unroll
      for (int i = 0; i < NN; ++i) acc = fmaf(P.Gu[j * NN + i], pu[i], acc);
      pl[j] = acc;
    }
#pragma unroll
    for (int j = 0; j < NN; ++j) res[j] = pl[j];

    if (P.energy_on) {
      // The energy iteration is covariant under phi -> c phi (gamma, alpha, beta scale by c^2, q by
      // c, s is invariant), so it runs on values scaled by a power of two to order one; elements
      // whose values lie below the normal float range carry no energy correction.
      float smax = fabsf(ref);
#pragma unroll
      for (int i = 0; i < NN; ++i) smax = fmaxf(smax, fmaxf(fabsf(ps[i]), fabsf(pu[i])));
      if (smax >= 1e-30f) {
        int ex;
        frexpf(smax, &ex);
        const float sc = ldexpf(1.0f, -ex), usc = ldexpf(1.0f, ex);
        const float rf = ref * sc;
        float qs[NN], qu[NN], ql[NN];
#pragma unroll
        for (int i = 0; i < NN; ++i) { qs[i] = ps[i] * sc; qu[i] = pu[i] * sc; ql[i] = pl[i] * sc; }
        // energy mismatch from increments: variance part, plus 2 ref x mass residual when the mass
        // row is not enforced (with it, that bracket vanishes identically)
        float gv = 0.0f, gm = 0.0f, escale = 0.0f;
#pragma unroll
        for (int i = 0; i < NN; ++i) {
          gv = fmaf(P.w[i], (ql[i] - qs[i]) * (ql[i] + qs[i]), gv);
          gm = fmaf(P.w[i], ql[i] - qs[i], gm);
          const float phv = rf + qs[i];
          escale = fmaf(P.w[i], phv * phv, escale);
        }
        for (int s = 0; s < P.nst; ++s) {
          float es = 0.0f, eu = 0.0f;
#pragma unroll
          for (int i = 0; i < NN; ++i) { es = fmaf(P.E[s][i], qs[i], es); eu = fmaf(P.E[s][i], qu[i], eu); }
          gv = fmaf(P.lam * P.fb[s], es * es - eu * eu, gv);
          gm = fmaf(P.lam * P.fb[s], es - eu, gm);
        }
        const float gamma = P.mass_on ? gv : fmaf(2.0f * rf, gm, gv);
        if (fabsf(gamma) > (float)ENERGY_SKIP_RTOL * escale) {
          float pmax = 0.0f;
#pragma unroll
          for (int i = 0; i < NN; ++i) pmax = fmaxf(pmax, fabsf(ql[i]));
          const float tol = fmaxf(P.picard_rtol * fabsf(rf), 2.4e-7f * pmax) + 1e-30f;
          float cur[NN];
#pragma unroll
          for (int i = 0; i < NN; ++i) cur[i] = ql[i];
          bool conv = false, feasible = true;
          for (int it = 0; it < P.picard_cap; ++it) {
            float av[NN], q[NN];
#pragma unroll
            for (int i = 0; i < NN; ++i) av[i] = P.w[i] * (P.mass_on ? cur[i] : rf + cur[i]);
            float ca[MMAX1D];
            for (int k = 0; k < P.m; ++k) {
              float acc = 0.0f;
#pragma unroll
              for (int i = 0; i < NN; ++i) acc = fmaf(P.C[k * NN + i], av[i], acc);
              ca[k] = acc;
            }
#pragma unroll
            for (int j = 0; j < NN; ++j) {
              float acc = av[j];
              for (int k = 0; k < P.m; ++k) acc = fmaf(-P.Cp[j * P.m + k], ca[k], acc);
              q[j] = acc;
            }
            float alpha = 0.0f, beta = 0.0f, wq = 0.0f;
#pragma unroll
            for (int i = 0; i < NN; ++i) {
              alpha = fmaf(P.w[i] * ql[i], q[i], alpha);
              beta = fmaf(P.w[i] * q[i], q[i], beta);
              wq = fmaf(P.w[i], q[i], wq);
            }
            if (!P.mass_on) alpha = fmaf(rf, wq, alpha);
            float s;
            if (beta <= 0.0f) { s = 0.0f; feasible = gamma <= 0.0f; }
            else {
              const float disc = alpha * alpha - beta * gamma;
              if (disc < 0.0f) { s = -alpha / beta; feasible = false; }
              else {
                const float root = sqrtf(disc);
                const float den = alpha + (alpha >= 0.0f ? root : -root);
                s = den == 0.0f ? 0.0f : -gamma / den;
                feasible = true;
              }
            }
            float delta = 0.0f;
#pragma unroll
            for (int i = 0; i < NN; ++i) {
              const float nv = fmaf(s, q[i], ql[i]);
              delta = fmaxf(delta, fabsf(nv - cur[i]));
              cur[i] = nv;
            }
            if (delta <= tol) { conv = feasible; break; }
          }
          if (conv) {
#pragma unroll
            for (int i = 0; i < NN; ++i) res[i] = cur[i] * usc;
          }                                   // else: keep the linear-constraint solution
          ok = conv;
        }
      }
    }
  }
  __syncthreads();                          // tile rows are rewritten below
  bool finite = true;
  if (active) {
#pragma unroll
    for (int j = 0; j < NN; ++j) {
      // TwoSum: hi + lo == ref + res exactly
      const float s = ref + res[j];
      const float bb = s - ref;
      const float err = (ref - (s - bb)) + (res[j] - bb);
      shi[tid * NN + j] = s;
      slo[tid * NN + j] = err;
      finite = finite && isfinite(s);
    }
  }
  __syncthreads();
  // coalesced write-back: e0 * NN is a multiple of 4 (TILE is), and so is the lo plane offset
  const int nact = min(TILE, K - e0);
  const int nout = nact * NN, nv = nout >> 2;
  float4* oh = reinterpret_cast<float4*>(out + (int64_t)e0 * NN);
  float4* ol = reinterpret_cast<float4*>(out + plane + (int64_t)e0 * NN);
  for (int v = tid; v < nv; v += TILE) {
    oh[v] = reinterpret_cast<const float4*>(shi)[v];
    ol[v] = reinterpret_cast<const float4*>(slo)[v];
  }
  for (int idx = 4 * nv + tid; idx < nout; idx += TILE) {
    out[(int64_t)e0 * NN + idx] = shi[idx];
    out[plane + (int64_t)e0 * NN + idx] = slo[idx];
  }
  const unsigned bits = (finite ? 0u : SL_ST_NONFINITE) | (ok ? 0u : SL_ST_PICARD_NOCONV);
  if (bits) atomicOr(status, bits);
}

template <int NN>
void launch_n(const Mixed1DParams& p, const float* in, float* out, unsigned* st, cudaStream_t s) {
  const int grid = (p.K + TILE - 1) / TILE;
  k_step1d_mixed<NN><<<grid, TILE, 0, s>>>(p, in, out, st);
}

}  // namespace k1m
}  // namespace sl
