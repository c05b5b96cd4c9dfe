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
//     lo = (ref + psi) - hi;
//   - with the mass row (hard fit), the element's mass target is also formed in float-float,
//     M^n - lam (F_own - F_up), where F is the outflow-flux functional applied to an element's hi + lo
//     (each element's F is computed bit for bit alike by the element itself and by its downstream
//     neighbour, so global mass telescopes); after the fit, the float-float miss of the written
//     element mass is moved along the pseudo-inverse column of the mass row into the lo words, so
//     that the element mass meets its target to about 1e-16 relative.
// The kernel is persistent: a CTA advances tiles of TILE elements, one thread per element.  A
// tile's rows (its elements and the upwind halo element) are one contiguous run of each plane;
// one thread moves both runs into shared memory with bulk asynchronous copies (TMA) that complete
// on an mbarrier, into one of two stages, so the next tile's load overlaps this tile's
// arithmetic.  Results are written back into the stage and stored with bulk copies.  The kernel
// reads 8 and writes 8 bytes per node from HBM.  Every wait on a copy is bounded: on a timeout
// the CTA stops, reports SL_ST_TIMEOUT, and drains its stores.
#include <algorithm>

#include "ffloat.cuh"
#include "sl_internal.h"

namespace sl {
namespace k1m {

constexpr int TILE = 256;                  // elements (threads) per tile
constexpr int WAIT_LIMIT = 1 << 22;        // polls of an mbarrier before a wait gives up

__device__ __forceinline__ int wrap_elem(int e, int K, bool periodic) {
  if (e >= 0 && e < K) return e;
  if (!periodic) return -1;
  e %= K;
  return e < 0 ? e + K : e;
}

// ---- bulk asynchronous copies (PTX cp.async.bulk) and mbarriers
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n"
      "  .reg .pred p;\n"
      "  mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "  selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// global -> shared, completion counted in bytes on bar; addresses and size multiples of 16 bytes
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

// shared -> global in the thread's bulk group; addresses and size multiples of 16 bytes
__device__ __forceinline__ void bulk_store(void* dst, const void* src, unsigned bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_addr(src)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// this thread's shared-memory writes become visible to later bulk copies (async proxy)
__device__ __forceinline__ void fence_to_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// floats of one plane of one stage: TILE + 1 rows, up to 3 floats of alignment shift, and the
// rounding of the copied run to 16 bytes at both ends
template <int NN>
__host__ __device__ constexpr int stage_floats() { return ((TILE + 1) * NN + 16 + 3) & ~3; }

// Where tile t's rows sit: rows r in [r_lo, r_hi) are elements first + r inside [0, K), one
// contiguous run of floats [g0, g1) of each plane, copied as the 16-byte-aligned window [a0, a1)
// to shared offset sbase; row r starts at shared offset sh + r NN.  sh in [0, 4) makes sbase a
// multiple of 4 floats.
struct TileGeo {
  int e0, first, r_lo, r_hi, sh, sbase, nvec;
  int64_t a0;
};

template <int NN>
__device__ __forceinline__ TileGeo tile_geo(const Mixed1DParams& P, int t) {
  TileGeo g;
  g.e0 = t * TILE;
  g.first = P.left_up ? g.e0 - 1 : g.e0;
  g.r_lo = max(0, -g.first);
  g.r_hi = min(TILE + 1, P.K - g.first);
  const int64_t g0 = (int64_t)(g.first + g.r_lo) * NN, g1 = (int64_t)(g.first + g.r_hi) * NN;
  g.a0 = g0 & ~int64_t(3);
  const int64_t a1 = (g1 + 3) & ~int64_t(3);   // within the plane: planes are padded to 64 floats
  const int d = (int)(g0 - g.a0);
  g.sh = (d - g.r_lo * NN) & 3;
  g.sbase = g.sh + g.r_lo * NN - d;
  g.nvec = (int)((a1 - g.a0) >> 2);
  return g;
}

// The outflow flux functional of one element's row: ref sum(f) + sum_i f_i ((hi_i - ref) + lo_i)
// with ref = hi_0, the same float operations whichever element evaluates it (the element itself or
// its downstream neighbour), so that both see the same number
template <int NN>
__device__ __forceinline__ float row_flux(const float* f, float sumf, const float* hi, const float* lo) {
  const float ref = hi[0];
  float acc = 0.0f;
#pragma unroll
  for (int i = 0; i < NN; ++i) acc = fmaf(f[i], __fadd_rn(__fsub_rn(hi[i], ref), lo[i]), acc);
  return fmaf(ref, sumf, acc);
}

// One element: rows own and up of the staged tile (shi, slo); writes res = phi^{n+1} - ref.
// Returns false when the energy iteration did not converge (the linear solution is kept).
template <int NN>
__device__ __forceinline__ bool element_step(const Mixed1DParams& P, const float* shi, const float* slo, int own,
                                             int up, bool has_up, float& ref, float (&res)[NN], ff& target) {
  bool ok = true;
  ref = shi[own];
  if (P.refine) {
    // M^{n+1} = M^n - lam (F_own - F_up) in float-float; the fluxes are exact floats by definition
    cdot mn;
#pragma unroll
    for (int i = 0; i < NN; ++i) mn.add(P.wh[i], P.wl[i], shi[own + i], slo[own + i]);
    const float fo = row_flux<NN>(P.Ff, P.sumf, shi + own, slo + own);
    const float fu = has_up ? row_flux<NN>(P.Ff, P.sumf, shi + up, slo + up) : (float)P.ghost * P.sumf;
    const ff net = two_sum(fo, -fu);
    target = ff_add(mn.get(), ff_neg(ff_mul(net, ff{P.lam, P.lam_lo})));
  }
  float ps[NN], pu[NN];
  if (has_up) {                             // own and upwind node i side by side (paired adds)
    const float2 mref = make_float2(-ref, -ref);
#pragma unroll
    for (int i = 0; i < NN; ++i) {
      const float2 d = __fadd2_rn(make_float2(shi[own + i], shi[up + i]), mref);
      const float2 v = __fadd2_rn(d, make_float2(slo[own + i], slo[up + i]));
      ps[i] = v.x;
      pu[i] = v.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < NN; ++i) ps[i] = (shi[own + i] - ref) + slo[own + i];
    const float g = (float)(P.ghost - (double)ref);   // ghost value at the inflow domain face
#pragma unroll
    for (int i = 0; i < NN; ++i) pu[i] = g;
  }
  // shared linear operator; rows 2p and 2p + 1 go through the paired FP32 FMA (each lane rounds
  // like fmaf and sums in the same order as a row on its own)
  float pl[NN];
#pragma unroll
  for (int pr = 0; pr < NN / 2; ++pr) {
    float2 acc = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int i = 0; i < NN; ++i) acc = __ffma2_rn(P.Gp[pr][i], make_float2(ps[i], ps[i]), acc);
#pragma unroll
    for (int i = 0; i < NN; ++i) acc = __ffma2_rn(P.Gp[pr][NN + i], make_float2(pu[i], pu[i]), acc);
    pl[2 * pr] = acc.x;
    pl[2 * pr + 1] = acc.y;
  }
  if (NN & 1) {
    constexpr int j = NN - 1;
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
        float2 eo = make_float2(0.0f, 0.0f);    // (own, upwind) basis sums, paired
#pragma unroll
        for (int i = 0; i < NN; ++i) eo = __ffma2_rn(make_float2(P.E[s][i], P.E[s][i]), make_float2(qs[i], qu[i]), eo);
        const float es = eo.x, eu = eo.y;
        gv = fmaf(P.lam * P.fb[s], es * es - eu * eu, gv);
        gm = fmaf(P.lam * P.fb[s], es - eu, gm);
      }
      const float gamma = P.mass_on ? gv : fmaf(2.0f * rf, gm, gv);
      if (fabsf(gamma) > (float)ENERGY_SKIP_RTOL_MIXED * escale) {
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
  return ok;
}

template <int NN>
__global__ void __launch_bounds__(TILE, NN <= 11 ? 3 : 2)
    k_step1d_mixed(const __grid_constant__ Mixed1DParams P, const float* __restrict__ in, float* __restrict__ out,
                   unsigned* status) {
  constexpr int SF = stage_floats<NN>();
  extern __shared__ __align__(16) float sm[];     // [stage][hi | lo][SF]
  __shared__ __align__(8) uint64_t bar[2];
  const int tid = threadIdx.x;
  const int K = P.K;
  const int64_t plane = P.plane;                  // float offset of the lo plane (multiple of 64)
  const int ntiles = (K + TILE - 1) / TILE;
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_init_fence();
  }
  __syncthreads();
  // thread 0: both planes of tile t into stage st
  auto issue = [&](int t, int st) {
    const TileGeo g = tile_geo<NN>(P, t);
    float* hi = sm + st * 2 * SF;
    const unsigned bytes = (unsigned)g.nvec * 16u;
    mbar_expect_tx(&bar[st], 2u * bytes);
    bulk_load(hi + g.sbase, in + g.a0, bytes, &bar[st]);
    bulk_load(hi + SF + g.sbase, in + plane + g.a0, bytes, &bar[st]);
  };
  if (tid == 0 && (int)blockIdx.x < ntiles) issue(blockIdx.x, 0);
  unsigned parity = 0;                            // bit st: phase parity awaited on stage st
  unsigned bits = 0;
  int st = 0;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x, st ^= 1) {
    // prefetch the next tile into the other stage once the stores that read it are done
    const int tn = t + (int)gridDim.x;
    if (tid == 0 && tn < ntiles) {
      bulk_wait_read_all();
      issue(tn, st ^ 1);
    }
    bool arrived = false;
    for (int it = 0; it < WAIT_LIMIT && !arrived; ++it) arrived = mbar_try_wait(&bar[st], (parity >> st) & 1u);
    if (__syncthreads_or(!arrived)) {             // every thread leaves together
      bits |= SL_ST_TIMEOUT;
      // the loads still in flight into this stage and into the prefetched one must land before
      // the CTA's shared memory is released: one more bounded wait on each (the output is left
      // incomplete either way)
      if (tid == 0) {
        bool done = false;
        for (int it = 0; it < WAIT_LIMIT && !done; ++it) done = mbar_try_wait(&bar[st], (parity >> st) & 1u);
        done = tn >= ntiles;
        for (int it = 0; it < WAIT_LIMIT && !done; ++it) done = mbar_try_wait(&bar[st ^ 1], (parity >> (st ^ 1)) & 1u);
      }
      __syncthreads();
      break;
    }
    parity ^= 1u << st;
    const TileGeo g = tile_geo<NN>(P, t);
    float* shi = sm + st * 2 * SF;
    float* slo = shi + SF;
    // the one halo row outside [0, K): periodic wrap, or zero at an inflow face (unused there)
    const int hrow = P.left_up ? 0 : g.r_hi;
    const bool hfix = P.left_up ? (g.r_lo == 1) : (g.r_hi <= TILE);
    if (hfix && tid < NN) {
      const int eh = wrap_elem(g.first + hrow, K, P.periodic != 0);
      shi[g.sh + hrow * NN + tid] = eh >= 0 ? in[(int64_t)eh * NN + tid] : 0.0f;
      slo[g.sh + hrow * NN + tid] = eh >= 0 ? in[plane + (int64_t)eh * NN + tid] : 0.0f;
    }
    __syncthreads();
    const int e = g.e0 + tid;
    const bool active = e < K;
    float res[NN];
    float ref = 0.0f;
    ff target = {0.0f, 0.0f};
    if (active) {
      const int own = g.sh + (P.left_up ? tid + 1 : tid) * NN;
      const int up = g.sh + (P.left_up ? tid : tid + 1) * NN;
      const bool has_up = wrap_elem(P.left_up ? e - 1 : e + 1, K, P.periodic != 0) >= 0;
      if (!element_step<NN>(P, shi, slo, own, up, has_up, ref, res, target)) bits |= SL_ST_PICARD_NOCONV;
    }
    __syncthreads();                              // the stage's rows are rewritten below
    if (active) {
      bool finite = true;
      // TwoSum: hi + lo == ref + res exactly; nodes j and j + 1 in paired operations
      // (a - b is formed as fma(b, -1, a), the same single rounding)
      float vh[NN], vl[NN];
      const float2 rr = make_float2(ref, ref), m1 = make_float2(-1.0f, -1.0f);
#pragma unroll
      for (int j = 0; j + 1 < NN; j += 2) {
        const float2 r = make_float2(res[j], res[j + 1]);
        const float2 s2 = __fadd2_rn(rr, r);
        const float2 bb = __ffma2_rn(rr, m1, s2);                  // s - ref
        const float2 t = __ffma2_rn(__ffma2_rn(bb, m1, s2), m1, rr);   // ref - (s - bb)
        const float2 err = __fadd2_rn(t, __ffma2_rn(bb, m1, r));    // + (res - bb)
        vh[j] = s2.x;
        vh[j + 1] = s2.y;
        vl[j] = err.x;
        vl[j + 1] = err.y;
      }
      if (NN & 1) {
        constexpr int j = NN - 1;
        const float s = ref + res[j];
        const float bb = s - ref;
        vh[j] = s;
        vl[j] = (ref - (s - bb)) + (res[j] - bb);
      }
      if (P.refine) {
        // float-float miss of the element mass, moved along the mass column into the lo words
        cdot mv;
#pragma unroll
        for (int i = 0; i < NN; ++i) mv.add(P.wh[i], P.wl[i], vh[i], vl[i]);
        const float miss = ff_to_f(ff_add(target, ff_neg(mv.get())));
#pragma unroll
        for (int j = 0; j < NN; ++j) {
          const ff v = fast_two_sum(vh[j], fmaf(miss, P.cmass[j], vl[j]));
          vh[j] = v.hi;
          vl[j] = v.lo;
        }
      }
#pragma unroll
      for (int j = 0; j < NN; ++j) {
        shi[tid * NN + j] = vh[j];
        slo[tid * NN + j] = vl[j];
        finite = finite && isfinite(vh[j]);
      }
      if (!finite) bits |= SL_ST_NONFINITE;
      fence_to_async();
    }
    __syncthreads();
    // the tile's own elements are one run starting at e0 NN (a multiple of 4 floats)
    const int nout = min(TILE, K - g.e0) * NN, nv = nout >> 2;
    if (tid == 0 && nv > 0) {
      bulk_store(out + (int64_t)g.e0 * NN, shi, (unsigned)nv * 16u);
      bulk_store(out + plane + (int64_t)g.e0 * NN, slo, (unsigned)nv * 16u);
      bulk_commit();
    }
    for (int idx = 4 * nv + tid; idx < nout; idx += TILE) {
      out[(int64_t)g.e0 * NN + idx] = shi[idx];
      out[plane + (int64_t)g.e0 * NN + idx] = slo[idx];
    }
    __syncthreads();                              // the stage is free once its stores have read it
  }
  if (tid == 0) bulk_wait_all();
  if (bits) atomicOr(status, bits);
}

template <int NN>
void launch_n(const Mixed1DParams& p, const float* in, float* out, unsigned* st, cudaStream_t s) {
  // persistent grid: resident CTAs per SM times the SM count (cached per device and kernel)
  constexpr size_t smem = (size_t)2 * 2 * stage_floats<NN>() * sizeof(float);
  const int cached_grid = persistent_grid((const void*)k_step1d_mixed<NN>, TILE, smem);
  const int ntiles = (p.K + TILE - 1) / TILE;
  k_step1d_mixed<NN><<<std::min(ntiles, cached_grid), TILE, smem, s>>>(p, in, out, st);
}

}  // namespace k1m
}  // namespace sl
