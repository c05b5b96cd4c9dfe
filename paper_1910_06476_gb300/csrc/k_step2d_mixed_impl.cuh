#pragma once
// 2D DSEM-SL step in mixed precision for any prescribed velocity (Sec. 4, two-dimensional scheme):
// particles seeded at the Gauss nodes and advected (eq. 4.4a), the collocation system eq. 5.4 solved for
// the remapped values, face traces (eq. 2dx/2dy_bnd_interpolate), upwinded interface values (eq. 4.12a),
// mass and energy targets (eq. 4.14, remap_mass, remap_energy) and the constrained fit (eq. matrix_a).
//
// State: double-float (hi + lo floats).  The bulk arithmetic is float on increments psi = phi - L
// relative to an element reference L, written back exactly, so float rounding scales with the
// variation inside the element:
//   - without the energy row L = r0 + gx (xi - 1/2) + gy (eta - 1/2) from the corner values, with the
//     energy row the constant r0.  L at a point is an exact float-float value (two-sum of r0 and the
//     once-rounded linear part), psi = (hi - L_hi) + (lo - L_lo) is therefore accurate relative to psi,
//     and the write-back L + psi is a float-float sum.  No FP64 instruction is used: this GPU's FP64
//     pipe runs at about 1/64 of the FP32 rate.
//   - Particles keep phi (divergence-free velocity), so the collocation data of psihat = phihat - L at a
//     particle displaced by d are psi - grad L . d.
//   - Mass: the element mass M^n = sum w (x) w (hi + lo) and each face's outflow flux G_f (outflow points
//     of the element, RK/Gauss quadrature at the backward characteristic feet, plus the ghost inflow on a
//     domain face) are float-float values.  An element's net outflow is its own G_f minus its
//     neighbours' G through the shared faces: every face flux enters two elements with opposite signs
//     as the same number, so global mass telescopes.  The fit itself works on float increments; one
//     refinement step then measures the element mass of the result in float-float and moves the
//     remaining miss along the pseudo-inverse column of the mass row into the lo word, which brings the
//     element mass to its target to about 1e-16 relative.
//   - Energy: target and mismatch from float increments (the energy row is decided at a 1e-9 relative
//     miss, its float resolution).
//
// Work layout: a group of G warps advances one element at a time (G = 1 up to n = 8, 5 at n = 17), two
// particles per thread (p0 = t, p1 = t + 32 G) with paired float operations across them where they
// share operands, several groups per CTA, each synchronising on its own named barrier (one warp:
// __syncwarp).  Reductions are butterflies (every lane gets the same bits) and, across the warps of a
// group, a fixed-order sum.  The kernels are persistent: group k of the grid walks the launch's elements
// k, k + groups, ...; per-group counters (solve and energy iterations, elements that stopped at the
// float floor or did not converge) are added to the context's counters once per group.
// Swirl velocity without transcendentals in the RK stages: sin and cos of pi x at the element's node
// and corner coordinates are taken once per element; at a displaced point they follow from the angle
// addition formulas, with the sine and cosine of the small angle pi h d from their Taylor series (used
// while h <= 1/4, so that |pi h d| <= pi / 4 where ten terms are exact to 1e-9; coarser meshes evaluate
// sinpi and cospi directly).  cos(pi t / T) is taken once per element at the stage-time fractions 0,
// 1/4, 1/2, 3/4, 1 of the step, which cover the RK schemes and their backward feet.
#include <type_traits>

#include "k_map2d.cuh"
#include "ffloat.cuh"

namespace sl {
namespace k2m {

// distinct stage times of the face-flux quadrature and their summed weights (RK4's two c = 1/2
// stages see the same face velocity and the same foot)
static __constant__ int c_ds_n[5] = {0, 1, 2, 3, 3};
static __constant__ float c_ds_c[5][3] = {{}, {0.0f}, {0.0f, 1.0f}, {0.0f, 0.5f, 1.0f}, {0.0f, 0.5f, 1.0f}};
static __constant__ float c_ds_b[5][3] = {
    {}, {1.0f}, {0.5f, 0.5f}, {1.0f / 6, 2.0f / 3, 1.0f / 6}, {1.0f / 6, 1.0f / 3 + 1.0f / 3, 1.0f / 6}};

constexpr int SOLVE_CAP = 40;
constexpr float SOLVE_RTOL = 3e-7f;          // target, relative to max |psi*|
constexpr float SOLVE_STALL = 4e-6f;         // a residual that stops improving below this is the float floor
constexpr float SOLVE_FLOOR = 1e-4f;         // best residual accepted (SL_ST_SOLVE_FLOOR) above the floor

// asynchronous 4-byte global-to-shared copies (the next element's inputs are staged while the current
// one is computed); a thread waits for its own copies, a group barrier then publishes them
__device__ __forceinline__ void cp_async4(float* smem, const float* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// element reference L at reference coordinates given as (a, b) = (xi - 1/2, eta - 1/2): the linear
// part is rounded once, L = r0 + t exactly as a float-float value.  Every use runs this same
// instruction sequence, so both kernels agree on L bit for bit.
__device__ __forceinline__ ff lref(float r0, float gx, float gy, float a, float b) {
  const float t = fmaf(gx, a, __fmul_rn(gy, b));
  return two_sum(r0, t);
}

// ------------------------------------------------------------------ groups of warps
template <int NN>
struct Shape {
  static constexpr int ND = NN * NN;
  static constexpr int G = (ND + 63) / 64;                 // warps per element
  static constexpr int GT = 32 * G;                        // threads per element
  static constexpr int EPC = G == 1 ? 8 : G == 2 ? 4 : G <= 4 ? 2 : 1;   // element groups per CTA
  static constexpr int NT = GT * EPC;
  static constexpr int NP = (NN + 3) & ~3;                 // row stride of psihat and psi^n (16 bytes)
  static constexpr int RS = NN | 1;                        // odd row stride of the preconditioner rows
  static constexpr int MINB = NN <= 12 ? 2 : 1;            // resident CTAs asked of the compiler: phase 1
  static constexpr int MINB2 = NN <= 8 ? 3 : NN <= 12 ? 2 : 1;   // phase 2 (measured: 3 beats 2 at n = 8)
};

template <int G>
struct Grp {
  int t, lane, w, slot;
  float* red;                                              // 4 G floats: two buffers of a pair per warp
  int rb;
  __device__ __forceinline__ void sync() const {
    if (G == 1) __syncwarp();
    else asm volatile("bar.sync %0, %1;" ::"r"(1 + slot), "r"(32 * G) : "memory");
  }
  // Cross-warp sums alternate between two scratch buffers: a buffer is rewritten two reductions
  // later, after every warp has passed the barrier of the reduction in between.
  __device__ __forceinline__ float sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (G == 1) return v;
    float* r = red + rb * 2 * G;
    rb ^= 1;
    if (lane == 0) r[w] = v;
    sync();
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < G; ++k) s += r[k];
    return s;
  }
  __device__ __forceinline__ float2 sum2(float a, float b) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (G == 1) return make_float2(a, b);
    float* r = red + rb * 2 * G;
    rb ^= 1;
    if (lane == 0) { r[w] = a; r[G + w] = b; }
    sync();
    float sa = 0.0f, sb = 0.0f;
#pragma unroll
    for (int k = 0; k < G; ++k) { sa += r[k]; sb += r[G + k]; }
    return make_float2(sa, sb);
  }
  __device__ __forceinline__ float max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (G == 1) return v;
    float* r = red + rb * 2 * G;
    rb ^= 1;
    if (lane == 0) r[w] = v;
    sync();
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < G; ++k) s = fmaxf(s, r[k]);
    return s;
  }
  __device__ __forceinline__ ff ffsum(ff v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ff u;
      u.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
      u.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
      v = ff_add(v, u);
    }
    if (G == 1) return v;
    float* r = red + rb * 2 * G;
    rb ^= 1;
    if (lane == 0) { r[w] = v.hi; r[G + w] = v.lo; }
    sync();
    ff s = {r[0], r[G]};
#pragma unroll
    for (int k = 1; k < G; ++k) s = ff_add(s, ff{r[k], r[G + k]});
    return s;
  }
};

// ------------------------------------------------------------------ velocity
// sine and cosine of a small angle by their Taylor series: five terms each (exact to 1e-9 for
// |x| <= pi / 4), or three when |x| <= 0.02 (the remainders x^7 / 7! and x^6 / 6! are then below
// 1e-13)
__device__ __forceinline__ void small_sincos(float x, bool shortser, float& s, float& c) {
  const float x2 = x * x;
  if (shortser) {
    s = fmaf(x * x2, fmaf(x2, 1.0f / 120.0f, -1.0f / 6.0f), x);
    c = fmaf(x2, fmaf(x2, 1.0f / 24.0f, -0.5f), 1.0f);
    return;
  }
  float ps = fmaf(x2, 1.0f / 362880.0f, -1.0f / 5040.0f);
  ps = fmaf(x2, ps, 1.0f / 120.0f);
  ps = fmaf(x2, ps, -1.0f / 6.0f);
  s = fmaf(x * x2, ps, x);
  float pc = fmaf(x2, -1.0f / 3628800.0f, 1.0f / 40320.0f);
  pc = fmaf(x2, pc, -1.0f / 720.0f);
  pc = fmaf(x2, pc, 1.0f / 24.0f);
  pc = fmaf(x2, pc, -0.5f);
  c = fmaf(x2, pc, 1.0f);
}

// paired float operations
__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

__device__ __forceinline__ void small_sincos2(float2 x, bool shortser, float2& s, float2& c) {
  const float2 x2 = mul2(x, x);
  if (shortser) {
    s = fma2(mul2(x, x2), fma2(x2, bc2(1.0f / 120.0f), bc2(-1.0f / 6.0f)), x);
    c = fma2(x2, fma2(x2, bc2(1.0f / 24.0f), bc2(-0.5f)), bc2(1.0f));
    return;
  }
  float2 ps = fma2(x2, bc2(1.0f / 362880.0f), bc2(-1.0f / 5040.0f));
  ps = fma2(x2, ps, bc2(1.0f / 120.0f));
  ps = fma2(x2, ps, bc2(-1.0f / 6.0f));
  s = fma2(mul2(x, x2), ps, x);
  float2 pc = fma2(x2, bc2(-1.0f / 3628800.0f), bc2(1.0f / 40320.0f));
  pc = fma2(x2, pc, bc2(-1.0f / 720.0f));
  pc = fma2(x2, pc, bc2(1.0f / 24.0f));
  pc = fma2(x2, pc, bc2(-0.5f));
  c = fma2(x2, pc, bc2(1.0f));
}

// The velocity of one element divided by its size (the time derivative of the reference
// coordinates).  A point is given by its base reference coordinates (bx, by), the sine and cosine of
// pi times the base's physical coordinates (swirl), and a displacement (dx, dy) in reference units;
// ct = cos(pi tau / T) at the stage time.
struct VelElem {
  int kind;
  bool direct;                   // evaluate sinpi/cospi at the point itself (coarse meshes)
  bool shortser;                 // pi h <= 0.02: three-term series for the small angle
  float x0, y0, hx, hy, ihx, ihy, pihx, pihy;
  float a, b, om, cx, cy;
};

__device__ __forceinline__ void vel_at(const VelElem& V, float bx, float by, float Sx, float Cx, float Sy, float Cy,
                                       float dx, float dy, float ct, float& u, float& v) {
  switch (V.kind) {
    case SL_VEL_ROTATION: {
      const float x = fmaf(V.hx, bx + dx, V.x0), y = fmaf(V.hy, by + dy, V.y0);
      u = -V.om * (y - V.cy) * V.ihx;
      v = V.om * (x - V.cx) * V.ihy;
      break;
    }
    case SL_VEL_SWIRL: {
      float sx, cx, sy, cy;
      if (V.direct) {
        sincospif(fmaf(V.hx, bx + dx, V.x0), &sx, &cx);
        sincospif(fmaf(V.hy, by + dy, V.y0), &sy, &cy);
      } else {
        float st, ctt;
        small_sincos(V.pihx * dx, V.shortser, st, ctt);
        sx = fmaf(Sx, ctt, Cx * st);
        cx = fmaf(Cx, ctt, -Sx * st);
        small_sincos(V.pihy * dy, V.shortser, st, ctt);
        sy = fmaf(Sy, ctt, Cy * st);
        cy = fmaf(Cy, ctt, -Sy * st);
      }
      // sin(2 pi y) = 2 sin(pi y) cos(pi y)
      u = sx * sx * (2.0f * sy * cy) * ct * V.ihx;
      v = -sy * sy * (2.0f * sx * cx) * ct * V.ihy;
      break;
    }
    default:
      u = V.a * V.ihx;
      v = V.b * V.ihy;
  }
}

// Butcher tableaux of the explicit RK schemes of orders 1-4 (forward Euler, Heun, Kutta's third
// order, classical), as compile-time functions so that the coefficients become immediates
template <int RK>
struct Tab {
  static constexpr int S = RK;
  __device__ static constexpr float a(int s, int j) {
    return RK == 2 ? (s == 1 && j == 0 ? 1.0f : 0.0f)
         : RK == 3 ? (s == 1 && j == 0 ? 0.5f : s == 2 && j == 0 ? -1.0f : s == 2 && j == 1 ? 2.0f : 0.0f)
         : RK == 4 ? ((s == 1 && j == 0) || (s == 2 && j == 1) ? 0.5f : s == 3 && j == 2 ? 1.0f : 0.0f)
                   : 0.0f;
  }
  __device__ static constexpr float b(int s) {
    return RK == 1 ? 1.0f
         : RK == 2 ? 0.5f
         : RK == 3 ? (s == 1 ? 2.0f / 3.0f : 1.0f / 6.0f)
                   : (s == 0 || s == 3 ? 1.0f / 6.0f : 1.0f / 3.0f);
  }
  __device__ static constexpr float c(int s) {
    return RK == 2 ? (s == 1 ? 1.0f : 0.0f)
         : RK == 3 ? (s == 1 ? 0.5f : s == 2 ? 1.0f : 0.0f)
         : RK == 4 ? (s == 1 || s == 2 ? 0.5f : s == 3 ? 1.0f : 0.0f)
                   : 0.0f;
  }
};

// One RK step of the displacement (dx, dy) of a point over a time step h (negative: backward), the
// stage time of stage s being the step fraction f0 + c_s fstep (one of 0, 1/4, 1/2, 3/4, 1, whose
// cos(pi tau / T) are ctab[0..4]).  The displacement is integrated by itself (not the position), so
// that its float rounding is relative to the displacement.
// velocity of the swirl at a displaced point from the tabulated sines (angle addition)
__device__ __forceinline__ void vel_swirl_tab(const VelElem& V, float Sx, float Cx, float Sy, float Cy, float dx,
                                              float dy, float ct, float& u, float& v) {
  float st, ctt;
  small_sincos(V.pihx * dx, V.shortser, st, ctt);
  const float sx = fmaf(Sx, ctt, Cx * st), cx = fmaf(Cx, ctt, -Sx * st);
  small_sincos(V.pihy * dy, V.shortser, st, ctt);
  const float sy = fmaf(Sy, ctt, Cy * st), cy = fmaf(Cy, ctt, -Sy * st);
  u = sx * sx * (2.0f * sy * cy) * ct * V.ihx;
  v = -sy * sy * (2.0f * sx * cx) * ct * V.ihy;
}

// TAB: the velocity is the swirl from the tabulated sines (chosen once per element)
template <int RK, bool TAB>
__device__ __forceinline__ void rk_disp_t(const VelElem& V, float bx, float by, float Sx, float Cx, float Sy, float Cy,
                                          float& dx, float& dy, float h, float f0, float fstep, const float* ctab) {
  using T = Tab<RK>;
  float kx[T::S], ky[T::S];
#pragma unroll
  for (int s = 0; s < T::S; ++s) {
    float xs = dx, ys = dy;
#pragma unroll
    for (int j = 0; j < s; ++j)
      if (T::a(s, j) != 0.0f) {
        xs = fmaf(h * T::a(s, j), kx[j], xs);
        ys = fmaf(h * T::a(s, j), ky[j], ys);
      }
    const int ci = __float2int_rn(4.0f * fmaf(T::c(s), fstep, f0));
    if (TAB) vel_swirl_tab(V, Sx, Cx, Sy, Cy, xs, ys, ctab[ci], kx[s], ky[s]);
    else vel_at(V, bx, by, Sx, Cx, Sy, Cy, xs, ys, ctab[ci], kx[s], ky[s]);
  }
  float sx = 0.0f, sy = 0.0f;
#pragma unroll
  for (int s = 0; s < T::S; ++s) {
    sx = fmaf(T::b(s), kx[s], sx);
    sy = fmaf(T::b(s), ky[s], sy);
  }
  dx = fmaf(h, sx, dx);
  dy = fmaf(h, sy, dy);
}

__device__ __forceinline__ void rk_disp(const VelElem& V, int rk, float bx, float by, float Sx, float Cx, float Sy,
                                        float Cy, float& dx, float& dy, float h, float f0, float fstep,
                                        const float* ctab) {
  if (rk == 4 && V.kind == SL_VEL_SWIRL && !V.direct) {
    rk_disp_t<4, true>(V, bx, by, Sx, Cx, Sy, Cy, dx, dy, h, f0, fstep, ctab);
    return;
  }
  switch (rk) {
    case 4: rk_disp_t<4, false>(V, bx, by, Sx, Cx, Sy, Cy, dx, dy, h, f0, fstep, ctab); break;
    case 3: rk_disp_t<3, false>(V, bx, by, Sx, Cx, Sy, Cy, dx, dy, h, f0, fstep, ctab); break;
    case 2: rk_disp_t<2, false>(V, bx, by, Sx, Cx, Sy, Cy, dx, dy, h, f0, fstep, ctab); break;
    default: rk_disp_t<1, false>(V, bx, by, Sx, Cx, Sy, Cy, dx, dy, h, f0, fstep, ctab);
  }
}

// vel_at at two points at once (paired float operations; the direct evaluation per component)
__device__ __forceinline__ void vel_at2(const VelElem& V, float2 bx, float2 by, float2 Sx, float2 Cx, float2 Sy,
                                        float2 Cy, float2 dx, float2 dy, float ct, float2& u, float2& v) {
  switch (V.kind) {
    case SL_VEL_ROTATION: {
      const float2 x = fma2(bc2(V.hx), add2(bx, dx), bc2(V.x0)), y = fma2(bc2(V.hy), add2(by, dy), bc2(V.y0));
      u = mul2(bc2(-V.om * V.ihx), add2(y, bc2(-V.cy)));
      v = mul2(bc2(V.om * V.ihy), add2(x, bc2(-V.cx)));
      break;
    }
    case SL_VEL_SWIRL: {
      float2 sx, cx, sy, cy;
      if (V.direct) {
        sincospif(fmaf(V.hx, bx.x + dx.x, V.x0), &sx.x, &cx.x);
        sincospif(fmaf(V.hx, bx.y + dx.y, V.x0), &sx.y, &cx.y);
        sincospif(fmaf(V.hy, by.x + dy.x, V.y0), &sy.x, &cy.x);
        sincospif(fmaf(V.hy, by.y + dy.y, V.y0), &sy.y, &cy.y);
      } else {
        float2 st, ctt;
        small_sincos2(mul2(bc2(V.pihx), dx), V.shortser, st, ctt);
        sx = fma2(Sx, ctt, mul2(Cx, st));
        cx = fma2(Cx, ctt, mul2(neg2(Sx), st));
        small_sincos2(mul2(bc2(V.pihy), dy), V.shortser, st, ctt);
        sy = fma2(Sy, ctt, mul2(Cy, st));
        cy = fma2(Cy, ctt, mul2(neg2(Sy), st));
      }
      u = mul2(mul2(sx, sx), mul2(mul2(sy, cy), bc2(2.0f * ct * V.ihx)));
      v = mul2(mul2(sy, sy), mul2(mul2(sx, cx), bc2(-2.0f * ct * V.ihy)));
      break;
    }
    default:
      u = bc2(V.a * V.ihx);
      v = bc2(V.b * V.ihy);
  }
}

// rk_disp for two points at once (paired float operations)
template <int RK, bool TAB>
__device__ __forceinline__ void rk_disp2_t(const VelElem& V, float2 bx, float2 by, float2 Sx, float2 Cx, float2 Sy,
                                           float2 Cy, float2& dx, float2& dy, float h, const float* ctab) {
  using T = Tab<RK>;
  float2 kx[T::S], ky[T::S];
#pragma unroll
  for (int s = 0; s < T::S; ++s) {
    float2 xs = dx, ys = dy;
#pragma unroll
    for (int j = 0; j < s; ++j)
      if (T::a(s, j) != 0.0f) {
        const float2 hj = bc2(h * T::a(s, j));
        xs = fma2(hj, kx[j], xs);
        ys = fma2(hj, ky[j], ys);
      }
    const float ct = ctab[__float2int_rn(4.0f * T::c(s))];
    if (TAB) {
      float2 st, ctt;
      small_sincos2(mul2(bc2(V.pihx), xs), V.shortser, st, ctt);
      const float2 sx = fma2(Sx, ctt, mul2(Cx, st)), cx = fma2(Cx, ctt, mul2(neg2(Sx), st));
      small_sincos2(mul2(bc2(V.pihy), ys), V.shortser, st, ctt);
      const float2 sy = fma2(Sy, ctt, mul2(Cy, st)), cy = fma2(Cy, ctt, mul2(neg2(Sy), st));
      kx[s] = mul2(mul2(sx, sx), mul2(mul2(sy, cy), bc2(2.0f * ct * V.ihx)));
      ky[s] = mul2(mul2(sy, sy), mul2(mul2(sx, cx), bc2(-2.0f * ct * V.ihy)));
    } else {
      vel_at2(V, bx, by, Sx, Cx, Sy, Cy, xs, ys, ct, kx[s], ky[s]);
    }
  }
  float2 sx = bc2(0.0f), sy = bc2(0.0f);
#pragma unroll
  for (int s = 0; s < T::S; ++s) {
    sx = fma2(bc2(T::b(s)), kx[s], sx);
    sy = fma2(bc2(T::b(s)), ky[s], sy);
  }
  dx = fma2(bc2(h), sx, dx);
  dy = fma2(bc2(h), sy, dy);
}

// forward step over the whole step h = dt from t^n
__device__ __forceinline__ void rk_disp2(const VelElem& V, int rk, float2 bx, float2 by, float2 Sx, float2 Cx,
                                         float2 Sy, float2 Cy, float2& dx, float2& dy, float h, const float* ctab) {
  if (rk == 4 && V.kind == SL_VEL_SWIRL && !V.direct) {
    rk_disp2_t<4, true>(V, bx, by, Sx, Cx, Sy, Cy, dx, dy, h, ctab);
    return;
  }
  switch (rk) {
    case 4: rk_disp2_t<4, false>(V, bx, by, Sx, Cx, Sy, Cy, dx, dy, h, ctab); break;
    case 3: rk_disp2_t<3, false>(V, bx, by, Sx, Cx, Sy, Cy, dx, dy, h, ctab); break;
    case 2: rk_disp2_t<2, false>(V, bx, by, Sx, Cx, Sy, Cy, dx, dy, h, ctab); break;
    default: rk_disp2_t<1, false>(V, bx, by, Sx, Cx, Sy, Cy, dx, dy, h, ctab);
  }
}

// velocity at a base point itself (no displacement): the tabulated sines and cosines directly
__device__ __forceinline__ void vel_base(const VelElem& V, float bx, float by, float Sx, float Cx, float Sy, float Cy,
                                         float ct, float& u, float& v) {
  if (V.kind == SL_VEL_SWIRL && !V.direct) {
    u = Sx * Sx * (2.0f * Sy * Cy) * ct * V.ihx;
    v = -Sy * Sy * (2.0f * Sx * Cx) * ct * V.ihy;
  } else {
    vel_at(V, bx, by, Sx, Cx, Sy, Cy, 0.0f, 0.0f, ct, u, v);
  }
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

// the same at two points at once, in paired float operations (same rounding per point)
template <int NN>
__device__ __forceinline__ void basis_at2(const float* xi, const float* lam, float z0a, float z0b, float dza, float dzb,
                                          float2* out) {
  float2 d[NN], pre[NN];
  const float2 dz = make_float2(dza, dzb);
#pragma unroll
  for (int k = 0; k < NN; ++k) d[k] = __fadd2_rn(make_float2(z0a - xi[k], z0b - xi[k]), dz);
  float2 acc = make_float2(1.0f, 1.0f);
#pragma unroll
  for (int k = 0; k < NN; ++k) { pre[k] = acc; acc = __fmul2_rn(acc, d[k]); }
  float2 suf = make_float2(1.0f, 1.0f);
#pragma unroll
  for (int l = NN - 1; l >= 0; --l) {
    out[l] = __fmul2_rn(__fmul2_rn(make_float2(lam[l], lam[l]), pre[l]), suf);
    suf = __fmul2_rn(suf, d[l]);
  }
}

// sum_l row[l] b[l] for two vectors b at once (paired FMAs), row 16-byte aligned with NN values
template <int NN>
__device__ __forceinline__ float2 row_dot2(const float* row, const float2 (&b)[NN]) {
  const float4* rowp = reinterpret_cast<const float4*>(row);
  float2 r = make_float2(0.0f, 0.0f);
#pragma unroll
  for (int q = 0; q < (NN + 3) / 4; ++q) {
    const float4 v = rowp[q];
    if (4 * q + 0 < NN) r = __ffma2_rn(make_float2(v.x, v.x), b[(4 * q + 0) % NN], r);
    if (4 * q + 1 < NN) r = __ffma2_rn(make_float2(v.y, v.y), b[(4 * q + 1) % NN], r);
    if (4 * q + 2 < NN) r = __ffma2_rn(make_float2(v.z, v.z), b[(4 * q + 2) % NN], r);
    if (4 * q + 3 < NN) r = __ffma2_rn(make_float2(v.w, v.w), b[(4 * q + 3) % NN], r);
  }
  return r;
}

// sum_l row[l] b[l] for one vector b: even and odd columns in the two lanes of paired FMAs
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

// per-problem float parameters of a batch element (the FP64 geometry is already in P)
__device__ __forceinline__ void batch_extra(const StepParams& P, const Map2D& M, Mixed2DExtra& X) {
  if (!M.geo) return;
  X.hx = (float)P.hx;
  X.hy = (float)P.hy;
  X.ihx = (float)(1.0 / P.hx);
  X.ihy = (float)(1.0 / P.hy);
  X.dt = (float)P.dt;
  const double lam = P.dt / (P.hx * P.hy);
  X.dt_area = (float)lam;
  X.lam_hi = (float)lam;
  X.lam_lo = (float)(lam - (double)X.lam_hi);
  if (X.Tper != 0.0) {
    X.tT = (float)(P.t / X.Tper);
    X.dtT = (float)(P.dt / X.Tper);
  }
}

__device__ __forceinline__ int nb_index(const StepParams& P, int ex, int ey, int face) {
  int jx = ex + (face == 0 ? -1 : face == 1 ? 1 : 0);
  int jy = ey + (face == 2 ? -1 : face == 3 ? 1 : 0);
  if (jx >= 0 && jx < P.kx && jy >= 0 && jy < P.ky) return jy * P.kx + jx;
  // the face's boundary condition by selection (a dynamic index would put P in local memory)
  const int bc = face == 0 ? P.bc[0] : face == 1 ? P.bc[1] : face == 2 ? P.bc[2] : P.bc[3];
  if (bc != SL_BC_PERIODIC) return -1;
  jx = (jx + P.kx) % P.kx;
  jy = (jy + P.ky) % P.ky;
  return jy * P.kx + jx;
}

// the element of launch-list index k; copies its problem's geometry and step into P (batches)
template <int NN>
__device__ __forceinline__ Elem elem_at(StepParams& P, const Map2D& M, int64_t k) {
  Elem E;
  E.g = M.list ? (int64_t)M.list[k] : k;
  E.gb = 0;
  if (M.geo) {
    const ProbGeom& G = M.geo[M.prob[E.g]];
    P.kx = G.kx;
    P.ky = G.ky;
    for (int f = 0; f < 4; ++f) P.bc[f] = G.bc[f];
    P.x0 = G.x0;
    P.hx = G.hx;
    P.y0 = G.y0;
    P.hy = G.hy;
    P.ghost = G.ghost;
    P.t = G.t;
    P.dt = G.dt;
    E.gb = G.gbase;
  }
  E.e = (int)(E.g - E.gb);
  E.ex = E.e % P.kx;
  E.ey = E.e / P.kx;
  E.base = M.off ? M.off[E.g] : E.g * (NN * NN);
  return E;
}

__device__ __forceinline__ VelElem make_vel(const StepParams& P, const Mixed2DExtra& X, float x0, float y0) {
  VelElem V;
  V.kind = P.vel_kind;
  V.x0 = x0;
  V.y0 = y0;
  V.hx = X.hx;
  V.hy = X.hy;
  V.ihx = X.ihx;
  V.ihy = X.ihy;
  V.pihx = 3.14159265358979f * X.hx;
  V.pihy = 3.14159265358979f * X.hy;
  V.direct = !(X.hx <= 0.25f && X.hy <= 0.25f);
  V.shortser = V.pihx <= 0.02f && V.pihy <= 0.02f;
  V.a = X.a;
  V.b = X.b;
  V.om = X.om;
  V.cx = X.cx;
  V.cy = X.cy;
  return V;
}

// Per-element sines and cosines of the swirl: sin and cos of pi x at the node x-coordinates n[0],
// n[1], y-coordinates n[2], n[3]; at the corner coordinates x0, x0 + hx, y0, y0 + hy (sines in
// corner[0..3], cosines in corner[4..7]); ct[k] = cos(pi (t + k dt / 4) / T).
template <int NN>
struct Trig {
  float n[4][NN];
  float corner[8];
  float ct[5];
};

template <int NN, int G>
__device__ __forceinline__ void trig_setup(const Grp<G>& g, const VelElem& V, const Mixed2DExtra& X, const float* xi,
                                           Trig<NN>& T) {
  const int t = g.t;
  if (V.kind == SL_VEL_SWIRL) {
    if (t < NN) sincospif(fmaf(V.hx, xi[t], V.x0), &T.n[0][t], &T.n[1][t]);
    else if (t < 2 * NN) sincospif(fmaf(V.hy, xi[t - NN], V.y0), &T.n[2][t - NN], &T.n[3][t - NN]);
    else if (t < 2 * NN + 4) {
      const int k = t - 2 * NN;
      const float z = k < 2 ? V.x0 + (k == 1 ? V.hx : 0.0f) : V.y0 + (k == 3 ? V.hy : 0.0f);
      sincospif(z, &T.corner[k], &T.corner[4 + k]);
    } else if (t < 2 * NN + 9) {
      const int k = t - 2 * NN - 4;
      T.ct[k] = cospif(fmaf(0.25f * (float)k, X.dtT, X.tT));
    }
  } else if (t < 5) {
    T.ct[t] = 1.0f;
  }
}

// ------------------------------------------------------------------ phase 1
template <int NN>
struct Smem1 {
  static constexpr int ND = Shape<NN>::ND, NP = Shape<NN>::NP, RS = Shape<NN>::RS, G = Shape<NN>::G;
  __align__(16) float ph[NN * NP];             // psihat rows
  __align__(16) float psi[NN * NP];            // psi^n rows
  union {
    struct {                                   // the collocation solve
      float r[ND], tt[ND], best[ND];
      float Rx[NN * RS], Ry[NN * RS];
    } sv;
    struct {                                   // the face outflow, after the solve
      float fbo[4][NMAX][3], fbi[4][NMAX][3];  // per face point and distinct stage: outflow, inflow weight
      float fv[4][NMAX][3];                    //   and the outflow value (phi - r0)
      float pt[4][NMAX][4];                    // per face point: U_out, U_in, P1, P2 over the step
      float fs[4][4];                          // per face: the same summed over its points
      int items[4 * NMAX * 2];                 // outflow (point, stage) pairs that need a foot
    } fc;
  } u;
  float red[4 * G];
  int cum[5];
  int nitems;
  Trig<NN> T;
  float sth[2][ND], stl[2][ND];                // staged input state (hi, lo) of this and the next element
};

template <int NN>
__global__ void __launch_bounds__(Shape<NN>::NT, Shape<NN>::MINB)
    k_p1(StepParams P0, const __grid_constant__ Mixed2DExtra X0, Map2D M, int64_t count, const float* __restrict__ in,
         Work2M W, unsigned* status) {
  using S = Shape<NN>;
  constexpr int ND = S::ND, NP = S::NP, RS = S::RS, G = S::G, GT = S::GT, EPC = S::EPC;
  __shared__ float s_xi[NN], s_lam[NN], s_w[NN], s_l0[NN], s_l1[NN];
  __shared__ Smem1<NN> sm_all[EPC];
  if (threadIdx.x < NN) {
    s_xi[threadIdx.x] = X0.xi[threadIdx.x];
    s_lam[threadIdx.x] = X0.lam[threadIdx.x];
    s_w[threadIdx.x] = X0.w[threadIdx.x];
    s_l0[threadIdx.x] = X0.l0[threadIdx.x];
    s_l1[threadIdx.x] = X0.l1[threadIdx.x];
  }
  __syncthreads();
  Grp<G> g;
  g.slot = threadIdx.x / GT;
  g.t = threadIdx.x % GT;
  g.lane = threadIdx.x & 31;
  g.w = g.t >> 5;
  Smem1<NN>& sm = sm_all[g.slot];
  g.red = sm.red;
  g.rb = 0;
  const int t = g.t;
  const int p0 = t, p1 = t + GT;
  const bool v0 = p0 < ND, v1 = p1 < ND;
  const int i0 = p0 % NN, j0 = (p0 / NN) % NN, i1 = p1 % NN, j1 = (p1 / NN) % NN;
  unsigned long long c_it = 0, c_floor = 0, c_nc = 0, c_feet = 0;
  unsigned bits = 0;
  const int64_t ngroups = (int64_t)gridDim.x * EPC;
  // asynchronous copies of element kk's input state into staging buffer b (one group per call)
  auto stage = [&](int64_t kk, int b) {
    if (kk < count) {
      StepParams Pn = P0;
      const Elem En = elem_at<NN>(Pn, M, kk);
      if (v0) { cp_async4(&sm.sth[b][p0], in + En.base + p0); cp_async4(&sm.stl[b][p0], in + X0.plane + En.base + p0); }
      if (v1) { cp_async4(&sm.sth[b][p1], in + En.base + p1); cp_async4(&sm.stl[b][p1], in + X0.plane + En.base + p1); }
    }
    cp_async_commit();
  };
  int64_t k = (int64_t)blockIdx.x * EPC + g.slot;
  stage(k, 0);
  for (int b = 0; k < count; k += ngroups, b ^= 1) {
    g.sync();                                    // the previous element's shared data is consumed
    stage(k + ngroups, b ^ 1);
    cp_async_wait1();
    StepParams P = P0;
    const Elem E = elem_at<NN>(P, M, k);
    Mixed2DExtra X = X0;
    batch_extra(P, M, X);
    const int ex = E.ex, ey = E.ey;
    const float x0 = (float)(P.x0 + ex * P.hx), y0 = (float)(P.y0 + ey * P.hy);
    const VelElem V = make_vel(P, X, x0, y0);
    trig_setup<NN>(g, V, X, s_xi, sm.T);
    g.sync();                                    // this element's staged state is visible
    const float* sh = sm.sth[b];
    const float* sl = sm.stl[b];
    // element reference: linear from the four corner values, or the first node value
    const float c00 = sh[0], c01 = sh[NN - 1], c10 = sh[(NN - 1) * NN], c11 = sh[ND - 1];
    float r0 = c00, gx = 0.0f, gy = 0.0f;
    if (X.linref) {
      r0 = 0.25f * ((c00 + c01) + (c10 + c11));
      gx = ((c01 + c11) - (c00 + c10)) * X.span;
      gy = ((c10 + c11) - (c00 + c01)) * X.span;
    }
    // psi^n at the own nodes, and the element mass in float-float
    float pn0 = 0.0f, pn1 = 0.0f;
    ff mn = {0.0f, 0.0f};
    if (v0) {
      const float hi = sh[p0], lo = sl[p0];
      const ff L = lref(r0, gx, gy, s_xi[i0] - 0.5f, s_xi[j0] - 0.5f);
      pn0 = __fadd_rn(__fsub_rn(hi, L.hi), __fsub_rn(lo, L.lo));
      sm.psi[j0 * NP + i0] = pn0;
      mn = ff_mul(ff{hi, lo}, ff{X.w2h[p0], X.w2l[p0]});
    }
    if (v1) {
      const float hi = sh[p1], lo = sl[p1];
      const ff L = lref(r0, gx, gy, s_xi[i1] - 0.5f, s_xi[j1] - 0.5f);
      pn1 = __fadd_rn(__fsub_rn(hi, L.hi), __fsub_rn(lo, L.lo));
      sm.psi[j1 * NP + i1] = pn1;
      mn = ff_add(mn, ff_mul(ff{hi, lo}, ff{X.w2h[p1], X.w2l[p1]}));
    }
    g.sync();
    // advect the particles of nodes p0, p1 in reference coordinates
    float2 d2x = bc2(0.0f), d2y = bc2(0.0f);
    rk_disp2(V, P.rk, make_float2(s_xi[i0], s_xi[i1]), make_float2(s_xi[j0], s_xi[j1]),
             make_float2(sm.T.n[0][i0], sm.T.n[0][i1]), make_float2(sm.T.n[1][i0], sm.T.n[1][i1]),
             make_float2(sm.T.n[2][j0], sm.T.n[2][j1]), make_float2(sm.T.n[3][j0], sm.T.n[3][j1]), d2x, d2y, X.dt,
             sm.T.ct);
    const float dx0 = v0 ? d2x.x : 0.0f, dy0 = v0 ? d2y.x : 0.0f, dx1 = v1 ? d2x.y : 0.0f, dy1 = v1 ? d2y.y : 0.0f;
    float2 Lx[NN], Ly[NN];
    basis_at2<NN>(s_xi, s_lam, s_xi[i0], s_xi[i1], dx0, dx1, Lx);
    basis_at2<NN>(s_xi, s_lam, s_xi[j0], s_xi[j1], dy0, dy1, Ly);
    // collocation data of psihat = phihat - L
    const float ps0 = v0 ? pn0 - fmaf(gx, dx0, gy * dy0) : 0.0f;
    const float ps1 = v1 ? pn1 - fmaf(gx, dx1, gy * dy1) : 0.0f;
    const float2 md = g.sum2(dx0 + dx1, dy0 + dy1);
    const float mdx = md.x / ND, mdy = md.y / ND;
    // preconditioner: interpolation back over the mean displacement, Rx[i][q] = l_q(xi_i - mdx)
    if (t < 2 * NN) {
      float b[NN];
      const int row = t < NN ? t : t - NN;
      basis_at<NN>(s_xi, s_lam, s_xi[row], t < NN ? -mdx : -mdy, b);
      float* R = (t < NN ? sm.u.sv.Rx : sm.u.sv.Ry) + row * RS;
#pragma unroll
      for (int q = 0; q < NN; ++q) R[q] = b[q];
    }
    if (v0) sm.u.sv.r[p0] = ps0;
    if (v1) sm.u.sv.r[p1] = ps1;
    g.sync();
    // psihat (+)= Ry r Rx^T
    auto precond = [&](bool first) {
      if (v0) {
        float acc = 0.0f;
#pragma unroll
        for (int q = 0; q < NN; ++q) acc = fmaf(sm.u.sv.Rx[i0 * RS + q], sm.u.sv.r[j0 * NN + q], acc);
        sm.u.sv.tt[p0] = acc;
      }
      if (v1) {
        float acc = 0.0f;
#pragma unroll
        for (int q = 0; q < NN; ++q) acc = fmaf(sm.u.sv.Rx[i1 * RS + q], sm.u.sv.r[j1 * NN + q], acc);
        sm.u.sv.tt[p1] = acc;
      }
      g.sync();
      if (v0) {
        float acc = 0.0f;
#pragma unroll
        for (int q = 0; q < NN; ++q) acc = fmaf(sm.u.sv.Ry[j0 * RS + q], sm.u.sv.tt[q * NN + i0], acc);
        sm.ph[j0 * NP + i0] = first ? acc : sm.ph[j0 * NP + i0] + acc;
      }
      if (v1) {
        float acc = 0.0f;
#pragma unroll
        for (int q = 0; q < NN; ++q) acc = fmaf(sm.u.sv.Ry[j1 * RS + q], sm.u.sv.tt[q * NN + i1], acc);
        sm.ph[j1 * NP + i1] = first ? acc : sm.ph[j1 * NP + i1] + acc;
      }
      g.sync();
    };
    precond(true);
    const float scale = g.max(fmaxf(fabsf(ps0), fabsf(ps1)));
    // iterate to the tolerance; a residual that stalls at the float floor is accepted; the best
    // iterate is kept against divergence, and accepting it above the floor is reported
    float prev = INFINITY, best = INFINITY, rmax = INFINITY;
    int it = 0;
    bool done = false;
    for (; it < SOLVE_CAP; ++it) {
      float2 acc = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int mm = 0; mm < NN; ++mm) {
        const float2 row = row_dot2<NN>(sm.ph + mm * NP, Lx);
        acc = __ffma2_rn(Ly[mm], row, acc);
      }
      const float r0v = ps0 - acc.x, r1v = ps1 - acc.y;
      rmax = g.max(fmaxf(v0 ? fabsf(r0v) : 0.0f, v1 ? fabsf(r1v) : 0.0f));
      // values below the normal float range carry no accuracy to refine
      if (rmax <= SOLVE_RTOL * scale || rmax == 0.0f || scale < 1e-30f) { done = true; break; }
      const bool stalled = rmax > 0.5f * prev && rmax <= SOLVE_STALL * scale;
      const bool diverging = !(rmax <= 4.0f * best);                             // or not finite
      if (stalled || diverging) break;
      if (rmax < best) {
        best = rmax;
        if (v0) sm.u.sv.best[p0] = sm.ph[j0 * NP + i0];
        if (v1) sm.u.sv.best[p1] = sm.ph[j1 * NP + i1];
      }
      prev = rmax;
      if (v0) sm.u.sv.r[p0] = r0v;
      if (v1) sm.u.sv.r[p1] = r1v;
      g.sync();
      precond(false);
    }
    c_it += (unsigned long long)(it < SOLVE_CAP ? it + 1 : SOLVE_CAP);
    if (!done) {
      // stalled, diverging or at the cap: the better of the last and the best iterate
      float acc_r = rmax;
      if (!(rmax <= best)) {
        if (v0) sm.ph[j0 * NP + i0] = sm.u.sv.best[p0];
        if (v1) sm.ph[j1 * NP + i1] = sm.u.sv.best[p1];
        acc_r = best;
        g.sync();
      }
      if (acc_r <= SOLVE_STALL * scale) {
        // the float floor of the residual: the solve is as accurate as float allows
      } else if (acc_r <= SOLVE_FLOOR * scale) {
        ++c_floor;
        bits |= SL_ST_SOLVE_FLOOR;
      } else {
        ++c_nc;
        bits |= SL_ST_SOLVE_NOCONV;
      }
    }
    if (v0) W.psihat[E.base + p0] = sm.ph[j0 * NP + i0];
    if (v1) W.psihat[E.base + p1] = sm.ph[j1 * NP + i1];
    // element sums of psi^n (reference measure) and the float-float element mass
    const float w20 = v0 ? s_w[i0] * s_w[j0] : 0.0f, w21 = v1 ? s_w[i1] * s_w[j1] : 0.0f;
    const float2 m12 = g.sum2(fmaf(w20, pn0, w21 * pn1), fmaf(w20 * pn0, pn0, w21 * pn1 * pn1));
    const ff Mn = g.ffsum(mn);
    float* el = W.elem + E.g * 8;
    if (t == 0) {
      el[0] = r0;
      el[1] = gx;
      el[2] = gy;
      el[3] = m12.x;
      el[4] = m12.y;
      el[5] = Mn.hi;
      el[6] = Mn.lo;
    }
    // interface values at the face points (relative to L): traces of psihat, or phi^n at the
    // backward characteristic foot of the face point from t^{n+1} (eq. 4.11; meshes of one node
    // count), L(foot) - L(face point) being the linear part over the foot's displacement
    if (t < 4 * NN) {
      const int f = t / NN, q = t % NN;
      float acc = 0.0f;
      if (P.bvalue == SL_BV_BACKTRACK) {
        const float xr = f == 0 ? 0.0f : f == 1 ? 1.0f : s_xi[q];
        const float yr = f == 2 ? 0.0f : f == 3 ? 1.0f : s_xi[q];
        float Sx = 0.0f, Cx = 0.0f, Sy = 0.0f, Cy = 0.0f;
        if (V.kind == SL_VEL_SWIRL && !V.direct) {
          Sx = f < 2 ? sm.T.corner[f] : sm.T.n[0][q];
          Cx = f < 2 ? sm.T.corner[4 + f] : sm.T.n[1][q];
          Sy = f < 2 ? sm.T.n[2][q] : sm.T.corner[f];
          Cy = f < 2 ? sm.T.n[3][q] : sm.T.corner[4 + f];
        }
        float fdx = 0.0f, fdy = 0.0f;
        rk_disp(V, P.rk, xr, yr, Sx, Cx, Sy, Cy, fdx, fdy, -X.dt, 1.0f, -1.0f, sm.T.ct);
        float bx[NN], by[NN];
        basis_at<NN>(s_xi, s_lam, xr, fdx, bx);
        basis_at<NN>(s_xi, s_lam, yr, fdy, by);
#pragma unroll
        for (int mm = 0; mm < NN; ++mm) acc = fmaf(by[mm], row_dot<NN>(sm.psi + mm * NP, bx), acc);
        acc += fmaf(gx, fdx, gy * fdy);
      } else {
        const float* Lb = (f == 1 || f == 3) ? s_l1 : s_l0;
#pragma unroll
        for (int kk = 0; kk < NN; ++kk) acc = fmaf(f < 2 ? sm.ph[q * NP + kk] : sm.ph[kk * NP + q], Lb[kk], acc);
      }
      W.traces[E.g * M.tstride + t] = acc;
    }
    // outflow over each face and step; a face shared with a neighbour of another node count takes
    // the rule of the finer side, so that both elements integrate the same points.  Pass 1 (one face
    // point per thread): the sign of u.n at each distinct stage time, the quadrature weights, and at
    // the stage time t^n the outflow value itself (the trace of psi^n, no foot).  Pass 2: the outflow
    // (point, stage) pairs of later stage times, compacted into a list, one backward characteristic
    // foot each.  Every pair writes its own slot; the face sums add the slots in a fixed order.
    if (P.cons & (SL_C_MASS | SL_C_ENERGY)) {
      if (t < 4) {
        // points of face t and their prefix sum (lanes 0-3 of the first warp)
        const int nb = nb_index(P, ex, ey, t);
        const int nq = nb < 0 ? NN : max(NN, order_of<NN>(M, E.gb + nb));
        int acc = nq;
#pragma unroll
        for (int o = 1; o < 4; o <<= 1) {
          const int v = __shfl_up_sync(0xfu, acc, o);
          if (t >= o) acc += v;
        }
        sm.cum[t + 1] = acc;
        if (t == 0) {
          sm.cum[0] = 0;
          sm.nitems = 0;
        }
      }
      g.sync();
      const int S = c_ds_n[P.rk];
      const int total = sm.cum[4];
      // Geometry of face point idx: face, point, rule, reference coordinates, sines and cosines.
      // CONF: every face takes the element's own rule (conforming neighbours), so that no lane
      // carries the general rule's branches.
      auto face_point = [&](auto conf, int idx, int& f, int& q, int& nq, float& xr, float& yr, float& Sx, float& Cx,
                            float& Sy, float& Cy) {
        constexpr bool CONF = decltype(conf)::value;
        if (CONF) {
          f = idx / NN;
          q = idx % NN;
          nq = NN;
        } else {
          f = (idx >= sm.cum[1]) + (idx >= sm.cum[2]) + (idx >= sm.cum[3]);
          q = idx - sm.cum[f];
          nq = sm.cum[f + 1] - sm.cum[f];
        }
        const float zq = (CONF || nq == NN) ? s_xi[q] : X.rules[(size_t)nq * 3 * NMAX + q];
        xr = f == 0 ? 0.0f : f == 1 ? 1.0f : zq;
        yr = f == 2 ? 0.0f : f == 3 ? 1.0f : zq;
        Sx = Cx = Sy = Cy = 0.0f;
        if (V.kind == SL_VEL_SWIRL && !V.direct) {
          if (f < 2) {
            Sx = sm.T.corner[f];
            Cx = sm.T.corner[4 + f];
            if (CONF || nq == NN) { Sy = sm.T.n[2][q]; Cy = sm.T.n[3][q]; }
            else sincospif(fmaf(V.hy, zq, V.y0), &Sy, &Cy);
          } else {
            Sy = sm.T.corner[f];
            Cy = sm.T.corner[4 + f];
            if (CONF || nq == NN) { Sx = sm.T.n[0][q]; Cx = sm.T.n[1][q]; }
            else sincospif(fmaf(V.hx, zq, V.x0), &Sx, &Cx);
          }
        }
      };
      const bool conforming = total == 4 * NN;
      const bool tab = V.kind == SL_VEL_SWIRL && !V.direct;
      // CONF: conforming faces; TAB: the swirl from the tabulated sines (both known per element)
      auto pass1 = [&](auto conf, auto tabc) {
      constexpr bool CONF = decltype(conf)::value;
      constexpr bool TAB = decltype(tabc)::value;
      for (int idx = t; idx < total; idx += GT) {
        int f, q, nq;
        float xr, yr, Sx, Cx, Sy, Cy;
        face_point(conf, idx, f, q, nq, xr, yr, Sx, Cx, Sy, Cy);
        const float hn = f < 2 ? X.hx : X.hy;            // velocity in reference units times this = u.n
        const float sg = (f == 0 || f == 2) ? -1.0f : 1.0f;
        const float Wq = (f < 2 ? X.hy : X.hx) *
                         ((CONF || nq == NN) ? s_w[q] : X.rules[(size_t)nq * 3 * NMAX + 2 * NMAX + q]);
        // phi - r0 at the face point itself (stage time t^n): the trace of psi^n plus (L - r0)
        float val0;
        if (CONF || nq == NN) {
          const float* Lb = (f == 1 || f == 3) ? s_l1 : s_l0;
          float acc = 0.0f;
#pragma unroll
          for (int kk = 0; kk < NN; ++kk) acc = fmaf(f < 2 ? sm.psi[q * NP + kk] : sm.psi[kk * NP + q], Lb[kk], acc);
          val0 = acc;
        } else {
          float bx[NN], by[NN];
          basis_at<NN>(s_xi, s_lam, xr, 0.0f, bx);
          basis_at<NN>(s_xi, s_lam, yr, 0.0f, by);
          float acc = 0.0f;
#pragma unroll
          for (int mm = 0; mm < NN; ++mm) acc = fmaf(by[mm], row_dot<NN>(sm.psi + mm * NP, bx), acc);
          val0 = acc;
        }
        val0 += fmaf(gx, xr - 0.5f, gy * (yr - 0.5f));
        // per distinct stage time: the sign of u.n, the weight; later stage times that flow out
        // are queued for their backward foot (their weight kept in fbo, 0 otherwise)
        float uo = 0.0f, ui = 0.0f, q1 = 0.0f, q2 = 0.0f;
        for (int s = 0; s < S; ++s) {
          const float cs = c_ds_c[P.rk][s];
          float ur, vr;
          const float ct = sm.T.ct[__float2int_rn(4.0f * cs)];
          if (TAB) {
            ur = Sx * Sx * (2.0f * Sy * Cy) * ct * V.ihx;
            vr = -Sy * Sy * (2.0f * Sx * Cx) * ct * V.ihy;
          } else {
            vel_at(V, xr, yr, Sx, Cx, Sy, Cy, 0.0f, 0.0f, ct, ur, vr);
          }
          const float un = sg * (f < 2 ? ur : vr) * hn;
          const float bw = c_ds_b[P.rk][s] * Wq * un;
          const bool out = un > (float)TIE;
          if (out) uo += bw;
          if (un < -(float)TIE) ui += bw;
          if (cs == 0.0f) {
            if (out) {
              q1 = fmaf(bw, val0, q1);
              q2 = fmaf(bw * val0, val0, q2);
            }
          } else {
            sm.u.fc.fbo[f][q][s] = out ? bw : 0.0f;
            // queue the pair: one shared atomic per warp (lane order within the warp)
            const unsigned act = __activemask();
            const unsigned want = __ballot_sync(act, out);
            if (want) {
              const int leader = __ffs(act) - 1;
              int base = 0;
              if (g.lane == leader) base = atomicAdd(&sm.nitems, __popc(want));
              base = __shfl_sync(act, base, leader);
              if (out) sm.u.fc.items[base + __popc(want & ((1u << g.lane) - 1u))] = idx * 4 + s;
            }
          }
        }
        sm.u.fc.pt[f][q][0] = uo;
        sm.u.fc.pt[f][q][1] = ui;
        sm.u.fc.pt[f][q][2] = q1;
        sm.u.fc.pt[f][q][3] = q2;
      }
      };
      if (conforming && tab) pass1(std::true_type{}, std::true_type{});
      else pass1(std::false_type{}, std::false_type{});
      g.sync();
      const int nitems = sm.nitems;
      c_feet += (unsigned long long)nitems;
      for (int it2 = t; it2 < nitems; it2 += GT) {
        const int code = sm.u.fc.items[it2];
        const int idx = code >> 2, s = code & 3;
        int f, q, nq;
        float xr, yr, Sx, Cx, Sy, Cy;
        if (conforming) face_point(std::true_type{}, idx, f, q, nq, xr, yr, Sx, Cx, Sy, Cy);
        else face_point(std::false_type{}, idx, f, q, nq, xr, yr, Sx, Cx, Sy, Cy);
        const float cs = c_ds_c[P.rk][s];
        float fdx = 0.0f, fdy = 0.0f;
        rk_disp(V, P.rk, xr, yr, Sx, Cx, Sy, Cy, fdx, fdy, -cs * X.dt, cs, -cs, sm.T.ct);
        float bx[NN], by[NN];
        basis_at<NN>(s_xi, s_lam, xr, fdx, bx);
        basis_at<NN>(s_xi, s_lam, yr, fdy, by);
        float val = 0.0f;
#pragma unroll
        for (int mm = 0; mm < NN; ++mm) val = fmaf(by[mm], row_dot<NN>(sm.psi + mm * NP, bx), val);
        val += fmaf(gx, (xr - 0.5f) + fdx, gy * ((yr - 0.5f) + fdy));   // phi - r0 = (L - r0) + psi
        sm.u.fc.fv[f][q][s] = val;
      }
      g.sync();
      // per face point: the outflow of the later stage times, added in stage order
      if (S > 1)
        for (int idx = t; idx < total; idx += GT) {
          const int f = (idx >= sm.cum[1]) + (idx >= sm.cum[2]) + (idx >= sm.cum[3]);
          const int q = idx - sm.cum[f];
          float q1 = sm.u.fc.pt[f][q][2], q2 = sm.u.fc.pt[f][q][3];
          for (int s = 1; s < S; ++s) {
            const float bo = sm.u.fc.fbo[f][q][s];
            if (bo != 0.0f) {
              const float v = sm.u.fc.fv[f][q][s];
              q1 = fmaf(bo, v, q1);
              q2 = fmaf(bo * v, v, q2);
            }
          }
          sm.u.fc.pt[f][q][2] = q1;
          sm.u.fc.pt[f][q][3] = q2;
        }
      g.sync();
      // per face and quantity (16 threads): the sum over the face's points in point order
      if (t < 16) {
        const int f = t >> 2, c = t & 3;
        const int nq = sm.cum[f + 1] - sm.cum[f];
        float acc = 0.0f;
#pragma unroll
        for (int q = 0; q < NMAX; ++q)
          if (q < nq) acc += sm.u.fc.pt[f][q][c];
        sm.u.fc.fs[f][c] = acc;
      }
      g.sync();
      if (t < 4) {
        const int f = t;
        const float uo = sm.u.fc.fs[f][0], ui = sm.u.fc.fs[f][1], q1 = sm.u.fc.fs[f][2], q2 = sm.u.fc.fs[f][3];
        // the face's outflow flux of phi as a float-float value: r0 U_out + sum bw (phi - r0), plus
        // the inflow of the ghost value through a domain face
        ff Gf = ff_add(two_prod(r0, uo), ff{q1, 0.0f});
        if (nb_index(P, ex, ey, f) < 0) Gf = ff_add(Gf, two_prod((float)P.ghost, ui));
        float* F = W.faces + E.g * 24 + 6 * f;
        F[0] = Gf.hi;
        F[1] = Gf.lo;
        F[2] = uo;
        F[3] = ui;
        F[4] = q1;
        F[5] = q2;
      }
    }
  }
  if (t == 0 && X0.counts) {
    atomicAdd(X0.counts + SL_CNT_SOLVE_ITERS, c_it);
    if (c_floor) atomicAdd(X0.counts + SL_CNT_SOLVE_FLOOR, c_floor);
    if (c_nc) atomicAdd(X0.counts + SL_CNT_SOLVE_NOCONV, c_nc);
    if (c_feet) atomicAdd(X0.counts + SL_CNT_FEET, c_feet);
  }
  if (bits) atomicOr(status, bits);
}

// ------------------------------------------------------------------ phase 2
template <int NN>
struct Smem2 {
  static constexpr int ND = Shape<NN>::ND, G = Shape<NN>::G;
  static constexpr int MMAX = 4 * NN + 1;
  float a[ND];
  float r[MMAX], ca[MMAX];
  float red[4 * G];
  float scal[8];
};

template <int NN>
__global__ void __launch_bounds__(Shape<NN>::NT, Shape<NN>::MINB2)
    k_p2(StepParams P0, const __grid_constant__ Mixed2DExtra X0, Map2D M, int64_t count, const float* __restrict__ in,
         Work2M W, float* __restrict__ out, unsigned* status) {
  using S = Shape<NN>;
  constexpr int ND = S::ND, G = S::G, GT = S::GT, EPC = S::EPC;
  __shared__ float s_xi[NN], s_w[NN], s_l0[NN], s_l1[NN];
  __shared__ Smem2<NN> sm_all[EPC];
  // the pseudo-inverse of the fit, [m][n^2], staged once per CTA (dynamic shared memory)
  extern __shared__ __align__(16) float s_Cp[];
  if (threadIdx.x < NN) {
    s_xi[threadIdx.x] = X0.xi[threadIdx.x];
    s_w[threadIdx.x] = X0.w[threadIdx.x];
    s_l0[threadIdx.x] = X0.l0[threadIdx.x];
    s_l1[threadIdx.x] = X0.l1[threadIdx.x];
  }
  for (int i = threadIdx.x; i < P0.m * ND; i += blockDim.x) s_Cp[i] = X0.Cp[i];
  __syncthreads();
  Grp<G> g;
  g.slot = threadIdx.x / GT;
  g.t = threadIdx.x % GT;
  g.lane = threadIdx.x & 31;
  g.w = g.t >> 5;
  Smem2<NN>& sm = sm_all[g.slot];
  g.red = sm.red;
  g.rb = 0;
  const int t = g.t;
  const int p0 = t, p1 = t + GT;
  const bool v0 = p0 < ND, v1 = p1 < ND;
  const int i0 = p0 % NN, j0 = (p0 / NN) % NN, i1 = p1 % NN, j1 = (p1 / NN) % NN;
  const float w20 = v0 ? s_w[i0] * s_w[j0] : 0.0f, w21 = v1 ? s_w[i1] * s_w[j1] : 0.0f;
  unsigned long long c_el = 0, c_eapp = 0, c_pit = 0, c_pnc = 0;
  unsigned bits = 0;
  const int64_t ngroups = (int64_t)gridDim.x * EPC;
  for (int64_t k = (int64_t)blockIdx.x * EPC + g.slot; k < count; k += ngroups) {
    g.sync();
    StepParams P = P0;
    const Elem E = elem_at<NN>(P, M, k);
    Mixed2DExtra X = X0;
    batch_extra(P, M, X);
    const int ex = E.ex, ey = E.ey;
    const float x0 = (float)(P.x0 + ex * P.hx), y0 = (float)(P.y0 + ey * P.hy);
    const VelElem V = make_vel(P, X, x0, y0);
    // every global read of the element first, so that they share one memory round trip: own
    // record, psihat, input (energy), face-point traces and the neighbours' records and faces
    const bool bnd = (P.cons & SL_C_BOUNDARY) != 0;
    const bool mass = (P.cons & SL_C_MASS) != 0, energy = (P.cons & SL_C_ENERGY) != 0;
    const int nb_rows = bnd ? 4 * NN : 0;
    const float* el = W.elem + E.g * 8;
    const float r0 = el[0], gx = el[1], gy = el[2], m1 = el[3], mn_hi = el[5], mn_lo = el[6];
    const float ph0 = v0 ? W.psihat[E.base + p0] : 0.0f;
    const float ph1 = v1 ? W.psihat[E.base + p1] : 0.0f;
    float in_hi0 = 0.0f, in_lo0 = 0.0f, in_hi1 = 0.0f, in_lo1 = 0.0f;
    if (energy) {
      if (v0) { in_hi0 = in[E.base + p0]; in_lo0 = in[X.plane + E.base + p0]; }
      if (v1) { in_hi1 = in[E.base + p1]; in_lo1 = in[X.plane + E.base + p1]; }
    }
    // boundary lanes: face point (f, q), own trace, neighbour's trace at this point and record
    int bf = 0, bq = 0, bnb = -1;
    float own = 0.0f, trn = 0.0f, en0 = 0.0f, en1 = 0.0f, en2 = 0.0f;
    if (bnd && t < 4 * NN) {
      bf = t / NN;
      bq = t % NN;
      bnb = nb_index(P, ex, ey, bf);
      own = W.traces[E.g * M.tstride + t];
      if (bnb >= 0) {
        const int64_t gn = E.gb + bnb;
        const int nn = order_of<NN>(M, gn);
        const float* tr = W.traces + gn * M.tstride + (bf ^ 1) * nn;
        const float* en = W.elem + gn * 8;
        en0 = en[0];
        en1 = en[1];
        en2 = en[2];
        trn = nn == NN ? tr[bq] : interp_rule(X.rules, nn, tr, s_xi[bq]);
      }
    }
    // face lanes (0-3): own face record, the neighbour's record of the shared face and its r0
    int fnb = -1;
    float F[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f}, Gn[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f}, rnb = 0.0f;
    if ((mass || energy) && t < 4) {
      fnb = nb_index(P, ex, ey, t);
      const float* Fp = W.faces + E.g * 24 + 6 * t;
#pragma unroll
      for (int c = 0; c < 6; ++c) F[c] = Fp[c];
      if (fnb >= 0) {
        const float* Gp = W.faces + (E.gb + fnb) * 24 + 6 * (t ^ 1);
#pragma unroll
        for (int c = 0; c < 6; ++c) Gn[c] = Gp[c];
        rnb = W.elem[(E.gb + fnb) * 8];
      }
    }
    if (bnd && t < 4 * NN) {
      const int f = bf, q = bq, nb = bnb;
      // neighbour's value at this element's face point relative to this element's L: the difference
      // of the two references (float-float, of the size of psi when both fit the same data) plus the
      // neighbour's trace of its own psihat
      const float aq = s_xi[q] - 0.5f;
      const float fa = f == 0 ? -0.5f : f == 1 ? 0.5f : aq, fb = f == 2 ? -0.5f : f == 3 ? 0.5f : aq;
      const ff lown = lref(r0, gx, gy, fa, fb);
      float other;
      if (nb >= 0) {
        const ff lnb = lref(en0, en1, en2, f == 0 ? 0.5f : f == 1 ? -0.5f : fa, f == 2 ? 0.5f : f == 3 ? -0.5f : fb);
        const float dl = __fadd_rn(__fsub_rn(lnb.hi, lown.hi), __fsub_rn(lnb.lo, lown.lo));
        other = dl + trn;
      } else {
        other = __fsub_rn(__fsub_rn((float)P.ghost, lown.hi), lown.lo);
      }
      const float xr = f == 0 ? 0.0f : f == 1 ? 1.0f : s_xi[q];
      const float yr = f == 2 ? 0.0f : f == 3 ? 1.0f : s_xi[q];
      // one velocity evaluation per face point at t^{n+1}: sinpi/cospi directly
      VelElem Vd = V;
      Vd.direct = true;
      const float ct = V.kind == SL_VEL_SWIRL ? cospif(X.tT + X.dtT) : 1.0f;
      float ur, vr;
      vel_at(Vd, xr, yr, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, ct, ur, vr);
      const float un = (f == 0 || f == 2 ? -1.0f : 1.0f) * (f < 2 ? ur * X.hx : vr * X.hy);
      float val;
      if (un > (float)TIE) val = own;
      else if (un < -(float)TIE) val = other;
      else val = nb < 0 ? own : 0.5f * (own + other);
      // the row's value at psihat: the own trace when the interface values are traces of psihat,
      // else the trace formed here from the stored psihat
      float trh = own;
      if (P.bvalue == SL_BV_BACKTRACK) {
        const float* Lb = (f == 1 || f == 3) ? s_l1 : s_l0;
        const float* ps = W.psihat + E.base;
        trh = 0.0f;
#pragma unroll
        for (int kk = 0; kk < NN; ++kk) trh = fmaf(f < 2 ? ps[q * NN + kk] : ps[kk * NN + q], Lb[kk], trh);
      }
      sm.r[t] = val - trh;
    }
    // net outflow of mass (increments), of the squared increments and of the velocity, lanes 0-3 of
    // the first warp one face each, summed in face order; the float-float mass target
    if ((mass || energy) && t < 32) {
      float cu = 0.0f, cm = 0.0f, cd = 0.0f;
      ff net = {0.0f, 0.0f};
      if (t < 4) {
        cu = F[2] + F[3];
        net = ff{F[0], F[1]};
        if (fnb >= 0) {
          const float dref = rnb - r0;
          // inflow part: u.n (dref + psi_nb) with the neighbour's u.n = -ours
          cm = F[4] + (dref * F[3] - Gn[4]);
          cd = F[5] + (dref * dref * F[3] - 2.0f * dref * Gn[4] - Gn[5]);
          net = ff_add(net, ff_neg(ff{Gn[0], Gn[1]}));
        } else {
          const float gg = (float)P.ghost - r0;
          cm = F[4] + gg * F[3];
          cd = F[5] + gg * gg * F[3];
        }
      }
      float su = 0.0f, smm = 0.0f, sd = 0.0f;
      ff sn = {0.0f, 0.0f};
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        su += __shfl_sync(0xffffffffu, cu, f);
        smm += __shfl_sync(0xffffffffu, cm, f);
        sd += __shfl_sync(0xffffffffu, cd, f);
        sn = ff_add(sn, ff{__shfl_sync(0xffffffffu, net.hi, f), __shfl_sync(0xffffffffu, net.lo, f)});
      }
      if (t == 0) {
        // M^{n+1} = M^n - dt / (hx hy) (net outflow), in float-float
        const ff ln = ff_mul(sn, ff{X.lam_hi, X.lam_lo});
        const ff target = ff_add(ff{mn_hi, mn_lo}, ff_neg(ln));
        sm.scal[0] = smm;
        sm.scal[1] = sd;
        sm.scal[2] = su;
        sm.scal[3] = target.hi;
        sm.scal[4] = target.lo;
      }
    }
    g.sync();
    const float netm = sm.scal[0], netd2 = sm.scal[1];
    const ff target = {sm.scal[3], sm.scal[4]};
    const float lam = X.dt_area;                  // dt / (hx hy)
    if (mass) {
      const float mh = g.sum(fmaf(w20, ph0, w21 * ph1));
      // target (increments): sum w psi^n - lam (net increment outflow + ref * closed-surface u.n);
      // ref * (closed-surface integral of u.n) is dropped: every 2D velocity here is divergence free
      // and the face quadrature integrates it to rounding (the refinement below meets the float-float
      // target whatever this residual leaves)
      if (t == 0) sm.r[nb_rows] = (m1 - lam * netm) - mh;
    }
    g.sync();
    const int m = P.m;
    float phL0 = ph0, phL1 = ph1;
#pragma unroll 4
    for (int kk = 0; kk < m; ++kk) {
      const float rk_ = sm.r[kk];
      phL0 = fmaf(s_Cp[kk * ND + (v0 ? p0 : 0)], rk_, phL0);
      phL1 = fmaf(s_Cp[kk * ND + (v1 ? p1 : 0)], rk_, phL1);
    }
    if (!v0) phL0 = 0.0f;
    if (!v1) phL1 = 0.0f;
    float cur0 = phL0, cur1 = phL1;
    bool ok = true;
    if (energy) {
      // energy mismatch from increments (mass enforced): sum w (psiL - psi)(psiL + psi) + lam net(delta^2);
      // without the mass row, add 2 ref times the mass residual (closed-surface u.n taken as zero)
      float psin0 = 0.0f, psin1 = 0.0f;
      if (v0) {
        const ff L = lref(r0, gx, gy, s_xi[i0] - 0.5f, s_xi[j0] - 0.5f);
        psin0 = __fadd_rn(__fsub_rn(in_hi0, L.hi), __fsub_rn(in_lo0, L.lo));
      }
      if (v1) {
        const ff L = lref(r0, gx, gy, s_xi[i1] - 0.5f, s_xi[j1] - 0.5f);
        psin1 = __fadd_rn(__fsub_rn(in_hi1, L.hi), __fsub_rn(in_lo1, L.lo));
      }
      const float dp0 = phL0 - psin0, dp1 = phL1 - psin1;
      const float2 evml = g.sum2(fmaf(w20 * dp0, phL0 + (phL0 - dp0), w21 * dp1 * (phL1 + (phL1 - dp1))),
                                 fmaf(w20, phL0, w21 * phL1));
      const float ev = evml.x, ml = evml.y;
      float gamma;
      if (mass) gamma = ev + lam * netd2;
      else gamma = fmaf(2.0f * r0, (ml - m1) + lam * netm, ev + lam * netd2);
      const float escale = g.sum(fmaf(w20 * (r0 + cur0), r0 + cur0, w21 * (r0 + cur1) * (r0 + cur1)));
      const float smax = g.max(fmaxf(fmaxf(fabsf(phL0), fabsf(phL1)), fabsf(r0)));
      if (smax >= 1e-30f && fabsf(gamma) > (float)ENERGY_SKIP_RTOL_MIXED * escale) {
        ++c_eapp;
        int exn;
        frexpf(smax, &exn);
        const float sc = ldexpf(1.0f, -exn), usc = ldexpf(1.0f, exn);
        const float rf = r0 * sc, gm = gamma * sc * sc;
        const float ql0 = phL0 * sc, ql1 = phL1 * sc;
        float c20 = ql0, c21 = ql1;
        const float tol = 2.4e-7f + 1e-30f;         // scaled units: values are of order one
        bool conv = false, feasible = true;
        int it = 0;
        for (; it < P.picard_cap; ++it) {
          const float a0 = w20 * (mass ? c20 : rf + c20), a1 = w21 * (mass ? c21 : rf + c21);
          if (v0) sm.a[p0] = a0;
          if (v1) sm.a[p1] = a1;
          g.sync();
          if (bnd && t < 4 * NN) {
            const int f = t / NN, qq = t % NN;
            const float* Lb = (f == 1 || f == 3) ? s_l1 : s_l0;
            float acc = 0.0f;
            for (int kk = 0; kk < NN; ++kk) acc = fmaf(f < 2 ? sm.a[qq * NN + kk] : sm.a[kk * NN + qq], Lb[kk], acc);
            sm.ca[t] = acc;
          }
          if (mass) {
            const float cmm = g.sum(fmaf(w20, a0, w21 * a1));
            if (t == 0) sm.ca[nb_rows] = cmm;
          }
          g.sync();
          float q0 = a0, q1 = a1;
#pragma unroll 4
          for (int kk = 0; kk < m; ++kk) {
            const float ck = sm.ca[kk];
            q0 = fmaf(-s_Cp[kk * ND + (v0 ? p0 : 0)], ck, q0);
            q1 = fmaf(-s_Cp[kk * ND + (v1 ? p1 : 0)], ck, q1);
          }
          if (!v0) q0 = 0.0f;
          if (!v1) q1 = 0.0f;
          const float2 ab = g.sum2(fmaf(w20 * ql0, q0, w21 * ql1 * q1), fmaf(w20 * q0, q0, w21 * q1 * q1));
          float alpha = ab.x;
          if (!mass) alpha = fmaf(rf, g.sum(fmaf(w20, q0, w21 * q1)), alpha);
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
          const float nv0 = v0 ? fmaf(s, q0, ql0) : 0.0f, nv1 = v1 ? fmaf(s, q1, ql1) : 0.0f;
          const float delta = g.max(fmaxf(fabsf(nv0 - c20), fabsf(nv1 - c21)));
          c20 = nv0;
          c21 = nv1;
          if (delta <= tol) { conv = feasible; break; }
        }
        c_pit += (unsigned long long)(it < P.picard_cap ? it + 1 : P.picard_cap);
        if (conv) {                                 // else keep the linear-constraint solution
          cur0 = c20 * usc;
          cur1 = c21 * usc;
        }
        ok = conv;
      }
    }
    // write-back v = L + psi as a float-float sum; with the mass row, one refinement step moves the
    // float-float miss of the element mass along the pseudo-inverse column of the mass row (lo word)
    ff vv0 = {0.0f, 0.0f}, vv1 = {0.0f, 0.0f};
    if (v0) {
      const ff L = lref(r0, gx, gy, s_xi[i0] - 0.5f, s_xi[j0] - 0.5f);
      const ff s = two_sum(L.hi, cur0);
      vv0 = fast_two_sum(s.hi, __fadd_rn(s.lo, L.lo));
    }
    if (v1) {
      const ff L = lref(r0, gx, gy, s_xi[i1] - 0.5f, s_xi[j1] - 0.5f);
      const ff s = two_sum(L.hi, cur1);
      vv1 = fast_two_sum(s.hi, __fadd_rn(s.lo, L.lo));
    }
    if (mass) {
      ff mv = {0.0f, 0.0f};
      if (v0) mv = ff_mul(vv0, ff{X.w2h[p0], X.w2l[p0]});
      if (v1) mv = ff_add(mv, ff_mul(vv1, ff{X.w2h[p1], X.w2l[p1]}));
      mv = g.ffsum(mv);
      const float miss = ff_to_f(ff_add(target, ff_neg(mv)));
      const float* cmcol = s_Cp + nb_rows * ND;
      if (v0) vv0 = fast_two_sum(vv0.hi, fmaf(miss, cmcol[p0], vv0.lo));
      if (v1) vv1 = fast_two_sum(vv1.hi, fmaf(miss, cmcol[p1], vv1.lo));
    }
    if (v0) {
      out[E.base + p0] = vv0.hi;
      out[X.plane + E.base + p0] = vv0.lo;
      if (!isfinite(vv0.hi)) bits |= SL_ST_NONFINITE;
    }
    if (v1) {
      out[E.base + p1] = vv1.hi;
      out[X.plane + E.base + p1] = vv1.lo;
      if (!isfinite(vv1.hi)) bits |= SL_ST_NONFINITE;
    }
    ++c_el;
    if (!ok) {
      bits |= SL_ST_PICARD_NOCONV;
      ++c_pnc;
    }
  }
  if (t == 0 && X0.counts) {
    atomicAdd(X0.counts + SL_CNT_ELEMS, c_el);
    if (c_eapp) atomicAdd(X0.counts + SL_CNT_ENERGY_APPLIED, c_eapp);
    if (c_pit) atomicAdd(X0.counts + SL_CNT_PICARD_ITERS, c_pit);
    if (c_pnc) atomicAdd(X0.counts + SL_CNT_PICARD_NOCONV, c_pnc);
  }
  if (bits) atomicOr(status, bits);
}

// persistent grid: the resident CTAs of the whole GPU, or one CTA per EPC elements if fewer
template <int NN>
void launch_n(int phase, const StepParams& p, const Mixed2DExtra& x, const Map2D& m, int64_t count, const float* in,
              float* out, const Work2M& w, unsigned* st, cudaStream_t s, int per_sm) {
  if (count <= 0) return;
  using S = Shape<NN>;
  // phase 2 stages the fit operator for the largest row set (4 n + 1 rows), whatever p.m is, so
  // that one occupancy figure serves every launch
  const size_t smem2 = (size_t)(4 * NN + 1) * S::ND * sizeof(float);
  const void* kern = phase == 1 ? (const void*)k_p1<NN> : (const void*)k_p2<NN>;
  int fill = persistent_grid(kern, S::NT, phase == 1 ? 0 : smem2);
  // per_sm > 0: that many resident CTAs per SM (the autotuner's choice), within the occupancy
  if (per_sm > 0) fill = std::min(fill, per_sm * sm_count());
  const int64_t want = (count + S::EPC - 1) / S::EPC;
  const unsigned grid = (unsigned)(want < fill ? want : fill);
  if (phase == 1) k_p1<NN><<<grid, S::NT, 0, s>>>(p, x, m, count, in, w, st);
  else k_p2<NN><<<grid, S::NT, smem2, s>>>(p, x, m, count, in, w, out, st);
}

}  // namespace k2m
}  // namespace sl
