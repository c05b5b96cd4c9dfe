#pragma once
// Float-float arithmetic of the mixed-precision kernels: error-free transformations (Knuth's two-sum
// and the FMA product error) and the sums and products built on them.  A float-float value is the
// unevaluated sum hi + lo with |lo| <= ulp(hi) / 2, about 48 significant bits.

namespace sl {

struct ff {
  float hi, lo;
};
__device__ __forceinline__ ff two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ ff fast_two_sum(float a, float b) {   // |a| >= |b| or a = 0
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ff two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, fmaf(a, b, -p)};
}
// sum of two float-float values; symmetric in its arguments bit for bit (the two-sum error term is
// exact whatever the order), so a butterfly leaves the same value in every lane
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  const ff s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, __fadd_rn(__fadd_rn(a.lo, b.lo), s.lo));
}
__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }
// product with a float-float weight, to about 2^-44 relative
__device__ __forceinline__ ff ff_mul(ff a, ff w) {
  const ff p = two_prod(a.hi, w.hi);
  return fast_two_sum(p.hi, fmaf(a.hi, w.lo, fmaf(a.lo, w.hi, p.lo)));
}
__device__ __forceinline__ float ff_to_f(ff a) { return __fadd_rn(a.hi, a.lo); }

// Compensated dot product sum_i (wh_i + wl_i)(hi_i + lo_i) (float-float weights and values): the
// products' high parts are added with their exact rounding errors (two-sum), everything of lower
// order goes into one float compensation.  About 2^-46 relative for sums whose terms do not cancel.
struct cdot {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add(float wh, float wl, float hi, float lo) {
    const float p = __fmul_rn(wh, hi);
    const float pe = fmaf(wh, hi, -p);
    const ff t = two_sum(s, p);
    s = t.hi;
    c = __fadd_rn(c, __fadd_rn(__fadd_rn(t.lo, pe), fmaf(wh, lo, __fmul_rn(wl, hi))));
  }
  __device__ __forceinline__ ff get() const { return fast_two_sum(s, c); }
};

}  // namespace sl
