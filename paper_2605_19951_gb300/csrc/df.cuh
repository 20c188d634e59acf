// Double-float ("pair") arithmetic on the FP32 pipes: a value is hi + lo
// with |lo| <= ulp(hi) / 2 (48-bit significand).  Error-free transformations:
// Knuth's TwoSum, the FMA form of Dekker's TwoProduct, and the compensated dot
// product Dot2 of Ogita, Rump and Oishi (2005).  Explicit _rn intrinsics keep
// the compiler from contracting or reassociating them.
#pragma once
#include <cuda_runtime.h>

namespace tem {

// rounding-exact primitives (explicit _rn forms: no contraction or reassociation)
struct dfl {
  float hi, lo;
};

__device__ __forceinline__ dfl two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ dfl fast_two_sum(float a, float b) {   // |a| >= |b| (or a == 0)
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ dfl df_add(dfl x, dfl y) {
  const dfl s = two_sum(x.hi, y.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ dfl df_mul(dfl x, dfl y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ dfl df_neg(dfl x) { return {-x.hi, -x.lo}; }

// Dot2 accumulator: s + c, products of pairs added error-free into s
struct Dot2 {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(dfl a, dfl b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    const dfl t = two_sum(s, p);
    s = t.hi;
    c = __fadd_rn(c, __fadd_rn(t.lo, e));
  }
  __device__ __forceinline__ dfl value() const { return fast_two_sum(s, c); }
};

__device__ __forceinline__ dfl split(double d) {
  const float h = __double2float_rn(d);
  return {h, __double2float_rn(d - double(h))};
}

__device__ __forceinline__ double df_to_double(dfl x) { return double(x.hi) + double(x.lo); }

}  // namespace tem
