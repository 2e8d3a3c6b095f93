// Double-word ("double-float") arithmetic on FP32 pairs.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// about 48 significant bits. On this part an FP64 instruction costs about 70
// cycles of its SM sub-partition, against about 2 for an FP32 one, so short
// FP64-class computations run faster as a dozen FP32 operations each. The
// building blocks are the error-free transformations: Knuth's TwoSum (the
// exact rounding error of a sum) and Dekker's product with an FMA (the exact
// rounding error of a product), as used for double-word arithmetic by
// Joldes, Muller and Popescu (ACM TOMS 44, 2017). The _rn intrinsics keep the
// compiler from contracting or reassociating them.
#pragma once

#include <cuda_runtime.h>

namespace rsv {

struct DW {
  float hi, lo;
};

// s + e = a + b exactly.
__device__ __forceinline__ float two_sum(float a, float b, float& e) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return s;
}

// s + e = a + b exactly, for |a| >= |b| (or a = 0).
__device__ __forceinline__ float fast_two_sum(float a, float b, float& e) {
  const float s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
  return s;
}

__device__ __forceinline__ DW dw_renorm(float s, float lo) {
  float e;
  const float h = fast_two_sum(s, lo, e);
  return DW{h, e};
}

// FP64 <-> double word (FP64 instructions: use outside inner loops).
__device__ __forceinline__ DW dw_from(double d) {
  const float h = __double2float_rn(d);
  return DW{h, __double2float_rn(d - (double)h)};
}
__device__ __forceinline__ double dw_value(DW a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ DW dw_neg(DW a) { return DW{-a.hi, -a.lo}; }

// a + c * x
__device__ __forceinline__ DW dw_axpy(DW a, DW c, DW x) {
  const float p = __fmul_rn(c.hi, x.hi);
  float e = __fmaf_rn(c.hi, x.hi, -p);
  e = __fmaf_rn(c.hi, x.lo, __fmaf_rn(c.lo, x.hi, e));
  float f;
  const float s = two_sum(a.hi, p, f);
  return dw_renorm(s, __fadd_rn(__fadd_rn(a.lo, e), f));
}

// a * x + b * y + c * z - w, with one renormalisation
__device__ __forceinline__ DW dw_stencil(DW a, DW x, DW b, DW y, DW c, DW z, DW w) {
  const float p1 = __fmul_rn(a.hi, x.hi), p2 = __fmul_rn(b.hi, y.hi), p3 = __fmul_rn(c.hi, z.hi);
  const float e1 = __fmaf_rn(a.hi, x.hi, -p1), e2 = __fmaf_rn(b.hi, y.hi, -p2), e3 = __fmaf_rn(c.hi, z.hi, -p3);
  const float t = __fmaf_rn(a.hi, x.lo, __fmaf_rn(a.lo, x.hi, __fmaf_rn(b.hi, y.lo, __fmaf_rn(b.lo, y.hi,
                  __fmaf_rn(c.hi, z.lo, __fmul_rn(c.lo, z.hi))))));
  float f1, f2, f3;
  float s = two_sum(p1, p2, f1);
  s = two_sum(s, p3, f2);
  s = two_sum(s, -w.hi, f3);
  const float lo = __fadd_rn(__fadd_rn(__fadd_rn(e1, e2), __fadd_rn(e3, t)),
                             __fadd_rn(__fadd_rn(f1, f2), __fsub_rn(f3, w.lo)));
  return dw_renorm(s, lo);
}

__device__ __forceinline__ DW dw_shfl_up(DW a, int d) {
  return DW{__shfl_up_sync(0xffffffffu, a.hi, d), __shfl_up_sync(0xffffffffu, a.lo, d)};
}
__device__ __forceinline__ DW dw_shfl_down(DW a, int d) {
  return DW{__shfl_down_sync(0xffffffffu, a.hi, d), __shfl_down_sync(0xffffffffu, a.lo, d)};
}

}  // namespace rsv
