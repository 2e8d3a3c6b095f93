// 16-byte complex vectors and the flip arithmetic on them, shared by the
// streaming tile passes and the batched kernel. complex64: one vector is two
// amplitudes held as packed FP32x2 words; complex128: one amplitude.
#pragma once

#include <type_traits>

#include "rsv_common.cuh"
#include "tma.cuh"

namespace rsv {

template <typename Real>
struct VecCfg {
  static constexpr bool kF = std::is_same<Real, float>::value;
};

// ---- complex helpers -------------------------------------------------------
// One 16-byte vector: complex64 = 2 amplitudes (two packed f32x2 words),
// complex128 = 1 amplitude (two doubles).
struct Vec {
  unsigned long long w0, w1;
};

__device__ __forceinline__ Vec lds_vec(const void* base, int idx) {
  const ulonglong2 v = reinterpret_cast<const ulonglong2*>(base)[idx];
  return Vec{v.x, v.y};
}
__device__ __forceinline__ void sts_vec(void* base, int idx, Vec v) {
  reinterpret_cast<ulonglong2*>(base)[idx] = make_ulonglong2(v.w0, v.w1);
}
// plain global load (coherent: for data written earlier in the same kernel)
__device__ __forceinline__ Vec ldv_vec(const void* base, int64_t idx) {
  const ulonglong2 v = reinterpret_cast<const ulonglong2*>(base)[idx];
  return Vec{v.x, v.y};
}
// read-only-path global load (data not written by the running kernel)
__device__ __forceinline__ Vec ldg_vec(const void* base, int64_t idx) {
  const ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2*>(base) + idx);
  return Vec{v.x, v.y};
}
__device__ __forceinline__ Vec ldcs_vec(const void* base, int64_t idx) {
  const ulonglong2 v = __ldcs(reinterpret_cast<const ulonglong2*>(base) + idx);
  return Vec{v.x, v.y};
}
__device__ __forceinline__ void stg_vec(void* base, int64_t idx, Vec v) {
  reinterpret_cast<ulonglong2*>(base)[idx] = make_ulonglong2(v.w0, v.w1);
}
__device__ __forceinline__ double dbl(unsigned long long w) { return __longlong_as_double((long long)w); }
__device__ __forceinline__ unsigned long long bits(double d) { return (unsigned long long)__double_as_longlong(d); }

// Coefficient of one flip in "apply" form. complex64: rr = (cr, cr), ii = (-ci, ci)
// as packed pairs; complex128: cr, ci as doubles (stored in the same words).
struct Coef {
  unsigned long long rr, ii;
};

template <typename Real, bool PHI>
__device__ __forceinline__ Coef make_coef(Real cr, Real ci) {
  if constexpr (VecCfg<Real>::kF) {
    return Coef{f2_pack(cr, cr), PHI ? f2_pack(-ci, ci) : 0ull};
  } else {
    return Coef{bits(cr), bits(ci)};
  }
}

// complex64 amplitude o += coef * p (packed re, im).
template <bool PHI>
__device__ __forceinline__ void cmac_word(unsigned long long& o, const Coef& c, unsigned long long p) {
  f2_fma(o, c.rr, p);
  if (PHI) {
    float re, im;
    f2_unpack(p, re, im);
    f2_fma(o, c.ii, f2_pack(im, re));
  }
}

// o += coef * p on every amplitude of the vector.
template <typename Real, bool PHI>
__device__ __forceinline__ void cmac(Vec& o, const Coef& c, const Vec& p) {
  if constexpr (VecCfg<Real>::kF) {
    cmac_word<PHI>(o.w0, c, p.w0);
    cmac_word<PHI>(o.w1, c, p.w1);
  } else {
    const double cr = dbl(c.rr), pr = dbl(p.w0), pi = dbl(p.w1);
    double orr = fma(cr, pr, dbl(o.w0)), oi = fma(cr, pi, dbl(o.w1));
    if (PHI) {
      const double ci = dbl(c.ii);
      orr = fma(-ci, pi, orr);
      oi = fma(ci, pr, oi);
    }
    o.w0 = bits(orr);
    o.w1 = bits(oi);
  }
}

// o = s * x (real s) per amplitude; e0/e1 are the per-amplitude scales (complex64
// has two amplitudes per vector, complex128 uses e0 only).
template <typename Real>
__device__ __forceinline__ Vec scale2(const Vec& x, Real e0, Real e1) {
  if constexpr (VecCfg<Real>::kF) {
    return Vec{f2_mul(f2_pack(e0, e0), x.w0), f2_mul(f2_pack(e1, e1), x.w1)};
  } else {
    return Vec{bits(e0 * dbl(x.w0)), bits(e0 * dbl(x.w1))};
  }
}

// o += s * x (real s, same for every amplitude)
template <typename Real>
__device__ __forceinline__ void axpy(Vec& o, Real s, const Vec& x) {
  if constexpr (VecCfg<Real>::kF) {
    const unsigned long long ss = f2_pack(s, s);
    f2_fma(o.w0, ss, x.w0);
    f2_fma(o.w1, ss, x.w1);
  } else {
    o.w0 = bits(fma(s, dbl(x.w0), dbl(o.w0)));
    o.w1 = bits(fma(s, dbl(x.w1), dbl(o.w1)));
  }
}

// x = (u - a v) * s
template <typename Real>
__device__ __forceinline__ Vec form(const Vec& u, const Vec& v, Real a, Real s, bool has_v) {
  Vec r = u;
  if (has_v) axpy<Real>(r, -a, v);
  return scale2<Real>(r, s, s);
}

// Re<x, o>, |o|^2, |x|^2 of one vector: four-term FP32 (or FP64) partials,
// accumulated across vectors with the compensated accumulator.
template <typename Real, typename Acc>
__device__ __forceinline__ void reduce_vec(const Vec& x, const Vec& o, Acc& r0, Acc& r1, Acc& r2) {
  if constexpr (VecCfg<Real>::kF) {
    float x0, x1, x2, x3, o0, o1, o2, o3;
    f2_unpack(x.w0, x0, x1);
    f2_unpack(x.w1, x2, x3);
    f2_unpack(o.w0, o0, o1);
    f2_unpack(o.w1, o2, o3);
    r0.add(fmaf(x3, o3, fmaf(x2, o2, fmaf(x1, o1, x0 * o0))));
    r1.add(fmaf(o3, o3, fmaf(o2, o2, fmaf(o1, o1, o0 * o0))));
    r2.add(fmaf(x3, x3, fmaf(x2, x2, fmaf(x1, x1, x0 * x0))));
  } else {
    const double x0 = dbl(x.w0), x1 = dbl(x.w1), o0 = dbl(o.w0), o1 = dbl(o.w1);
    r0.dot(x0, o0);
    r0.dot(x1, o1);
    r1.dot(o0, o0);
    r1.dot(o1, o1);
    r2.dot(x0, x0);
    r2.dot(x1, x1);
  }
}

}  // namespace rsv
