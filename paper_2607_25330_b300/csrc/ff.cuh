// Double-float arithmetic for the refinement residual.
//
// B300 runs FP64 at a small fraction of its FP32 rate, and the outer residual b - A E of the
// mixed-precision solve only has to be accurate well below the 1e-6 target.  A value is kept as
// an unevaluated sum hi + lo of two floats (|lo| <= ulp(hi) / 2, about 48 significant bits),
// and the operations are the error-free transformations of Dekker (1971) and Knuth (TAOCP
// vol. 2, 4.2.2): Knuth's two-sum for the exact rounding error of a sum, Dekker's fast two-sum
// when the larger operand is known, and an FMA for the exact rounding error of a product.
// Sums are the "sloppy" variant (lo parts added once), whose error is about 2^-44 of
// |a| + |b|: the same error model as the FFT butterflies they sit in.  The fields stay FP64 in
// memory; they are split on load and joined on store.
#pragma once
#include "common.cuh"

struct ff {
  float hi, lo;
  ff() = default;
  __host__ __device__ constexpr ff(float h, float l) : hi(h), lo(l) {}
  // nearest float, then the float nearest to the remainder
  __host__ __device__ constexpr ff(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
};

__device__ __forceinline__ ff ff_fast_two_sum(float a, float b) {   // |a| >= |b| or a == 0
  const float s = __fadd_rn(a, b);
  return ff(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ ff ff_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float v = __fsub_rn(s, a);
  return ff(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v)));
}
__device__ __forceinline__ ff operator+(ff a, ff b) {
  const ff s = ff_two_sum(a.hi, b.hi);
  return ff_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ ff operator-(ff a) { return ff(-a.hi, -a.lo); }
__device__ __forceinline__ ff operator-(ff a, ff b) { return a + (-b); }
__device__ __forceinline__ ff operator*(ff a, ff b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);   // exact rounding error of a.hi b.hi
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return ff_fast_two_sum(p, e);
}
__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }

// complex double-float
struct cff {
  ff x, y;
};
__device__ __forceinline__ cff mkc(ff re, ff im) { cff c; c.x = re; c.y = im; return c; }
__device__ __forceinline__ cff to_cff(zd a) { return mkc(ff(a.x), ff(a.y)); }
__device__ __forceinline__ zd to_zd(cff a) { return make_double2(ff_to_double(a.x), ff_to_double(a.y)); }
__device__ __forceinline__ cff cadd(cff a, cff b) { return mkc(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ cff csub(cff a, cff b) { return mkc(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ cff cmul(cff a, cff b) { return mkc(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ cff cscale(cff a, ff s) { return mkc(a.x * s, a.y * s); }
__device__ __forceinline__ cff ctimesi(cff a) { return mkc(-a.y, a.x); }
__device__ __forceinline__ cff ctimesmi(cff a) { return mkc(a.y, -a.x); }
__device__ __forceinline__ cff cfma(cff a, cff b, cff c) { return cadd(cmul(a, b), c); }

template <> struct CTraits<cff> {
  using R = ff;
  static __device__ __forceinline__ cff zero() { return mkc(ff(0.f, 0.f), ff(0.f, 0.f)); }
  static __device__ __forceinline__ cff make(ff a, ff b) { return mkc(a, b); }
};

__device__ __forceinline__ ff shfl_xor_r(ff v, int m) {
  return ff(__shfl_xor_sync(0xffffffffu, v.hi, m), __shfl_xor_sync(0xffffffffu, v.lo, m));
}
__device__ __forceinline__ cff ld_tw(const cff* p) {
  const float4 q = __ldg(reinterpret_cast<const float4*>(p));
  return mkc(ff(q.x, q.y), ff(q.z, q.w));
}

// generic helpers over the compute type C (cff or zd) of the extended-precision kernels
template <class C> __device__ __forceinline__ C from_zd(zd a);
template <> __device__ __forceinline__ cff from_zd<cff>(zd a) { return to_cff(a); }
template <> __device__ __forceinline__ zd from_zd<zd>(zd a) { return a; }
__device__ __forceinline__ zd to_zd(zd a) { return a; }

// the table of the compute type: double-float copy or the FP64 original
template <class C> __device__ __forceinline__ const C* pick_tab(const cff* f, const zd* d);
template <> __device__ __forceinline__ const cff* pick_tab<cff>(const cff* f, const zd*) { return f; }
template <> __device__ __forceinline__ const zd* pick_tab<zd>(const cff*, const zd* d) { return d; }
template <class C> __device__ __forceinline__ const typename CTraits<C>::R* pick_real(const ff* f, const double* d);
template <> __device__ __forceinline__ const ff* pick_real<cff>(const ff* f, const double*) { return f; }
template <> __device__ __forceinline__ const double* pick_real<zd>(const ff*, const double* d) { return d; }

// double-float where a thread holds at most 16 points of a transform; larger register codelets in
// double-float take ptxas tens of minutes, so those stay FP64
template <int N, int T>
using ExtC = typename std::conditional<(N / T <= 16), cff, zd>::type;
