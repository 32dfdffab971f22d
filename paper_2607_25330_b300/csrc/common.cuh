// Common device helpers: complex64 arithmetic, compile-time trigonometry,
// compile-time loops and error reporting.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <type_traits>

typedef float2 cf;

__host__ __device__ __forceinline__ cf mk(float re, float im) { return make_float2(re, im); }
__device__ __forceinline__ cf cadd(cf a, cf b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ cf csub(cf a, cf b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ cf cmul(cf a, cf b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ cf cmulc(cf a, cf b) {  // a * conj(b)
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ cf cconj(cf a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ cf cscale(cf a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ cf ctimesi(cf a) { return make_float2(-a.y, a.x); }     // i a
__device__ __forceinline__ cf ctimesmi(cf a) { return make_float2(a.y, -a.x); }    // -i a
__device__ __forceinline__ cf cfma(cf a, cf b, cf c) {                                 // a*b + c
  return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y)));
}
__device__ __forceinline__ cf czero() { return make_float2(0.f, 0.f); }
__device__ __forceinline__ cf cneg(cf a) { return make_float2(-a.x, -a.y); }

// complex128 overloads (same names) for the FP64 residual path
typedef double2 zd;
__device__ __forceinline__ zd cadd(zd a, zd b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ zd csub(zd a, zd b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ zd cmul(zd a, zd b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ zd cscale(zd a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ zd ctimesi(zd a) { return make_double2(-a.y, a.x); }
__device__ __forceinline__ zd ctimesmi(zd a) { return make_double2(a.y, -a.x); }
__device__ __forceinline__ zd cfma(zd a, zd b, zd c) {
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}

// warp shuffle and twiddle-table load by value type (overloaded for the double-float type)
__device__ __forceinline__ float shfl_xor_r(float v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
__device__ __forceinline__ double shfl_xor_r(double v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
__device__ __forceinline__ cf ld_tw(const cf* p) { return __ldg(p); }
__device__ __forceinline__ zd ld_tw(const zd* p) { return __ldg(p); }

template <class C> struct CTraits;
template <> struct CTraits<cf> {
  using R = float;
  static __device__ __forceinline__ cf zero() { return make_float2(0.f, 0.f); }
  static __device__ __forceinline__ cf make(float a, float b) { return make_float2(a, b); }
};
template <> struct CTraits<zd> {
  using R = double;
  static __device__ __forceinline__ zd zero() { return make_double2(0.0, 0.0); }
  static __device__ __forceinline__ zd make(double a, double b) { return make_double2(a, b); }
};

// ------------------------------------------------------------ compile-time loops
template <int B, int E, class F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    static_for<B + 1, E>(f);
  }
}

// ------------------------------------------------------------ compile-time trigonometry
// sin / cos of 2*pi*J/N evaluated at compile time: exact integer reduction to
// [0, pi/4] followed by a Taylor series (error far below float rounding).
namespace ct {
constexpr double kPi = 3.14159265358979323846264338327950288;
constexpr double sin_small(double x) {
  double t = x, s = x;
  for (int n = 1; n < 16; ++n) { t *= -x * x / double((2 * n) * (2 * n + 1)); s += t; }
  return s;
}
constexpr double cos_small(double x) {
  double t = 1.0, s = 1.0;
  for (int n = 1; n < 16; ++n) { t *= -x * x / double((2 * n - 1) * (2 * n)); s += t; }
  return s;
}
struct SinCos { double s, c; };
constexpr SinCos sincos2pi(long J, long N) {
  long j = ((J % N) + N) % N;
  long q = (4 * j) / N;
  long rem = 4 * j - q * N;  // angle = q*pi/2 + (pi/2) * rem / N
  double s = 0, c = 0;
  if (2 * rem <= N) {
    double x = (kPi / 2) * double(rem) / double(N);
    s = sin_small(x); c = cos_small(x);
  } else {
    double x = (kPi / 2) * double(N - rem) / double(N);
    s = cos_small(x); c = sin_small(x);
  }
  switch (q & 3) {
    case 0: return {s, c};
    case 1: return {c, -s};
    case 2: return {-s, -c};
    default: return {-c, s};
  }
}
}  // namespace ct

// a * exp(sign * 2 pi i J / N) with sign = -1 (forward) or +1 (INV); the
// special angles become sign flips and swaps.
template <int N, int J, bool INV, class C>
__device__ __forceinline__ C twmul(C a) {
  using R = typename CTraits<C>::R;
  constexpr int j = ((J % N) + N) % N;
  if constexpr (j == 0) {
    return a;
  } else if constexpr (2 * j == N) {
    return CTraits<C>::make(-a.x, -a.y);
  } else if constexpr (4 * j == N) {
    return INV ? ctimesi(a) : ctimesmi(a);
  } else if constexpr (4 * j == 3 * N) {
    return INV ? ctimesmi(a) : ctimesi(a);
  } else {
    constexpr ct::SinCos sc = ct::sincos2pi(j, N);
    constexpr R c = (R)sc.c;
    constexpr R s = INV ? (R)sc.s : (R)(-sc.s);
    return CTraits<C>::make(a.x * c - a.y * s, a.x * s + a.y * c);
  }
}

// ------------------------------------------------------------ host error helpers
#define PSFD_CUDA_TRY(expr)                                                  \
  do {                                                                       \
    cudaError_t err__ = (expr);                                              \
    if (err__ != cudaSuccess) {                                              \
      psfd_set_error("%s:%d: %s: %s", __FILE__, __LINE__, #expr,             \
                     cudaGetErrorString(err__));                             \
      return PSFD_ERR_CUDA;                                                  \
    }                                                                        \
  } while (0)

#define PSFD_CHECK_LAUNCH()                                                  \
  do {                                                                       \
    psfd_count_launch();                                                     \
    cudaError_t err__ = cudaGetLastError();                                  \
    if (err__ != cudaSuccess) {                                              \
      psfd_set_error("%s:%d: launch: %s", __FILE__, __LINE__,                \
                     cudaGetErrorString(err__));                             \
      return PSFD_ERR_CUDA;                                                  \
    }                                                                        \
  } while (0)

void psfd_set_error(const char* fmt, ...);
void psfd_count_launch();

// Optional per-stage timing with CUDA events on the launching stream.
enum { ST_AXIAL = 0, ST_CONTRAST = 1, ST_KRYLOV = 2, ST_TRANSFORM = 3, ST_FNO = 4, ST_PRECOND = 5, ST_LAYBUILD = 6,
       ST_N = 7 };
// `bytes` is the stage's algorithmic traffic: the compulsory reads and writes of its
// inputs and outputs (intermediate passes of a multi-kernel stage are not counted).
void stage_mark(cudaStream_t s, int stage, bool begin, double bytes = 0.0);
struct StageScope {
  cudaStream_t s;
  int st;
  double bytes;
  StageScope(cudaStream_t s_, int st_, double bytes_ = 0.0) : s(s_), st(st_), bytes(bytes_) {
    stage_mark(s, st, true);
  }
  ~StageScope() { stage_mark(s, st, false, bytes); }
};
