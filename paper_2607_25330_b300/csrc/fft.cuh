// Register FFT codelets and warp-distributed pencil FFTs.
//
// A length-N transform ("pencil") is held by T lanes of one warp, N = T * R,
// with T dividing R.  Two register layouts are used:
//   time layout:  lane t, slot m      holds x[t + T*m]            (m < R)
//   freq layout:  lane t, slot k2*B+i holds X[t*B + i + R*k2]      (B = R/T)
// to_freq() maps time -> freq layout (four-step: R-point DFT in registers,
// twiddle w_N^(t*k1), all-to-all through warp shuffles, T-point DFTs);
// to_time() is the mirror image.  Either may use the forward (e^-) or the
// inverse (e^+) sign; transforms are unnormalised.
#pragma once
#include "common.cuh"

// ------------------------------------------------------------ register DFTs
template <int N, bool INV>
struct DFT;

template <bool INV>
struct DFT<1, INV> {
  static __device__ __forceinline__ void run(cf*) {}
};

template <bool INV>
struct DFT<2, INV> {
  static __device__ __forceinline__ void run(cf* x) {
    cf a = x[0], b = x[1];
    x[0] = cadd(a, b);
    x[1] = csub(a, b);
  }
};

template <bool INV>
struct DFT<3, INV> {
  static __device__ __forceinline__ void run(cf* x) {
    constexpr float h = 0.86602540378443864676f;  // sqrt(3)/2
    cf a = x[0], b = x[1], c = x[2];
    cf s = cadd(b, c);
    cf d = csub(b, c);
    cf m = make_float2(a.x - 0.5f * s.x, a.y - 0.5f * s.y);
    cf r = INV ? make_float2(-h * d.y, h * d.x) : make_float2(h * d.y, -h * d.x);  // +-i h d
    x[0] = cadd(a, s);
    x[1] = cadd(m, r);
    x[2] = csub(m, r);
  }
};

template <bool INV>
struct DFT<4, INV> {
  static __device__ __forceinline__ void run(cf* x) {
    cf a = x[0], b = x[1], c = x[2], d = x[3];
    cf s0 = cadd(a, c), d0 = csub(a, c);
    cf s1 = cadd(b, d), d1 = csub(b, d);
    cf r = INV ? ctimesi(d1) : ctimesmi(d1);
    x[0] = cadd(s0, s1);
    x[2] = csub(s0, s1);
    x[1] = cadd(d0, r);
    x[3] = csub(d0, r);
  }
};

// Mixed-radix decimation in time: N = P * Q, P in {4, 2, 3}.
template <int N, bool INV>
struct DFT {
  static constexpr int P = (N % 4 == 0) ? 4 : ((N % 2 == 0) ? 2 : 3);
  static constexpr int Q = N / P;
  static_assert(P * Q == N, "DFT size must be 2^a 3^b");
  static __device__ __forceinline__ void run(cf* x) {
    cf t[N];
    static_for<0, P>([&](auto pp) {
      constexpr int p = decltype(pp)::value;
      cf s[Q];
#pragma unroll
      for (int q = 0; q < Q; ++q) s[q] = x[q * P + p];
      DFT<Q, INV>::run(s);
#pragma unroll
      for (int q = 0; q < Q; ++q) t[p * Q + q] = s[q];
    });
    static_for<0, Q>([&](auto kk) {
      constexpr int k = decltype(kk)::value;
      cf u[P];
      static_for<0, P>([&](auto pp) {
        constexpr int p = decltype(pp)::value;
        u[p] = twmul<N, p * k, INV>(t[p * Q + k]);
      });
      DFT<P, INV>::run(u);
#pragma unroll
      for (int m = 0; m < P; ++m) x[k + Q * m] = u[m];
    });
  }
};

// ------------------------------------------------------------ warp pencils
// LS: lane stride between the T lanes of one pencil (partner of lane bit b is
// lane ^ (b * LS)).  tw: device table exp(-2 pi i m / N), m < N.
template <int N, int T, int LS>
struct Pencil {
  static constexpr int R = N / T;
  static constexpr int B = R / T;
  static_assert(T * R == N && (T == 1 || B * T == R), "pencil needs N = T*R with T | R");

  // all-to-all among the T lanes: slot (x, i) of lane t ends holding slot (t, i) of lane x
  static __device__ __forceinline__ void all2all(cf* v, int t) {
    static_for<0, 5>([&](auto bb) {
      constexpr int b = 1 << decltype(bb)::value;
      if constexpr (b < T) {
        const bool tb = (t & b) != 0;
        static_for<0, T>([&](auto xx) {
          constexpr int x0 = decltype(xx)::value;
          if constexpr ((x0 & b) == 0) {
#pragma unroll
            for (int i = 0; i < B; ++i) {
              const int s0 = x0 * B + i, s1 = (x0 | b) * B + i;
              cf send = tb ? v[s0] : v[s1];
              cf got;
              got.x = __shfl_xor_sync(0xffffffffu, send.x, b * LS);
              got.y = __shfl_xor_sync(0xffffffffu, send.y, b * LS);
              if (tb) v[s0] = got; else v[s1] = got;
            }
          }
        });
      }
    });
  }

  template <bool INV>
  static __device__ __forceinline__ void twiddle(cf* v, int t, const cf* __restrict__ tw) {
    if constexpr (T > 1) {
#pragma unroll
      for (int k = 1; k < R; ++k) {
        cf w = __ldg(tw + t * k);   // t*k < T*R = N
        if (INV) w.y = -w.y;
        v[k] = cmul(v[k], w);
      }
    }
  }

  // time layout -> freq layout
  template <bool INV>
  static __device__ __forceinline__ void to_freq(cf* v, int t, const cf* __restrict__ tw) {
    DFT<R, INV>::run(v);
    if constexpr (T > 1) {
      twiddle<INV>(v, t, tw);
      all2all(v, t);
#pragma unroll
      for (int i = 0; i < B; ++i) {
        cf u[T];
#pragma unroll
        for (int x = 0; x < T; ++x) u[x] = v[x * B + i];
        DFT<T, INV>::run(u);
#pragma unroll
        for (int x = 0; x < T; ++x) v[x * B + i] = u[x];
      }
    }
  }

  // freq layout -> time layout
  template <bool INV>
  static __device__ __forceinline__ void to_time(cf* v, int t, const cf* __restrict__ tw) {
    if constexpr (T > 1) {
#pragma unroll
      for (int i = 0; i < B; ++i) {
        cf u[T];
#pragma unroll
        for (int x = 0; x < T; ++x) u[x] = v[x * B + i];
        DFT<T, INV>::run(u);
#pragma unroll
        for (int x = 0; x < T; ++x) v[x * B + i] = u[x];
      }
      all2all(v, t);
      twiddle<INV>(v, t, tw);
    }
    DFT<R, INV>::run(v);
  }

  // index helpers
  static __device__ __forceinline__ int time_index(int t, int m) { return t + T * m; }
  static __device__ __forceinline__ int freq_index(int t, int slot) {
    const int k2 = slot / B, i = slot - k2 * B;
    return t * B + i + R * k2;
  }
};

// signed FFT-order index: i -> i for i <= (n-1)/2, else i - n
__device__ __forceinline__ int fft_signed(int i, int n) { return (i <= (n - 1) / 2) ? i : i - n; }
