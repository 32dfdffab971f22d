// Register FFT codelets and warp-distributed pencil FFTs.
//
// A length-N transform ("pencil") is held by T lanes of one warp, N = T * R,
// with T dividing R.  Two register layouts are used:
//   time layout:  lane t, slot m      holds x[t + T*m]            (m < R)
//   freq layout:  lane t, slot k2*B+i holds X[t*B + i + R*k2]      (B = R/T)
// to_freq() maps time -> freq layout (four-step: R-point DFT in registers,
// twiddle w_N^(t*k1), all-to-all through warp shuffles or a shared-memory tile,
// T-point DFTs);
// to_time() is the mirror image.  Either may use the forward (e^-) or the
// inverse (e^+) sign; transforms are unnormalised.
#pragma once
#include "common.cuh"

// ------------------------------------------------------------ register DFTs
template <int N, bool INV, class C = cf>
struct DFT;

template <bool INV, class C>
struct DFT<1, INV, C> {
  static __device__ __forceinline__ void run(C*) {}
};

template <bool INV, class C>
struct DFT<2, INV, C> {
  static __device__ __forceinline__ void run(C* x) {
    C a = x[0], b = x[1];
    x[0] = cadd(a, b);
    x[1] = csub(a, b);
  }
};

template <bool INV, class C>
struct DFT<3, INV, C> {
  static __device__ __forceinline__ void run(C* x) {
    using R = typename CTraits<C>::R;
    constexpr R h = (R)0.86602540378443864676;  // sqrt(3)/2
    C a = x[0], b = x[1], c = x[2];
    C s = cadd(b, c);
    C d = csub(b, c);
    C m = CTraits<C>::make(a.x - (R)0.5 * s.x, a.y - (R)0.5 * s.y);
    C r = INV ? CTraits<C>::make(-h * d.y, h * d.x) : CTraits<C>::make(h * d.y, -h * d.x);  // +-i h d
    x[0] = cadd(a, s);
    x[1] = cadd(m, r);
    x[2] = csub(m, r);
  }
};

template <bool INV, class C>
struct DFT<4, INV, C> {
  static __device__ __forceinline__ void run(C* x) {
    C a = x[0], b = x[1], c = x[2], d = x[3];
    C s0 = cadd(a, c), d0 = csub(a, c);
    C s1 = cadd(b, d), d1 = csub(b, d);
    C r = INV ? ctimesi(d1) : ctimesmi(d1);
    x[0] = cadd(s0, s1);
    x[2] = csub(s0, s1);
    x[1] = cadd(d0, r);
    x[3] = csub(d0, r);
  }
};

// Mixed-radix decimation in time: N = P * Q, P in {4, 2, 3}.
template <int N, bool INV, class C>
struct DFT {
  static constexpr int P = (N % 4 == 0) ? 4 : ((N % 2 == 0) ? 2 : 3);
  static constexpr int Q = N / P;
  static_assert(P * Q == N, "DFT size must be 2^a 3^b");
  static __device__ __forceinline__ void run(C* x) {
    C t[N];
    static_for<0, P>([&](auto pp) {
      constexpr int p = decltype(pp)::value;
      C s[Q];
#pragma unroll
      for (int q = 0; q < Q; ++q) s[q] = x[q * P + p];
      DFT<Q, INV, C>::run(s);
#pragma unroll
      for (int q = 0; q < Q; ++q) t[p * Q + q] = s[q];
    });
    static_for<0, Q>([&](auto kk) {
      constexpr int k = decltype(kk)::value;
      C u[P];
      static_for<0, P>([&](auto pp) {
        constexpr int p = decltype(pp)::value;
        u[p] = twmul<N, p * k, INV>(t[p * Q + k]);
      });
      DFT<P, INV, C>::run(u);
#pragma unroll
      for (int m = 0; m < P; ++m) x[k + Q * m] = u[m];
    });
  }
};

// ------------------------------------------------------------ warp pencils
// LS: lane stride between the T lanes of one pencil (partner of lane bit b is
// lane ^ (b * LS)).  tw: device table exp(-2 pi i m / N), m < N.
template <int N, int T, int LS, class C = cf>
struct Pencil {
  static constexpr int R = N / T;
  static constexpr int B = R / T;
  static_assert(T * R == N && (T == 1 || B * T == R), "pencil needs N = T*R with T | R");

  // all-to-all among the T lanes: slot (x, i) of lane t ends holding slot (t, i) of lane x
  static __device__ __forceinline__ void all2all(C* v, int t) {
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
              C send = tb ? v[s0] : v[s1];
              C got;
              got.x = shfl_xor_r(send.x, b * LS);
              got.y = shfl_xor_r(send.y, b * LS);
              if (tb) v[s0] = got; else v[s1] = got;
            }
          }
        });
      }
    });
  }

  // The same all-to-all through a per-warp shared-memory tile of TILE elements (kernels that
  // can spare the shared memory use it: 2R stores and 2R loads per lane instead of
  // B T/2 log2(T) shuffle pairs with their selects).  Lane (t, p) stores its slot (x, i) at
  // tile[(i T + x) XS + lane] and loads slot (s, i) from the entry that lane (s, p) stored for
  // it, tile[(i T + t) XS + lane + (s - t) LS].  With XS = 32 + 1 (LS = 1) or 32 + LS both
  // phases touch 16 distinct 8-byte bank pairs per half warp (and 8 distinct 16-byte ones per
  // quarter warp).
  static constexpr int XS = 32 + (LS == 1 ? 1 : LS);
  static constexpr int TILE = (T > 1) ? R * XS : 1;
  static __device__ __forceinline__ void all2all_smem(C* v, int t, C* tile) {
    static_assert(LS == 1 || LS * T == 32, "pencil lanes are consecutive or 32/T apart");
    const int lane = threadIdx.x & 31;
    __syncwarp();   // the previous exchange through this tile has been read by every lane
    C* w = tile + lane;
#pragma unroll
    for (int i = 0; i < B; ++i)
#pragma unroll
      for (int x = 0; x < T; ++x) w[(i * T + x) * XS] = v[x * B + i];
    __syncwarp();
    const C* r = tile + t * XS + lane - t * LS;
#pragma unroll
    for (int i = 0; i < B; ++i)
#pragma unroll
      for (int s = 0; s < T; ++s) v[s * B + i] = r[i * T * XS + s * LS];
  }

  template <bool INV>
  static __device__ __forceinline__ void twiddle(C* v, int t, const C* __restrict__ tw) {
    if constexpr (T > 1) {
#pragma unroll
      for (int k = 1; k < R; ++k) {
        C w = ld_tw(tw + t * k);   // t*k < T*R = N
        if (INV) w.y = -w.y;
        v[k] = cmul(v[k], w);
      }
    }
  }

  // time layout -> freq layout; SM: exchange through this warp's tile (all2all_smem), else shuffles
  template <bool INV, bool SM>
  static __device__ __forceinline__ void to_freq_impl(C* v, int t, const C* __restrict__ tw, C* tile) {
    DFT<R, INV, C>::run(v);
    if constexpr (T > 1) {
      twiddle<INV>(v, t, tw);
      if constexpr (SM) all2all_smem(v, t, tile);
      else all2all(v, t);
#pragma unroll
      for (int i = 0; i < B; ++i) {
        C u[T];
#pragma unroll
        for (int x = 0; x < T; ++x) u[x] = v[x * B + i];
        DFT<T, INV, C>::run(u);
#pragma unroll
        for (int x = 0; x < T; ++x) v[x * B + i] = u[x];
      }
    }
  }

  // freq layout -> time layout
  template <bool INV, bool SM>
  static __device__ __forceinline__ void to_time_impl(C* v, int t, const C* __restrict__ tw, C* tile) {
    if constexpr (T > 1) {
#pragma unroll
      for (int i = 0; i < B; ++i) {
        C u[T];
#pragma unroll
        for (int x = 0; x < T; ++x) u[x] = v[x * B + i];
        DFT<T, INV, C>::run(u);
#pragma unroll
        for (int x = 0; x < T; ++x) v[x * B + i] = u[x];
      }
      if constexpr (SM) all2all_smem(v, t, tile);
      else all2all(v, t);
      twiddle<INV>(v, t, tw);
    }
    DFT<R, INV, C>::run(v);
  }

  template <bool INV>
  static __device__ __forceinline__ void to_freq(C* v, int t, const C* __restrict__ tw) {
    to_freq_impl<INV, false>(v, t, tw, nullptr);
  }
  template <bool INV>
  static __device__ __forceinline__ void to_freq(C* v, int t, const C* __restrict__ tw, C* tile) {
    to_freq_impl<INV, true>(v, t, tw, tile);
  }
  template <bool INV>
  static __device__ __forceinline__ void to_time(C* v, int t, const C* __restrict__ tw) {
    to_time_impl<INV, false>(v, t, tw, nullptr);
  }
  template <bool INV>
  static __device__ __forceinline__ void to_time(C* v, int t, const C* __restrict__ tw, C* tile) {
    to_time_impl<INV, true>(v, t, tw, tile);
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
