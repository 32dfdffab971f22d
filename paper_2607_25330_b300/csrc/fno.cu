// Factorised Fourier neural operator forward pass (Sec. 2.1, Eqs. 1-5) and
// spectral zero-padding upsampling of a coarse prediction.
//
// Layout: hidden fields are float32 [B][C][nz][ny][nx] (channel planes).
// Per layer:
//   xy branch (Eq. 2): x-FFT of every row keeping the mx retained kx, y-FFT of
//     the retained columns keeping my ky -> V[mode][i][b*nz+z]; per-mode channel
//     mixing U = K V (operands rounded to bfloat16, float32 accumulation);
//     zero-padded inverse y- and x-FFTs, real part -> u_xy.
//   z branch (Eq. 3): z-FFT of u_xy keeping mz kz -> per-kz mixing -> zero-padded
//     inverse z-FFT, real part -> u_z.
//   pointwise MLP with residual (Eq. 4), GELU (erf form) inside and, except in
//     the last layer, outside.
// Lift: (a, x/nx, y/ny, z/nz) -> dv.  Projection: dv -> dq -> 6 (Re/Im of E).
#include <mutex>
#include <cuda_bf16.h>

#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <vector>

#include "fft.cuh"
#include "internal.h"
#include "pdl.cuh"

namespace {

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

struct Dims {
  int B, C, nx, ny, nz;   // C = channels of the transformed field
  int mx, my, mz;          // retained modes actually present on this grid
  int MX, MY, MZ;          // mode-table sizes of the weights
};

// FFT index -> kept index j in [0, m) (signed k = j - m/2), or -1
__device__ __forceinline__ int fft_to_kept(int idx, int m, int n) {
  int k = fft_signed(idx, n);
  int lo = -(m / 2), hi = m - m / 2;  // [lo, hi)
  return (k >= lo && k < hi) ? k - lo : -1;
}

// ---------------------------------------------------------------- x-FFT of real rows -> kept kx
// rows r over [B*C*nz*ny]; out T1[r][mx] complex
template <int NX, int T>
__global__ void __launch_bounds__(128) k_xfwd(const float* __restrict__ v, cf* __restrict__ T1, long nrows, int mx,
                                              const cf* __restrict__ tw) {
  pdl_enter();
  constexpr int P = 32 / T, R = NX / T;
  using PX = Pencil<NX, T, 1>;
  __shared__ cf xch[4][PX::TILE];   // per-warp exchange tiles (4 warps per block)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  cf* const xt = xch[warp];
  const int p = lane / T, t = lane - p * T;
  const long row = ((long)blockIdx.x * (blockDim.x >> 5) + warp) * P + p;
  const bool act = row < nrows;
  const float* src = v + (act ? row : 0) * NX;
  cf w[R];
#pragma unroll
  for (int m = 0; m < R; ++m) w[m] = make_float2(act ? src[t + T * m] : 0.f, 0.f);
  PX::template to_freq<false>(w, t, tw, xt);
#pragma unroll
  for (int s = 0; s < R; ++s) {
    const int j = fft_to_kept(PX::freq_index(t, s), mx, NX);
    if (act && j >= 0) T1[row * mx + j] = w[s];
  }
}

// ---------------------------------------------------------------- y-FFT of kept columns -> V[mode][c][n]
// columns over [B*C*nz] planes x mx; plane (b, c, z) -> n = b*nz + z
template <int NY, int T>
__global__ void __launch_bounds__(128) k_yfwd(const cf* __restrict__ T1, cf* __restrict__ V, Dims d,
                                              const cf* __restrict__ tw) {
  pdl_enter();
  constexpr int P = 32 / T, R = NY / T;
  using PY = Pencil<NY, T, P>;
  __shared__ cf xch[4][PY::TILE];   // per-warp exchange tiles (4 warps per block)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  cf* const xt = xch[warp];
  const int t = lane / P, p = lane - t * P;
  const long colid = ((long)blockIdx.x * (blockDim.x >> 5) + warp) * P + p;
  const long ncol = (long)d.B * d.C * d.nz * d.mx;
  const bool act = colid < ncol;
  const long cid = act ? colid : 0;
  const long plane = cid / d.mx;
  const int kx = (int)(cid - plane * d.mx);
  const cf* base = T1 + plane * (long)NY * d.mx + kx;
  cf w[R];
#pragma unroll
  for (int m = 0; m < R; ++m) w[m] = act ? base[(long)(t + T * m) * d.mx] : czero();
  PY::template to_freq<false>(w, t, tw, xt);
  const int z = (int)(plane % d.nz);
  const long bc = plane / d.nz;
  const int c = (int)(bc % d.C);
  const long b = bc / d.C;
  const long n = b * d.nz + z, NB = (long)d.B * d.nz;
#pragma unroll
  for (int s = 0; s < R; ++s) {
    const int jy = fft_to_kept(PY::freq_index(t, s), d.my, NY);
    if (act && jy >= 0) {
      const long mode = (long)jy * d.mx + kx;
      V[(mode * d.C + c) * NB + n] = w[s];
    }
  }
}

// ---------------------------------------------------------------- per-mode channel mixing
// U[mode][o][n] = sum_i K[row(mode)][o][i] V[mode][i][n]; bf16 operands, fp32 accumulation.
// K table rows: xy -> (jy + (MY-my)/2) * MX + (jx + (MX-mx)/2); z -> jz + (MZ-mz)/2.
constexpr int MIX_TN = 64;
__global__ void __launch_bounds__(256) k_mix(const cf* __restrict__ V, cf* __restrict__ U, const cf* __restrict__ K,
                                             int C, long NB, int mx, int MX, int offy, int offx, bool conjT = false,
                                             bool round_v = true, bool round_k = true) {
  pdl_enter();
  extern __shared__ float sm[];
  float* Kr = sm;                       // [C][C]
  float* Ki = Kr + C * C;
  float* Vr = Ki + C * C;               // [C][MIX_TN]
  float* Vi = Vr + C * MIX_TN;
  const long mode = blockIdx.y;
  const int jy = (int)(mode / mx), jx = (int)(mode - (long)jy * mx);
  const long krow = (long)(jy + offy) * MX + (jx + offx);
  const cf* Km = K + krow * C * C;
  for (int e = threadIdx.x; e < C * C; e += blockDim.x) {
    // conjT: the adjoint mixing uses K^H, i.e. entry (o, i) = conj(K[i][o])
    const int o = e / C, i = e - o * C;
    cf k = conjT ? Km[i * C + o] : Km[e];
    const float kr = round_k ? bf16r(k.x) : k.x, ki = round_k ? bf16r(k.y) : k.y;
    Kr[e] = kr;
    Ki[e] = conjT ? -ki : ki;
  }
  const long n0 = (long)blockIdx.x * MIX_TN;
  const cf* Vm = V + mode * C * NB;
  for (int e = threadIdx.x; e < C * MIX_TN; e += blockDim.x) {
    const int i = e / MIX_TN, j = e - i * MIX_TN;
    cf x = (n0 + j < NB) ? Vm[(long)i * NB + n0 + j] : czero();
    Vr[e] = round_v ? bf16r(x.x) : x.x;
    Vi[e] = round_v ? bf16r(x.y) : x.y;
  }
  __syncthreads();
  cf* Um = U + mode * C * NB;
  for (int e = threadIdx.x; e < C * MIX_TN; e += blockDim.x) {
    const int o = e / MIX_TN, j = e - o * MIX_TN;
    float re = 0.f, im = 0.f;
#pragma unroll 8
    for (int i = 0; i < C; ++i) {
      const float kr = Kr[o * C + i], ki = Ki[o * C + i];
      const float vr = Vr[i * MIX_TN + j], vi = Vi[i * MIX_TN + j];
      re = fmaf(kr, vr, fmaf(-ki, vi, re));
      im = fmaf(kr, vi, fmaf(ki, vr, im));
    }
    if (n0 + j < NB) Um[(long)o * NB + n0 + j] = make_float2(re, im);
  }
}

// ---------------------------------------------------------------- mixing weight gradient
// dK[row(mode)][o][i] += sum_n Ubar[mode][o][n] conj(bf16(V[mode][i][n])): the gradient of the
// bf16-rounded mixing with the rounding passed straight through.  Each block reduces a chunk
// of n in tiles of MIX_TN and adds its partial sums to dK with atomics.
constexpr int GRAD_CHUNK = 2048;
__global__ void __launch_bounds__(256) k_mixgrad(const cf* __restrict__ Ubar, const cf* __restrict__ V,
                                                 float* __restrict__ dK, int C, long NB, int mx, int MX, int offy,
                                                 int offx, float scale) {
  pdl_enter();
  __shared__ float Ur[32][MIX_TN + 1], Ui[32][MIX_TN + 1], Vr[32][MIX_TN + 1], Vi[32][MIX_TN + 1];
  const long mode = blockIdx.y;
  const int jy = (int)(mode / mx), jx = (int)(mode - (long)jy * mx);
  const long krow = (long)(jy + offy) * MX + (jx + offx);
  const cf* Um = Ubar + mode * C * NB;
  const cf* Vm = V + mode * C * NB;
  // each thread owns 4 (o, i) entries: e = threadIdx.x + 256 q; each tile's fp32 partial sum is
  // added to an FP64 total (a chunk is up to GRAD_CHUNK terms of mixed sign)
  double ar[4] = {0, 0, 0, 0}, ai[4] = {0, 0, 0, 0};
  const long n_begin = (long)blockIdx.x * GRAD_CHUNK;
  const long n_end = min(NB, n_begin + GRAD_CHUNK);
  for (long n0 = n_begin; n0 < n_end; n0 += MIX_TN) {
    __syncthreads();
    for (int e = threadIdx.x; e < C * MIX_TN; e += blockDim.x) {
      const int c = e / MIX_TN, j = e - c * MIX_TN;
      const bool in = n0 + j < n_end;
      const cf u = in ? Um[(long)c * NB + n0 + j] : czero();
      const cf v = in ? Vm[(long)c * NB + n0 + j] : czero();
      Ur[c][j] = u.x; Ui[c][j] = u.y;
      Vr[c][j] = bf16r(v.x); Vi[c][j] = bf16r(v.y);
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = threadIdx.x + 256 * q;
      const int o = e / 32, i = e - o * 32;
      float tr = 0.f, ti = 0.f;
#pragma unroll 8
      for (int j = 0; j < MIX_TN; ++j) {
        // u * conj(v)
        tr = fmaf(Ur[o][j], Vr[i][j], fmaf(Ui[o][j], Vi[i][j], tr));
        ti = fmaf(Ui[o][j], Vr[i][j], fmaf(-Ur[o][j], Vi[i][j], ti));
      }
      ar[q] += tr;
      ai[q] += ti;
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int e = threadIdx.x + 256 * q;
    float* dst = dK + 2 * (krow * C * C + e);
    atomicAdd(dst, (float)(ar[q] * scale));
    atomicAdd(dst + 1, (float)(ai[q] * scale));
  }
}

// ---------------------------------------------------------------- inverse y: U -> T2[plane][y][mx]
template <int NY, int T>
__global__ void __launch_bounds__(128) k_yinv(const cf* __restrict__ U, cf* __restrict__ T2, Dims d,
                                              const cf* __restrict__ tw) {
  pdl_enter();
  constexpr int P = 32 / T, R = NY / T;
  using PY = Pencil<NY, T, P>;
  __shared__ cf xch[4][PY::TILE];   // per-warp exchange tiles (4 warps per block)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  cf* const xt = xch[warp];
  const int t = lane / P, p = lane - t * P;
  const long colid = ((long)blockIdx.x * (blockDim.x >> 5) + warp) * P + p;
  const long ncol = (long)d.B * d.C * d.nz * d.mx;
  const bool act = colid < ncol;
  const long cid = act ? colid : 0;
  const long plane = cid / d.mx;
  const int kx = (int)(cid - plane * d.mx);
  const int z = (int)(plane % d.nz);
  const long bc = plane / d.nz;
  const int c = (int)(bc % d.C);
  const long b = bc / d.C;
  const long n = b * d.nz + z, NB = (long)d.B * d.nz;
  cf w[R];
#pragma unroll
  for (int s = 0; s < R; ++s) {
    const int jy = fft_to_kept(PY::freq_index(t, s), d.my, NY);
    w[s] = (act && jy >= 0) ? U[(((long)jy * d.mx + kx) * d.C + c) * NB + n] : czero();
  }
  PY::template to_time<true>(w, t, tw, xt);
  cf* base = T2 + plane * (long)NY * d.mx + kx;
#pragma unroll
  for (int m = 0; m < R; ++m)
    if (act) base[(long)(t + T * m) * d.mx] = w[m];
}

// ---------------------------------------------------------------- inverse x: T2 rows -> real out * scale
template <int NX, int T>
__global__ void __launch_bounds__(128) k_xinv(const cf* __restrict__ T2, float* __restrict__ out, long nrows, int mx,
                                              float scale, const cf* __restrict__ tw) {
  pdl_enter();
  constexpr int P = 32 / T, R = NX / T;
  using PX = Pencil<NX, T, 1>;
  __shared__ cf xch[4][PX::TILE];   // per-warp exchange tiles (4 warps per block)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  cf* const xt = xch[warp];
  const int p = lane / T, t = lane - p * T;
  const long row = ((long)blockIdx.x * (blockDim.x >> 5) + warp) * P + p;
  const bool act = row < nrows;
  const long r = act ? row : 0;
  cf w[R];
#pragma unroll
  for (int s = 0; s < R; ++s) {
    const int j = fft_to_kept(PX::freq_index(t, s), mx, NX);
    w[s] = (act && j >= 0) ? T2[r * mx + j] : czero();
  }
  PX::template to_time<true>(w, t, tw, xt);
#pragma unroll
  for (int m = 0; m < R; ++m)
    if (act) out[r * NX + t + T * m] = w[m].x * scale;
}

// ---------------------------------------------------------------- z branch
// forward: columns (b, c, yx) along z of real u -> W[kz][c][b*nxy + yx]
template <int NZ, int T>
__global__ void __launch_bounds__(128) k_zfwd(const float* __restrict__ u, cf* __restrict__ W, Dims d,
                                              const cf* __restrict__ tw) {
  pdl_enter();
  constexpr int P = 32 / T, R = NZ / T;
  using PZ = Pencil<NZ, T, P>;
  __shared__ cf xch[4][PZ::TILE];   // per-warp exchange tiles (4 warps per block)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  cf* const xt = xch[warp];
  const int t = lane / P, p = lane - t * P;
  const long nxy = (long)d.nx * d.ny;
  const long colid = ((long)blockIdx.x * (blockDim.x >> 5) + warp) * P + p;
  const long ncol = (long)d.B * d.C * nxy;
  const bool act = colid < ncol;
  const long cid = act ? colid : 0;
  const long bc = cid / nxy, yx = cid - bc * nxy;
  const int c = (int)(bc % d.C);
  const long b = bc / d.C;
  const float* base = u + bc * NZ * nxy + yx;
  cf w[R];
#pragma unroll
  for (int m = 0; m < R; ++m) w[m] = make_float2(act ? base[(long)(t + T * m) * nxy] : 0.f, 0.f);
  PZ::template to_freq<false>(w, t, tw, xt);
  const long NB = (long)d.B * nxy, n = b * nxy + yx;
#pragma unroll
  for (int s = 0; s < R; ++s) {
    const int jz = fft_to_kept(PZ::freq_index(t, s), d.mz, NZ);
    if (act && jz >= 0) W[((long)jz * d.C + c) * NB + n] = w[s];
  }
}

template <int NZ, int T>
__global__ void __launch_bounds__(128) k_zinv(const cf* __restrict__ U, float* __restrict__ out, Dims d, float scale,
                                              const cf* __restrict__ tw) {
  pdl_enter();
  constexpr int P = 32 / T, R = NZ / T;
  using PZ = Pencil<NZ, T, P>;
  __shared__ cf xch[4][PZ::TILE];   // per-warp exchange tiles (4 warps per block)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  cf* const xt = xch[warp];
  const int t = lane / P, p = lane - t * P;
  const long nxy = (long)d.nx * d.ny;
  const long colid = ((long)blockIdx.x * (blockDim.x >> 5) + warp) * P + p;
  const long ncol = (long)d.B * d.C * nxy;
  const bool act = colid < ncol;
  const long cid = act ? colid : 0;
  const long bc = cid / nxy, yx = cid - bc * nxy;
  const int c = (int)(bc % d.C);
  const long b = bc / d.C;
  const long NB = (long)d.B * nxy, n = b * nxy + yx;
  cf w[R];
#pragma unroll
  for (int s = 0; s < R; ++s) {
    const int jz = fft_to_kept(PZ::freq_index(t, s), d.mz, NZ);
    w[s] = (act && jz >= 0) ? U[((long)jz * d.C + c) * NB + n] : czero();
  }
  PZ::template to_time<true>(w, t, tw, xt);
  float* base = out + bc * NZ * nxy + yx;
#pragma unroll
  for (int m = 0; m < R; ++m)
    if (act) base[(long)(t + T * m) * nxy] = w[m].x * scale;
}

// ---------------------------------------------------------------- pointwise layers
__global__ void k_lift(const float* __restrict__ a, float* __restrict__ v, const float* __restrict__ W,
                       const float* __restrict__ bias, int B, int C, int nx, int ny, int nz) {
  pdl_enter();
  const long N = (long)nx * ny * nz;
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long)B * N) return;
  const long b = i / N, pt = i - b * N;
  const int x = (int)(pt % nx), y = (int)((pt / nx) % ny), z = (int)(pt / ((long)nx * ny));
  const float in0 = a[i], in1 = (float)x / nx, in2 = (float)y / ny, in3 = (float)z / nz;
  for (int c = 0; c < C; ++c) {
    const float* w = W + c * 4;
    v[(b * C + c) * N + pt] = fmaf(w[0], in0, fmaf(w[1], in1, fmaf(w[2], in2, fmaf(w[3], in3, bias[c]))));
  }
}

// v_out = v_in + s(W2 gelu(W1 (uxy + uz) + b1) + b2); C = dv <= 64, H = dh <= 128; v_out may alias v_in
template <int C, int H>
__global__ void __launch_bounds__(128) k_mlp(const float* vin, float* vout, const float* __restrict__ uxy,
                                             const float* __restrict__ uz, const float* __restrict__ W1,
                                             const float* __restrict__ b1, const float* __restrict__ W2,
                                             const float* __restrict__ b2, long N, int B, bool outer_gelu) {
  pdl_enter();
  __shared__ float w1[H * C], w2[C * H], sb1[H], sb2[C];
  for (int e = threadIdx.x; e < H * C; e += blockDim.x) { w1[e] = W1[e]; w2[e] = W2[e]; }
  for (int e = threadIdx.x; e < H; e += blockDim.x) sb1[e] = b1[e];
  for (int e = threadIdx.x; e < C; e += blockDim.x) sb2[e] = b2[e];
  __syncthreads();
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long)B * N) return;
  const long b = i / N, pt = i - b * N;
  const long base = b * C * N + pt;
  float h[C], o[C];
#pragma unroll
  for (int c = 0; c < C; ++c) { h[c] = uxy[base + c * N] + uz[base + c * N]; o[c] = sb2[c]; }
#pragma unroll 2
  for (int j = 0; j < H; ++j) {
    float s = sb1[j];
#pragma unroll
    for (int c = 0; c < C; ++c) s = fmaf(w1[j * C + c], h[c], s);
    const float g = gelu(s);
#pragma unroll
    for (int c = 0; c < C; ++c) o[c] = fmaf(w2[c * H + j], g, o[c]);
  }
#pragma unroll
  for (int c = 0; c < C; ++c) vout[base + c * N] = vin[base + c * N] + (outer_gelu ? gelu(o[c]) : o[c]);
}

template <int C, int Q>
__global__ void __launch_bounds__(128) k_proj(const float* __restrict__ v, cf* __restrict__ E, const float* __restrict__ Q1,
                                              const float* __restrict__ qb1, const float* __restrict__ Q2,
                                              const float* __restrict__ qb2, long N, int B) {
  pdl_enter();
  __shared__ float q1[Q * C], q2[6 * Q], sb1[Q], sb2[6];
  for (int e = threadIdx.x; e < Q * C; e += blockDim.x) q1[e] = Q1[e];
  for (int e = threadIdx.x; e < 6 * Q; e += blockDim.x) q2[e] = Q2[e];
  for (int e = threadIdx.x; e < Q; e += blockDim.x) sb1[e] = qb1[e];
  if (threadIdx.x < 6) sb2[threadIdx.x] = qb2[threadIdx.x];
  __syncthreads();
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long)B * N) return;
  const long b = i / N, pt = i - b * N;
  float h[C], o[6];
#pragma unroll
  for (int c = 0; c < C; ++c) h[c] = v[(b * C + c) * N + pt];
#pragma unroll
  for (int k = 0; k < 6; ++k) o[k] = sb2[k];
#pragma unroll 2
  for (int j = 0; j < Q; ++j) {
    float s = sb1[j];
#pragma unroll
    for (int c = 0; c < C; ++c) s = fmaf(q1[j * C + c], h[c], s);
    const float g = gelu(s);
#pragma unroll
    for (int k = 0; k < 6; ++k) o[k] = fmaf(q2[k * Q + j], g, o[k]);
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) E[(b * 3 + c) * N + pt] = make_float2(o[2 * c], o[2 * c + 1]);
}

// ---------------------------------------------------------------- pointwise backward
// One point per thread.  The per-point gradients go to global memory; the point's
// vectors are also staged in shared memory ([feature][point], a tile of BW_TILE
// points, row stride BW_LD so that the column reads below hit distinct banks),
// and the weight gradients (sums over points of outer products) are accumulated
// in 4x4 register blocks and added to global memory once per block.
constexpr int BW_TILE = 128;
constexpr int BW_LD = BW_TILE + 1;

// acc[u][w] += sum_p X[a0+u][p] Y[b0+w][p]
__device__ __forceinline__ void outer4(float (&acc)[4][4], const float* X, int a0, const float* Y, int b0) {
#pragma unroll 4
  for (int p = 0; p < BW_TILE; ++p) {
    float x[4], y[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) { x[u] = X[(a0 + u) * BW_LD + p]; y[u] = Y[(b0 + u) * BW_LD + p]; }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int w = 0; w < 4; ++w) acc[u][w] = fmaf(x[u], y[w], acc[u][w]);
  }
}

// d/dx of the erf-form GELU: Phi(x) + x phi(x)
__device__ __forceinline__ float gelu_grad(float x) {
  const float cdf = 0.5f * (1.0f + erff(x * 0.70710678118654752f));
  const float pdf = 0.39894228040143268f * expf(-0.5f * x * x);
  return fmaf(x, pdf, cdf);
}

template <int C, int H>
constexpr size_t mlp_bwd_smem() { return (size_t)(2 * H * C + H + C + (2 * H + 2 * C) * BW_LD) * sizeof(float); }

// Backward of v_out = v_in + s(W2 gelu(W1 h + b1) + b2), h = uxy + uz (C = 32, H = 64):
// dh_out = W1^T [gelu'(a1) * (W2^T (dv_out * s'(o)))]; dW1, db1, dW2, db2 accumulate.
// The residual part of dv_in (= dv_out) is left to the caller.
template <int C, int H>
__global__ void __launch_bounds__(BW_TILE) k_mlp_bwd(const float* __restrict__ uxy, const float* __restrict__ uz,
                                                   const float* __restrict__ dvout, float* __restrict__ dh_out,
                                                   const float* __restrict__ W1, const float* __restrict__ b1,
                                                   const float* __restrict__ W2, const float* __restrict__ b2,
                                                   float* __restrict__ dW1, float* __restrict__ db1,
                                                   float* __restrict__ dW2, float* __restrict__ db2, long N, int B,
                                                   bool outer_gelu) {
  pdl_enter();
  extern __shared__ float sm[];
  float* w1 = sm;                  // [H][C]
  float* w2 = w1 + H * C;          // [C][H]
  float* sb1 = w2 + C * H;
  float* sb2 = sb1 + H;
  float* sDA = sb2 + C;            // [H][BW_LD]  gelu'(a1) * (W2^T do)
  float* sG = sDA + H * BW_LD;     // [H][BW_LD]  gelu(a1)
  float* sH = sG + H * BW_LD;      // [C][BW_LD]  h
  float* sDO = sH + C * BW_LD;     // [C][BW_LD]  do
  for (int e = threadIdx.x; e < H * C; e += blockDim.x) { w1[e] = W1[e]; w2[e] = W2[e]; }
  for (int e = threadIdx.x; e < H; e += blockDim.x) sb1[e] = b1[e];
  for (int e = threadIdx.x; e < C; e += blockDim.x) sb2[e] = b2[e];
  const int t = threadIdx.x;
  const int r1 = (t / 8) * 4, c1 = (t % 8) * 4;    // dW1 block rows j (H = 16 x 4), cols c (C = 8 x 4)
  const int r2 = (t / 16) * 4, c2 = (t % 16) * 4;  // dW2 block rows o (C = 8 x 4), cols j (H = 16 x 4)
  float g1[4][4] = {}, g2[4][4] = {};
  float gb = 0.f;
  const long total = (long)B * N;
  for (long tile = (long)blockIdx.x * BW_TILE; tile < total; tile += (long)gridDim.x * BW_TILE) {
    __syncthreads();
    const long i = tile + t;
    const bool act = i < total;
    const long b = act ? i / N : 0, pt = act ? i - b * N : 0;
    const long base = b * C * N + pt;
    float h[C], o[C];
#pragma unroll
    for (int c = 0; c < C; ++c) { h[c] = act ? uxy[base + c * N] + uz[base + c * N] : 0.f; o[c] = sb2[c]; }
#pragma unroll 4
    for (int j = 0; j < H; ++j) {
      float s = sb1[j];
#pragma unroll
      for (int c = 0; c < C; ++c) s = fmaf(w1[j * C + c], h[c], s);
      sDA[j * BW_LD + t] = s;   // pre-activation a1, replaced by its gradient below
      const float gj = gelu(s);
      sG[j * BW_LD + t] = act ? gj : 0.f;
#pragma unroll
      for (int c = 0; c < C; ++c) o[c] = fmaf(w2[c * H + j], gj, o[c]);
    }
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const float dv = act ? dvout[base + c * N] : 0.f;
      const float d = outer_gelu ? dv * gelu_grad(o[c]) : dv;
      o[c] = d;
      sDO[c * BW_LD + t] = d;
      sH[c * BW_LD + t] = h[c];
    }
    float dh[C];
#pragma unroll
    for (int c = 0; c < C; ++c) dh[c] = 0.f;
#pragma unroll 4
    for (int j = 0; j < H; ++j) {
      float s = 0.f;
#pragma unroll
      for (int c = 0; c < C; ++c) s = fmaf(w2[c * H + j], o[c], s);
      const float d = act ? s * gelu_grad(sDA[j * BW_LD + t]) : 0.f;
      sDA[j * BW_LD + t] = d;
#pragma unroll
      for (int c = 0; c < C; ++c) dh[c] = fmaf(w1[j * C + c], d, dh[c]);
    }
    if (act)
#pragma unroll
      for (int c = 0; c < C; ++c) dh_out[base + c * N] = dh[c];
    __syncthreads();
    outer4(g1, sDA, r1, sH, c1);
    outer4(g2, sDO, r2, sG, c2);
    if (t < H) {
      for (int p = 0; p < BW_TILE; ++p) gb += sDA[t * BW_LD + p];
    } else if (t < H + C) {
      for (int p = 0; p < BW_TILE; ++p) gb += sDO[(t - H) * BW_LD + p];
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      atomicAdd(dW1 + (r1 + u) * C + c1 + w, g1[u][w]);
      atomicAdd(dW2 + (r2 + u) * H + c2 + w, g2[u][w]);
    }
  if (t < H) atomicAdd(db1 + t, gb);
  else if (t < H + C) atomicAdd(db2 + (t - H), gb);
}

template <int C, int Q>
constexpr size_t proj_bwd_smem() { return (size_t)(Q * C + 6 * Q + Q + (2 * Q + C + 6) * BW_LD) * sizeof(float); }

// Backward of E = Q2 gelu(Q1 v + qb1) + qb2 (C = 32 -> Q = 128 -> 6 = Re/Im of Ex, Ey, Ez):
// dv = Q1^T [gelu'(a) * (Q2^T d6)] with d6 = (Re, Im) of dE; dQ1, dqb1, dQ2, dqb2 accumulate.
template <int C, int Q>
__global__ void __launch_bounds__(BW_TILE) k_proj_bwd(const float* __restrict__ v, const cf* __restrict__ dE,
                                                    float* __restrict__ dv_out, const float* __restrict__ Q1,
                                                    const float* __restrict__ qb1, const float* __restrict__ Q2,
                                                    float* __restrict__ dQ1, float* __restrict__ dqb1,
                                                    float* __restrict__ dQ2, float* __restrict__ dqb2, long N, int B) {
  pdl_enter();
  static_assert(Q == 128 && BW_TILE == 128, "thread-to-block mapping assumes Q = 128 = BW_TILE");
  extern __shared__ float sm[];
  float* q1 = sm;                  // [Q][C]
  float* q2 = q1 + Q * C;          // [6][Q]
  float* sb1 = q2 + 6 * Q;         // [Q]
  float* sDA = sb1 + Q;            // [Q][BW_LD]
  float* sG = sDA + Q * BW_LD;     // [Q][BW_LD]
  float* sV = sG + Q * BW_LD;      // [C][BW_LD]
  float* sD6 = sV + C * BW_LD;     // [6][BW_LD]
  for (int e = threadIdx.x; e < Q * C; e += blockDim.x) q1[e] = Q1[e];
  for (int e = threadIdx.x; e < 6 * Q; e += blockDim.x) q2[e] = Q2[e];
  for (int e = threadIdx.x; e < Q; e += blockDim.x) sb1[e] = qb1[e];
  const int t = threadIdx.x;
  const int r0 = (t / 8) * 4, c0 = (t % 8) * 4;   // dQ1 rows 0..63 (and 64..127), cols 0..31
  float g1[4][4] = {}, g1b[4][4] = {};
  float gq2[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  float gqb1 = 0.f, gqb2 = 0.f;
  const long total = (long)B * N;
  for (long tile = (long)blockIdx.x * BW_TILE; tile < total; tile += (long)gridDim.x * BW_TILE) {
    __syncthreads();
    const long i = tile + t;
    const bool act = i < total;
    const long b = act ? i / N : 0, pt = act ? i - b * N : 0;
    float h[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
      h[c] = act ? v[(b * C + c) * N + pt] : 0.f;
      sV[c * BW_LD + t] = h[c];
    }
    float d6[6];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const cf d = act ? dE[(b * 3 + c) * N + pt] : czero();
      d6[2 * c] = d.x;
      d6[2 * c + 1] = d.y;
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) sD6[k * BW_LD + t] = d6[k];
    float dh[C];
#pragma unroll
    for (int c = 0; c < C; ++c) dh[c] = 0.f;
#pragma unroll 2
    for (int j = 0; j < Q; ++j) {
      float s = sb1[j];
#pragma unroll
      for (int c = 0; c < C; ++c) s = fmaf(q1[j * C + c], h[c], s);
      sG[j * BW_LD + t] = act ? gelu(s) : 0.f;
      float dg = 0.f;
#pragma unroll
      for (int k = 0; k < 6; ++k) dg = fmaf(q2[k * Q + j], d6[k], dg);
      const float da = act ? dg * gelu_grad(s) : 0.f;
      sDA[j * BW_LD + t] = da;
#pragma unroll
      for (int c = 0; c < C; ++c) dh[c] = fmaf(q1[j * C + c], da, dh[c]);
    }
    if (act)
#pragma unroll
      for (int c = 0; c < C; ++c) dv_out[(b * C + c) * N + pt] = dh[c];
    __syncthreads();
    outer4(g1, sDA, r0, sV, c0);
    outer4(g1b, sDA, 64 + r0, sV, c0);
    // thread t owns row t of dQ2^T (6 entries) and qb1[t]
    for (int p = 0; p < BW_TILE; ++p) {
      const float gp = sG[t * BW_LD + p];
#pragma unroll
      for (int k = 0; k < 6; ++k) gq2[k] = fmaf(sD6[k * BW_LD + p], gp, gq2[k]);
      gqb1 += sDA[t * BW_LD + p];
    }
    if (t < 6)
      for (int p = 0; p < BW_TILE; ++p) gqb2 += sD6[t * BW_LD + p];
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      atomicAdd(dQ1 + (r0 + u) * C + c0 + w, g1[u][w]);
      atomicAdd(dQ1 + (64 + r0 + u) * C + c0 + w, g1b[u][w]);
    }
#pragma unroll
  for (int k = 0; k < 6; ++k) atomicAdd(dQ2 + k * Q + t, gq2[k]);
  atomicAdd(dqb1 + t, gqb1);
  if (t < 6) atomicAdd(dqb2 + t, gqb2);
}

// lift backward: dW[c][k] += sum dv0[c] in_k with in = (a, x/nx, y/ny, z/nz); db[c] += sum dv0[c]
// (C <= 32; one thread per point; per-thread partials reduced in shared memory)
__global__ void __launch_bounds__(256) k_lift_bwd(const float* __restrict__ a, const float* __restrict__ dv0,
                                                float* __restrict__ dW, float* __restrict__ db, int B, int C, int nx,
                                                int ny, int nz) {
  pdl_enter();
  __shared__ float acc[32 * 5];
  for (int e = threadIdx.x; e < 32 * 5; e += blockDim.x) acc[e] = 0.f;
  __syncthreads();
  const long N = (long)nx * ny * nz, total = (long)B * N;
  for (int c = 0; c < C; ++c) {
    float r[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
      const long b = i / N, pt = i - b * N;
      const int x = (int)(pt % nx), y = (int)((pt / nx) % ny), z = (int)(pt / ((long)nx * ny));
      const float d = dv0[(b * C + c) * N + pt];
      r[0] = fmaf(d, a[i], r[0]);
      r[1] = fmaf(d, (float)x / nx, r[1]);
      r[2] = fmaf(d, (float)y / ny, r[2]);
      r[3] = fmaf(d, (float)z / nz, r[3]);
      r[4] += d;
    }
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      float x = r[k];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
      if ((threadIdx.x & 31) == 0) atomicAdd(&acc[c * 5 + k], x);
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < C * 5; e += blockDim.x) {
    const int c = e / 5, k = e - c * 5;
    if (k < 4) atomicAdd(dW + c * 4 + k, acc[e]);
    else atomicAdd(db + c, acc[e]);
  }
}

__global__ void k_axpy_f(float* __restrict__ y, const float* __restrict__ x, long n) {
  pdl_enter();
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] += x[i];
}

// ---------------------------------------------------------------- dispatch helpers
#define LAT_CASES(F, n, ...)                 \
  switch (n) {                               \
    case 16: F(16, 4, __VA_ARGS__); break;   \
    case 32: F(32, 4, __VA_ARGS__); break;   \
    case 64: F(64, 8, __VA_ARGS__); break;   \
    case 96: F(96, 4, __VA_ARGS__); break;   \
    case 128: F(128, 8, __VA_ARGS__); break; \
    case 256: F(256, 16, __VA_ARGS__); break;\
    case 512: F(512, 16, __VA_ARGS__); break;\
    default: bad = true;                     \
  }
#define COL_CASES(F, n, ...)                 \
  switch (n) {                               \
    case 16: F(16, 2, __VA_ARGS__); break;   \
    case 32: F(32, 4, __VA_ARGS__); break;   \
    case 48: F(48, 4, __VA_ARGS__); break;   \
    case 64: F(64, 4, __VA_ARGS__); break;   \
    case 96: F(96, 4, __VA_ARGS__); break;   \
    case 128: F(128, 8, __VA_ARGS__); break; \
    case 256: F(256, 8, __VA_ARGS__); break; \
    case 512: F(512, 16, __VA_ARGS__); break;\
    default: bad = true;                     \
  }

static unsigned blocks_for(long items, int per_block) { return (unsigned)((items + per_block - 1) / per_block); }

struct Tw {
  cf *x = nullptr, *y = nullptr, *z = nullptr;
};

static void host_tw(int n, std::vector<cf>& out) {
  out.resize(n);
  for (int m = 0; m < n; ++m) {
    double a = -2.0 * M_PI * (double)m / (double)n;
    out[m] = make_float2((float)cos(a), (float)sin(a));
  }
}

static size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

struct FnoWs {
  float *v, *uxy, *uz;
  cf *T1, *Vm, *Um, *T2, *Wm, *Wu;
  cf *twx, *twy, *twz;
  // training only.  Stored mode: per-layer branch outputs and spectra.  Checkpoint mode: per-layer
  // inputs v_l (the branches are recomputed in the backward) and separate gradient buffers.
  float *uxyL = nullptr, *uzL = nullptr, *vL = nullptr, *dv = nullptr, *dh = nullptr, *tmp = nullptr;
  cf *VmL = nullptr, *WmL = nullptr, *Vg = nullptr, *Wg = nullptr;
  size_t act = 0, vm = 0, wm = 0;   // elements per layer: activations (float), V and W spectra (complex)
};

enum { FNO_INFER = 0, FNO_STORE = 1, FNO_CHECKPOINT = 2 };

static size_t fno_ws(const fno_weights_t* w, int B, int nx, int ny, int nz, FnoWs* o, char* base,
                     int mode = FNO_INFER) {
  const int mx = w->mx < nx ? w->mx : nx, my = w->my < ny ? w->my : ny, mz = w->mz < nz ? w->mz : nz;
  const size_t N = (size_t)nx * ny * nz;
  o->act = (size_t)B * w->dv * N;
  o->vm = (size_t)mx * my * w->dv * B * nz;
  o->wm = (size_t)mz * w->dv * B * nx * ny;
  const size_t act = o->act * sizeof(float);
  const size_t t1 = (size_t)B * w->dv * nz * ny * mx * sizeof(cf);
  const size_t vm = o->vm * sizeof(cf), wm = o->wm * sizeof(cf);
  size_t off = 0;
  auto take = [&](size_t bytes) -> char* { char* q = base ? base + off : nullptr; off += al(bytes); return q; };
  o->v = (float*)take(act); o->uxy = (float*)take(act); o->uz = (float*)take(act);
  o->T1 = (cf*)take(t1); o->T2 = (cf*)take(t1);
  o->Vm = (cf*)take(vm); o->Um = (cf*)take(vm);
  o->Wm = (cf*)take(wm); o->Wu = (cf*)take(wm);
  o->twx = (cf*)take(nx * sizeof(cf)); o->twy = (cf*)take(ny * sizeof(cf)); o->twz = (cf*)take(nz * sizeof(cf));
  const size_t L = (size_t)w->layers;
  if (mode == FNO_STORE) {
    o->uxyL = (float*)take(L * act); o->uzL = (float*)take(L * act);
    o->VmL = (cf*)take(L * vm); o->WmL = (cf*)take(L * wm);
    o->dv = (float*)take(act);
    o->dh = o->uxy; o->tmp = o->uz; o->Vg = o->Vm; o->Wg = o->Wm;   // free during the backward
  } else if (mode == FNO_CHECKPOINT) {
    o->vL = (float*)take(L * act);
    o->dv = (float*)take(act); o->dh = (float*)take(act); o->tmp = (float*)take(act);
    o->Vg = (cf*)take(vm); o->Wg = (cf*)take(wm);
  }
  return off;
}

static int check_weights(const fno_weights_t* w, int B, int nx, int ny, int nz, const char* who) {
  if (w->dv != 32 || w->dh != 64 || w->dq != 128) {
    psfd_set_error("%s: this build is compiled for dv=32, dh=64, dq=128", who);
    return PSFD_ERR_ARG;
  }
  if (w->layers <= 0 || w->mx <= 0 || w->my <= 0 || w->mz <= 0 || B <= 0) {
    psfd_set_error("%s: bad layer count, mode counts or batch", who);
    return PSFD_ERR_ARG;
  }
  if (!lateral_supported(nx) || !lateral_supported(ny) || !axial_supported(nz)) {
    psfd_set_error("%s: unsupported grid %dx%dx%d", who, nx, ny, nz);
    return PSFD_ERR_ARG;
  }
  return PSFD_OK;
}

static Dims make_dims(const fno_weights_t* w, int B, int nx, int ny, int nz) {
  Dims d;
  d.B = B; d.C = w->dv; d.nx = nx; d.ny = ny; d.nz = nz;
  d.mx = w->mx < nx ? w->mx : nx; d.my = w->my < ny ? w->my : ny; d.mz = w->mz < nz ? w->mz : nz;
  d.MX = w->mx; d.MY = w->my; d.MZ = w->mz;
  return d;
}

// ---- the four halves of the two spectral branches (kernels above); each returns false on an unsupported size
// xy analysis: real in [B][C][nz][ny][nx] -> V[mode][c][b*nz+z] (unnormalised DFT on the kept modes)
static bool xy_analysis(const Dims& d, const FnoWs& ws, const float* in, cf* V, cudaStream_t s) {
  bool bad = false;
  const long rows = (long)d.B * d.C * d.nz * d.ny, ycols = (long)d.B * d.C * d.nz * d.mx;
#define XF(NX_, T_, ...) (void)launch_pdl(k_xfwd<NX_, T_>, dim3(blocks_for(rows, 4 * (32 / T_))), dim3(128), 0, s, in, ws.T1, rows, d.mx, ws.twx)
  LAT_CASES(XF, d.nx, 0);
#undef XF
#define YF(NY_, T_, ...) (void)launch_pdl(k_yfwd<NY_, T_>, dim3(blocks_for(ycols, 4 * (32 / T_))), dim3(128), 0, s, ws.T1, V, d, ws.twy)
  LAT_CASES(YF, d.ny, 0);
#undef YF
  return !bad;
}
// xy synthesis: U on the kept modes -> real out = scale * Re(unnormalised inverse DFT of the zero-padded U)
static bool xy_synthesis(const Dims& d, const FnoWs& ws, const cf* U, float* out, float scale, cudaStream_t s) {
  bool bad = false;
  const long rows = (long)d.B * d.C * d.nz * d.ny, ycols = (long)d.B * d.C * d.nz * d.mx;
#define YI(NY_, T_, ...) (void)launch_pdl(k_yinv<NY_, T_>, dim3(blocks_for(ycols, 4 * (32 / T_))), dim3(128), 0, s, U, ws.T2, d, ws.twy)
  LAT_CASES(YI, d.ny, 0);
#undef YI
#define XI(NX_, T_, ...) (void)launch_pdl(k_xinv<NX_, T_>, dim3(blocks_for(rows, 4 * (32 / T_))), dim3(128), 0, s, ws.T2, out, rows, d.mx, scale, ws.twx)
  LAT_CASES(XI, d.nx, 0);
#undef XI
  return !bad;
}
static bool z_analysis(const Dims& d, const FnoWs& ws, const float* in, cf* W, cudaStream_t s) {
  bool bad = false;
  const long zcols = (long)d.B * d.C * d.nx * d.ny;
#define ZF(NZ_, T_, ...) (void)launch_pdl(k_zfwd<NZ_, T_>, dim3(blocks_for(zcols, 4 * (32 / T_))), dim3(128), 0, s, in, W, d, ws.twz)
  COL_CASES(ZF, d.nz, 0);
#undef ZF
  return !bad;
}
static bool z_synthesis(const Dims& d, const FnoWs& ws, const cf* U, float* out, float scale, cudaStream_t s) {
  bool bad = false;
  const long zcols = (long)d.B * d.C * d.nx * d.ny;
#define ZI(NZ_, T_, ...) (void)launch_pdl(k_zinv<NZ_, T_>, dim3(blocks_for(zcols, 4 * (32 / T_))), dim3(128), 0, s, U, out, d, scale, ws.twz)
  COL_CASES(ZI, d.nz, 0);
#undef ZI
  return !bad;
}

static size_t mix_smem_bytes(int C) { return (2 * C * C + 2 * C * MIX_TN) * sizeof(float); }

// PSFD_MIX_FP32=1: the forward mixing keeps float32 operands (no bfloat16 rounding), on the SIMT kernel
static bool mix_fp32() {
  const char* e = getenv("PSFD_MIX_FP32");
  return e && e[0] == '1';
}

// per-mode mixing of a branch; xy modes: grid (n-tiles, mx*my); z modes: grid (n-tiles, mz) with mx = MX = 1
static void mix_xy(const Dims& d, const cf* V, cf* U, const cf* K, bool adjoint, cudaStream_t s) {
  const long NB = (long)d.B * d.nz;
  const bool exact = !adjoint && mix_fp32();
  if (!adjoint && !exact && fno_mix_tc_enabled(d.C)) {
    fno_mix_tc(V, U, K, NB, d.mx * d.my, d.mx, d.MX, (d.MY - d.my) / 2, (d.MX - d.mx) / 2, s);
    return;
  }
  dim3 g(blocks_for(NB, MIX_TN), (unsigned)(d.mx * d.my));
  (void)launch_pdl(k_mix, dim3(g), dim3(256), mix_smem_bytes(d.C), s, V, U, K, d.C, NB, d.mx, d.MX, (d.MY - d.my) / 2, (d.MX - d.mx) / 2,
                                           adjoint, !adjoint && !exact, !exact);
}
static void mix_z(const Dims& d, const cf* V, cf* U, const cf* K, bool adjoint, cudaStream_t s) {
  const long NB = (long)d.B * d.nx * d.ny;
  const bool exact = !adjoint && mix_fp32();
  if (!adjoint && !exact && fno_mix_tc_enabled(d.C)) {
    fno_mix_tc(V, U, K, NB, d.mz, 1, 1, (d.MZ - d.mz) / 2, 0, s);
    return;
  }
  dim3 g(blocks_for(NB, MIX_TN), (unsigned)d.mz);
  (void)launch_pdl(k_mix, dim3(g), dim3(256), mix_smem_bytes(d.C), s, V, U, K, d.C, NB, 1, 1, (d.MZ - d.mz) / 2, 0, adjoint, !adjoint && !exact,
                                           !exact);
}
static void mixgrad_xy(const Dims& d, const cf* Ubar, const cf* V, cf* dK, float scale, cudaStream_t s) {
  const long NB = (long)d.B * d.nz;
  dim3 g(blocks_for(NB, GRAD_CHUNK), (unsigned)(d.mx * d.my));
  (void)launch_pdl(k_mixgrad, dim3(g), dim3(256), 0, s, Ubar, V, (float*)dK, d.C, NB, d.mx, d.MX, (d.MY - d.my) / 2, (d.MX - d.mx) / 2, scale);
}
static void mixgrad_z(const Dims& d, const cf* Ubar, const cf* V, cf* dK, float scale, cudaStream_t s) {
  const long NB = (long)d.B * d.nx * d.ny;
  dim3 g(blocks_for(NB, GRAD_CHUNK), (unsigned)d.mz);
  (void)launch_pdl(k_mixgrad, dim3(g), dim3(256), 0, s, Ubar, V, (float*)dK, d.C, NB, 1, 1, (d.MZ - d.mz) / 2, 0, scale);
}

static int upload_twiddles(const FnoWs& ws, int nx, int ny, int nz, cudaStream_t s) {
  std::vector<cf> tx, ty, tz;
  host_tw(nx, tx); host_tw(ny, ty); host_tw(nz, tz);
  PSFD_CUDA_TRY(cudaMemcpyAsync(ws.twx, tx.data(), nx * sizeof(cf), cudaMemcpyHostToDevice, s));
  PSFD_CUDA_TRY(cudaMemcpyAsync(ws.twy, ty.data(), ny * sizeof(cf), cudaMemcpyHostToDevice, s));
  PSFD_CUDA_TRY(cudaMemcpyAsync(ws.twz, tz.data(), nz * sizeof(cf), cudaMemcpyHostToDevice, s));
  PSFD_CUDA_TRY(cudaStreamSynchronize(s));  // the host vectors go out of scope
  return PSFD_OK;
}

static int set_smem_attrs() {
  static std::once_flag once;   // complete before any host thread launches
  static cudaError_t init = cudaSuccess;
  std::call_once(once, [] {
    init = cudaFuncSetAttribute(k_mlp_bwd<32, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)mlp_bwd_smem<32, 64>());
    if (init == cudaSuccess)
      init = cudaFuncSetAttribute(k_proj_bwd<32, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)proj_bwd_smem<32, 128>());
  });
  if (init != cudaSuccess) {
    psfd_set_error("fno: shared-memory attributes: %s", cudaGetErrorString(init));
    return PSFD_ERR_CUDA;
  }
  return PSFD_OK;
}

// forward pass; with train = true the per-layer spectra and branch outputs are kept in the workspace
// one layer's spectral branches: v -> u_xy (Eq. 2) -> u_z (Eq. 3), spectra V and W kept where given
static bool branches(const Dims& d, const FnoWs& ws, const fno_weights_t* w, int l, const float* v, float* uxy,
                     float* uz, cf* Vm, cf* Wm, cudaStream_t s) {
  const int C = d.C;
  const float sxy = 1.0f / ((float)d.nx * (float)d.ny), sz = 1.0f / (float)d.nz;
  const cf* Kxy = (const cf*)w->kxy + (size_t)l * w->my * w->mx * C * C;
  const cf* Kz = (const cf*)w->kz + (size_t)l * w->mz * C * C;
  bool ok = xy_analysis(d, ws, v, Vm, s);
  mix_xy(d, Vm, ws.Um, Kxy, false, s);
  ok &= xy_synthesis(d, ws, ws.Um, uxy, sxy, s);
  ok &= z_analysis(d, ws, uxy, Wm, s);
  mix_z(d, Wm, ws.Wu, Kz, false, s);
  ok &= z_synthesis(d, ws, ws.Wu, uz, sz, s);
  return ok;
}

static int fno_run(const fno_weights_t* w, const float* a, int B, int nx, int ny, int nz, psfd_c64* E_out,
                   const FnoWs& ws, int mode, cudaStream_t s) {
  int rc = upload_twiddles(ws, nx, ny, nz, s);
  if (rc) return rc;
  const Dims d = make_dims(w, B, nx, ny, nz);
  const int C = d.C;
  const long N = (long)nx * ny * nz;
  bool ok = true;
  const int L = w->layers;
  // layer inputs: in checkpoint mode v_l lives in vL[l] (kept), else the layers update ws.v in place
  auto vin = [&](int l) -> float* { return mode == FNO_CHECKPOINT ? ws.vL + l * ws.act : ws.v; };
  const bool tc = fno_mlp_tc_enabled(C, w->dh, w->dq);
  (void)launch_pdl(k_lift, dim3(blocks_for((long)B * N, 256)), dim3(256), 0, s, a, vin(0), w->lift_w, w->lift_b, B, C, nx, ny, nz);
  PSFD_CHECK_LAUNCH();
  for (int l = 0; l < L; ++l) {
    const bool st = mode == FNO_STORE;
    float* uxy = st ? ws.uxyL + l * ws.act : ws.uxy;
    float* uz = st ? ws.uzL + l * ws.act : ws.uz;
    cf* Vm = st ? ws.VmL + l * ws.vm : ws.Vm;
    cf* Wm = st ? ws.WmL + l * ws.wm : ws.Wm;
    ok &= branches(d, ws, w, l, vin(l), uxy, uz, Vm, Wm, s);
    PSFD_CHECK_LAUNCH();
    // MLP + residual (Eq. 4)
    float* vout = (mode == FNO_CHECKPOINT && l + 1 < L) ? vin(l + 1) : ws.v;
    if (tc) {
      rc = fno_mlp_tc(vin(l), vout, uxy, uz, w->w1 + (size_t)l * 64 * 32, w->b1 + (size_t)l * 64,
                      w->w2 + (size_t)l * 32 * 64, w->b2 + (size_t)l * 32, N, B, l < L - 1, s);
      if (rc) return rc;
    } else {
      (void)launch_pdl(k_mlp<32, 64>, dim3(blocks_for((long)B * N, 128)), dim3(128), 0, s,
          vin(l), vout, uxy, uz, w->w1 + (size_t)l * 64 * 32, w->b1 + (size_t)l * 64, w->w2 + (size_t)l * 32 * 64,
          w->b2 + (size_t)l * 32, N, B, l < L - 1);
      PSFD_CHECK_LAUNCH();
    }
  }
  if (!ok) { psfd_set_error("fno: unsupported size"); return PSFD_ERR_ARG; }
  if (tc) return fno_proj_tc(ws.v, (cf*)E_out, w->q1, w->qb1, w->q2, w->qb2, N, B, s);
  (void)launch_pdl(k_proj<32, 128>, dim3(blocks_for((long)B * N, 128)), dim3(128), 0, s, ws.v, (cf*)E_out, w->q1, w->qb1, w->q2, w->qb2, N, B);
  PSFD_CHECK_LAUNCH();
  return PSFD_OK;
}

}  // namespace

extern "C" size_t fno_workspace_size(const fno_weights_t* w, int B, int nx, int ny, int nz) {
  if (!w || B <= 0) return 0;
  FnoWs o;
  return fno_ws(w, B, nx, ny, nz, &o, nullptr);
}

extern "C" size_t fno_train_workspace_size(const fno_weights_t* w, int B, int nx, int ny, int nz, int checkpoint) {
  if (!w || B <= 0 || w->layers <= 0) return 0;
  FnoWs o;
  return fno_ws(w, B, nx, ny, nz, &o, nullptr, checkpoint ? FNO_CHECKPOINT : FNO_STORE);
}

extern "C" int fno_forward(const fno_weights_t* w, const float* a, int B, int nx, int ny, int nz, psfd_c64* E_out,
                           void* workspace, size_t workspace_bytes, void* stream) {
  if (!w || !a || !E_out || !workspace || B <= 0) { psfd_set_error("fno_forward: null argument"); return PSFD_ERR_ARG; }
  int rc = check_weights(w, B, nx, ny, nz, "fno_forward");
  if (rc) return rc;
  FnoWs ws;
  const size_t need = fno_ws(w, B, nx, ny, nz, &ws, nullptr);
  if (workspace_bytes < need) { psfd_set_error("fno_forward: workspace too small"); return PSFD_ERR_ARG; }
  fno_ws(w, B, nx, ny, nz, &ws, (char*)workspace);
  cudaStream_t s = (cudaStream_t)stream;
  StageScope scope(s, ST_FNO);
  return fno_run(w, a, B, nx, ny, nz, E_out, ws, FNO_INFER, s);
}

extern "C" int fno_forward_train(const fno_weights_t* w, const float* a, int B, int nx, int ny, int nz,
                                 psfd_c64* E_out, void* workspace, size_t workspace_bytes, int checkpoint,
                                 void* stream) {
  if (!w || !a || !E_out || !workspace || B <= 0) {
    psfd_set_error("fno_forward_train: null argument");
    return PSFD_ERR_ARG;
  }
  int rc = check_weights(w, B, nx, ny, nz, "fno_forward_train");
  if (rc) return rc;
  const int mode = checkpoint ? FNO_CHECKPOINT : FNO_STORE;
  FnoWs ws;
  const size_t need = fno_ws(w, B, nx, ny, nz, &ws, nullptr, mode);
  if (workspace_bytes < need) { psfd_set_error("fno_forward_train: workspace too small"); return PSFD_ERR_ARG; }
  fno_ws(w, B, nx, ny, nz, &ws, (char*)workspace, mode);
  cudaStream_t s = (cudaStream_t)stream;
  StageScope scope(s, ST_FNO);
  return fno_run(w, a, B, nx, ny, nz, E_out, ws, mode, s);
}

extern "C" int fno_backward(const fno_weights_t* w, const fno_grads_t* g, const float* a, int B, int nx, int ny,
                            int nz, const psfd_c64* dE, void* workspace, size_t workspace_bytes, int checkpoint,
                            void* stream) {
  if (!w || !g || !a || !dE || !workspace || B <= 0) {
    psfd_set_error("fno_backward: null argument");
    return PSFD_ERR_ARG;
  }
  if (!g->lift_w || !g->lift_b || !g->kxy || !g->kz || !g->w1 || !g->b1 || !g->w2 || !g->b2 || !g->q1 || !g->qb1 ||
      !g->q2 || !g->qb2) {
    psfd_set_error("fno_backward: null gradient buffer");
    return PSFD_ERR_ARG;
  }
  int rc = check_weights(w, B, nx, ny, nz, "fno_backward");
  if (rc) return rc;
  const int mode = checkpoint ? FNO_CHECKPOINT : FNO_STORE;
  FnoWs ws;
  const size_t need = fno_ws(w, B, nx, ny, nz, &ws, nullptr, mode);
  if (workspace_bytes < need) { psfd_set_error("fno_backward: workspace too small"); return PSFD_ERR_ARG; }
  fno_ws(w, B, nx, ny, nz, &ws, (char*)workspace, mode);
  if ((rc = set_smem_attrs())) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  StageScope scope(s, ST_FNO);
  const Dims d = make_dims(w, B, nx, ny, nz);
  const int C = d.C;
  const long N = (long)nx * ny * nz;
  const float sxy = 1.0f / ((float)nx * (float)ny), sz = 1.0f / (float)nz;
  const unsigned pw_all = blocks_for((long)B * N, BW_TILE);
  const unsigned pw_blocks = pw_all < 4u * 148u ? pw_all : 4u * 148u;
  (void)launch_pdl(k_proj_bwd<32, 128>, dim3(pw_blocks), dim3(BW_TILE), proj_bwd_smem<32, 128>(), s,
      ws.v, (const cf*)dE, ws.dv, w->q1, w->qb1, w->q2, g->q1, g->qb1, g->q2, g->qb2, N, B);
  PSFD_CHECK_LAUNCH();
  bool ok = true;
  const long nact = (long)ws.act;
  for (int l = w->layers - 1; l >= 0; --l) {
    const float *uxy, *uz;
    const cf *Vm, *Wm;
    if (mode == FNO_CHECKPOINT) {
      // recompute the layer's branches from its kept input v_l
      ok &= branches(d, ws, w, l, ws.vL + l * ws.act, ws.uxy, ws.uz, ws.Vm, ws.Wm, s);
      uxy = ws.uxy; uz = ws.uz; Vm = ws.Vm; Wm = ws.Wm;
    } else {
      uxy = ws.uxyL + l * ws.act; uz = ws.uzL + l * ws.act; Vm = ws.VmL + l * ws.vm; Wm = ws.WmL + l * ws.wm;
    }
    const cf* Kxy = (const cf*)w->kxy + (size_t)l * w->my * w->mx * C * C;
    const cf* Kz = (const cf*)w->kz + (size_t)l * w->mz * C * C;
    cf* dKxy = (cf*)g->kxy + (size_t)l * w->my * w->mx * C * C;
    cf* dKz = (cf*)g->kz + (size_t)l * w->mz * C * C;
    // MLP (Eq. 4): dh = d(loss)/d(uxy + uz); the residual keeps dv as part of d(loss)/d(v_l)
    (void)launch_pdl(k_mlp_bwd<32, 64>, dim3(pw_blocks), dim3(BW_TILE), mlp_bwd_smem<32, 64>(), s,
        uxy, uz, ws.dv, ws.dh, w->w1 + (size_t)l * 64 * 32, w->b1 + (size_t)l * 64, w->w2 + (size_t)l * 32 * 64,
        w->b2 + (size_t)l * 32, g->w1 + (size_t)l * 64 * 32, g->b1 + (size_t)l * 64, g->w2 + (size_t)l * 32 * 64,
        g->b2 + (size_t)l * 32, N, B, l < w->layers - 1);
    PSFD_CHECK_LAUNCH();
    // z branch adjoint (Eq. 3): d(uxy) = dh + Z^T dh; dKz += (1/nz) F_z(dh) conj(W)
    ok &= z_analysis(d, ws, ws.dh, ws.Wg, s);
    mixgrad_z(d, ws.Wg, Wm, dKz, sz, s);
    mix_z(d, ws.Wg, ws.Wu, Kz, true, s);
    ok &= z_synthesis(d, ws, ws.Wu, ws.tmp, sz, s);
    (void)launch_pdl(k_axpy_f, dim3(blocks_for(nact, 256)), dim3(256), 0, s, ws.dh, ws.tmp, nact);
    PSFD_CHECK_LAUNCH();
    // xy branch adjoint (Eq. 2): dv += XY^T d(uxy); dKxy += (1/(nx ny)) F_xy(d uxy) conj(V)
    ok &= xy_analysis(d, ws, ws.dh, ws.Vg, s);
    mixgrad_xy(d, ws.Vg, Vm, dKxy, sxy, s);
    mix_xy(d, ws.Vg, ws.Um, Kxy, true, s);
    ok &= xy_synthesis(d, ws, ws.Um, ws.tmp, sxy, s);
    (void)launch_pdl(k_axpy_f, dim3(blocks_for(nact, 256)), dim3(256), 0, s, ws.dv, ws.tmp, nact);
    PSFD_CHECK_LAUNCH();
  }
  if (!ok) { psfd_set_error("fno_backward: unsupported size"); return PSFD_ERR_ARG; }
  (void)launch_pdl(k_lift_bwd, dim3((unsigned)(2 * 148)), dim3(256), 0, s, a, ws.dv, g->lift_w, g->lift_b, B, C, nx, ny, nz);
  PSFD_CHECK_LAUNCH();
  return PSFD_OK;
}

// ---------------------------------------------------------------- spectral upsampling
__global__ void k_pad_spectrum(const cf* __restrict__ src, cf* __restrict__ dst, int nx0, int ny0, int nz0, int nx,
                               int ny, int nz, long nb, float scale) {
  pdl_enter();
  const long n0 = (long)nx0 * ny0 * nz0;
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb * n0) return;
  const long b = i / n0, r = i - b * n0;
  const int x = (int)(r % nx0), y = (int)((r / nx0) % ny0), z = (int)(r / ((long)nx0 * ny0));
  // signed frequencies of the coarse grid; the coarse Nyquist index maps to -n0/2
  auto map = [](int k, int n0_, int n) { int s = (k <= (n0_ - 1) / 2) ? k : k - n0_; return s < 0 ? s + n : s; };
  const long o = ((b * nz + map(z, nz0, nz)) * ny + map(y, ny0, ny)) * (long)nx + map(x, nx0, nx);
  dst[o] = cscale(src[i], scale);
}

// the transforms of psfd_spectral_upsample on caller-provided scratch (tmp: nb * n0, tw: twiddles)
static int upsample_run(const psfd_c64* src, int nb, int nx0, int ny0, int nz0, psfd_c64* dst, int nx, int ny, int nz,
                        cf* tmp, cf* tw, const std::vector<cf>* t6, const int* sizes, const size_t* twoff,
                        cudaStream_t s) {
  const long n0 = (long)nx0 * ny0 * nz0, n1 = (long)nx * ny * nz;
  for (int k = 0; k < 6; ++k)
    PSFD_CUDA_TRY(cudaMemcpy(tw + twoff[k], t6[k].data(), sizes[k] * sizeof(cf), cudaMemcpyHostToDevice));
  PSFD_CUDA_TRY(cudaMemcpyAsync(tmp, src, (size_t)nb * n0 * sizeof(cf), cudaMemcpyDeviceToDevice, s));
  int rc;
  // forward 3-D FFT of the coarse field: x rows, y columns, z columns (stride nx*ny)
  if ((rc = launch_rows(nx0, tmp, (long)nb * nz0 * ny0, true, 1.f, tw + twoff[0], s))) return rc;
  if ((rc = launch_cols(ny0, nx0, tmp, (long)nb * nz0 * nx0, true, 1.f, tw + twoff[1], s))) return rc;
  if ((rc = launch_cols(nz0, nx0 * ny0, tmp, (long)nb * nx0 * ny0, true, 1.f, tw + twoff[2], s))) return rc;
  PSFD_CUDA_TRY(cudaMemsetAsync(dst, 0, (size_t)nb * n1 * sizeof(cf), s));
  (void)launch_pdl(k_pad_spectrum, dim3(blocks_for((long)nb * n0, 256)), dim3(256), 0, s, tmp, (cf*)dst, nx0, ny0, nz0, nx, ny, nz, nb,
                                                                1.0f / (float)n0);
  PSFD_CHECK_LAUNCH();
  if ((rc = launch_cols(nz, nx * ny, (cf*)dst, (long)nb * nx * ny, false, 1.f, tw + twoff[5], s))) return rc;
  if ((rc = launch_cols(ny, nx, (cf*)dst, (long)nb * nz * nx, false, 1.f, tw + twoff[4], s))) return rc;
  if ((rc = launch_rows(nx, (cf*)dst, (long)nb * nz * ny, false, 1.f, tw + twoff[3], s))) return rc;
  PSFD_CUDA_TRY(cudaStreamSynchronize(s));
  return PSFD_OK;
}

extern "C" int psfd_spectral_upsample(const psfd_c64* src, int nb, int nx0, int ny0, int nz0, psfd_c64* dst, int nx,
                                      int ny, int nz, void* stream) {
  if (!src || !dst || nb <= 0) { psfd_set_error("psfd_spectral_upsample: null argument"); return PSFD_ERR_ARG; }
  if (nx < nx0 || ny < ny0 || nz < nz0 || !lateral_supported(nx0) || !lateral_supported(ny0) ||
      !axial_supported(nz0) || !lateral_supported(nx) || !lateral_supported(ny) || !axial_supported(nz)) {
    psfd_set_error("psfd_spectral_upsample: unsupported sizes");
    return PSFD_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const long n0 = (long)nx0 * ny0 * nz0;
  cf *tmp = nullptr, *tw = nullptr;
  std::vector<cf> t6[6];
  int sizes[6] = {nx0, ny0, nz0, nx, ny, nz};
  size_t twoff[7] = {0};
  for (int k = 0; k < 6; ++k) { host_tw(sizes[k], t6[k]); twoff[k + 1] = twoff[k] + sizes[k]; }
  int rc = PSFD_OK;
  cudaError_t e = cudaMalloc((void**)&tmp, (size_t)nb * n0 * sizeof(cf));
  if (e == cudaSuccess) e = cudaMalloc((void**)&tw, twoff[6] * sizeof(cf));
  if (e != cudaSuccess) {
    psfd_set_error("psfd_spectral_upsample: cudaMalloc: %s", cudaGetErrorString(e));
    rc = PSFD_ERR_CUDA;
  } else {
    rc = upsample_run(src, nb, nx0, ny0, nz0, dst, nx, ny, nz, tmp, tw, t6, sizes, twoff, s);
    if (rc != PSFD_OK) cudaStreamSynchronize(s);   // nothing queued may still read the scratch when it is freed
  }
  // the scratch is released on every path, failing ones included
  if (tmp) cudaFree(tmp);
  if (tw) cudaFree(tw);
  return rc;
}
