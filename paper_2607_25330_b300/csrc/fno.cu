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
#include <cuda_bf16.h>

#include <cmath>
#include <cstdio>
#include <vector>

#include "fft.cuh"
#include "internal.h"

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
  constexpr int P = 32 / T, R = NX / T;
  using PX = Pencil<NX, T, 1>;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int p = lane / T, t = lane - p * T;
  const long row = ((long)blockIdx.x * (blockDim.x >> 5) + warp) * P + p;
  const bool act = row < nrows;
  const float* src = v + (act ? row : 0) * NX;
  cf w[R];
#pragma unroll
  for (int m = 0; m < R; ++m) w[m] = make_float2(act ? src[t + T * m] : 0.f, 0.f);
  PX::template to_freq<false>(w, t, tw);
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
  constexpr int P = 32 / T, R = NY / T;
  using PY = Pencil<NY, T, P>;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
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
  PY::template to_freq<false>(w, t, tw);
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
                                             int C, long NB, int mx, int MX, int offy, int offx) {
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
    cf k = Km[e];
    Kr[e] = bf16r(k.x);
    Ki[e] = bf16r(k.y);
  }
  const long n0 = (long)blockIdx.x * MIX_TN;
  const cf* Vm = V + mode * C * NB;
  for (int e = threadIdx.x; e < C * MIX_TN; e += blockDim.x) {
    const int i = e / MIX_TN, j = e - i * MIX_TN;
    cf x = (n0 + j < NB) ? Vm[(long)i * NB + n0 + j] : czero();
    Vr[e] = bf16r(x.x);
    Vi[e] = bf16r(x.y);
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

// ---------------------------------------------------------------- inverse y: U -> T2[plane][y][mx]
template <int NY, int T>
__global__ void __launch_bounds__(128) k_yinv(const cf* __restrict__ U, cf* __restrict__ T2, Dims d,
                                              const cf* __restrict__ tw) {
  constexpr int P = 32 / T, R = NY / T;
  using PY = Pencil<NY, T, P>;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
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
  PY::template to_time<true>(w, t, tw);
  cf* base = T2 + plane * (long)NY * d.mx + kx;
#pragma unroll
  for (int m = 0; m < R; ++m)
    if (act) base[(long)(t + T * m) * d.mx] = w[m];
}

// ---------------------------------------------------------------- inverse x: T2 rows -> real out * scale
template <int NX, int T>
__global__ void __launch_bounds__(128) k_xinv(const cf* __restrict__ T2, float* __restrict__ out, long nrows, int mx,
                                              float scale, const cf* __restrict__ tw) {
  constexpr int P = 32 / T, R = NX / T;
  using PX = Pencil<NX, T, 1>;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
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
  PX::template to_time<true>(w, t, tw);
#pragma unroll
  for (int m = 0; m < R; ++m)
    if (act) out[r * NX + t + T * m] = w[m].x * scale;
}

// ---------------------------------------------------------------- z branch
// forward: columns (b, c, yx) along z of real u -> W[kz][c][b*nxy + yx]
template <int NZ, int T>
__global__ void __launch_bounds__(128) k_zfwd(const float* __restrict__ u, cf* __restrict__ W, Dims d,
                                              const cf* __restrict__ tw) {
  constexpr int P = 32 / T, R = NZ / T;
  using PZ = Pencil<NZ, T, P>;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
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
  PZ::template to_freq<false>(w, t, tw);
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
  constexpr int P = 32 / T, R = NZ / T;
  using PZ = Pencil<NZ, T, P>;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
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
  PZ::template to_time<true>(w, t, tw);
  float* base = out + bc * NZ * nxy + yx;
#pragma unroll
  for (int m = 0; m < R; ++m)
    if (act) base[(long)(t + T * m) * nxy] = w[m].x * scale;
}

// ---------------------------------------------------------------- pointwise layers
__global__ void k_lift(const float* __restrict__ a, float* __restrict__ v, const float* __restrict__ W,
                       const float* __restrict__ bias, int B, int C, int nx, int ny, int nz) {
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

// v <- v + s(W2 gelu(W1 (uxy + uz) + b1) + b2); C = dv <= 64, H = dh <= 128
template <int C, int H>
__global__ void __launch_bounds__(128) k_mlp(float* __restrict__ v, const float* __restrict__ uxy,
                                             const float* __restrict__ uz, const float* __restrict__ W1,
                                             const float* __restrict__ b1, const float* __restrict__ W2,
                                             const float* __restrict__ b2, long N, int B, bool outer_gelu) {
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
  for (int c = 0; c < C; ++c) v[base + c * N] += outer_gelu ? gelu(o[c]) : o[c];
}

template <int C, int Q>
__global__ void __launch_bounds__(128) k_proj(const float* __restrict__ v, cf* __restrict__ E, const float* __restrict__ Q1,
                                              const float* __restrict__ qb1, const float* __restrict__ Q2,
                                              const float* __restrict__ qb2, long N, int B) {
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
};

static size_t fno_ws(const fno_weights_t* w, int B, int nx, int ny, int nz, FnoWs* o, char* base) {
  const int mx = w->mx < nx ? w->mx : nx, my = w->my < ny ? w->my : ny, mz = w->mz < nz ? w->mz : nz;
  const size_t N = (size_t)nx * ny * nz;
  const size_t act = (size_t)B * w->dv * N * sizeof(float);
  const size_t t1 = (size_t)B * w->dv * nz * ny * mx * sizeof(cf);
  const size_t vm = (size_t)mx * my * w->dv * B * nz * sizeof(cf);
  const size_t wm = (size_t)mz * w->dv * B * nx * ny * sizeof(cf);
  size_t off = 0;
  auto take = [&](size_t bytes) -> char* { char* q = base ? base + off : nullptr; off += al(bytes); return q; };
  o->v = (float*)take(act); o->uxy = (float*)take(act); o->uz = (float*)take(act);
  o->T1 = (cf*)take(t1); o->T2 = (cf*)take(t1);
  o->Vm = (cf*)take(vm); o->Um = (cf*)take(vm);
  o->Wm = (cf*)take(wm); o->Wu = (cf*)take(wm);
  o->twx = (cf*)take(nx * sizeof(cf)); o->twy = (cf*)take(ny * sizeof(cf)); o->twz = (cf*)take(nz * sizeof(cf));
  return off;
}

}  // namespace

extern "C" size_t fno_workspace_size(const fno_weights_t* w, int B, int nx, int ny, int nz) {
  if (!w || B <= 0) return 0;
  FnoWs o;
  return fno_ws(w, B, nx, ny, nz, &o, nullptr);
}

extern "C" int fno_forward(const fno_weights_t* w, const float* a, int B, int nx, int ny, int nz, psfd_c64* E_out,
                           void* workspace, size_t workspace_bytes, void* stream) {
  if (!w || !a || !E_out || !workspace || B <= 0) { psfd_set_error("fno_forward: null argument"); return PSFD_ERR_ARG; }
  if (w->dv != 32 || w->dh != 64 || w->dq != 128) {
    psfd_set_error("fno_forward: this build is compiled for dv=32, dh=64, dq=128");
    return PSFD_ERR_ARG;
  }
  if (!lateral_supported(nx) || !lateral_supported(ny) || !axial_supported(nz)) {
    psfd_set_error("fno_forward: unsupported grid %dx%dx%d", nx, ny, nz);
    return PSFD_ERR_ARG;
  }
  FnoWs ws;
  const size_t need = fno_ws(w, B, nx, ny, nz, &ws, nullptr);
  if (workspace_bytes < need) { psfd_set_error("fno_forward: workspace too small"); return PSFD_ERR_ARG; }
  fno_ws(w, B, nx, ny, nz, &ws, (char*)workspace);
  cudaStream_t s = (cudaStream_t)stream;
  StageScope scope(s, ST_FNO);
  {
    std::vector<cf> tx, ty, tz;
    host_tw(nx, tx); host_tw(ny, ty); host_tw(nz, tz);
    PSFD_CUDA_TRY(cudaMemcpyAsync(ws.twx, tx.data(), nx * sizeof(cf), cudaMemcpyHostToDevice, s));
    PSFD_CUDA_TRY(cudaMemcpyAsync(ws.twy, ty.data(), ny * sizeof(cf), cudaMemcpyHostToDevice, s));
    PSFD_CUDA_TRY(cudaMemcpyAsync(ws.twz, tz.data(), nz * sizeof(cf), cudaMemcpyHostToDevice, s));
    PSFD_CUDA_TRY(cudaStreamSynchronize(s));  // host vectors go out of scope
  }
  const int C = w->dv;
  Dims d;
  d.B = B; d.C = C; d.nx = nx; d.ny = ny; d.nz = nz;
  d.mx = w->mx < nx ? w->mx : nx; d.my = w->my < ny ? w->my : ny; d.mz = w->mz < nz ? w->mz : nz;
  d.MX = w->mx; d.MY = w->my; d.MZ = w->mz;
  const long N = (long)nx * ny * nz;
  const long rows = (long)B * C * nz * ny;
  bool bad = false;
  k_lift<<<blocks_for((long)B * N, 256), 256, 0, s>>>(a, ws.v, w->lift_w, w->lift_b, B, C, nx, ny, nz);
  PSFD_CHECK_LAUNCH();
  const size_t mix_smem = (2 * C * C + 2 * C * MIX_TN) * sizeof(float);
  for (int l = 0; l < w->layers; ++l) {
    // ---- xy branch
#define XF(NX_, T_, ...) k_xfwd<NX_, T_><<<blocks_for(rows, 4 * (32 / T_)), 128, 0, s>>>(ws.v, ws.T1, rows, d.mx, ws.twx)
    LAT_CASES(XF, nx, 0);
#undef XF
    PSFD_CHECK_LAUNCH();
    const long ycols = (long)B * C * nz * d.mx;
#define YF(NY_, T_, ...) k_yfwd<NY_, T_><<<blocks_for(ycols, 4 * (32 / T_)), 128, 0, s>>>(ws.T1, ws.Vm, d, ws.twy)
    LAT_CASES(YF, ny, 0);
#undef YF
    PSFD_CHECK_LAUNCH();
    const long NB = (long)B * nz;
    dim3 gm(blocks_for(NB, MIX_TN), (unsigned)(d.mx * d.my));
    const cf* Kxy = (const cf*)w->kxy + (size_t)l * w->my * w->mx * C * C;
    k_mix<<<gm, 256, mix_smem, s>>>(ws.Vm, ws.Um, Kxy, C, NB, d.mx, w->mx, (w->my - d.my) / 2,
                                    (w->mx - d.mx) / 2);
    PSFD_CHECK_LAUNCH();
#define YI(NY_, T_, ...) k_yinv<NY_, T_><<<blocks_for(ycols, 4 * (32 / T_)), 128, 0, s>>>(ws.Um, ws.T2, d, ws.twy)
    LAT_CASES(YI, ny, 0);
#undef YI
    PSFD_CHECK_LAUNCH();
    const float sxy = 1.0f / ((float)nx * (float)ny);
#define XI(NX_, T_, ...) k_xinv<NX_, T_><<<blocks_for(rows, 4 * (32 / T_)), 128, 0, s>>>(ws.T2, ws.uxy, rows, d.mx, sxy, ws.twx)
    LAT_CASES(XI, nx, 0);
#undef XI
    PSFD_CHECK_LAUNCH();
    // ---- z branch
    const long zcols = (long)B * C * nx * ny;
#define ZF(NZ_, T_, ...) k_zfwd<NZ_, T_><<<blocks_for(zcols, 4 * (32 / T_)), 128, 0, s>>>(ws.uxy, ws.Wm, d, ws.twz)
    COL_CASES(ZF, nz, 0);
#undef ZF
    PSFD_CHECK_LAUNCH();
    const long NBz = (long)B * nx * ny;
    dim3 gz(blocks_for(NBz, MIX_TN), (unsigned)d.mz);
    const cf* Kz = (const cf*)w->kz + (size_t)l * w->mz * C * C;
    // z table rows: mode jz -> row jz + (MZ - mz)/2 ; reuse the xy row formula with my=1 layout
    k_mix<<<gz, 256, mix_smem, s>>>(ws.Wm, ws.Wu, Kz, C, NBz, 1, 1, (w->mz - d.mz) / 2, 0);
    PSFD_CHECK_LAUNCH();
    const float sz = 1.0f / (float)nz;
#define ZI(NZ_, T_, ...) k_zinv<NZ_, T_><<<blocks_for(zcols, 4 * (32 / T_)), 128, 0, s>>>(ws.Wu, ws.uz, d, sz, ws.twz)
    COL_CASES(ZI, nz, 0);
#undef ZI
    PSFD_CHECK_LAUNCH();
    // ---- MLP + residual
    k_mlp<32, 64><<<blocks_for((long)B * N, 128), 128, 0, s>>>(
        ws.v, ws.uxy, ws.uz, w->w1 + (size_t)l * 64 * 32, w->b1 + (size_t)l * 64, w->w2 + (size_t)l * 32 * 64,
        w->b2 + (size_t)l * 32, N, B, l < w->layers - 1);
    PSFD_CHECK_LAUNCH();
  }
  if (bad) { psfd_set_error("fno_forward: unsupported size"); return PSFD_ERR_ARG; }
  k_proj<32, 128><<<blocks_for((long)B * N, 128), 128, 0, s>>>(ws.v, (cf*)E_out, w->q1, w->qb1, w->q2, w->qb2, N, B);
  PSFD_CHECK_LAUNCH();
  return PSFD_OK;
}

// ---------------------------------------------------------------- spectral upsampling
__global__ void k_pad_spectrum(const cf* __restrict__ src, cf* __restrict__ dst, int nx0, int ny0, int nz0, int nx,
                               int ny, int nz, long nb, float scale) {
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

extern "C" int psfd_spectral_upsample(const psfd_c64* src, int nb, int nx0, int ny0, int nz0, psfd_c64* dst, int nx,
                                      int ny, int nz, void* stream) {
  if (!src || !dst || nb <= 0) { psfd_set_error("psfd_spectral_upsample: null argument"); return PSFD_ERR_ARG; }
  if (nx < nx0 || ny < ny0 || nz < nz0 || !lateral_supported(nx0) || !lateral_supported(ny0) ||
      !axial_supported(nz0) || !lateral_supported(nx) || !lateral_supported(ny) || !axial_supported(nz)) {
    psfd_set_error("psfd_spectral_upsample: unsupported sizes");
    return PSFD_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const long n0 = (long)nx0 * ny0 * nz0, n1 = (long)nx * ny * nz;
  cf *tmp = nullptr, *tw = nullptr;
  std::vector<cf> t6[6];
  int sizes[6] = {nx0, ny0, nz0, nx, ny, nz};
  size_t twoff[7] = {0};
  for (int k = 0; k < 6; ++k) { host_tw(sizes[k], t6[k]); twoff[k + 1] = twoff[k] + sizes[k]; }
  PSFD_CUDA_TRY(cudaMalloc((void**)&tmp, (size_t)nb * n0 * sizeof(cf)));
  PSFD_CUDA_TRY(cudaMalloc((void**)&tw, twoff[6] * sizeof(cf)));
  for (int k = 0; k < 6; ++k)
    PSFD_CUDA_TRY(cudaMemcpy(tw + twoff[k], t6[k].data(), sizes[k] * sizeof(cf), cudaMemcpyHostToDevice));
  PSFD_CUDA_TRY(cudaMemcpyAsync(tmp, src, (size_t)nb * n0 * sizeof(cf), cudaMemcpyDeviceToDevice, s));
  int rc;
  // forward 3-D FFT of the coarse field: x rows, y columns, z columns (stride nx*ny)
  if ((rc = launch_rows(nx0, tmp, (long)nb * nz0 * ny0, true, 1.f, tw + twoff[0], s))) return rc;
  if ((rc = launch_cols(ny0, nx0, tmp, (long)nb * nz0 * nx0, true, 1.f, tw + twoff[1], s))) return rc;
  if ((rc = launch_cols(nz0, nx0 * ny0, tmp, (long)nb * nx0 * ny0, true, 1.f, tw + twoff[2], s))) return rc;
  PSFD_CUDA_TRY(cudaMemsetAsync(dst, 0, (size_t)nb * n1 * sizeof(cf), s));
  k_pad_spectrum<<<blocks_for((long)nb * n0, 256), 256, 0, s>>>(tmp, (cf*)dst, nx0, ny0, nz0, nx, ny, nz, nb,
                                                                1.0f / (float)n0);
  PSFD_CHECK_LAUNCH();
  if ((rc = launch_cols(nz, nx * ny, (cf*)dst, (long)nb * nx * ny, false, 1.f, tw + twoff[5], s))) return rc;
  if ((rc = launch_cols(ny, nx, (cf*)dst, (long)nb * nz * nx, false, 1.f, tw + twoff[4], s))) return rc;
  if ((rc = launch_rows(nx, (cf*)dst, (long)nb * nz * ny, false, 1.f, tw + twoff[3], s))) return rc;
  PSFD_CUDA_TRY(cudaStreamSynchronize(s));
  cudaFree(tmp);
  cudaFree(tw);
  return PSFD_OK;
}
