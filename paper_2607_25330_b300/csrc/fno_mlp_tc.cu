// Pointwise layers of the factorised FNO (Eq. 4 and the projection of Eq. 5) on the
// fifth-generation tensor cores.
//
// Per point the layer is a pair of small dense products: h (C) -> W1 h + b1 (H) -> GELU ->
// W2 (.) + b2 (C) for the MLP, and v (C) -> Q1 v + qb1 (Q) -> GELU -> Q2 (.) + qb2 (6) for the
// projection.  A tile of 128 points is a GEMM with M = 128: D1 (128 x H) = A (128 x C) * W1^T, in
// tcgen05.mma kind::tf32 with FP32 accumulation in tensor memory, issued by one thread.  The paper
// fixes no precision for these layers, so they keep FP32 accuracy: every operand x enters as
// x_hi + x_lo with x_hi = x with its 13 low mantissa bits cleared (exact in TF32) and
// x_lo = x - x_hi (exact in FP32, read by the tensor core as TF32), and each product is
// A_hi B_hi + A_hi B_lo + A_lo B_hi (relative error about 2^-20).  The GELU between the two
// products runs on the CUDA cores after tcgen05.ld of the accumulator rows; the second product of
// the MLP is a second pair of MMAs (K = H) on the same tile; the projection's last product (Q x 6)
// stays on the CUDA cores (N = 6 is below the MMA's minimum).
// Operands are staged in shared memory in the canonical K-major layout without swizzle: 8-row x
// 16-byte core matrices, K-adjacent core matrices 128 B apart, 8-row groups (K bytes / 16) x 128 B
// apart.  Every wait on the tensor core is bounded; on a timeout the kernel records it in the same
// device flag as the mode mixing, waits once more, frees its tensor memory and returns.
#include <mutex>
#include <algorithm>
#include <cstdint>
#include <cstdlib>

#include "internal.h"
#include "pdl.cuh"

namespace {

constexpr int MT = 128;                 // points per tile (MMA M), one thread per point
constexpr int MLP_C = 32, MLP_H = 64;   // the FNO's dv and dh
constexpr int PROJ_Q = 128;             // dq
constexpr uint32_t TMEM_COLS = 128;

__device__ __forceinline__ uint32_t saddr(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

// byte offset of element (row, k) of a K-major tile with K 4-byte elements per row
template <int K>
__device__ __forceinline__ int koff(int row, int k) {
  return (((row >> 3) * (K / 4) + (k >> 2)) << 7) + ((row & 7) << 4) + ((k & 3) << 2);
}

template <int K>
__device__ __forceinline__ uint64_t kdesc(uint32_t a) {
  constexpr uint64_t LBO = 128, SBO = (uint64_t)(K / 4) * 128;
  return (uint64_t)((a >> 4) & 0x3FFF) | ((uint64_t)((LBO >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((SBO >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// kind::tf32 instruction descriptor: FP32 accumulate, TF32 A and B, both K-major, M = 128
template <int N>
constexpr uint32_t idesc_tf32() {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(MT >> 4) << 24);
}

__device__ __forceinline__ void split(float x, float& hi, float& lo) {
  hi = __uint_as_float(__float_as_uint(x) & 0xffffe000u);
  lo = x - hi;
}

__device__ __forceinline__ float gelu_f(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752440f)); }

__device__ __forceinline__ bool mbar_wait(uint32_t mb, uint32_t parity, long limit) {
  uint32_t ok = 0;
  for (long it = 0; it < limit && !ok; ++it) {
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok) : "r"(mb), "r"(parity) : "memory");
  }
  return ok != 0;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];\n"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// D (TMEM, N columns at tcol) = A (128 x K) * B^T (N x K), split operands: (Ahi, Bhi), (Ahi, Blo), (Alo, Bhi)
template <int K, int N>
__device__ __forceinline__ void mma3(uint32_t tcol, uint32_t ahi, uint32_t alo, uint32_t bhi, uint32_t blo) {
  constexpr uint32_t id = idesc_tf32<N>();
  const uint32_t as[3] = {ahi, ahi, alo}, bs[3] = {bhi, blo, bhi};
#pragma unroll
  for (int p = 0; p < 3; ++p)
#pragma unroll
    for (int kk = 0; kk < K / 8; ++kk) {   // K = 8 TF32 elements = 32 bytes = two core matrices
      const uint64_t ad = kdesc<K>(as[p] + kk * 256), bd = kdesc<K>(bs[p] + kk * 256);
      const uint32_t acc = (p > 0 || kk > 0) ? 1u : 0u;
      asm volatile(
          "{\n .reg .pred q;\n setp.ne.u32 q, %4, 0;\n"
          " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, q;\n}"
          :: "r"(tcol), "l"(ad), "l"(bd), "r"(id), "r"(acc) : "memory");
    }
}

__device__ __forceinline__ void commit(uint32_t mb) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(mb) : "memory");
}

__device__ __forceinline__ void to_tensor_core() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// a bounded wait for the CTA's products; false (after recording, waiting once more and freeing
// tensor memory) when they did not complete
__device__ bool wait_products(uint32_t mb, uint32_t parity, uint32_t taddr, int* err) {
  const bool done = mbar_wait(mb, parity, 1L << 24);
  if (__syncthreads_or(!done)) {
    if (threadIdx.x == 0) atomicExch(err, 1);
    mbar_wait(mb, parity, 1L << 24);
    __syncthreads();
    if ((threadIdx.x >> 5) == 0)
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(taddr), "r"(TMEM_COLS) : "memory");
    return false;
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  return true;
}

__device__ __forceinline__ void free_tmem(uint32_t taddr) {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if ((threadIdx.x >> 5) == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(taddr), "r"(TMEM_COLS) : "memory");
  }
}

__device__ __forceinline__ uint32_t alloc_tmem(uint32_t* slot, uint32_t mb) {
  if ((threadIdx.x >> 5) == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(saddr(slot)), "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(mb) : "memory");
  return 0;
}

// shared-memory plan of k_mlp_tc (bytes): A (hi, lo) at K = H (the first product's K = C tile
// uses its first half), B1 (hi, lo), B2 (hi, lo)
constexpr int MLP_A = MT * MLP_H * 4;        // 32 KB per part
constexpr int MLP_B1 = MLP_H * MLP_C * 4;    // 8 KB per part
constexpr int MLP_B2 = MLP_C * MLP_H * 4;    // 8 KB per part
constexpr int MLP_SMEM = 2 * MLP_A + 2 * MLP_B1 + 2 * MLP_B2;

// split x into TF32 high and low parts and store four consecutive K entries of one row (16 bytes)
template <int K>
__device__ __forceinline__ void stage4(unsigned char* hi, unsigned char* lo, int row, int k, const float* x) {
  float4 h, l;
  split(x[0], h.x, l.x);
  split(x[1], h.y, l.y);
  split(x[2], h.z, l.z);
  split(x[3], h.w, l.w);
  *reinterpret_cast<float4*>(hi + koff<K>(row, k)) = h;
  *reinterpret_cast<float4*>(lo + koff<K>(row, k)) = l;
}

// Persistent, 8 warps: each CTA stages the weights once, keeps its tensor memory, and walks tiles
// blockIdx.x, blockIdx.x + gridDim.x, ...  Two threads serve a point: warp w reads TMEM lanes
// 32 (w % 4) .. + 31 (its quarter of the tile's points) and owns half hh = w / 4 of every
// accumulator row and of the point's channels.  The next tile's inputs are loaded into registers
// while the current tile's products run.
constexpr int NT2 = 2 * MT;   // threads per CTA

// v_out = v_in + s(W2 gelu(W1 (uxy + uz) + b1) + b2), s = GELU when outer_gelu; v_out may alias v_in
__global__ void __launch_bounds__(NT2) k_mlp_tc(const float* vin, float* vout, const float* __restrict__ uxy,
                                                const float* __restrict__ uz, const float* __restrict__ W1,
                                                const float* __restrict__ b1, const float* __restrict__ W2,
                                                const float* __restrict__ b2, long N, int B, int outer_gelu,
                                                int* err) {
  pdl_enter();
  constexpr int HC = MLP_C / 2, HH = MLP_H / 2;   // channels and hidden units per thread
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char* Ahi = sm;
  unsigned char* Alo = sm + MLP_A;
  unsigned char* B1hi = sm + 2 * MLP_A;
  unsigned char* B1lo = B1hi + MLP_B1;
  unsigned char* B2hi = B1lo + MLP_B1;
  unsigned char* B2lo = B2hi + MLP_B2;
  __shared__ __align__(8) unsigned long long mbar;
  __shared__ uint32_t tmem_base;
  __shared__ float sb1[MLP_H], sb2[MLP_C];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row = 32 * (warp & 3) + lane, hh = warp >> 2;
  const uint32_t mb = saddr(&mbar);
  alloc_tmem(&tmem_base, mb);
  for (int e = 4 * tid; e < MLP_H * MLP_C; e += 4 * NT2) {
    const int j = e / MLP_C, c = e - j * MLP_C;      // W1 [H][C]: row j of B1 (N = H, K = C)
    stage4<MLP_C>(B1hi, B1lo, j, c, W1 + e);
    const int o = e / MLP_H, k = e - o * MLP_H;      // W2 [C][H]: row o of B2 (N = C, K = H)
    stage4<MLP_H>(B2hi, B2lo, o, k, W2 + e);
  }
  if (tid < MLP_H) sb1[tid] = b1[tid];
  if (tid < MLP_C) sb2[tid] = b2[tid];
  const long total = (long)B * N;
  const long ntiles = (total + MT - 1) / MT;
  // point `row` of a tile; channels HC hh .. HC hh + HC - 1 of uxy + uz and of v_in
  auto load = [&](long tile, float* h, float* r) {
    const long i = tile * MT + row;
    const bool in = tile < ntiles && i < total;
    const long b = in ? i / N : 0, pt = in ? i - b * N : 0;
    const long base = (b * MLP_C + HC * hh) * N + pt;
#pragma unroll
    for (int c = 0; c < HC; ++c) {
      h[c] = in ? uxy[base + c * N] + uz[base + c * N] : 0.f;
      r[c] = in ? vin[base + c * N] : 0.f;
    }
  };
  float h[HC], r[HC];
  load(blockIdx.x, h, r);
  uint32_t ph = 0;
  for (long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
#pragma unroll
    for (int c = 0; c < HC; c += 4) stage4<MLP_C>(Ahi, Alo, row, HC * hh + c, h + c);
    float rin[HC];
#pragma unroll
    for (int c = 0; c < HC; ++c) rin[c] = r[c];
    to_tensor_core();
    const uint32_t taddr = tmem_base;
    if (tid == 0) {
      mma3<MLP_C, MLP_H>(taddr, saddr(Ahi), saddr(Alo), saddr(B1hi), saddr(B1lo));
      commit(mb);
    }
    load(tile + gridDim.x, h, r);                    // next tile, while the products run
    if (!wait_products(mb, ph, taddr, err)) return;
    ph ^= 1u;
    const uint32_t trow = taddr + ((uint32_t)(32 * (warp & 3)) << 16);
    // GELU(W1 h + b1) -> A2 (row = point, K = H): this thread's half of the hidden units
#pragma unroll
    for (int q = 0; q < HH / 16; ++q) {
      float d[16];
      const int j0 = HH * hh + 16 * q;
      tmem_ld16(trow + j0, d);
#pragma unroll
      for (int u = 0; u < 16; ++u) d[u] = gelu_f(d[u] + sb1[j0 + u]);
#pragma unroll
      for (int u = 0; u < 16; u += 4) stage4<MLP_H>(Ahi, Alo, row, j0 + u, d + u);
    }
    to_tensor_core();
    if (tid == 0) {
      mma3<MLP_H, MLP_C>(taddr + MLP_H, saddr(Ahi), saddr(Alo), saddr(B2hi), saddr(B2lo));
      commit(mb);
    }
    if (!wait_products(mb, ph, taddr, err)) return;
    ph ^= 1u;
    float o[HC];
    tmem_ld16(trow + MLP_H + HC * hh, o);
    const long i = tile * MT + row;
    if (i < total) {
      const long b = i / N, pt = i - b * N;
      const long base = (b * MLP_C + HC * hh) * N + pt;
#pragma unroll
      for (int c = 0; c < HC; ++c) {
        const float t = o[c] + sb2[HC * hh + c];
        vout[base + c * N] = rin[c] + (outer_gelu ? gelu_f(t) : t);
      }
    }
  }
  free_tmem(tmem_base);
}

constexpr int PROJ_A = MT * MLP_C * 4;       // 16 KB per part
constexpr int PROJ_B = PROJ_Q * MLP_C * 4;   // 16 KB per part
constexpr int PROJ_SMEM = 2 * PROJ_A + 2 * PROJ_B;

// E = (Q2 gelu(Q1 v + qb1) + qb2) as (Re, Im) of (Ex, Ey, Ez); persistent, 8 warps as k_mlp_tc
// (each half of the hidden units gives partial sums of the six outputs; the halves meet in
// shared memory)
__global__ void __launch_bounds__(NT2) k_proj_tc(const float* __restrict__ v, cf* __restrict__ E,
                                                 const float* __restrict__ Q1, const float* __restrict__ qb1,
                                                 const float* __restrict__ Q2, const float* __restrict__ qb2, long N,
                                                 int B, int* err) {
  pdl_enter();
  constexpr int HC = MLP_C / 2, HQ = PROJ_Q / 2;
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char* Ahi = sm;
  unsigned char* Alo = sm + PROJ_A;
  unsigned char* Bhi = sm + 2 * PROJ_A;
  unsigned char* Blo = Bhi + PROJ_B;
  __shared__ __align__(8) unsigned long long mbar;
  __shared__ uint32_t tmem_base;
  __shared__ float sq1[PROJ_Q], sq2[6 * PROJ_Q], sqb2[6];
  __shared__ float part[MT][7];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row = 32 * (warp & 3) + lane, hh = warp >> 2;
  const uint32_t mb = saddr(&mbar);
  alloc_tmem(&tmem_base, mb);
  for (int e = 4 * tid; e < PROJ_Q * MLP_C; e += 4 * NT2) {
    const int j = e / MLP_C, c = e - j * MLP_C;      // Q1 [Q][C]
    stage4<MLP_C>(Bhi, Blo, j, c, Q1 + e);
  }
  for (int e = tid; e < 6 * PROJ_Q; e += NT2) sq2[e] = Q2[e];
  if (tid < PROJ_Q) sq1[tid] = qb1[tid];
  if (tid < 6) sqb2[tid] = qb2[tid];
  const long total = (long)B * N;
  const long ntiles = (total + MT - 1) / MT;
  auto load = [&](long tile, float* x) {
    const long i = tile * MT + row;
    const bool in = tile < ntiles && i < total;
    const long b = in ? i / N : 0, pt = in ? i - b * N : 0;
    const long base = (b * MLP_C + HC * hh) * N + pt;
#pragma unroll
    for (int c = 0; c < HC; ++c) x[c] = in ? v[base + c * N] : 0.f;
  };
  float x[HC];
  load(blockIdx.x, x);
  uint32_t ph = 0;
  for (long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
#pragma unroll
    for (int c = 0; c < HC; c += 4) stage4<MLP_C>(Ahi, Alo, row, HC * hh + c, x + c);
    to_tensor_core();
    const uint32_t taddr = tmem_base;
    if (tid == 0) {
      mma3<MLP_C, PROJ_Q>(taddr, saddr(Ahi), saddr(Alo), saddr(Bhi), saddr(Blo));
      commit(mb);
    }
    load(tile + gridDim.x, x);
    if (!wait_products(mb, ph, taddr, err)) return;
    ph ^= 1u;
    const uint32_t trow = taddr + ((uint32_t)(32 * (warp & 3)) << 16);
    float o[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) o[k] = hh == 0 ? sqb2[k] : 0.f;
#pragma unroll 1
    for (int q = 0; q < HQ / 16; ++q) {
      float d[16];
      const int j0 = HQ * hh + 16 * q;
      tmem_ld16(trow + j0, d);
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int j = j0 + u;
        const float g = gelu_f(d[u] + sq1[j]);
#pragma unroll
        for (int k = 0; k < 6; ++k) o[k] = fmaf(sq2[k * PROJ_Q + j], g, o[k]);
      }
    }
    if (hh == 1) {
#pragma unroll
      for (int k = 0; k < 6; ++k) part[row][k] = o[k];
    }
    __syncthreads();
    const long i = tile * MT + row;
    if (hh == 0 && i < total) {
      const long b = i / N, pt = i - b * N;
#pragma unroll
      for (int c = 0; c < 3; ++c)
        E[(b * 3 + c) * N + pt] = make_float2(o[2 * c] + part[row][2 * c], o[2 * c + 1] + part[row][2 * c + 1]);
    }
  }
  free_tmem(tmem_base);
}

int* g_mlp_err = nullptr;

}  // namespace

// 1 when the pointwise layers run on the tensor cores (C = 32, H = 64, Q = 128; PSFD_MLP_TC=0
// selects the CUDA-core kernels)
bool fno_mlp_tc_enabled(int C, int H, int Q) {
  const char* e = getenv("PSFD_MLP_TC");
  return C == MLP_C && H == MLP_H && Q == PROJ_Q && !(e && e[0] == '0');
}

static int mlp_err_ptr() {
  // once per process, complete before any host thread launches
  static std::once_flag once;
  static cudaError_t init = cudaSuccess;
  std::call_once(once, [] {
    int* p = nullptr;
    init = cudaMalloc((void**)&p, sizeof(int));
    if (init == cudaSuccess) init = cudaMemset(p, 0, sizeof(int));
    if (init == cudaSuccess) init = cudaFuncSetAttribute(k_mlp_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, MLP_SMEM);
    if (init == cudaSuccess) init = cudaFuncSetAttribute(k_proj_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, PROJ_SMEM);
    if (init == cudaSuccess) g_mlp_err = p;
  });
  if (init != cudaSuccess || !g_mlp_err) {
    psfd_set_error("fno tensor-core layers: set-up: %s", cudaGetErrorString(init));
    return PSFD_ERR_CUDA;
  }
  return PSFD_OK;
}

// persistent grid: CTAs per SM (shared memory bound) x SMs, at most one CTA per tile
static unsigned persistent_grid(long ntiles, int per_sm) {
  static const int nsm = [] {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        n <= 0)
      n = 148;
    return n;
  }();
  return (unsigned)std::min<long>(ntiles, (long)nsm * per_sm);
}

int fno_mlp_tc(const float* vin, float* vout, const float* uxy, const float* uz, const float* W1, const float* b1,
               const float* W2, const float* b2, long N, int B, bool outer_gelu, cudaStream_t s) {
  int rc = mlp_err_ptr();
  if (rc) return rc;
  const unsigned grid = persistent_grid(((long)B * N + MT - 1) / MT, 2);
  (void)launch_pdl(k_mlp_tc, dim3(grid), dim3(NT2), MLP_SMEM, s, vin, vout, uxy, uz, W1, b1, W2, b2, N, B, outer_gelu ? 1 : 0, g_mlp_err);
  PSFD_CHECK_LAUNCH();
  return PSFD_OK;
}

int fno_proj_tc(const float* v, cf* E, const float* Q1, const float* qb1, const float* Q2, const float* qb2, long N,
                int B, cudaStream_t s) {
  int rc = mlp_err_ptr();
  if (rc) return rc;
  const unsigned grid = persistent_grid(((long)B * N + MT - 1) / MT, 2);
  (void)launch_pdl(k_proj_tc, dim3(grid), dim3(NT2), PROJ_SMEM, s, v, E, Q1, qb1, Q2, qb2, N, B, g_mlp_err);
  PSFD_CHECK_LAUNCH();
  return PSFD_OK;
}

// reads and clears the timeout flag of the pointwise tensor-core kernels
int fno_mlp_tc_error(int* host_flag) {
  *host_flag = 0;
  if (!g_mlp_err) return PSFD_OK;
  PSFD_CUDA_TRY(cudaMemcpy(host_flag, g_mlp_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (*host_flag) PSFD_CUDA_TRY(cudaMemset(g_mlp_err, 0, sizeof(int)));
  return PSFD_OK;
}
