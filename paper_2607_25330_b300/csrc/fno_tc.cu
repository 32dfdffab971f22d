// Per-mode channel mixing of the factorised FNO (Eqs. 2-3) on the fifth-generation tensor cores.
//
// For one retained mode the mixing is U = K V with K a C x C complex matrix and V the C x NB
// complex spectra (NB = batch * planes, or batch * lateral points).  In real form
//     [Ur; Ui] = [[Kr, -Ki], [Ki, Kr]] [Vr; Vi],
// so a tile of 128 columns n is the real GEMM  D (128 x 2C) = A (128 x 2C) * B^T with
// A[n][k] = (Vr; Vi)[k][n] and B[o][k] = Kreal[o][k], operands rounded to bfloat16 (round to
// nearest even, the precision the workload prescribes for the mixing) and accumulated in FP32
// in tensor memory: tcgen05.mma kind::f16, M = 128, N = 2C = 64, four K = 16 steps, issued by
// one thread; operands staged in shared memory in the canonical K-major layout without swizzle
// (8-row x 16-byte core matrices: K-adjacent core matrices 128 B apart, 8-row groups 1024 B apart).
#include <mutex>
#include <cuda_bf16.h>

#include <cstdint>
#include <cstdlib>

#include "internal.h"
#include "pdl.cuh"

namespace {

constexpr int TC_C = 32;            // channels
constexpr int TC_K = 2 * TC_C;      // real-form K = N = 64
constexpr int TC_M = 128;           // columns n per tile (MMA M)
constexpr int TC_THREADS = 128;     // one thread per tile row; four warps cover the 128 TMEM lanes
constexpr uint32_t TC_TMEM_COLS = 64;
constexpr int A_BYTES = TC_M * TC_K * 2;     // 16 KB
constexpr int B_BYTES = TC_K * TC_K * 2;     // 8 KB

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// byte offset of element (row, k) in the K-major, no-swizzle core-matrix layout (K = 64)
__device__ __forceinline__ int kmajor_off(int row, int k) {
  return (((row >> 3) * (TC_K / 8) + (k >> 3)) << 7) + ((row & 7) << 4) + ((k & 7) << 1);
}

// shared-memory matrix descriptor: start address, leading (K) and stride (8-row) byte offsets,
// descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) {
  constexpr uint64_t LBO = 128, SBO = 1024;
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((LBO >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((SBO >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: FP32 accumulate, BF16 A and B, both K-major, N = 64, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TC_K >> 3) << 17) |
                            ((uint32_t)(TC_M >> 4) << 24);

__device__ __forceinline__ bool mbar_wait(uint32_t mb, uint32_t parity, long limit) {
  uint32_t ok = 0;
  for (long it = 0; it < limit && !ok; ++it) {
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok) : "r"(mb), "r"(parity) : "memory");
  }
  return ok != 0;
}

// 16 consecutive FP32 columns of this thread's TMEM lane; the wait is in the same statement, so
// the destination registers are complete before the compiler can touch them
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
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

// grid (ceil(NB / 128), modes); U[mode][o][n] = sum_i K[row(mode)][o][i] V[mode][i][n]
__global__ void __launch_bounds__(TC_THREADS) k_mix_tc(const cf* __restrict__ V, cf* __restrict__ U,
                                                       const cf* __restrict__ K, long NB, int mx, int MX, int offy,
                                                       int offx, int* err) {
  pdl_enter();
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char* As = sm;
  unsigned char* Bs = sm + A_BYTES;
  __shared__ __align__(8) unsigned long long mbar;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5;
  const long mode = blockIdx.y;
  const int jy = (int)(mode / mx), jx = (int)(mode - (long)jy * mx);
  const long krow = (long)(jy + offy) * MX + (jx + offx);
  const cf* Km = K + krow * TC_C * TC_C;
  const cf* Vm = V + mode * TC_C * NB;
  const long n0 = (long)blockIdx.x * TC_M;

  // TMEM columns for the 128 x 64 FP32 accumulator (one warp allocates for the CTA)
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_addr(&tmem_base)), "r"(TC_TMEM_COLS) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_addr(&mbar)) : "memory");
  }
  // A: row t = column n0 + t of V in real form (bf16); B: the real form of K (bf16)
  {
    const long n = n0 + tid;
    const bool in = n < NB;
#pragma unroll 4
    for (int c = 0; c < TC_C; ++c) {
      const cf v = in ? Vm[(long)c * NB + n] : make_float2(0.f, 0.f);
      *reinterpret_cast<__nv_bfloat16*>(As + kmajor_off(tid, c)) = __float2bfloat16_rn(v.x);
      *reinterpret_cast<__nv_bfloat16*>(As + kmajor_off(tid, TC_C + c)) = __float2bfloat16_rn(v.y);
    }
    for (int e = tid; e < TC_C * TC_C; e += TC_THREADS) {
      const int o = e / TC_C, i = e - o * TC_C;
      const cf kv = Km[e];
      const __nv_bfloat16 kr = __float2bfloat16_rn(kv.x), ki = __float2bfloat16_rn(kv.y);
      const __nv_bfloat16 nki = __float2bfloat16_rn(-kv.y);   // exact negation of the rounded value
      *reinterpret_cast<__nv_bfloat16*>(Bs + kmajor_off(o, i)) = kr;
      *reinterpret_cast<__nv_bfloat16*>(Bs + kmajor_off(o, TC_C + i)) = nki;
      *reinterpret_cast<__nv_bfloat16*>(Bs + kmajor_off(TC_C + o, i)) = ki;
      *reinterpret_cast<__nv_bfloat16*>(Bs + kmajor_off(TC_C + o, TC_C + i)) = kr;
    }
  }
  // generic-proxy shared stores -> visible to the tensor core (async proxy); TMEM address visible
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t taddr = tmem_base;
  const uint32_t mb = smem_addr(&mbar);
  if (tid == 0) {
    const uint32_t a0 = smem_addr(As), b0 = smem_addr(Bs);
#pragma unroll
    for (int kk = 0; kk < TC_K / 16; ++kk) {
      // K = 16 elements = two core matrices along K
      const uint64_t ad = make_desc(a0 + kk * 256), bd = make_desc(b0 + kk * 256);
      const uint32_t acc = kk > 0 ? 1u : 0u;
      asm volatile(
          "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
          " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
          :: "r"(taddr), "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc) : "memory");
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(mb)
                 : "memory");
  }
  const bool done = mbar_wait(mb, 0, 1L << 24);
  if (__syncthreads_or(!done)) {
    // the products did not complete in time: report, wait once more for them, free TMEM, leave
    if (tid == 0) atomicExch(err, 1);
    mbar_wait(mb, 0, 1L << 24);
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(taddr), "r"(TC_TMEM_COLS)
                                : "memory");
    return;
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // row n0 + tid lives in TMEM lane tid (warp w reads lanes 32 w .. 32 w + 31)
  const uint32_t trow = taddr + ((uint32_t)(warp * 32) << 16);
  float d[TC_K];
#pragma unroll
  for (int q = 0; q < TC_K / 16; ++q) {
    float v[16];
    tmem_ld16(trow + q * 16, v);
#pragma unroll
    for (int i = 0; i < 16; ++i) d[q * 16 + i] = v[i];
  }
  const long n = n0 + tid;
  if (n < NB) {
    cf* Um = U + mode * TC_C * NB;
#pragma unroll
    for (int o = 0; o < TC_C; ++o) Um[(long)o * NB + n] = make_float2(d[o], d[TC_C + o]);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(taddr), "r"(TC_TMEM_COLS) : "memory");
  }
}

int* g_tc_err = nullptr;

}  // namespace

// 1 when the forward mixing runs on the tensor cores (PSFD_MIX_SIMT=1 selects the SIMT kernel)
bool fno_mix_tc_enabled(int C) {
  const char* e = getenv("PSFD_MIX_SIMT");
  return C == TC_C && !(e && e[0] == '1');
}

int fno_mix_tc(const cf* V, cf* U, const cf* K, long NB, int modes, int mx, int MX, int offy, int offx,
               cudaStream_t s) {
  static std::once_flag once;   // once per process, complete before any host thread launches
  static cudaError_t init = cudaSuccess;
  std::call_once(once, [] {
    int* p = nullptr;
    init = cudaMalloc((void**)&p, sizeof(int));
    if (init == cudaSuccess) init = cudaMemset(p, 0, sizeof(int));
    if (init == cudaSuccess) g_tc_err = p;
  });
  if (init != cudaSuccess || !g_tc_err) {
    psfd_set_error("fno mixing: set-up: %s", cudaGetErrorString(init));
    return PSFD_ERR_CUDA;
  }
  dim3 g((unsigned)((NB + TC_M - 1) / TC_M), (unsigned)modes);
  (void)launch_pdl(k_mix_tc, dim3(g), dim3(TC_THREADS), A_BYTES + B_BYTES, s, V, U, K, NB, mx, MX, offy, offx, g_tc_err);
  PSFD_CHECK_LAUNCH();
  return PSFD_OK;
}

int fno_mix_tc_error(int* host_flag) {
  *host_flag = 0;
  if (!g_tc_err) return PSFD_OK;
  PSFD_CUDA_TRY(cudaMemcpy(host_flag, g_tc_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (*host_flag) PSFD_CUDA_TRY(cudaMemset(g_tc_err, 0, sizeof(int)));
  return PSFD_OK;
}
