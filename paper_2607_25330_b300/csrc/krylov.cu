// Right-preconditioned Krylov solves with the affine warm start (Sec. 3:
// Eqs. right_preconditioned, right_correction_solution,
// right_preconditioned_system, relative_residual).
//
// All vectors are complex64 in the HYBRID domain, batched over the plan's
// right-hand sides; every scalar is FP64 and stays on the device.  Inner
// products use error-free transformations: each thread accumulates exact
// float products (TwoProduct via fma) with a compensated float sum (TwoSum),
// which gives twice-float accuracy per thread; the per-thread results are then
// summed in FP64 in a fixed order (warp tree, block tree, blocks in index
// order by the last block to finish), so results are reproducible run to run.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <thread>
#include <cstdio>
#include <vector>

#include "fft.cuh"
#include "internal.h"
#include "pdl.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kMaxQ = 4;  // reals reduced per kernel

struct KScal {
  double2 rho, rho_old, alpha, omega, rv, ts;
  double tt, rr, bnorm2, rr0, res0, res1;
  int status, iters, maxit, pad;
  double tol2;
};

// Per-thread compensated accumulator (Kahan): the BiCGSTAB kernels add the plain FP32 partial of
// one batch of elements (at most 16 products, exact inside each FMA, error about 16 u sum|p| with
// u = 2^-24) into it once per batch, so the compensated chain runs once per batch instead of once
// per product; partials of threads and blocks are then summed in FP64.
struct Acc2 {
  float s, c, e;
};

__device__ __forceinline__ void acc_add(Acc2& A, float v) {
  const float y = __fsub_rn(v, A.c);
  const float t = __fadd_rn(A.s, y);
  A.c = __fsub_rn(__fsub_rn(t, A.s), y);
  A.s = t;
}

__device__ __forceinline__ double acc_value(const Acc2& A) {
  return (double)A.s - (double)A.c + (double)A.e;
}
// |a|^2 into the running sum, uncompensated: a sum of positive terms has no cancellation, so the
// per-thread FP32 partial (a few tens of terms) keeps about 1e-6 relative accuracy, ample for
// omega's denominator and the convergence tests; the partials are summed in FP64
__device__ __forceinline__ void acc_norm(Acc2& A, cf a) { A.s = fmaf(a.x, a.x, fmaf(a.y, a.y, A.s)); }

// re/im of conj(a) * b into a batch partial (plain FMA chains)
__device__ __forceinline__ void acc_cdot_plain(Acc2& re, Acc2& im, cf a, cf b) {
  re.s = fmaf(a.x, b.x, fmaf(a.y, b.y, re.s));
  im.s = fmaf(a.x, b.y, fmaf(-a.y, b.x, im.s));
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-reduce NQ doubles; write partials; the last block of this rhs sums the
// partials in index order and returns true with the totals in out[].
// Generic form: `pbase` holds gridDim.x * QS doubles for this reduction group,
// `counter` counts finished blocks of the group.
template <int NQ, int QS>
__device__ bool reduce_group(double (&val)[NQ], double* pbase, unsigned* counter, double* out) {
  __shared__ double sh[kThreads / 32][QS];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    double v = warp_sum(val[q]);
    if (lane == 0) sh[warp][q] = v;
  }
  __syncthreads();
  double* part = pbase + (long)blockIdx.x * QS;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      double s = 0;
      for (int w = 0; w < kThreads / 32; ++w) s += sh[w][q];
      part[q] = s;
    }
    __threadfence();
    unsigned prev = atomicAdd(counter, 1u);
    last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  // last block: every thread sums a fixed strided subset of the partials, then the
  // same fixed tree as above (deterministic for a given grid)
  const volatile double* base = pbase;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    double s = 0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) s += base[b * QS + q];
    s = warp_sum(s);
    if (lane == 0) sh[warp][q] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      double s = 0;
      for (int w = 0; w < kThreads / 32; ++w) s += sh[w][q];
      out[q] = s;
    }
    *counter = 0;  // ready for the next reduction
  }
  return true;
}

template <int NQ>
__device__ bool reduce_finish(double (&val)[NQ], double* partials, unsigned* counters, double* out) {
  const int rhs = blockIdx.y;
  return reduce_group<NQ, kMaxQ>(val, partials + (long)rhs * gridDim.x * kMaxQ, counters + rhs, out);
}

__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 zdiv(double2 a, double2 b) {
  const double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
__device__ __forceinline__ double zabs(double2 a) { return hypot(a.x, a.y); }
__device__ __forceinline__ cf zf(double2 a) { return make_float2((float)a.x, (float)a.y); }

enum {
  OK_INIT = 0,   // rhat = r, p = v = y = 0; <r, r> -> rho, rr, rr0
  OK_P = 1,      // p = r + beta (p - omega v)
  OK_RV = 2,     // <rhat, v> -> alpha
  OK_S = 3,      // s = r - alpha v
  OK_TS = 4,     // <t, s>, <t, t> -> omega
  OK_XR = 5,     // y += alpha p + omega s ; r = s - omega t ; <rhat, r>, <r, r>
  OK_NORM = 6,   // <a, a> -> res0
  OK_SUB = 7,    // c = a - b ; <c, c> -> res1
  OK_AXPY = 8    // c = a + b
};

struct VArgs {
  cf* v0;  // meaning depends on the op
  cf* v1;
  cf* v2;
  cf* v3;
  cf* v4;
  cf* v5;
  long n;  // complex entries per rhs
  KScal* sc;
  int* done;
  double* partials;
  unsigned* counters;
  double* hist;
  int hist_cap;
  bool use_done;
  int* prog;   // nullable, host-mapped [2][nrhs]: iterations completed and done flag per rhs
};

// the progress word of a rhs for the host (a hint: the kernels decide on a.done alone)
__device__ __forceinline__ void post_progress(int* prog, int rhs, int iters, int done) {
  if (!prog) return;
  volatile int* q = prog;
  q[rhs] = iters;
  q[gridDim.y + rhs] = done;
  __threadfence_system();
}

template <int OP>
__global__ void __launch_bounds__(kThreads) k_vec(VArgs a) {
  pdl_enter();
  const int rhs = blockIdx.y;
  KScal* S = a.sc + rhs;
  if (a.use_done && a.done[rhs]) return;
  const long off = (long)rhs * a.n;
  const long n2 = a.n / 2;  // float4 = 2 complex
  const long stride = (long)gridDim.x * blockDim.x;
  Acc2 acc[kMaxQ];
#pragma unroll
  for (int q = 0; q < kMaxQ; ++q) acc[q] = {0.f, 0.f, 0.f};

  cf beta = czero(), omg = czero(), alp = czero();
  if constexpr (OP == OK_P) {
    // beta = (rho / rho_old) (alpha / omega)
    const double2 b = zmul(zdiv(S->rho, S->rho_old), zdiv(S->alpha, S->omega));
    beta = zf(b);
    omg = zf(S->omega);
  }
  if constexpr (OP == OK_S || OP == OK_XR) alp = zf(S->alpha);
  if constexpr (OP == OK_XR) omg = zf(S->omega);

  // Batches of kU elements per thread: every load of a batch is issued before the first use,
  // so that kU x (vectors read) float4 loads are in flight; the batch's products are summed in
  // plain FMA chains and enter the compensated sums once per batch.
  constexpr int NIN = (OP == OK_XR) ? 5 : (OP == OK_P) ? 3 : (OP == OK_INIT || OP == OK_NORM) ? 1 : 2;
  constexpr int kU = (NIN >= 3) ? 2 : 4;
  auto ld4 = [&](const cf* v, long e) { return __ldg(reinterpret_cast<const float4*>(v) + e); };
  auto load = [&](long e, float4 (&L)[5]) {
    if constexpr (OP == OK_INIT || OP == OK_NORM) {
      L[0] = ld4(a.v0, e);
    } else if constexpr (OP == OK_P) {          // p, r, v
      L[0] = ld4(a.v0, e); L[1] = ld4(a.v1, e); L[2] = ld4(a.v2, e);
    } else if constexpr (OP == OK_S) {          // r, v
      L[1] = ld4(a.v1, e); L[2] = ld4(a.v2, e);
    } else if constexpr (OP == OK_XR) {         // y, p, s, t, rhat
      L[0] = ld4(a.v0, e); L[1] = ld4(a.v2, e); L[2] = ld4(a.v3, e); L[3] = ld4(a.v4, e); L[4] = ld4(a.v5, e);
    } else {                                    // RV, TS, SUB, AXPY: v0, v1
      L[0] = ld4(a.v0, e); L[1] = ld4(a.v1, e);
    }
  };
  auto body = [&](long e, const float4 (&L)[5], Acc2* A) {
    if constexpr (OP == OK_INIT) {
      // v0 = r, v1 = rhat, v2 = p, v3 = v, v4 = y
      const float4 r = L[0];
      reinterpret_cast<float4*>(a.v1)[e] = r;
      const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
      reinterpret_cast<float4*>(a.v2)[e] = z;
      reinterpret_cast<float4*>(a.v3)[e] = z;
      reinterpret_cast<float4*>(a.v4)[e] = z;
      acc_norm(A[0], make_float2(r.x, r.y));
      acc_norm(A[0], make_float2(r.z, r.w));
    } else if constexpr (OP == OK_P) {
      // v0 = p (in/out), v1 = r, v2 = v
      const float4 pp = L[0], rr = L[1], vv = L[2];
      cf p0 = make_float2(pp.x, pp.y), p1 = make_float2(pp.z, pp.w);
      cf t0 = csub(p0, cmul(omg, make_float2(vv.x, vv.y)));
      cf t1 = csub(p1, cmul(omg, make_float2(vv.z, vv.w)));
      cf o0 = cfma(beta, t0, make_float2(rr.x, rr.y));
      cf o1 = cfma(beta, t1, make_float2(rr.z, rr.w));
      reinterpret_cast<float4*>(a.v0)[e] = make_float4(o0.x, o0.y, o1.x, o1.y);
    } else if constexpr (OP == OK_RV) {
      // v0 = rhat, v1 = v
      const float4 h = L[0], v = L[1];
      acc_cdot_plain(A[0], A[1], make_float2(h.x, h.y), make_float2(v.x, v.y));
      acc_cdot_plain(A[0], A[1], make_float2(h.z, h.w), make_float2(v.z, v.w));
    } else if constexpr (OP == OK_S) {
      // v0 = s (out), v1 = r, v2 = v
      const float4 rr = L[1], vv = L[2];
      cf s0 = csub(make_float2(rr.x, rr.y), cmul(alp, make_float2(vv.x, vv.y)));
      cf s1 = csub(make_float2(rr.z, rr.w), cmul(alp, make_float2(vv.z, vv.w)));
      reinterpret_cast<float4*>(a.v0)[e] = make_float4(s0.x, s0.y, s1.x, s1.y);
    } else if constexpr (OP == OK_TS) {
      // v0 = t, v1 = s
      const float4 tt = L[0], ss = L[1];
      cf t0 = make_float2(tt.x, tt.y), t1 = make_float2(tt.z, tt.w);
      acc_cdot_plain(A[0], A[1], t0, make_float2(ss.x, ss.y));
      acc_cdot_plain(A[0], A[1], t1, make_float2(ss.z, ss.w));
      acc_norm(A[2], t0);
      acc_norm(A[2], t1);
    } else if constexpr (OP == OK_XR) {
      // v0 = y, v1 = r (out), v2 = p, v3 = s, v4 = t, v5 = rhat
      const float4 yy = L[0], pp = L[1], ss = L[2], tt = L[3], hh = L[4];
      cf s0 = make_float2(ss.x, ss.y), s1 = make_float2(ss.z, ss.w);
      cf y0 = cfma(alp, make_float2(pp.x, pp.y), make_float2(yy.x, yy.y));
      cf y1 = cfma(alp, make_float2(pp.z, pp.w), make_float2(yy.z, yy.w));
      y0 = cfma(omg, s0, y0);
      y1 = cfma(omg, s1, y1);
      cf r0 = csub(s0, cmul(omg, make_float2(tt.x, tt.y)));
      cf r1 = csub(s1, cmul(omg, make_float2(tt.z, tt.w)));
      reinterpret_cast<float4*>(a.v0)[e] = make_float4(y0.x, y0.y, y1.x, y1.y);
      reinterpret_cast<float4*>(a.v1)[e] = make_float4(r0.x, r0.y, r1.x, r1.y);
      acc_cdot_plain(A[0], A[1], make_float2(hh.x, hh.y), r0);
      acc_cdot_plain(A[0], A[1], make_float2(hh.z, hh.w), r1);
      acc_norm(A[2], r0);
      acc_norm(A[2], r1);
    } else if constexpr (OP == OK_NORM) {
      const float4 x = L[0];
      acc_norm(A[0], make_float2(x.x, x.y));
      acc_norm(A[0], make_float2(x.z, x.w));
    } else if constexpr (OP == OK_SUB) {
      // v2 = v0 - v1
      const float4 x = L[0], y = L[1];
      const float4 c = make_float4(x.x - y.x, x.y - y.y, x.z - y.z, x.w - y.w);
      reinterpret_cast<float4*>(a.v2)[e] = c;
      acc_norm(A[0], make_float2(c.x, c.y));
      acc_norm(A[0], make_float2(c.z, c.w));
    } else if constexpr (OP == OK_AXPY) {
      const float4 x = L[0], y = L[1];
      reinterpret_cast<float4*>(a.v2)[e] = make_float4(x.x + y.x, x.y + y.y, x.z + y.z, x.w + y.w);
    }
  };
  for (long i0 = (long)blockIdx.x * blockDim.x + threadIdx.x; i0 < n2; i0 += kU * stride) {
    float4 L[kU][5];
#pragma unroll
    for (int u = 0; u < kU; ++u)
      if (i0 + u * stride < n2) load(off / 2 + i0 + u * stride, L[u]);
    Acc2 Bt[kMaxQ];   // this batch's plain partials
#pragma unroll
    for (int q = 0; q < kMaxQ; ++q) Bt[q] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int u = 0; u < kU; ++u)
      if (i0 + u * stride < n2) body(off / 2 + i0 + u * stride, L[u], Bt);
#pragma unroll
    for (int q = 0; q < kMaxQ; ++q) acc_add(acc[q], Bt[q].s);
  }

  constexpr int NQ = (OP == OK_TS || OP == OK_XR) ? 4 : ((OP == OK_INIT || OP == OK_RV || OP == OK_NORM || OP == OK_SUB) ? 2 : 0);
  if constexpr (NQ > 0) {
    double val[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) val[q] = acc_value(acc[q]);
    double tot[NQ];
    if (!reduce_finish<NQ>(val, a.partials, a.counters, tot)) return;
    if (threadIdx.x != 0) return;
    // ---- scalar updates (one thread per rhs)
    if constexpr (OP == OK_INIT) {
      S->rho = make_double2(tot[0], 0.0);
      S->rho_old = make_double2(1.0, 0.0);
      S->alpha = make_double2(1.0, 0.0);
      S->omega = make_double2(1.0, 0.0);
      S->rr = tot[0];
      S->rr0 = tot[0];
      S->iters = 0;
      S->status = PSFD_NOT_CONVERGED;
      int d = 0;
      if (tot[0] <= S->tol2 * S->bnorm2) { d = 1; S->status = PSFD_OK; }
      if (S->maxit <= 0) d = 1;
      a.done[rhs] = d;
      post_progress(a.prog, rhs, 0, d);
    } else if constexpr (OP == OK_RV) {
      S->rv = make_double2(tot[0], tot[1]);
      const double arv = zabs(S->rv);
      if (!(arv > 1e-300) || !isfinite(arv)) {
        S->status = PSFD_ERR_BREAKDOWN;
        S->alpha = make_double2(0.0, 0.0);
        a.done[rhs] = 1;
        post_progress(a.prog, rhs, S->iters, 1);
      } else {
        S->alpha = zdiv(S->rho, S->rv);
      }
    } else if constexpr (OP == OK_TS) {
      S->ts = make_double2(tot[0], tot[1]);
      S->tt = tot[2];
      S->omega = (tot[2] > 0.0) ? make_double2(tot[0] / tot[2], tot[1] / tot[2]) : make_double2(0.0, 0.0);
    } else if constexpr (OP == OK_XR) {
      S->rho_old = S->rho;
      S->rho = make_double2(tot[0], tot[1]);
      S->rr = tot[2];
      const int it = ++S->iters;
      const double rel = sqrt(tot[2] / S->bnorm2);
      if (a.hist && it - 1 < a.hist_cap) a.hist[(long)rhs * a.hist_cap + it - 1] = rel;
      int d = 0;
      if (!isfinite(tot[2])) { S->status = PSFD_ERR_BREAKDOWN; d = 1; }
      else if (tot[2] <= S->tol2 * S->bnorm2) { S->status = PSFD_OK; d = 1; }
      else if (!(zabs(S->rho) > 1e-300) || !(zabs(S->omega) > 0.0)) { S->status = PSFD_ERR_BREAKDOWN; d = 1; }
      else if (it >= S->maxit) { S->status = PSFD_NOT_CONVERGED; d = 1; }
      a.done[rhs] = d;
      post_progress(a.prog, rhs, it, d);
    } else if constexpr (OP == OK_NORM) {
      S->res0 = tot[0];
    } else if constexpr (OP == OK_SUB) {
      S->res1 = tot[0];
    }
  }
}

// SMs of the current device (thread-safe one-time query; 148 when it fails)
int device_sms() {
  static const int n = [] {
    int dev = 0, m = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&m, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        m <= 0)
      m = 148;
    return m;
  }();
  return n;
}

// CTAs of KERNEL resident per SM at kThreads threads (one-time query per kernel; 1 when it fails)
template <auto KERNEL>
int per_sm_of() {
  static const int b = [] {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, KERNEL, kThreads, 0) != cudaSuccess || n < 1) n = 1;
    return n;
  }();
  return b;
}

// Grid-stride streaming kernels run as one wave of resident CTAs shared by `groups` grid slices
// (right-hand sides, basis chunks), at most `cap` CTAs per slice (what the reduction partials were
// sized for): a fraction of a second wave would leave SMs idle at the end of every pass.
template <auto KERNEL>
int one_wave(int cap, int groups) {
  const long w = (long)per_sm_of<KERNEL>() * device_sms() / std::max(1, groups);
  return (int)std::max(1L, std::min<long>(cap, w));
}

// compulsory complex64 vector passes (reads + writes) of each vector kernel
constexpr int vec_passes(int op) {
  return op == OK_INIT ? 5 : op == OK_P ? 4 : op == OK_RV ? 2 : op == OK_S ? 3 : op == OK_TS ? 2
       : op == OK_XR ? 7 : op == OK_NORM ? 1 : op == OK_SUB ? 3 : 3;
}

template <int OP>
int launch_vec(const VArgs& a, int nrhs, cudaStream_t s, int nblocks) {
  StageScope sc(s, ST_KRYLOV, (double)vec_passes(OP) * nrhs * a.n * sizeof(cf));
  dim3 grid((unsigned)one_wave<k_vec<OP>>(nblocks, nrhs), (unsigned)nrhs);
  (void)launch_pdl(k_vec<OP>, grid, dim3(kThreads), 0, s, a);
  PSFD_CHECK_LAUNCH();
  return PSFD_OK;
}

__global__ void k_set_scalars(KScal* sc, int nrhs, double tol2, int maxit) {
  pdl_enter();
  int r = threadIdx.x;
  if (r < nrhs) {
    KScal z{};
    z.tol2 = tol2;
    z.maxit = maxit;
    z.status = PSFD_NOT_CONVERGED;
    sc[r] = z;
  }
}
__global__ void k_copy_bnorm(KScal* sc, int nrhs) {
  pdl_enter();
  int r = threadIdx.x;
  if (r < nrhs) sc[r].bnorm2 = sc[r].res0;
}

// per-rhs flags from the host, passed as a kernel argument (one bit per rhs) instead of a copy
struct RhsBits {
  static constexpr int kMax = 1024;
  unsigned long long w[kMax / 64];
};
__global__ void k_set_flags(int* f, int nrhs, RhsBits b) {
  pdl_enter();
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < nrhs) f[r] = (int)((b.w[r >> 6] >> (r & 63)) & 1ull);
}

}  // namespace


// ======================================================================= GMRES(m)
// Arnoldi with classical Gram-Schmidt applied twice (CGS2); the Hessenberg
// matrix, the Givens rotations and the small triangular solve are FP64 on the
// device (one thread per right-hand side).
namespace {

constexpr int GCH = 8;       // basis vectors per multi-dot block
constexpr int GMAX = 256;    // largest restart length supported

struct GState {
  double2 H[(GMAX + 1) * GMAX];  // column-major: H[i + j*(m+1)]
  double2 cs[GMAX], sn[GMAX], g[GMAX + 1], z[GMAX];
  double beta, bnorm2, tol2;
  int jd, iters, maxit, status, m, active, pad0, pad1;
};

struct GArgs {
  cf* V;           // basis, V_i at V + i * vs (each [nrhs][n])
  long vs;
  long n;
  int nv;          // vectors used (multi-dot / update)
  int j;           // Arnoldi column being built
  GState* gs;
  const int* mask; // skip rhs with mask != 0 (nullable)
  double* partials;
  unsigned* counters;
  double2* hout;   // [nrhs][GMAX] results of the multi-dot
  cf* w;           // target vector (V_{j+1})
  cf* y;           // solution accumulator
  KScal* sc;       // per-rhs scalars: res0 <- ||w||^2 after an update, tt <- ||w||^2 before
  bool save_norm;  // k_gdot: also reduce ||w||^2 (chunk 0) into sc.tt
};

// mask: nonzero = skip this right-hand side (same convention as the operator kernels)
__device__ __forceinline__ bool skip_rhs(const GArgs& a, int rhs) { return a.mask && a.mask[rhs]; }

// h[i] = <V_i, w>, i in [chunk*GCH, min(nv, chunk*GCH+GCH)).  Per-thread partial sums are
// plain float over ~20 elements (two interleaved accumulators), summed in FP64 across
// threads and blocks; a second Gram-Schmidt pass is taken whenever the first one
// cancels more than half of ||w||^2, which also absorbs the rounding of these partials.
__global__ void __launch_bounds__(kThreads) k_gdot(GArgs a) {
  pdl_enter();
  const int rhs = blockIdx.y, chunk = blockIdx.z;
  if (skip_rhs(a, rhs)) return;
  const int i0 = chunk * GCH;
  const int nq = min(GCH, a.nv - i0);
  if (nq <= 0) return;
  float sr[GCH], si[GCH];
#pragma unroll
  for (int q = 0; q < GCH; ++q) { sr[q] = 0.f; si[q] = 0.f; }
  float ww = 0.f;
  const bool want_ww = a.save_norm && chunk == 0;
  const long n2 = a.n / 2, off2 = (long)rhs * a.n / 2;
  const float4* w4 = reinterpret_cast<const float4*>(a.w);
  // two elements per thread and pass, all (nq + 1) x 2 loads issued before the arithmetic
  const long stride = (long)gridDim.x * blockDim.x;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += 2 * stride) {
    const bool two = i + stride < n2;
    const float4 wv0 = __ldg(w4 + off2 + i);
    const float4 wv1 = two ? __ldg(w4 + off2 + i + stride) : make_float4(0.f, 0.f, 0.f, 0.f);
    float4 v0[GCH], v1[GCH];
#pragma unroll
    for (int q = 0; q < GCH; ++q) {
      if (q < nq) {
        const float4* vq = reinterpret_cast<const float4*>(a.V + (i0 + q) * a.vs) + off2;
        v0[q] = __ldg(vq + i);
        v1[q] = two ? __ldg(vq + i + stride) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    if (want_ww) {
      ww = fmaf(wv0.x, wv0.x, fmaf(wv0.y, wv0.y, fmaf(wv0.z, wv0.z, fmaf(wv0.w, wv0.w, ww))));
      ww = fmaf(wv1.x, wv1.x, fmaf(wv1.y, wv1.y, fmaf(wv1.z, wv1.z, fmaf(wv1.w, wv1.w, ww))));
    }
#pragma unroll
    for (int q = 0; q < GCH; ++q) {
      if (q < nq) {
        // conj(v) * w for the four complex entries
        const float4 a0 = v0[q], b0 = v1[q];
        sr[q] = fmaf(a0.x, wv0.x, fmaf(a0.y, wv0.y, fmaf(a0.z, wv0.z, fmaf(a0.w, wv0.w, sr[q]))));
        si[q] = fmaf(a0.x, wv0.y, fmaf(-a0.y, wv0.x, fmaf(a0.z, wv0.w, fmaf(-a0.w, wv0.z, si[q]))));
        sr[q] = fmaf(b0.x, wv1.x, fmaf(b0.y, wv1.y, fmaf(b0.z, wv1.z, fmaf(b0.w, wv1.w, sr[q]))));
        si[q] = fmaf(b0.x, wv1.y, fmaf(-b0.y, wv1.x, fmaf(b0.z, wv1.w, fmaf(-b0.w, wv1.z, si[q]))));
      }
    }
  }
  constexpr int NQ = 2 * GCH + 1;
  double val[NQ];
#pragma unroll
  for (int q = 0; q < GCH; ++q) { val[2 * q] = (double)sr[q]; val[2 * q + 1] = (double)si[q]; }
  val[2 * GCH] = (double)ww;
  double tot[NQ];
  double* pbase = a.partials + ((long)rhs * gridDim.z + chunk) * gridDim.x * (NQ + 1);
  if (!reduce_group<NQ, NQ + 1>(val, pbase, a.counters + rhs * gridDim.z + chunk, tot)) return;
  if (threadIdx.x == 0) {
    for (int q = 0; q < nq; ++q) a.hout[rhs * GMAX + i0 + q] = make_double2(tot[2 * q], tot[2 * q + 1]);
    if (want_ww) a.sc[rhs].tt = tot[2 * GCH];
  }
}

// per rhs: keep the norm of w before orthogonalisation (res0 -> tt), zero the second-pass
// coefficients, and after the first pass decide whether a second one is needed
__global__ void k_gsave(double2* h2, int nrhs, int nv) {
  pdl_enter();
  const int r = blockIdx.x;
  if (r >= nrhs) return;
  for (int i = threadIdx.x; i < nv; i += blockDim.x) h2[r * GMAX + i] = make_double2(0.0, 0.0);
}
__global__ void k_greorth(const KScal* sc, const int* skip, int* skip2, int nrhs) {
  pdl_enter();
  const int r = threadIdx.x;
  if (r >= nrhs) return;
  // second pass when ||w_after||^2 < ||w_before||^2 / 2 (Daniel-Gragg-Kaufman-Stewart, eta = 1/sqrt(2))
  skip2[r] = (skip && skip[r]) || !(sc[r].res0 < 0.5 * sc[r].tt);
}

// w -= sum_i h[i] V_i  (h from hout)   or   y += sum_i z[i] V_i (ADD, count jd per rhs)
template <bool ADD>
__global__ void __launch_bounds__(kThreads) k_gupd(GArgs a) {
  pdl_enter();
  const int rhs = blockIdx.y;
  if (skip_rhs(a, rhs)) return;
  const int nv = ADD ? a.gs[rhs].jd : a.nv;
  if (nv <= 0) return;
  __shared__ cf coef[GMAX];
  for (int i = threadIdx.x; i < nv; i += blockDim.x) {
    const double2 c = ADD ? a.gs[rhs].z[i] : a.hout[rhs * GMAX + i];
    coef[i] = ADD ? make_float2((float)c.x, (float)c.y) : make_float2((float)-c.x, (float)-c.y);
  }
  __syncthreads();
  const long n2 = a.n / 2, off2 = (long)rhs * a.n / 2;
  float4* t4 = reinterpret_cast<float4*>(ADD ? a.y : a.w);
  float ww = 0.f;
  // two elements per thread and pass; the basis vectors in groups of four, loads first
  const long stride = (long)gridDim.x * blockDim.x;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += 2 * stride) {
    const bool two = i + stride < n2;
    const float4 acc0 = t4[off2 + i];
    const float4 acc1 = two ? t4[off2 + i + stride] : make_float4(0.f, 0.f, 0.f, 0.f);
    cf a0 = make_float2(acc0.x, acc0.y), a1 = make_float2(acc0.z, acc0.w);
    cf b0 = make_float2(acc1.x, acc1.y), b1 = make_float2(acc1.z, acc1.w);
    int q = 0;
    for (; q + 4 <= nv; q += 4) {
      float4 u[4], v[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float4* vq = reinterpret_cast<const float4*>(a.V + (q + k) * a.vs) + off2;
        u[k] = __ldg(vq + i);
        v[k] = two ? __ldg(vq + i + stride) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const cf c = coef[q + k];
        a0 = cfma(c, make_float2(u[k].x, u[k].y), a0);
        a1 = cfma(c, make_float2(u[k].z, u[k].w), a1);
        b0 = cfma(c, make_float2(v[k].x, v[k].y), b0);
        b1 = cfma(c, make_float2(v[k].z, v[k].w), b1);
      }
    }
    for (; q < nv; ++q) {
      const float4* vq = reinterpret_cast<const float4*>(a.V + q * a.vs) + off2;
      const float4 u = __ldg(vq + i);
      const float4 v = two ? __ldg(vq + i + stride) : make_float4(0.f, 0.f, 0.f, 0.f);
      a0 = cfma(coef[q], make_float2(u.x, u.y), a0);
      a1 = cfma(coef[q], make_float2(u.z, u.w), a1);
      b0 = cfma(coef[q], make_float2(v.x, v.y), b0);
      b1 = cfma(coef[q], make_float2(v.z, v.w), b1);
    }
    t4[off2 + i] = make_float4(a0.x, a0.y, a1.x, a1.y);
    if (two) t4[off2 + i + stride] = make_float4(b0.x, b0.y, b1.x, b1.y);
    if (!ADD) {
      ww = fmaf(a0.x, a0.x, fmaf(a0.y, a0.y, fmaf(a1.x, a1.x, fmaf(a1.y, a1.y, ww))));
      ww = fmaf(b0.x, b0.x, fmaf(b0.y, b0.y, fmaf(b1.x, b1.x, fmaf(b1.y, b1.y, ww))));
    }
  }
  if constexpr (!ADD) {
    // ||w||^2 after the update (per-thread float partials, FP64 across threads)
    double val[2] = {(double)ww, 0.0};
    double tot[2];
    if (!reduce_group<2, kMaxQ>(val, a.partials + (long)rhs * gridDim.x * kMaxQ, a.counters + rhs, tot)) return;
    if (threadIdx.x == 0) a.sc[rhs].res0 = tot[0];
  }
}

// V_0 = r / beta, or V_{j+1} = w / H[j+1][j]
__global__ void k_gscale(GArgs a, bool first) {
  pdl_enter();
  const int rhs = blockIdx.y;
  if (skip_rhs(a, rhs)) return;
  const GState& G = a.gs[rhs];
  const double b = first ? G.beta : G.H[(a.j + 1) + a.j * (G.m + 1)].x;
  const float inv = b > 0 ? (float)(1.0 / b) : 0.f;
  const long n2 = a.n / 2, off2 = (long)rhs * a.n / 2;
  float4* t4 = reinterpret_cast<float4*>(a.w);
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += (long)gridDim.x * blockDim.x) {
    float4 v = t4[off2 + i];
    t4[off2 + i] = make_float4(v.x * inv, v.y * inv, v.z * inv, v.w * inv);
  }
}

__global__ void k_ginit(GState* gs, const KScal* sc, int nrhs, int m, double tol2, int maxit) {
  pdl_enter();
  const int r = threadIdx.x;
  if (r >= nrhs) return;
  GState& G = gs[r];
  G.m = m; G.tol2 = tol2; G.maxit = maxit; G.iters = 0; G.status = PSFD_NOT_CONVERGED;
  G.bnorm2 = sc[r].bnorm2; G.jd = 0; G.active = 0;
}

// start of a cycle: beta = ||r|| (from res1 of the scalar block); skip[r] = 1 for
// right-hand sides that are finished
__global__ void k_gstart(GState* gs, KScal* sc, int* skip, int* done, int nrhs) {
  pdl_enter();
  const int r = threadIdx.x;
  if (r >= nrhs) return;
  GState& G = gs[r];
  G.jd = 0;
  if (done[r]) { skip[r] = 1; G.active = 0; return; }
  const double rr = sc[r].res1;
  G.beta = sqrt(rr);
  sc[r].rr = rr;
  if (G.iters == 0) sc[r].rr0 = rr;
  for (int i = 0; i <= G.m; ++i) G.g[i] = make_double2(0.0, 0.0);
  G.g[0] = make_double2(G.beta, 0.0);
  int act = 1;
  if (rr <= G.tol2 * G.bnorm2 || G.bnorm2 == 0.0) { G.status = PSFD_OK; act = 0; done[r] = 1; }
  else if (G.iters >= G.maxit) { G.status = PSFD_NOT_CONVERGED; act = 0; done[r] = 1; }
  else if (!isfinite(rr)) { G.status = PSFD_ERR_BREAKDOWN; act = 0; done[r] = 1; }
  skip[r] = !act;
  G.active = act;
}

// Hessenberg column j: h = h1 + h2 (two CGS passes), H[j+1][j] = ||w||, Givens update
__global__ void k_givens(GState* gs, const double2* h1, const double2* h2, const KScal* sc, int* skip,
                         double* hist, int hist_cap, int nrhs, int j) {
  pdl_enter();
  const int r = threadIdx.x;
  if (r >= nrhs || skip[r]) return;
  GState& G = gs[r];
  const int ld = G.m + 1;
  double2* Hc = G.H + j * ld;
  for (int i = 0; i <= j; ++i) {
    const double2 a = h1[r * GMAX + i], b = h2[r * GMAX + i];
    Hc[i] = make_double2(a.x + b.x, a.y + b.y);
  }
  const double beta = sqrt(sc[r].res0);
  Hc[j + 1] = make_double2(beta, 0.0);
  for (int i = 0; i < j; ++i) {
    const double2 a = Hc[i], b = Hc[i + 1];
    const double2 c = G.cs[i], s = G.sn[i];
    // [conj(c) conj(s); -s c] [a; b]
    Hc[i] = make_double2(c.x * a.x + c.y * a.y + s.x * b.x + s.y * b.y, c.x * a.y - c.y * a.x + s.x * b.y - s.y * b.x);
    Hc[i + 1] = make_double2(-(s.x * a.x - s.y * a.y) + (c.x * b.x - c.y * b.y),
                             -(s.x * a.y + s.y * a.x) + (c.x * b.y + c.y * b.x));
  }
  const double2 a = Hc[j];
  const double den = sqrt(a.x * a.x + a.y * a.y + beta * beta);
  double2 c = make_double2(1.0, 0.0), s = make_double2(0.0, 0.0);
  if (den > 0) { c = make_double2(a.x / den, a.y / den); s = make_double2(beta / den, 0.0); }
  G.cs[j] = c; G.sn[j] = s;
  Hc[j] = make_double2(den, 0.0);
  const double2 gj = G.g[j];
  G.g[j + 1] = make_double2(-(s.x * gj.x - s.y * gj.y), -(s.x * gj.y + s.y * gj.x));
  G.g[j] = make_double2(c.x * gj.x + c.y * gj.y, c.x * gj.y - c.y * gj.x);
  G.iters += 1;
  G.jd = j + 1;
  const double res2 = G.g[j + 1].x * G.g[j + 1].x + G.g[j + 1].y * G.g[j + 1].y;
  if (hist && G.iters - 1 < hist_cap) hist[(long)r * hist_cap + G.iters - 1] = sqrt(res2 / G.bnorm2);
  if (res2 <= G.tol2 * G.bnorm2 || beta == 0.0 || G.iters >= G.maxit || !isfinite(res2) || j + 1 == G.m) {
    skip[r] = 1;
    G.active = 0;
  }
}

// z = H^-1 g on the leading jd x jd triangle (FP64 back substitution)
__global__ void k_gtri(GState* gs, int nrhs) {
  pdl_enter();
  const int r = threadIdx.x;
  if (r >= nrhs) return;
  GState& G = gs[r];
  const int ld = G.m + 1, n = G.jd;
  for (int i = n - 1; i >= 0; --i) {
    double2 acc = G.g[i];
    for (int k = i + 1; k < n; ++k) {
      const double2 h = G.H[i + k * ld], zk = G.z[k];
      acc.x -= h.x * zk.x - h.y * zk.y;
      acc.y -= h.x * zk.y + h.y * zk.x;
    }
    const double2 d = G.H[i + i * ld];
    const double dd = d.x * d.x + d.y * d.y;
    G.z[i] = dd > 0 ? make_double2((acc.x * d.x + acc.y * d.y) / dd, (acc.y * d.x - acc.x * d.y) / dd)
                    : make_double2(0.0, 0.0);
  }
}

__global__ void k_gfinish(GState* gs, KScal* sc, int nrhs) {
  pdl_enter();
  const int r = threadIdx.x;
  if (r >= nrhs) return;
  sc[r].iters = gs[r].iters;
  sc[r].status = gs[r].status;
}

}  // namespace

struct SolveWs {
  cf *bH, *r, *rhat, *p, *v, *s, *t, *y, *Eb;
  cf* V;            // GMRES basis (m + 1 vectors)
  KScal* sc;
  int* done;
  int* active;
  int* skip2;
  double* partials;
  unsigned* counters;
  GState* gs;
  double2* h1;
  double2* h2;
};

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static int nblocks_for(long n) {
  long per = (n / 2 + kThreads - 1) / kThreads;
  long nb = per < 4 * 148 ? per : 4 * 148;
  return (int)(nb < 1 ? 1 : nb);
}

static size_t ws_layout(psfd_plan_s* P, int method, int restart, SolveWs* w, char* base) {
  const size_t vb = align256((size_t)P->nrhs * P->nvec * sizeof(cf));
  const int nb = nblocks_for(P->nvec);
  const int nr = P->nrhs;
  const int nch = (GMAX + GCH - 1) / GCH;
  size_t off = 0;
  auto take = [&](size_t bytes) -> char* { char* q = base ? base + off : nullptr; off += align256(bytes); return q; };
  const bool gm = method == PSFD_GMRES;
  cf** common[] = {&w->bH, &w->r, &w->v, &w->t, &w->y, &w->Eb};
  for (cf** q : common) *q = (cf*)take(vb);
  if (gm) {
    w->rhat = w->p = w->s = nullptr;
    w->V = (cf*)take(vb * (size_t)(restart + 1));
  } else {
    cf** bic[] = {&w->rhat, &w->p, &w->s};
    for (cf** q : bic) *q = (cf*)take(vb);
    w->V = nullptr;
  }
  w->sc = (KScal*)take(sizeof(KScal) * nr);
  w->done = (int*)take(sizeof(int) * nr);
  w->active = (int*)take(sizeof(int) * nr);
  w->skip2 = (int*)take(sizeof(int) * nr);
  w->partials = (double*)take(sizeof(double) * (size_t)nr * nb * (gm ? nch * (2 * GCH + 2) : kMaxQ));
  w->counters = (unsigned*)take(sizeof(unsigned) * nr * (gm ? nch : 1));
  w->gs = gm ? (GState*)take(sizeof(GState) * nr) : nullptr;
  w->h1 = gm ? (double2*)take(sizeof(double2) * nr * GMAX) : nullptr;
  w->h2 = gm ? (double2*)take(sizeof(double2) * nr * GMAX) : nullptr;
  return off;
}

extern "C" size_t psfd_solve_workspace_size(psfd_plan P, int method, int restart) {
  if (!P) return 0;
  SolveWs w;
  return ws_layout(P, method, restart, &w, nullptr);
}

// Pinned, device-mapped progress words of the plan (allocated on first use); nullptr when the
// allocation fails, and the loop then checks convergence by synchronising every 8 iterations.
static int* plan_progress(psfd_plan_s* P) {
  if (!P->prog_h) {
    int* h = nullptr;
    if (cudaHostAlloc((void**)&h, sizeof(int) * 2 * P->nrhs, cudaHostAllocMapped) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    int* d = nullptr;
    if (cudaHostGetDevicePointer((void**)&d, h, 0) != cudaSuccess) {
      cudaGetLastError();
      cudaFreeHost(h);
      return nullptr;
    }
    P->prog_h = h;
    P->prog_d = d;
  }
  return P->prog_d;
}

static int bicgstab_loop(psfd_plan_s* P, SolveWs& w, VArgs va, int maxit, int aflags, int nb) {
  const int nr = P->nrhs;
  cudaStream_t st = P->stream;
  int rc;
  // The host enqueues one iteration at a time and, before the next, waits (without a stream
  // synchronisation) until the one before has completed on every rhs that is still running, as
  // the vector kernels post it to host-mapped memory: the GPU always has the next iteration queued,
  // and at most one iteration of early-returning launches follows convergence.
  va.prog = plan_progress(P);
  volatile int* prog = P->prog_h;
  if (va.prog)
    for (int r = 0; r < 2 * nr; ++r) prog[r] = 0;
  va.v0 = w.r; va.v1 = w.rhat; va.v2 = w.p; va.v3 = w.v; va.v4 = w.y;
  if ((rc = launch_vec<OK_INIT>(va, nr, st, nb))) return rc;
  va.use_done = true;
  std::vector<int> hdone(nr);
  const int check_every = 8;
  for (int it = 0; it < maxit; ++it) {
    va.v0 = w.p; va.v1 = w.r; va.v2 = w.v;
    if ((rc = launch_vec<OK_P>(va, nr, st, nb))) return rc;
    if ((rc = apply_hybrid(P, w.p, w.v, aflags, w.done))) return rc;
    va.v0 = w.rhat; va.v1 = w.v;
    if ((rc = launch_vec<OK_RV>(va, nr, st, nb))) return rc;
    va.v0 = w.s; va.v1 = w.r; va.v2 = w.v;
    if ((rc = launch_vec<OK_S>(va, nr, st, nb))) return rc;
    if ((rc = apply_hybrid(P, w.s, w.t, aflags, w.done))) return rc;
    va.v0 = w.t; va.v1 = w.s;
    if ((rc = launch_vec<OK_TS>(va, nr, st, nb))) return rc;
    va.v0 = w.y; va.v1 = w.r; va.v2 = w.p; va.v3 = w.s; va.v4 = w.t; va.v5 = w.rhat;
    if ((rc = launch_vec<OK_XR>(va, nr, st, nb))) return rc;
    if (va.prog) {
      // iteration it - 1 complete (it iterations) on every running rhs, or every rhs done
      auto state = [&](bool& all_done) {
        all_done = true;
        bool ready = true;
        for (int r = 0; r < nr; ++r) {
          if (prog[nr + r]) continue;
          all_done = false;
          ready = ready && prog[r] >= it;
        }
        return ready || all_done;
      };
      bool all_done = false;
      const auto t0 = std::chrono::steady_clock::now();
      while (!state(all_done)) {
        if (std::chrono::steady_clock::now() - t0 > std::chrono::seconds(2)) {
          // a long iteration: wait for the queue instead of spinning
          PSFD_CUDA_TRY(cudaStreamSynchronize(st));
          state(all_done);
          break;
        }
        std::this_thread::yield();
      }
      if (all_done) break;
    } else if ((it + 1) % check_every == 0 || it + 1 == maxit) {
      PSFD_CUDA_TRY(cudaMemcpyAsync(hdone.data(), w.done, sizeof(int) * nr, cudaMemcpyDeviceToHost, st));
      PSFD_CUDA_TRY(cudaStreamSynchronize(st));
      bool all = true;
      for (int r = 0; r < nr; ++r) all = all && hdone[r];
      if (all) break;
    }
  }
  return PSFD_OK;
}

static int gmres_loop(psfd_plan_s* P, SolveWs& w, VArgs va, double tol, int maxit, int m, int aflags, int nb) {
  // the multi-dot and update kernels stream (j + 2) vectors per launch, one wave of CTAs each
  const int nr = P->nrhs;
  const int nbu = one_wave<k_gupd<false>>(nb, nr), nby = one_wave<k_gupd<true>>(nb, nr);
  cudaStream_t st = P->stream;
  const long n = P->nvec;
  const size_t vbytes = (size_t)nr * n * sizeof(cf);
  const long vs = (long)(align256(vbytes) / sizeof(cf));
  const int nch_max = (GMAX + GCH - 1) / GCH;
  int rc;
  const unsigned tpb = 32 * ((nr + 31) / 32);
  PSFD_CUDA_TRY(cudaMemsetAsync(w.done, 0, sizeof(int) * nr, st));
  PSFD_CUDA_TRY(cudaMemsetAsync(w.y, 0, vbytes, st));
  PSFD_CUDA_TRY(cudaMemsetAsync(w.counters, 0, sizeof(unsigned) * nr * nch_max, st));
  (void)launch_pdl(k_ginit, dim3(1), dim3(tpb), 0, st, w.gs, w.sc, nr, m, tol * tol, maxit);
  PSFD_CHECK_LAUNCH();
  GArgs g{};
  g.V = w.V; g.vs = vs; g.n = n; g.gs = w.gs; g.partials = w.partials; g.counters = w.counters; g.y = w.y;
  g.sc = w.sc; g.save_norm = false;
  std::vector<int> hv(nr);
  bool first = true;
  for (int cycle = 0;; ++cycle) {
    // restart residual r = c - B y (c kept in w.r), written into V_0 with ||r||^2 -> res1
    va.use_done = false;
    if (first) {
      va.v0 = w.r;
      va.v1 = w.t;  // t = 0
      PSFD_CUDA_TRY(cudaMemsetAsync(w.t, 0, vbytes, st));
    } else {
      if ((rc = apply_hybrid(P, w.y, w.t, aflags, w.done))) return rc;
      va.v0 = w.r; va.v1 = w.t;
    }
    va.v2 = w.V;
    if ((rc = launch_vec<OK_SUB>(va, nr, st, nb))) return rc;
    first = false;
    (void)launch_pdl(k_gstart, dim3(1), dim3(tpb), 0, st, w.gs, w.sc, w.active, w.done, nr);
    PSFD_CHECK_LAUNCH();
    PSFD_CUDA_TRY(cudaMemcpyAsync(hv.data(), w.active, sizeof(int) * nr, cudaMemcpyDeviceToHost, st));
    PSFD_CUDA_TRY(cudaStreamSynchronize(st));
    bool any = false;
    for (int r = 0; r < nr; ++r) any = any || !hv[r];
    if (!any) break;
    g.mask = w.active; g.w = w.V; g.j = 0;
    (void)launch_pdl(k_gscale, dim3(nb, nr), dim3(kThreads), 0, st, g, true);
    PSFD_CHECK_LAUNCH();
    for (int j = 0; j < m; ++j) {
      cf* Vj = w.V + (long)j * vs;
      cf* Wn = w.V + (long)(j + 1) * vs;
      if ((rc = apply_hybrid(P, Vj, Wn, aflags, w.active))) return rc;
      g.w = Wn; g.nv = j + 1; g.j = j;
      const int nch = (j + 1 + GCH - 1) / GCH;
      (void)launch_pdl(k_gsave, dim3(nr), dim3(64), 0, st, w.h2, nr, j + 1);
      PSFD_CHECK_LAUNCH();
      {
        // dot (+ ||w||^2 before): read w + (j+1) basis vectors; update (+ ||w||^2 after):
        // read (j+1) + read/write w
        StageScope sc(st, ST_KRYLOV, (2.0 * (j + 1) + 3.0) * nr * n * sizeof(cf));
        g.hout = w.h1;
        g.save_norm = true;
        (void)launch_pdl(k_gdot, dim3(one_wave<k_gdot>(nb, nr * nch), nr, nch), dim3(kThreads), 0, st, g);
        PSFD_CHECK_LAUNCH();
        g.save_norm = false;
        (void)launch_pdl(k_gupd<false>, dim3(nbu, nr), dim3(kThreads), 0, st, g);
        PSFD_CHECK_LAUNCH();
      }
      (void)launch_pdl(k_greorth, dim3(1), dim3(tpb), 0, st, w.sc, w.active, w.skip2, nr);
      PSFD_CHECK_LAUNCH();
      {
        StageScope sc(st, ST_KRYLOV, 0.0);   // second pass: data-dependent, not counted as algorithmic
        const int* keep = g.mask;
        g.mask = w.skip2;
        g.hout = w.h2;
        (void)launch_pdl(k_gdot, dim3(one_wave<k_gdot>(nb, nr * nch), nr, nch), dim3(kThreads), 0, st, g);
        PSFD_CHECK_LAUNCH();
        (void)launch_pdl(k_gupd<false>, dim3(nbu, nr), dim3(kThreads), 0, st, g);
        PSFD_CHECK_LAUNCH();
        g.mask = keep;
      }
      (void)launch_pdl(k_givens, dim3(1), dim3(tpb), 0, st, w.gs, w.h1, w.h2, w.sc, w.active, va.hist, va.hist_cap, nr, j);
      PSFD_CHECK_LAUNCH();
      (void)launch_pdl(k_gscale, dim3(nb, nr), dim3(kThreads), 0, st, g, false);
      PSFD_CHECK_LAUNCH();
      if ((j & 3) == 3 || j == m - 1) {
        PSFD_CUDA_TRY(cudaMemcpyAsync(hv.data(), w.active, sizeof(int) * nr, cudaMemcpyDeviceToHost, st));
        PSFD_CUDA_TRY(cudaStreamSynchronize(st));
        bool a = false;
        for (int r = 0; r < nr; ++r) a = a || !hv[r];
        if (!a) break;
      }
    }
    // y += V z for every rhs that ran this cycle
    (void)launch_pdl(k_gtri, dim3(1), dim3(tpb), 0, st, w.gs, nr);
    PSFD_CHECK_LAUNCH();
    g.mask = nullptr;  // every rhs with jd > 0 updates y
    (void)launch_pdl(k_gupd<true>, dim3(nby, nr), dim3(kThreads), 0, st, g);
    PSFD_CHECK_LAUNCH();
  }
  (void)launch_pdl(k_gfinish, dim3(1), dim3(tpb), 0, st, w.gs, w.sc, nr);
  PSFD_CHECK_LAUNCH();
  return PSFD_OK;
}

extern "C" int psfd_solve(psfd_plan P, const psfd_c64* b, const psfd_c64* x0, psfd_c64* E, double tol, int maxit,
                          int method, int restart, int use_precond, psfd_info_t* info, void* workspace,
                          size_t workspace_bytes) {
  if (!P || !b || !E || !info) { psfd_set_error("psfd_solve: null argument"); return PSFD_ERR_ARG; }
  if (!P->have_background) { psfd_set_error("psfd_solve: call psfd_background first"); return PSFD_ERR_STATE; }
  if (!(tol > 0) || maxit < 0) { psfd_set_error("psfd_solve: bad tol / maxit"); return PSFD_ERR_ARG; }
  if (method != PSFD_BICGSTAB && method != PSFD_GMRES) { psfd_set_error("psfd_solve: unknown method"); return PSFD_ERR_ARG; }
  if (method == PSFD_GMRES && (restart < 1 || restart > GMAX)) {
    psfd_set_error("psfd_solve: GMRES restart must be in [1, %d]", GMAX);
    return PSFD_ERR_ARG;
  }
  if (use_precond < 0 || use_precond > 2) { psfd_set_error("psfd_solve: use_precond must be 0, 1 or 2"); return PSFD_ERR_ARG; }
  if (use_precond == 2 && !P->lay_built) { psfd_set_error("psfd_solve: call psfd_layered_build first"); return PSFD_ERR_STATE; }
  cudaStream_t st = P->stream;
  SolveWs w;
  const size_t need = ws_layout(P, method, restart, &w, nullptr);
  char* base = (char*)workspace;
  bool own = false;
  if (!base) {
    PSFD_CUDA_TRY(cudaMallocAsync((void**)&base, need, st));
    own = true;
  } else if (workspace_bytes < need) {
    psfd_set_error("psfd_solve: workspace too small (%zu < %zu)", workspace_bytes, need);
    return PSFD_ERR_ARG;
  }
  ws_layout(P, method, restart, &w, base);
  const int nr = P->nrhs;
  const long n = P->nvec;
  const size_t vbytes = (size_t)nr * n * sizeof(cf);
  const int nb = nblocks_for(n);
  const float us = 1.0f / sqrtf((float)P->ncols);
  const long nplanes = (long)nr * 3 * P->nz;
  const unsigned tpb = 32 * ((nr + 31) / 32);
  int rc = PSFD_OK;
  double* dhist = nullptr;
  auto fail = [&](int code) {
    if (own) cudaFreeAsync(base, st);
    if (dhist) cudaFreeAsync(dhist, st);
    return code;
  };

  PSFD_CUDA_TRY(cudaMemsetAsync(w.counters, 0, sizeof(unsigned) * nr, st));
  (void)launch_pdl(k_set_scalars, dim3(1), dim3(tpb), 0, st, w.sc, nr, tol * tol, maxit);
  PSFD_CHECK_LAUNCH();
  VArgs va{};
  va.n = n; va.sc = w.sc; va.done = w.done; va.partials = w.partials; va.counters = w.counters;
  va.hist = nullptr; va.hist_cap = 0; va.use_done = false;
  if (P->hist && P->hist_cap > 0) {
    PSFD_CUDA_TRY(cudaMallocAsync((void**)&dhist, sizeof(double) * nr * P->hist_cap, st));
    PSFD_CUDA_TRY(cudaMemsetAsync(dhist, 0, sizeof(double) * nr * P->hist_cap, st));
    va.hist = dhist; va.hist_cap = P->hist_cap;
  }
  // b -> HYBRID, ||b||^2
  PSFD_CUDA_TRY(cudaMemcpyAsync(w.bH, b, vbytes, cudaMemcpyDeviceToDevice, st));
  if ((rc = launch_lateral_transform(P, w.bH, nplanes, true, us))) return fail(rc);
  va.v0 = w.bH;
  if ((rc = launch_vec<OK_NORM>(va, nr, st, nb))) return fail(rc);
  (void)launch_pdl(k_copy_bnorm, dim3(1), dim3(tpb), 0, st, w.sc, nr);
  PSFD_CHECK_LAUNCH();
  // c = b - A E_base (the right-hand side of A M y = c)
  if (x0) {
    PSFD_CUDA_TRY(cudaMemcpyAsync(w.Eb, x0, vbytes, cudaMemcpyDeviceToDevice, st));
    if ((rc = launch_lateral_transform(P, w.Eb, nplanes, true, us))) return fail(rc);
    if ((rc = apply_hybrid(P, w.Eb, w.v, 0, nullptr))) return fail(rc);
    va.v0 = w.bH; va.v1 = w.v; va.v2 = w.r;
    if ((rc = launch_vec<OK_SUB>(va, nr, st, nb))) return fail(rc);
  } else {
    PSFD_CUDA_TRY(cudaMemcpyAsync(w.r, w.bH, vbytes, cudaMemcpyDeviceToDevice, st));
  }
  const int aflags = use_precond == 2 ? PSFD_LAYERED : (use_precond ? PSFD_PRECOND : 0);
  if (method == PSFD_BICGSTAB) rc = bicgstab_loop(P, w, va, maxit, aflags, nb);
  else rc = gmres_loop(P, w, va, tol, maxit, restart, aflags, nb);
  if (rc) return fail(rc);
  // ---- E = E_base + M y ; true residual (FP64 norm)
  va.use_done = false;
  cf* My = w.t;
  if (use_precond == 2) {
    if ((rc = layered_apply(P, w.y, My))) return fail(rc);
  } else if (use_precond) {
    if ((rc = launch_axial(P, w.y, My, 2, nullptr, nr))) return fail(rc);
  } else {
    PSFD_CUDA_TRY(cudaMemcpyAsync(My, w.y, vbytes, cudaMemcpyDeviceToDevice, st));
  }
  cf* EH = w.r;
  if (x0) {
    va.v0 = w.Eb; va.v1 = My; va.v2 = EH;
    if ((rc = launch_vec<OK_AXPY>(va, nr, st, nb))) return fail(rc);
  } else {
    PSFD_CUDA_TRY(cudaMemcpyAsync(EH, My, vbytes, cudaMemcpyDeviceToDevice, st));
  }
  if ((rc = apply_hybrid(P, EH, w.v, 0, nullptr))) return fail(rc);
  va.v0 = w.bH; va.v1 = w.v; va.v2 = w.t;
  if ((rc = launch_vec<OK_SUB>(va, nr, st, nb))) return fail(rc);
  PSFD_CUDA_TRY(cudaMemcpyAsync(E, EH, vbytes, cudaMemcpyDeviceToDevice, st));
  if ((rc = launch_lateral_transform(P, (cf*)E, nplanes, false, us))) return fail(rc);
  std::vector<KScal> hs(nr);
  PSFD_CUDA_TRY(cudaMemcpyAsync(hs.data(), w.sc, sizeof(KScal) * nr, cudaMemcpyDeviceToHost, st));
  if (dhist) {
    PSFD_CUDA_TRY(cudaMemcpyAsync(P->hist, dhist, sizeof(double) * nr * P->hist_cap, cudaMemcpyDeviceToHost, st));
  }
  PSFD_CUDA_TRY(cudaStreamSynchronize(st));
  if (dhist) { cudaFree(dhist); dhist = nullptr; }
  int worst = PSFD_OK;
  for (int r = 0; r < nr; ++r) {
    const double bn = hs[r].bnorm2;
    info[r].iters = hs[r].iters;
    info[r].status = (bn == 0.0) ? PSFD_OK : hs[r].status;
    info[r].r_rel = bn > 0 ? sqrt(hs[r].res1 / bn) : 0.0;
    info[r].r_rel_recursive = bn > 0 ? sqrt(hs[r].rr / bn) : 0.0;
    info[r].r_rel_initial = bn > 0 ? sqrt(hs[r].rr0 / bn) : 0.0;
    info[r].outer = 0;
    info[r].r_rel_output = info[r].r_rel;
    if (info[r].status != PSFD_OK && worst == PSFD_OK) worst = info[r].status;
  }
  if (own) PSFD_CUDA_TRY(cudaFreeAsync(base, st));
  if ((rc = plan_wait_status(P))) return rc;
  return worst;
}

// ======================================================================= mixed-precision refinement
// Outer loop in FP64:  r = b - A E (FP64 operator apply, FP64 field E),
// inner complex64 Krylov solve of A M d = r to a relative tolerance, E += M d.
namespace {

enum { V64_PROMOTE = 0, V64_RES = 1, V64_CAST = 2, V64_ADD = 3, V64_NORM = 4 };

struct V64Args {
  const zd* a64;
  zd* o64;
  const cf* a32;
  cf* o32;
  const zd* b64;
  long n;
  KScal* sc;
  const int* skip;   // V64_CAST: write zero for rhs with skip != 0
  double* partials;
  unsigned* counters;
};

template <int OP>
__global__ void __launch_bounds__(kThreads) k_v64(V64Args a) {
  pdl_enter();
  const int rhs = blockIdx.y;
  const long off = (long)rhs * a.n;
  const long stride = (long)gridDim.x * blockDim.x;
  double acc = 0.0;
  const bool zero = (OP == V64_CAST) && a.skip && a.skip[rhs];
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
    const long e = off + i;
    if constexpr (OP == V64_PROMOTE) {
      const cf x = a.a32[e];
      a.o64[e] = make_double2((double)x.x, (double)x.y);
    } else if constexpr (OP == V64_RES) {
      const zd b = a.b64[e], v = a.a64[e];
      const zd r = make_double2(b.x - v.x, b.y - v.y);
      a.o64[e] = r;
      acc = fma(r.x, r.x, fma(r.y, r.y, acc));
    } else if constexpr (OP == V64_CAST) {
      const zd x = a.a64[e];
      a.o32[e] = zero ? czero() : make_float2((float)x.x, (float)x.y);
    } else if constexpr (OP == V64_ADD) {
      const cf d = a.a32[e];
      zd x = a.o64[e];
      x.x += (double)d.x;
      x.y += (double)d.y;
      a.o64[e] = x;
    } else {
      const zd x = a.a64[e];
      acc = fma(x.x, x.x, fma(x.y, x.y, acc));
    }
  }
  if constexpr (OP == V64_RES || OP == V64_NORM) {
    double val[2] = {acc, 0.0};
    double tot[2];
    if (!reduce_finish<2>(val, a.partials, a.counters, tot)) return;
    if (threadIdx.x == 0) {
      if (OP == V64_RES) a.sc[rhs].res1 = tot[0];
      else a.sc[rhs].res0 = tot[0];
    }
  }
}

template <int OP>
int launch_v64(const V64Args& a, int nrhs, cudaStream_t s, int nb) {
  StageScope sc(s, ST_KRYLOV);
  (void)launch_pdl(k_v64<OP>, dim3(nb, nrhs), dim3(kThreads), 0, s, a);
  PSFD_CHECK_LAUNCH();
  return PSFD_OK;
}

}  // namespace

static size_t refine_extra_bytes(psfd_plan_s* P) {
  return 3 * align256((size_t)P->nrhs * P->nvec * sizeof(zd));
}

extern "C" size_t psfd_solve_ex_workspace_size(psfd_plan P, const psfd_solve_opts_t* o) {
  if (!P || !o) return 0;
  SolveWs w;
  size_t base = ws_layout(P, o->method, o->restart, &w, nullptr);
  return base + (o->refine ? refine_extra_bytes(P) : 0);
}

extern "C" int psfd_solve_ex(psfd_plan P, const psfd_c64* b, const psfd_c64* x0, psfd_c64* E,
                             const psfd_solve_opts_t* o, psfd_info_t* info, void* workspace,
                             size_t workspace_bytes) {
  if (!P || !b || !E || !info || !o) { psfd_set_error("psfd_solve_ex: null argument"); return PSFD_ERR_ARG; }
  if (o->out_c128 && !o->refine) {
    psfd_set_error("psfd_solve_ex: out_c128 needs refine = 1 (the FP64 field)");
    return PSFD_ERR_ARG;
  }
  if (!o->refine) {
    int rc = psfd_solve(P, b, x0, E, o->tol, o->maxit, o->method, o->restart, o->use_precond, info, workspace,
                        workspace_bytes);
    for (int r = 0; r < P->nrhs; ++r) { info[r].outer = 0; info[r].r_rel_output = info[r].r_rel; }
    return rc;
  }
  if (!P->have_background) { psfd_set_error("psfd_solve_ex: call psfd_background first"); return PSFD_ERR_STATE; }
  if (!(o->tol > 0) || o->maxit < 0 || !(o->inner_tol > 0 && o->inner_tol < 1)) {
    psfd_set_error("psfd_solve_ex: bad tol / inner_tol / maxit");
    return PSFD_ERR_ARG;
  }
  if (o->method != PSFD_BICGSTAB && o->method != PSFD_GMRES) { psfd_set_error("psfd_solve_ex: unknown method"); return PSFD_ERR_ARG; }
  if (o->method == PSFD_GMRES && (o->restart < 1 || o->restart > GMAX)) {
    psfd_set_error("psfd_solve_ex: GMRES restart must be in [1, %d]", GMAX);
    return PSFD_ERR_ARG;
  }
  if (o->use_precond < 0 || o->use_precond > 2) {
    psfd_set_error("psfd_solve_ex: use_precond must be 0, 1 or 2");
    return PSFD_ERR_ARG;
  }
  if (o->use_precond == 2 && !P->lay_built) {
    psfd_set_error("psfd_solve_ex: call psfd_layered_build first");
    return PSFD_ERR_STATE;
  }
  int rc = fp64_prepare(P);
  if (rc) return rc;
  cudaStream_t st = P->stream;
  SolveWs w;
  const size_t base_need = ws_layout(P, o->method, o->restart, &w, nullptr);
  const size_t need = base_need + refine_extra_bytes(P);
  char* base = (char*)workspace;
  bool own = false;
  if (!base) {
    PSFD_CUDA_TRY(cudaMallocAsync((void**)&base, need, st));
    own = true;
  } else if (workspace_bytes < need) {
    psfd_set_error("psfd_solve_ex: workspace too small (%zu < %zu)", workspace_bytes, need);
    return PSFD_ERR_ARG;
  }
  ws_layout(P, o->method, o->restart, &w, base);
  const size_t v64b = align256((size_t)P->nrhs * P->nvec * sizeof(zd));
  zd* b64 = (zd*)(base + base_need);
  zd* E64 = (zd*)(base + base_need + v64b);
  zd* r64 = (zd*)(base + base_need + 2 * v64b);
  const int nr = P->nrhs;
  const long n = P->nvec;
  const size_t vbytes = (size_t)nr * n * sizeof(cf);
  const int nb = nblocks_for(n);
  const long nplanes = (long)nr * 3 * P->nz;
  const double us = 1.0 / sqrt((double)P->ncols);
  const unsigned tpb = 32 * ((nr + 31) / 32);
  auto fail = [&](int code) { if (own) cudaFreeAsync(base, st); return code; };

  const int nch_max = (GMAX + GCH - 1) / GCH;
  PSFD_CUDA_TRY(cudaMemsetAsync(w.counters, 0, sizeof(unsigned) * nr * (o->method == PSFD_GMRES ? nch_max : 1), st));
  (void)launch_pdl(k_set_scalars, dim3(1), dim3(tpb), 0, st, w.sc, nr, 0.0, 0);
  PSFD_CHECK_LAUNCH();
  V64Args a64{};
  a64.n = n; a64.sc = w.sc; a64.partials = w.partials; a64.counters = w.counters;
  // b (complex64, real space) -> FP64 HYBRID
  a64.a32 = (const cf*)b; a64.o64 = b64;
  if ((rc = launch_v64<V64_PROMOTE>(a64, nr, st, nb))) return fail(rc);
  // b usually vanishes outside the absorber planes (it carries the factor delta-eps): the zero
  // planes, flagged from b itself, are left out of its lateral transform
  if ((rc = plane_flags(P, (const cf*)b, nplanes, P->F.plane_nz))) return fail(rc);
  if ((rc = transform64(P, b64, nplanes, true, us, P->F.plane_nz))) return fail(rc);
  a64.a64 = b64;
  if ((rc = launch_v64<V64_NORM>(a64, nr, st, nb))) return fail(rc);
  // ||b||^2 stays in res0 until the first inner solve: it is read with the first residual
  std::vector<KScal> hs(nr);
  std::vector<double> bnorm2(nr), rr(nr, 0.0), rr0(nr, 0.0);
  // E64 = x0 (HYBRID, FP64) or 0.  The warm start only sets where the refinement begins, so its
  // lateral transform runs in complex64 (kept in w.t, where the first residual reads it)
  if (x0) {
    PSFD_CUDA_TRY(cudaMemcpyAsync(w.t, x0, vbytes, cudaMemcpyDeviceToDevice, st));
    if ((rc = launch_lateral_transform(P, w.t, nplanes, true, (float)us))) return fail(rc);
    a64.a32 = w.t; a64.o64 = E64;
    if ((rc = launch_v64<V64_PROMOTE>(a64, nr, st, nb))) return fail(rc);
  } else {
    PSFD_CUDA_TRY(cudaMemsetAsync(E64, 0, (size_t)nr * n * sizeof(zd), st));
  }
  std::vector<int> conv(nr, 0), status(nr, PSFD_NOT_CONVERGED), inner_its(nr, 0);
  int* dskip = w.active;  // reused as the per-rhs "outer converged" flag
  int outer = 0;
  const int max_outer = o->max_outer > 0 ? o->max_outer : 100;
  const int aflags = o->use_precond == 2 ? PSFD_LAYERED : (o->use_precond ? PSFD_PRECOND : 0);
  VArgs va{};
  va.n = n; va.sc = w.sc; va.done = w.done; va.partials = w.partials; va.counters = w.counters;
  for (;; ++outer) {
    // r = b - A E with the extended-precision apply.  The first residual only feeds an inner solve
    // to inner_tol, so a cold start takes r = b (E = 0) and a warm start forms A E with the
    // complex64 operator; convergence is only ever decided on an extended-precision residual.
    bool exact = !(outer == 0 && x0);
    if (outer == 0 && !x0) {
      PSFD_CUDA_TRY(cudaMemsetAsync(r64, 0, (size_t)nr * n * sizeof(zd), st));
    } else if (outer == 0) {
      if ((rc = apply_hybrid(P, w.t, w.v, 0, nullptr))) return fail(rc);   // w.t = complex64 E (above)
      a64.a32 = w.v; a64.o64 = r64;
      if ((rc = launch_v64<V64_PROMOTE>(a64, nr, st, nb))) return fail(rc);
    } else {
      if ((rc = apply64_hybrid(P, E64, r64))) return fail(rc);
    }
    a64.b64 = b64; a64.a64 = r64; a64.o64 = r64;
    if ((rc = launch_v64<V64_RES>(a64, nr, st, nb))) return fail(rc);
    PSFD_CUDA_TRY(cudaMemcpyAsync(hs.data(), w.sc, sizeof(KScal) * nr, cudaMemcpyDeviceToHost, st));
    PSFD_CUDA_TRY(cudaStreamSynchronize(st));
    if (outer == 0) {
      for (int r = 0; r < nr; ++r) bnorm2[r] = hs[r].res0;
    } else {
      // the last inner solve's iteration counts are still in the scalar block
      for (int r = 0; r < nr; ++r)
        if (!conv[r]) inner_its[r] += hs[r].iters;
    }
    if (!exact) {
      // a warm start that may already meet the tolerance is decided on the exact residual
      bool near = false;
      for (int r = 0; r < nr; ++r) near = near || hs[r].res1 <= 4.0 * o->tol * o->tol * bnorm2[r];
      if (near) {
        if ((rc = apply64_hybrid(P, E64, r64))) return fail(rc);
        a64.b64 = b64; a64.a64 = r64; a64.o64 = r64;
        if ((rc = launch_v64<V64_RES>(a64, nr, st, nb))) return fail(rc);
        PSFD_CUDA_TRY(cudaMemcpyAsync(hs.data(), w.sc, sizeof(KScal) * nr, cudaMemcpyDeviceToHost, st));
        PSFD_CUDA_TRY(cudaStreamSynchronize(st));
        exact = true;
      }
    }
    bool all = true;
    int total_max = 0;
    for (int r = 0; r < nr; ++r) {
      rr[r] = hs[r].res1;
      if (outer == 0) rr0[r] = rr[r];
      if (bnorm2[r] == 0.0 || (exact && rr[r] <= o->tol * o->tol * bnorm2[r])) { conv[r] = 1; status[r] = PSFD_OK; }
      else if (!std::isfinite(rr[r])) { conv[r] = 1; status[r] = PSFD_ERR_BREAKDOWN; }
      else if (inner_its[r] >= o->maxit || outer >= max_outer) { conv[r] = 1; status[r] = PSFD_NOT_CONVERGED; }
      all = all && conv[r];
      total_max = std::max(total_max, inner_its[r]);
    }
    if (all) break;
    if (nr <= RhsBits::kMax) {
      RhsBits bits{};
      for (int r = 0; r < nr; ++r)
        if (conv[r]) bits.w[r >> 6] |= 1ull << (r & 63);
      (void)launch_pdl(k_set_flags, dim3((nr + 255) / 256), dim3(256), 0, st, dskip, nr, bits);
      PSFD_CHECK_LAUNCH();
    } else {
      PSFD_CUDA_TRY(cudaMemcpyAsync(dskip, conv.data(), sizeof(int) * nr, cudaMemcpyHostToDevice, st));
    }
    a64.a64 = r64; a64.o32 = w.r; a64.skip = dskip;
    if ((rc = launch_v64<V64_CAST>(a64, nr, st, nb))) return fail(rc);
    // inner complex64 solve of A M y = r to inner_tol (relative to ||r||), or only as far as the
    // final tolerance needs: 0.5 tol ||b|| / ||r|| when that is looser (strictest over the rhs)
    const int inner_max = std::max(1, o->maxit - total_max);
    double itol = 0.5;
    for (int r = 0; r < nr; ++r)
      if (!conv[r] && rr[r] > 0) itol = std::min(itol, 0.5 * o->tol * sqrt(bnorm2[r] / rr[r]));
    itol = std::max(itol, o->inner_tol);
    (void)launch_pdl(k_set_scalars, dim3(1), dim3(tpb), 0, st, w.sc, nr, itol * itol, inner_max);
    PSFD_CHECK_LAUNCH();
    va.use_done = false;
    va.v0 = w.r;
    if ((rc = launch_vec<OK_NORM>(va, nr, st, nb))) return fail(rc);
    (void)launch_pdl(k_copy_bnorm, dim3(1), dim3(tpb), 0, st, w.sc, nr);
    PSFD_CHECK_LAUNCH();
    if (o->method == PSFD_BICGSTAB) rc = bicgstab_loop(P, w, va, inner_max, aflags, nb);
    else rc = gmres_loop(P, w, va, itol, inner_max, o->restart, aflags, nb);
    if (rc) return fail(rc);
    // E += M y
    cf* My = w.t;
    if (o->use_precond == 2) {
      if ((rc = layered_apply(P, w.y, My))) return fail(rc);
    } else if (o->use_precond) {
      if ((rc = launch_axial(P, w.y, My, 2, nullptr, nr))) return fail(rc);
    } else {
      PSFD_CUDA_TRY(cudaMemcpyAsync(My, w.y, vbytes, cudaMemcpyDeviceToDevice, st));
    }
    a64.a32 = My; a64.o64 = E64;
    if ((rc = launch_v64<V64_ADD>(a64, nr, st, nb))) return fail(rc);
  }
  if (o->out_c128) {
    // output: E = F^-1 E64 in FP64 (complex128); its residual is the last outer residual
    zd* E128 = (zd*)E;
    PSFD_CUDA_TRY(cudaMemcpyAsync(E128, E64, (size_t)nr * n * sizeof(zd), cudaMemcpyDeviceToDevice, st));
    if ((rc = transform64(P, E128, nplanes, false, us))) return fail(rc);
    for (int r = 0; r < nr; ++r) hs[r].res1 = rr[r];
  } else {
    // output: E = complex64(F^-1 E64), transformed in FP64
    PSFD_CUDA_TRY(cudaMemcpyAsync(r64, E64, (size_t)nr * n * sizeof(zd), cudaMemcpyDeviceToDevice, st));
    if ((rc = transform64(P, r64, nplanes, false, us))) return fail(rc);
    a64.a64 = r64; a64.o32 = (cf*)E; a64.skip = nullptr;
    if ((rc = launch_v64<V64_CAST>(a64, nr, st, nb))) return fail(rc);
    // FP64 residual of the returned complex64 field
    a64.a32 = (const cf*)E; a64.o64 = r64;
    if ((rc = launch_v64<V64_PROMOTE>(a64, nr, st, nb))) return fail(rc);
    if ((rc = transform64(P, r64, nplanes, true, us))) return fail(rc);
    if ((rc = apply64_hybrid(P, r64, E64))) return fail(rc);
    a64.b64 = b64; a64.a64 = E64; a64.o64 = E64;
    if ((rc = launch_v64<V64_RES>(a64, nr, st, nb))) return fail(rc);
    PSFD_CUDA_TRY(cudaMemcpyAsync(hs.data(), w.sc, sizeof(KScal) * nr, cudaMemcpyDeviceToHost, st));
  }
  PSFD_CUDA_TRY(cudaStreamSynchronize(st));
  int worst = PSFD_OK;
  for (int r = 0; r < nr; ++r) {
    info[r].iters = inner_its[r];
    info[r].status = status[r];
    info[r].outer = outer;
    info[r].r_rel = bnorm2[r] > 0 ? sqrt(rr[r] / bnorm2[r]) : 0.0;
    info[r].r_rel_recursive = info[r].r_rel;
    info[r].r_rel_initial = bnorm2[r] > 0 ? sqrt(rr0[r] / bnorm2[r]) : 0.0;
    info[r].r_rel_output = bnorm2[r] > 0 ? sqrt(hs[r].res1 / bnorm2[r]) : 0.0;
    if (status[r] != PSFD_OK && worst == PSFD_OK) worst = status[r];
  }
  if (own) PSFD_CUDA_TRY(cudaFreeAsync(base, st));
  if ((rc = plan_wait_status(P))) return rc;
  return worst;
}
