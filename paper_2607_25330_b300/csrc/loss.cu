// Physics-informed loss of Sec. 3 (Eq. loss) and its gradient, in the library.
//
//   J_a = (1/N) ||r_a||^2 + (lambda_hf / N) ||w(nu) F3[r_a]||^2,   r_a = A E_a - b_a,
//   w(nu) = w0 + eta_hf |nu|, nu in cycles per sample, F3 the unitary 3-D DFT,
//   dJ_a/dRe E_a + i dJ_a/dIm E_a = (2/N) A^H [ r_a + lambda_hf F3^H (w^2 F3 r_a) ]
// (the gradient in the convention of torch's complex autograd: for a real J of a complex E it is
// twice the derivative with respect to conj(E)).  A and A^H are the library's operator applies;
// the 3-D DFT is the library's own row and column FFTs (x rows, y columns, z columns of stride
// nx ny); the two sums accumulate in FP64.
#include <cuda_runtime.h>

#include <cmath>

#include "internal.h"

namespace {

constexpr int kLossThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// block sum of v added into *acc (one FP64 atomic per block)
__device__ __forceinline__ void block_add(double v, double* acc) {
  __shared__ double part[kLossThreads / 32];
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) part[warp] = v;
  __syncthreads();
  if (warp == 0) {
    double s = lane < kLossThreads / 32 ? part[lane] : 0.0;
    s = warp_sum(s);
    if (lane == 0) atomicAdd(acc, s);
  }
}

// r <- r - b; acc[rhs] += sum |r|^2 (grid: blocks over one rhs's entries, rhs in blockIdx.y)
__global__ void __launch_bounds__(kLossThreads) k_loss_residual(cf* __restrict__ r, const cf* __restrict__ b,
                                                              long n, double* acc) {
  const long off = (long)blockIdx.y * n;
  double s = 0.0;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    cf v = r[off + i];
    const cf bb = b[off + i];
    v = make_float2(v.x - bb.x, v.y - bb.y);
    r[off + i] = v;
    s += (double)v.x * v.x + (double)v.y * v.y;
  }
  block_add(s, acc + blockIdx.y);
}

// cycles per sample of FFT index i of a length-n transform (Nyquist counted negative)
__device__ __forceinline__ float freq(int i, int n) { return (float)((i <= (n - 1) / 2) ? i : i - n) / (float)n; }

// spectrum U of r (unitary): acc[rhs] += sum w^2 |U|^2 and U <- lambda w^2 U
__global__ void __launch_bounds__(kLossThreads) k_loss_weight(cf* __restrict__ U, int nx, int ny, int nz, long n,
                                                            float w0, float eta, float lam, int scale_u,
                                                            double* acc) {
  const long off = (long)blockIdx.y * n;
  const long plane = (long)nx * ny;
  double s = 0.0;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const long q = i % ((long)nz * plane);           // index within one component
    const int z = (int)(q / plane);
    const long rem = q - (long)z * plane;
    const int y = (int)(rem / nx), x = (int)(rem - (long)y * nx);
    const float fx = freq(x, nx), fy = freq(y, ny), fz = freq(z, nz);
    const float w = w0 + eta * sqrtf(fx * fx + fy * fy + fz * fz);
    const float w2 = w * w;
    cf v = U[off + i];
    s += (double)w2 * ((double)v.x * v.x + (double)v.y * v.y);
    if (scale_u) U[off + i] = make_float2(lam * w2 * v.x, lam * w2 * v.y);
  }
  block_add(s, acc + blockIdx.y);
}

// U <- U + R (the bracket of the gradient)
__global__ void k_loss_add(cf* __restrict__ U, const cf* __restrict__ R, long n) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const cf a = U[i], c = R[i];
    U[i] = make_float2(a.x + c.x, a.y + c.y);
  }
}

// g <- s g
__global__ void k_loss_scale(cf* __restrict__ g, long n, float s) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const cf a = g[i];
    g[i] = make_float2(s * a.x, s * a.y);
  }
}

// unitary 3-D DFT of every component plane stack of every rhs (in place)
int fft3(psfd_plan_s* P, cf* buf, bool forward) {
  const long comps = (long)P->nrhs * 3;
  const float us = (float)(1.0 / sqrt((double)P->nvec / 3.0));
  cudaStream_t s = P->stream;
  int rc;
  if (forward) {
    if ((rc = launch_rows(P->nx, buf, comps * P->nz * P->ny, true, 1.f, P->tw_x, s))) return rc;
    if ((rc = launch_cols(P->ny, P->nx, buf, comps * P->nz * P->nx, true, 1.f, P->tw_y, s))) return rc;
    return launch_cols(P->nz, P->nx * P->ny, buf, comps * P->nx * P->ny, true, us, P->tw_z, s);
  }
  if ((rc = launch_cols(P->nz, P->nx * P->ny, buf, comps * P->nx * P->ny, false, 1.f, P->tw_z, s))) return rc;
  if ((rc = launch_cols(P->ny, P->nx, buf, comps * P->nz * P->nx, false, 1.f, P->tw_y, s))) return rc;
  return launch_rows(P->nx, buf, comps * P->nz * P->ny, false, us, P->tw_x, s);
}

unsigned grid_for(long n) {
  const long b = (n + kLossThreads - 1) / kLossThreads;
  return (unsigned)(b < 4 * 148 ? (b > 0 ? b : 1) : 4 * 148);
}

}  // namespace

extern "C" size_t psfd_physics_loss_workspace_size(psfd_plan P) {
  if (!P) return 0;
  const size_t v = (size_t)P->nrhs * P->nvec * sizeof(cf);
  return 2 * ((v + 255) / 256 * 256) + 256;
}

extern "C" int psfd_physics_loss(psfd_plan P, const psfd_c64* E, const psfd_c64* b, double lam_hf, double w0,
                                 double eta_hf, double* J, psfd_c64* grad, void* workspace,
                                 size_t workspace_bytes) {
  if (!P || !E || !b || !J || !workspace) { psfd_set_error("psfd_physics_loss: null argument"); return PSFD_ERR_ARG; }
  if (!P->have_background) { psfd_set_error("psfd_physics_loss: call psfd_background first"); return PSFD_ERR_STATE; }
  if (workspace_bytes < psfd_physics_loss_workspace_size(P)) {
    psfd_set_error("psfd_physics_loss: workspace of %zu bytes, %zu needed", workspace_bytes,
                   psfd_physics_loss_workspace_size(P));
    return PSFD_ERR_ARG;
  }
  if (!std::isfinite(lam_hf) || !std::isfinite(w0) || !std::isfinite(eta_hf)) {
    psfd_set_error("psfd_physics_loss: non-finite constant");
    return PSFD_ERR_ARG;
  }
  if ((const void*)grad == (const void*)E || (const void*)grad == (const void*)b) {
    psfd_set_error("psfd_physics_loss: grad must not overlap E or b");
    return PSFD_ERR_ARG;
  }
  cudaStream_t s = P->stream;
  const long n = P->nvec;                     // entries per rhs
  const long ntot = (long)P->nrhs * n;
  const size_t vb = (size_t)ntot * sizeof(cf);
  char* ws = (char*)workspace;
  cf* R = (cf*)ws;
  cf* U = (cf*)(ws + (vb + 255) / 256 * 256);
  double* acc = (double*)(ws + 2 * ((vb + 255) / 256 * 256));   // [2][nrhs]
  int rc;
  PSFD_CUDA_TRY(cudaMemsetAsync(acc, 0, 2 * sizeof(double) * P->nrhs, s));
  // r = A E - b and ||r||^2
  if ((rc = psfd_apply(P, E, (psfd_c64*)R, 0))) return rc;
  dim3 g1(grid_for(n), (unsigned)P->nrhs);
  k_loss_residual<<<g1, kLossThreads, 0, s>>>(R, (const cf*)b, n, acc);
  PSFD_CHECK_LAUNCH();
  // F3 r, sum w^2 |F3 r|^2, and lambda w^2 F3 r
  PSFD_CUDA_TRY(cudaMemcpyAsync(U, R, vb, cudaMemcpyDeviceToDevice, s));
  if ((rc = fft3(P, U, true))) return rc;
  k_loss_weight<<<g1, kLossThreads, 0, s>>>(U, P->nx, P->ny, P->nz, n, (float)w0, (float)eta_hf, (float)lam_hf,
                                            grad ? 1 : 0, acc + P->nrhs);
  PSFD_CHECK_LAUNCH();
  if (grad) {
    // (2/N) A^H [ r + F3^H (lambda w^2 F3 r) ]
    if ((rc = fft3(P, U, false))) return rc;
    k_loss_add<<<grid_for(ntot), kLossThreads, 0, s>>>(U, R, ntot);
    PSFD_CHECK_LAUNCH();
    if ((rc = psfd_apply(P, (const psfd_c64*)U, grad, PSFD_ADJOINT))) return rc;
    const double npts = (double)n / 3.0;
    k_loss_scale<<<grid_for(ntot), kLossThreads, 0, s>>>((cf*)grad, ntot, (float)(2.0 / npts));
    PSFD_CHECK_LAUNCH();
  }
  std::vector<double> h(2 * P->nrhs);
  PSFD_CUDA_TRY(cudaMemcpyAsync(h.data(), acc, sizeof(double) * 2 * P->nrhs, cudaMemcpyDeviceToHost, s));
  PSFD_CUDA_TRY(cudaStreamSynchronize(s));
  const double npts = (double)n / 3.0;
  for (int r = 0; r < P->nrhs; ++r) J[r] = (h[r] + lam_hf * h[P->nrhs + r]) / npts;
  return PSFD_OK;
}
