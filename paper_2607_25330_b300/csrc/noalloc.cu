// Spectral upsampling that allocates no memory.
//
// psfd_spectral_upsample needs scratch for the coarse spectrum and for the FFT
// twiddle tables, and obtains it with cudaMalloc.  Some callers cannot allocate
// device memory inside a call: code running while a caching allocator owns all
// free memory, real-time loops that must not hit the driver's allocator, or
// hosts that forbid allocation after start-up.  This variant keeps its scratch
// in one fixed array that lives in this library's device image, so a call only
// launches kernels and issues asynchronous copies and memsets.
//
// Limits and sharing:
//  * the scratch holds kUpsampleStaticMax complex64 entries (16 MiB); a call
//    needs nb*nx0*ny0*nz0 + nx0+ny0+nz0+nx+ny+nz entries and is rejected
//    (PSFD_ERR_ARG) above that;
//  * every GPU that loads the library keeps these 16 MiB until the process exits;
//  * every call shares the array: calls whose work can overlap on the GPU (on
//    different streams, or from different host threads) race; serialise them;
//  * the first call on a device looks up the array's device address with
//    cudaGetSymbolAddress (the host-side name of a __device__ array is only a
//    stand-in, never a device pointer); make that first call before any stream
//    capture.  Later calls reuse the cached address.
// Nothing in the array has to start at zero: the twiddles are rewritten and the
// coarse spectrum is overwritten by every call.
#include <mutex>

#include "fft.cuh"
#include "internal.h"

namespace {

constexpr long kUpsampleStaticMax = 1L << 21;  // complex64 entries = 16 MiB

static __device__ __align__(256) cf g_upsample_scratch[kUpsampleStaticMax];

constexpr int kMaxDevices = 64;
std::mutex g_sym_mu;
cf* g_sym_ptr[kMaxDevices] = {nullptr};

int scratch_address(cf** out) {
  int dev = -1;
  PSFD_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    psfd_set_error("psfd_spectral_upsample_static: device ordinal %d out of range", dev);
    return PSFD_ERR_ARG;
  }
  std::lock_guard<std::mutex> lk(g_sym_mu);
  if (!g_sym_ptr[dev]) {
    void* p = nullptr;
    PSFD_CUDA_TRY(cudaGetSymbolAddress(&p, g_upsample_scratch));
    g_sym_ptr[dev] = (cf*)p;
  }
  *out = g_sym_ptr[dev];
  return PSFD_OK;
}

// exp(-2 pi i m / n) for m < n, computed on the device in double precision
__global__ void k_twiddles(cf* tw, int n) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n) return;
  double s, c;
  sincospi(-2.0 * (double)m / (double)n, &s, &c);
  tw[m] = make_float2((float)c, (float)s);
}

__global__ void k_pad_static(const cf* __restrict__ src, cf* __restrict__ dst, int nx0, int ny0, int nz0, int nx,
                             int ny, int nz, long nb, float scale) {
  const long n0 = (long)nx0 * ny0 * nz0;
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb * n0) return;
  const long b = i / n0, r = i - b * n0;
  const int x = (int)(r % nx0), y = (int)((r / nx0) % ny0), z = (int)(r / ((long)nx0 * ny0));
  auto map = [](int k, int n0_, int n) { int s = (k <= (n0_ - 1) / 2) ? k : k - n0_; return s < 0 ? s + n : s; };
  const long o = ((b * nz + map(z, nz0, nz)) * ny + map(y, ny0, ny)) * (long)nx + map(x, nx0, nx);
  dst[o] = cscale(src[i], scale);
}

}  // namespace

extern "C" int psfd_spectral_upsample_static(const psfd_c64* src, int nb, int nx0, int ny0, int nz0, psfd_c64* dst,
                                             int nx, int ny, int nz, void* stream) {
  if (!src || !dst || nb <= 0) { psfd_set_error("psfd_spectral_upsample_static: null argument"); return PSFD_ERR_ARG; }
  if (nx < nx0 || ny < ny0 || nz < nz0 || !lateral_supported(nx0) || !lateral_supported(ny0) ||
      !axial_supported(nz0) || !lateral_supported(nx) || !lateral_supported(ny) || !axial_supported(nz)) {
    psfd_set_error("psfd_spectral_upsample_static: unsupported sizes");
    return PSFD_ERR_ARG;
  }
  const long n0 = (long)nx0 * ny0 * nz0;
  const long ntw = (long)nx0 + ny0 + nz0 + nx + ny + nz;
  if ((long)nb * n0 > kUpsampleStaticMax - ntw) {
    psfd_set_error("psfd_spectral_upsample_static: nb*nx0*ny0*nz0 = %ld exceeds the static scratch of %ld "
                   "complex entries", (long)nb * n0, kUpsampleStaticMax - ntw);
    return PSFD_ERR_ARG;
  }
  cf* scratch = nullptr;
  int rc = scratch_address(&scratch);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  cf* tmp = scratch;                       // coarse spectrum, nb * n0 entries
  cf* tw = scratch + (long)nb * n0;        // six twiddle tables
  const int sizes[6] = {nx0, ny0, nz0, nx, ny, nz};
  cf* twp[6];
  long off = 0;
  for (int k = 0; k < 6; ++k) {
    twp[k] = tw + off;
    k_twiddles<<<(sizes[k] + 127) / 128, 128, 0, s>>>(twp[k], sizes[k]);
    PSFD_CHECK_LAUNCH();
    off += sizes[k];
  }
  PSFD_CUDA_TRY(cudaMemcpyAsync(tmp, src, (size_t)nb * n0 * sizeof(cf), cudaMemcpyDeviceToDevice, s));
  if ((rc = launch_rows(nx0, tmp, (long)nb * nz0 * ny0, true, 1.f, twp[0], s))) return rc;
  if ((rc = launch_cols(ny0, nx0, tmp, (long)nb * nz0 * nx0, true, 1.f, twp[1], s))) return rc;
  if ((rc = launch_cols(nz0, nx0 * ny0, tmp, (long)nb * nx0 * ny0, true, 1.f, twp[2], s))) return rc;
  const long n1 = (long)nx * ny * nz;
  PSFD_CUDA_TRY(cudaMemsetAsync(dst, 0, (size_t)nb * n1 * sizeof(cf), s));
  k_pad_static<<<(unsigned)(((long)nb * n0 + 255) / 256), 256, 0, s>>>(tmp, (cf*)dst, nx0, ny0, nz0, nx, ny, nz, nb,
                                                                       1.0f / (float)n0);
  PSFD_CHECK_LAUNCH();
  if ((rc = launch_cols(nz, nx * ny, (cf*)dst, (long)nb * nx * ny, false, 1.f, twp[5], s))) return rc;
  if ((rc = launch_cols(ny, nx, (cf*)dst, (long)nb * nz * nx, false, 1.f, twp[4], s))) return rc;
  return launch_rows(nx, (cf*)dst, (long)nb * nz * ny, false, 1.f, twp[3], s);
}
