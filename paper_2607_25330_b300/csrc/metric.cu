// Threshold-contour width metric of the scattered near field (Sec. 4, practical assessment of
// scattered-field convergence; Eq. logistic_sigmoid).
//
// I = |E_comp|^2 on one z-plane; the S = 0.5 contour of the logistic map is I = I_th.  Along
// every scan line (m = min(n_lines, n) rows at floor(i n / m), the same for columns; periodic)
// the contour crosses between samples j and j + 1 where (I_j >= I_th) != (I_{j+1} >= I_th), at
// j + (I_th - I_j) / (I_{j+1} - I_j).  A segment runs from an upward crossing to the next
// downward one (with the periodic wrap); its width times the pixel size is d.  Each reference
// segment is matched to the segment under test whose centre lies inside it (nearest centre if
// several): |d_ref - d| / demag is accumulated; a reference segment without a match is unresolved.
#include <cmath>
#include <vector>

#include "internal.h"

namespace {

constexpr int MET_THREADS = 128;

struct LineArgs {
  const cf* E;        // field plane base: E[(comp * nz + z) * ny * nx], per rhs offset applied
  int nx, ny, my, mx; // grid and scan-line counts
  float I_th;
  int cap;            // segment capacity per line
  float2* segs;       // [lines][cap] (start, end) in samples, end > start
  int* count;         // [lines]
};

__device__ __forceinline__ float intensity(cf e) {
  // rounded products and sum (no contraction), the float32 arithmetic the metric is defined in
  return __fadd_rn(__fmul_rn(e.x, e.x), __fmul_rn(e.y, e.y));
}

// one thread per scan line: rows first (along x), then columns (along y)
__global__ void k_line_segments(LineArgs a) {
  const int line = blockIdx.x * blockDim.x + threadIdx.x;
  if (line >= a.my + a.mx) return;
  const bool row = line < a.my;
  const int n = row ? a.nx : a.ny;
  const long stride = row ? 1 : a.nx;
  const long base = row ? (long)((line * (long)a.ny) / a.my) * a.nx : (long)(((line - a.my) * (long)a.nx) / a.mx);
  float2* out = a.segs + (long)line * a.cap;
  // first pass: is there any crossing; find a downward crossing to start from so that every
  // segment is closed when it is emitted
  int start = -1;
  for (int j = 0; j < n; ++j) {
    const bool a0 = intensity(a.E[base + j * stride]) >= a.I_th;
    const bool a1 = intensity(a.E[base + ((j + 1) % n) * stride]) >= a.I_th;
    if (a0 && !a1) { start = j; break; }
  }
  int cnt = 0;
  if (start >= 0) {
    float up = 0.f;
    bool open = false;
    for (int s = 1; s <= n; ++s) {
      const int j = (start + s) % n, j1 = (j + 1) % n;
      const float i0 = intensity(a.E[base + j * stride]), i1 = intensity(a.E[base + j1 * stride]);
      const bool a0 = i0 >= a.I_th, a1 = i1 >= a.I_th;
      if (a0 == a1) continue;
      const float x = (float)j + (a.I_th - i0) / (i1 - i0);
      if (a1) {            // upward
        up = x;
        open = true;
      } else if (open) {   // downward, closes the open segment
        float e = x;
        if (e <= up) e += (float)n;
        float u = up;
        if (u >= (float)n) { u -= (float)n; e -= (float)n; }
        if (cnt < a.cap) out[cnt] = make_float2(u, e);
        ++cnt;
        open = false;
      }
    }
  }
  a.count[line] = cnt < a.cap ? cnt : a.cap;
}

}  // namespace

extern "C" int psfd_width_metric(psfd_plan P, const psfd_c64* E, const psfd_c64* E_ref, int rhs, int comp, int z,
                                 float I_th, int n_lines, double demag, double* out) {
  if (!P || !E || !E_ref || !out) { psfd_set_error("psfd_width_metric: null argument"); return PSFD_ERR_ARG; }
  if (rhs < 0 || rhs >= P->nrhs || comp < 0 || comp > 2 || z < 0 || z >= P->nz || n_lines < 1 || !(demag > 0)) {
    psfd_set_error("psfd_width_metric: bad rhs / component / plane / line count / demagnification");
    return PSFD_ERR_ARG;
  }
  cudaStream_t s = P->stream;
  const int nx = P->nx, ny = P->ny;
  const int my = n_lines < ny ? n_lines : ny, mx = n_lines < nx ? n_lines : nx;
  const int lines = my + mx;
  const int cap = (nx > ny ? nx : ny) / 2 + 1;
  const long off = (long)rhs * P->nvec + ((long)comp * P->nz + z) * P->ncols;
  float2* segs = nullptr;
  int* count = nullptr;
  PSFD_CUDA_TRY(cudaMallocAsync((void**)&segs, 2 * (size_t)lines * cap * sizeof(float2), s));
  PSFD_CUDA_TRY(cudaMallocAsync((void**)&count, 2 * (size_t)lines * sizeof(int), s));
  for (int f = 0; f < 2; ++f) {
    LineArgs a{};
    a.E = (const cf*)(f == 0 ? E : E_ref) + off;
    a.nx = nx; a.ny = ny; a.my = my; a.mx = mx; a.I_th = I_th; a.cap = cap;
    a.segs = segs + (size_t)f * lines * cap;
    a.count = count + (size_t)f * lines;
    k_line_segments<<<(lines + MET_THREADS - 1) / MET_THREADS, MET_THREADS, 0, s>>>(a);
    PSFD_CHECK_LAUNCH();
  }
  std::vector<float2> hs(2 * (size_t)lines * cap);
  std::vector<int> hc(2 * (size_t)lines);
  PSFD_CUDA_TRY(cudaMemcpyAsync(hs.data(), segs, hs.size() * sizeof(float2), cudaMemcpyDeviceToHost, s));
  PSFD_CUDA_TRY(cudaMemcpyAsync(hc.data(), count, hc.size() * sizeof(int), cudaMemcpyDeviceToHost, s));
  PSFD_CUDA_TRY(cudaStreamSynchronize(s));
  PSFD_CUDA_TRY(cudaFreeAsync(segs, s));
  PSFD_CUDA_TRY(cudaFreeAsync(count, s));
  // matching of the (at most a few thousand) segments on the host
  double sum = 0, sum2 = 0, mx_dev = 0;
  long matched = 0, unresolved = 0, above = 0;
  for (int l = 0; l < lines; ++l) {
    const int n = l < my ? nx : ny;
    const double px = l < my ? P->p.dx : P->p.dy;
    const float2* sg = hs.data() + (size_t)l * cap;
    const float2* rf = hs.data() + ((size_t)lines + l) * cap;
    for (int r = 0; r < hc[lines + l]; ++r) {
      const double a = rf[r].x, b = rf[r].y, mid = 0.5 * (a + b);
      int best = -1;
      double bd = 0;
      for (int q = 0; q < hc[l]; ++q) {
        const double ctr = 0.5 * ((double)sg[q].x + (double)sg[q].y);
        for (int sh = -1; sh <= 1; ++sh) {
          const double cc = ctr + sh * n;
          if (a <= cc && cc <= b) {
            const double dist = fabs(cc - mid);
            if (best < 0 || dist < bd) { best = q; bd = dist; }
          }
        }
      }
      if (best < 0) { ++unresolved; continue; }
      const double dev = fabs((b - a) - ((double)sg[best].y - (double)sg[best].x)) * px / demag;
      sum += dev; sum2 += dev * dev; mx_dev = dev > mx_dev ? dev : mx_dev; ++matched;
      if (dev > 1.0) ++above;
    }
  }
  const double mean = matched ? sum / matched : 0.0;
  out[0] = mean;
  out[1] = matched ? sqrt(fmax(0.0, sum2 / matched - mean * mean)) : 0.0;
  out[2] = mx_dev;
  out[3] = (double)matched;
  out[4] = (double)unresolved;
  out[5] = matched ? (double)above / matched : 0.0;
  return PSFD_OK;
}
