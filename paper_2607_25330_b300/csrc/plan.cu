// Plan set-up, geometry (mask -> fill), FP64 multilayer reflection and the
// background source b (Sec. 2.2, Eq. bg_source).
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "fft.cuh"
#include "internal.h"

static thread_local char g_err[1024] = "";
static std::atomic<long long> g_launches{0};

void psfd_count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
extern "C" long long psfd_launch_count(void) { return g_launches.load(); }

// ---------------------------------------------------------------- stage timing
namespace {
struct StageRec {
  int stage;
  cudaEvent_t a, b;
  double bytes;
};
std::mutex g_tmu;
bool g_timing = false;
std::vector<StageRec> g_open[ST_N];   // begun, not yet ended (stack per stage)
std::vector<StageRec> g_done;
std::vector<cudaEvent_t> g_pool;
double g_ms[ST_N];
double g_bytes[ST_N];
long long g_calls[ST_N];

cudaEvent_t ev_get() {
  if (!g_pool.empty()) { cudaEvent_t e = g_pool.back(); g_pool.pop_back(); return e; }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}
void harvest(bool wait) {
  std::vector<StageRec> keep;
  for (auto& r : g_done) {
    if (wait) cudaEventSynchronize(r.b);
    if (cudaEventQuery(r.b) == cudaSuccess) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, r.a, r.b);
      g_ms[r.stage] += ms;
      g_bytes[r.stage] += r.bytes;
      g_calls[r.stage] += 1;
      g_pool.push_back(r.a);
      g_pool.push_back(r.b);
    } else {
      keep.push_back(r);
    }
  }
  g_done.swap(keep);
}
}  // namespace

void stage_mark(cudaStream_t s, int stage, bool begin, double bytes) {
  if (!g_timing) return;
  std::lock_guard<std::mutex> lk(g_tmu);
  if (begin) {
    StageRec r{stage, ev_get(), nullptr, 0.0};
    cudaEventRecord(r.a, s);
    g_open[stage].push_back(r);
  } else if (!g_open[stage].empty()) {
    StageRec r = g_open[stage].back();
    g_open[stage].pop_back();
    r.b = ev_get();
    r.bytes = bytes;
    cudaEventRecord(r.b, s);
    g_done.push_back(r);
    if (g_done.size() > 4096) harvest(true);
  }
}

extern "C" int psfd_timing_enable(int on) {
  std::lock_guard<std::mutex> lk(g_tmu);
  harvest(true);
  for (int i = 0; i < ST_N; ++i) { g_ms[i] = 0; g_bytes[i] = 0; g_calls[i] = 0; g_open[i].clear(); }
  g_timing = on != 0;
  return PSFD_OK;
}

extern "C" int psfd_timing_read(double* ms, long long* calls, int nstages) {
  return psfd_timing_read_bytes(ms, calls, nullptr, nstages);
}

extern "C" int psfd_timing_read_bytes(double* ms, long long* calls, double* bytes, int nstages) {
  std::lock_guard<std::mutex> lk(g_tmu);
  harvest(true);
  for (int i = 0; i < nstages && i < ST_N; ++i) {
    if (ms) ms[i] = g_ms[i];
    if (calls) calls[i] = g_calls[i];
    if (bytes) bytes[i] = g_bytes[i];
  }
  return PSFD_OK;
}

void psfd_set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

extern "C" const char* psfd_last_error(void) { return g_err; }
extern "C" const char* psfd_version(void) { return "psfd-b300 0.1 (sm_103a)"; }

// The bounded device-side waits record a timeout instead of hanging: the operator's plane kernel
// in P->err, the layered apply in P->lay_err[1], the FNO mode mixing in a global flag.  Read and
// clear them (synchronises the plan's stream).
int plan_wait_status(psfd_plan_s* P) {
  int h[2] = {0, 0}, tc = 0;
  cudaStream_t s = P->stream;
  if (P->err) PSFD_CUDA_TRY(cudaMemcpyAsync(&h[0], P->err, sizeof(int), cudaMemcpyDeviceToHost, s));
  if (P->lay_err) PSFD_CUDA_TRY(cudaMemcpyAsync(&h[1], P->lay_err + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
  PSFD_CUDA_TRY(cudaStreamSynchronize(s));
  int rc = fno_mix_tc_error(&tc);
  if (rc) return rc;
  int tm = 0;
  if ((rc = fno_mlp_tc_error(&tm))) return rc;
  tc = tc || tm;
  if (!h[0] && !h[1] && !tc) return PSFD_OK;
  if (h[0]) PSFD_CUDA_TRY(cudaMemsetAsync(P->err, 0, sizeof(int), s));
  if (h[1]) PSFD_CUDA_TRY(cudaMemsetAsync(P->lay_err + 1, 0, sizeof(int), s));
  PSFD_CUDA_TRY(cudaStreamSynchronize(s));
  psfd_set_error("a bounded device-side wait gave up (%s)",
                 h[0] ? "operator plane kernel" : h[1] ? "layered preconditioner apply"
                                                : (tm ? "FNO pointwise layers" : "FNO mode mixing"));
  return PSFD_ERR_TIMEOUT;
}

extern "C" int psfd_device_status(psfd_plan P) {
  if (!P) { psfd_set_error("psfd_device_status: null plan"); return PSFD_ERR_ARG; }
  return plan_wait_status(P);
}

extern "C" int psfd_supported(int nx, int ny, int nz) {
  return lateral_supported(nx) && lateral_supported(ny) && axial_supported(nz) ? 1 : 0;
}

// ------------------------------------------------------------ FP64 complex helpers
struct cd {
  double re, im;
};
__device__ __forceinline__ cd cd_(double r, double i) { return {r, i}; }
__device__ __forceinline__ cd operator+(cd a, cd b) { return {a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ cd operator-(cd a, cd b) { return {a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ cd operator*(cd a, cd b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
__device__ __forceinline__ cd operator*(double s, cd a) { return {s * a.re, s * a.im}; }
__device__ __forceinline__ cd cdiv(cd a, cd b) {
  // scaled division
  if (fabs(b.re) >= fabs(b.im)) {
    double r = b.im / b.re, den = b.re + b.im * r;
    return {(a.re + a.im * r) / den, (a.im - a.re * r) / den};
  } else {
    double r = b.re / b.im, den = b.re * r + b.im;
    return {(a.re * r + a.im) / den, (a.im * r - a.re) / den};
  }
}
__device__ __forceinline__ double cabs_(cd a) { return hypot(a.re, a.im); }
// principal square root, then the branch with Im >= 0
__device__ __forceinline__ cd csqrt_up(cd z) {
  double r = hypot(z.re, z.im);
  cd s;
  if (r == 0.0) return {0.0, 0.0};
  if (z.re >= 0) {
    double u = sqrt(0.5 * (r + z.re));
    s = {u, z.im / (2.0 * u)};
  } else {
    double u = sqrt(0.5 * (r - z.re));
    s = {fabs(z.im) / (2.0 * u), (z.im >= 0 ? u : -u)};
  }
  if (s.im < 0) s = {-s.re, -s.im};
  return s;
}
__device__ __forceinline__ cd ccos_(cd z) { return {cos(z.re) * cosh(z.im), -sin(z.re) * sinh(z.im)}; }
__device__ __forceinline__ cd csin_(cd z) { return {sin(z.re) * cosh(z.im), cos(z.re) * sinh(z.im)}; }

// ------------------------------------------------------------ transfer matrix (FP64)
// Reflection of the stack below z_ml for every lateral Bloch mode (Sec. 2.2,
// TMM-based R_ml).  Characteristic matrix of the tangential fields per layer,
//   [[cos d, i sin d / q], [i q sin d, cos d]],  d = kz_j t_j,
// q = kz (s) or kz / eps (p); the product is renormalised after each layer
// (the reflection is a ratio, so scale does not matter).  r = (a + c)/(c - a)
// with a = P21 - q_s P11, c = q_0 (P22 - q_s P12); r_p (tangential E) = -r.
struct StackDev {
  int nl;
  const double* n_re;
  const double* n_im;
  const double* d;
  double sub_re, sub_im;
};

__device__ cd tmm_r(double kp2, double k0, const StackDev& st, bool ppol) {
  cd P11 = {1, 0}, P12 = {0, 0}, P21 = {0, 0}, P22 = {1, 0};
  for (int j = 0; j < st.nl; ++j) {
    cd n = {st.n_re[j], st.n_im[j]};
    cd eps = n * n;
    cd kzj = csqrt_up(k0 * k0 * eps - cd_(kp2, 0.0));
    cd q = ppol ? cdiv(kzj, eps) : kzj;
    cd dl = st.d[j] * kzj;
    cd c = ccos_(dl), s = csin_(dl);
    cd is = {-s.im, s.re};                 // i sin
    cd m12 = cdiv(is, q), m21 = is * q;
    cd N11 = c * P11 + m12 * P21, N12 = c * P12 + m12 * P22;
    cd N21 = m21 * P11 + c * P21, N22 = m21 * P12 + c * P22;
    double mx = fmax(fmax(cabs_(N11), cabs_(N12)), fmax(cabs_(N21), cabs_(N22)));
    double inv = (mx > 0) ? 1.0 / mx : 1.0;
    P11 = inv * N11; P12 = inv * N12; P21 = inv * N21; P22 = inv * N22;
  }
  cd ns = {st.sub_re, st.sub_im};
  cd es = ns * ns;
  cd kzs = csqrt_up(k0 * k0 * es - cd_(kp2, 0.0));
  cd qs = ppol ? cdiv(kzs, es) : kzs;
  cd q0 = csqrt_up(cd_(k0 * k0 - kp2, 0.0));
  cd a = P21 - qs * P11;
  cd c = q0 * (P22 - qs * P12);
  cd r = cdiv(a + c, c - a);
  return ppol ? cd_(-r.re, -r.im) : r;
}

__global__ void k_tmm(int nx, int ny, double dkx, double dky, double kx_inc, double ky_inc, double k0,
                      StackDev st, double2* rs64, double2* rp64, double2* kz064, float4* refl, cf* kz0f) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= nx * ny) return;
  int ix = m % nx, iy = m / nx;
  double kx = dkx * fft_signed(ix, nx) + kx_inc;
  double ky = dky * fft_signed(iy, ny) + ky_inc;
  double kp2 = kx * kx + ky * ky;
  cd rs = tmm_r(kp2, k0, st, false);
  cd rp = tmm_r(kp2, k0, st, true);
  cd kz0 = csqrt_up(cd_(k0 * k0 - kp2, 0.0));
  rs64[m] = make_double2(rs.re, rs.im);
  rp64[m] = make_double2(rp.re, rp.im);
  kz064[m] = make_double2(kz0.re, kz0.im);
  refl[m] = make_float4((float)rs.re, (float)rs.im, (float)rp.re, (float)rp.im);
  kz0f[m] = make_float2((float)kz0.re, (float)kz0.im);
}

// ------------------------------------------------------------ source b (Eq. bg_source)
// b = k0^2 deps (E_inc + R E_inc): the incident plane wave is the lateral mode
// (0,0); its reflection uses that mode's FP64 r_s, r_p.  Computed in FP64.
struct SourceArgs {
  const float* fill;
  cf* b;
  int nx, ny, nz, z_ml;
  long ncols;
  double dz, k0, theta, phi;
  const double2* pc64;     // per-plane contrast c[z]
  const double2* rs64;
  const double2* rp64;
  const double2* kz064;
  int pol;
};

// grid: (ceil(ncols / blockDim), nz); the z-only factors are computed once per block
// per plane z: (re, im) of E_inc + R E_inc for the three components (one thread per plane; the
// FP64 trigonometry runs once per plane instead of once per block)
__global__ void k_source_z(SourceArgs a, double* ftab) {
  const int z = blockIdx.x * blockDim.x + threadIdx.x;
  if (z >= a.nz) return;
  double st = sin(a.theta), ctt = cos(a.theta), sp = sin(a.phi), cp = cos(a.phi);
  double e[3];
  if (a.pol == 0) { e[0] = -sp; e[1] = cp; e[2] = 0.0; }
  else { e[0] = ctt * cp; e[1] = ctt * sp; e[2] = st; }
  double kx = a.k0 * st * cp, ky = a.k0 * st * sp;
  double kpar = sqrt(kx * kx + ky * ky);
  double sx, sy, tx, ty;
  if (kpar < 1e-12 * a.k0) { sx = 0; sy = 1; tx = 1; ty = 0; }
  else { sx = -ky / kpar; sy = kx / kpar; tx = kx / kpar; ty = ky / kpar; }
  cd rs = {a.rs64[0].x, a.rs64[0].y}, rp = {a.rp64[0].x, a.rp64[0].y};
  cd kz0 = {a.kz064[0].x, a.kz064[0].y};
  double as = sx * e[0] + sy * e[1], at = tx * e[0] + ty * e[1];
  cd r0 = as * sx * rs + at * tx * rp;
  cd r1 = as * sy * rs + at * ty * rp;
  cd r2 = cdiv(cd_(-1, 0) * (kx * r0 + ky * r1), kz0);
  double zr = (z - a.z_ml) * a.dz;
  double kzi = a.k0 * ctt;
  cd einc = {cos(kzi * zr), -sin(kzi * zr)};
  cd prof = {0, 0};
  if (zr >= 0) {
    double mag = exp(-kz0.im * zr);
    prof = {mag * cos(kz0.re * zr), mag * sin(kz0.re * zr)};
  }
  cd tot[3] = {e[0] * einc + r0 * prof, e[1] * einc + r1 * prof, e[2] * einc + r2 * prof};
  for (int c = 0; c < 3; ++c) { ftab[z * 6 + 2 * c] = tot[c].re; ftab[z * 6 + 2 * c + 1] = tot[c].im; }
}

__global__ void k_source(SourceArgs a, const double* __restrict__ ftab) {
  __shared__ double f_tot[6];   // (re, im) of E_inc + R E_inc for the three components at this z
  const int z = blockIdx.y;
  if (threadIdx.x < 6) f_tot[threadIdx.x] = ftab[z * 6 + threadIdx.x];
  __syncthreads();
  const long xy = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (xy >= a.ncols) return;
  const long i = (long)z * a.ncols + xy;
  const double f = a.fill[i];
  const double k02 = a.k0 * a.k0;
  const cd de = {f * a.pc64[z].x * k02, f * a.pc64[z].y * k02};
  const long plane = a.ncols * a.nz;
  for (int c = 0; c < 3; ++c) {
    const cd v = de * cd_(f_tot[2 * c], f_tot[2 * c + 1]);
    a.b[c * plane + i] = make_float2((float)v.re, (float)v.im);
  }
}

// ------------------------------------------------------------ geometry kernels
__global__ void k_u8_to_c(const uint8_t* a, cf* out, long n) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = make_float2((float)a[i], 0.f);
}

__global__ void k_extrude(const cf* plane, const float* zprof, float* fill, long ncols, int nz) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ncols * nz) return;
  int z = (int)(i / ncols);
  fill[i] = zprof[z] * plane[i % ncols].x;
}

// planes with any nonzero fill
__global__ void k_fill_range(const float* fill, long ncols, int nz, int* zr) {
  int z = blockIdx.x;
  int any = 0;
  for (long i = threadIdx.x; i < ncols; i += blockDim.x) any |= (fill[(long)z * ncols + i] != 0.f);
  any = __syncthreads_or(any);
  if (threadIdx.x == 0 && any) {
    atomicMin(&zr[0], z);
    atomicMax(&zr[1], z + 1);
  }
}

// ------------------------------------------------------------ plan
static void host_twiddles(int n, std::vector<cf>& out) {
  out.resize(n);
  for (int m = 0; m < n; ++m) {
    double a = -2.0 * M_PI * (double)m / (double)n;
    out[m] = make_float2((float)cos(a), (float)sin(a));
  }
}

static double host_fftk(int i, int n, double d) {
  int m = (i <= (n - 1) / 2) ? i : i - n;
  return 2.0 * M_PI * m / (n * d);
}

double fft_wavenumber(int i, int n, double d) { return host_fftk(i, n, d); }

// 1/s(z) of the stretched-coordinate PML: s = 1 + i alpha (d/d_pml)^3, alpha = 4 ln(1/R0) / (2 k0 d_pml)
// sigma(z) of the PML's absorbing backing: on the outermost nb = max(1, np / 4) planes of each end
// of the box (where the two PMLs meet across the periodic wrap), pml_backing ((nb - j) / nb)^2 on
// the j-th plane from the end; 0 elsewhere
void pml_backing64(const psfd_params_t& p, std::vector<double>& sb) {
  sb.assign(p.nz, 0.0);
  if (p.pml_planes <= 0 || !(p.pml_backing > 0)) return;
  const int nb = std::max(1, p.pml_planes / 4);
  for (int j = 0; j < nb; ++j) {
    const double w = (double)(nb - j) / nb;
    sb[j] = sb[p.nz - 1 - j] = p.pml_backing * w * w;
  }
}

void pml_sinv64(const psfd_plan_s* P, std::vector<zd>& sinv) {
  const psfd_params_t& p = P->p;
  sinv.resize(p.nz);
  const int np = p.pml_planes;
  const double dpml = np * p.dz;
  const double alpha = np > 0 ? 4.0 * log(1.0 / p.pml_R0) / (2.0 * P->k0 * dpml) : 0.0;
  for (int k = 0; k < p.nz; ++k) {
    double d = 0.0;
    if (k < np) d = (np - k) * p.dz;
    else if (k >= p.nz - np) d = (k - (p.nz - np - 1)) * p.dz;
    const double sig = np > 0 ? alpha * pow(d / dpml, 3.0) : 0.0;
    const double den = 1.0 + sig * sig;            // 1/(1 + i sig) = (1 - i sig)/(1 + sig^2)
    sinv[k] = make_double2(1.0 / den, -sig / den);
  }
}

static int upload_pc32(psfd_plan_s* P) {
  std::vector<cf> h(P->pc_host.size());
  for (size_t z = 0; z < h.size(); ++z) h[z] = make_float2((float)P->pc_host[z].x, (float)P->pc_host[z].y);
  if (!P->pc) PSFD_CUDA_TRY(cudaMalloc((void**)&P->pc, h.size() * sizeof(cf)));
  PSFD_CUDA_TRY(cudaMemcpy(P->pc, h.data(), h.size() * sizeof(cf), cudaMemcpyHostToDevice));
  return PSFD_OK;
}

static int upload(void** dst, const void* src, size_t bytes) {
  PSFD_CUDA_TRY(cudaMalloc(dst, bytes));
  PSFD_CUDA_TRY(cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice));
  return PSFD_OK;
}

static void plan_free(psfd_plan_s* P) {
  fp64_free(P);
  layered_free(P);
  void* ptrs[] = {P->kx, P->ky, P->kz, P->sinv, P->kbg, P->sback, P->tw_x, P->tw_y, P->tw_z, P->R.rs64, P->R.rp64,
                  P->R.kz064, P->R.refl, P->R.kz0, P->G, P->tmpA, P->tmpB, P->err, P->pc, P->pc64};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  if (P->prog_h) cudaFreeHost(P->prog_h);
}

extern "C" int psfd_plan_create(psfd_plan* out, const psfd_params_t* prm) {
  if (!out || !prm) { psfd_set_error("psfd_plan_create: null argument"); return PSFD_ERR_ARG; }
  *out = nullptr;
  const psfd_params_t& p = *prm;
  if (p.nrhs < 1 || p.dx <= 0 || p.dy <= 0 || p.dz <= 0 || p.lambda <= 0) {
    psfd_set_error("psfd_plan_create: invalid sizes or spacing");
    return PSFD_ERR_ARG;
  }
  if (!psfd_supported(p.nx, p.ny, p.nz)) {
    psfd_set_error("psfd_plan_create: unsupported grid %dx%dx%d", p.nx, p.ny, p.nz);
    return PSFD_ERR_ARG;
  }
  if (p.pml_planes < 0 || 2 * p.pml_planes >= p.nz || p.z_ml < 0 || p.z_ml >= p.nz ||
      (p.pml_planes > 0 && !(p.pml_R0 > 0 && p.pml_R0 < 1)) || !(p.pml_backing >= 0) ||
      !std::isfinite(p.pml_backing)) {
    psfd_set_error("psfd_plan_create: invalid PML / z_ml");
    return PSFD_ERR_ARG;
  }
  psfd_plan_s* P = new psfd_plan_s();
  P->p = p;
  P->stream = (cudaStream_t)p.stream;
  P->nx = p.nx; P->ny = p.ny; P->nz = p.nz; P->nrhs = p.nrhs;
  P->ncols = (long)p.nx * p.ny;
  P->nvec = 3L * p.nz * P->ncols;
  P->k0 = 2.0 * M_PI / p.lambda;
  double th = p.theta_deg * M_PI / 180.0, ph = p.phi_deg * M_PI / 180.0;
  P->kx_inc = P->k0 * sin(th) * cos(ph);
  P->ky_inc = P->k0 * sin(th) * sin(ph);
  P->kz_inc = P->k0 * cos(th);
  P->deps_re = p.eps_abs_re - 1.0;
  P->deps_im = p.eps_abs_im;
  // light-cone check (k_z = 0 exactly is not representable)
  for (int iy = 0; iy < p.ny; ++iy)
    for (int ix = 0; ix < p.nx; ++ix) {
      double kx = host_fftk(ix, p.nx, p.dx) + P->kx_inc, ky = host_fftk(iy, p.ny, p.dy) + P->ky_inc;
      if (fabs(P->k0 * P->k0 - kx * kx - ky * ky) < 1e-18 * P->k0 * P->k0) {
        psfd_set_error("psfd_plan_create: a lateral mode lies on the light cone");
        delete P;
        return PSFD_ERR_ARG;
      }
    }
  std::vector<float> kx(p.nx), ky(p.ny), kz(p.nz);
  for (int i = 0; i < p.nx; ++i) kx[i] = (float)(host_fftk(i, p.nx, p.dx) + P->kx_inc);
  for (int i = 0; i < p.ny; ++i) ky[i] = (float)(host_fftk(i, p.ny, p.dy) + P->ky_inc);
  for (int i = 0; i < p.nz; ++i) kz[i] = (float)host_fftk(i, p.nz, p.dz);
  P->pc_host.assign(p.nz, make_double2(P->deps_re, P->deps_im));
  std::vector<zd> sinv64;
  pml_sinv64(P, sinv64);
  std::vector<cf> sinv(p.nz);
  for (int k = 0; k < p.nz; ++k) sinv[k] = make_float2((float)sinv64[k].x, (float)sinv64[k].y);
  pml_backing64(p, P->sback_host);
  std::vector<cf> kbg(p.nz);
  std::vector<float> sback(p.nz);
  for (int k = 0; k < p.nz; ++k) {
    kbg[k] = make_float2((float)(P->k0 * P->k0), (float)(P->k0 * P->k0 * P->sback_host[k]));
    sback[k] = (float)P->sback_host[k];
  }
  std::vector<cf> twx, twy, twz;
  host_twiddles(p.nx, twx);
  host_twiddles(p.ny, twy);
  host_twiddles(p.nz, twz);
  int rc = PSFD_OK;
  if ((rc = upload((void**)&P->kx, kx.data(), kx.size() * 4)) ||
      (rc = upload((void**)&P->ky, ky.data(), ky.size() * 4)) ||
      (rc = upload((void**)&P->kz, kz.data(), kz.size() * 4)) ||
      (rc = upload((void**)&P->sinv, sinv.data(), sinv.size() * 8)) ||
      (rc = upload((void**)&P->kbg, kbg.data(), kbg.size() * 8)) ||
      (rc = upload((void**)&P->sback, sback.data(), sback.size() * 4)) ||
      (rc = upload((void**)&P->pc64, P->pc_host.data(), P->pc_host.size() * sizeof(zd))) ||
      (rc = upload((void**)&P->tw_x, twx.data(), twx.size() * 8)) ||
      (rc = upload((void**)&P->tw_y, twy.data(), twy.size() * 8)) ||
      (rc = upload((void**)&P->tw_z, twz.data(), twz.size() * 8)) ||
      (rc = upload_pc32(P))) {
    plan_free(P);
    delete P;
    return rc;
  }
  // damping
  double kref = p.k_ref > 0 ? p.k_ref : P->k0;
  P->m_min = (float)p.m_min;
  P->kref2 = (float)(kref * kref);
  P->gamma = (float)p.gamma;
  P->damp_eps = (float)(p.damp_eps_rel * P->k0 * P->k0);
  // scratch
  size_t nm = (size_t)P->ncols;
  size_t vec_bytes = (size_t)p.nrhs * P->nvec * sizeof(cf);
  cudaError_t e1 = cudaMalloc((void**)&P->R.rs64, nm * 16);
  cudaError_t e2 = cudaMalloc((void**)&P->R.rp64, nm * 16);
  cudaError_t e3 = cudaMalloc((void**)&P->R.kz064, nm * 16);
  cudaError_t e4 = cudaMalloc((void**)&P->R.refl, nm * 16);
  cudaError_t e5 = cudaMalloc((void**)&P->R.kz0, nm * 8);
  cudaError_t e6 = cudaMalloc((void**)&P->tmpA, vec_bytes);
  cudaError_t e7 = cudaMalloc((void**)&P->tmpB, vec_bytes);
  if (e1 || e2 || e3 || e4 || e5 || e6 || e7) {
    psfd_set_error("psfd_plan_create: cudaMalloc failed (%s)", cudaGetErrorString(cudaGetLastError()));
    plan_free(P);
    delete P;
    return PSFD_ERR_CUDA;
  }
  // PSFD_PLANE=1 selects the single-pass plane kernel for the lateral contrast where it applies
  // (square planes up to 128^2).  Default: the three-pass path, which measured slightly faster at
  // 128x128x64 (0.141 vs 0.144 ms per A M apply): 186 one-CTA-per-SM planes make two waves.
  const char* po = getenv("PSFD_PLANE");
  P->use_plane = po && po[0] == '1';
  *out = P;
  return PSFD_OK;
}

extern "C" int psfd_plan_destroy(psfd_plan P) {
  if (!P) return PSFD_OK;
  cudaStreamSynchronize(P->stream);
  plan_free(P);
  delete P;
  return PSFD_OK;
}

extern "C" int psfd_set_history(psfd_plan P, double* hist, int capacity) {
  if (!P || capacity < 0) { psfd_set_error("psfd_set_history: bad argument"); return PSFD_ERR_ARG; }
  P->hist = hist;
  P->hist_cap = hist ? capacity : 0;
  return PSFD_OK;
}

extern "C" int psfd_mask_fill(psfd_plan P, const uint8_t* a_bin, const float* zprof, float* fill) {
  if (!P || !a_bin || !zprof || !fill) { psfd_set_error("psfd_mask_fill: null argument"); return PSFD_ERR_ARG; }
  cudaStream_t s = P->stream;
  long n = P->ncols;
  cf* buf = P->tmpA;  // one plane
  float* zp = nullptr;
  PSFD_CUDA_TRY(cudaMallocAsync((void**)&zp, P->nz * sizeof(float), s));
  PSFD_CUDA_TRY(cudaMemcpyAsync(zp, zprof, P->nz * sizeof(float), cudaMemcpyHostToDevice, s));
  k_u8_to_c<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a_bin, buf, n);
  PSFD_CHECK_LAUNCH();
  int rc;
  if ((rc = launch_rows(P->nx, buf, P->ny, true, 1.0f, P->tw_x, s))) return rc;
  if ((rc = launch_cols_gauss(P->ny, P->nx, buf, (float)P->p.sigma_px, P->tw_y, s))) return rc;
  if ((rc = launch_rows(P->nx, buf, P->ny, false, 1.0f / (float)n, P->tw_x, s))) return rc;
  k_extrude<<<(unsigned)((n * P->nz + 255) / 256), 256, 0, s>>>(buf, zp, fill, n, P->nz);
  PSFD_CHECK_LAUNCH();
  PSFD_CUDA_TRY(cudaFreeAsync(zp, s));
  return PSFD_OK;
}

extern "C" int psfd_background(psfd_plan P, const psfd_stack_t* stack, const float* fill, const int* pol,
                               psfd_c64* b) {
  if (!P || !stack || !fill || !pol || !b) { psfd_set_error("psfd_background: null argument"); return PSFD_ERR_ARG; }
  if (stack->n_layers < 0 || (stack->n_layers > 0 && (!stack->n_re || !stack->n_im || !stack->d))) {
    psfd_set_error("psfd_background: bad stack");
    return PSFD_ERR_ARG;
  }
  for (int r = 0; r < P->nrhs; ++r)
    if (pol[r] != PSFD_TE && pol[r] != PSFD_TM) { psfd_set_error("psfd_background: bad polarisation"); return PSFD_ERR_ARG; }
  cudaStream_t s = P->stream;
  int nl = stack->n_layers;
  double* dstack = nullptr;
  long nm = P->ncols;
  // the reflection tables depend on the grid, the illumination and the stack, not on the mask:
  // recompute them only when the stack differs from the one they were built for
  std::vector<double> sig;
  sig.reserve(3 * nl + 3);
  sig.push_back((double)nl);
  for (int l = 0; l < nl; ++l) { sig.push_back(stack->n_re[l]); sig.push_back(stack->n_im[l]); sig.push_back(stack->d[l]); }
  sig.push_back(stack->sub_re);
  sig.push_back(stack->sub_im);
  if (!P->have_background || sig != P->stack_sig) {
    if (nl > 0) {
      PSFD_CUDA_TRY(cudaMalloc((void**)&dstack, 3 * nl * sizeof(double)));
      PSFD_CUDA_TRY(cudaMemcpy(dstack, stack->n_re, nl * 8, cudaMemcpyHostToDevice));
      PSFD_CUDA_TRY(cudaMemcpy(dstack + nl, stack->n_im, nl * 8, cudaMemcpyHostToDevice));
      PSFD_CUDA_TRY(cudaMemcpy(dstack + 2 * nl, stack->d, nl * 8, cudaMemcpyHostToDevice));
    }
    StackDev st{nl, dstack, dstack ? dstack + nl : nullptr, dstack ? dstack + 2 * nl : nullptr, stack->sub_re,
                stack->sub_im};
    double dkx = 2.0 * M_PI / (P->nx * P->p.dx), dky = 2.0 * M_PI / (P->ny * P->p.dy);
    k_tmm<<<(unsigned)((nm + 127) / 128), 128, 0, s>>>(P->nx, P->ny, dkx, dky, P->kx_inc, P->ky_inc, P->k0, st,
                                                       P->R.rs64, P->R.rp64, P->R.kz064, P->R.refl, P->R.kz0);
    PSFD_CHECK_LAUNCH();
    P->stack_sig = sig;
  }
  // absorber plane range
  int* zr = nullptr;
  int hz[2] = {P->nz, 0};
  PSFD_CUDA_TRY(cudaMallocAsync((void**)&zr, 2 * sizeof(int), s));
  PSFD_CUDA_TRY(cudaMemcpyAsync(zr, hz, 8, cudaMemcpyHostToDevice, s));
  k_fill_range<<<P->nz, 256, 0, s>>>(fill, nm, P->nz, zr);
  PSFD_CHECK_LAUNCH();
  PSFD_CUDA_TRY(cudaMemcpyAsync(hz, zr, 8, cudaMemcpyDeviceToHost, s));
  PSFD_CUDA_TRY(cudaStreamSynchronize(s));
  PSFD_CUDA_TRY(cudaFreeAsync(zr, s));
  if (dstack) PSFD_CUDA_TRY(cudaFree(dstack));
  if (hz[1] <= hz[0]) { hz[0] = 0; hz[1] = 0; }
  P->za0 = hz[0];
  P->za1 = hz[1];
  size_t need = (size_t)P->nrhs * 3 * (size_t)(P->za1 - P->za0) * nm;
  if (need > P->G_elems) {
    if (P->G) cudaFree(P->G);
    P->G = nullptr;
    P->G_elems = 0;
    PSFD_CUDA_TRY(cudaMalloc((void**)&P->G, need * sizeof(cf)));
    P->G_elems = need;
  }
  P->fill = fill;
  // sources
  double* ftab = nullptr;
  PSFD_CUDA_TRY(cudaMallocAsync((void**)&ftab, (size_t)P->nz * 6 * sizeof(double), s));
  for (int r = 0; r < P->nrhs; ++r) {
    SourceArgs a;
    a.fill = fill; a.b = (cf*)b + (long)r * P->nvec;
    a.nx = P->nx; a.ny = P->ny; a.nz = P->nz; a.z_ml = P->p.z_ml; a.ncols = nm;
    a.dz = P->p.dz; a.k0 = P->k0;
    a.theta = P->p.theta_deg * M_PI / 180.0; a.phi = P->p.phi_deg * M_PI / 180.0;
    a.pc64 = P->pc64;
    a.rs64 = P->R.rs64; a.rp64 = P->R.rp64; a.kz064 = P->R.kz064;
    a.pol = pol[r];
    k_source_z<<<(unsigned)((P->nz + 127) / 128), 128, 0, s>>>(a, ftab);
    PSFD_CHECK_LAUNCH();
    dim3 grid((unsigned)((nm + 255) / 256), (unsigned)P->nz);
    k_source<<<grid, 256, 0, s>>>(a, ftab);
    PSFD_CHECK_LAUNCH();
  }
  PSFD_CUDA_TRY(cudaFreeAsync(ftab, s));
  P->have_background = true;
  return PSFD_OK;
}

extern "C" int psfd_set_plane_contrast(psfd_plan P, const double* re, const double* im) {
  if (!P) { psfd_set_error("psfd_set_plane_contrast: null plan"); return PSFD_ERR_ARG; }
  if ((re == nullptr) != (im == nullptr)) {
    psfd_set_error("psfd_set_plane_contrast: give both re and im, or neither");
    return PSFD_ERR_ARG;
  }
  for (int z = 0; z < P->nz; ++z) {
    P->pc_host[z] = re ? make_double2(re[z], im[z]) : make_double2(P->deps_re, P->deps_im);
    if (!std::isfinite(P->pc_host[z].x) || !std::isfinite(P->pc_host[z].y)) {
      psfd_set_error("psfd_set_plane_contrast: non-finite entry at plane %d", z);
      return PSFD_ERR_ARG;
    }
  }
  PSFD_CUDA_TRY(cudaStreamSynchronize(P->stream));
  PSFD_CUDA_TRY(cudaMemcpy(P->pc64, P->pc_host.data(), P->nz * sizeof(zd), cudaMemcpyHostToDevice));
  int rc = upload_pc32(P);
  if (rc) return rc;
  P->have_background = false;   // b and the registered fill must be set again with psfd_background
  return PSFD_OK;
}

extern "C" int psfd_set_layer_stack_contrast(psfd_plan P, const psfd_stack_t* layers, double z_top, float* zmask) {
  if (!P || !layers) { psfd_set_error("psfd_set_layer_stack_contrast: null argument"); return PSFD_ERR_ARG; }
  if (layers->n_layers < 0 || (layers->n_layers > 0 && (!layers->n_re || !layers->n_im || !layers->d))) {
    psfd_set_error("psfd_set_layer_stack_contrast: bad stack");
    return PSFD_ERR_ARG;
  }
  // layer k occupies [top_k - d_k, top_k] (top to bottom from z_top), the substrate everything
  // below, vacuum everything above; cell z covers [z dz - dz/2, z dz + dz/2]
  struct Slab { double top, bot; std::complex<double> eps; };
  std::vector<Slab> slabs;
  double zc = z_top;
  for (int l = 0; l < layers->n_layers; ++l) {
    const std::complex<double> n(layers->n_re[l], layers->n_im[l]);
    slabs.push_back({zc, zc - layers->d[l], n * n});
    zc -= layers->d[l];
  }
  const std::complex<double> ns(layers->sub_re, layers->sub_im);
  slabs.push_back({zc, -1e300, ns * ns});
  const double dz = P->p.dz;
  std::vector<double> re(P->nz), im(P->nz);
  for (int z = 0; z < P->nz; ++z) {
    const double lo = z * dz - 0.5 * dz, hi = z * dz + 0.5 * dz;
    std::complex<double> acc(0.0, 0.0);
    for (const Slab& s : slabs) {
      const double ov = std::max(0.0, std::min(hi, s.top) - std::max(lo, s.bot));
      acc += ov * (s.eps - 1.0);
    }
    acc /= dz;
    re[z] = acc.real();
    im[z] = acc.imag();
    if (zmask) zmask[z] = (acc != std::complex<double>(0.0, 0.0)) ? 1.f : 0.f;
  }
  return psfd_set_plane_contrast(P, re.data(), im.data());
}

extern "C" int psfd_reflection_tables(psfd_plan P, double* rs, double* rp, double* kz0) {
  if (!P || !P->have_background) { psfd_set_error("psfd_reflection_tables: no background yet"); return PSFD_ERR_STATE; }
  size_t bytes = (size_t)P->ncols * 16;
  PSFD_CUDA_TRY(cudaStreamSynchronize(P->stream));
  if (rs) PSFD_CUDA_TRY(cudaMemcpy(rs, P->R.rs64, bytes, cudaMemcpyDeviceToHost));
  if (rp) PSFD_CUDA_TRY(cudaMemcpy(rp, P->R.rp64, bytes, cudaMemcpyDeviceToHost));
  if (kz0) PSFD_CUDA_TRY(cudaMemcpy(kz0, P->R.kz064, bytes, cudaMemcpyDeviceToHost));
  return PSFD_OK;
}
