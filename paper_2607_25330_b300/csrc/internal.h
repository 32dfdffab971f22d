// Host-side plan structure and internal launch interfaces shared by the .cu files.
#pragma once
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>
#include <vector>
#include "../../include/psfd.h"
#include "common.cuh"

struct ReflTables {
  double2* rs64 = nullptr;   // [ny*nx]
  double2* rp64 = nullptr;
  double2* kz064 = nullptr;
  float4* refl = nullptr;    // (rs.re, rs.im, rp.re, rp.im) per mode
  cf* kz0 = nullptr;         // kz0 per mode (float)
};

struct Fp64Tables {
  double* kx = nullptr;
  double* ky = nullptr;
  double* kz = nullptr;
  double2* sinv = nullptr;
  double* sback = nullptr;   // [nz] sigma_b(z) of the PML backing
  double2* twx = nullptr;
  double2* twy = nullptr;
  double2* twz = nullptr;
  double2* G = nullptr;
  size_t G_elems = 0;
  double2* X = nullptr;      // [nrhs][3][nz][ny][nx] input copy of the real-space psfd_apply64
  int* plane_nz = nullptr;   // [nrhs][3][nz] 1 where a plane of the refined solve's b is not zero
  // double-float (hi, lo) copies used by the extended-precision transforms
  float* kz_f = nullptr;
  float* sinv_f = nullptr;
  float* twx_f = nullptr;
  float* twy_f = nullptr;
  float* twz_f = nullptr;
};

struct psfd_plan_s {
  psfd_params_t p{};
  cudaStream_t stream = nullptr;
  int nx = 0, ny = 0, nz = 0, nrhs = 0;
  long ncols = 0;            // nx * ny
  long nvec = 0;             // 3 * nz * ncols (complex entries per right-hand side)
  double k0 = 0, kx_inc = 0, ky_inc = 0, kz_inc = 0;
  double deps_re = 0, deps_im = 0;  // eps_abs - 1 (default per-plane contrast)
  // per-plane material contrast c[z]: deps(x, y, z) = fill(x, y, z) * c[z]; defaults to eps_abs - 1
  cf* pc = nullptr;                  // [nz] complex64
  zd* pc64 = nullptr;                // [nz] FP64
  std::vector<zd> pc_host;
  // device tables
  float* kx = nullptr;       // [nx] Bloch-shifted lateral wavenumbers
  float* ky = nullptr;       // [ny]
  float* kz = nullptr;       // [nz] axial wavenumbers (FFT order)
  cf* sinv = nullptr;        // [nz] 1 / s(z)
  cf* kbg = nullptr;         // [nz] k0^2 eps_bg(z) = k0^2 (1 + i sigma_b(z)) (the PML backing)
  float* sback = nullptr;    // [nz] sigma_b(z)
  std::vector<double> sback_host;
  cf* tw_x = nullptr;        // [nx] exp(-2 pi i m / nx)
  cf* tw_y = nullptr;
  cf* tw_z = nullptr;
  ReflTables R;
  // geometry
  const float* fill = nullptr;
  int za0 = 0, za1 = 0;      // planes with nonzero fill: [za0, za1)
  bool have_background = false;
  std::vector<double> stack_sig;   // stack the reflection tables were computed for
  // damping
  float m_min = 0, kref2 = 0, gamma = 1, damp_eps = 0;
  // scratch (plan-owned)
  cf* G = nullptr;           // [nrhs][3][nab][ny][nx]
  size_t G_elems = 0;
  cf* tmpA = nullptr;        // [nrhs][3][nz][ny][nx]
  cf* tmpB = nullptr;        // [nrhs][3][nz][ny][nx]
  // history (host)
  double* hist = nullptr;
  int hist_cap = 0;
  // BiCGSTAB progress that the host reads without synchronising the stream: pinned, device-mapped
  // [2][nrhs] ints (iterations completed, done flag), written by the vector kernels
  int* prog_h = nullptr;
  int* prog_d = nullptr;
  // launch choices (set by the tuner)
  int axial_T = 0;
  // FP64 residual path (built on first refined solve)
  Fp64Tables F;
  // single-pass plane kernel: error word of its bounded waits; use_plane enables the kernel
  int* err = nullptr;
  bool use_plane = false;
  // layered-background preconditioner (per-column TE/TM inverses, built by psfd_layered_build)
  cf* lay = nullptr;         // [ncols][5 nz^2]
  cf* lay_D = nullptr;       // [nz][nz] stretched axial derivative
  cf* lay_DT = nullptr;      // [nz][nz] its transpose
  cf* lay_D2 = nullptr;      // [nz][nz]
  cf* lay_deps = nullptr;    // [nz] laterally averaged contrast
  int* lay_err = nullptr;
  double* lay_fmean = nullptr;          // [nz] device scratch for plane means
  void* lay16 = nullptr;                // half-precision blocks (storage PSFD_LAY_HALF)
  float* lay_scale = nullptr;           // their per-block power-of-two scales
  bool lay_half = false;
  bool lay_schur = false;               // blocks in the Schur form (TE^-1 and S^-1, 2 nz^2 per column)
  int lay_form = 0;                     // requested form: PSFD_LAY_FORM_AUTO or PSFD_LAY_FORM_SCHUR
  std::vector<double> lay_mean;         // plane means of the fill the blocks were built for
  bool lay_built = false;
};

// apply64.cu
int fp64_prepare(psfd_plan_s* P);
void fp64_free(psfd_plan_s* P);
int apply64_hybrid(psfd_plan_s* P, const double2* x, double2* y);
int transform64(psfd_plan_s* P, double2* buf, long nplanes, bool forward, double scale,
                const int* plane_nz = nullptr);
int plane_flags(psfd_plan_s* P, const cf* a, long nplanes, int* flags);

// apply.cu
int launch_axial(psfd_plan_s* P, const cf* x, cf* y, int mode, const int* done, int nrhs_active);
int launch_lateral_contrast(psfd_plan_s* P, cf* y, const int* done, bool adjoint);
int launch_lateral_transform(psfd_plan_s* P, cf* buf, long nplanes, bool forward, float scale);
int apply_hybrid(psfd_plan_s* P, const cf* x, cf* y, int flags, const int* done);
int launch_rows(int n, cf* buf, long nrows, bool forward, float scale, const cf* tw, cudaStream_t s);
int launch_cols(int n, int nx, cf* buf, long ncols_total, bool forward, float scale, const cf* tw,
                cudaStream_t s);
int launch_cols_gauss(int ny, int nx, cf* buf, float sigma, const cf* tw, cudaStream_t s);
int axial_supported(int nz);
int axial_candidates(int nz, int* out);
int lateral_supported(int n);

// plan.cu
void psfd_set_error(const char* fmt, ...);
double fft_wavenumber(int i, int n, double d);           // 2 pi m / (n d), FFT order, Nyquist negative
void pml_sinv64(const psfd_plan_s* P, std::vector<zd>& sinv);   // 1 / s(z) in FP64

// fno_tc.cu: forward per-mode mixing on the tensor cores (C = 32)
bool fno_mix_tc_enabled(int C);
int fno_mix_tc(const cf* V, cf* U, const cf* K, long NB, int modes, int mx, int MX, int offy, int offx,
               cudaStream_t s);
int fno_mix_tc_error(int* host_flag);   // reads and clears the flag
// fno_mlp_tc.cu: the pointwise MLP (C = 32, H = 64) and projection (Q = 128) on the tensor cores
bool fno_mlp_tc_enabled(int C, int H, int Q);
int fno_mlp_tc(const float* vin, float* vout, const float* uxy, const float* uz, const float* W1, const float* b1,
               const float* W2, const float* b2, long N, int B, bool outer_gelu, cudaStream_t s);
int fno_proj_tc(const float* v, cf* E, const float* Q1, const float* qb1, const float* Q2, const float* qb2, long N,
                int B, cudaStream_t s);
int fno_mlp_tc_error(int* host_flag);   // reads and clears the flag
int plan_wait_status(psfd_plan_s* P);   // PSFD_ERR_TIMEOUT if a bounded device wait gave up

// layered.cu
int layered_supported(const psfd_plan_s* P);
bool layered_pairs(const psfd_plan_s* P);
long layered_columns(const psfd_plan_s* P);
bool layered_schur_for(const psfd_plan_s* P);   // the block form a build of this plan uses
bool layered_half(const psfd_plan_s* P);        // half-precision blocks in effect
size_t layered_bytes(const psfd_plan_s* P);
// done (nullable, device [nrhs]): when every right-hand side is done the apply returns at once
int layered_apply(psfd_plan_s* P, const cf* x, cf* y, const int* done = nullptr);
void layered_free(psfd_plan_s* P);
