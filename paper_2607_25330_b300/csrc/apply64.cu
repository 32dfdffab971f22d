// Extended-precision operator apply for the outer residual of the mixed-precision solve.
//
// A complex64 field cannot represent the solution to much better than a
// relative residual of ~1e-6 (rounding the exact FP64 solution to complex64
// already leaves 5e-7..8e-7 on the 32x32x16 and 32x32x32 cases), so the solver
// refines: complex64 inner Krylov solves of A M d = r, and an FP64 field
// E <- E + M d whose residual r = b - A E is computed here.  Same operator as
// apply.cu (A = curl_s curl_s - k0^2 - k0^2 deps (I + R), Sec. 2.2).  Fields and
// tables are FP64 in memory; the transforms and products run in double-float
// arithmetic (ff.cuh, about 48 bits, on the FP32 units: B300's FP64 rate is a
// small fraction of its FP32 rate), and the per-column reflection terms in FP64.
#include <cmath>
#include <vector>

#include "ff.cuh"
#include "fft.cuh"
#include "internal.h"
#include "pdl.cuh"

namespace {

struct Ax64 {
  const zd* x;
  zd* y;
  zd* G;
  const double* kx;
  const double* ky;
  const ff* kzf;      // [nz] wavenumbers, double-float, and FP64
  const double* kz;
  const cff* sinvf;   // [nz] PML stretch 1/s
  const zd* sinv;
  const double* sback;  // [nz] loss sigma_b(z) of the PML backing (eps_bg = 1 + i sigma_b)
  const cff* twf;     // [nz] twiddles
  const zd* tw;
  const double2* rs;
  const double2* rp;
  const double2* kz0;
  int nx;
  long ncols, vstride, gstride;
  int z_ml, za0, za1;
  double dz, k02;
};

// Same job structure as k_axial (mode A): jobs 0, 1, 3 copy the input.
template <int NZ, int T, class C>
__global__ void __launch_bounds__(64) k_axial64(Ax64 a) {
  pdl_enter();
  constexpr int P = 32 / T;
  constexpr int R = NZ / T;
  using PZ = Pencil<NZ, T, P, C>;
  using RT = typename CTraits<C>::R;
  const RT* kzt = pick_real<C>(a.kzf, a.kz);
  const C* sinv = pick_tab<C>(a.sinvf, a.sinv);
  const C* tw = pick_tab<C>(a.twf, a.tw);
  extern __shared__ zd smem64[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int t = lane / P, p = lane - t * P;
  const int rhs = blockIdx.y;
  const long col = ((long)blockIdx.x * (blockDim.x >> 5) + warp) * P + p;
  const bool act = col < a.ncols;
  const long cc = act ? col : 0;
  const long nc = a.ncols;
  const zd* __restrict__ x = a.x + rhs * a.vstride;
  zd* __restrict__ y = a.y + rhs * a.vstride;
  const double kx = a.kx[cc % a.nx], ky = a.ky[cc / a.nx];
  const RT inv_n(1.0 / (double)NZ), k02(a.k02), zero(0.0);
  const C ikx = CTraits<C>::make(zero, RT(kx)), iky = CTraits<C>::make(zero, RT(ky));
  C* st = reinterpret_cast<C*>(smem64) + (size_t)warp * 4 * R * 32;
  auto unst = [&](int sl, int m) -> C { return st[(sl * R + m) * 32 + lane]; };
  auto stash = [&](int sl, int m, C v) { st[(sl * R + m) * 32 + lane] = v; };
#pragma unroll 1
  for (int job = 0; job < 7; ++job) {
    const bool copy_only = (job == 0 || job == 1 || job == 3);
    C v[R];
    if (job < 5) {
      const int c = (job == 0) ? 2 : (job <= 2 ? 1 : 0);
      const zd* src = x + (long)(c * NZ + t) * nc + col;
#pragma unroll
      for (int m = 0; m < R; ++m) v[m] = act ? from_zd<C>(src[(long)(T * m) * nc]) : CTraits<C>::zero();
    } else {
      const int sl = (job == 5) ? 2 : 0;
#pragma unroll
      for (int m = 0; m < R; ++m) v[m] = unst(sl, m);
    }
    if (!copy_only) {
      PZ::template to_freq<false>(v, t, tw);
#pragma unroll
      for (int s = 0; s < R; ++s) {
        const RT kzv = kzt[PZ::freq_index(t, s)] * inv_n;
        v[s] = CTraits<C>::make(-(kzv * v[s].y), kzv * v[s].x);
      }
      PZ::template to_time<true>(v, t, tw);
    }
    if (copy_only) {
      const int sl = (job == 0) ? 0 : (job == 1 ? 1 : 3);
#pragma unroll
      for (int m = 0; m < R; ++m) stash(sl, m, v[m]);
    } else if (job == 2) {
#pragma unroll
      for (int m = 0; m < R; ++m) stash(2, m, csub(cmul(iky, unst(0, m)), cmul(v[m], sinv[t + T * m])));
    } else if (job == 4) {
#pragma unroll
      for (int m = 0; m < R; ++m) v[m] = csub(cmul(v[m], sinv[t + T * m]), cmul(ikx, unst(0, m)));
      __syncwarp();
      // reflection of the field at z_ml (Sec. 2.2): per column, in FP64
      const int tml = a.z_ml % T, mml = a.z_ml / T;
      const zd exm = to_zd(st[(3 * R + mml) * 32 + tml * P + p]);
      const zd eym = to_zd(st[(1 * R + mml) * 32 + tml * P + p]);
      const zd rs = a.rs[cc], rp = a.rp[cc], kz0 = a.kz0[cc];
      const double kp = sqrt(kx * kx + ky * ky);
      double sx, sy, tx, ty;
      if (kp > 0.0) { sx = -ky / kp; sy = kx / kp; tx = kx / kp; ty = ky / kp; }
      else { sx = 0.0; sy = 1.0; tx = 1.0; ty = 0.0; }
      const zd as = make_double2(sx * exm.x + sy * eym.x, sx * exm.y + sy * eym.y);
      const zd at = make_double2(tx * exm.x + ty * eym.x, tx * exm.y + ty * eym.y);
      const zd ras = cmul(rs, as), rat = cmul(rp, at);
      const zd r0 = make_double2(ras.x * sx + rat.x * tx, ras.y * sx + rat.y * tx);
      const zd r1 = make_double2(ras.x * sy + rat.x * ty, ras.y * sy + rat.y * ty);
      const zd num = make_double2(-(kx * r0.x + ky * r1.x), -(kx * r0.y + ky * r1.y));
      const double kd = kz0.x * kz0.x + kz0.y * kz0.y;
      const zd r2 = make_double2((num.x * kz0.x + num.y * kz0.y) / kd, (num.y * kz0.x - num.x * kz0.y) / kd);
      const C r0c = from_zd<C>(r0), r1c = from_zd<C>(r1), r2c = from_zd<C>(r2);
      const int nab = a.za1 - a.za0;
      zd* __restrict__ G = a.G + rhs * a.gstride;
#pragma unroll
      for (int m = 0; m < R; ++m) {
        const int z = t + T * m;
        const C qz = unst(0, m), cx = unst(2, m), cy = v[m];
        const C Wz = csub(csub(csub(cmul(ikx, cy), cmul(iky, cx)), cscale(qz, k02)),
                          ctimesi(cscale(qz, k02 * RT(a.sback[z]))));
        if (act) y[(long)(2 * NZ + z) * nc + col] = to_zd(Wz);
        if (z >= a.za0 && z < a.za1 && act) {
          zd prof = make_double2(0.0, 0.0);
          if (z >= a.z_ml) {
            const double zr = (double)(z - a.z_ml) * a.dz;
            double sn, cs;
            sincos(kz0.x * zr, &sn, &cs);
            const double mag = exp(-kz0.y * zr);
            prof = make_double2(mag * cs, mag * sn);
          }
          const C pc = from_zd<C>(prof);
          const long o = (long)(z - a.za0) * nc + col;
          G[o] = to_zd(cfma(r0c, pc, unst(3, m)));
          G[(long)nab * nc + o] = to_zd(cfma(r1c, pc, unst(1, m)));
          G[2L * nab * nc + o] = to_zd(cfma(r2c, pc, qz));
        }
      }
#pragma unroll
      for (int m = 0; m < R; ++m) stash(0, m, v[m]);
    } else {
      const int c = (job == 5) ? 1 : 0;
#pragma unroll
      for (int m = 0; m < R; ++m) {
        const C d = cmul(v[m], sinv[t + T * m]);
        const C qx = unst(3, m), qy = unst(1, m);
        const C cz = csub(cmul(ikx, qy), cmul(iky, qx));
        const C q = (job == 5) ? qy : qx;
        const C W0 = (job == 5) ? csub(csub(d, cmul(ikx, cz)), cscale(qy, k02))
                                : csub(csub(cmul(iky, cz), d), cscale(qx, k02));
        const C W = csub(W0, ctimesi(cscale(q, k02 * RT(a.sback[t + T * m]))));
        if (act) y[(long)(c * NZ + t + T * m) * nc + col] = to_zd(W);
      }
    }
  }
}

// ---------------------------------------------------------------- FP64 lateral passes
enum { R64_FWD = 0, R64_INV = 1, R64_FWD_SUB = 2 };
struct Row64 {
  zd* buf;
  long nrows;
  double scale;
  const cff* twf;   // twiddles, double-float and FP64
  const zd* tw;
  zd* y;
  int ny, nz, nab, za0;
  const int* plane_nz;   // nullable (forward transforms): planes flagged 0 are zero and are skipped
};

template <int NX, int T, int OP, class C>
__global__ void __launch_bounds__(64) k_rows64(Row64 a) {
  pdl_enter();
  constexpr int P = 32 / T, R = NX / T;
  using PX = Pencil<NX, T, 1, C>;
  using RT = typename CTraits<C>::R;
  const C* tw = pick_tab<C>(a.twf, a.tw);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int p = lane / T, t = lane - p * T;
  const long row = ((long)blockIdx.x * (blockDim.x >> 5) + warp) * P + p;
  const bool act = row < a.nrows;
  // a zero plane transforms to zero: a warp whose rows all lie in zero planes has nothing to do
  if (a.plane_nz && __all_sync(0xffffffffu, !act || !a.plane_nz[row / a.ny])) return;
  zd* src = a.buf + (act ? row : 0) * NX;
  const RT scale(a.scale);
  C v[R];
  if constexpr (OP == R64_INV) {
#pragma unroll
    for (int s = 0; s < R; ++s) v[s] = act ? from_zd<C>(src[PX::freq_index(t, s)]) : CTraits<C>::zero();
    PX::template to_time<true>(v, t, tw);
#pragma unroll
    for (int m = 0; m < R; ++m)
      if (act) src[t + T * m] = to_zd(cscale(v[m], scale));
  } else {
#pragma unroll
    for (int m = 0; m < R; ++m) v[m] = act ? from_zd<C>(src[t + T * m]) : CTraits<C>::zero();
    PX::template to_freq<false>(v, t, tw);
    if constexpr (OP == R64_FWD) {
#pragma unroll
      for (int s = 0; s < R; ++s)
        if (act) src[PX::freq_index(t, s)] = to_zd(cscale(v[s], scale));
    } else {
      const long per_c = (long)a.nab * a.ny;
      const long r = act ? row : 0;
      const long rhs = r / (3 * per_c), rem = r - rhs * 3 * per_c;
      const long c = rem / per_c, rem2 = rem - c * per_c;
      const long zz = rem2 / a.ny, iy = rem2 - zz * a.ny;
      zd* dst = a.y + (((rhs * 3 + c) * a.nz + a.za0 + zz) * a.ny + iy) * NX;
#pragma unroll
      for (int s = 0; s < R; ++s)
        if (act) {
          const int k = PX::freq_index(t, s);
          dst[k] = csub(dst[k], to_zd(v[s]));
        }
    }
  }
}

enum { C64_FWD = 0, C64_INV = 1, C64_CONTRAST = 2 };
struct Col64 {
  zd* buf;
  long ncolumns;
  int nx;
  double scale;
  const cff* twf;   // twiddles, double-float and FP64
  const zd* tw;
  const float* fill;
  const zd* pc;   // per-plane contrast; multiplier cs * c[z]
  double cs;
  int nab, za0;
  const int* plane_nz;   // nullable (forward transforms): planes flagged 0 are zero and are skipped
  long plane_elems;
};

template <int NY, int T, int OP, class C>
__global__ void __launch_bounds__(64) k_cols64(Col64 a) {
  pdl_enter();
  constexpr int P = 32 / T, R = NY / T;
  using PY = Pencil<NY, T, P, C>;
  using RT = typename CTraits<C>::R;
  const C* tw = pick_tab<C>(a.twf, a.tw);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int t = lane / P, p = lane - t * P;
  const long colid = ((long)blockIdx.x * (blockDim.x >> 5) + warp) * P + p;
  const bool act = colid < a.ncolumns;
  const long cid = act ? colid : 0;
  const long plane = cid / a.nx;
  if (a.plane_nz && __all_sync(0xffffffffu, !act || !a.plane_nz[plane])) return;   // zero planes stay zero
  const int ix = (int)(cid - plane * a.nx);
  zd* base = a.buf + plane * a.plane_elems + ix;
  const long sx = a.nx;
  const RT scale(a.scale);
  C v[R];
  if constexpr (OP == C64_FWD) {
#pragma unroll
    for (int m = 0; m < R; ++m) v[m] = act ? from_zd<C>(base[(long)(t + T * m) * sx]) : CTraits<C>::zero();
    PY::template to_freq<false>(v, t, tw);
#pragma unroll
    for (int s = 0; s < R; ++s)
      if (act) base[(long)PY::freq_index(t, s) * sx] = to_zd(cscale(v[s], scale));
  } else if constexpr (OP == C64_INV) {
#pragma unroll
    for (int s = 0; s < R; ++s) v[s] = act ? from_zd<C>(base[(long)PY::freq_index(t, s) * sx]) : CTraits<C>::zero();
    PY::template to_time<true>(v, t, tw);
#pragma unroll
    for (int m = 0; m < R; ++m)
      if (act) base[(long)(t + T * m) * sx] = to_zd(cscale(v[m], scale));
  } else {
    const long zz = plane % a.nab;
    const float* f = a.fill + (a.za0 + zz) * a.plane_elems + ix;
    const zd c0 = a.pc[a.za0 + zz];
    const RT dre(a.cs * c0.x), dim(a.cs * c0.y);
#pragma unroll
    for (int s = 0; s < R; ++s) v[s] = act ? from_zd<C>(base[(long)PY::freq_index(t, s) * sx]) : CTraits<C>::zero();
    PY::template to_time<true>(v, t, tw);
#pragma unroll
    for (int m = 0; m < R; ++m) {
      const RT fv((double)(act ? f[(long)(t + T * m) * sx] : 0.f));   // the fill is a float: exact
      v[m] = cmul(v[m], CTraits<C>::make(dre * fv, dim * fv));
    }
    PY::template to_freq<false>(v, t, tw);
#pragma unroll
    for (int s = 0; s < R; ++s)
      if (act) base[(long)PY::freq_index(t, s) * sx] = to_zd(v[s]);
  }
}

template <int NX, int T>
int rows64_op(const Row64& a, int op, cudaStream_t s) {
  const int warps = 2;
  const long per = warps * (32 / T);
  dim3 g((unsigned)((a.nrows + per - 1) / per));
  if (!g.x) return PSFD_OK;
  using C = ExtC<NX, T>;
  if (op == R64_FWD) (void)launch_pdl(k_rows64<NX, T, R64_FWD, C>, dim3(g), dim3(warps * 32), 0, s, a);
  else if (op == R64_INV) (void)launch_pdl(k_rows64<NX, T, R64_INV, C>, dim3(g), dim3(warps * 32), 0, s, a);
  else (void)launch_pdl(k_rows64<NX, T, R64_FWD_SUB, C>, dim3(g), dim3(warps * 32), 0, s, a);
  PSFD_CHECK_LAUNCH();
  return PSFD_OK;
}
int rows64(int nx, const Row64& a, int op, cudaStream_t s) {
  switch (nx) {
    case 16: return rows64_op<16, 4>(a, op, s);
    case 32: return rows64_op<32, 4>(a, op, s);
    case 64: return rows64_op<64, 8>(a, op, s);
    case 96: return rows64_op<96, 4>(a, op, s);
    case 128: return rows64_op<128, 8>(a, op, s);
    case 256: return rows64_op<256, 16>(a, op, s);
    case 512: return rows64_op<512, 16>(a, op, s);
  }
  psfd_set_error("rows64: unsupported %d", nx);
  return PSFD_ERR_ARG;
}
template <int NY, int T>
int cols64_op(const Col64& a, int op, cudaStream_t s) {
  const int warps = 2;
  const long per = warps * (32 / T);
  dim3 g((unsigned)((a.ncolumns + per - 1) / per));
  if (!g.x) return PSFD_OK;
  using C = ExtC<NY, T>;
  if (op == C64_FWD) (void)launch_pdl(k_cols64<NY, T, C64_FWD, C>, dim3(g), dim3(warps * 32), 0, s, a);
  else if (op == C64_INV) (void)launch_pdl(k_cols64<NY, T, C64_INV, C>, dim3(g), dim3(warps * 32), 0, s, a);
  else (void)launch_pdl(k_cols64<NY, T, C64_CONTRAST, C>, dim3(g), dim3(warps * 32), 0, s, a);
  PSFD_CHECK_LAUNCH();
  return PSFD_OK;
}
int cols64(int ny, const Col64& a, int op, cudaStream_t s) {
  switch (ny) {
    case 16: return cols64_op<16, 2>(a, op, s);
    case 32: return cols64_op<32, 4>(a, op, s);
    case 64: return cols64_op<64, 4>(a, op, s);
    case 96: return cols64_op<96, 4>(a, op, s);
    case 128: return cols64_op<128, 8>(a, op, s);
    case 256: return cols64_op<256, 8>(a, op, s);
    case 512: return cols64_op<512, 16>(a, op, s);
  }
  psfd_set_error("cols64: unsupported %d", ny);
  return PSFD_ERR_ARG;
}

template <int NZ, int T>
int axial64_run(psfd_plan_s* P, const zd* x, zd* y) {
  constexpr int R = NZ / T;
  Ax64 a;
  a.x = x; a.y = y; a.G = P->F.G;
  a.kx = P->F.kx; a.ky = P->F.ky;
  a.kz = P->F.kz; a.kzf = reinterpret_cast<const ff*>(P->F.kz_f);
  a.sinv = P->F.sinv; a.sinvf = reinterpret_cast<const cff*>(P->F.sinv_f);
  a.tw = P->F.twz; a.twf = reinterpret_cast<const cff*>(P->F.twz_f);
  a.rs = P->R.rs64; a.rp = P->R.rp64; a.kz0 = P->R.kz064;
  a.nx = P->nx; a.ncols = P->ncols; a.vstride = P->nvec;
  a.gstride = 3L * (P->za1 - P->za0) * P->ncols;
  a.z_ml = P->p.z_ml; a.za0 = P->za0; a.za1 = P->za1;
  a.dz = P->p.dz; a.k02 = P->k0 * P->k0; a.sback = P->F.sback;
  const int warps = 2;
  const long per = warps * (32 / T);
  dim3 g((unsigned)((P->ncols + per - 1) / per), (unsigned)P->nrhs);
  const size_t smem = (size_t)warps * 4 * R * 32 * sizeof(zd);
  using C = ExtC<NZ, T>;
  if (smem > 48 * 1024) cudaFuncSetAttribute(k_axial64<NZ, T, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  (void)launch_pdl(k_axial64<NZ, T, C>, dim3(g), dim3(warps * 32), smem, P->stream, a);
  PSFD_CHECK_LAUNCH();
  return PSFD_OK;
}

void host_tw64(int n, std::vector<zd>& out) {
  out.resize(n);
  for (int m = 0; m < n; ++m) {
    const double ang = -2.0 * M_PI * (double)m / (double)n;
    out[m] = make_double2(cos(ang), sin(ang));
  }
}

// FP64 values as double-float pairs (hi = nearest float, lo = nearest float to the remainder)
void split_ff(const double* d, size_t n, std::vector<float>& out) {
  out.resize(2 * n);
  for (size_t i = 0; i < n; ++i) {
    const float hi = (float)d[i];
    out[2 * i] = hi;
    out[2 * i + 1] = (float)(d[i] - (double)hi);
  }
}

double host_k(int i, int n, double d) {
  const int m = (i <= (n - 1) / 2) ? i : i - n;
  return 2.0 * M_PI * m / (n * d);
}

}  // namespace

// Build the FP64 tables and scratch on first use (plan-owned, freed with the plan).
int fp64_prepare(psfd_plan_s* P) {
  Fp64Tables& F = P->F;
  const size_t nab = (size_t)(P->za1 - P->za0);
  const size_t gneed = (size_t)P->nrhs * 3 * nab * P->ncols;
  if (F.kx && F.G_elems >= gneed) return PSFD_OK;
  if (!F.kx) {
    std::vector<double> kx(P->nx), ky(P->ny), kz(P->nz);
    for (int i = 0; i < P->nx; ++i) kx[i] = host_k(i, P->nx, P->p.dx) + P->kx_inc;
    for (int i = 0; i < P->ny; ++i) ky[i] = host_k(i, P->ny, P->p.dy) + P->ky_inc;
    for (int i = 0; i < P->nz; ++i) kz[i] = host_k(i, P->nz, P->p.dz);
    std::vector<zd> sinv, twx, twy, twz;
    pml_sinv64(P, sinv);
    host_tw64(P->nx, twx); host_tw64(P->ny, twy); host_tw64(P->nz, twz);
    PSFD_CUDA_TRY(cudaMalloc((void**)&F.plane_nz, (size_t)P->nrhs * 3 * P->nz * sizeof(int)));
    PSFD_CUDA_TRY(cudaMalloc((void**)&F.kx, P->nx * 8));
    PSFD_CUDA_TRY(cudaMalloc((void**)&F.ky, P->ny * 8));
    PSFD_CUDA_TRY(cudaMalloc((void**)&F.kz, P->nz * 8));
    PSFD_CUDA_TRY(cudaMalloc((void**)&F.sinv, P->nz * 16));
    PSFD_CUDA_TRY(cudaMalloc((void**)&F.sback, P->nz * 8));
    PSFD_CUDA_TRY(cudaMemcpy(F.sback, P->sback_host.data(), P->nz * 8, cudaMemcpyHostToDevice));
    PSFD_CUDA_TRY(cudaMalloc((void**)&F.twx, P->nx * 16));
    PSFD_CUDA_TRY(cudaMalloc((void**)&F.twy, P->ny * 16));
    PSFD_CUDA_TRY(cudaMalloc((void**)&F.twz, P->nz * 16));
    PSFD_CUDA_TRY(cudaMemcpy(F.kx, kx.data(), P->nx * 8, cudaMemcpyHostToDevice));
    PSFD_CUDA_TRY(cudaMemcpy(F.ky, ky.data(), P->ny * 8, cudaMemcpyHostToDevice));
    PSFD_CUDA_TRY(cudaMemcpy(F.kz, kz.data(), P->nz * 8, cudaMemcpyHostToDevice));
    PSFD_CUDA_TRY(cudaMemcpy(F.sinv, sinv.data(), P->nz * 16, cudaMemcpyHostToDevice));
    PSFD_CUDA_TRY(cudaMemcpy(F.twx, twx.data(), P->nx * 16, cudaMemcpyHostToDevice));
    PSFD_CUDA_TRY(cudaMemcpy(F.twy, twy.data(), P->ny * 16, cudaMemcpyHostToDevice));
    PSFD_CUDA_TRY(cudaMemcpy(F.twz, twz.data(), P->nz * 16, cudaMemcpyHostToDevice));
    // double-float copies for the transforms and products
    std::vector<float> f;
    struct T2 { const double* src; size_t n; float** dst; };
    const T2 tabs[] = {{kz.data(), (size_t)P->nz, &F.kz_f},
                       {reinterpret_cast<const double*>(sinv.data()), 2 * (size_t)P->nz, &F.sinv_f},
                       {reinterpret_cast<const double*>(twx.data()), 2 * (size_t)P->nx, &F.twx_f},
                       {reinterpret_cast<const double*>(twy.data()), 2 * (size_t)P->ny, &F.twy_f},
                       {reinterpret_cast<const double*>(twz.data()), 2 * (size_t)P->nz, &F.twz_f}};
    for (const T2& tb : tabs) {
      split_ff(tb.src, tb.n, f);
      PSFD_CUDA_TRY(cudaMalloc((void**)tb.dst, f.size() * sizeof(float)));
      PSFD_CUDA_TRY(cudaMemcpy(*tb.dst, f.data(), f.size() * sizeof(float), cudaMemcpyHostToDevice));
    }
  }
  if (F.G_elems < gneed) {
    if (F.G) cudaFree(F.G);
    F.G = nullptr;
    F.G_elems = 0;
    if (gneed) PSFD_CUDA_TRY(cudaMalloc((void**)&F.G, gneed * sizeof(zd)));
    F.G_elems = gneed;
  }
  return PSFD_OK;
}

// flags[q] = 1 if plane q of a (nplanes planes of ncols complex64 entries) has a nonzero (or NaN)
// entry, else 0
__global__ void k_plane_any(const cf* __restrict__ a, long plane_elems, int* flags) {
  const cf* p = a + (long)blockIdx.x * plane_elems;
  int any = 0;
  for (long i = threadIdx.x; i < plane_elems; i += blockDim.x) {
    const cf v = p[i];
    any |= (v.x != 0.f) || (v.y != 0.f);
  }
  any = __syncthreads_or(any);
  if (threadIdx.x == 0) flags[blockIdx.x] = any;
}

int plane_flags(psfd_plan_s* P, const cf* a, long nplanes, int* flags) {
  k_plane_any<<<(unsigned)nplanes, 256, 0, P->stream>>>(a, P->ncols, flags);
  PSFD_CHECK_LAUNCH();
  return PSFD_OK;
}

void fp64_free(psfd_plan_s* P) {
  Fp64Tables& F = P->F;
  void* ptrs[] = {F.kx, F.ky, F.kz, F.sinv, F.sback, F.twx, F.twy, F.twz, F.G, F.X, F.kz_f, F.sinv_f, F.twx_f, F.twy_f, F.twz_f,
                  F.plane_nz};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  F = Fp64Tables();
}

// y = A x in FP64, HYBRID domain (no preconditioner)
int apply64_hybrid(psfd_plan_s* P, const zd* x, zd* y) {
  int rc;
  {
    StageScope sc(P->stream, ST_AXIAL);
    switch (P->nz) {
      case 16: rc = axial64_run<16, 2>(P, x, y); break;
      case 32: rc = axial64_run<32, 4>(P, x, y); break;
      case 48: rc = axial64_run<48, 4>(P, x, y); break;
      case 64: rc = axial64_run<64, 8>(P, x, y); break;
      case 96: rc = axial64_run<96, 4>(P, x, y); break;
      case 128: rc = axial64_run<128, 8>(P, x, y); break;
      case 256: rc = axial64_run<256, 16>(P, x, y); break;
      case 512: rc = axial64_run<512, 16>(P, x, y); break;
      case 1024: rc = axial64_run<1024, 32>(P, x, y); break;
      default: psfd_set_error("apply64: nz %d", P->nz); return PSFD_ERR_ARG;
    }
    if (rc) return rc;
  }
  const int nab = P->za1 - P->za0;
  if (nab <= 0) return PSFD_OK;
  StageScope sc(P->stream, ST_CONTRAST);
  const long nplanes = (long)P->nrhs * 3 * nab;
  Row64 r{};
  r.buf = P->F.G; r.nrows = nplanes * P->ny; r.scale = 1.0; r.tw = P->F.twx; r.twf = reinterpret_cast<const cff*>(P->F.twx_f);
  if ((rc = rows64(P->nx, r, R64_INV, P->stream))) return rc;
  Col64 c{};
  const double scl = P->k0 * P->k0 / (double)P->ncols;
  c.buf = P->F.G; c.ncolumns = nplanes * P->nx; c.nx = P->nx; c.scale = 1.0;
  c.tw = P->F.twy; c.twf = reinterpret_cast<const cff*>(P->F.twy_f);
  c.fill = P->fill; c.pc = P->pc64; c.cs = scl; c.nab = nab; c.za0 = P->za0;
  c.plane_elems = P->ncols;
  if ((rc = cols64(P->ny, c, C64_CONTRAST, P->stream))) return rc;
  Row64 w{};
  w.buf = P->F.G; w.nrows = nplanes * P->ny; w.tw = P->F.twx; w.twf = reinterpret_cast<const cff*>(P->F.twx_f); w.y = y;
  w.ny = P->ny; w.nz = P->nz; w.nab = nab; w.za0 = P->za0;
  return rows64(P->nx, w, R64_FWD_SUB, P->stream);
}

// real space <-> HYBRID in FP64 over nplanes planes (unitary scale applied once)
int transform64(psfd_plan_s* P, zd* buf, long nplanes, bool forward, double scale, const int* plane_nz) {
  StageScope sc(P->stream, ST_TRANSFORM);
  int rc;
  Row64 r{};
  r.buf = buf; r.nrows = nplanes * P->ny; r.tw = P->F.twx; r.twf = reinterpret_cast<const cff*>(P->F.twx_f);
  r.ny = P->ny; r.plane_nz = forward ? plane_nz : nullptr;
  Col64 c{};
  c.buf = buf; c.ncolumns = nplanes * P->nx; c.nx = P->nx; c.tw = P->F.twy; c.twf = reinterpret_cast<const cff*>(P->F.twy_f);
  c.plane_elems = P->ncols; c.plane_nz = forward ? plane_nz : nullptr;
  if (forward) {
    r.scale = 1.0;
    if ((rc = rows64(P->nx, r, R64_FWD, P->stream))) return rc;
    c.scale = scale;
    return cols64(P->ny, c, C64_FWD, P->stream);
  }
  c.scale = 1.0;
  if ((rc = cols64(P->ny, c, C64_INV, P->stream))) return rc;
  r.scale = scale;
  return rows64(P->nx, r, R64_INV, P->stream);
}

// y = A x in FP64 through the C ABI (the operator of the refinement residual).
extern "C" int psfd_apply64(psfd_plan P, const double* x, double* y, int flags) {
  if (!P || !x || !y) { psfd_set_error("psfd_apply64: null argument"); return PSFD_ERR_ARG; }
  if (!P->have_background) { psfd_set_error("psfd_apply64: call psfd_background first"); return PSFD_ERR_STATE; }
  if ((const void*)x == (void*)y) { psfd_set_error("psfd_apply64: x and y must not overlap"); return PSFD_ERR_ARG; }
  if (flags & ~PSFD_HYBRID) { psfd_set_error("psfd_apply64: only PSFD_HYBRID is accepted"); return PSFD_ERR_ARG; }
  int rc = fp64_prepare(P);
  if (rc) return rc;
  const zd* xi = reinterpret_cast<const zd*>(x);
  zd* yo = reinterpret_cast<zd*>(y);
  if (flags & PSFD_HYBRID) return apply64_hybrid(P, xi, yo);
  const size_t n = (size_t)P->nrhs * P->nvec;
  if (!P->F.X) PSFD_CUDA_TRY(cudaMalloc((void**)&P->F.X, n * sizeof(zd)));
  PSFD_CUDA_TRY(cudaMemcpyAsync(P->F.X, xi, n * sizeof(zd), cudaMemcpyDeviceToDevice, P->stream));
  const double us = 1.0 / sqrt((double)P->ncols);
  const long nplanes = (long)P->nrhs * 3 * P->nz;
  if ((rc = transform64(P, P->F.X, nplanes, true, us))) return rc;
  if ((rc = apply64_hybrid(P, P->F.X, yo))) return rc;
  return transform64(P, yo, nplanes, false, us);
}
