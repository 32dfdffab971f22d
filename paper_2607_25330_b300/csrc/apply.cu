// The PSFD operator apply (Sec. 2.2) on the device.
//
// Krylov vectors live in the HYBRID domain (kx, ky, z) (unitary lateral DFT).
// In that domain every term except the contrast is local to one (kx, ky)
// column: the spectral-damping preconditioner M (a 3-D Fourier multiplier:
// FFT_z, x m(k), IFFT_z), the stretched-coordinate curl-curl (i kx, i ky and
// D_z = s^-1 F_z^-1 i kz F_z), -k0^2 E and the multilayer reflection R
// (tangential field at z_ml -> r_s/r_p -> upgoing profile).  One fused kernel
// ("axial") does all of that per column and emits
//   W = curl_s curl_s q - k0^2 q           for every plane, into y
//   G = q + R q                            for the absorber planes, into scratch
// with q = M x (or x).  The contrast term is then added on the absorber planes
// only by three lateral passes: IFFT_x (rows), IFFT_y * k0^2 deps / N * FFT_y
// (columns), FFT_x with y -= result (rows).
#include <mutex>
#include <cstdio>

#include "fft.cuh"
#include "internal.h"
#include "pdl.cuh"

// ======================================================================= axial kernel
struct AxialArgs {
  const cf* x;
  cf* y;
  cf* G;
  const float* kx;
  const float* ky;
  const float* kz;
  const cf* sinv;
  const cf* kbg;    // [nz] k0^2 eps_bg(z)
  const cf* tw;
  const float4* refl;
  const cf* kz0;
  const int* done;
  int nx;
  long ncols, vstride, gstride;
  int z_ml, za0, za1;
  float dz, k02;
  float m_min, kref2, gamma, damp_eps;
};

enum { AX_AM = 0, AX_A = 1, AX_M = 2, AX_AH = 3 };

// k0^2 eps_bg(z) of the operator (its conjugate in the adjoint)
template <int MODE>
__device__ __forceinline__ cf kbg_at_(const AxialArgs& a, int z) {
  const cf v = __ldg(a.kbg + z);
  return MODE == AX_AH ? make_float2(v.x, -v.y) : v;
}
#define kbg_at(a, z) kbg_at_<MODE>(a, z)

// The column work is a loop over "jobs"; each job is
//   source (time layout) -> FFT_z -> one spectral factor -> IFFT_z -> post-op
// so that each transform direction is instantiated once (the fully inlined
// 12-transform body overflowed the instruction cache).  Jobs (q = M x):
//   0: x_z -> m/N          -> q_z                     -> slot 0
//   1: x_y -> m/N          -> q_y                     -> slot 1
//   2: x_y -> m i kz / N   -> D q_y  -> c_x = i ky q_z - D q_y       -> slot 2
//   3: x_x -> m/N          -> q_x                     -> slot 3
//   4: x_x -> m i kz / N   -> D q_x  -> c_y = D q_x - i kx q_z; emit W_z, G; c_y -> slot 0
//   5: c_x -> i kz / N     -> D c_x  -> W_y = D c_x - i kx c_z - k0^2 q_y
//   6: c_y -> i kz / N     -> D c_y  -> W_x = i ky c_z - D c_y - k0^2 q_x
// with D = s^-1 (.) applied after the inverse transform, c_z = i kx q_y - i ky q_x.
// Without M (mode A) jobs 0, 1, 3 copy the input.  Mode M runs jobs 0, 1, 3 only
// and writes q to y.  Mode AH applies the adjoint A^H x = curl~ curl~ x - k0^2 x
// - G - R^H G with D~ = F^-1 i kz F conj(s^-1) (the PML factor moves in front of
// the transform) and G = k0^2 F_xy[conj(deps) F_xy^-1 x] on the absorber planes,
// prepared by the contrast passes before this kernel; R^H G sums conj(profile) G
// over the column and is subtracted at z_ml.
template <int NZ, int T, int MODE>
__global__ void __launch_bounds__(128) k_axial(AxialArgs a) {
  pdl_enter();
  constexpr int P = 32 / T;
  constexpr int R = NZ / T;
  using PZ = Pencil<NZ, T, P>;
  extern __shared__ cf smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int t = lane / P, p = lane - t * P;
  const int rhs = blockIdx.y;
  if (a.done && a.done[rhs]) return;
  const long col = ((long)blockIdx.x * (blockDim.x >> 5) + warp) * P + p;
  const bool act = col < a.ncols;
  const long cc = act ? col : 0;
  const long nc = a.ncols;
  const cf* __restrict__ x = a.x + rhs * a.vstride;
  cf* __restrict__ y = a.y + rhs * a.vstride;
  const float kx = __ldg(a.kx + cc % a.nx), ky = __ldg(a.ky + cc / a.nx);
  const float inv_n = 1.0f / (float)NZ;
  const cf ikx = make_float2(0.f, kx), iky = make_float2(0.f, ky);
  cf* st = smem + (size_t)warp * 4 * R * 32;
  auto unst = [&](int sl, int m) -> cf { return st[(sl * R + m) * 32 + lane]; };
  auto stash = [&](int sl, int m, cf v) { st[(sl * R + m) * 32 + lane] = v; };

  // adjoint: (rh0, rh1) = T^H sum_z conj(profile(z)) G(z), the R^H term at z_ml
  cf rh0 = czero(), rh1 = czero();
  if constexpr (MODE == AX_AH) {
    const int nab = a.za1 - a.za0;
    const cf* __restrict__ G = a.G + rhs * a.gstride;
    const cf kz0 = __ldg(a.kz0 + cc);
    cf v0 = czero(), v1 = czero(), v2 = czero();
#pragma unroll
    for (int m = 0; m < R; ++m) {
      const int z = t + T * m;
      if (z >= a.za0 && z < a.za1 && z >= a.z_ml && act) {
        const float zr = (float)(z - a.z_ml) * a.dz;
        float sn, cs;
        sincosf(kz0.x * zr, &sn, &cs);
        const float mag = expf(-kz0.y * zr);
        const cf pc = make_float2(mag * cs, -mag * sn);     // conj(profile)
        const long o = (long)(z - a.za0) * nc + col;
        v0 = cfma(pc, G[o], v0);
        v1 = cfma(pc, G[(long)nab * nc + o], v1);
        v2 = cfma(pc, G[2L * nab * nc + o], v2);
      }
    }
#pragma unroll
    for (int b = 1; b < T; b <<= 1) {
      v0.x += __shfl_xor_sync(0xffffffffu, v0.x, b * P); v0.y += __shfl_xor_sync(0xffffffffu, v0.y, b * P);
      v1.x += __shfl_xor_sync(0xffffffffu, v1.x, b * P); v1.y += __shfl_xor_sync(0xffffffffu, v1.y, b * P);
      v2.x += __shfl_xor_sync(0xffffffffu, v2.x, b * P); v2.y += __shfl_xor_sync(0xffffffffu, v2.y, b * P);
    }
    const float4 rr = __ldg(a.refl + cc);
    const cf rs = make_float2(rr.x, rr.y), rp = make_float2(rr.z, rr.w);
    const float kp = sqrtf(kx * kx + ky * ky);
    float sx, sy, tx, ty;
    if (kp > 0.f) { sx = -ky / kp; sy = kx / kp; tx = kx / kp; ty = ky / kp; }
    else { sx = 0.f; sy = 1.f; tx = 1.f; ty = 0.f; }
    // T = [[rs sx sx + rp tx tx, rs sx sy + rp tx ty], [rs sy sx + rp ty tx, rs sy sy + rp ty ty],
    //      [-(kx T00 + ky T10)/kz0, -(kx T01 + ky T11)/kz0]];  e = T^H v
    const cf T00 = cfma(rs, make_float2(sx * sx, 0.f), cscale(rp, tx * tx));
    const cf T01 = cfma(rs, make_float2(sx * sy, 0.f), cscale(rp, tx * ty));
    const cf T10 = cfma(rs, make_float2(sy * sx, 0.f), cscale(rp, ty * tx));
    const cf T11 = cfma(rs, make_float2(sy * sy, 0.f), cscale(rp, ty * ty));
    const float kd = kz0.x * kz0.x + kz0.y * kz0.y;
    auto divkz = [&](cf n) { return make_float2((n.x * kz0.x + n.y * kz0.y) / kd, (n.y * kz0.x - n.x * kz0.y) / kd); };
    const cf T20 = divkz(make_float2(-(kx * T00.x + ky * T10.x), -(kx * T00.y + ky * T10.y)));
    const cf T21 = divkz(make_float2(-(kx * T01.x + ky * T11.x), -(kx * T01.y + ky * T11.y)));
    rh0 = cadd(cadd(cmulc(v0, T00), cmulc(v1, T10)), cmulc(v2, T20));   // conj(T_i0) v_i
    rh1 = cadd(cadd(cmulc(v0, T01), cmulc(v1, T11)), cmulc(v2, T21));
  }

  // modes A and A^H read the components z, y, y, x, x in jobs 0-4: load each once, all three
  // up front, so that their latencies overlap (where a thread holds at most 8 points of a pencil)
  constexpr bool PRE = (MODE == AX_A || MODE == AX_AH) && R <= 8;
  cf pre0[PRE ? R : 1], pre1[PRE ? R : 1], pre2[PRE ? R : 1];
  if constexpr (PRE) {
#pragma unroll
    for (int m = 0; m < R; ++m) {
      const long o = (long)(t + T * m) * nc + col;
      pre2[m] = act ? __ldg(x + 2L * NZ * nc + o) : czero();
      pre1[m] = act ? __ldg(x + (long)NZ * nc + o) : czero();
      pre0[m] = act ? __ldg(x + o) : czero();
    }
  }

#pragma unroll 1
  for (int job = 0; job < 7; ++job) {
    if (MODE == AX_M && (job == 2 || job >= 4)) continue;
    const bool copy_only = (MODE == AX_A || MODE == AX_AH) && (job == 0 || job == 1 || job == 3);
    cf v[R];
    // ---- source
    if (job < 5) {
      if constexpr (PRE) {
        if (job == 0) {
#pragma unroll
          for (int m = 0; m < R; ++m) v[m] = pre2[m];
        } else if (job <= 2) {
#pragma unroll
          for (int m = 0; m < R; ++m) v[m] = pre1[m];
        } else {
#pragma unroll
          for (int m = 0; m < R; ++m) v[m] = pre0[m];
        }
      } else {
        const int c = (job == 0) ? 2 : (job <= 2 ? 1 : 0);
        const cf* src = x + (long)(c * NZ + t) * nc + col;
#pragma unroll
        for (int m = 0; m < R; ++m) v[m] = act ? __ldg(src + (long)(T * m) * nc) : czero();
      }
    } else {
      const int sl = (job == 5) ? 2 : 0;
#pragma unroll
      for (int m = 0; m < R; ++m) v[m] = unst(sl, m);
    }
    if (MODE == AX_AH && (job == 2 || job >= 4)) {
#pragma unroll
      for (int m = 0; m < R; ++m) v[m] = cmulc(v[m], __ldg(a.sinv + t + T * m));   // v * conj(1/s)
    }
    // ---- spectral filter along z
    if (!copy_only) {
      PZ::template to_freq<false>(v, t, a.tw);
      const bool with_m = (MODE == AX_AM || MODE == AX_M) && job < 5;
      const bool with_d = (job == 2 || job >= 4);
#pragma unroll
      for (int s = 0; s < R; ++s) {
        const float kzv = __ldg(a.kz + PZ::freq_index(t, s));
        float f = inv_n;
        if (with_m) {
          const float k2 = fmaf(kx, kx, fmaf(ky, ky, kzv * kzv));
          float d = 1.0f;
          if (k2 > a.kref2) {
            const float ratio = a.kref2 / (k2 + a.damp_eps);
            d = (a.gamma == 1.0f) ? ratio : powf(ratio, a.gamma);
          }
          f *= a.m_min + (1.0f - a.m_min) * d;
        }
        cf w = cscale(v[s], f);
        v[s] = with_d ? make_float2(-kzv * w.y, kzv * w.x) : w;
      }
      PZ::template to_time<true>(v, t, a.tw);
    }
    // ---- post-op (time layout, z = t + T m)
    if (MODE == AX_M) {
      const int c = (job == 0) ? 2 : (job == 1 ? 1 : 0);
#pragma unroll
      for (int m = 0; m < R; ++m)
        if (act) y[(long)(c * NZ + t + T * m) * nc + col] = v[m];
      continue;
    }
    if (job == 0 || job == 1 || job == 3) {
      const int sl = (job == 0) ? 0 : (job == 1 ? 1 : 3);
#pragma unroll
      for (int m = 0; m < R; ++m) stash(sl, m, v[m]);
    } else if (job == 2) {
#pragma unroll
      for (int m = 0; m < R; ++m) {
        const cf dq = (MODE == AX_AH) ? v[m] : cmul(v[m], __ldg(a.sinv + t + T * m));
        stash(2, m, csub(cmul(iky, unst(0, m)), dq));
      }
    } else if (job == 4 && MODE == AX_AH) {
#pragma unroll
      for (int m = 0; m < R; ++m) v[m] = csub(v[m], cmul(ikx, unst(0, m)));   // c~_y
      const int nab = a.za1 - a.za0;
      const cf* __restrict__ G = a.G + rhs * a.gstride;
#pragma unroll
      for (int m = 0; m < R; ++m) {
        const int z = t + T * m;
        const cf qz = unst(0, m), cx = unst(2, m), cy = v[m];
        cf Wz = csub(csub(cmul(ikx, cy), cmul(iky, cx)), cmul(qz, kbg_at(a, z)));
        if (z >= a.za0 && z < a.za1 && act) Wz = csub(Wz, G[(2L * nab + z - a.za0) * nc + col]);
        if (act) y[(long)(2 * NZ + z) * nc + col] = Wz;
      }
#pragma unroll
      for (int m = 0; m < R; ++m) stash(0, m, v[m]);
    } else if (job == 4) {
#pragma unroll
      for (int m = 0; m < R; ++m) {
        const cf dq = cmul(v[m], __ldg(a.sinv + t + T * m));
        v[m] = csub(dq, cmul(ikx, unst(0, m)));   // c_y
      }
      __syncwarp();
      // reflected vector of this column from the tangential q at z_ml (Sec. 2.2, R_ml)
      const int tml = a.z_ml % T, mml = a.z_ml / T;
      const cf exm = st[(3 * R + mml) * 32 + tml * P + p];
      const cf eym = st[(1 * R + mml) * 32 + tml * P + p];
      const float4 rr = __ldg(a.refl + cc);
      const cf rs = make_float2(rr.x, rr.y), rp = make_float2(rr.z, rr.w);
      const cf kz0 = __ldg(a.kz0 + cc);
      const float kp = sqrtf(kx * kx + ky * ky);
      float sx, sy, tx, ty;
      if (kp > 0.f) { sx = -ky / kp; sy = kx / kp; tx = kx / kp; ty = ky / kp; }
      else { sx = 0.f; sy = 1.f; tx = 1.f; ty = 0.f; }
      const cf as = make_float2(sx * exm.x + sy * eym.x, sx * exm.y + sy * eym.y);
      const cf at = make_float2(tx * exm.x + ty * eym.x, tx * exm.y + ty * eym.y);
      const cf ras = cmul(rs, as), rat = cmul(rp, at);
      const cf r0 = make_float2(ras.x * sx + rat.x * tx, ras.y * sx + rat.y * tx);
      const cf r1 = make_float2(ras.x * sy + rat.x * ty, ras.y * sy + rat.y * ty);
      const cf num = make_float2(-(kx * r0.x + ky * r1.x), -(kx * r0.y + ky * r1.y));
      const float kd = kz0.x * kz0.x + kz0.y * kz0.y;
      const cf r2 = make_float2((num.x * kz0.x + num.y * kz0.y) / kd, (num.y * kz0.x - num.x * kz0.y) / kd);
      const int nab = a.za1 - a.za0;
      cf* __restrict__ G = a.G + rhs * a.gstride;
#pragma unroll
      for (int m = 0; m < R; ++m) {
        const int z = t + T * m;
        const cf qz = unst(0, m), cx = unst(2, m), cy = v[m];
        const cf Wz = csub(csub(cmul(ikx, cy), cmul(iky, cx)), cmul(qz, kbg_at(a, z)));
        if (act) y[(long)(2 * NZ + z) * nc + col] = Wz;
        if (z >= a.za0 && z < a.za1 && act) {
          cf prof = czero();
          if (z >= a.z_ml) {
            const float zr = (float)(z - a.z_ml) * a.dz;
            float sn, cs;
            sincosf(kz0.x * zr, &sn, &cs);
            const float mag = expf(-kz0.y * zr);
            prof = make_float2(mag * cs, mag * sn);
          }
          const long o = (long)(z - a.za0) * nc + col;
          G[o] = cfma(r0, prof, unst(3, m));
          G[(long)nab * nc + o] = cfma(r1, prof, unst(1, m));
          G[2L * nab * nc + o] = cfma(r2, prof, qz);
        }
      }
#pragma unroll
      for (int m = 0; m < R; ++m) stash(0, m, v[m]);   // c_y replaces q_z (lane-private entries)
    } else {
      const int c = (job == 5) ? 1 : 0;
      const int nab = a.za1 - a.za0;
      const cf* __restrict__ G = a.G + rhs * a.gstride;
#pragma unroll
      for (int m = 0; m < R; ++m) {
        const int z = t + T * m;
        const cf d = (MODE == AX_AH) ? v[m] : cmul(v[m], __ldg(a.sinv + z));
        const cf qx = unst(3, m), qy = unst(1, m);
        const cf cz = csub(cmul(ikx, qy), cmul(iky, qx));
        const cf kb = kbg_at(a, z);
        cf W = (job == 5) ? csub(csub(d, cmul(ikx, cz)), cmul(qy, kb))
                          : csub(csub(cmul(iky, cz), d), cmul(qx, kb));
        if (MODE == AX_AH) {
          if (z >= a.za0 && z < a.za1 && act) W = csub(W, G[((long)c * nab + z - a.za0) * nc + col]);
          if (z == a.z_ml) W = csub(W, c == 0 ? rh0 : rh1);
        }
        if (act) y[(long)(c * NZ + z) * nc + col] = W;
      }
    }
  }
}

template <int NZ, int T, int MODE>
static int run_axial(psfd_plan_s* P, const cf* x, cf* y, const int* done) {
  constexpr int P_ = 32 / T, R = NZ / T;
  AxialArgs a;
  a.x = x; a.y = y; a.G = P->G;
  a.kx = P->kx; a.ky = P->ky; a.kz = P->kz; a.sinv = P->sinv; a.kbg = P->kbg; a.tw = P->tw_z;
  a.refl = P->R.refl; a.kz0 = P->R.kz0; a.done = done;
  a.nx = P->nx; a.ncols = P->ncols; a.vstride = P->nvec;
  a.gstride = 3L * (P->za1 - P->za0) * P->ncols;
  a.z_ml = P->p.z_ml; a.za0 = P->za0; a.za1 = P->za1;
  a.dz = (float)P->p.dz; a.k02 = (float)(P->k0 * P->k0);
  a.m_min = P->m_min; a.kref2 = P->kref2; a.gamma = P->gamma; a.damp_eps = P->damp_eps;
  const int warps = 4;
  const long cols_per_block = warps * P_;
  dim3 grid((unsigned)((P->ncols + cols_per_block - 1) / cols_per_block), (unsigned)P->nrhs);
  size_t smem = (MODE == AX_M) ? 0 : (size_t)warps * 4 * R * 32 * sizeof(cf);
  static_assert(R > 0, "");
  if (smem > 48 * 1024) {
    cudaFuncSetAttribute(k_axial<NZ, T, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  }
  (void)launch_pdl(k_axial<NZ, T, MODE>, grid, dim3(warps * 32), smem, P->stream, a);
  PSFD_CHECK_LAUNCH();
  return PSFD_OK;
}

template <int NZ, int T>
static int run_axial_mode(psfd_plan_s* P, const cf* x, cf* y, int mode, const int* done) {
  switch (mode) {
    case AX_AM: return run_axial<NZ, T, AX_AM>(P, x, y, done);
    case AX_A: return run_axial<NZ, T, AX_A>(P, x, y, done);
    case AX_AH: return run_axial<NZ, T, AX_AH>(P, x, y, done);
    default: return run_axial<NZ, T, AX_M>(P, x, y, done);
  }
}

int axial_supported(int nz) {
  switch (nz) {
    case 16: case 32: case 48: case 64: case 96: case 128: case 256: case 512: case 1024: return 1;
    default: return 0;
  }
}

int launch_axial(psfd_plan_s* P, const cf* x, cf* y, int mode, const int* done, int) {
  // read x, write y (all planes); the operator modes also write (or, adjoint, read) G
  const double vb = (double)P->nrhs * P->nvec * sizeof(cf);
  const double gb = (mode == AX_M) ? 0.0 : (double)P->nrhs * 3 * (P->za1 - P->za0) * P->ncols * sizeof(cf);
  StageScope sc(P->stream, ST_AXIAL, 2.0 * vb + gb);
  const int T = P->axial_T;
  switch (P->nz) {
    case 16: return (T == 4) ? run_axial_mode<16, 4>(P, x, y, mode, done) : run_axial_mode<16, 2>(P, x, y, mode, done);
    case 32: return (T == 2) ? run_axial_mode<32, 2>(P, x, y, mode, done) : run_axial_mode<32, 4>(P, x, y, mode, done);
    case 48: return (T == 2) ? run_axial_mode<48, 2>(P, x, y, mode, done) : run_axial_mode<48, 4>(P, x, y, mode, done);
    case 64: return (T == 4) ? run_axial_mode<64, 4>(P, x, y, mode, done) : run_axial_mode<64, 8>(P, x, y, mode, done);
    case 96: return run_axial_mode<96, 4>(P, x, y, mode, done);
    case 128: return (T == 4) ? run_axial_mode<128, 4>(P, x, y, mode, done) : run_axial_mode<128, 8>(P, x, y, mode, done);
    // long columns (layer stacks meshed in the domain): one warp per column above 256 planes
    case 256: return run_axial_mode<256, 16>(P, x, y, mode, done);
    case 512: return run_axial_mode<512, 16>(P, x, y, mode, done);
    case 1024: return run_axial_mode<1024, 32>(P, x, y, mode, done);
  }
  psfd_set_error("axial: unsupported nz %d", P->nz);
  return PSFD_ERR_ARG;
}

// lanes per axial pencil that the kernels are compiled for (the autotuner's choices)
int axial_candidates(int nz, int* out) {
  switch (nz) {
    case 16: out[0] = 2; out[1] = 4; return 2;
    case 32: out[0] = 4; out[1] = 2; return 2;
    case 48: out[0] = 4; out[1] = 2; return 2;
    case 64: out[0] = 8; out[1] = 4; return 2;
    case 96: out[0] = 4; return 1;
    case 128: out[0] = 8; out[1] = 4; return 2;
    case 256: out[0] = 16; return 1;
    case 512: out[0] = 16; return 1;
    case 1024: out[0] = 32; return 1;
  }
  return 0;
}

// ======================================================================= lateral passes
// Rows (x axis, contiguous): lane = p*T + t, P = 32/T rows per warp.  The lateral passes
// exchange through shared-memory tiles (measured faster than shuffles here; the axial kernel
// keeps shuffles, whose shared memory already limits its occupancy).
enum { ROW_FWD = 0, ROW_INV = 1, ROW_FWD_SUB = 2 };

struct RowArgs {
  cf* buf;
  long nrows;
  float scale;
  const cf* tw;
  // ROW_FWD_SUB: y[row'] -= scale * FFT_x(buf[row])
  cf* y;
  int ny, nz, nab, za0;
  const int* done;
  long rows_per_rhs;
};

template <int NX, int T, int OP>
__global__ void __launch_bounds__(128) k_rows(RowArgs a) {
  pdl_enter();
  constexpr int P = 32 / T, R = NX / T;
  using PX = Pencil<NX, T, 1>;
  __shared__ cf xch[4][PX::TILE];   // per-warp exchange tiles (4 warps per block)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int p = lane / T, t = lane - p * T;
  const long row = ((long)blockIdx.x * (blockDim.x >> 5) + warp) * P + p;
  cf* const xt = xch[warp];
  bool act = row < a.nrows;
  if (act && a.done && a.done[row / a.rows_per_rhs]) act = false;
  cf* __restrict__ src = a.buf + (act ? row : 0) * NX;
  cf v[R];
  if constexpr (OP == ROW_INV) {
#pragma unroll
    for (int s = 0; s < R; ++s) v[s] = act ? src[PX::freq_index(t, s)] : czero();
    PX::template to_time<true>(v, t, a.tw, xt);
#pragma unroll
    for (int m = 0; m < R; ++m)
      if (act) src[t + T * m] = cscale(v[m], a.scale);
  } else if constexpr (OP == ROW_FWD) {
#pragma unroll
    for (int m = 0; m < R; ++m) v[m] = act ? src[t + T * m] : czero();
    PX::template to_freq<false>(v, t, a.tw, xt);
#pragma unroll
    for (int s = 0; s < R; ++s)
      if (act) src[PX::freq_index(t, s)] = cscale(v[s], a.scale);
  } else {
    // map the G row (rhs, c, zz, iy) to the y row (rhs, c, za0 + zz, iy); the y row is read with
    // the G row, so that both latencies overlap
    const long per_c = (long)a.nab * a.ny;
    const long r = act ? row : 0;
    const long rhs = r / (3 * per_c), rem = r - rhs * 3 * per_c;
    const long c = rem / per_c, rem2 = rem - c * per_c;
    const long zz = rem2 / a.ny, iy = rem2 - zz * a.ny;
    cf* __restrict__ dst = a.y + (((rhs * 3 + c) * a.nz + a.za0 + zz) * a.ny + iy) * NX;
    cf o[R];
#pragma unroll
    for (int m = 0; m < R; ++m) v[m] = act ? src[t + T * m] : czero();
#pragma unroll
    for (int s = 0; s < R; ++s) o[s] = act ? dst[PX::freq_index(t, s)] : czero();
    PX::template to_freq<false>(v, t, a.tw, xt);
#pragma unroll
    for (int s = 0; s < R; ++s)
      if (act) dst[PX::freq_index(t, s)] = make_float2(fmaf(-a.scale, v[s].x, o[s].x), fmaf(-a.scale, v[s].y, o[s].y));
  }
}

// Columns (y axis, stride nx): lane = t*P + p, P = 32/T consecutive x per warp.
enum { COL_FWD = 0, COL_INV = 1, COL_CONTRAST = 2, COL_GAUSS = 3 };

struct ColArgs {
  cf* buf;
  long ncolumns;   // nplanes * nx
  int nx;
  float scale;
  const cf* tw;
  // COL_CONTRAST
  const float* fill;
  const cf* pc;    // per-plane contrast c[z]; the multiplier is cs * c[z] (conjugated if pc_conj)
  float cs;
  int pc_conj;
  int nab, za0;
  long plane_elems;  // nx * ny
  const int* done;
  long planes_per_rhs;
  // COL_GAUSS
  float sigma;
};

template <int NY, int T, int OP>
__global__ void __launch_bounds__(128) k_cols(ColArgs a) {
  pdl_enter();
  constexpr int P = 32 / T, R = NY / T;
  using PY = Pencil<NY, T, P>;
  __shared__ cf xch[4][PY::TILE];   // per-warp exchange tiles (4 warps per block)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int t = lane / P, p = lane - t * P;
  cf* const xt = xch[warp];
  const long colid = ((long)blockIdx.x * (blockDim.x >> 5) + warp) * P + p;
  bool act = colid < a.ncolumns;
  const long cid = act ? colid : 0;
  const long plane = cid / a.nx;
  const int ix = (int)(cid - plane * a.nx);
  if (act && a.done && a.done[plane / a.planes_per_rhs]) act = false;
  cf* __restrict__ base = a.buf + plane * a.plane_elems + ix;
  const long sx = a.nx;
  cf v[R];
  if constexpr (OP == COL_FWD) {
#pragma unroll
    for (int m = 0; m < R; ++m) v[m] = act ? base[(long)(t + T * m) * sx] : czero();
    PY::template to_freq<false>(v, t, a.tw, xt);
#pragma unroll
    for (int s = 0; s < R; ++s)
      if (act) base[(long)PY::freq_index(t, s) * sx] = cscale(v[s], a.scale);
  } else if constexpr (OP == COL_INV) {
#pragma unroll
    for (int s = 0; s < R; ++s) v[s] = act ? base[(long)PY::freq_index(t, s) * sx] : czero();
    PY::template to_time<true>(v, t, a.tw, xt);
#pragma unroll
    for (int m = 0; m < R; ++m)
      if (act) base[(long)(t + T * m) * sx] = cscale(v[m], a.scale);
  } else if constexpr (OP == COL_CONTRAST) {
    // IFFT_y -> * scale * deps * fill(x, y, z) -> FFT_y
    const long zz = plane % a.nab;
    const float* __restrict__ f = a.fill + (a.za0 + zz) * a.plane_elems + ix;
    const cf c0 = a.pc[a.za0 + zz];
    const float dre = a.cs * c0.x, dim = a.cs * (a.pc_conj ? -c0.y : c0.y);
#pragma unroll
    for (int s = 0; s < R; ++s) v[s] = act ? base[(long)PY::freq_index(t, s) * sx] : czero();
    float fv[R];   // the fill is loaded with the column, so that both latencies overlap
#pragma unroll
    for (int m = 0; m < R; ++m) fv[m] = act ? __ldg(f + (long)(t + T * m) * sx) : 0.f;
    PY::template to_time<true>(v, t, a.tw, xt);
#pragma unroll
    for (int m = 0; m < R; ++m) v[m] = cmul(v[m], make_float2(dre * fv[m], dim * fv[m]));
    PY::template to_freq<false>(v, t, a.tw, xt);
#pragma unroll
    for (int s = 0; s < R; ++s)
      if (act) base[(long)PY::freq_index(t, s) * sx] = v[s];
  } else {
    // Gaussian smoothing of a single plane: FFT_y -> * exp(-sigma^2 |kappa|^2 / 2) -> IFFT_y
    const float kxp = 6.283185307179586f * (float)fft_signed(ix, a.nx) / (float)a.nx;
#pragma unroll
    for (int m = 0; m < R; ++m) v[m] = act ? base[(long)(t + T * m) * sx] : czero();
    PY::template to_freq<false>(v, t, a.tw, xt);
#pragma unroll
    for (int s = 0; s < R; ++s) {
      const float kyp = 6.283185307179586f * (float)fft_signed(PY::freq_index(t, s), NY) / (float)NY;
      const float g = expf(-0.5f * a.sigma * a.sigma * (kxp * kxp + kyp * kyp));
      v[s] = cscale(v[s], g);
    }
    PY::template to_time<true>(v, t, a.tw, xt);
#pragma unroll
    for (int m = 0; m < R; ++m)
      if (act) base[(long)(t + T * m) * sx] = v[m];
  }
}

int lateral_supported(int n) {
  switch (n) {
    case 16: case 32: case 64: case 96: case 128: case 256: case 512: return 1;
    default: return 0;
  }
}

template <int NX, int T>
static int rows_op(const RowArgs& a, int op, cudaStream_t s) {
  constexpr int P = 32 / T;
  const int warps = 4;
  const long per_block = warps * P;
  dim3 grid((unsigned)((a.nrows + per_block - 1) / per_block));
  if (grid.x == 0) return PSFD_OK;
  switch (op) {
    case ROW_FWD: (void)launch_pdl(k_rows<NX, T, ROW_FWD>, grid, dim3(warps * 32), 0, s, a); break;
    case ROW_INV: (void)launch_pdl(k_rows<NX, T, ROW_INV>, grid, dim3(warps * 32), 0, s, a); break;
    default: (void)launch_pdl(k_rows<NX, T, ROW_FWD_SUB>, grid, dim3(warps * 32), 0, s, a); break;
  }
  PSFD_CHECK_LAUNCH();
  return PSFD_OK;
}

static int rows_dispatch(int nx, const RowArgs& a, int op, cudaStream_t s) {
  switch (nx) {
    case 16: return rows_op<16, 4>(a, op, s);
    case 32: return rows_op<32, 4>(a, op, s);
    case 64: return rows_op<64, 8>(a, op, s);
    case 96: return rows_op<96, 4>(a, op, s);
    case 128: return rows_op<128, 8>(a, op, s);
    case 256: return rows_op<256, 16>(a, op, s);
    case 512: return rows_op<512, 16>(a, op, s);
  }
  psfd_set_error("rows: unsupported n %d", nx);
  return PSFD_ERR_ARG;
}

template <int NY, int T>
static int cols_op(const ColArgs& a, int op, cudaStream_t s) {
  constexpr int P = 32 / T;
  if (a.nx % P != 0) {
    psfd_set_error("cols: nx %d not a multiple of %d", a.nx, P);
    return PSFD_ERR_ARG;
  }
  const int warps = 4;
  const long per_block = warps * P;
  dim3 grid((unsigned)((a.ncolumns + per_block - 1) / per_block));
  if (grid.x == 0) return PSFD_OK;
  switch (op) {
    case COL_FWD: (void)launch_pdl(k_cols<NY, T, COL_FWD>, grid, dim3(warps * 32), 0, s, a); break;
    case COL_INV: (void)launch_pdl(k_cols<NY, T, COL_INV>, grid, dim3(warps * 32), 0, s, a); break;
    case COL_CONTRAST: (void)launch_pdl(k_cols<NY, T, COL_CONTRAST>, grid, dim3(warps * 32), 0, s, a); break;
    default: (void)launch_pdl(k_cols<NY, T, COL_GAUSS>, grid, dim3(warps * 32), 0, s, a); break;
  }
  PSFD_CHECK_LAUNCH();
  return PSFD_OK;
}

static int cols_dispatch(int ny, const ColArgs& a, int op, cudaStream_t s) {
  switch (ny) {
    case 16: return cols_op<16, 2>(a, op, s);
    case 32: return cols_op<32, 4>(a, op, s);
    case 48: return cols_op<48, 4>(a, op, s);
    case 64: return cols_op<64, 4>(a, op, s);
    case 96: return cols_op<96, 4>(a, op, s);
    case 128: return cols_op<128, 8>(a, op, s);
    case 256: return cols_op<256, 8>(a, op, s);
    case 512: return cols_op<512, 16>(a, op, s);
  }
  psfd_set_error("cols: unsupported n %d", ny);
  return PSFD_ERR_ARG;
}

int launch_rows(int n, cf* buf, long nrows, bool forward, float scale, const cf* tw, cudaStream_t s) {
  RowArgs a{};
  a.buf = buf; a.nrows = nrows; a.scale = scale; a.tw = tw; a.rows_per_rhs = 1;
  return rows_dispatch(n, a, forward ? ROW_FWD : ROW_INV, s);
}

int launch_cols(int n, int nx, cf* buf, long ncols_total, bool forward, float scale, const cf* tw,
                cudaStream_t s) {
  ColArgs a{};
  a.buf = buf; a.ncolumns = ncols_total; a.nx = nx; a.scale = scale; a.tw = tw;
  a.plane_elems = (long)n * nx; a.planes_per_rhs = 1;
  return cols_dispatch(n, a, forward ? COL_FWD : COL_INV, s);
}

int launch_cols_gauss(int ny, int nx, cf* buf, float sigma, const cf* tw, cudaStream_t s) {
  ColArgs a{};
  a.buf = buf; a.ncolumns = nx; a.nx = nx; a.scale = 1.f; a.tw = tw; a.sigma = sigma;
  a.plane_elems = (long)nx * ny; a.planes_per_rhs = 1;
  return cols_dispatch(ny, a, COL_GAUSS, s);
}

// real space <-> HYBRID over nplanes planes: forward = rows then columns (unitary scale)
int launch_lateral_transform(psfd_plan_s* P, cf* buf, long nplanes, bool forward, float scale) {
  StageScope sc(P->stream, ST_TRANSFORM, 2.0 * nplanes * P->ncols * sizeof(cf));
  int rc;
  const long rows = nplanes * P->ny, cols = nplanes * P->nx;
  if (forward) {
    if ((rc = launch_rows(P->nx, buf, rows, true, 1.f, P->tw_x, P->stream))) return rc;
    return launch_cols(P->ny, P->nx, buf, cols, true, scale, P->tw_y, P->stream);
  }
  if ((rc = launch_cols(P->ny, P->nx, buf, cols, false, 1.f, P->tw_y, P->stream))) return rc;
  return launch_rows(P->nx, buf, rows, false, scale, P->tw_x, P->stream);
}

// ======================================================================= single-pass plane kernel
// One CTA per (rhs, component, absorber plane) of a square N x N grid (N <= 128):
// the G plane and the fill plane are brought into shared memory with bulk async
// copies (cp.async.bulk, completion on an mbarrier, bounded wait), then
//   row IFFT_x -> column IFFT_y * k0^2 deps fill / N^2 * FFT_y -> row FFT_x,
// and the result is subtracted from y (forward operator) or written back to G
// (adjoint preparation).  The plane crosses HBM once instead of three times.
// Rows of the staged plane are padded by 4 complex entries so that the column
// pass (T rows x P consecutive columns per warp access) is free of bank conflicts.
constexpr int kPlaneThreads = 512;
constexpr int kRowPad = 4;

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

struct PlaneArgs {
  cf* G;
  cf* y;
  const float* fill;
  const cf* twx;
  const cf* twy;
  const int* done;
  int* err;
  int nz, nab, za0;
  const cf* pc;     // per-plane contrast; multiplier cs * c[z] (conjugated if pc_conj)
  float cs;
  int pc_conj;
  bool to_y;   // true: y -= result (forward); false: G <- result (adjoint preparation)
};

template <int N, int TR, int TC>
__global__ void __launch_bounds__(kPlaneThreads) k_plane(PlaneArgs a) {
  constexpr int RS = N + kRowPad;
  constexpr int PR = 32 / TR, RR = N / TR;   // rows: lane = p*TR + t
  constexpr int PC = 32 / TC, RC = N / TC;   // columns: lane = t*PC + p
  using PX = Pencil<N, TR, 1>;
  using PY = Pencil<N, TC, PC>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  cf* S = reinterpret_cast<cf*>(smem_raw);                             // N x RS complex
  float* F = reinterpret_cast<float*>(smem_raw + sizeof(cf) * N * RS);  // N x N fill
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem_raw + sizeof(cf) * N * RS + sizeof(float) * N * N);
  const long plane = blockIdx.x;
  const long per_rhs = 3L * a.nab;
  const long rhs = plane / per_rhs;
  if (a.done && a.done[rhs]) return;
  const int c = (int)((plane / a.nab) % 3);
  const int zz = (int)(plane % a.nab);
  const cf c0 = a.pc[a.za0 + zz];
  const float dre = a.cs * c0.x, dim = a.cs * (a.pc_conj ? -c0.y : c0.y);
  cf* Gp = a.G + plane * (long)N * N;
  const float* Fp = a.fill + (long)(a.za0 + zz) * N * N;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int nwarps = kPlaneThreads / 32;

  // ---- stage G (row by row, padded) and the fill plane with bulk async copies
  const unsigned mb = smem_u32(bar);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(mb) : "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0) {
    const unsigned tx = (unsigned)(sizeof(cf) * N * N + sizeof(float) * N * N);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(mb), "r"(tx) : "memory");
    for (int r = 0; r < N; ++r) {
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                   :: "r"(smem_u32(S + r * RS)), "l"(Gp + (long)r * N), "r"((unsigned)(sizeof(cf) * N)), "r"(mb)
                   : "memory");
    }
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(smem_u32(F)), "l"(Fp), "r"((unsigned)(sizeof(float) * N * N)), "r"(mb) : "memory");
  }
  // bounded wait on phase 0 of the barrier
  {
    unsigned ok = 0;
    for (long it = 0; it < (1L << 26) && !ok; ++it) {
      asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}"
                   : "=r"(ok) : "r"(mb) : "memory");
    }
    // leave together: a thread that gave up makes the whole block return
    if (__syncthreads_or(!ok)) {
      if (tid == 0) atomicExch(a.err, 1);
      return;
    }
  }

  // ---- row IFFT_x (kx -> x)
  for (int r0 = warp * PR; r0 < N; r0 += nwarps * PR) {
    const int p = lane / TR, t = lane - p * TR;
    const int row = r0 + p;
    cf v[RR];
#pragma unroll
    for (int s = 0; s < RR; ++s) v[s] = S[row * RS + PX::freq_index(t, s)];
    PX::template to_time<true>(v, t, a.twx);
#pragma unroll
    for (int m = 0; m < RR; ++m) S[row * RS + t + TR * m] = v[m];
  }
  __syncthreads();
  // ---- columns: IFFT_y (ky -> y), * k0^2 deps fill / N^2, FFT_y
  for (int c0 = warp * PC; c0 < N; c0 += nwarps * PC) {
    const int t = lane / PC, p = lane - t * PC;
    const int col = c0 + p;
    cf v[RC];
#pragma unroll
    for (int s = 0; s < RC; ++s) v[s] = S[PY::freq_index(t, s) * RS + col];
    PY::template to_time<true>(v, t, a.twy);
#pragma unroll
    for (int m = 0; m < RC; ++m) {
      const float fv = F[(t + TC * m) * N + col];
      v[m] = cmul(v[m], make_float2(dre * fv, dim * fv));
    }
    PY::template to_freq<false>(v, t, a.twy);
#pragma unroll
    for (int s = 0; s < RC; ++s) S[PY::freq_index(t, s) * RS + col] = v[s];
  }
  __syncthreads();
  // ---- row FFT_x (x -> kx) and combine
  cf* yp = a.to_y ? a.y + (((rhs * 3 + c) * a.nz + a.za0 + zz) * (long)N) * N : Gp;
  for (int r0 = warp * PR; r0 < N; r0 += nwarps * PR) {
    const int p = lane / TR, t = lane - p * TR;
    const int row = r0 + p;
    cf v[RR];
#pragma unroll
    for (int m = 0; m < RR; ++m) v[m] = S[row * RS + t + TR * m];
    PX::template to_freq<false>(v, t, a.twx);
#pragma unroll
    for (int s = 0; s < RR; ++s) {
      const long o = (long)row * N + PX::freq_index(t, s);
      if (a.to_y) {
        const cf old = yp[o];
        yp[o] = csub(old, v[s]);
      } else {
        yp[o] = v[s];
      }
    }
  }
}

template <int N, int TR, int TC>
static int run_plane(psfd_plan_s* P, const PlaneArgs& a, long nplanes) {
  const size_t smem = sizeof(cf) * N * (N + kRowPad) + sizeof(float) * N * N + 16;
  static std::once_flag once;   // complete before any host thread launches
  static cudaError_t init = cudaSuccess;
  std::call_once(once, [smem] {
    init = cudaFuncSetAttribute(k_plane<N, TR, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  if (init != cudaSuccess) {
    psfd_set_error("plane contrast: %s", cudaGetErrorString(init));
    return PSFD_ERR_CUDA;
  }
  k_plane<N, TR, TC><<<(unsigned)nplanes, kPlaneThreads, smem, P->stream>>>(a);
  PSFD_CHECK_LAUNCH();
  return PSFD_OK;
}

// 1 if the single-pass plane kernel handles this grid, and launches it
static int plane_contrast(psfd_plan_s* P, cf* y, const int* done, bool adjoint, bool to_y, bool* handled) {
  *handled = false;
  if (P->nx != P->ny || P->nx > 128 || !P->use_plane) return PSFD_OK;
  if (!P->err) {
    PSFD_CUDA_TRY(cudaMalloc((void**)&P->err, sizeof(int)));
    PSFD_CUDA_TRY(cudaMemset(P->err, 0, sizeof(int)));
  }
  const int nab = P->za1 - P->za0;
  PlaneArgs a;
  a.G = P->G; a.y = y; a.fill = P->fill; a.twx = P->tw_x; a.twy = P->tw_y; a.done = done; a.err = P->err;
  a.nz = P->nz; a.nab = nab; a.za0 = P->za0;
  a.pc = P->pc;
  a.cs = (float)(P->k0 * P->k0 / (double)P->ncols);
  a.pc_conj = adjoint ? 1 : 0;
  a.to_y = to_y;
  const long nplanes = (long)P->nrhs * 3 * nab;
  int rc = PSFD_OK;
  switch (P->nx) {
    case 16: rc = run_plane<16, 4, 2>(P, a, nplanes); break;
    case 32: rc = run_plane<32, 4, 4>(P, a, nplanes); break;
    case 64: rc = run_plane<64, 8, 4>(P, a, nplanes); break;
    case 96: rc = run_plane<96, 4, 4>(P, a, nplanes); break;
    case 128: rc = run_plane<128, 8, 8>(P, a, nplanes); break;
    default: return PSFD_OK;
  }
  if (rc) return rc;
  *handled = true;
  return PSFD_OK;
}

// y (absorber planes) -= k0^2 F_xy[deps F_xy^-1 G] / (nx ny): G is consumed.
int launch_lateral_contrast(psfd_plan_s* P, cf* y, const int* done, bool adjoint) {
  const int nab = P->za1 - P->za0;
  if (nab <= 0) return PSFD_OK;
  // read G, read fill, read y, write y on the absorber planes
  StageScope scope(P->stream, ST_CONTRAST,
                   (double)P->nrhs * nab * P->ncols * (3.0 * 3 * sizeof(cf) + sizeof(float)));
  const long nplanes = (long)P->nrhs * 3 * nab;
  int rc;
  bool handled = false;
  if ((rc = plane_contrast(P, y, done, adjoint, true, &handled))) return rc;
  if (handled) return PSFD_OK;
  RowArgs r{};
  r.buf = P->G; r.nrows = nplanes * P->ny; r.scale = 1.f; r.tw = P->tw_x; r.done = done;
  r.rows_per_rhs = 3L * nab * P->ny;
  if ((rc = rows_dispatch(P->nx, r, ROW_INV, P->stream))) return rc;
  ColArgs c{};
  const double sc = P->k0 * P->k0 / (double)P->ncols;
  c.buf = P->G; c.ncolumns = nplanes * P->nx; c.nx = P->nx; c.scale = 1.f; c.tw = P->tw_y;
  c.fill = P->fill; c.pc = P->pc; c.cs = (float)sc; c.pc_conj = adjoint ? 1 : 0;
  c.nab = nab; c.za0 = P->za0; c.plane_elems = P->ncols; c.done = done; c.planes_per_rhs = 3L * nab;
  if ((rc = cols_dispatch(P->ny, c, COL_CONTRAST, P->stream))) return rc;
  RowArgs w{};
  w.buf = P->G; w.nrows = nplanes * P->ny; w.scale = 1.f; w.tw = P->tw_x; w.y = y;
  w.ny = P->ny; w.nz = P->nz; w.nab = nab; w.za0 = P->za0; w.done = done; w.rows_per_rhs = 3L * nab * P->ny;
  return rows_dispatch(P->nx, w, ROW_FWD_SUB, P->stream);
}

// G <- k0^2 F_xy[conj(deps) F_xy^-1 x] on the absorber planes (first half of the adjoint)
static int adjoint_contrast(psfd_plan_s* P, const cf* x) {
  const int nab = P->za1 - P->za0;
  if (nab <= 0) return PSFD_OK;
  StageScope scope(P->stream, ST_CONTRAST);
  const long pe = (long)nab * P->ncols;
  for (int r = 0; r < P->nrhs; ++r)
    for (int c = 0; c < 3; ++c) {
      const cf* src = x + (long)r * P->nvec + ((long)c * P->nz + P->za0) * P->ncols;
      cf* dst = P->G + ((long)r * 3 + c) * pe;
      PSFD_CUDA_TRY(cudaMemcpyAsync(dst, src, pe * sizeof(cf), cudaMemcpyDeviceToDevice, P->stream));
    }
  const long nplanes = (long)P->nrhs * 3 * nab;
  int rc;
  bool handled = false;
  if ((rc = plane_contrast(P, nullptr, nullptr, true, false, &handled))) return rc;
  if (handled) return PSFD_OK;
  RowArgs r{};
  r.buf = P->G; r.nrows = nplanes * P->ny; r.scale = 1.f; r.tw = P->tw_x; r.rows_per_rhs = 3L * nab * P->ny;
  if ((rc = rows_dispatch(P->nx, r, ROW_INV, P->stream))) return rc;
  ColArgs c{};
  const double sc = P->k0 * P->k0 / (double)P->ncols;
  c.buf = P->G; c.ncolumns = nplanes * P->nx; c.nx = P->nx; c.scale = 1.f; c.tw = P->tw_y;
  c.fill = P->fill; c.pc = P->pc; c.cs = (float)sc; c.pc_conj = 1;
  c.nab = nab; c.za0 = P->za0; c.plane_elems = P->ncols; c.planes_per_rhs = 3L * nab;
  if ((rc = cols_dispatch(P->ny, c, COL_CONTRAST, P->stream))) return rc;
  return rows_dispatch(P->nx, r, ROW_FWD, P->stream);
}

// y = A x, A M x, A^H x or M A^H x, all in the HYBRID domain
int apply_hybrid(psfd_plan_s* P, const cf* x, cf* y, int flags, const int* done) {
  int rc;
  if (flags & PSFD_ADJOINT) {
    if (flags & PSFD_LAYERED) { psfd_set_error("psfd_apply: PSFD_LAYERED has no adjoint"); return PSFD_ERR_ARG; }
    if ((rc = adjoint_contrast(P, x))) return rc;
    if (!(flags & PSFD_PRECOND)) return launch_axial(P, x, y, AX_AH, done, P->nrhs);
    if ((rc = launch_axial(P, x, P->tmpB, AX_AH, done, P->nrhs))) return rc;
    return launch_axial(P, P->tmpB, y, AX_M, done, P->nrhs);
  }
  if (flags & PSFD_LAYERED) {
    // A P x: the per-column inverses first, then the operator
    if ((rc = layered_apply(P, x, P->tmpB, done))) return rc;
    x = P->tmpB;
  }
  rc = launch_axial(P, x, y, (flags & PSFD_PRECOND) && !(flags & PSFD_LAYERED) ? AX_AM : AX_A, done, P->nrhs);
  if (rc) return rc;
  return launch_lateral_contrast(P, y, done, false);
}

extern "C" int psfd_apply(psfd_plan P, const psfd_c64* x, psfd_c64* y, int flags) {
  if (!P || !x || !y) { psfd_set_error("psfd_apply: null argument"); return PSFD_ERR_ARG; }
  if (!P->have_background) { psfd_set_error("psfd_apply: call psfd_background first"); return PSFD_ERR_STATE; }
  if (x == y) { psfd_set_error("psfd_apply: x and y must not overlap"); return PSFD_ERR_ARG; }
  if ((flags & PSFD_LAYERED) && !P->lay_built) {
    psfd_set_error("psfd_apply: call psfd_layered_build first");
    return PSFD_ERR_STATE;
  }
  const cf* xi = (const cf*)x;
  cf* yo = (cf*)y;
  const long bytes = (long)P->nrhs * P->nvec * sizeof(cf);
  if (flags & PSFD_HYBRID) return apply_hybrid(P, xi, yo, flags, nullptr);
  const float us = 1.0f / sqrtf((float)P->ncols);
  const long nplanes = (long)P->nrhs * 3 * P->nz;
  PSFD_CUDA_TRY(cudaMemcpyAsync(P->tmpA, xi, bytes, cudaMemcpyDeviceToDevice, P->stream));
  int rc;
  if ((rc = launch_lateral_transform(P, P->tmpA, nplanes, true, us))) return rc;
  if ((rc = apply_hybrid(P, P->tmpA, yo, flags, nullptr))) return rc;
  return launch_lateral_transform(P, yo, nplanes, false, us);
}

extern "C" int psfd_precond(psfd_plan P, const psfd_c64* x, psfd_c64* y, int flags) {
  if (!P || !x || !y) { psfd_set_error("psfd_precond: null argument"); return PSFD_ERR_ARG; }
  const long bytes = (long)P->nrhs * P->nvec * sizeof(cf);
  const bool lay = (flags & PSFD_LAYERED) != 0;
  if (lay && !P->lay_built) { psfd_set_error("psfd_precond: call psfd_layered_build first"); return PSFD_ERR_STATE; }
  auto op = [&](const cf* in, cf* out) {
    return lay ? layered_apply(P, in, out) : launch_axial(P, in, out, AX_M, nullptr, P->nrhs);
  };
  if (flags & PSFD_HYBRID) {
    if ((const void*)x == (void*)y) {
      PSFD_CUDA_TRY(cudaMemcpyAsync(P->tmpA, x, bytes, cudaMemcpyDeviceToDevice, P->stream));
      return op(P->tmpA, (cf*)y);
    }
    return op((const cf*)x, (cf*)y);
  }
  const float us = 1.0f / sqrtf((float)P->ncols);
  const long nplanes = (long)P->nrhs * 3 * P->nz;
  PSFD_CUDA_TRY(cudaMemcpyAsync(P->tmpA, x, bytes, cudaMemcpyDeviceToDevice, P->stream));
  int rc;
  if ((rc = launch_lateral_transform(P, P->tmpA, nplanes, true, us))) return rc;
  if ((rc = op(P->tmpA, (cf*)y))) return rc;
  return launch_lateral_transform(P, (cf*)y, nplanes, false, us);
}
