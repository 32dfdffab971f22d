// Layered-background preconditioner: the exact inverse, per lateral Bloch mode, of the operator
// with the permittivity contrast replaced by its lateral average on each plane.
//
// With the fill averaged over every z-plane, Δε̄(z) = c(z) · mean_xy f(z) (c = ε_abs − 1 unless a
// per-plane contrast table is set), the operator of
// Eqs. bg_source / vector_helmholtz_operator no longer couples lateral modes.  For the mode
// (kx, ky), κ = |k∥|, ŝ = (−ky, kx)/κ, t̂ = (kx, ky)/κ (ŝ = ŷ, t̂ = x̂ at κ = 0) and the
// stretched axial derivative D = s⁻¹ F⁻¹ i k_z F, the curl-curl is
//     (cc)_s = (κ² − D²) E_s,   (cc)_t = −D² E_t + iκ D E_z,   (cc)_z = iκ D E_t + κ² E_z,
// and the reflection R (Sec. 2.2) maps E_s(z_ml) to r_s e(z) ŝ and E_t(z_ml) to
// r_p e(z) (t̂ − κ/k_z ẑ), e(z) = exp(i k_z (z − z_ml)) for z ≥ z_ml.  So the averaged operator
// splits into a TE block (E_s, nz × nz) and a TM block ((E_t, E_z), 2nz × 2nz):
//     TE = κ² − D² − k0² (1 + Δε̄) − k0² Δε̄ r_s e e_mlᵀ
//     TM = [ −D² − k0² (1 + Δε̄) − k0² Δε̄ r_p e e_mlᵀ      iκ D                 ]
//          [ iκ D + k0² Δε̄ (κ r_p / k_z) e e_mlᵀ          κ² − k0² (1 + Δε̄)   ]
// Both are assembled per column on the device and inverted in FP32 by Gauss-Jordan exchange
// steps with partial pivoting (one CTA per matrix, the matrix held in registers), then applied as
// dense per-column matrix-vector products in the HYBRID (kx, ky, z) domain.  Used as the right
// preconditioner P in A P y = b − A E_base, E = E_base + P y, in place of the spectral damping
// M of Eq. spectral_damping_action (an addition to the paper's method: the damping alone leaves
// restarted Krylov stalling near 1e-5 at oblique incidence, where near-grazing diffraction orders
// are barely absorbed by the axial PML; the averaged operator resolves those modes exactly).
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include <cuda_fp16.h>

#include "internal.h"

namespace {

using zc = std::complex<double>;
constexpr int LAY_THREADS = 256;   // 16 x 16 thread grid over an N x N matrix
constexpr int LAY_GROUP = 4;       // lateral columns (consecutive kx) per apply CTA

// PSFD_LAY_TC=1 applies the half-precision blocks on the tensor cores (nz a multiple of 32);
// the default is the SIMT kernel, measured faster on 128x128x64 (0.20 vs 0.30 ms per apply)
bool lay_apply_tc_enabled() {
  const char* e = getenv("PSFD_LAY_TC");
  return e && e[0] == '1';
}

struct LayArgs {
  const float* kx;
  const float* ky;
  const float4* refl;   // (r_s, r_p) per mode
  const cf* kz0;        // upgoing k_z per mode
  const cf* D;          // [nz][nz] stretched axial derivative
  const cf* D2;         // [nz][nz] D * D
  const cf* deps;       // [nz] laterally averaged contrast
  float k0sq, dz;
  int nx, ny, nz, zml;
  int pair;             // 1: blocks stored for rows 0 .. ny/2 only (ky and -ky share them)
  cf* mats;             // [ncols][5 nz^2]: TE inverse (nz^2) then TM inverse (4 nz^2), column-major
  __half2* mats16;      // the same in half precision (storage 1), entries divided by the block's scale
  float* scales;        // [ncols][2] power-of-two scale of the TE and TM block (storage 1)
  int half;             // 1: half-precision storage
  int* err;             // [0] set to 1 if a pivot vanished, [1] if an apply gave up waiting for its blocks
  int no_copy;          // test of the bounded wait: the tensor-core apply requests no blocks
};

__device__ __forceinline__ cf cdiv1(cf a) {  // 1 / a
  const float d = a.x * a.x + a.y * a.y;
  return make_float2(a.x / d, -a.y / d);
}

// per-column mode data
struct Mode {
  float kap, kap2;
  cf rs, rp, kz;
};
__device__ __forceinline__ Mode mode_of(const LayArgs& a, long col) {
  Mode m;
  const int ix = (int)(col % a.nx), iy = (int)(col / a.nx);
  const float kx = a.kx[ix], ky = a.ky[iy];
  m.kap2 = kx * kx + ky * ky;
  m.kap = sqrtf(m.kap2);
  const float4 r = a.refl[col];
  m.rs = make_float2(r.x, r.y);
  m.rp = make_float2(r.z, r.w);
  m.kz = a.kz0[col];
  return m;
}

// e(z) = exp(i k_z (z − z_ml) dz) for z ≥ z_ml, else 0
__device__ __forceinline__ cf upgoing(const LayArgs& a, const Mode& m, int z) {
  if (z < a.zml) return czero();
  const float d = (float)(z - a.zml) * a.dz;
  const float mag = expf(-m.kz.y * d);
  float sn, cs;
  sincosf(m.kz.x * d, &sn, &cs);
  return make_float2(mag * cs, mag * sn);
}

// entry (i, j) of the TE (TM = false, N = nz) or TM (TM = true, N = 2 nz) block of a column
template <bool TM>
__device__ cf entry(const LayArgs& a, const Mode& m, int i, int j) {
  const int nz = a.nz;
  if (!TM) {
    cf v = cneg(a.D2[i * nz + j]);
    const cf de = a.deps[i];
    if (i == j) v = cadd(v, make_float2(m.kap2 - a.k0sq * (1.f + de.x), -a.k0sq * de.y));
    if (j == a.zml && i >= a.zml) v = csub(v, cscale(cmul(cmul(de, m.rs), upgoing(a, m, i)), a.k0sq));
    return v;
  }
  const int bi = i / nz, bj = j / nz, ii = i - bi * nz, jj = j - bj * nz;
  const cf de = a.deps[ii];
  if (bi == 0 && bj == 0) {
    cf v = cneg(a.D2[ii * nz + jj]);
    if (ii == jj) v = cadd(v, make_float2(-a.k0sq * (1.f + de.x), -a.k0sq * de.y));
    if (jj == a.zml && ii >= a.zml) v = csub(v, cscale(cmul(cmul(de, m.rp), upgoing(a, m, ii)), a.k0sq));
    return v;
  }
  if (bi == 0) return ctimesi(cscale(a.D[ii * nz + jj], m.kap));   // iκ D
  if (bj == 0) {
    cf v = ctimesi(cscale(a.D[ii * nz + jj], m.kap));
    if (jj == a.zml && ii >= a.zml) {
      // + k0² Δε̄ (κ r_p / k_z) e
      const cf c = cmul(cmul(de, m.rp), cmul(upgoing(a, m, ii), cdiv1(m.kz)));
      v = cadd(v, cscale(c, a.k0sq * m.kap));
    }
    return v;
  }
  if (ii == jj) return make_float2(m.kap2 - a.k0sq * (1.f + de.x), -a.k0sq * de.y);
  return czero();
}

// Assemble and invert one N x N block per CTA.  Thread (rg, cg) of the 16 x 16 grid owns rows
// rg + 16 u and columns cg + 16 v (u, v < N/16).  Step k exchanges the roles of x_k and y_p for
// the pivot row p (largest |T[p][k]| among rows not yet used):
//     T[p][k] <- 1/π,  T[p][j] <- −T[p][j]/π,  T[i][k] <- T[i][k]/π,  T[i][j] <- T[i][j] − T[i][k] T[p][j]/π
// with π = T[p][k].  After N steps, row p_k holds x_k and column k' holds y_{p_k'}:
// Minv[k][p_k'] = T[p_k][k'].
template <int N, bool TM>
__global__ void __launch_bounds__(LAY_THREADS) k_lay_inv(LayArgs a, int block_off) {
  constexpr int TT = N / 16;
  __shared__ cf colv[2][N], rowv[2][N];
  __shared__ float mag[2][N];
  __shared__ int pivrow[N], rowvar[N];
  const long col = blockIdx.x;
  const int tid = threadIdx.x, rg = tid >> 4, cg = tid & 15, lane = tid & 31;
  const Mode m = mode_of(a, col);
  cf T[TT][TT];
#pragma unroll
  for (int u = 0; u < TT; ++u)
#pragma unroll
    for (int v = 0; v < TT; ++v) T[u][v] = entry<TM>(a, m, rg + 16 * u, cg + 16 * v);
  unsigned used = 0;   // bit u: owned row rg + 16 u has been a pivot row
  for (int k = 0; k < N; ++k) {
    const int buf = k & 1;
    // column k -> shared (owners: cg == k % 16); used rows get magnitude -1 and a non-finite
    // magnitude counts as 0, so the pivot is always a row not used before
    if (cg == (k & 15)) {
      const int vk = k >> 4;
#pragma unroll
      for (int v = 0; v < TT; ++v) {
        if (v != vk) continue;   // static register indexing: select the column by predicate
#pragma unroll
        for (int u = 0; u < TT; ++u) {
          const int i = rg + 16 * u;
          const cf t = T[u][v];
          const float mg = t.x * t.x + t.y * t.y;
          colv[buf][i] = t;
          mag[buf][i] = ((used >> u) & 1u) ? -1.f : (mg <= 3.0e38f ? mg : 0.f);
        }
      }
    }
    __syncthreads();
    // every warp finds the pivot itself (no broadcast barrier): argmax, ties to the lower row
    float best = -2.f;
    int p = 0;
    for (int i = lane; i < N; i += 32) {
      const float mv = mag[buf][i];
      if (mv > best) { best = mv; p = i; }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const float ob = __shfl_xor_sync(0xffffffffu, best, off);
      const int oi = __shfl_xor_sync(0xffffffffu, p, off);
      if (ob > best || (ob == best && oi < p)) { best = ob; p = oi; }
    }
    const bool ok = best > 0.f;
    const cf pinv = ok ? cdiv1(colv[buf][p]) : czero();
    if (tid == 0) {
      pivrow[k] = p;
      if (!ok) atomicExch(a.err, 1);
    }
    // pivot row p -> shared (owners: rg == p % 16)
    if (rg == (p & 15)) {
      const int up = p >> 4;
      used |= 1u << up;
#pragma unroll
      for (int u = 0; u < TT; ++u) {
        if (u != up) continue;
#pragma unroll
        for (int v = 0; v < TT; ++v) rowv[buf][cg + 16 * v] = T[u][v];
      }
    }
    __syncthreads();
    cf ci[TT], rj[TT];
#pragma unroll
    for (int u = 0; u < TT; ++u) ci[u] = cmul(colv[buf][rg + 16 * u], pinv);
#pragma unroll
    for (int v = 0; v < TT; ++v) rj[v] = rowv[buf][cg + 16 * v];
    // rank-1 update of every owned entry; the pivot row and column are overwritten below
#pragma unroll
    for (int u = 0; u < TT; ++u)
#pragma unroll
      for (int v = 0; v < TT; ++v) T[u][v] = csub(T[u][v], cmul(ci[u], rj[v]));
    const bool own_row = rg == (p & 15), own_col = cg == (k & 15);
    const int up = p >> 4, vk = k >> 4;
    if (own_row) {
#pragma unroll
      for (int u = 0; u < TT; ++u) {
        if (u != up) continue;
#pragma unroll
        for (int v = 0; v < TT; ++v) T[u][v] = cneg(cmul(rj[v], pinv));
      }
    }
    if (own_col) {
#pragma unroll
      for (int v = 0; v < TT; ++v) {
        if (v != vk) continue;
#pragma unroll
        for (int u = 0; u < TT; ++u) T[u][v] = (own_row && u == up) ? pinv : ci[u];
      }
    }
  }
  __syncthreads();
  // pivrow is a permutation: each step picks a row not used before
  for (int k = tid; k < N; k += LAY_THREADS) rowvar[pivrow[k]] = k;
  __syncthreads();
  // column-major output: element (r, c) of the inverse at c * N + r
  if (!a.half) {
    cf* out = a.mats + col * (5L * a.nz * a.nz) + block_off;
#pragma unroll
    for (int u = 0; u < TT; ++u)
#pragma unroll
      for (int v = 0; v < TT; ++v) {
        const int r = rowvar[rg + 16 * u], c = pivrow[cg + 16 * v];
        out[(long)c * N + r] = T[u][v];
      }
    return;
  }
  // half precision: divide by the power of two at or above the block's largest |re|, |im| (the
  // entries then lie in [-1, 1], where half keeps 11 significant bits)
  float mx = 0.f;
#pragma unroll
  for (int u = 0; u < TT; ++u)
#pragma unroll
    for (int v = 0; v < TT; ++v) mx = fmaxf(mx, fmaxf(fabsf(T[u][v].x), fabsf(T[u][v].y)));
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  __shared__ float wmax[LAY_THREADS / 32];
  if (lane == 0) wmax[tid >> 5] = mx;
  __syncthreads();
  mx = 0.f;
  for (int w = 0; w < LAY_THREADS / 32; ++w) mx = fmaxf(mx, wmax[w]);
  int e = 0;
  if (mx > 0.f && mx <= 3.0e38f) frexpf(mx, &e);   // mx = f 2^e with f in [0.5, 1)
  const float scale = ldexpf(1.f, e), inv = ldexpf(1.f, -e);
  if (tid == 0) a.scales[col * 2 + (TM ? 1 : 0)] = scale;
  __half2* out = a.mats16 + col * (5L * a.nz * a.nz) + block_off;
#pragma unroll
  for (int u = 0; u < TT; ++u)
#pragma unroll
    for (int v = 0; v < TT; ++v) {
      const int r = rowvar[rg + 16 * u], c = pivrow[cg + 16 * v];
      out[(long)c * N + r] = __floats2half2_rn(T[u][v].x * inv, T[u][v].y * inv);
    }
}

// mean fill of every z-plane (FP64 sum)
__global__ void k_plane_mean(const float* __restrict__ fill, long plane, double* mean) {
  __shared__ double sh[LAY_THREADS / 32];
  const int z = blockIdx.x;
  double s = 0.0;
  for (long i = threadIdx.x; i < plane; i += blockDim.x) s += (double)fill[(long)z * plane + i];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < LAY_THREADS / 32; ++w) t += sh[w];
    mean[z] = t / (double)plane;
  }
}

// y = P x in the HYBRID domain: per column, rotate (x, y) -> (s, t), apply the TE and TM
// inverses, rotate back.  The blocks depend on a column only through kappa = |k_par|; with no
// Bloch shift along y the columns ky and -ky share them, so blocks are stored for the rows
// h = 0 .. ny/2 only and a CTA serves LAY_GROUP consecutive kx columns of row h and of its partner
// row ny - h, reading each block once for both rows and all right-hand sides.  Each thread
// produces two adjacent output rows of one block (16-byte loads of the column-major blocks); a
// CTA has LAY_GROUP * 3 NZ / 2 threads.
// rows of a block per thread: 2 for complex64 blocks (16-byte loads of two entries), 4 for half
// blocks (16-byte loads of four entries)
template <bool HALF>
constexpr int apply_rpt() { return HALF ? 4 : 2; }
template <int NZ, bool HALF>
constexpr int apply_threads() { return LAY_GROUP * 3 * NZ / apply_rpt<HALF>(); }

template <int NZ, int NR, bool HALF>
__global__ void __launch_bounds__(apply_threads<NZ, HALF>(), (HALF ? 4 : (NR <= 2 ? 3 : 2)))
    k_lay_apply(LayArgs a, const cf* __restrict__ x, cf* __restrict__ y, long ncols) {
  constexpr int nrhs = NR;
  constexpr int G = LAY_GROUP, NT = apply_threads<NZ, HALF>(), RPT = apply_rpt<HALF>();
  extern __shared__ cf xs[];       // [2G][3][NZ][nrhs]: (s, t, z) components after rotation
  __shared__ float rot[2 * G][4];  // sx, sy, tx, ty per virtual column
  const long hc0 = (long)blockIdx.x * G;               // first block column: row h, kx index ix0
  const int ix0 = (int)(hc0 % a.nx), h = (int)(hc0 / a.nx);
  const int ny = a.ny;
  const int iyB = a.pair ? (ny - h) % ny : h;
  const bool two = a.pair && iyB != h;                 // a partner row exists
  const int nv = two ? 2 * G : G;                      // virtual columns: row h, then row iyB
  const int tid = threadIdx.x;
  if (tid < nv) {
    const int iy = tid < G ? h : iyB;
    const float kx = a.kx[ix0 + (tid % G)], ky = a.ky[iy];
    const float kap = sqrtf(kx * kx + ky * ky);
    const bool small = !(kap > 0.f);
    rot[tid][0] = small ? 0.f : -ky / kap;
    rot[tid][1] = small ? 1.f : kx / kap;
    rot[tid][2] = small ? 1.f : kx / kap;
    rot[tid][3] = small ? 0.f : ky / kap;
  }
  __syncthreads();
  const long n = 3L * NZ * ncols;   // entries per right-hand side
  auto colof = [&](int v) -> long { return (long)(v < G ? h : iyB) * a.nx + ix0 + (v % G); };
  // gather + rotate: item = ((r * NZ + z) * nv + v)
  for (int it = tid; it < nrhs * NZ * nv; it += NT) {
    const int v = it % nv, z = (it / nv) % NZ, r = it / (nv * NZ);
    const long base = (long)r * n + (long)z * ncols + colof(v);
    const cf ex = x[base], ey = x[base + (long)NZ * ncols], ez = x[base + 2L * NZ * ncols];
    const float sx = rot[v][0], sy = rot[v][1], tx = rot[v][2], ty = rot[v][3];
    xs[((v * 3 + 0) * NZ + z) * nrhs + r] = cadd(cscale(ex, sx), cscale(ey, sy));
    xs[((v * 3 + 1) * NZ + z) * nrhs + r] = cadd(cscale(ex, tx), cscale(ey, ty));
    xs[((v * 3 + 2) * NZ + z) * nrhs + r] = ez;
  }
  __syncthreads();
  constexpr long MS = 5L * NZ * NZ;
  // thread -> (block column g, rows rr .. rr + RPT - 1) of the 3 NZ stacked rows (TE, then TM)
  constexpr int TPC = 3 * NZ / RPT;                         // threads per block column
  const int g = tid / TPC, rr = RPT * (tid - g * TPC);
  const bool te = rr < NZ;
  const int nb = te ? NZ : 2 * NZ;                         // block size
  const int i = te ? rr : rr - NZ;                         // first row inside the block
  const cf* Mb = a.mats + (hc0 + g) * MS + (te ? 0 : (long)NZ * NZ);
  const __half2* Mh = a.mats16 + (hc0 + g) * MS + (te ? 0 : (long)NZ * NZ);
  const int comp0 = te ? 0 : 1;                            // TE: s; TM: t then z (contiguous)
  const cf* xa = xs + (g * 3 + comp0) * NZ * nrhs;
  const cf* xb = xs + ((g + G) * 3 + comp0) * NZ * nrhs;
  cf A[RPT][NR], Bv[RPT][NR];
#pragma unroll
  for (int q = 0; q < RPT; ++q)
#pragma unroll
    for (int r = 0; r < NR; ++r) { A[q][r] = czero(); Bv[q][r] = czero(); }
  auto load = [&](int j, cf (&m)[RPT]) {
    if constexpr (HALF) {
      const uint4 hv = __ldg(reinterpret_cast<const uint4*>(Mh + (long)j * nb + i));
      m[0] = __half22float2(*reinterpret_cast<const __half2*>(&hv.x));
      m[1] = __half22float2(*reinterpret_cast<const __half2*>(&hv.y));
      m[2] = __half22float2(*reinterpret_cast<const __half2*>(&hv.z));
      m[3] = __half22float2(*reinterpret_cast<const __half2*>(&hv.w));
    } else {
      const float4 mv = __ldg(reinterpret_cast<const float4*>(Mb + (long)j * nb + i));
      m[0] = make_float2(mv.x, mv.y);
      m[1] = make_float2(mv.z, mv.w);
    }
  };
  if (two) {
#pragma unroll 8
    for (int j = 0; j < nb; ++j) {
      cf m[RPT];
      load(j, m);
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        const cf xv = xa[j * NR + r], xw = xb[j * NR + r];
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
          A[q][r] = cfma(m[q], xv, A[q][r]);
          Bv[q][r] = cfma(m[q], xw, Bv[q][r]);
        }
      }
    }
  } else {
#pragma unroll 8
    for (int j = 0; j < nb; ++j) {
      cf m[RPT];
      load(j, m);
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        const cf xv = xa[j * NR + r];
#pragma unroll
        for (int q = 0; q < RPT; ++q) A[q][r] = cfma(m[q], xv, A[q][r]);
      }
    }
  }
  if constexpr (HALF) {
    const float s = a.scales[(hc0 + g) * 2 + (te ? 0 : 1)];
#pragma unroll
    for (int q = 0; q < RPT; ++q)
#pragma unroll
      for (int r = 0; r < NR; ++r) { A[q][r] = cscale(A[q][r], s); Bv[q][r] = cscale(Bv[q][r], s); }
  }
  __syncthreads();   // every thread has read its inputs: the outputs overwrite xs in place
  {
    // rows i .. i + RPT - 1 never straddle the t / z boundary (NZ is a multiple of RPT)
    const int comp = te ? 0 : (i < NZ ? 1 : 2);
    const int z = te ? rr : (i < NZ ? i : i - NZ);
#pragma unroll
    for (int q = 0; q < RPT; ++q)
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        xs[((g * 3 + comp) * NZ + z + q) * nrhs + r] = A[q][r];
        if (two) xs[(((g + G) * 3 + comp) * NZ + z + q) * nrhs + r] = Bv[q][r];
      }
  }
  __syncthreads();
  for (int it = tid; it < nrhs * NZ * nv; it += NT) {
    const int v = it % nv, z = (it / nv) % NZ, r = it / (nv * NZ);
    const long base = (long)r * n + (long)z * ncols + colof(v);
    const cf es = xs[((v * 3 + 0) * NZ + z) * nrhs + r], et = xs[((v * 3 + 1) * NZ + z) * nrhs + r];
    const float sx = rot[v][0], sy = rot[v][1], tx = rot[v][2], ty = rot[v][3];
    y[base] = cadd(cscale(es, sx), cscale(et, tx));
    y[base + (long)NZ * ncols] = cadd(cscale(es, sy), cscale(et, ty));
    y[base + 2L * NZ * ncols] = xs[((v * 3 + 2) * NZ + z) * nrhs + r];
  }
}

// ---------------------------------------------------------------------------------------------
// Tensor-core apply of the half-precision blocks.  For one stored block column the V vectors
// (right-hand sides x rows ky, -ky) form an nb x V complex panel, and M X is, in real arithmetic,
// A' (nb x 2nb) times B' (2nb x 2V) with the entries of M as (re, im) pairs along k -- exactly the
// stored half2 layout -- and the columns of vector v holding (Re x, -Im x) and (Im x, Re x) along
// k.  That is an f16 matrix product with FP32 accumulation (mma.sync m16n8k16, N = 8 = two output
// columns for each of four vectors).  The vector enters as a two-term f16 split: with s a power of
// two putting the column's largest entry in [2^13, 2^14), hi = f16(s x) and lo = f16(s x - hi)
// carry about 22 bits, so P stays linear to about FP32 rounding (the Krylov solvers need a fixed
// linear P) while every stored entry costs a quarter of an instruction instead of the SIMT
// kernel's four complex FMAs.
//
// One warp per (slab of 32 block rows, k range of nz): nz / 32 TE slabs and nz / 16 TM slabs x two
// k halves (the TM input's t and z parts, summed in the output).  Lane (g, t) reads 16 B = rows
// 4g .. 4g + 3 of the slab at k columns j and j + 4; the MMA row order is permuted so that those
// four rows are the fragment rows g, g + 8 of the slab's two 16-row tiles, and the k order within
// an 8-column step is the stored one.
__device__ __forceinline__ void mma_f16(float (&d)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                        unsigned b0, unsigned b1) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ unsigned h2bits(__half2 h) { return *reinterpret_cast<unsigned*>(&h); }

// 2^e for e in [-126, 127]
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }

__device__ __forceinline__ unsigned smem_u32a(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// wait for phase `parity` of an mbarrier, giving up after about max_cycles SM clocks
__device__ __forceinline__ bool mbar_wait_cycles(unsigned mb, unsigned parity, long long max_cycles) {
  const long long t0 = clock64();
  unsigned ok = 0;
  while (!ok) {
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok) : "r"(mb), "r"(parity) : "memory");
    if (!ok && clock64() - t0 > max_cycles) return false;
  }
  return true;
}

template <int NZ, int NR>
struct MmaCfg {
  static constexpr int V = 2 * NR;            // vector slots: rhs r of row h is r, of row ny - h is NR + r
  static constexpr int NT = (V + 3) / 4;      // n8 tiles (four vectors each)
  static constexpr int TES = NZ / 32;         // TE slabs
  static constexpr int TMS = NZ / 16;         // TM slabs
  static constexpr int W = TES + 2 * TMS;     // warps
  static constexpr int KT = NZ / 8;           // 8-column k steps per warp
  static constexpr int R3 = 3 * NZ;           // stacked (s, t, z) rows
  static constexpr size_t S_BYTES = (size_t)NT * R3 * 8 * sizeof(uint2);    // B' fragments (hi, lo)
  static constexpr size_t X_BYTES = (size_t)V * R3 * sizeof(cf);             // rotated x, FP32
  static constexpr size_t O_BYTES = (size_t)V * 5 * NZ * sizeof(cf);         // outputs (s, t, z + upper-k t, z)
};

// Persistent, pipelined form of the tensor-core apply.  One CTA per SM walks the stored block
// columns blockIdx.x, + gridDim.x, ...; the column's blocks stream through a ring of shared-memory
// slots of 4 nz^2 bytes (the TE block, then the TM block in four quarters of nz/2 columns each),
// filled by bulk asynchronous copies that one producer lane issues as soon as a slot is released,
// so the HBM stream never waits for the per-column work.  Two groups of worker warps take
// alternate columns: while one gathers, splits and scatters, the other multiplies.  Each worker
// warp passes every chunk of its column in order (waits until it has landed, uses it if it holds
// the warp's k range, then releases it), and prefetches the vectors of its group's next column
// into registers before the multiplications.  Every wait is bounded (about a second); the first
// that gives up sets a CTA-wide abort flag, after which nothing waits any more, no copy is issued,
// the producer waits (bounded) for the copies it issued, and the flag err[1] reports it.
template <int NZ, int NR>
struct PipeCfg {
  using M = MmaCfg<NZ, NR>;
  static constexpr int W = M::W;                                      // worker warps per group
  static constexpr int GT = 32 * W;                                   // worker threads per group
  static constexpr int THREADS = 32 + 2 * GT;                         // producer warp + two groups
  static constexpr size_t CH = (size_t)4 * NZ * NZ;                   // bytes per chunk (nz^2 half2)
  static constexpr size_t G_BYTES = M::S_BYTES + M::O_BYTES + 16 * ((M::V * sizeof(float) + 15) / 16);
  // two columns of chunks: slot 5 g + q only ever holds chunk q of group g's columns, so every
  // wait on a slot's barriers follows the same warps' wait on the previous round (the parity
  // of a phase identifies it only within one phase)
  static constexpr int RING = 10;
  static constexpr size_t SMEM = RING * CH + 2 * G_BYTES;
  static constexpr int ITEMS = NR * NZ * 2;                           // gather items per column
  static constexpr int IPT = (ITEMS + GT - 1) / GT;                   // per worker thread
  static_assert(M::X_BYTES <= M::O_BYTES, "the rotated vectors reuse the output area");
};

template <int NZ, int NR>
constexpr bool pipe_fits() { return PipeCfg<NZ, NR>::SMEM <= (size_t)227 * 1024; }

__device__ __forceinline__ void group_sync(int grp, int nthreads) {
  asm volatile("bar.sync %0, %1;" :: "r"(1 + grp), "r"(nthreads) : "memory");
}

template <int NZ, int NR>
__global__ void __launch_bounds__(PipeCfg<NZ, NR>::THREADS, 1)
    k_lay_apply_pipe(LayArgs a, const cf* __restrict__ x, cf* __restrict__ y, long ncols, long ncolsB) {
  using P = PipeCfg<NZ, NR>;
  using M = MmaCfg<NZ, NR>;
  constexpr int V = M::V, NT = M::NT, R3 = M::R3, W = P::W, RING = P::RING;
  constexpr long long WAIT = 2000000000LL;   // SM clocks, about a second
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) unsigned long long full[RING], empty[RING];
  __shared__ int abort_flag;
  __shared__ float rot[2][2][4];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const long ncta = blockIdx.x < ncolsB ? (ncolsB - 1 - blockIdx.x) / gridDim.x + 1 : 0;   // columns here
  if (tid == 0) {
    for (int s = 0; s < RING; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32a(&full[s])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32a(&empty[s])), "r"(W) : "memory");
    }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const long n = 3L * NZ * ncols;
  auto give_up = [&]() {
    if (atomicExch(&abort_flag, 1) == 0) atomicExch(a.err + 1, 1);
  };
  // ------------------------------------------------------------------ producer
  if (warp == 0) {
    if (lane == 0) {
      long issued = 0;
      for (long k = 0; k < ncta; ++k) {
        const char* src = reinterpret_cast<const char*>(a.mats16 + (blockIdx.x + k * gridDim.x) * (5L * NZ * NZ));
        for (int q = 0; q < 5; ++q) {
          const long c = 5 * k + q;
          const int slot = (int)(c % RING);
          if (c >= RING && !mbar_wait_cycles(smem_u32a(&empty[slot]), (unsigned)(((c / RING) - 1) & 1), WAIT))
            give_up();
          if (*(volatile int*)&abort_flag) break;
          if (!a.no_copy) {
            const unsigned fb = smem_u32a(&full[slot]);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(fb), "r"((unsigned)P::CH)
                         : "memory");
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                         :: "r"(smem_u32a(smem + (size_t)slot * P::CH)), "l"(src + q * P::CH), "r"((unsigned)P::CH),
                            "r"(fb)
                         : "memory");
            issued = c + 1;
          }
        }
        if (*(volatile int*)&abort_flag) break;
      }
      // leave only when every copy issued has landed (bounded)
      for (long c = issued > RING ? issued - RING : 0; c < issued; ++c)
        mbar_wait_cycles(smem_u32a(&full[c % RING]), (unsigned)((c / RING) & 1), WAIT);
    }
    return;
  }
  // ------------------------------------------------------------------ workers
  const int grp = (warp - 1) / W, w = (warp - 1) % W, gt = tid - 32 - grp * P::GT;
  unsigned char* gbase = smem + (size_t)RING * P::CH + (size_t)grp * P::G_BYTES;
  uint2* S = reinterpret_cast<uint2*>(gbase);                                  // [NT][R3][8]
  cf* O = reinterpret_cast<cf*>(gbase + M::S_BYTES);                           // [V][5 NZ]
  cf* X = O;                                                                   // [V][R3], before the MMAs
  float* isv = reinterpret_cast<float*>(gbase + M::S_BYTES + M::O_BYTES);      // [V]
  const int g = lane >> 2, t = lane & 3;
  const bool te = w < M::TES;
  const int slab = te ? w : (w - M::TES) % M::TMS, kh = te ? 0 : (w - M::TES) / M::TMS;
  const int nb = te ? NZ : 2 * NZ;
  const int jjb = te ? 0 : NZ + kh * NZ;
  // the warp's chunks: TE -> chunk 0 (all KT k steps); TM (slab, kh) -> chunks 1 + 2 kh, 2 + 2 kh
  // (KT / 2 k steps each, over the chunk's nz/2 columns of the 2nz x 2nz block)
  const int qa = te ? 0 : 1 + 2 * kh;
  constexpr int KT = M::KT;
  // prefetched vector entries of the group's next column: item it = gt + i GT -> (p, z, r)
  cf pre[P::IPT][3];
  auto fetch = [&](long k) {
    const long hc = blockIdx.x + k * gridDim.x;
    const int ix = (int)(hc % a.nx), h = (int)(hc / a.nx);
    const int iyB = a.pair ? (a.ny - h) % a.ny : h;
    const bool two = a.pair && iyB != h;
#pragma unroll
    for (int i = 0; i < P::IPT; ++i) {
      const int it = gt + i * P::GT;
      const int p = it & 1, z = (it >> 1) % NZ, r = (it >> 1) / NZ;
      if (it < P::ITEMS && !(p && !two)) {
        const long base = (long)r * n + (long)z * ncols + (long)(p ? iyB : h) * a.nx + ix;
        pre[i][0] = x[base]; pre[i][1] = x[base + (long)NZ * ncols]; pre[i][2] = x[base + 2L * NZ * ncols];
      } else {
        pre[i][0] = czero(); pre[i][1] = czero(); pre[i][2] = czero();
      }
    }
  };
  if (grp < ncta) fetch(grp);
  for (long k = grp; k < ncta; k += 2) {
    const long hc = blockIdx.x + k * gridDim.x;
    const int ix = (int)(hc % a.nx), h = (int)(hc / a.nx);
    const int iyB = a.pair ? (a.ny - h) % a.ny : h;
    const bool two = a.pair && iyB != h;
    if (gt < 2) {
      const float kx = a.kx[ix], ky = a.ky[gt == 0 ? h : iyB];
      const float kap = sqrtf(kx * kx + ky * ky);
      const bool small = !(kap > 0.f);
      rot[grp][gt][0] = small ? 0.f : -ky / kap;
      rot[grp][gt][1] = small ? 1.f : kx / kap;
      rot[grp][gt][2] = small ? 1.f : kx / kap;
      rot[grp][gt][3] = small ? 0.f : ky / kap;
    }
    group_sync(grp, P::GT);
    // 1. rotate the prefetched entries into X
#pragma unroll
    for (int i = 0; i < P::IPT; ++i) {
      const int it = gt + i * P::GT;
      if (it < P::ITEMS) {
        const int p = it & 1, z = (it >> 1) % NZ, r = (it >> 1) / NZ;
        cf* Xv = X + (p * NR + r) * R3;
        const float* q = rot[grp][p];
        Xv[z] = cadd(cscale(pre[i][0], q[0]), cscale(pre[i][1], q[1]));
        Xv[NZ + z] = cadd(cscale(pre[i][0], q[2]), cscale(pre[i][1], q[3]));
        Xv[2 * NZ + z] = pre[i][2];
      }
    }
    group_sync(grp, P::GT);
    // 2. per-vector power-of-two scale
    for (int v = w; v < V; v += W) {
      const cf* Xv = X + v * R3;
      float m = 0.f;
      for (int i = lane; i < R3; i += 32) m = fmaxf(m, fmaxf(fabsf(Xv[i].x), fabsf(Xv[i].y)));
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
      if (lane == 0) {
        int e = 0;
        if (m > 0.f && m <= 3.0e38f) frexpf(m, &e);
        isv[v] = pow2f(-min(120, max(-120, 14 - e)));
      }
    }
    group_sync(grp, P::GT);
    // 3. B' fragments
    for (int it = gt; it < NT * R3 * 8; it += P::GT) {
      const int nn = it & 7, jj = (it >> 3) % R3, nt = (it >> 3) / R3;
      const int v = 4 * nt + (nn >> 1);
      float p0 = 0.f, p1 = 0.f;
      if (v < V) {
        const float s = 1.f / isv[v];
        const cf xv = X[v * R3 + jj];
        if (nn & 1) { p0 = xv.y * s; p1 = xv.x * s; }
        else { p0 = xv.x * s; p1 = -xv.y * s; }
      }
      const __half2 hi = __floats2half2_rn(p0, p1);
      const __half2 lo = __floats2half2_rn(p0 - __low2float(hi), p1 - __high2float(hi));
      S[it] = make_uint2(h2bits(hi), h2bits(lo));
    }
    group_sync(grp, P::GT);
    // prefetch the group's next column while this one is multiplied
    if (k + 2 < ncta) fetch(k + 2);
    // 4. the chunks of this column, in order
    float acc[NT][2][4];
#pragma unroll
    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
      for (int m = 0; m < 2; ++m)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[nt][m][q] = 0.f;
    const uint2* Sb = S + (jjb + t) * 8 + g;
    for (int q = 0; q < 5; ++q) {
      const long c = 5 * k + q;
      const int slot = (int)(c % RING);
      bool ok = !*(volatile int*)&abort_flag;
      if (ok) ok = mbar_wait_cycles(smem_u32a(&full[slot]), (unsigned)((c / RING) & 1), WAIT);
      if (!ok && lane == 0) give_up();
      ok = __all_sync(0xffffffffu, ok) && !*(volatile int*)&abort_flag;
      if (ok && (q == qa || (!te && q == qa + 1))) {
        // k steps of this chunk: TE all KT from column 0; TM KT / 2 from the chunk's first column
        const int k0 = te ? 0 : (q - qa) * (KT / 2);
        const int nk = te ? KT : KT / 2;
        const uint4* Ab = reinterpret_cast<const uint4*>(
            reinterpret_cast<const __half2*>(smem + (size_t)slot * P::CH) + t * nb + slab * 32 + 4 * g);
#pragma unroll
        for (int kk = 0; kk < KT; ++kk) {
          if (kk >= nk) break;
          const uint4 aj = Ab[kk * 2 * nb];
          const uint4 aj4 = Ab[kk * 2 * nb + nb];
          const int kt = k0 + kk;
#pragma unroll
          for (int nt = 0; nt < NT; ++nt) {
            const uint2 b0 = Sb[(nt * R3 + 8 * kt) * 8], b1 = Sb[(nt * R3 + 8 * kt + 4) * 8];
            mma_f16(acc[nt][0], aj.x, aj.y, aj4.x, aj4.y, b0.x, b1.x);
            mma_f16(acc[nt][0], aj.x, aj.y, aj4.x, aj4.y, b0.y, b1.y);
            mma_f16(acc[nt][1], aj.z, aj.w, aj4.z, aj4.w, b0.x, b1.x);
            mma_f16(acc[nt][1], aj.z, aj.w, aj4.z, aj4.w, b0.y, b1.y);
          }
        }
      }
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_u32a(&empty[slot])) : "memory");
    }
    group_sync(grp, P::GT);   // X (under O) and S are no longer read
    // 5. epilogue into O, then rotate back and scatter
    {
      const float bs = a.scales[hc * 2 + (te ? 0 : 1)];
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
        const int v = 4 * nt + t;
        if (v >= V) continue;
        const float sc = bs * isv[v];
        cf* Ov = O + v * 5 * NZ + (te ? 0 : (kh == 0 ? NZ : 3 * NZ)) + slab * 32 + 4 * g;
#pragma unroll
        for (int m = 0; m < 2; ++m) {
          Ov[2 * m] = make_float2(acc[nt][m][0] * sc, acc[nt][m][1] * sc);
          Ov[2 * m + 1] = make_float2(acc[nt][m][2] * sc, acc[nt][m][3] * sc);
        }
      }
    }
    group_sync(grp, P::GT);
    for (int it = gt; it < P::ITEMS; it += P::GT) {
      const int p = it & 1, z = (it >> 1) % NZ, r = (it >> 1) / NZ;
      if (p && !two) continue;
      const cf* Ov = O + (p * NR + r) * 5 * NZ;
      const cf es = Ov[z], et = cadd(Ov[NZ + z], Ov[3 * NZ + z]), ez = cadd(Ov[2 * NZ + z], Ov[4 * NZ + z]);
      const float* rq = rot[grp][p];
      const long base = (long)r * n + (long)z * ncols + (long)(p ? iyB : h) * a.nx + ix;
      y[base] = cadd(cscale(es, rq[0]), cscale(et, rq[2]));
      y[base + (long)NZ * ncols] = cadd(cscale(es, rq[1]), cscale(et, rq[3]));
      y[base + 2L * NZ * ncols] = ez;
    }
    group_sync(grp, P::GT);   // O and rot are free for the next column
  }
}

LayArgs lay_args(psfd_plan_s* P) {
  LayArgs a{};
  a.kx = P->kx; a.ky = P->ky; a.refl = P->R.refl; a.kz0 = P->R.kz0;
  a.D = P->lay_D; a.D2 = P->lay_D2; a.deps = P->lay_deps;
  a.k0sq = (float)(P->k0 * P->k0); a.dz = (float)P->p.dz;
  a.nx = P->nx; a.ny = P->ny; a.nz = P->nz; a.zml = P->p.z_ml;
  a.pair = layered_pairs(P) ? 1 : 0;
  a.mats = P->lay; a.err = P->lay_err;
  a.mats16 = (__half2*)P->lay16; a.scales = P->lay_scale; a.half = P->lay_half ? 1 : 0;
  const char* e = getenv("PSFD_TEST_LAY_NO_COPY");
  a.no_copy = (e && e[0] == '1') ? 1 : 0;
  return a;
}

template <int NZ>
int build_nz(psfd_plan_s* P) {
  LayArgs a = lay_args(P);
  const unsigned nblk = (unsigned)layered_columns(P);
  k_lay_inv<NZ, false><<<nblk, LAY_THREADS, 0, P->stream>>>(a, 0);
  PSFD_CHECK_LAUNCH();
  k_lay_inv<2 * NZ, true><<<nblk, LAY_THREADS, 0, P->stream>>>(a, NZ * NZ);
  PSFD_CHECK_LAUNCH();
  return PSFD_OK;
}

template <int NZ, int NR>
int apply_nr(psfd_plan_s* P, const LayArgs& a, const cf* x, cf* y) {
  if constexpr (NZ % 32 == 0) {
    if (pipe_fits<NZ, NR>() && a.half && lay_apply_tc_enabled()) {
      using C = PipeCfg<NZ, NR>;
      static int nsm = 0;
      if (!nsm) {
        int dev = 0;
        PSFD_CUDA_TRY(cudaGetDevice(&dev));
        PSFD_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        PSFD_CUDA_TRY(cudaFuncSetAttribute(k_lay_apply_pipe<NZ, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)C::SMEM));
      }
      const long cols = layered_columns(P);
      const unsigned grid = (unsigned)std::min<long>(cols, nsm);
      k_lay_apply_pipe<NZ, NR><<<grid, C::THREADS, C::SMEM, P->stream>>>(a, x, y, P->ncols, cols);
      PSFD_CHECK_LAUNCH();
      return PSFD_OK;
    }
  }
  const size_t smem = (size_t)2 * LAY_GROUP * 3 * NZ * NR * sizeof(cf);
  const unsigned grid = (unsigned)(layered_columns(P) / LAY_GROUP);
  if (a.half)
    k_lay_apply<NZ, NR, true><<<grid, apply_threads<NZ, true>(), smem, P->stream>>>(a, x, y, P->ncols);
  else
    k_lay_apply<NZ, NR, false><<<grid, apply_threads<NZ, false>(), smem, P->stream>>>(a, x, y, P->ncols);
  PSFD_CHECK_LAUNCH();
  return PSFD_OK;
}

template <int NZ>
int apply_nz(psfd_plan_s* P, const cf* x, cf* y) {
  LayArgs a = lay_args(P);
  switch (P->nrhs) {
    case 1: return apply_nr<NZ, 1>(P, a, x, y);
    case 2: return apply_nr<NZ, 2>(P, a, x, y);
    case 3: return apply_nr<NZ, 3>(P, a, x, y);
    default: return apply_nr<NZ, 4>(P, a, x, y);
  }
}

}  // namespace

int layered_supported(const psfd_plan_s* P) {
  return (P->nz == 16 || P->nz == 32 || P->nz == 48 || P->nz == 64) && P->nx % LAY_GROUP == 0 && P->nrhs <= 4;
}

// ky and -ky share their blocks when there is no Bloch shift along y (the blocks depend on kappa)
bool layered_pairs(const psfd_plan_s* P) { return P->ky_inc == 0.0 && P->ny % 2 == 0; }

// number of stored block columns
long layered_columns(const psfd_plan_s* P) {
  return layered_pairs(P) ? (long)(P->ny / 2 + 1) * P->nx : P->ncols;
}

size_t layered_bytes(const psfd_plan_s* P) {
  const size_t per = (size_t)5 * P->nz * P->nz * (P->lay_half ? sizeof(__half2) : sizeof(cf));
  return (size_t)layered_columns(P) * per;
}

int layered_apply(psfd_plan_s* P, const cf* x, cf* y) {
  if (!P->lay_built) { psfd_set_error("layered preconditioner: call psfd_layered_build first"); return PSFD_ERR_STATE; }
  StageScope scope(P->stream, ST_PRECOND, (double)layered_bytes(P) + 2.0 * P->nrhs * P->nvec * sizeof(cf));
  switch (P->nz) {
    case 16: return apply_nz<16>(P, x, y);
    case 32: return apply_nz<32>(P, x, y);
    case 48: return apply_nz<48>(P, x, y);
    case 64: return apply_nz<64>(P, x, y);
    default: psfd_set_error("layered preconditioner: unsupported nz %d", P->nz); return PSFD_ERR_ARG;
  }
}

void layered_free(psfd_plan_s* P) {
  void* ptrs[] = {P->lay, P->lay_D, P->lay_D2, P->lay_deps, P->lay_err, P->lay_fmean, P->lay16, P->lay_scale};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  P->lay = nullptr; P->lay_D = nullptr; P->lay_D2 = nullptr; P->lay_deps = nullptr; P->lay_err = nullptr;
  P->lay_fmean = nullptr; P->lay16 = nullptr; P->lay_scale = nullptr;
  P->lay_built = false;
  P->lay_mean.clear();
}

// per-plane mean of the registered fill, copied to the host (synchronises the plan's stream)
static int plane_means(psfd_plan_s* P, std::vector<double>& mean) {
  cudaStream_t s = P->stream;
  if (!P->lay_fmean) PSFD_CUDA_TRY(cudaMalloc((void**)&P->lay_fmean, (size_t)P->nz * sizeof(double)));
  k_plane_mean<<<P->nz, LAY_THREADS, 0, s>>>(P->fill, P->ncols, P->lay_fmean);
  PSFD_CHECK_LAUNCH();
  mean.resize(P->nz);
  PSFD_CUDA_TRY(cudaMemcpyAsync(mean.data(), P->lay_fmean, P->nz * sizeof(double), cudaMemcpyDeviceToHost, s));
  PSFD_CUDA_TRY(cudaStreamSynchronize(s));
  return PSFD_OK;
}

extern "C" int psfd_layered_storage(psfd_plan P, int storage) {
  if (!P || (storage != PSFD_LAY_C64 && storage != PSFD_LAY_HALF)) {
    psfd_set_error("psfd_layered_storage: null plan or unknown storage");
    return PSFD_ERR_ARG;
  }
  const bool half = storage == PSFD_LAY_HALF;
  if (half != P->lay_half) {
    PSFD_CUDA_TRY(cudaStreamSynchronize(P->stream));
    layered_free(P);   // blocks are rebuilt in the new storage by the next psfd_layered_build
    P->lay_half = half;
  }
  return PSFD_OK;
}

extern "C" size_t psfd_layered_bytes(psfd_plan P) {
  if (!P || !layered_supported(P)) return 0;
  return layered_bytes(P);
}

extern "C" int psfd_layered_build(psfd_plan P) {
  if (!P) { psfd_set_error("psfd_layered_build: null plan"); return PSFD_ERR_ARG; }
  if (!P->have_background) { psfd_set_error("psfd_layered_build: call psfd_background first"); return PSFD_ERR_STATE; }
  if (!layered_supported(P)) {
    psfd_set_error("psfd_layered_build: supported for nz in {16, 32, 48, 64}, nx a multiple of 4, nrhs <= 4");
    return PSFD_ERR_ARG;
  }
  const int nz = P->nz;
  cudaStream_t s = P->stream;
  StageScope scope(s, ST_LAYBUILD);
  if (P->lay_half ? !P->lay16 : !P->lay) {
    if (P->lay_half) {
      PSFD_CUDA_TRY(cudaMalloc((void**)&P->lay16, layered_bytes(P)));
      PSFD_CUDA_TRY(cudaMalloc((void**)&P->lay_scale, (size_t)layered_columns(P) * 2 * sizeof(float)));
    } else {
      PSFD_CUDA_TRY(cudaMalloc((void**)&P->lay, layered_bytes(P)));
    }
  }
  if (!P->lay_D) {
    PSFD_CUDA_TRY(cudaMalloc((void**)&P->lay_D, (size_t)nz * nz * sizeof(cf)));
    PSFD_CUDA_TRY(cudaMalloc((void**)&P->lay_D2, (size_t)nz * nz * sizeof(cf)));
    PSFD_CUDA_TRY(cudaMalloc((void**)&P->lay_deps, (size_t)nz * sizeof(cf)));
    PSFD_CUDA_TRY(cudaMalloc((void**)&P->lay_err, 2 * sizeof(int)));   // [0] singular pivot, [1] apply wait
    PSFD_CUDA_TRY(cudaMemset(P->lay_err, 0, 2 * sizeof(int)));
    // D = s^-1 C, C[z][z'] = (1/nz) sum_m i k_m exp(2 pi i m (z - z') / nz) (FFT-order k_m, Nyquist
    // negative), and D^2, in FP64 on the host
    std::vector<zd> sinv;
    pml_sinv64(P, sinv);
    std::vector<zc> Cc(nz), D((size_t)nz * nz), D2((size_t)nz * nz, zc(0.0, 0.0));
    for (int d = 0; d < nz; ++d) {
      zc acc(0.0, 0.0);
      for (int m = 0; m < nz; ++m) {
        const double km = fft_wavenumber(m, nz, P->p.dz);
        const double ph = 2.0 * M_PI * (double)m * (double)d / (double)nz;
        acc += zc(0.0, km) * zc(cos(ph), sin(ph));
      }
      Cc[d] = acc / (double)nz;
    }
    for (int i = 0; i < nz; ++i)
      for (int j = 0; j < nz; ++j) D[(size_t)i * nz + j] = zc(sinv[i].x, sinv[i].y) * Cc[((i - j) % nz + nz) % nz];
    for (int i = 0; i < nz; ++i)
      for (int k = 0; k < nz; ++k) {
        const zc dik = D[(size_t)i * nz + k];
        for (int j = 0; j < nz; ++j) D2[(size_t)i * nz + j] += dik * D[(size_t)k * nz + j];
      }
    std::vector<cf> hD((size_t)nz * nz), hD2((size_t)nz * nz);
    for (size_t e = 0; e < hD.size(); ++e) {
      hD[e] = make_float2((float)D[e].real(), (float)D[e].imag());
      hD2[e] = make_float2((float)D2[e].real(), (float)D2[e].imag());
    }
    PSFD_CUDA_TRY(cudaMemcpy(P->lay_D, hD.data(), hD.size() * sizeof(cf), cudaMemcpyHostToDevice));
    PSFD_CUDA_TRY(cudaMemcpy(P->lay_D2, hD2.data(), hD2.size() * sizeof(cf), cudaMemcpyHostToDevice));
  }
  std::vector<double> mean;
  int rc = plane_means(P, mean);
  if (rc) return rc;
  std::vector<cf> deps(nz);
  for (int z = 0; z < nz; ++z)
    deps[z] = make_float2((float)(mean[z] * P->pc_host[z].x), (float)(mean[z] * P->pc_host[z].y));
  PSFD_CUDA_TRY(cudaMemcpyAsync(P->lay_deps, deps.data(), nz * sizeof(cf), cudaMemcpyHostToDevice, s));
  PSFD_CUDA_TRY(cudaMemsetAsync(P->lay_err, 0, sizeof(int), s));
  switch (nz) {
    case 16: rc = build_nz<16>(P); break;
    case 32: rc = build_nz<32>(P); break;
    case 48: rc = build_nz<48>(P); break;
    default: rc = build_nz<64>(P); break;
  }
  if (rc) return rc;
  int herr = 0;
  PSFD_CUDA_TRY(cudaMemcpyAsync(&herr, P->lay_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  PSFD_CUDA_TRY(cudaStreamSynchronize(s));
  if (herr) { psfd_set_error("psfd_layered_build: a column block is singular"); return PSFD_ERR_BREAKDOWN; }
  P->lay_built = true;
  P->lay_mean = mean;
  return PSFD_OK;
}

extern "C" int psfd_layered_refresh(psfd_plan P, double max_shift, int* rebuilt) {
  if (rebuilt) *rebuilt = 0;
  if (!P) { psfd_set_error("psfd_layered_refresh: null plan"); return PSFD_ERR_ARG; }
  if (!P->have_background) { psfd_set_error("psfd_layered_refresh: call psfd_background first"); return PSFD_ERR_STATE; }
  if (P->lay_built && (int)P->lay_mean.size() == P->nz) {
    std::vector<double> mean;
    int rc = plane_means(P, mean);
    if (rc) return rc;
    double shift = 0.0;
    for (int z = 0; z < P->nz; ++z) shift = std::max(shift, fabs(mean[z] - P->lay_mean[z]));
    if (shift <= max_shift) return PSFD_OK;
  }
  if (rebuilt) *rebuilt = 1;
  return psfd_layered_build(P);
}
