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
// dense per-column matrix-vector products in the HYBRID (kx, ky, z) domain.
//
// Schur form (nz = 96, 128, where a 2nz x 2nz block no longer fits one CTA's registers; any nz
// with PSFD_LAY_SCHUR=1): the E_z-E_z block of TM is diagonal, Dg = κ² − k0² ε̄(z) with
// ε̄ = 1 + Δε̄ + i σ_b (the PML backing), so E_z is eliminated.  With B = iκ D and
// C = iκ D + c e_mlᵀ, c(z) = k0² Δε̄ κ r_p e(z) / k_z, the complement on E_t is
//     S = TM_tt − B Dg⁻¹ C = TM_tt + κ² D Dg⁻¹ D − iκ (D Dg⁻¹ c) e_mlᵀ
// and the TM solve of (u_t, u_z) is  y_t = S⁻¹ (u_t − iκ D Dg⁻¹ u_z),
// y_z = Dg⁻¹ (u_z − iκ D y_t − c y_t(z_ml)).  Only TE⁻¹ and S⁻¹ are stored (2 nz² entries per
// column); D is shared by every column and Dg, c are formed on the fly.  Used as the right
// preconditioner P in A P y = b − A E_base, E = E_base + P y, in place of the spectral damping
// M of Eq. spectral_damping_action (an addition to the paper's method: the damping alone leaves
// restarted Krylov stalling near 1e-5 at oblique incidence, where near-grazing diffraction orders
// are barely absorbed by the axial PML; the averaged operator resolves those modes exactly).
#include <mutex>
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include <cuda.h>
#include <cuda_fp16.h>

#include "internal.h"
#include "pdl.cuh"

namespace {

using zc = std::complex<double>;
constexpr int LAY_THREADS = 256;   // 16 x 16 thread grid over an N x N matrix
constexpr int LAY_GROUP = 4;       // lateral columns (consecutive kx) per apply CTA

// the half-precision blocks are applied on the tensor cores where the pipeline fits (nz a multiple
// of 32); PSFD_LAY_TC=0 selects the SIMT kernel
bool lay_apply_tc_enabled() {
  const char* e = getenv("PSFD_LAY_TC");
  return !(e && e[0] == '0');
}

struct LayArgs {
  const float* kx;
  const float* ky;
  const float4* refl;   // (r_s, r_p) per mode
  const cf* kz0;        // upgoing k_z per mode
  const cf* D;          // [nz][nz] stretched axial derivative
  const cf* DT;         // [nz][nz] its transpose (row k holds column k of D: coalesced over rows i)
  const cf* D2;         // [nz][nz] D * D
  const cf* deps;       // [nz] laterally averaged contrast
  const float* sb;      // [nz] loss sigma_b(z) of the PML backing (eps_bg = 1 + i sigma_b)
  float k0sq, dz;
  int nx, ny, nz, zml;
  int pair;             // 1: blocks stored for rows 0 .. ny/2 only (ky and -ky share them)
  cf* mats;             // [ncols][5 nz^2]: TE inverse (nz^2) then TM inverse (4 nz^2), column-major
  __half2* mats16;      // the same in half precision (storage 1), entries divided by the block's scale,
                        // each block laid out by half_pos
  float* scales;        // [ncols][2] power-of-two scale of the TE and TM block (storage 1)
  int half;             // 1: half-precision storage
  int* err;             // [0] set to 1 if a pivot vanished, [1] if an apply gave up waiting for its blocks
  int no_copy;          // test of the bounded wait: the tensor-core apply requests no blocks
  const int* done;      // nullable [nrhs]: the apply does nothing when every right-hand side is done
  int nrhs;
  int schur;            // 1: per column TE^-1 then S^-1 (2 nz^2 entries, the TM block reduced to its
                        // Schur complement on E_t); 0: TE^-1 then the TM inverse (5 nz^2 entries)
};

// entries stored per block column
__host__ __device__ __forceinline__ long block_stride(const LayArgs& a) {
  return (a.schur ? 2L : 5L) * a.nz * a.nz;
}

// 1 when every right-hand side of the solve is done (the whole block returns, before any copy)
__device__ __forceinline__ bool all_done(const LayArgs& a) {
  if (!a.done) return false;
  for (int r = 0; r < a.nrhs; ++r)
    if (!a.done[r]) return false;
  return true;
}

// Half-precision block layout: column-major, with the 16-byte chunks of four rows permuted
// within each column by an XOR with 2 (j mod 4) when the block size is a multiple of 32, so
// that the tensor-core apply's fragment reads (lanes at columns j .. j + 3, same row chunk) fall
// in distinct shared-memory banks.  Half2 index of entry (i, j) of an nb x nb block:
__host__ __device__ __forceinline__ int half_pos(int i, int j, int nb) {
  return (nb % 32 == 0) ? j * nb + ((((i >> 2) ^ (2 * (j & 3))) << 2) | (i & 3)) : j * nb + i;
}

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
    if (i == j) v = cadd(v, make_float2(m.kap2 - a.k0sq * (1.f + de.x), -a.k0sq * (de.y + a.sb[i])));
    if (j == a.zml && i >= a.zml) v = csub(v, cscale(cmul(cmul(de, m.rs), upgoing(a, m, i)), a.k0sq));
    return v;
  }
  const int bi = i / nz, bj = j / nz, ii = i - bi * nz, jj = j - bj * nz;
  const cf de = a.deps[ii];
  if (bi == 0 && bj == 0) {
    cf v = cneg(a.D2[ii * nz + jj]);
    if (ii == jj) v = cadd(v, make_float2(-a.k0sq * (1.f + de.x), -a.k0sq * (de.y + a.sb[ii])));
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
  if (ii == jj) return make_float2(m.kap2 - a.k0sq * (1.f + de.x), -a.k0sq * (de.y + a.sb[ii]));
  return czero();
}

// Assemble and invert one N x N block per CTA.  Thread (rg, cg) of the RG x 16 grid owns rows
// rg + RG u and columns cg + 16 v (u < N/RG, v < N/16).  Step k exchanges the roles of x_k and y_p for
// the pivot row p (largest |T[p][k]| among rows not yet used):
//     T[p][k] <- 1/π,  T[p][j] <- −T[p][j]/π,  T[i][k] <- T[i][k]/π,  T[i][j] <- T[i][j] − T[i][k] T[p][j]/π
// with π = T[p][k].  After N steps, row p_k holds x_k and column k' holds y_{p_k'}:
// Minv[k][p_k'] = T[p_k][k'].
template <int N, bool TM, bool SCHUR = false, int RG = 16>
__global__ void __launch_bounds__(RG * 16) k_lay_inv(LayArgs a, int block_off) {
  // thread grid RG x 16 over the N x N matrix: thread (rg, cg) owns rows rg + RG u and columns
  // cg + 16 v, a TU x TV complex tile in registers
  constexpr int NTH = RG * 16, TU = N / RG, TV = N / 16;
  static_assert(TU * RG == N && TV * 16 == N && TU <= 32, "tile");
  __shared__ cf colv[2][N], rowv[2][N];
  __shared__ float mag[2][N];
  __shared__ int pivrow[N], rowvar[N];
  const long col = blockIdx.x;
  const int tid = threadIdx.x, rg = tid >> 4, cg = tid & 15, lane = tid & 31;
  const Mode m = mode_of(a, col);
  cf T[TU][TV];
  if constexpr (SCHUR) {
    // S = TM_tt + κ² D Dg⁻¹ D − iκ (D Dg⁻¹ c) e_mlᵀ (N = nz); Dg⁻¹ and Dg⁻¹ c in shared memory
    cf* gs = colv[0];
    cf* gc = rowv[0];
    for (int z = tid; z < N; z += NTH) {
      const cf de = a.deps[z];
      const cf dg = make_float2(m.kap2 - a.k0sq * (1.f + de.x), -a.k0sq * (de.y + a.sb[z]));
      const cf g = cdiv1(dg);
      gs[z] = g;
      cf c = czero();
      if (z >= a.zml) c = cscale(cmul(cmul(de, m.rp), cmul(upgoing(a, m, z), cdiv1(m.kz))), a.k0sq * m.kap);
      gc[z] = cmul(g, c);
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < TU; ++u)
#pragma unroll
      for (int v = 0; v < TV; ++v) T[u][v] = entry<false>(a, m, rg + RG * u, cg + 16 * v);
    // the TE entry carries κ² on the diagonal, TM_tt does not
#pragma unroll
    for (int u = 0; u < TU; ++u)
#pragma unroll
      for (int v = 0; v < TV; ++v)
        if (rg + RG * u == cg + 16 * v) T[u][v].x -= m.kap2;
    // TE uses r_s in its reflection column where TM_tt uses r_p
    {
      const int jm = a.zml;
#pragma unroll
      for (int v = 0; v < TV; ++v) {
        if (cg + 16 * v != jm) continue;
#pragma unroll
        for (int u = 0; u < TU; ++u) {
          const int i = rg + RG * u;
          if (i < a.zml) continue;
          const cf e = cscale(cmul(a.deps[i], upgoing(a, m, i)), a.k0sq);
          T[u][v] = cadd(T[u][v], csub(cmul(e, m.rs), cmul(e, m.rp)));
        }
      }
    }
    const cf ik = make_float2(0.f, -m.kap);   // −iκ
    for (int k = 0; k < N; ++k) {
      const cf g = gs[k];
      cf dik[TU], dkj[TV];
#pragma unroll
      for (int u = 0; u < TU; ++u) dik[u] = __ldg(a.D + (long)(rg + RG * u) * N + k);
#pragma unroll
      for (int v = 0; v < TV; ++v) dkj[v] = cscale(cmul(g, __ldg(a.D + (long)k * N + cg + 16 * v)), m.kap2);
#pragma unroll
      for (int u = 0; u < TU; ++u)
#pragma unroll
        for (int v = 0; v < TV; ++v) T[u][v] = cfma(dik[u], dkj[v], T[u][v]);
      const cf gck = cmul(ik, gc[k]);
#pragma unroll
      for (int v = 0; v < TV; ++v) {
        if (cg + 16 * v != a.zml) continue;
#pragma unroll
        for (int u = 0; u < TU; ++u) T[u][v] = cfma(dik[u], gck, T[u][v]);
      }
    }
    __syncthreads();   // colv / rowv are reused by the elimination below
  } else {
#pragma unroll
    for (int u = 0; u < TU; ++u)
#pragma unroll
      for (int v = 0; v < TV; ++v) T[u][v] = entry<TM>(a, m, rg + RG * u, cg + 16 * v);
  }
  unsigned used = 0;   // bit u: owned row rg + RG u has been a pivot row
  for (int k = 0; k < N; ++k) {
    const int buf = k & 1;
    // column k -> shared (owners: cg == k % 16); used rows get magnitude -1 and a non-finite
    // magnitude counts as 0, so the pivot is always a row not used before
    if (cg == (k & 15)) {
      const int vk = k >> 4;
#pragma unroll
      for (int v = 0; v < TV; ++v) {
        if (v != vk) continue;   // static register indexing: select the column by predicate
#pragma unroll
        for (int u = 0; u < TU; ++u) {
          const int i = rg + RG * u;
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
    // pivot row p -> shared (owners: rg == p % RG)
    if (rg == (p % RG)) {
      const int up = p / RG;
      used |= 1u << up;
#pragma unroll
      for (int u = 0; u < TU; ++u) {
        if (u != up) continue;
#pragma unroll
        for (int v = 0; v < TV; ++v) rowv[buf][cg + 16 * v] = T[u][v];
      }
    }
    __syncthreads();
    cf ci[TU], rj[TV];
#pragma unroll
    for (int u = 0; u < TU; ++u) ci[u] = cmul(colv[buf][rg + RG * u], pinv);
#pragma unroll
    for (int v = 0; v < TV; ++v) rj[v] = rowv[buf][cg + 16 * v];
    // rank-1 update of every owned entry; the pivot row and column are overwritten below
#pragma unroll
    for (int u = 0; u < TU; ++u)
#pragma unroll
      for (int v = 0; v < TV; ++v) T[u][v] = csub(T[u][v], cmul(ci[u], rj[v]));
    const bool own_row = rg == (p % RG), own_col = cg == (k & 15);
    const int up = p / RG, vk = k >> 4;
    if (own_row) {
#pragma unroll
      for (int u = 0; u < TU; ++u) {
        if (u != up) continue;
#pragma unroll
        for (int v = 0; v < TV; ++v) T[u][v] = cneg(cmul(rj[v], pinv));
      }
    }
    if (own_col) {
#pragma unroll
      for (int v = 0; v < TV; ++v) {
        if (v != vk) continue;
#pragma unroll
        for (int u = 0; u < TU; ++u) T[u][v] = (own_row && u == up) ? pinv : ci[u];
      }
    }
  }
  __syncthreads();
  // pivrow is a permutation: each step picks a row not used before
  for (int k = tid; k < N; k += NTH) rowvar[pivrow[k]] = k;
  __syncthreads();
  // column-major output: element (r, c) of the inverse at c * N + r
  if (!a.half) {
    cf* out = a.mats + col * block_stride(a) + block_off;
#pragma unroll
    for (int u = 0; u < TU; ++u)
#pragma unroll
      for (int v = 0; v < TV; ++v) {
        const int r = rowvar[rg + RG * u], c = pivrow[cg + 16 * v];
        out[(long)c * N + r] = T[u][v];
      }
    return;
  }
  // half precision: divide by the power of two at or above the block's largest |re|, |im| (the
  // entries then lie in [-1, 1], where half keeps 11 significant bits)
  float mx = 0.f;
#pragma unroll
  for (int u = 0; u < TU; ++u)
#pragma unroll
    for (int v = 0; v < TV; ++v) mx = fmaxf(mx, fmaxf(fabsf(T[u][v].x), fabsf(T[u][v].y)));
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  __shared__ float wmax[NTH / 32];
  if (lane == 0) wmax[tid >> 5] = mx;
  __syncthreads();
  mx = 0.f;
  for (int w = 0; w < NTH / 32; ++w) mx = fmaxf(mx, wmax[w]);
  int e = 0;
  if (mx > 0.f && mx <= 3.0e38f) frexpf(mx, &e);   // mx = f 2^e with f in [0.5, 1)
  const float scale = ldexpf(1.f, e), inv = ldexpf(1.f, -e);
  if (tid == 0) a.scales[col * 2 + ((TM || SCHUR) ? 1 : 0)] = scale;
  __half2* out = a.mats16 + col * block_stride(a) + block_off;
#pragma unroll
  for (int u = 0; u < TU; ++u)
#pragma unroll
    for (int v = 0; v < TV; ++v) {
      const int r = rowvar[rg + RG * u], c = pivrow[cg + 16 * v];
      out[half_pos(r, c, N)] = __floats2half2_rn(T[u][v].x * inv, T[u][v].y * inv);
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
  pdl_enter();
  if (all_done(a)) return;
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
  const long MS = block_stride(a);
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
      const uint4 hv = __ldg(reinterpret_cast<const uint4*>(Mh + half_pos(i, j, nb)));   // rows i .. i + 3
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

// Schur-form apply (blocks TE^-1 and S^-1 per column, see the top of this file):
//   y_s = TE^-1 u_s,  w = u_t - i kappa D (Dg^-1 u_z),  y_t = S^-1 w,
//   y_z = Dg^-1 (u_z - i kappa D y_t - c y_t(z_ml)).
// Same CTA layout as k_lay_apply (LAY_GROUP kx columns of row h and of its partner row, every
// right-hand side); the products with the shared derivative matrix D run one output row per
// thread over every vector of the CTA, the block products as in k_lay_apply on 2 NZ stacked rows.
template <int NZ, bool HALF>
constexpr int schur_threads() { return LAY_GROUP * 2 * NZ / apply_rpt<HALF>(); }

template <int NZ, int NR, bool HALF>
__global__ void __launch_bounds__(schur_threads<NZ, HALF>())
    k_lay_apply_schur(LayArgs a, const cf* __restrict__ x, cf* __restrict__ y, long ncols) {
  pdl_enter();
  if (all_done(a)) return;
  constexpr int G = LAY_GROUP, NT = schur_threads<NZ, HALF>(), RPT = apply_rpt<HALF>();
  static_assert(NT >= NZ && NT % NZ == 0, "whole groups of NZ threads in the D products");
  extern __shared__ cf sh[];
  cf* xs = sh;                                   // [2G][3][NZ][NR] (s, t, z) after rotation
  cf* ws = xs + 2 * G * 3 * NZ * NR;             // [2G][NZ][NR]   w
  cf* gs = ws + 2 * G * NZ * NR;                 // [G][NZ]        Dg^-1
  cf* cs = gs + G * NZ;                          // [G][NZ]        c
  __shared__ float rot[2 * G][4];
  __shared__ float kapv[G];
  const long hc0 = (long)blockIdx.x * G;
  const int ix0 = (int)(hc0 % a.nx), h = (int)(hc0 / a.nx);
  const int ny = a.ny;
  const int iyB = a.pair ? (ny - h) % ny : h;
  const bool two = a.pair && iyB != h;
  const int nv = two ? 2 * G : G;
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
  // Dg^-1 and c of each block column (both rows of a pair share kappa, r_p and k_z)
  for (int it = tid; it < G * NZ; it += NT) {
    const int g = it / NZ, z = it - g * NZ;
    const Mode m = mode_of(a, hc0 + g);
    if (z == 0) kapv[g] = m.kap;
    const cf de = a.deps[z];
    const cf gz = cdiv1(make_float2(m.kap2 - a.k0sq * (1.f + de.x), -a.k0sq * (de.y + a.sb[z])));
    gs[it] = gz;
    cs[it] = (z >= a.zml) ? cscale(cmul(cmul(de, m.rp), cmul(upgoing(a, m, z), cdiv1(m.kz))), a.k0sq * m.kap)
                          : czero();
  }
  __syncthreads();
  const long n = 3L * NZ * ncols;
  auto colof = [&](int v) -> long { return (long)(v < G ? h : iyB) * a.nx + ix0 + (v % G); };
  for (int it = tid; it < NR * NZ * nv; it += NT) {
    const int v = it % nv, z = (it / nv) % NZ, r = it / (nv * NZ);
    const long base = (long)r * n + (long)z * ncols + colof(v);
    const cf ex = x[base], ey = x[base + (long)NZ * ncols], ez = x[base + 2L * NZ * ncols];
    const float sx = rot[v][0], sy = rot[v][1], tx = rot[v][2], ty = rot[v][3];
    xs[((v * 3 + 0) * NZ + z) * NR + r] = cadd(cscale(ex, sx), cscale(ey, sy));
    xs[((v * 3 + 1) * NZ + z) * NR + r] = cadd(cscale(ex, tx), cscale(ey, ty));
    xs[((v * 3 + 2) * NZ + z) * NR + r] = cmul(gs[(v % G) * NZ + z], ez);   // Dg^-1 u_z
  }
  __syncthreads();
  // w = u_t - i kappa D (Dg^-1 u_z): thread (group q, row i) owns output row i of the vectors
  // v = q, q + NG, ... (NG = NT / NZ groups share the virtual columns)
  constexpr int NG = NT / NZ, VPG = (2 * G + NG - 1) / NG;
  const int grp = tid / NZ, irow = tid - (tid / NZ) * NZ;
  if (grp < NG) {
    cf acc[VPG][NR];
#pragma unroll
    for (int u = 0; u < VPG; ++u)
#pragma unroll
      for (int r = 0; r < NR; ++r) acc[u][r] = czero();
#pragma unroll 8
    for (int k = 0; k < NZ; ++k) {
      const cf d = __ldg(a.DT + (long)k * NZ + irow);
#pragma unroll
      for (int u = 0; u < VPG; ++u) {
        const int v = grp + NG * u;
        if (v >= nv) continue;
#pragma unroll
        for (int r = 0; r < NR; ++r) acc[u][r] = cfma(d, xs[((v * 3 + 2) * NZ + k) * NR + r], acc[u][r]);
      }
    }
#pragma unroll
    for (int u = 0; u < VPG; ++u) {
      const int v = grp + NG * u;
      if (v >= nv) continue;
      const cf mik = make_float2(0.f, -kapv[v % G]);
#pragma unroll
      for (int r = 0; r < NR; ++r)
        ws[(v * NZ + irow) * NR + r] = cfma(mik, acc[u][r], xs[((v * 3 + 1) * NZ + irow) * NR + r]);
    }
  }
  __syncthreads();
  // block products: thread -> (block column g, rows rr .. rr + RPT - 1 of [TE; S])
  {
    constexpr long NN = (long)NZ * NZ;
    constexpr int TPC = 2 * NZ / RPT;
    const int g = tid / TPC, rr = RPT * (tid - g * TPC);
    const bool te = rr < NZ;
    const int i = te ? rr : rr - NZ;
    const long MS = block_stride(a);
    const cf* Mb = a.mats + (hc0 + g) * MS + (te ? 0 : NN);
    const __half2* Mh = a.mats16 + (hc0 + g) * MS + (te ? 0 : NN);
    const cf* xa = te ? xs + (g * 3) * NZ * NR : ws + g * NZ * NR;
    const cf* xb = te ? xs + ((g + G) * 3) * NZ * NR : ws + (g + G) * NZ * NR;
    cf A[RPT][NR], Bv[RPT][NR];
#pragma unroll
    for (int q = 0; q < RPT; ++q)
#pragma unroll
      for (int r = 0; r < NR; ++r) { A[q][r] = czero(); Bv[q][r] = czero(); }
    auto load = [&](int j, cf (&m)[RPT]) {
      if constexpr (HALF) {
        const uint4 hv = __ldg(reinterpret_cast<const uint4*>(Mh + half_pos(i, j, NZ)));
        m[0] = __half22float2(*reinterpret_cast<const __half2*>(&hv.x));
        m[1] = __half22float2(*reinterpret_cast<const __half2*>(&hv.y));
        m[2] = __half22float2(*reinterpret_cast<const __half2*>(&hv.z));
        m[3] = __half22float2(*reinterpret_cast<const __half2*>(&hv.w));
      } else {
        const float4 mv = __ldg(reinterpret_cast<const float4*>(Mb + (long)j * NZ + i));
        m[0] = make_float2(mv.x, mv.y);
        m[1] = make_float2(mv.z, mv.w);
      }
    };
#pragma unroll 4
    for (int j = 0; j < NZ; ++j) {
      cf mm[RPT];
      load(j, mm);
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        const cf xv = xa[j * NR + r];
        const cf xw = two ? xb[j * NR + r] : czero();
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
          A[q][r] = cfma(mm[q], xv, A[q][r]);
          Bv[q][r] = cfma(mm[q], xw, Bv[q][r]);
        }
      }
    }
    if constexpr (HALF) {
      const float sc = a.scales[(hc0 + g) * 2 + (te ? 0 : 1)];
#pragma unroll
      for (int q = 0; q < RPT; ++q)
#pragma unroll
        for (int r = 0; r < NR; ++r) { A[q][r] = cscale(A[q][r], sc); Bv[q][r] = cscale(Bv[q][r], sc); }
    }
    __syncthreads();   // every thread has read u_s and w: y_s, y_t overwrite components 0 and 1
    const int comp = te ? 0 : 1;
#pragma unroll
    for (int q = 0; q < RPT; ++q)
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        xs[((g * 3 + comp) * NZ + i + q) * NR + r] = A[q][r];
        if (two) xs[(((g + G) * 3 + comp) * NZ + i + q) * NR + r] = Bv[q][r];
      }
  }
  __syncthreads();
  // y_z = Dg^-1 (u_z - i kappa D y_t - c y_t(z_ml)): thread (group q, row i) as above
  cf acc[VPG][NR];
#pragma unroll
  for (int u = 0; u < VPG; ++u)
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[u][r] = czero();
  if (grp < NG) {
#pragma unroll 8
    for (int k = 0; k < NZ; ++k) {
      const cf d = __ldg(a.DT + (long)k * NZ + irow);
#pragma unroll
      for (int u = 0; u < VPG; ++u) {
        const int v = grp + NG * u;
        if (v >= nv) continue;
#pragma unroll
        for (int r = 0; r < NR; ++r) acc[u][r] = cfma(d, xs[((v * 3 + 1) * NZ + k) * NR + r], acc[u][r]);
      }
    }
#pragma unroll
    for (int u = 0; u < VPG; ++u) {
      const int v = grp + NG * u;
      if (v >= nv) continue;
      const int g = v % G;
      const cf mik = make_float2(0.f, -kapv[g]);
      const cf gi = gs[g * NZ + irow], ci = cs[g * NZ + irow];
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        // y_z = Dg^-1 u_z + Dg^-1 (-i kappa D y_t - c y_t(z_ml)), the first term stored by the gather
        const cf ytm = xs[((v * 3 + 1) * NZ + a.zml) * NR + r];
        const cf t = csub(cmul(mik, acc[u][r]), cmul(ci, ytm));
        acc[u][r] = cfma(gi, t, xs[((v * 3 + 2) * NZ + irow) * NR + r]);
      }
    }
  }
  __syncthreads();   // every row's reads of u_z and y_t are done
  if (grp < NG) {
#pragma unroll
    for (int u = 0; u < VPG; ++u) {
      const int v = grp + NG * u;
      if (v >= nv) continue;
#pragma unroll
      for (int r = 0; r < NR; ++r) xs[((v * 3 + 2) * NZ + irow) * NR + r] = acc[u][r];
    }
  }
  __syncthreads();
  for (int it = tid; it < NR * NZ * nv; it += NT) {
    const int v = it % nv, z = (it / nv) % NZ, r = it / (nv * NZ);
    const long base = (long)r * n + (long)z * ncols + colof(v);
    const cf es = xs[((v * 3 + 0) * NZ + z) * NR + r], et = xs[((v * 3 + 1) * NZ + z) * NR + r];
    const float sx = rot[v][0], sy = rot[v][1], tx = rot[v][2], ty = rot[v][3];
    y[base] = cadd(cscale(es, sx), cscale(et, tx));
    y[base + (long)NZ * ncols] = cadd(cscale(es, sy), cscale(et, ty));
    y[base + 2L * NZ * ncols] = xs[((v * 3 + 2) * NZ + z) * NR + r];
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
  static constexpr int TES = NZ / 32;         // TE slabs (warps) per column
  static constexpr int TMS = NZ / 16;         // TM slabs (warps) per column
  static constexpr int CW = TES + TMS;        // warps per column
  static constexpr int KT = NZ / 8;           // 8-column k steps of a TE block
  static constexpr int R3 = 3 * NZ;           // stacked (s, t, z) rows
  static constexpr int VS = 4 * NT;           // vector slots of the B' operand (unused ones zero)
  static constexpr int R3S = R3 + 4;          // row stride of the split vectors (16 B rows; 64 mod 128 B)
  static constexpr int R3O = R3 + 1;          // row stride of the products (8 B rows; 8 mod 128 B)
};

// Persistent, pipelined form of the tensor-core apply.  One CTA per SM walks pairs of stored
// block columns (kx, kx + 1 of one row; blockIdx.x, + gridDim.x, ...).  The blocks stream through
// a ring of ten shared-memory slots of 4 nz^2 bytes (per column: the TE block, then the TM block
// in four quarters of nz/2 columns), filled by bulk asynchronous copies that one producer lane
// issues as soon as a slot is released, so the HBM stream never waits for the per-pair work.
// The vectors move as tensor-memory-access boxes (2 kx x 1 row x nz x 3 components x nrhs, 16 B
// rows): the next pair's boxes are loaded while this pair is multiplied, and the result box is
// stored from the same buffer, so neither touches the load/store pipe that the fragment reads
// use.  Six warps per column (nz = 64: two TE slabs over 8 k steps, four TM slabs over 16): both
// columns of a pair are multiplied at once, and slot 5 c + q only ever holds chunk q of column c
// of a pair, consumed by the same warps every round (the parity of a phase identifies it only
// within one phase).  Every wait is bounded (about a second); the first that gives up sets a
// CTA-wide abort flag, after which nothing waits any more and no copy is issued, every copy
// issued is waited for (bounded) before its issuer leaves, and err[1] reports it.
template <int NZ, int NR>
struct PipeCfg {
  using M = MmaCfg<NZ, NR>;
  static constexpr int WW = 2 * M::CW;                                // worker warps
  static constexpr int WT = 32 * WW;                                  // worker threads
  static constexpr int THREADS = 32 + WT;                             // + producer warp
  static constexpr size_t CH = (size_t)4 * NZ * NZ;                   // bytes per chunk (nz^2 half2)
  static constexpr int RING = 10;                                     // one pair of columns
  static constexpr size_t BOX = (size_t)2 * NZ * 3 * NR * sizeof(cf); // one row's vector box
  static constexpr int NBUF = 2;                                      // box buffers (pairs k, k + 1)
  static constexpr size_t XT_OFF = RING * CH;                         // [NBUF][2 rows] boxes
  static constexpr size_t XS_OFF = XT_OFF + 2 * NBUF * BOX;           // [2 cols][VS][R3S] uint4
  static constexpr size_t O_OFF = XS_OFF + (size_t)2 * M::VS * M::R3S * sizeof(uint4);   // [2][V][R3O]
  static constexpr size_t IS_OFF = O_OFF + (size_t)2 * M::V * M::R3O * sizeof(cf);       // [2][V] 1 / s
  static constexpr size_t SMEM = IS_OFF + 2 * M::V * sizeof(float);
  static constexpr int ITEMS = 2 * 2 * NR * NZ;                       // (col, row, rhs, z) per pair
};

template <int NZ, int NR>
constexpr bool pipe_fits() { return PipeCfg<NZ, NR>::SMEM <= (size_t)227 * 1024; }

__device__ __forceinline__ void group_sync(int nthreads) {
  asm volatile("bar.sync 1, %0;" :: "r"(nthreads) : "memory");
}

template <int NZ, int NR>
__global__ void __launch_bounds__(PipeCfg<NZ, NR>::THREADS, 1)
    k_lay_apply_pipe(LayArgs a, const __grid_constant__ CUtensorMap tx, const __grid_constant__ CUtensorMap ty,
                     long npairs) {
  pdl_enter();
  if (all_done(a)) return;
  using P = PipeCfg<NZ, NR>;
  using M = MmaCfg<NZ, NR>;
  constexpr int V = M::V, NT = M::NT, R3 = M::R3, VS = M::VS, R3S = M::R3S, R3O = M::R3O, CW = M::CW;
  constexpr int RING = P::RING;
  constexpr long long WAIT = 2000000000LL;   // SM clocks, about a second
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) unsigned long long full[RING], empty[RING], xfull[P::NBUF];
  __shared__ int abort_flag;
  __shared__ float rot[2][2][4];   // [col][row] sx, sy, tx, ty
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const long npc = blockIdx.x < npairs ? (npairs - 1 - blockIdx.x) / gridDim.x + 1 : 0;   // pairs here
  if (tid == 0) {
    for (int s = 0; s < RING; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32a(&full[s])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32a(&empty[s])), "r"(CW) : "memory");
    }
    for (int b = 0; b < P::NBUF; ++b)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32a(&xfull[b])) : "memory");
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  auto aborted = [&]() { return *(volatile int*)&abort_flag != 0; };
  auto give_up = [&]() {
    if (atomicExch(&abort_flag, 1) == 0) atomicExch(a.err + 1, 1);
  };
  // ------------------------------------------------------------------ producer
  if (warp == 0) {
    if (lane == 0) {
      long issued = 0;   // chunks c = 10 k + 5 col + q
      for (long k = 0; k < npc && !aborted(); ++k) {
        const char* src = reinterpret_cast<const char*>(a.mats16 + 2 * (blockIdx.x + k * gridDim.x) * (5L * NZ * NZ));
        for (int sl = 0; sl < RING; ++sl) {
          if (k > 0 && !mbar_wait_cycles(smem_u32a(&empty[sl]), (unsigned)((k - 1) & 1), WAIT)) give_up();
          if (aborted()) break;
          if (!a.no_copy) {
            const unsigned fb = smem_u32a(&full[sl]);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(fb), "r"((unsigned)P::CH)
                         : "memory");
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                         :: "r"(smem_u32a(smem + (size_t)sl * P::CH)), "l"(src + sl * P::CH), "r"((unsigned)P::CH),
                            "r"(fb)
                         : "memory");
            issued = 10 * k + sl + 1;
          }
        }
      }
      // leave only when every copy issued has landed (bounded)
      for (long c = issued > RING ? issued - RING : 0; c < issued; ++c)
        mbar_wait_cycles(smem_u32a(&full[c % RING]), (unsigned)((c / RING) & 1), WAIT);
    }
    return;
  }
  // ------------------------------------------------------------------ workers
  const int wt = tid - 32, ww = warp - 1;
  const bool leader = wt == 0;
  // split vectors: entry (col, v, jj) = {hi, lo} of (Re w, -Im w), then {hi, lo} of (Im w, Re w),
  // w = s x the rotated, scaled entry; lane (g, t) of an MMA warp reads the half with o = g & 1
  uint4* XS = reinterpret_cast<uint4*>(smem + P::XS_OFF);
  cf* O = reinterpret_cast<cf*>(smem + P::O_OFF);       // [2][V][R3O] products
  float* isv = reinterpret_cast<float*>(smem + P::IS_OFF);
  auto xtile = [&](int b, int p) { return reinterpret_cast<cf*>(smem + P::XT_OFF + (size_t)(2 * b + p) * P::BOX); };
  auto pair_rows = [&](long k, int& ix0, int& h, int& iyB, bool& two) {
    const long hc = 2 * (blockIdx.x + k * gridDim.x);
    ix0 = (int)(hc % a.nx); h = (int)(hc / a.nx);
    iyB = a.pair ? (a.ny - h) % a.ny : h;
    two = a.pair && iyB != h;
  };
  // the leader loads pair k's vector boxes into buffer k % NBUF
  long xissued = 0;   // boxes requested: pair index + 1
  auto load_boxes = [&](long k) {
    int ix0, h, iyB; bool two;
    pair_rows(k, ix0, h, iyB, two);
    const int b = (int)(k % P::NBUF);
    const unsigned mb = smem_u32a(&xfull[b]);
    const unsigned bytes = (unsigned)((two ? 2 : 1) * P::BOX);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(mb), "r"(bytes) : "memory");
    for (int p = 0; p < (two ? 2 : 1); ++p)
      asm volatile("cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                   " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];"
                   :: "r"(smem_u32a(xtile(b, p))), "l"(reinterpret_cast<const void*>(&tx)), "r"(ix0),
                      "r"(p ? iyB : h), "r"(0), "r"(0), "r"(0), "r"(mb)
                   : "memory");
    xissued = k + 1;
  };
  if (leader && npc > 0 && !a.no_copy) load_boxes(0);
  if constexpr (VS > V) {   // slots past the vectors stay zero
    for (int i = wt; i < 2 * (VS - V) * R3S; i += P::WT) {
      const int c = i / ((VS - V) * R3S), e = i % ((VS - V) * R3S);
      XS[(c * VS + V) * R3S + e] = make_uint4(0u, 0u, 0u, 0u);
    }
  }
  // this warp's column and slab
  const int col = ww / CW, cw = ww % CW;
  const bool te = cw < M::TES;
  const int slab = te ? cw : cw - M::TES;
  const int nb = te ? NZ : 2 * NZ;
  const int g = lane >> 2, t = lane & 3;
  const int q0 = te ? 0 : 1, nq = te ? 1 : 4;               // chunks: TE 0; TM 1 .. 4
  constexpr int KQ_TE = NZ / 8, KQ_TM = NZ / 16;            // 8-column k steps per chunk
  for (long k = 0; k < npc; ++k) {
    int ix0, h, iyB; bool two;
    pair_rows(k, ix0, h, iyB, two);
    const int b = (int)(k % P::NBUF);
    const float bs = a.scales[(2 * (blockIdx.x + k * gridDim.x) + col) * 2 + (te ? 0 : 1)];   // used in step 4
    if (wt < 4) {   // rotation of (col, row) = (wt & 1, wt >> 1)
      const int c = wt & 1, p = wt >> 1;
      const float kx = a.kx[ix0 + c], ky = a.ky[p ? iyB : h];
      const float kap = sqrtf(kx * kx + ky * ky);
      const bool small = !(kap > 0.f);
      rot[c][p][0] = small ? 0.f : -ky / kap;
      rot[c][p][1] = small ? 1.f : kx / kap;
      rot[c][p][2] = small ? 1.f : kx / kap;
      rot[c][p][3] = small ? 0.f : ky / kap;
    }
    // this pair's boxes
    bool ok = !aborted() && !a.no_copy;
    if (ok) ok = mbar_wait_cycles(smem_u32a(&xfull[b]), (unsigned)((k / P::NBUF) & 1), WAIT);
    if (!ok && !a.no_copy && !aborted()) give_up();
    group_sync(P::WT);
    // 1. per-vector power-of-two scale from the raw entries: a rotated entry is at most sqrt 2
    //    times the largest raw one (|sx| + |sy| <= sqrt 2), so s puts the rotated vector below
    //    2^14 and its largest entry at or above 2^12 (one bit of the split at most is lost)
    for (int cv = ww; cv < 2 * V; cv += P::WW) {
      const int c = cv / V, v = cv % V, p = v / NR, r = v % NR;
      float m = 0.f;
      if (!(p && !two)) {
        const cf* bx = xtile(b, p);
        for (int i = lane; i < R3; i += 32) {
          const cf e = bx[((r * 3 + i / NZ) * NZ + i % NZ) * 2 + c];
          m = fmaxf(m, fmaxf(fabsf(e.x), fabsf(e.y)));
        }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
      if (lane == 0) {
        const float mb = m * 1.41421356f;
        int e = 0;
        if (mb > 0.f && mb <= 3.0e38f) frexpf(mb, &e);   // mb = f 2^e, f in [0.5, 1)
        isv[cv] = pow2f(-min(120, max(-120, 14 - e)));     // s mb in [2^13, 2^14)
      }
    }
    group_sync(P::WT);
    // 2. rotate, scale and split into XS: item (c, p, r, z)
    for (int it = wt; it < P::ITEMS; it += P::WT) {
      const int z = it % NZ, r = (it / NZ) % NR, p = (it / (NZ * NR)) & 1, c = it / (NZ * NR * 2);
      const int v = p * NR + r;
      uint4* Xv = XS + (c * VS + v) * R3S;
      if (p && !two) {
        Xv[z] = Xv[NZ + z] = Xv[2 * NZ + z] = make_uint4(0u, 0u, 0u, 0u);
        continue;
      }
      const cf* bx = xtile(b, p);
      const cf ex = bx[((r * 3 + 0) * NZ + z) * 2 + c], ey = bx[((r * 3 + 1) * NZ + z) * 2 + c];
      const cf ez = bx[((r * 3 + 2) * NZ + z) * 2 + c];
      const float* q = rot[c][p];
      const float sc = 1.f / isv[c * V + v];
      const cf w[3] = {cscale(cadd(cscale(ex, q[0]), cscale(ey, q[1])), sc),
                       cscale(cadd(cscale(ex, q[2]), cscale(ey, q[3])), sc), cscale(ez, sc)};
#pragma unroll
      for (int comp = 0; comp < 3; ++comp) {
        const __half hr = __float2half_rn(w[comp].x), hm = __float2half_rn(w[comp].y);
        const __half lr = __float2half_rn(w[comp].x - __half2float(hr));
        const __half lm = __float2half_rn(w[comp].y - __half2float(hm));
        Xv[comp * NZ + z] = make_uint4(h2bits(__halves2half2(hr, __hneg(hm))), h2bits(__halves2half2(lr, __hneg(lm))),
                                       h2bits(__halves2half2(hm, hr)), h2bits(__halves2half2(lm, lr)));
      }
    }
    group_sync(P::WT);
    // 3. multiply this warp's slab of its column: chunks q0 .. q0 + nq - 1 of slots 5 col + q
    // four independent accumulations per tile (hi and lo products, even and odd k steps), summed
    // at the end, so consecutive MMAs do not wait on each other
    float acc[NT][2][4][4];
#pragma unroll
    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
      for (int m = 0; m < 2; ++m)
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int e = 0; e < 4; ++e) acc[nt][m][u][e] = 0.f;
    // B' columns of lane (g, t): n = g -> vector 4 nt + g / 2, (re, im) part g & 1: the (hi, lo)
    // pair at uint2 2 (row index) + (g & 1) of XS
    const uint2* Xg[NT];
#pragma unroll
    for (int nt = 0; nt < NT; ++nt)
      Xg[nt] = reinterpret_cast<const uint2*>(XS + (col * VS + 4 * nt + (g >> 1)) * R3S + (te ? 0 : NZ) + t) + (g & 1);
    for (int qq = 0; qq < 5; ++qq) {
      const int sl = col * 5 + qq;
      bool okc = !aborted();
      if (okc) okc = mbar_wait_cycles(smem_u32a(&full[sl]), (unsigned)(k & 1), WAIT);
      if (!okc && lane == 0) give_up();
      okc = __all_sync(0xffffffffu, okc) && !aborted();
      if (okc && qq >= q0 && qq < q0 + nq) {
        const int kq = te ? KQ_TE : KQ_TM;
        const int kbase = te ? 0 : (qq - 1) * KQ_TM;         // first 8-column step of this chunk
        // lane (g, t): rows 4g .. 4g + 3 of the slab (chunk g ^ 2t of 4 rows), columns 8 kk + t, + 4
        const uint4* Ab = reinterpret_cast<const uint4*>(
            reinterpret_cast<const __half2*>(smem + (size_t)sl * P::CH) + t * nb + slab * 32 + 4 * (g ^ (2 * t)));
#pragma unroll 2
        for (int k2 = 0; k2 < kq; k2 += 2) {
#pragma unroll
          for (int par = 0; par < 2; ++par) {
            const int kk = k2 + par;
            const uint4 aj = Ab[kk * 2 * nb];
            const uint4 aj4 = Ab[kk * 2 * nb + nb];
            const int j = 8 * (kbase + kk);
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) {
              const uint2 b0 = Xg[nt][2 * j], b1 = Xg[nt][2 * (j + 4)];
              mma_f16(acc[nt][0][2 * par], aj.x, aj.y, aj4.x, aj4.y, b0.x, b1.x);
              mma_f16(acc[nt][0][2 * par + 1], aj.x, aj.y, aj4.x, aj4.y, b0.y, b1.y);
              mma_f16(acc[nt][1][2 * par], aj.z, aj.w, aj4.z, aj4.w, b0.x, b1.x);
              mma_f16(acc[nt][1][2 * par + 1], aj.z, aj.w, aj4.z, aj4.w, b0.y, b1.y);
            }
          }
        }
      }
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_u32a(&empty[sl])) : "memory");
    }
    // the next pair's boxes go to the other buffer, once pair k - 1's store (issued a whole
    // multiplication ago) has read it
    if (leader && k + 1 < npc && !aborted() && !a.no_copy) {
      asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
      load_boxes(k + 1);
    }
    // 4. products into O (rows of the stacked s, t, z vector): lane (g, t) holds vector 4 nt + t
    //    at slab rows 4g + 2m (c0, c1) and 4g + 2m + 1 (c2, c3)
    {
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
        const int v = 4 * nt + t;
        if (v >= V) continue;
        const float sc = bs * isv[col * V + v];
        cf* Ov = O + (col * V + v) * R3O + (te ? 0 : NZ) + slab * 32 + 4 * g;
#pragma unroll
        for (int m = 0; m < 2; ++m) {
          float f[4];
#pragma unroll
          for (int e = 0; e < 4; ++e)
            f[e] = (acc[nt][m][0][e] + acc[nt][m][2][e]) + (acc[nt][m][1][e] + acc[nt][m][3][e]);
          Ov[2 * m] = make_float2(f[0] * sc, f[1] * sc);
          Ov[2 * m + 1] = make_float2(f[2] * sc, f[3] * sc);
        }
      }
    }
    group_sync(P::WT);
    // 5. rotate back into the box buffer b (its input was consumed in step 1) and store it
    for (int it = wt; it < P::ITEMS; it += P::WT) {
      const int z = it % NZ, r = (it / NZ) % NR, p = (it / (NZ * NR)) & 1, c = it / (NZ * NR * 2);
      if (p && !two) continue;
      const cf* Ov = O + (c * V + p * NR + r) * R3O;
      const cf es = Ov[z], et = Ov[NZ + z], ez = Ov[2 * NZ + z];
      const float* q = rot[c][p];
      cf* by = xtile(b, p);
      by[((r * 3 + 0) * NZ + z) * 2 + c] = cadd(cscale(es, q[0]), cscale(et, q[2]));
      by[((r * 3 + 1) * NZ + z) * 2 + c] = cadd(cscale(es, q[1]), cscale(et, q[3]));
      by[((r * 3 + 2) * NZ + z) * 2 + c] = ez;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic writes -> tensor store
    group_sync(P::WT);
    if (leader && !aborted()) {
      for (int p = 0; p < (two ? 2 : 1); ++p)
        asm volatile("cp.async.bulk.tensor.5d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3, %4, %5}], [%6];"
                     :: "l"(reinterpret_cast<const void*>(&ty)), "r"(ix0), "r"(p ? iyB : h), "r"(0), "r"(0), "r"(0),
                        "r"(smem_u32a(xtile(b, p)))
                     : "memory");
      asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    }
  }
  if (leader) {
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");   // stores complete before the CTA leaves
    // boxes requested but not consumed (abort): wait for them (bounded)
    if (xissued > 0)
      mbar_wait_cycles(smem_u32a(&xfull[(xissued - 1) % P::NBUF]), (unsigned)(((xissued - 1) / P::NBUF) & 1), WAIT);
  }
}

// Tensor map of a vector [nrhs][3][nz][ny][nx] (complex64, as 8-byte elements) with boxes of
// 2 kx x 1 row x nz x 3 x nrhs; false if the driver entry point is missing or the encoding is
// refused (an address not 16-byte aligned), in which case the SIMT apply runs.
bool vector_box_map(const psfd_plan_s* P, int nz, int nrhs, const void* base, CUtensorMap* m) {
  using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static Encode enc = nullptr;
  static std::once_flag once;   // the batched solve calls this from several host threads
  std::call_once(once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      enc = reinterpret_cast<Encode>(fn);
  });
  if (!enc || (reinterpret_cast<uintptr_t>(base) & 15)) return false;
  const cuuint64_t e = sizeof(cf);
  const cuuint64_t dims[5] = {(cuuint64_t)P->nx, (cuuint64_t)P->ny, (cuuint64_t)nz, 3, (cuuint64_t)nrhs};
  const cuuint64_t strides[4] = {e * P->nx, e * P->ncols, e * P->ncols * nz, e * P->ncols * nz * 3};
  const cuuint32_t box[5] = {2, 1, (cuuint32_t)nz, 3, (cuuint32_t)nrhs};
  const cuuint32_t es[5] = {1, 1, 1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 5, const_cast<void*>(base), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

LayArgs lay_args(psfd_plan_s* P) {
  LayArgs a{};
  a.kx = P->kx; a.ky = P->ky; a.refl = P->R.refl; a.kz0 = P->R.kz0;
  a.D = P->lay_D; a.DT = P->lay_DT; a.D2 = P->lay_D2; a.deps = P->lay_deps;
  a.k0sq = (float)(P->k0 * P->k0); a.dz = (float)P->p.dz; a.sb = P->sback;
  a.nx = P->nx; a.ny = P->ny; a.nz = P->nz; a.zml = P->p.z_ml;
  a.pair = layered_pairs(P) ? 1 : 0;
  a.mats = P->lay; a.err = P->lay_err;
  a.mats16 = (__half2*)P->lay16; a.scales = P->lay_scale; a.half = layered_half(P) ? 1 : 0;
  a.schur = P->lay_schur ? 1 : 0;
  const char* e = getenv("PSFD_TEST_LAY_NO_COPY");
  a.no_copy = (e && e[0] == '1') ? 1 : 0;
  return a;
}

// rows of the inversion's thread grid: 32 x 16 threads (16 warps) for blocks of 128, whose
// 16 x 16 version held an 8 x 8 tile per thread at one CTA (8 warps) per SM (measured: 14.2 -> 12.9 ms
// per build at 128x128x64; at 96 the 16 x 16 grid is faster, 11.6 against 16.9 ms at 128x128x96)
constexpr int lay_rg(int n) { return n == 128 ? 32 : 16; }

template <int NZ>
int build_nz(psfd_plan_s* P) {
  LayArgs a = lay_args(P);
  const unsigned nblk = (unsigned)layered_columns(P);
  k_lay_inv<NZ, false, false, lay_rg(NZ)><<<nblk, 16 * lay_rg(NZ), 0, P->stream>>>(a, 0);
  PSFD_CHECK_LAUNCH();
  if (a.schur) {
    if constexpr (NZ % 32 == 0) {
      k_lay_inv<NZ, false, true, lay_rg(NZ)><<<nblk, 16 * lay_rg(NZ), 0, P->stream>>>(a, NZ * NZ);
    } else {
      psfd_set_error("layered preconditioner: the Schur form is built for nz in {32, 64, 96, 128}");
      return PSFD_ERR_ARG;
    }
  } else {
    if constexpr (2 * NZ <= 128) {
      k_lay_inv<2 * NZ, true, false, lay_rg(2 * NZ)><<<nblk, 16 * lay_rg(2 * NZ), 0, P->stream>>>(a, NZ * NZ);
    } else {
      psfd_set_error("layered preconditioner: nz %d needs the Schur form", NZ);
      return PSFD_ERR_ARG;
    }
  }
  PSFD_CHECK_LAUNCH();
  return PSFD_OK;
}

template <int NZ, int NR>
int apply_schur_nr(psfd_plan_s* P, const LayArgs& a, const cf* x, cf* y) {
  const size_t smem = (size_t)(2 * LAY_GROUP * 3 * NZ * NR + 2 * LAY_GROUP * NZ * NR + 2 * LAY_GROUP * NZ) * sizeof(cf);
  const unsigned grid = (unsigned)(layered_columns(P) / LAY_GROUP);
  if (a.half) {
    PSFD_CUDA_TRY(cudaFuncSetAttribute(k_lay_apply_schur<NZ, NR, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem));
    (void)launch_pdl(k_lay_apply_schur<NZ, NR, true>, dim3(grid), dim3(schur_threads<NZ, true>()), smem, P->stream, a, x,
                     y, P->ncols);
  } else {
    PSFD_CUDA_TRY(cudaFuncSetAttribute(k_lay_apply_schur<NZ, NR, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem));
    (void)launch_pdl(k_lay_apply_schur<NZ, NR, false>, dim3(grid), dim3(schur_threads<NZ, false>()), smem, P->stream, a,
                     x, y, P->ncols);
  }
  PSFD_CHECK_LAUNCH();
  return PSFD_OK;
}

template <int NZ, int NR>
int apply_nr(psfd_plan_s* P, const LayArgs& a, const cf* x, cf* y) {
  if constexpr (NZ % 32 == 0) {
    if (pipe_fits<NZ, NR>() && a.half && lay_apply_tc_enabled()) {
      using C = PipeCfg<NZ, NR>;
      CUtensorMap tx, ty;
      if (vector_box_map(P, NZ, NR, x, &tx) && vector_box_map(P, NZ, NR, y, &ty)) {
        // once per instantiation and process, complete before any thread launches (the batched
        // solve applies P from several host threads)
        static std::once_flag once;
        static int nsm = 0;
        static cudaError_t init = cudaSuccess;
        std::call_once(once, [] {
          int dev = 0;
          init = cudaGetDevice(&dev);
          if (init == cudaSuccess) init = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
          if (init == cudaSuccess)
            init = cudaFuncSetAttribute(k_lay_apply_pipe<NZ, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)C::SMEM);
        });
        if (init != cudaSuccess || nsm <= 0) {
          psfd_set_error("layered apply: set-up of the tensor-core pipeline: %s", cudaGetErrorString(init));
          return PSFD_ERR_CUDA;
        }
        const long npairs = layered_columns(P) / 2;
        const unsigned grid = (unsigned)std::min<long>(npairs, nsm);
        (void)launch_pdl(k_lay_apply_pipe<NZ, NR>, dim3(grid), dim3(C::THREADS), (size_t)C::SMEM, P->stream, a, tx, ty,
                         npairs);
        PSFD_CHECK_LAUNCH();
        return PSFD_OK;
      }
    }
  }
  const size_t smem = (size_t)2 * LAY_GROUP * 3 * NZ * NR * sizeof(cf);
  const unsigned grid = (unsigned)(layered_columns(P) / LAY_GROUP);
  if (a.half)
    (void)launch_pdl(k_lay_apply<NZ, NR, true>, dim3(grid), dim3(apply_threads<NZ, true>()), smem, P->stream, a, x, y,
                     P->ncols);
  else
    (void)launch_pdl(k_lay_apply<NZ, NR, false>, dim3(grid), dim3(apply_threads<NZ, false>()), smem, P->stream, a, x, y,
                     P->ncols);
  PSFD_CHECK_LAUNCH();
  return PSFD_OK;
}

template <int NZ>
int apply_nz(psfd_plan_s* P, const cf* x, cf* y, const int* done) {
  LayArgs a = lay_args(P);
  a.done = done;
  a.nrhs = P->nrhs;
  if (a.schur) {
    if constexpr (NZ % 32 == 0) {
      switch (P->nrhs) {
        case 1: return apply_schur_nr<NZ, 1>(P, a, x, y);
        case 2: return apply_schur_nr<NZ, 2>(P, a, x, y);
        case 3: return apply_schur_nr<NZ, 3>(P, a, x, y);
        default: return apply_schur_nr<NZ, 4>(P, a, x, y);
      }
    }
    psfd_set_error("layered preconditioner: the Schur form is built for nz in {32, 64, 96, 128}");
    return PSFD_ERR_ARG;
  }
  if constexpr (NZ <= 64) {
    switch (P->nrhs) {
      case 1: return apply_nr<NZ, 1>(P, a, x, y);
      case 2: return apply_nr<NZ, 2>(P, a, x, y);
      case 3: return apply_nr<NZ, 3>(P, a, x, y);
      default: return apply_nr<NZ, 4>(P, a, x, y);
    }
  }
  psfd_set_error("layered preconditioner: nz %d needs the Schur form", NZ);
  return PSFD_ERR_ARG;
}

}  // namespace

int layered_supported(const psfd_plan_s* P) {
  return (P->nz == 16 || P->nz == 32 || P->nz == 48 || P->nz == 64 || P->nz == 96 || P->nz == 128) &&
         P->nx % LAY_GROUP == 0 && P->nrhs <= 4;
}

// half-precision storage in effect: requested, and not the Schur form (S^-1 carries the large
// kappa^2 D Dg^-1 D part near grazing, and an 11-bit mantissa measured 3e-2 off the complex64
// apply, with some 256^2 x 96 solves diverging; its blocks stay complex64)
bool layered_half(const psfd_plan_s* P) { return P->lay_half && !P->lay_schur; }

// the Schur form for nz above 64 (a 2 nz x 2 nz TM block no longer fits one CTA's registers), and
// for nz a multiple of 32 when the plan asks for it (psfd_layered_form) or PSFD_LAY_SCHUR=1
bool layered_schur_for(const psfd_plan_s* P) {
  const char* e = getenv("PSFD_LAY_SCHUR");
  const bool asked = P->lay_form == PSFD_LAY_FORM_SCHUR || (e && e[0] == '1');
  return P->nz > 64 || (asked && P->nz % 32 == 0);
}

// ky and -ky share their blocks when there is no Bloch shift along y (the blocks depend on kappa)
bool layered_pairs(const psfd_plan_s* P) { return P->ky_inc == 0.0 && P->ny % 2 == 0; }

// number of stored block columns
long layered_columns(const psfd_plan_s* P) {
  return layered_pairs(P) ? (long)(P->ny / 2 + 1) * P->nx : P->ncols;
}

size_t layered_bytes(const psfd_plan_s* P) {
  const size_t per = (size_t)(P->lay_schur ? 2 : 5) * P->nz * P->nz * (layered_half(P) ? sizeof(__half2) : sizeof(cf));
  return (size_t)layered_columns(P) * per;
}

int layered_apply(psfd_plan_s* P, const cf* x, cf* y, const int* done) {
  if (!P->lay_built) { psfd_set_error("layered preconditioner: call psfd_layered_build first"); return PSFD_ERR_STATE; }
  StageScope scope(P->stream, ST_PRECOND, (double)layered_bytes(P) + 2.0 * P->nrhs * P->nvec * sizeof(cf));
  switch (P->nz) {
    case 16: return apply_nz<16>(P, x, y, done);
    case 32: return apply_nz<32>(P, x, y, done);
    case 48: return apply_nz<48>(P, x, y, done);
    case 64: return apply_nz<64>(P, x, y, done);
    case 96: return apply_nz<96>(P, x, y, done);
    case 128: return apply_nz<128>(P, x, y, done);
    default: psfd_set_error("layered preconditioner: unsupported nz %d", P->nz); return PSFD_ERR_ARG;
  }
}

void layered_free(psfd_plan_s* P) {
  void* ptrs[] = {P->lay, P->lay_D, P->lay_DT, P->lay_D2, P->lay_deps, P->lay_err, P->lay_fmean, P->lay16,
                  P->lay_scale};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  P->lay = nullptr; P->lay_D = nullptr; P->lay_DT = nullptr; P->lay_D2 = nullptr; P->lay_deps = nullptr;
  P->lay_err = nullptr;
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

extern "C" int psfd_layered_form(psfd_plan P, int form) {
  if (!P || (form != PSFD_LAY_FORM_AUTO && form != PSFD_LAY_FORM_SCHUR)) {
    psfd_set_error("psfd_layered_form: null plan or unknown form");
    return PSFD_ERR_ARG;
  }
  P->lay_form = form;   // the next psfd_layered_build releases blocks of the other form
  return PSFD_OK;
}

extern "C" size_t psfd_layered_bytes(psfd_plan P) {
  if (!P || !layered_supported(P)) return 0;
  const bool built_form = P->lay_schur;
  P->lay_schur = (P->lay || P->lay16) ? built_form : layered_schur_for(P);
  const size_t b = layered_bytes(P);
  P->lay_schur = built_form;
  return b;
}

extern "C" int psfd_layered_build(psfd_plan P) {
  if (!P) { psfd_set_error("psfd_layered_build: null plan"); return PSFD_ERR_ARG; }
  if (!P->have_background) { psfd_set_error("psfd_layered_build: call psfd_background first"); return PSFD_ERR_STATE; }
  if (!layered_supported(P)) {
    psfd_set_error("psfd_layered_build: supported for nz in {16, 32, 48, 64, 96, 128}, nx a multiple of 4, "
                   "nrhs <= 4");
    return PSFD_ERR_ARG;
  }
  const int nz = P->nz;
  cudaStream_t s = P->stream;
  StageScope scope(s, ST_LAYBUILD);
  if (layered_schur_for(P) != P->lay_schur) {
    // the block form changes the storage: release the blocks, keep the storage precision
    PSFD_CUDA_TRY(cudaStreamSynchronize(s));
    layered_free(P);
    P->lay_schur = layered_schur_for(P);
  }
  if (layered_half(P) ? !P->lay16 : !P->lay) {
    if (layered_half(P)) {
      PSFD_CUDA_TRY(cudaMalloc((void**)&P->lay16, layered_bytes(P)));
      PSFD_CUDA_TRY(cudaMalloc((void**)&P->lay_scale, (size_t)layered_columns(P) * 2 * sizeof(float)));
    } else {
      PSFD_CUDA_TRY(cudaMalloc((void**)&P->lay, layered_bytes(P)));
    }
  }
  if (!P->lay_D) {
    PSFD_CUDA_TRY(cudaMalloc((void**)&P->lay_D, (size_t)nz * nz * sizeof(cf)));
    PSFD_CUDA_TRY(cudaMalloc((void**)&P->lay_DT, (size_t)nz * nz * sizeof(cf)));
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
    std::vector<cf> hD((size_t)nz * nz), hDT((size_t)nz * nz), hD2((size_t)nz * nz);
    for (size_t e = 0; e < hD.size(); ++e) {
      hD[e] = make_float2((float)D[e].real(), (float)D[e].imag());
      hD2[e] = make_float2((float)D2[e].real(), (float)D2[e].imag());
    }
    for (int i = 0; i < nz; ++i)
      for (int k = 0; k < nz; ++k) hDT[(size_t)k * nz + i] = hD[(size_t)i * nz + k];
    PSFD_CUDA_TRY(cudaMemcpy(P->lay_D, hD.data(), hD.size() * sizeof(cf), cudaMemcpyHostToDevice));
    PSFD_CUDA_TRY(cudaMemcpy(P->lay_DT, hDT.data(), hDT.size() * sizeof(cf), cudaMemcpyHostToDevice));
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
    case 64: rc = build_nz<64>(P); break;
    case 96: rc = build_nz<96>(P); break;
    default: rc = build_nz<128>(P); break;
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
