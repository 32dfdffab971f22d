/*
 * psfd.h - C ABI of the B300 library for the background-decomposed,
 * preconditioned pseudo-spectral frequency-domain (PSFD) solve of the
 * scattered field of a 3-D EUV mask, with a factorised-FNO warm start
 * (Kim & Gillijns, "Physics-Informed Neural Operator for Warm-Starting
 * Background-Decomposed and Preconditioned PSFD").
 *
 * Conventions shared by every call
 * --------------------------------
 * - Complex numbers are complex64, stored as interleaved (re, im) float pairs
 *   (psfd_c64).  Fields are arrays [nrhs][3][nz][ny][nx] (x fastest) holding
 *   the Bloch envelopes of (Ex, Ey, Ez): physical field = envelope *
 *   exp(i (kx_inc x + ky_inc y)).  Grid points sit at x = i dx, y = j dy,
 *   z = k dz.  Time dependence exp(-i w t); illumination comes from +z.
 * - "Real-space" arrays use that layout directly.  Arrays marked HYBRID hold
 *   the same field after the unitary lateral DFT (1/sqrt(nx ny) scaling),
 *   indexed [nrhs][3][nz][ky][kx] with kx, ky in FFT order.  Norms and inner
 *   products are the same in both domains.
 * - Every array pointer is caller-owned DEVICE memory unless the argument is
 *   documented as host memory.  Calls are asynchronous on the plan's stream
 *   unless stated otherwise; the library allocates only inside
 *   psfd_plan_create, psfd_mask_fill and psfd_background (plan-owned tables and
 *   scratch; stream-ordered temporaries freed within the call),
 *   psfd_layered_build (the blocks), on the first psfd_apply64 or refined solve
 *   of a plan (plan-owned FP64 tables), on the first BiCGSTAB solve of a plan
 *   (2 nrhs pinned, device-mapped host ints through which the kernels report
 *   their progress to the host loop), inside psfd_solve / psfd_solve_ex when the
 *   caller passes no workspace (see psfd_solve_workspace_size) and, temporarily,
 *   inside psfd_spectral_upsample.
 * - The kernels of a Krylov iteration are launched with programmatic dependent
 *   launch; each one's first instruction waits for the completion of the work
 *   before it on the stream, so stream order holds for anything the caller
 *   interleaves.
 * - Return codes: PSFD_OK (0) or one of the PSFD_ERR_* / PSFD_NOT_CONVERGED
 *   values; psfd_last_error() returns a message for the last failing call on
 *   the calling thread.  Argument errors are detected before any launch.
 * - Threads: different plans may be used from different host threads at once
 *   (a plan from one thread at a time); the library's one-time kernel set-up
 *   completes before any thread launches.
 */
#ifndef PSFD_H
#define PSFD_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define PSFD_API __attribute__((visibility("default")))
#else
#define PSFD_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { float re, im; } psfd_c64;
typedef struct psfd_plan_s* psfd_plan;

enum {
  PSFD_OK = 0,
  PSFD_ERR_ARG = 1,          /* invalid argument or unsupported size            */
  PSFD_ERR_CUDA = 2,         /* a CUDA runtime call failed                      */
  PSFD_NOT_CONVERGED = 3,    /* maxit reached before the tolerance (solve)      */
  PSFD_ERR_BREAKDOWN = 4,    /* Krylov breakdown (rho or <rhat,v> vanished)     */
  PSFD_ERR_TIMEOUT = 5,      /* a bounded device-side wait gave up              */
  PSFD_ERR_STATE = 6         /* call order violated (e.g. apply before background) */
};

enum { PSFD_TE = 0, PSFD_TM = 1 };

/* psfd_apply / psfd_precond flags */
enum {
  PSFD_PRECOND = 1,          /* apply A M instead of A                          */
  PSFD_HYBRID = 2,           /* x and y are in the HYBRID (kx, ky, z) domain    */
  PSFD_ADJOINT = 4,          /* apply A^H (or (A M)^H = M A^H with PSFD_PRECOND) */
  PSFD_LAYERED = 8           /* apply A P with the layered-background preconditioner P
                                (psfd_layered_build); not combined with ADJOINT    */
};

enum { PSFD_BICGSTAB = 0, PSFD_GMRES = 1 };

/* Problem description (lengths in nm).  Sec. 2.2 of the paper states the
 * operator; the discretisation constants it leaves to the companion PSFD
 * paper are explicit fields here. */
typedef struct {
  int nx, ny, nz;            /* grid; nx, ny, nz in {16,32,48,64,96,128,256,512}-type sizes, see psfd_supported */
  int nrhs;                  /* right-hand sides sharing this operator (e.g. TE + TM)      */
  double dx, dy, dz;         /* grid spacing                                                */
  double lambda;             /* vacuum wavelength (13.5 nm for EUV)                         */
  double theta_deg, phi_deg; /* incidence polar / azimuth angle; sets the Bloch shift       */
  int pml_planes;            /* PML thickness in planes at each z end (0 = periodic)        */
  double pml_R0;             /* nominal normal-incidence PML reflection (sets the strength) */
  double pml_backing;        /* peak loss sigma_b of the PML's absorbing backing: eps_bg = 1 + i sigma
                                on the outermost nb = max(1, pml_planes / 4) planes at each z end,
                                where the two PMLs meet across the periodic wrap, with sigma =
                                sigma_b ((nb - j) / nb)^2 on the j-th plane from the end (0 = none).
                                A z-stretch leaves fields that are constant in z untouched, so
                                without it a lateral mode near grazing keeps an undamped mode */
  int z_ml;                  /* plane index of the multilayer interface z_ml                */
  double eps_abs_re, eps_abs_im;  /* absorber permittivity; deps = fill * (eps_abs - 1)     */
  double m_min, k_ref, gamma, damp_eps_rel;  /* spectral damping (Eq. spectral_damping_mask);
                                                k_ref <= 0 means k0; eps = damp_eps_rel * k0^2 */
  double sigma_px;           /* lateral Gaussian smoothing width of the mask (pixels)       */
  void* stream;              /* cudaStream_t for every call on this plan (NULL = legacy)    */
} psfd_params_t;

/* Multilayer below z_ml, top to bottom, host memory (Sec. 3: 40 Mo/Si pairs). */
typedef struct {
  int n_layers;
  const double* n_re;        /* [n_layers] refractive index, real part  */
  const double* n_im;        /* [n_layers] imaginary part (absorbing > 0) */
  const double* d;           /* [n_layers] thickness, nm                 */
  double sub_re, sub_im;     /* substrate index                          */
} psfd_stack_t;

typedef struct {
  int iters;                 /* Krylov iterations (operator applications for GMRES)      */
  int status;                /* PSFD_OK / PSFD_NOT_CONVERGED / PSFD_ERR_BREAKDOWN          */
  double r_rel;              /* true relative residual ||b - A E|| / ||b|| (FP64), Eq. relative_residual */
  double r_rel_recursive;    /* the solver's recursive estimate at exit                   */
  double r_rel_initial;      /* ||b - A E_base|| / ||b|| before the first iteration; for a
                                refined warm start (psfd_solve_ex, refine = 1) it is formed
                                with the complex64 operator unless that estimate is already
                                at the tolerance, then with the extended-precision one     */
  int outer;                 /* outer FP64 refinement steps (psfd_solve_ex with refine)   */
  double r_rel_output;       /* FP64 relative residual of the returned complex64 field    */
} psfd_info_t;

/* ---------------------------------------------------------------- plan */

/* Create a plan: validates sizes, builds the PML profile s(z), the Bloch-shifted
 * wavenumbers, the FFT twiddle tables, and allocates plan-owned scratch.  Blocks
 * until the tables are on the device.  The multilayer reflection is computed by
 * psfd_background.  Returns PSFD_ERR_ARG for unsupported sizes. */
PSFD_API int psfd_plan_create(psfd_plan* plan, const psfd_params_t* params);
PSFD_API int psfd_plan_destroy(psfd_plan plan);

/* 1 if (n along a lateral axis, nz) is supported by the FFT kernels, else 0. */
PSFD_API int psfd_supported(int nx, int ny, int nz);

/* ---------------------------------------------------------------- geometry (Sec. 2.1 / Sec. 3)
 * a_bin: device uint8 [ny][nx], binary indicator of the absorber layout.
 * zprof: HOST float [nz], fraction of each z cell covered by the absorber.
 * fill:  device float [nz][ny][nx] (output): Gaussian-smoothed indicator
 *        (spectral, periodic, width sigma_px) times zprof[z].
 */
PSFD_API int psfd_mask_fill(psfd_plan plan, const uint8_t* a_bin, const float* zprof, float* fill);

/* ---------------------------------------------------------------- background (Eq. bg_source)
 * Computes in FP64 on the device the reflection coefficients r_s, r_p (ratios of
 * reflected to incident tangential E) of the stack for every lateral Bloch mode
 * (transfer-matrix method; recomputed only when the stack differs from the
 * previous call's, since they do not depend on the mask), registers `fill`
 * (device [nz][ny][nx], kept by
 * pointer: it must stay alive while the plan is used), and writes the source
 *   b = k0^2 deps (E_inc + R E_inc)
 * for each right-hand side r with polarisation pol[r] (HOST int array [nrhs],
 * PSFD_TE = E along s, PSFD_TM).  b: device [nrhs][3][nz][ny][nx], real space. */
PSFD_API int psfd_background(psfd_plan plan, const psfd_stack_t* stack, const float* fill,
                    const int* pol, psfd_c64* b);

/* Per-plane material contrast: deps(x, y, z) = fill(x, y, z) * c[z] with c[z] =
 * re[z] + i im[z] (HOST double arrays [nz]); NULL, NULL restores c[z] = eps_abs - 1
 * (the absorber of psfd_params_t).  With fill = 1 on the planes of a layered
 * structure and c[z] its cell-averaged eps - 1, and an empty stack (r = 0, so
 * R = 0), the operator is the standard full-domain scattered-field PSFD with
 * that structure meshed (e.g. a bare multilayer, whose specular reflection can
 * be compared with the transfer-matrix result).  Call psfd_background again
 * afterwards (the source depends on c); PSFD_ERR_ARG on a non-finite entry. */
PSFD_API int psfd_set_plane_contrast(psfd_plan plan, const double* re, const double* im);
/* The per-plane table of a layer stack meshed in the domain: layers (top to
 * bottom, refractive indices and thicknesses in nm) with the top face at height
 * z_top (nm, plane k at k dz), the stack's substrate below it down through the
 * bottom PML, vacuum above; c[z] = cell average of eps - 1 over
 * [z dz - dz/2, z dz + dz/2].  zmask (HOST float [nz], nullable) receives 1 on
 * planes with nonzero contrast (the zprof of psfd_mask_fill for fill = 1). */
PSFD_API int psfd_set_layer_stack_contrast(psfd_plan plan, const psfd_stack_t* layers, double z_top, float* zmask);

/* Copy the FP64 reflection tables to host: rs, rp, kz0 as [ny][nx] complex
 * double pairs (re, im), each array 2*nx*ny doubles.  Synchronous. */
PSFD_API int psfd_reflection_tables(psfd_plan plan, double* rs, double* rp, double* kz0);

/* ---------------------------------------------------------------- operator (Sec. 2.2)
 * y = A x with
 *   A E = curl_s curl_s E - k0^2 eps_bg E - k0^2 deps (E + R E)    (Eqs. bg_source,
 *         vector_helmholtz_operator; derivatives pseudo-spectral, PML in z;
 *         eps_bg = 1 except on the PML backing, see psfd_params_t.pml_backing)
 * flags: PSFD_PRECOND -> y = A M x (Eq. right_preconditioned);
 *        PSFD_ADJOINT -> y = A^H x (with PRECOND: M A^H x);
 *        PSFD_LAYERED -> y = A P x (P: layered-background preconditioner);
 *        PSFD_HYBRID  -> x, y in the HYBRID domain (no lateral transforms of x, y).
 * x, y: device [nrhs][3][nz][ny][nx]; x and y must not overlap. */
PSFD_API int psfd_apply(psfd_plan plan, const psfd_c64* x, psfd_c64* y, int flags);

/* y = A x in FP64, the operator of Sec. 2.2 exactly as psfd_apply defines it
 * (no preconditioner).  x, y: device complex128 arrays [nrhs][3][nz][ny][nx]
 * of interleaved (re, im) doubles, real space, or HYBRID with PSFD_HYBRID (the
 * only flag accepted; others give PSFD_ERR_ARG); x and y must not overlap.  The
 * lateral and axial transforms and the products run in double-float arithmetic
 * (about 48 significant bits) where a thread holds at most 16 points of a
 * transform, in FP64 elsewhere; the multilayer tables are the FP64 ones.  This
 * is the apply of the FP64 refinement residual of psfd_solve_ex.  The first call
 * on a plan builds the FP64 tables (plan-owned, freed with the plan) and the
 * first real-space call a plan-owned copy buffer of x. */
PSFD_API int psfd_apply64(psfd_plan plan, const double* x, double* y, int flags);

/* y = M x, spectral damping (Eq. spectral_damping_action): componentwise 3-D
 * Fourier multiplier m(k); with PSFD_LAYERED in flags, y = P x instead.
 * flags: PSFD_HYBRID, PSFD_LAYERED.  In-place (x == y) allowed. */
PSFD_API int psfd_precond(psfd_plan plan, const psfd_c64* x, psfd_c64* y, int flags);

/* ---------------------------------------------------------------- layered-background preconditioner
 * Not in the paper: an alternative right preconditioner P = A0^-1, where A0 is A
 * with the contrast replaced on every z-plane by its lateral mean
 * (deps_bar(z) = (eps_abs - 1) * mean_xy fill(z)).  A0 does not couple lateral
 * Bloch modes; per mode it splits into a TE block (nz x nz, E along s) and a TM
 * block (2nz x 2nz, (E_t, E_z)), which psfd_layered_build assembles and inverts
 * (FP32, partial pivoting) on the device and stores in the plan:
 * psfd_layered_bytes() bytes = columns * 5 nz^2 entries (2 nz^2 in the Schur form
 * below), where columns = nx*ny, or
 * nx*(ny/2+1) without a Bloch shift along y (the blocks depend on |k_par| only,
 * so ky and -ky share them): 1.36 GB at 128x128x64 at 6 deg in complex64.
 * psfd_layered_build makes the blocks exact for the fill registered by the last
 * psfd_background.  They stay usable as a preconditioner after later
 * psfd_background calls on the same plan (any fill): P only changes how fast the
 * solve converges, never the solution.  psfd_layered_refresh rebuilds them only
 * when some plane's mean fill moved by more than max_shift (fill fraction units)
 * since the last build, and sets *rebuilt (nullable) to 1 if it did.
 * With half storage and nz a multiple of 32 (nz = 64: nrhs <= 2) P is applied on
 * the tensor cores: the columns' blocks stream through shared memory in bulk
 * copies and are multiplied as f16 matrices with FP32 accumulation, the vector
 * entering as a two-term f16 split with a power-of-two scale per column (about
 * 22 bits), so P stays linear to FP32 level.  PSFD_LAY_TC=0 in the environment
 * selects the FP32 SIMT kernel.
 * For nz = 96 and 128 (and any nz in {32, 64} with PSFD_LAY_SCHUR=1) the blocks
 * are stored in the Schur form: the E_z-E_z part of the TM block is diagonal in z,
 * so E_z is eliminated and only TE^-1 and S^-1 (S the nz x nz Schur complement on
 * E_t) are stored, 2 nz^2 entries per column, always in complex64 (a half-precision
 * request applies to the full-block form only: S^-1 carries the large
 * kappa^2 D Dg^-1 D part of near-grazing columns); the apply forms the E_z part with
 * the shared stretched derivative matrix (SIMT kernel).
 * Supported for nz in {16, 32, 48, 64, 96, 128}, nx a multiple of 4 and nrhs <= 4
 * (else PSFD_ERR_ARG / psfd_layered_bytes() = 0); PSFD_ERR_STATE before
 * psfd_background; PSFD_ERR_BREAKDOWN if a block is singular.  Both synchronise
 * the plan's stream. */
PSFD_API int psfd_layered_build(psfd_plan plan);
/* Storage of the blocks, taking effect at the next build (the current blocks are
 * released): PSFD_LAY_C64 (default) complex64; PSFD_LAY_HALF complex half
 * precision, each block divided by the power of two at or above its largest
 * |re|, |im| (the scale is kept per block and applied in FP32 after the
 * product).  Half storage halves the bytes of every P apply; P changes only the
 * convergence, never the solution, and the iteration counts measured with it
 * match complex64 storage.  PSFD_ERR_ARG for an unknown storage. */
enum { PSFD_LAY_C64 = 0, PSFD_LAY_HALF = 1 };
PSFD_API int psfd_layered_storage(psfd_plan plan, int storage);
/* Form of the blocks, taking effect at the next psfd_layered_build (blocks of the
 * other form are released then): PSFD_LAY_FORM_AUTO (default) full TE / TM
 * inverses for nz <= 64 and the Schur form above; PSFD_LAY_FORM_SCHUR the Schur
 * form for every nz that is a multiple of 32 (nz 16 and 48 keep the full blocks).
 * The Schur build inverts two nz x nz blocks per column instead of an nz x nz and a
 * 2 nz x 2 nz one (about 3x faster at nz = 64), while its apply is FP32-arithmetic
 * bound (about 1.4x slower at nz = 64 than the half-precision tensor-core apply):
 * the better choice when the blocks are built for a single solve.  The environment
 * variable PSFD_LAY_SCHUR=1 requests the Schur form for every plan.  PSFD_ERR_ARG
 * for a null plan or an unknown form. */
enum { PSFD_LAY_FORM_AUTO = 0, PSFD_LAY_FORM_SCHUR = 1 };
PSFD_API int psfd_layered_form(psfd_plan plan, int form);
PSFD_API int psfd_layered_refresh(psfd_plan plan, double max_shift, int* rebuilt);
PSFD_API size_t psfd_layered_bytes(psfd_plan plan);

/* ---------------------------------------------------------------- solve (Sec. 3, warm start)
 * Solves A E = b for every right-hand side with right preconditioning and an
 * affine warm start: E = E_base + M y with A M y = b - A E_base
 * (Eqs. right_correction_solution, right_preconditioned_system); x0 = NULL is
 * the null initialisation (Eq. right_preconditioned).  use_precond: 1 = the
 * spectral damping M; 0 = identity (the paper's "null preconditioner");
 * 2 = the layered-background preconditioner P in place of M (psfd_layered_build
 * at least once on the plan, else PSFD_ERR_STATE).  Convergence: recursive
 * relative residual <= tol with ||b|| of the original b (Eq. relative_residual);
 * the true residual is recomputed in FP64 at exit.
 *   b, x0 (nullable), E: device [nrhs][3][nz][ny][nx], real space.
 *   method: PSFD_BICGSTAB (the paper's solver) or PSFD_GMRES (restart m).
 *   info: HOST array [nrhs].  Blocks until the solve has finished.
 *   workspace: device scratch of psfd_solve_workspace_size() bytes, or NULL to
 *   let the library allocate (and free) it inside the call.
 * Returns PSFD_OK when every right-hand side converged, else the worst status. */
PSFD_API int psfd_solve(psfd_plan plan, const psfd_c64* b, const psfd_c64* x0, psfd_c64* E,
               double tol, int maxit, int method, int restart, int use_precond,
               psfd_info_t* info, void* workspace, size_t workspace_bytes);
PSFD_API size_t psfd_solve_workspace_size(psfd_plan plan, int method, int restart);

/* Solve with options; refine = 1 selects mixed precision: the field is kept in
 * FP64, the outer residual b - A E is computed with an FP64 operator apply, and
 * each outer step solves A M d = r in complex64 (method, restart, preconditioner
 * as above) to the relative tolerance inner_tol (or only to 0.5 tol ||b|| / ||r||
 * when that is looser: the correction is not solved more accurately than the
 * final tolerance needs), then E += M d.  The first residual only feeds that
 * first inner solve: it is b itself for a cold start and is formed with the
 * complex64 operator for a warm start (so info.r_rel_initial of a refined warm
 * solve carries complex64 rounding); every later residual, and the convergence
 * test, use the extended-precision apply.  Convergence is
 * the FP64 relative residual <= tol (Eq. relative_residual); maxit bounds the
 * total number of inner iterations, max_outer (0 = 100) the outer steps.  The
 * returned field is the complex64 rounding of the FP64 field, or with out_c128
 * the FP64 field itself; info.r_rel_output is the returned field's own FP64
 * relative residual (rounding a field to complex64 leaves a residual of about
 * 1.3e-6 at 128x128x64, so a 1e-6 target needs out_c128 to hold in the
 * output).  refine = 0 is psfd_solve.
 * Workspace: psfd_solve_ex_workspace_size() bytes or NULL (allocated inside). */
typedef struct {
  double tol;
  int maxit;
  int method;
  int restart;
  int use_precond;
  int refine;
  double inner_tol;
  int max_outer;
  int out_c128;   /* 1: E receives the FP64 field as complex128 (double re, im) [nrhs][3][nz][ny][nx]
                     (pass a buffer of that size, cast to psfd_c64*); needs refine = 1.  0: complex64 */
} psfd_solve_opts_t;
PSFD_API int psfd_solve_ex(psfd_plan plan, const psfd_c64* b, const psfd_c64* x0, psfd_c64* E,
                           const psfd_solve_opts_t* opts, psfd_info_t* info, void* workspace,
                           size_t workspace_bytes);
PSFD_API size_t psfd_solve_ex_workspace_size(psfd_plan plan, const psfd_solve_opts_t* opts);

/* FFT tile autotuner: times every compiled lane split of the axial transforms for
 * this plan's shape (CUDA events, after psfd_background) and keeps the fastest;
 * cached per (nx, ny, nz, nrhs) for the process.  *chosen_T (nullable) receives the
 * lanes per pencil.  Synchronous. */
PSFD_API int psfd_autotune(psfd_plan plan, int* chosen_T);

/* Batched solve of independent problems (masks of different size, angles,
 * polarisations): plans[i] with its b[i], optional x0[i] (x0 may be NULL) and
 * output E[i]; every plan must have its own stream for the solves to overlap.
 * info: HOST array of sum(plans[i].nrhs) entries, in plan order.  nworkers host
 * threads (<= 0: 8) take plans in order and run psfd_solve_ex on each.  Blocks
 * until all solves finish; returns the worst status (an argument, state or CUDA
 * error of any plan is returned with that plan's index and message). */
PSFD_API int psfd_solve_batched(const psfd_plan* plans, int nplans, const psfd_c64* const* b,
                                const psfd_c64* const* x0, psfd_c64* const* E,
                                const psfd_solve_opts_t* opts, psfd_info_t* info, int nworkers);

/* Optional residual history: if set, psfd_solve writes ||r_k|| / ||b|| for every
 * iteration k < capacity and right-hand side r to hist[r * capacity + k] (HOST). */
PSFD_API int psfd_set_history(psfd_plan plan, double* hist, int capacity);

/* ---------------------------------------------------------------- physics-informed loss (Sec. 3, Eq. loss)
 * For every right-hand side a of the plan (the fill and b of the last psfd_background):
 *   J[a] = (1/N) ||r_a||^2 + (lam_hf / N) ||w(nu) F3[r_a]||^2,   r_a = A E_a - b_a,
 * N = nx ny nz, w(nu) = w0 + eta_hf |nu| with nu the 3-D DFT frequency in cycles per
 * sample (|nu| <= sqrt(3)/2, the Nyquist index counted negative), F3 the unitary 3-D
 * DFT (the paper fixes none of lam_hf, w0, eta_hf or the normalisation of F3).  grad
 * (nullable) receives dJ[a]/dRe E_a + i dJ[a]/dIm E_a =
 *   (2/N) A^H [ r_a + lam_hf F3^H (w^2 F3 r_a) ]
 * (torch's convention for the gradient of a real function of a complex tensor).
 * E, b, grad: device real-space [nrhs][3][nz][ny][nx]; grad must not overlap E or b.
 * J: HOST double [nrhs].  workspace: device scratch of
 * psfd_physics_loss_workspace_size() bytes (PSFD_ERR_ARG if smaller or NULL).  Operator
 * applies and transforms in complex64, the two sums in FP64; synchronises the plan's
 * stream.  PSFD_ERR_STATE before psfd_background. */
PSFD_API size_t psfd_physics_loss_workspace_size(psfd_plan plan);
PSFD_API int psfd_physics_loss(psfd_plan plan, const psfd_c64* E, const psfd_c64* b, double lam_hf, double w0,
                               double eta_hf, double* J, psfd_c64* grad, void* workspace, size_t workspace_bytes);

/* ---------------------------------------------------------------- factorised FNO (Sec. 2.1, Eqs. 1-5)
 * Device pointers to float32 parameters; complex kernels as psfd_c64.
 *   lift_w [dv][4], lift_b [dv]                         (inputs: a, x/Lx, y/Ly, z/Lz)
 *   kxy [L][my][mx][dv][dv]  (modes k = -m/2..m/2-1, centred order; [out][in])
 *   kz  [L][mz][dv][dv]
 *   w1 [L][dh][dv], b1 [L][dh], w2 [L][dv][dh], b2 [L][dv]
 *   q1 [dq][dv], qb1 [dq], q2 [6][dq], qb2 [6]           (6 = Re/Im of Ex, Ey, Ez)
 * Mode mixing rounds both operands to bfloat16 and accumulates in float32.
 * PSFD_MIX_FP32=1 in the environment keeps both operands in float32 instead (a
 * verification mode: the network without the bfloat16 rounding, on the SIMT
 * mixing kernel).  The pointwise layers (the MLP of Eq. 4 and the projection)
 * run on the tensor cores at FP32 accuracy (TF32 products of split operands) for
 * dv = 32, dh = 64, dq = 128; PSFD_MLP_TC=0 selects the CUDA-core kernels. */
typedef struct {
  int dv, dh, layers, mx, my, mz, dq;
  const float* lift_w; const float* lift_b;
  const psfd_c64* kxy; const psfd_c64* kz;
  const float* w1; const float* b1; const float* w2; const float* b2;
  const float* q1; const float* qb1; const float* q2; const float* qb2;
} fno_weights_t;

/* E_out = G_theta(a): a device float [B][nz][ny][nx] (smoothed indicator),
 * E_out device [B][3][nz][ny][nx] complex64.  workspace of
 * fno_workspace_size() bytes (device).  stream: cudaStream_t or NULL. */
PSFD_API size_t fno_workspace_size(const fno_weights_t* w, int B, int nx, int ny, int nz);
PSFD_API int fno_forward(const fno_weights_t* w, const float* a, int B, int nx, int ny, int nz,
                psfd_c64* E_out, void* workspace, size_t workspace_bytes, void* stream);

/* ---------------------------------------------------------------- FNO training (physics-informed, Sec. 2.2)
 * Gradient buffers of the same shapes as fno_weights_t (device, float32 /
 * complex64).  fno_backward ADDS to them, so zero them before a step.  For a
 * complex kernel entry K the gradient is dJ/dRe K + i dJ/dIm K (the convention
 * of torch's complex autograd).  The bfloat16 rounding of the mixing operands is
 * passed straight through: dK = dU conj(bf16(V)), dV = bf16(K)^H dU. */
typedef struct {
  float* lift_w; float* lift_b;
  psfd_c64* kxy; psfd_c64* kz;
  float* w1; float* b1; float* w2; float* b2;
  float* q1; float* qb1; float* q2; float* qb2;
} fno_grads_t;

/* Workspace of a training pass.  checkpoint = 0 (stored): the forward keeps,
 * per layer, the branch outputs u_xy, u_z and the retained spectra V, W
 * (Eqs. 2-3) for the backward.  checkpoint != 0 (activation checkpointing): it
 * keeps only each layer's input v_l, and the backward recomputes that layer's
 * branches first (one more forward pass of the spectral branches, about a
 * third of the memory at dv = 32).  Both give the same gradients. */
PSFD_API size_t fno_train_workspace_size(const fno_weights_t* w, int B, int nx, int ny, int nz, int checkpoint);
/* Same result as fno_forward; keeps what fno_backward needs in the workspace
 * (fno_train_workspace_size bytes for the same checkpoint flag). */
PSFD_API int fno_forward_train(const fno_weights_t* w, const float* a, int B, int nx, int ny, int nz,
                               psfd_c64* E_out, void* workspace, size_t workspace_bytes, int checkpoint,
                               void* stream);
/* Reverse pass of the fno_forward_train that last used `workspace` (same w, a,
 * sizes and checkpoint flag; w unchanged since): dE device [B][3][nz][ny][nx]
 * complex64 = dJ/dRe E + i dJ/dIm E; the gradients of every parameter are
 * added into g.  Errors: PSFD_ERR_ARG for null pointers, unsupported sizes or a
 * small workspace. */
PSFD_API int fno_backward(const fno_weights_t* w, const fno_grads_t* g, const float* a, int B, int nx, int ny,
                          int nz, const psfd_c64* dE, void* workspace, size_t workspace_bytes, int checkpoint,
                          void* stream);

/* Zero-pad the 3-D spectrum of src [nb][nz0][ny0][nx0] to dst [nb][nz][ny][nx]
 * (spectral interpolation of a coarse prediction, amplitude preserving). */
PSFD_API int psfd_spectral_upsample(const psfd_c64* src, int nb, int nx0, int ny0, int nz0,
                           psfd_c64* dst, int nx, int ny, int nz, void* stream);

/* Allocation-free variant of psfd_spectral_upsample (the paper has no
 * counterpart; it exists for callers that cannot allocate device memory inside
 * a call, e.g. while a caching allocator holds the free memory or in loops that
 * must not enter the driver's allocator).  Same arguments and result as
 * psfd_spectral_upsample.  Its scratch is one fixed device array of 2^21
 * complex64 entries (16 MiB) inside the library, held by every GPU that loads
 * the library until the process exits: requests with
 * nb*nx0*ny0*nz0 + nx0+ny0+nz0+nx+ny+nz > 2^21 return PSFD_ERR_ARG.  The call
 * allocates nothing (no cudaMalloc, no host allocation); it launches kernels
 * and issues asynchronous copies / memsets on `stream`.  All calls share the
 * scratch, so calls that may overlap on the GPU race and must be serialised.
 * The first call on each device looks up the scratch address
 * (cudaGetSymbolAddress) and caches it; make that first call before any stream
 * capture. */
PSFD_API int psfd_spectral_upsample_static(const psfd_c64* src, int nb, int nx0, int ny0, int nz0,
                                           psfd_c64* dst, int nx, int ny, int nz, void* stream);

/* ---------------------------------------------------------------- threshold-width metric (Sec. 4)
 * Practical convergence measure of the paper: intensity I = |E_comp|^2 on plane z
 * of right-hand side rhs; contour I = I_th (the S = 0.5 level of the logistic map
 * of Eq. logistic_sigmoid); min(n_lines, ny) rows and min(n_lines, nx) columns of
 * the periodic grid; threshold-bounded segment widths by linear interpolation of
 * the crossings; every segment of E_ref (the converged field) matched to the
 * segment of E whose centre lies inside it.  out (HOST double[6]) = mean, std and
 * max of |d_ref - d| * pixel / demag (nm; demag = 4 for wafer units), matched
 * count, unresolved reference segments, fraction with deviation > 1 nm.
 * E, E_ref: device real-space fields [nrhs][3][nz][ny][nx].  Synchronises the
 * plan's stream.  PSFD_ERR_ARG on bad indices. */
PSFD_API int psfd_width_metric(psfd_plan plan, const psfd_c64* E, const psfd_c64* E_ref, int rhs, int comp, int z,
                               float I_th, int n_lines, double demag, double* out);

/* ---------------------------------------------------------------- observability
 * psfd_launch_count: number of kernels this library has launched in the process.
 * psfd_timing_enable(1) starts per-stage timing with CUDA events recorded on each
 * call's stream around the launches of a stage (0 fused axial operator kernel,
 * 1 lateral contrast passes, 2 Krylov vector kernels, 3 lateral real<->HYBRID
 * transforms, 4 FNO forward and backward, 5 layered preconditioner apply,
 * 6 layered preconditioner build) and clears the totals; 0 stops it.
 * psfd_timing_read synchronises on the recorded events and returns the summed
 * milliseconds and the number of timed launches groups per stage (HOST arrays). */
PSFD_API long long psfd_launch_count(void);
PSFD_API int psfd_timing_enable(int on);
PSFD_API int psfd_timing_read(double* ms, long long* calls, int nstages);
/* As psfd_timing_read, plus the summed algorithmic bytes of each stage: the
 * compulsory reads and writes of its inputs and outputs (HOST array). */
PSFD_API int psfd_timing_read_bytes(double* ms, long long* calls, double* bytes, int nstages);

/* ---------------------------------------------------------------- misc */
/* Every wait of a kernel on its own bulk copies or tensor-core products (the
 * operator's single-pass plane kernel, the tensor-core apply of the layered P,
 * the FNO mode mixing) gives up after a
 * bounded time instead of hanging, and records that in a device flag.
 * psfd_device_status reads and clears the flags: PSFD_ERR_TIMEOUT (with a
 * message naming the kernel) if a wait gave up since the last call, else
 * PSFD_OK.  Synchronises the plan's stream.  psfd_solve and psfd_solve_ex call
 * it before they return; callers of psfd_apply, psfd_precond and fno_forward
 * call it themselves. */
PSFD_API int psfd_device_status(psfd_plan plan);
PSFD_API const char* psfd_last_error(void);
PSFD_API const char* psfd_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PSFD_H */
