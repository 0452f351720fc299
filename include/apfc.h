/*
 * apfc.h - C ABI of the GB300 library for the semi-implicit time step of the
 * amplitude expansion of the phase-field crystal model (APFC).
 *
 * Method: Praetorius, Salvalaglio, Voigt, "An efficient numerical framework
 * for the amplitude expansion of the phase-field crystal model",
 * arXiv:1902.09761.
 *
 *   Model (Sec. II, Eqs. energyamplitude, amplitudetime, gs), standard
 *   parameters (dB, Bx, t, v) = (2 a1, a0, a3, 4 a2 / 3):
 *     d eta_j/dt = -|k_j|^2 [ (dB + Bx G_j^2) eta_j + N_j(eta) ],
 *     G_j = Laplacian + 2i k_j . grad.
 *   Space: uniform periodic grid, second-order central differences
 *   (G_h = L_h + 2i k_j . D_h), replacing the paper's P1 finite elements.
 *   Time (Alg. 1, one nonlinear iterate, nonlinear term explicit): per
 *   amplitude the split block system of Eq. linear_system2 with M = I,
 *     [ I             -G_h              ] [zeta]   [ 0                      ]
 *     [ kap Bx G_h    (1/dt + kap dB) I ] [eta ] = [ eta^n/dt - kap N(eta^n) ]
 *   solved by a Krylov method right-preconditioned with the factorised
 *   Schur-complement preconditioner of Eq. preconditioner (Sec. II.B), whose
 *   diffusion solves are Chebyshev polynomials of a stencil.
 *
 * Every entry point returns an apfc_status and never aborts.  Errors are
 * sticky on a context: after a failure, apfc_last_error() describes it and
 * calls that advance the state refuse to run until apfc_set_amplitudes()
 * resets the context.
 *
 * Buffers: complex numbers are interleaved (re, im) doubles (complex128).
 * "where" says whether a caller pointer is host (APFC_HOST) or device
 * (APFC_DEVICE) memory.  The caller owns every buffer it passes; the library
 * copies in or out and keeps no caller pointer.  Device copies run on the
 * context's stream; every call that takes "where" returns after its copies
 * have completed.
 *
 * Field layout: amplitude arrays are [J][nz][ny][nx] (x fastest).  Block
 * vectors (the unknowns (zeta_j, eta_j) of the block system) are
 * [J][2][nz][ny][nx]: for amplitude j first the zeta-part, then the eta-part.
 *
 * Threading: one context per stream; calls on one context must not overlap.
 */
#ifndef APFC_H
#define APFC_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct apfc_ctx apfc_ctx;

typedef enum {
  APFC_OK = 0,
  APFC_EINVAL = 1,  /* bad argument; nothing was changed                          */
  APFC_ENOMEM = 2,  /* device or host allocation failed                           */
  APFC_ECUDA = 3,   /* a CUDA call failed; see apfc_last_error                    */
  APFC_ENOCONV = 4, /* Krylov solve hit max_iter; the best iterate is kept        */
  APFC_ENAN = 5,    /* a residual norm became NaN/Inf (e.g. NaN amplitudes)       */
  APFC_ESTATE = 6,  /* context is in a failed state or has no amplitudes yet      */
  APFC_ETOOBIG = 7  /* problem exceeds the fixed scratch of the no-allocation entry point */
} apfc_status;

enum { APFC_HOST = 0, APFC_DEVICE = 1 };

/* Element type of an amplitude buffer of apfc_set_amplitudes / apfc_get_amplitudes:
 * complex128 (interleaved doubles) or complex64 (interleaved floats; converted
 * on the device to and from the FP64 state, rounding to nearest on the way out). */
enum { APFC_C128 = 0, APFC_C64 = 1 };

/* Lattices.  HEX2D: triangular lattice, J = 3, dim = 2, k_1 + k_2 + k_3 = 0,
 * nonlinear term in the closed form of Sec. II.  BCC3D / CUSTOM: the nonlinear
 * term is generated from k by keeping the resonant (zero-sum) wavevector
 * combinations of the cell-averaged density powers <n^3>, <n^4>, with
 * n = sum_j (eta_j e^{i k_j.r} + c.c.) (Eq. density). */
enum { APFC_LATTICE_CUSTOM = 0, APFC_LATTICE_HEX2D = 1, APFC_LATTICE_BCC3D = 2 };

enum { APFC_FP64 = 0,         /* fields, Krylov iterates and reductions in FP64 */
       APFC_FP32_REFINED = 1  /* FP32 Krylov inside FP64 iterative refinement   */ };
enum { APFC_BICGSTAB = 0 };
enum { APFC_TAU_FOLD = 0,     /* preconditioner uses 1/tau = 1/dt + kap dB      */
       APFC_TAU_PLAIN = 1     /* preconditioner uses tau = dt                    */ };

#define APFC_MAX_J 8

typedef struct {
  int lattice;               /* APFC_LATTICE_*                                   */
  int dim;                   /* 2 or 3                                           */
  int J;                     /* number of amplitudes, 1..APFC_MAX_J              */
  double k[APFC_MAX_J][3];   /* reciprocal vectors k_j (x, y, z); z ignored in 2D */
} apfc_lattice;

typedef struct { double dB, Bx, t, v; } apfc_params;

typedef struct {
  int n[3];                  /* grid points (nx, ny, nz); nz = 1 in 2D; each >= 3 */
  double h[3];               /* spacings (hx, hy, hz) > 0                          */
} apfc_grid;

typedef struct {
  int precision;             /* APFC_FP64 or APFC_FP32_REFINED                     */
  int krylov;                /* APFC_BICGSTAB                                       */
  int max_iter;              /* cap on Krylov iterations per solve (per refinement) */
  int cheb_degree;           /* applications of D per diffusion solve in P^{-1}, 0..16 */
  int tau_mode;              /* APFC_TAU_FOLD or APFC_TAU_PLAIN                     */
  int max_refine;            /* cap on FP64 refinement sweeps (FP32_REFINED)        */
  int check_every;           /* Krylov iterations between convergence checks        */
  int fused;                 /* 1: fused row-streaming A P^{-1} kernels on 2D grids (default);
                                0: one kernel per stencil pass                         */
  double tol;                /* stop at ||b - A x||_2 <= tol ||b||_2 (block norm, per amplitude) */
  double tol_inner;          /* relative tolerance of each FP32 inner solve         */
  int tile;                  /* fused 2D kernel variant 0..5 (columns per block and
                                rows of look-ahead), default 3                     */
  int tile_rows;             /* rows per block of the fused 2D kernels of the Krylov
                                iteration; 0 (default): the tallest of 128, 64, 32
                                rows that gives the first fused kernel's launch
                                >= 1.5 blocks per SM (x += P^{-1} u always takes
                                that automatic height)                             */
  int picard_iters;          /* K of Alg. 1: Picard iterations per step, 1..100;
                                1 (default) with jacobian 0 is the explicit step   */
  int jacobian;              /* 1: linearise N_j with D_j = dN_j/d eta_j (the
                                paper's J^j, h^j) in every Picard iteration        */
  int tile_t;                /* variant 0..5 of the fused kernel t = A P^{-1} s of
                                the merged iteration (-1: same as tile), default 1 */
  int guess;                 /* initial guess of each explicit step's solve:
                                APFC_GUESS_PREV (the previous state, Alg. 1) or
                                APFC_GUESS_EXTRAP (2 x^n - x^(n-1), after a
                                completed step of the same dt; else the previous state) */
} apfc_opts;
enum { APFC_GUESS_PREV = 0, APFC_GUESS_EXTRAP = 1 };

typedef struct {
  long long steps;           /* steps taken since apfc_set_amplitudes             */
  long long iters_total;     /* Krylov iterations summed over steps (of each solve,
                                the iterations of its slowest amplitude)           */
  int iters_last;            /* max over amplitudes of iterations in the last step */
  int refine_last;           /* refinement sweeps in the last step (FP32_REFINED)  */
  double resid_last;         /* max over amplitudes of ||b-Ax||/||b|| after the last step */
} apfc_stats_t;

/* Fill *o with defaults: FP64, BiCGStab, tol 1e-10, max_iter 500,
 * cheb_degree 1, tau fold, max_refine 10, tol_inner 1e-4, check_every 4, fused 1,
 * tile 3, tile_rows 0 (automatic), picard_iters 1, jacobian 0, tile_t 1. */
apfc_status apfc_default_opts(apfc_opts* o);

/* Relaxed-solid amplitude phi of a uniform crystal (eta_j = phi for all j):
 * the larger root of the uniform stationarity condition.  HEX2D:
 * phi = (t + sqrt(t^2 - 15 v dB)) / (15 v).  BCC3D: phi = (2t + sqrt(4t^2 -
 * 45 v dB)) / (45 v).  EINVAL for CUSTOM or when the root is not real. */
apfc_status apfc_uniform_amplitude(const apfc_lattice* lat, const apfc_params* p, double* phi);

/* Create a context (Sec. II model on the given grid).  Validates arguments,
 * builds per-amplitude stencil coefficients and the nonlinear-term table, and
 * allocates all device memory it needs (the context owns it).  stream: a
 * cudaStream_t (NULL = legacy default stream) used for every launch.  opts may
 * be NULL (defaults).  Amplitudes start unset (apfc_step returns ESTATE).
 * On failure *ctx is NULL and apfc_last_error(NULL) describes the failure
 * (per calling thread): EINVAL for arguments, ECUDA without a usable CUDA
 * device or for a failed CUDA call, ENOMEM when device or host memory runs out. */
apfc_status apfc_init(apfc_ctx** ctx, const apfc_lattice* lat, const apfc_params* p,
                      const apfc_grid* g, const apfc_opts* opts, void* stream);

/* Replace the solver options (precision, tolerances, degree). */
apfc_status apfc_set_opts(apfc_ctx* ctx, const apfc_opts* opts);

/* Copy amplitudes eta in ([J][nz][ny][nx], element type dtype: APFC_C128 or
 * APFC_C64) and set zeta = G_h eta (the auxiliary field of Sec. II.A).  The
 * state is FP64 either way.  Clears a sticky error and the stats.  EINVAL for
 * another dtype. */
apfc_status apfc_set_amplitudes(apfc_ctx* ctx, const void* eta, int where, int dtype);

/* Copy the current amplitudes eta out as dtype (APFC_C128 or APFC_C64), or the
 * auxiliary field zeta (complex128). */
apfc_status apfc_get_amplitudes(apfc_ctx* ctx, void* eta, int where, int dtype);
apfc_status apfc_get_zeta(apfc_ctx* ctx, void* zeta, int where);

/* Advance n steps of size dt (Alg. 1).  Default (picard_iters 1, jacobian 0):
 * one nonlinear iterate, explicit nonlinear right-hand side from eta^n for all
 * amplitudes, then one preconditioned Krylov solve per amplitude from the
 * initial guess (zeta^n, eta^n).  With picard_iters K > 1 or jacobian 1: K
 * iterations k, each solving per amplitude (all amplitudes reading eta^(k-1))
 *   [ I, -G_h ; kap Bx G_h, (1/dt + kap dB) I + kap D_j ] (zeta, eta)
 *     = (0, eta^n/dt - kap (N_j - D_j eta_j)(eta^(k-1))),
 * D_j = dN_j/d eta_j at eta^(k-1) with the Jacobian (a real diagonal), else 0,
 * from the previous iterate; the preconditioner keeps its constant coefficients
 * and the Jacobian runs the per-pass kernels.  Returns after the last step;
 * ENOCONV / ENAN if a solve failed (the state then holds the last iterate). */
apfc_status apfc_step(apfc_ctx* ctx, double dt, int n);

/* Choose the rows per segment of the fused 2D kernels (opts.tile_rows) and the
 * variant of the merged iteration's t-kernel (opts.tile_t) by timing: from the
 * current state, one step of size dt per candidate, each from the same state,
 * after one untimed step; first the automatic height, 32, 48 and 64 rows and every
 * height ceil(ny / s) between 96 and 256 rows (t-kernel variant as set), then every
 * t-kernel variant at the best height.  Keeps the fastest in the context's options.  The state and the
 * statistics are restored (the next step takes a stencil initial residual).  Only
 * the FP32-refined fused path on 2D grids has a choice to make: other
 * configurations return APFC_OK with their options unchanged and ms_per_step 0.
 * tile_rows, tile_t and ms_per_step (nullable) receive the choice and its step
 * time.  Allocates one copy of the state block for the duration of the call;
 * ENOMEM (context still usable) if it cannot. */
apfc_status apfc_autotune(apfc_ctx* ctx, double dt, int* tile_rows, int* tile_t, double* ms_per_step);

/* Discrete free energy (Eq. energyamplitude with the gradient term scaled so
 * that its Wirtinger derivative is the flow's Bx G_h^2 eta_j):
 *   F = h^d sum_points [ dB/2 A^2 + t-, v-terms of the bulk polynomial
 *                        + Bx sum_j |G_h eta_j|^2 ],  in FP64. */
apfc_status apfc_energy(apfc_ctx* ctx, double* F);

apfc_status apfc_stats(const apfc_ctx* ctx, apfc_stats_t* out);
const char* apfc_last_error(const apfc_ctx* ctx);
void apfc_destroy(apfc_ctx* ctx);

/* ---- operator-level entry points (FP64; same kernels as the step) ---------- */

/* y = A_j x for every amplitude (block operator of Eq. linear_system2, M = I);
 * x, y: block vectors [J][2][pts] complex128. */
apfc_status apfc_apply_operator(apfc_ctx* ctx, double dt, const void* x, void* y, int where);

/* x = P_j^{-1} b for every amplitude: the four-step application of the
 * preconditioner of Eq. preconditioner (Sec. II.B) with M = I and the
 * diffusion solves D^{-1} replaced by cheb_degree-application Chebyshev
 * polynomials on D's spectral interval; step 4 uses the sign that inverts the
 * displayed factorisation.  b, x: block vectors [J][2][pts]. */
apfc_status apfc_apply_preconditioner(apfc_ctx* ctx, double dt, const void* b, void* x, int where);

/* rhs_j = eta_j/dt - |k_j|^2 N_j(eta) for every amplitude (the explicit
 * nonlinear right-hand side); eta, rhs: [J][pts] complex128. */
apfc_status apfc_nonlinear_rhs(apfc_ctx* ctx, double dt, const void* eta, void* rhs, int where);

/* ---- preconditioner apply without allocation ----------------------------------
 * The paper has no counterpart to this entry point; it exists for callers that
 * may not allocate device memory where they apply the preconditioner (a
 * framework that owns the allocator, a latency-critical path where cudaMalloc
 * would synchronise the device, a plugin handed buffers and a stream only).
 *
 * x = P_j^{-1} b for every amplitude: the same operator as
 * apfc_apply_preconditioner (same coefficients, same Chebyshev polynomial of
 * degree cheb_degree, same tau_mode), computed with the unfused FP64 per-pass
 * kernels, so the two agree to rounding (not bit for bit: the context path may
 * run the fused 2D pipeline or fold step 4 into the last 3D pass).  There is no
 * context: the caller passes lattice, parameters, grid, dt, and DEVICE buffers
 * b and x (block vectors [J][2][pts] complex128).  The five intermediate fields
 * live in one file-scope device array of 5 * APFC_STATIC_MAX_DOF complex128
 * (20 MB) that every GPU which loads the library holds until the process
 * exits; the call performs no cudaMalloc/cudaFree and calls no allocating
 * library routine.
 *
 * Limits and behaviour:
 *  - J * nx * ny * nz must be <= APFC_STATIC_MAX_DOF, else APFC_ETOOBIG
 *    (nothing is launched).  Bad arguments give APFC_EINVAL (nothing is
 *    launched): the lattice, parameters, grid and dt checks of apfc_init and
 *    of a step, and b and x overlapping (the last pass reads b while it writes
 *    x, so the call cannot work in place).
 *  - A CUDA error left pending by the caller's earlier work makes the call
 *    return APFC_ECUDA without launching and without clearing that error;
 *    otherwise APFC_ECUDA reports a failed launch of this call.
 *  - The first call on a device resolves the array's device address with
 *    cudaGetSymbolAddress (with that device current); make that first call
 *    before any stream capture.  stream must belong to the current device.
 *  - Work is enqueued on stream (NULL = legacy default stream) and the call
 *    returns without waiting; x is ready when the stream reaches that point.
 *  - Every call shares the one array and it keeps the last call's contents;
 *    no intermediate needs to start at zero (each is written in full before it
 *    is read).  Calls that overlap on the GPU (different streams, or threads)
 *    race on the array and give wrong results: serialise them. */
#define APFC_STATIC_MAX_DOF 262144
apfc_status apfc_apply_preconditioner_static(const apfc_lattice* lat, const apfc_params* p, const apfc_grid* g,
                                             int cheb_degree, int tau_mode, double dt, const void* b, void* x,
                                             void* stream);

/* ---- measurement (tracing) ------------------------------------------------
 * Kernel ids run 0..apfc_kernel_count()-1 (FP64 variants, then FP32 ones);
 * apfc_kernel_name(id) names them.  Measurement is process-wide and serves
 * one context at a time.
 *
 * apfc_profile_start(ctx, timed_id): zeroes the counters.  From then on every
 * kernel adds the algorithmic bytes it moves (its whole-field reads and
 * writes, counted once per active amplitude) to a device counter of its id,
 * the host counts launches per id, and each launch of kernel timed_id
 * (-1: none; -2: every kernel) is bracketed by CUDA events recorded on the
 * context stream.
 * apfc_profile_read(ctx, id, ...): synchronises the stream; returns since the
 * start the summed event time of id in ms (0 unless id is timed), its
 * launches, its algorithmic bytes, and the launches of all library kernels.
 * Null output pointers are skipped.  apfc_profile_stop(ctx) ends it. */
int apfc_kernel_count(void);
const char* apfc_kernel_name(int id);
apfc_status apfc_profile_start(apfc_ctx* ctx, int timed_id);
apfc_status apfc_profile_read(apfc_ctx* ctx, int id, double* ms, long long* launches, double* bytes,
                              long long* all_launches);
apfc_status apfc_profile_stop(apfc_ctx* ctx);

/* Arithmetic rates of the current device, for the arithmetic roofline of the
 * FP64 kernels (the paper has no counterpart; it reports no GPU rates).
 * kind APFC_ALU_FMA64 / APFC_ALU_FMA32: independent FMA chains in FP64 / FP32,
 * *rate = FLOP/s (2 per FMA); APFC_ALU_CVT64: FP64 -> FP32 -> FP64 conversion
 * chains, *rate = conversions/s.  8 blocks of 256 threads per SM, best of three
 * launches timed with CUDA events on stream (NULL = legacy default stream).
 * Allocates and frees a small device buffer and synchronises the stream.
 * EINVAL for another kind or a NULL output, ECUDA / ENOMEM on failure. */
enum { APFC_ALU_FMA64 = 0, APFC_ALU_FMA32 = 1, APFC_ALU_CVT64 = 2 };
apfc_status apfc_measure_alu_rate(int kind, void* stream, double* rate);

/* ---- parameters and the adjoint of the step ---------------------------------
 * Gradient convention: for a real loss L of complex fields, the gradient with
 * respect to a field eta is the complex field dL/dRe(eta) + i dL/dIm(eta) (twice
 * the Wirtinger derivative dL/d conj(eta); PyTorch's convention), so that
 * dL = Re sum conj(grad) d(eta).  Fields are [J][nz][ny][nx] complex128. */

/* Replace (dB, Bx, t, v) (validated as in apfc_init); the state is kept.  The
 * next step rebuilds the coefficients; a recorded rollout is dropped. */
apfc_status apfc_set_params(apfc_ctx* ctx, const apfc_params* p);

/* Adjoint of one step of size dt (the map eta^n -> eta^{n+1} of apfc_step with
 * picard_iters 1 and jacobian 0, else EINVAL; per
 * amplitude eta_j^{n+1} = S_j^{-1} (eta_j^n/dt - kap_j N_j(eta^n)) with
 * S_j = (1/dt + kap_j dB) I + kap_j Bx G_h^2, kap_j = |k_j|^2).  Given
 * lam_np1 = grad of L wrt eta^{n+1}, returns lam_n = grad of L wrt eta^n
 * through this step and *dB_grad = dL/d dB through S:
 *   g_j = S_j^{-1} lam_np1_j   (S_j is Hermitian since G_h is: the adjoint solve
 *                               is the block solve of the step with right-hand
 *                               side (0, lam_np1_j), to opts.tol in opts.precision),
 *   lam_n_k = g_k/dt - sum_j kap_j [g_j conj(dN_j/d eta_k) + conj(g_j) dN_j/d conj(eta_k)],
 *   *dB_grad = -sum_j kap_j Re sum_points conj(g_j) eta_np1_j.
 * eta_n, eta_np1: the step's input and output.  The solve starts from zero. */
apfc_status apfc_adjoint_step(apfc_ctx* ctx, double dt, const void* eta_n, const void* eta_np1,
                              const void* lam_np1, void* lam_n, double* dB_grad, int where);

/* Gradient of the free energy F of apfc_energy at eta:
 *   grad_j = 2 h^d [ (dB + Bx G_h^2) eta_j + N_j(eta) ],
 * and *dF_ddB = h^d sum_points sum_j |eta_j|^2 (F is affine in dB); dF_ddB may be NULL. */
apfc_status apfc_energy_gradient(apfc_ctx* ctx, const void* eta, void* grad, double* dF_ddB, int where);

/* Checkpointed rollout.  apfc_rollout_forward advances the state n steps of size
 * dt like apfc_step, keeping eta every `every` steps and at the end on the device
 * (owned by the context: (ceil(n/every) + 1) fields).  At each checkpoint the
 * step restarts from (G_h eta, eta) without the previous step's residual, so that
 * the backward pass can recompute every segment bit for bit.
 * apfc_rollout_backward takes lam_n = grad of L wrt eta^n and returns
 * lam_0 = grad of L wrt eta^0 through all n steps and *dB_grad = the sum over the
 * steps of their dL/d dB (as apfc_adjoint_step; each adjoint solve starts from
 * the previous one's solution).  It recomputes each segment's states from its
 * checkpoint (one more forward pass in total; every + 1 fields of scratch) and
 * leaves the state at eta^n.  ESTATE without a recorded rollout. */
apfc_status apfc_rollout_forward(apfc_ctx* ctx, double dt, int n, int every);
apfc_status apfc_rollout_backward(apfc_ctx* ctx, const void* lam_n, void* lam_0, double* dB_grad, int where);

/* ---- rotation diagnostic and adaptivity map (Sec. II.D) ----------------------
 * Analysis output of the current state (nothing of the step depends on it).
 * omega: the rotation tensor omega_il = 1/2 (du_i/dx_l - du_l/dx_i) (Eq. rot) of
 * the displacement u solving k_j . u = arg(eta_j) in the least-squares sense,
 * u = M^{-1} sum_j k_j arg(eta_j), M = sum_j k_j k_j^T; the phase gradients are
 * central differences of the unwrapped phase, arg(eta_j(r+h e_d) conj(eta_j(r-h e_d)))/(2h_d),
 * so a grain rotated by theta about z gives omega_12 = sin(theta) (each phase
 * difference is taken by an FP32 atan2 of the FP64 product scaled to unit size:
 * omega to about 1e-7 absolute; A, grad A and h's branches in FP64).
 * Layout: [ncomp][nz][ny][nx] doubles, ncomp = 1 in 2D (omega_12) and 3 in 3D
 * (omega_23, omega_31, omega_12); 0 where some |eta_j|^2 < 1e-12 (the liquid).
 * amp (may be NULL): A = sqrt(2 sum_j |eta_j|^2), [nz][ny][nx] doubles.
 * hmap (may be NULL; needs adapt): the local grid size of Eq. hhh,
 *   h_int                              where |grad A| >= eps (central differences),
 *   min(max(h_amp, h_int), h_max)      where A > A_min,
 *   h_max                              elsewhere,
 * with h_amp = pi / (n max_j |k_j| sin(theta/2)), theta = asin(min(max_d |omega_d|, 1))
 * (lambda_j(theta) = 2 pi / |dk_j(theta)| at |dk_j| = 2 |k_j| sin(theta/2); theta = 0
 * gives h_amp = infinity).  EINVAL for n <= 0, h_int <= 0, h_max < h_int or eps < 0. */
typedef struct {
  double n;      /* grid points per smallest amplitude wavelength (the paper uses >= 10) */
  double h_int;  /* grid size at interfaces and defects                                 */
  double h_max;  /* largest grid size                                                   */
  double eps;    /* threshold on |grad A|                                               */
  double A_min;  /* "A > 0" threshold of the solid                                      */
} apfc_adapt;
apfc_status apfc_rotation_field(apfc_ctx* ctx, void* omega, void* amp, void* hmap, const apfc_adapt* adapt,
                                int where);

/* ---- batched independent runs ----------------------------------------------
 * Many independent 2D simulations of one lattice, one parameter set and one
 * spacing (hx, hy) on periodic grids of different sizes nx[r] x ny[r], advanced
 * together by the step of apfc_step (Alg. 1 with one nonlinear iterate; the
 * Sec. II.B preconditioner inside BiCGStab) in precision APFC_FP32_REFINED with
 * the fused pipeline.  Every stage of the step is one launch over the work of
 * all runs; each (run, amplitude) keeps its own Krylov scalars and stops on its
 * own, and a run whose refinement has converged waits unchanged for the
 * others.  Run r follows the same arithmetic as run r alone on an apfc_ctx
 * with the same options (the same per-run reductions in the same order).
 *
 * Storage: the batch owns the concatenated block vectors of all runs (FP64
 * state, right-hand sides and residuals; FP32 Krylov vectors), about
 * 2 J sum_r(nx ny) x (4 x 16 + 10 x 8) bytes.  Amplitude buffers of run r are
 * [J][ny[r]][nx[r]] complex128, owned by the caller, copied in or out.
 *
 * flags: APFC_BATCH_GRAPH replays the Krylov iteration blocks (check_every
 * merged iterations) from captured CUDA graphs; the first block of each solve
 * runs uncaptured.  With that flag a NULL stream makes the batch create and own
 * a non-blocking stream (graphs cannot be captured on the legacy stream).
 * Errors are sticky as on a context; ENAN / ENOCONV name the failing run in
 * apfc_batch_last_error(). */
typedef struct apfc_batch apfc_batch;
#define APFC_BATCH_GRAPH 1

/* Validate (lattice and parameters as apfc_init, dim 2, 1 <= nruns <= 65536,
 * 3 <= nx[r], ny[r] <= 2^20, opts: precision APFC_FP32_REFINED, fused 1,
 * cheb_degree 1..4; opts NULL = defaults with APFC_FP32_REFINED) and allocate.
 * EINVAL on bad arguments, ETOOBIG if a launch over all runs would exceed the
 * grid limit, ENOMEM if the device memory does not fit, ECUDA without a usable
 * CUDA device.  On failure *b is NULL and apfc_batch_last_error(NULL)
 * describes the failure (per calling thread). */
apfc_status apfc_batch_init(apfc_batch** b, const apfc_lattice* lat, const apfc_params* p, int nruns,
                            const int* nx, const int* ny, double hx, double hy, const apfc_opts* opts,
                            int flags, void* stream);
apfc_status apfc_batch_set_opts(apfc_batch* b, const apfc_opts* opts);
apfc_status apfc_batch_get_opts(const apfc_batch* b, apfc_opts* out);

/* Per-run state: as apfc_set_amplitudes / apfc_get_amplitudes for run r. */
apfc_status apfc_batch_set_amplitudes(apfc_batch* b, int run, const void* eta, int where);
apfc_status apfc_batch_get_amplitudes(apfc_batch* b, int run, void* eta, int where);

/* Advance every run n steps of size dt (all runs must have amplitudes). */
apfc_status apfc_batch_step(apfc_batch* b, double dt, int n);

/* Free energy of run r (as apfc_energy) and its solver statistics. */
apfc_status apfc_batch_energy(apfc_batch* b, int run, double* F);
apfc_status apfc_batch_stats(const apfc_batch* b, int run, apfc_stats_t* out);

/* Tile autotuner: from the first refinement residual of a step of the current
 * state (the state itself is not changed), time a fixed number of merged
 * BiCGStab iterations over all runs, first for every tile variant (0..5) and
 * segment height (32, 48, 64, 96, 128, 192, 256 rows) shared by both fused
 * kernels, then for every variant of the t-kernel alone with the rest fixed;
 * keep the fastest in the
 * batch's options (tile, tile_rows, tile_t; see apfc_batch_get_opts) and return
 * tile, rows and ms per iteration (null pointers skipped). */
apfc_status apfc_batch_autotune(apfc_batch* b, double dt, int* tile, int* tile_rows, double* ms_per_iter);

/* Number of captured-graph replays since creation (-1 for a null batch). */
long long apfc_batch_graph_replays(const apfc_batch* b);

const char* apfc_batch_last_error(const apfc_batch* b);
void apfc_batch_destroy(apfc_batch* b);

/* Measurement as apfc_profile_* on the batch's stream (graph replay is off
 * while measuring, so that every launch is counted and can be timed). */
apfc_status apfc_batch_profile_start(apfc_batch* b, int timed_id);
apfc_status apfc_batch_profile_read(apfc_batch* b, int id, double* ms, long long* launches, double* bytes,
                                    long long* all_launches);
apfc_status apfc_batch_profile_stop(apfc_batch* b);

#ifdef __cplusplus
}
#endif
#endif /* APFC_H */
