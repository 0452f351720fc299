// Internal declarations shared by the CUDA translation units of libapfc.
//
// Notation follows arXiv:1902.09761, Sec. II: amplitudes eta_j, auxiliary
// fields zeta_j = G_j eta_j, G_h = L_h + 2i k_j . D_h on a periodic grid.
//
// Storage: a "field" is [J][pts] complex; a "block vector" is [J][2][pts]
// complex (zeta-part, then eta-part, per amplitude).  A FieldRef addresses
// amplitude j of a field or of one part of a block vector through a stride.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "apfc.h"

namespace apfc {

constexpr int kMaxJ = APFC_MAX_J;
constexpr int kMaxCheb = 16;     // Chebyshev applications per diffusion solve
constexpr int kMaxTerms = 96;    // derivative / energy monomials of table lattices
constexpr int kDotBlocks = 304;  // partial-sum blocks per amplitude (2 x 152 SMs)
constexpr int kDotSlots = 6;     // inner products per amplitude that one reduction can carry
constexpr int kThreads = 256;

// ---------------------------------------------------------------------------
// Complex helpers (interleaved double2 / float2)
// ---------------------------------------------------------------------------
template <typename T> struct CT;
template <> struct CT<double> { using c = double2; };
template <> struct CT<float> { using c = float2; };
template <typename T> using cplx = typename CT<T>::c;

template <typename T>
__host__ __device__ __forceinline__ cplx<T> mkc(T re, T im) {
  cplx<T> r;
  r.x = re;
  r.y = im;
  return r;
}

template <typename T>
struct FieldRef {
  cplx<T>* p;
  long long ld;  // elements between amplitude j and j+1
  __host__ __device__ __forceinline__ cplx<T>* at(int j) const { return p + (long long)j * ld; }
};
template <typename T>
struct CFieldRef {
  const cplx<T>* p;
  long long ld;
  __host__ __device__ __forceinline__ const cplx<T>* at(int j) const { return p + (long long)j * ld; }
};

// ---------------------------------------------------------------------------
// Operator coefficients (rebuilt when dt changes)
// ---------------------------------------------------------------------------
struct OpCoef {
  int J, dim, nx, ny, nz;
  long long pts;            // nx * ny * nz
  double ih2[3];            // 1/h_d^2
  double c0;                // -2 sum_d 1/h_d^2 (centre weight of L_h)
  double kh[kMaxJ][3];      // k_{j,d} / h_d: 2i k_d D_d u = i (k_d/h_d)(u+ - u-)
  double kap[kMaxJ];        // |k_j|^2
  double kt[kMaxJ];         // |k_j|^2 Bx: coefficient of G_h in the (2,1) block
  double a[kMaxJ];          // 1/dt + |k_j|^2 dB: the (2,2) block
  double inv_dt;
  double sD[kMaxJ];         // D = sD I + mu (-L_h), sD = 1/sqrt(tau~)
  double mu[kMaxJ];         //                       mu = sqrt(kt)
  double inv_mu[kMaxJ];
  double inv_theta[kMaxJ];  // Chebyshev: 1/theta, theta = centre of D's interval
  unsigned long long* prof; // device byte counters per kernel id (nullptr: not measuring)
  const double* jd;         // Picard with Jacobian: kap_j D_j per point, [J][pts] (nullptr: none)
  const float2* jd32;       // the same as {value, 0} for the FP32 fused kernels' staged fetch
};

// (2,2) block of A_j at point p: a_j, plus kap_j D_j(p) when the Jacobian is on.
__host__ __device__ __forceinline__ double a_at(const OpCoef& c, int j, long long p) {
  return c.jd == nullptr ? c.a[j] : c.a[j] + c.jd[(long long)j * c.pts + p];
}

// ---------------------------------------------------------------------------
// Measurement: every kernel adds the algorithmic bytes it moves (whole-field
// reads and writes, once per active amplitude) to prof[id]; the launch
// wrappers count launches and bracket one selected kernel id with events.
// FP32 variants use id + KID_COUNT.
// ---------------------------------------------------------------------------
enum KernelId {
  KID_APPLY_A = 0,
  KID_RESIDUAL,
  KID_PC_RHS,
  KID_CHEB_ZERO,
  KID_CHEB_FIRST,
  KID_CHEB_SWEEP,
  KID_PC_FINAL,
  KID_P_UPDATE,
  KID_S_UPDATE,
  KID_R_UPDATE,
  KID_ADD_TO,
  KID_DOTS,
  KID_FINALIZE,
  KID_RHS,
  KID_ZETA,
  KID_RESID_REFINE,
  KID_ENERGY,
  KID_FUSED_APINV,
  KID_FUSED_PINV,
  KID_BICG_UPDATE,
  KID_FUSED_APINV_T,
  KID_ADJ_NONLIN,
  KID_ENERGY_GRAD,
  KID_ROTATION,
  KID_EXTRAP,
  KID_COUNT
};
template <typename T>
__host__ __device__ constexpr int kid_of(int k) {
  return k + (sizeof(T) == 4 ? KID_COUNT : 0);
}

// Host side (api.cu): called by every launch wrapper around its launch.
void prof_launch_begin(int kid, cudaStream_t s);
void prof_launch_end(int kid, cudaStream_t s);
struct ProfScope {
  int kid;
  cudaStream_t s;
  ProfScope(int k, cudaStream_t st) : kid(k), s(st) { prof_launch_begin(kid, s); }
  ~ProfScope() { prof_launch_end(kid, s); }
};

__device__ __forceinline__ void prof_add(const OpCoef& c, int kid, unsigned long long bytes) {
  if (c.prof != nullptr && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(c.prof + kid, bytes);
}

// Batched runs: every run's block vectors sit one after another in shared
// arrays; elem_off is the run's first element (of [J][2][pts]), part_off its
// first 16-byte partial-sum slot.
struct RunGeom {
  int nx, ny;
  long long pts, elem_off;
  long long part_off, part_off_t;  // first partial-sum slot: v-kernel layout, t-kernel layout
  int npart, npart_t;              // partial-sum slots per amplitude in each layout
};
struct BatchLaunch {
  const RunGeom* dev;   // device copy of the run table (per-point kernels, reductions)
  const RunGeom* host;  // host copy (the fused kernels carry it in their parameters)
  int R;
  int tlay;  // 1: partial sums in the t-kernel layout (its own tile variant)
};

// Point a kernel's grid sizes at run `run`; returns the run's first element.
__device__ __forceinline__ long long select_run(const RunGeom* rg, int run, OpCoef& c) {
  const RunGeom& q = rg[run];
  c.nx = q.nx;
  c.ny = q.ny;
  c.nz = 1;
  c.pts = q.pts;
  return q.elem_off;
}

// Chebyshev recurrence weights for one application (per amplitude):
// d_{k+1} = c1 d_k + c2 r_{k+1}.
struct ChebStep {
  double c1[kMaxJ];
  double c2[kMaxJ];
};

// Nonlinear term N_j.  hex = 1: closed form of the triangular lattice.
// Otherwise N_j = sum_{terms of j} coef * prod_f mode(f) with
// mode(f) = eta_{f>>1} if (f & 1) == 0 else conj(eta_{f>>1}).
struct NonlinTable {
  int hex;
  double t, v;
  int start[kMaxJ + 1];
  double coef[kMaxTerms];
  int nf[kMaxTerms];
  int f[kMaxTerms][3];
  // the same N_j with its |eta_m|^2 eta_j monomials gathered: N_j = eta_j sum_m
  // wdiag[j][m] |eta_m|^2 + the monomials ridx[rstart[j] .. rstart[j+1]) of the list above
  double wdiag[kMaxJ][kMaxJ];
  int rstart[kMaxJ + 1];
  int ridx[kMaxTerms];
};

// Bulk energy density beyond dB/2 A^2 for table lattices: sum_e ecoef Re(prod).
struct EnergyTable {
  int hex;
  double dB, t, v;
  int ne;
  double coef[kMaxTerms];
  int nf[kMaxTerms];
  int f[kMaxTerms][4];
};

// Per-amplitude Krylov scalars, resident on the device.
struct KScal {
  double2 rho, alpha, omega, beta;
  double bnorm2, rnorm2, tol2, tolrel2;
  int active, iters, status, max_iter;
  int just_done;  // stopped in this iteration, its last update of u still pending
  int pad;
};

enum KStatus { KS_RUNNING = 0, KS_CONVERGED = 1, KS_NOCONV = 2, KS_BREAKDOWN = 3, KS_NAN = 4 };
enum KOp { OP_INIT = 0, OP_ALPHA = 1, OP_SNORM = 2, OP_OMEGA = 3, OP_RHO = 4, OP_NORMS = 5, OP_OMEGA3 = 6, OP_RNORM = 7, OP_BNORM = 8, OP_OMEGA5 = 9, OP_INIT3 = 10 };

// Up to three (u, v) pairs of block vectors for conj(u).v per amplitude.
template <typename T>
struct DotPairs {
  const cplx<T>* u[3];
  const cplx<T>* v[3];
};

// ---------------------------------------------------------------------------
// kernels.cu (per-pass 2D kernels, nonlinear terms, vector updates, diagnostics;
// their 3D branches and the launch*3d / stream3d_parts entries: stream3d.cu)
// ---------------------------------------------------------------------------
template <typename T>
void launch_apply_A(const cplx<T>* x, cplx<T>* y, const OpCoef& c, const KScal* act, cudaStream_t s);
template <typename T>
void launch_residual(const cplx<T>* b, const cplx<T>* x, cplx<T>* r, cplx<T>* rhat, const OpCoef& c,
                     cudaStream_t s);
template <typename T>
void launch_pc_rhs(const cplx<T>* beta, FieldRef<T> f, const OpCoef& c, const KScal* act, cudaStream_t s);
template <typename T>
void launch_cheb_zero(CFieldRef<T> f, FieldRef<T> X, const OpCoef& c, const KScal* act, cudaStream_t s);

template <typename T>
void launch_pc_final(const cplx<T>* beta, CFieldRef<T> b2p, cplx<T>* chi, const OpCoef& c, const KScal* act,
                     cudaStream_t s);
template <typename T>
void launch_p_update(const cplx<T>* r, cplx<T>* p, const cplx<T>* v, const OpCoef& c, const KScal* k,
                     cudaStream_t s);
// s = r - alpha v (in r); then u += alpha p + omega s, r = s - omega t.  partials !=
// nullptr: the inner products of the updated vectors, (s, s) for the s-update and
// (rhat, r), (r, r) for the r-update, in the k_dots layout [J][kDotSlots][kDotBlocks]
template <typename T>
void launch_s_update(cplx<T>* r, const cplx<T>* v, const OpCoef& c, const KScal* k, cudaStream_t s,
                     void* partials = nullptr);
template <typename T>
void launch_r_update(cplx<T>* r, const cplx<T>* t, cplx<T>* u, const cplx<T>* p, const OpCoef& c, const KScal* k,
                     cudaStream_t s, const cplx<T>* rhat = nullptr, void* partials = nullptr);
// 3D grids: y = A x with inner products of y in the same pass: nd = 1 gives (du, y),
// nd = 2 gives (y, du) and (y, y).  Partials use the layout [J][kDotSlots][npart] with
// npart = stream3d_parts(c, sizeof(cplx<T>)) (one per block of the pass).
template <typename T>
void launch_apply_A_dots(const cplx<T>* x, cplx<T>* y, const cplx<T>* du, int nd, void* partials, const OpCoef& c,
                         const KScal* act, cudaStream_t s);
int stream3d_parts(const OpCoef& c, int elem_bytes);
// Step 4 of P^{-1} folded into the last Chebyshev pass of the second diffusion solve
// (3D grids): chi1 = beta1 + (beta2' - sD chi2) / mu, from the chi2 just computed.
template <typename T>
struct PcFin {
  CFieldRef<T> b1;   // beta1 (stride 2 pts)
  CFieldRef<T> b2p;  // beta2'
  FieldRef<T> chi1;  // chi1 (stride 2 pts)
};
// 3D grids (stream3d.cu): the passes behind launch_apply_A, launch_residual, launch_pc_rhs,
// launch_cheb_first / _sweep (fin: step 4 of P^{-1} in this last pass) and launch_zeta.
template <typename T>
void launch3d_apply_A(const cplx<T>* x, cplx<T>* y, const OpCoef& c, const KScal* act, cudaStream_t s);
template <typename T>
void launch3d_residual(const cplx<T>* b, const cplx<T>* x, cplx<T>* r, cplx<T>* rhat, const OpCoef& c,
                       cudaStream_t s);
template <typename T>
void launch3d_pc_rhs(const cplx<T>* beta, FieldRef<T> f, const OpCoef& c, const KScal* act, cudaStream_t s);
template <typename T>
void launch3d_cheb_first(CFieldRef<T> f, FieldRef<T> X, FieldRef<T> R, FieldRef<T> Dn, const ChebStep& w, int last,
                         const OpCoef& c, const KScal* act, cudaStream_t s, const PcFin<T>* fin);
template <typename T>
void launch3d_cheb_sweep(CFieldRef<T> Dd, FieldRef<T> X, FieldRef<T> R, FieldRef<T> Dn, const ChebStep& w, int last,
                         const OpCoef& c, const KScal* act, cudaStream_t s, const PcFin<T>* fin);
void launch3d_zeta(double2* x, const OpCoef& c, cudaStream_t s);
// fin != nullptr (3D grids, last pass only): also step 4 of P^{-1}, see PcFin
template <typename T>
void launch_cheb_first(CFieldRef<T> f, FieldRef<T> X, FieldRef<T> R, FieldRef<T> Dn, const ChebStep& w, int last,
                       const OpCoef& c, const KScal* act, cudaStream_t s, const PcFin<T>* fin = nullptr);
template <typename T>
void launch_cheb_sweep(CFieldRef<T> Dd, FieldRef<T> X, FieldRef<T> R, FieldRef<T> Dn, const ChebStep& w, int last,
                       const OpCoef& c, const KScal* act, cudaStream_t s, const PcFin<T>* fin = nullptr);
template <typename T>
void launch_add_to(const cplx<T>* d, double2* x, const OpCoef& c, cudaStream_t s);

// bl != nullptr (here and below): one launch over every run of a batch, c holding the
// largest run's sizes; FP64 partials of run r start at slot r J kDotSlots kDotBlocks
void launch_rhs(const double2* x, double2* b, const OpCoef& c, const NonlinTable& nt, cudaStream_t s,
                const BatchLaunch* bl = nullptr);
void launch_zeta(double2* x, const OpCoef& c, cudaStream_t s);
// x <- 2 x - xp, xp <- x over the state block (the extrapolated initial guess)
void launch_extrapolate(double2* x, double2* xp, const OpCoef& c, cudaStream_t s);
// complex64 [J][pts] <-> part (0 zeta, 1 eta) of the FP64 state block, rounding to nearest
void launch_c64_to_part(const float2* src, double2* x, long long pts, int J, int part, cudaStream_t s);
void launch_part_to_c64(const double2* x, float2* dst, long long pts, int J, int part, cudaStream_t s);
void launch_residual_refine(const double2* b, const double2* x, float2* r32, double* partials, const OpCoef& c,
                            cudaStream_t s);
// 2D only: FP64 residual with FP32 (and optional FP64) output
void launch_residual_refine2d(const double2* b, const double2* x, float2* r32, double2* r64, double* partials,
                              const OpCoef& c, cudaStream_t s, const BatchLaunch* bl = nullptr);
// One 2D or 3D grid: the residual with its tiles staged by TMA and the partial ||r||^2
// per amplitude (resid2d.cu); false, with *err set, if the tensor maps cannot be built
// (nothing is launched then)
bool launch_residual_refine_tma(const double2* b, const double2* x, float2* r32, double2* r64, double* partials,
                                const OpCoef& c, cudaStream_t s, const char** err);
// bounded waits of the TMA kernels that gave up since the library was loaded
// (stream3d_timeouts: those of the 3D passes alone)
unsigned long long tma_timeouts();
unsigned long long stream3d_timeouts();
// Start of an FP32 solve from x0 = 0: r = b, rhat = b rounded to bf16 with its packed copy
// rh16 [J][pts] (bf16pair.cuh), partials of (r, r), (b, b), (rhat, r) in slots 0-2 (k_dots' layout)
void launch_init32(const float2* b, float2* r, float2* rhat, uint2* rh16, void* partials, const OpCoef& c,
                   cudaStream_t s, const BatchLaunch* bl = nullptr);
// new RHS and initial residual r0 = b - b_prev + r_prev (pointwise); b_prev = r_prev = null:
// the RHS and the ||b||^2 partials only (the ||r0||^2 slot holds 0, r32 is not written)
void launch_rhs_resid(const double2* x, double2* b, const double2* b_prev, const double2* r_prev, float2* r32,
                      double* partials, const OpCoef& c, const NonlinTable& nt, cudaStream_t s,
                      const BatchLaunch* bl = nullptr);
void launch_energy(const double2* x, double* partials, double* out, const OpCoef& c, const EnergyTable& et,
                   double Bx, cudaStream_t s);
// Adjoint of the explicit right-hand side of a step (eta0, eta1: [J][pts]; xg: block whose
// eta-part is g = S^{-1} lam_{n+1}): lam = g/dt - sum_j kap_j [g_j conj(dN_j/deta) +
// conj(g_j) dN_j/dconj(eta)]; *out = sum_j kap_j Re sum conj(g_j) eta1_j (device scalar)
void launch_adj_nonlin(const double2* eta0, const double2* xg, const double2* eta1, double2* lam, double* partials,
                       double* out, const OpCoef& c, const NonlinTable& nt, cudaStream_t s);
// Picard iteration of Alg. 1: b_j = eta_prev_j/dt - kap_j (N_j - D_j eta_j) from the
// previous iterate (eta-parts of x); jd (nullable) receives kap_j D_j, D_j = dN_j/d eta_j
void launch_rhs_picard(const double2* x, const double2* eta_prev, double2* b, double* jd, float2* jd32,
                       const OpCoef& c, const NonlinTable& nt, cudaStream_t s);
// Rotation diagnostic and adaptivity map (Sec. II.D): per point the rotation
// tensor components omega (1 in 2D: omega_12; 3 in 3D: omega_23, omega_31,
// omega_12), A = sqrt(2 sum |eta_j|^2) and the local grid size h of Eq. hhh.
struct RotParams {
  float Wf[kMaxJ][3];  // M^{-1} k_j, M = sum_j k_j k_j^T
  float inv2h[3];      // 1 / (2 h_d)
  double inv2hd[3];
  double h_int, h_max, eps, A_min, amp_floor;
  double pi_over_nk;   // pi / (n max_j |k_j|)
};
void launch_rotation(const double2* x, double* omega, double* amp, double* hmap, const RotParams& rp,
                     const OpCoef& c, cudaStream_t s);
// Real gradient of the free energy: grad_j = scale [dB eta_j + Bx G_h zeta_j + N_j(eta)] from a
// block x with zeta = G_h eta; *out = sum_j sum |eta_j|^2 (device scalar)
void launch_energy_grad(const double2* x, double2* grad, double scale, double dB, double Bx, double* partials,
                        double* out, const OpCoef& c, const NonlinTable& nt, cudaStream_t s);

// ---------------------------------------------------------------------------
// fused2d.cu: row-streaming fused P^{-1} / A P^{-1} for 2D grids, Chebyshev
// degree m in 1..fused2d_max_degree(); each returns false when it cannot run.
// Dot partials use layout [J][kDotSlots][npart], npart = fused2d_npart(c, m, Ly).
// ---------------------------------------------------------------------------
int fused2d_max_degree(int elem_bytes);
int fused2d_npart(const OpCoef& c, int m, int Ly, int elem_bytes, int tile);  // elem_bytes = sizeof(complex)
int fused2d_tiles();  // number of tile variants
// p_new = r + beta (p_old - omega v_old); v_new = A P^{-1} p_new; partial (rhat, v_new)
template <typename T>
bool launch_fused_v(int m, int Ly, int tile, const OpCoef& c, const ChebStep* w, const cplx<T>* r, const cplx<T>* p_old,
                    const cplx<T>* v_old, cplx<T>* p_new, cplx<T>* v_new, const cplx<T>* rhat, const uint2* rh16,
                    const KScal* act, void* partials, cudaStream_t s);
// t = A P^{-1} (r - alpha v); partials (t, s), (t, t), (s, s)
template <typename T>
bool launch_fused_t(int m, int Ly, int tile, const OpCoef& c, const ChebStep* w, const cplx<T>* r, const cplx<T>* v,
                    cplx<T>* t_out, const KScal* act, void* partials, cudaStream_t s);
// x64 += P^{-1} u
template <typename T>
bool launch_fused_pinv_add(int m, int Ly, int tile, const OpCoef& c, const ChebStep* w, const cplx<T>* u, double2* x64,
                           cudaStream_t s, const BatchLaunch* bl = nullptr);
// blocks of one fused launch over an nx x ny grid (J amplitudes); *npart = blocks per amplitude
int fused2d_blocks(int nx, int ny, int J, int m, int Ly, int elem_bytes, int tile, bool with_a, int* npart);
// x = P^{-1} b
template <typename T>
bool launch_fused_pinv_store(int m, int Ly, int tile, const OpCoef& c, const ChebStep* w, const cplx<T>* b, cplx<T>* x,
                             cudaStream_t s);
// Merged BiCGStab iteration (buffers of the previous iteration -> the next):
// r' = r - alpha v - omega t, p' = r' + beta (p - omega v), u += alpha p + omega (r - alpha v)
// (the last at owned points), v' = A P^{-1} p'; partial (rhat, v').
template <typename T>
bool launch_fused_merged_v(int m, int Ly, int tile, const OpCoef& c, const ChebStep* w, const cplx<T>* r, const cplx<T>* v,
                           const cplx<T>* t, const cplx<T>* p, cplx<T>* u, cplx<T>* r_new, cplx<T>* p_new,
                           cplx<T>* v_new, const cplx<T>* rhat, const uint2* rh16, const KScal* act, void* partials,
                           cudaStream_t s, const BatchLaunch* bl = nullptr);
// t = A P^{-1} s, s = r - alpha v; partials (t, s), (t, t), (s, s), (rhat, s), (rhat, t)
template <typename T>
bool launch_fused_merged_t(int m, int Ly, int tile, const OpCoef& c, const ChebStep* w, const cplx<T>* r, const cplx<T>* v,
                           cplx<T>* t_out, const cplx<T>* rhat, const KScal* act, void* partials, cudaStream_t s,
                           const BatchLaunch* bl = nullptr);
// the pending u += alpha p + omega (r - alpha v) of amplitudes that stopped in this iteration
template <typename T>
void launch_final_update(const cplx<T>* r, const cplx<T>* v, const cplx<T>* p, cplx<T>* u, const KScal* ks,
                         const OpCoef& c, cudaStream_t s, const BatchLaunch* bl = nullptr);
// s = r - alpha v; u += alpha p + omega s; r = s - omega t; partials (rhat, r), (r, r) in [J][kDotSlots][kDotBlocks]
template <typename T>
void launch_bicg_update(cplx<T>* r, const cplx<T>* v, const cplx<T>* p, cplx<T>* u, const cplx<T>* t,
                        const cplx<T>* rhat, const KScal* ks, void* partials, const OpCoef& c, cudaStream_t s);

// ---------------------------------------------------------------------------
// reduce.cu
// ---------------------------------------------------------------------------
// bl != nullptr: one launch over every run of a batch (partials of run r from slot r J kDotSlots kDotBlocks)
template <typename T>
void launch_dots(int npair, const DotPairs<T>& pr, void* partials, const OpCoef& c, const KScal* act,
                 cudaStream_t s, const BatchLaunch* bl = nullptr);
// npart: partial-sum slots per (amplitude, pair); layout [J][kDotSlots][npart].
template <typename T>
void launch_finalize(int npair, const void* partials, KScal* k, int op, int J, cudaStream_t s,
                     int npart = kDotBlocks);
// partials in FP64 double2 layout regardless of T (for the fused FP64 residual)
void launch_finalize64(int npair, const void* partials, KScal* k, int op, int J, cudaStream_t s);
// batched runs: Krylov scalars k[run J + j]; npart_fixed > 0 for the k_dots layout
// (kDotBlocks), 0 for the fused-pipeline layout (RunGeom part_off, npart)
template <typename T>
void launch_finalize_batch(int npair, const void* partials, int npart_fixed, const BatchLaunch& bl, int J, KScal* k,
                           int op, cudaStream_t s);

}  // namespace apfc
