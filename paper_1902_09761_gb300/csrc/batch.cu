// Batched independent runs: many 2D simulations of one lattice, parameter set
// and spacing on grids of different sizes, advanced together.  Every stage of
// the step (arXiv:1902.09761, Alg. 1 with the nonlinear term explicit; the
// Sec. II.B preconditioner inside BiCGStab, FP32 Krylov in FP64 iterative
// refinement) is one launch over the work items of all runs: the block vectors
// of the runs sit one after another in shared arrays, a run table maps each
// block of a fused launch to (run, strip, row segment, amplitude), and each
// (run, amplitude) keeps its own Krylov scalars and convergence flag.  A run
// that has converged idles (its blocks return at once) while the others go on.
// The Krylov iteration blocks can be replayed from captured CUDA graphs.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "host_common.h"

using namespace apfc;

namespace {

constexpr int kBlocks = 10;        // r, rhat, p, v, u, t, r32, p', v', r'
constexpr int kDefaultRows = 128;  // rows per block segment of the fused pipeline
constexpr int kMaxRuns = 65536;
constexpr int kTuneIters = 6;      // merged iterations timed per autotuner candidate
constexpr int kTuneRows[] = {32, 48, 64, 96, 128, 192, 256};

}  // namespace

struct apfc_batch {
  apfc_lattice lat{};
  apfc_params par{};
  apfc_opts opts{};
  apfc_grid gmax{};  // largest nx, largest ny, and the spacings
  int R = 0, J = 0, flags = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<int> nx, ny;
  std::vector<RunGeom> rg;  // run table of the current tile / rows
  RunGeom* rg_dev = nullptr;
  BatchLaunch bl{};    // v-kernel partial layout
  BatchLaunch bl_t{};  // t-kernel partial layout (its own tile variant)
  long long elems = 0;  // complex entries of one concatenated block vector
  NonlinTable nt{};
  EnergyTable et{};
  OpCoef coef{};  // sizes of the largest run; kernels take each run's own from the table
  double coef_dt = -1.0;
  std::vector<ChebStep> cw;
  double2* x64 = nullptr;
  double2* b64 = nullptr;
  double2* b64_prev = nullptr;
  double2* r64_prev = nullptr;
  float2* blk[kBlocks] = {};
  uint2* rh16 = nullptr;  // rhat as packed bf16 pairs, [run][J][pts] (bf16pair.cuh)
  void* part_pipe = nullptr;  // fused-pipeline partials (run table layout)
  long long part_pipe_cap = 0;
  void* part_fix = nullptr;  // k_dots / FP64 residual partials: R J kDotSlots kDotBlocks slots
  KScal* ks = nullptr;
  KScal* ks_host = nullptr;
  KScal* ks64 = nullptr;
  KScal* ks64_host = nullptr;
  double* epart = nullptr;
  double* eout = nullptr;
  double* eout_host = nullptr;
  bool have_prev = false;
  double prev_dt = 0.0;
  std::vector<char> has_state;
  std::vector<apfc_stats_t> stats;
  bool failed = false;
  std::string err;
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};  // by starting side of the ping-pong buffers
  long long graph_replays = 0;
};

namespace {

apfc_status bfail(apfc_batch* b, apfc_status s, const std::string& msg) {
  if (b) {
    b->err = msg;
    if (s == APFC_ECUDA || s == APFC_ENAN || s == APFC_ENOMEM || s == APFC_ENOCONV) b->failed = true;
  }
  return s;
}

#define BK(call)                                                                              \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return bfail(b, e_ == cudaErrorMemoryAllocation ? APFC_ENOMEM : APFC_ECUDA,             \
                   std::string(#call) + ": " + cudaGetErrorString(e_));                       \
  } while (0)

int rows_of(const apfc_opts& o) { return o.tile_rows > 0 ? o.tile_rows : kDefaultRows; }
int tile_t_of(const apfc_opts& o) { return o.tile_t >= 0 ? o.tile_t : o.tile; }

// Run table for (tile, rows) of the v-kernel and tile_t of the t-kernel: element
// offsets and the partial-sum offsets of both layouts for every run.  Returns the
// partial slots the larger layout needs (the two kernels use the buffer in turn),
// or -1 when a fused launch would exceed the grid limit.
long long make_table(const apfc_batch* b, int tile, int rows, int tile_t, std::vector<RunGeom>& t) {
  t.resize(b->R);
  long long eoff = 0, poff = 0, poff_t = 0;
  const int m = b->opts.cheb_degree, eb = (int)sizeof(float2);
  for (int r = 0; r < b->R; ++r) {
    RunGeom& g = t[r];
    std::memset(&g, 0, sizeof(g));
    g.nx = b->nx[r];
    g.ny = b->ny[r];
    g.pts = (long long)g.nx * g.ny;
    g.elem_off = eoff;
    g.part_off = poff;
    g.part_off_t = poff_t;
    int np = 0, np_t = 0;
    const long long nb = fused2d_blocks(g.nx, g.ny, b->J, m, rows, eb, tile, false, nullptr);
    fused2d_blocks(g.nx, g.ny, b->J, m, rows, eb, tile, true, &np);
    fused2d_blocks(g.nx, g.ny, b->J, m, rows, eb, tile_t, true, &np_t);
    g.npart = np;
    g.npart_t = np_t;
    eoff += 2LL * b->J * g.pts;
    poff += (long long)b->J * kDotSlots * np;
    poff_t += (long long)b->J * kDotSlots * np_t;
    if (nb > 0x7fffffffLL) return -1;
  }
  return std::max(poff, poff_t);
}

void drop_graphs(apfc_batch* b) {
  for (auto& g : b->gexec)
    if (g) cudaGraphExecDestroy(g), g = nullptr;
}

// Install the run table of (tile, rows, tile_t) on the device.
apfc_status use_table(apfc_batch* b, int tile, int rows, int tile_t) {
  std::vector<RunGeom> t;
  const long long need = make_table(b, tile, rows, tile_t, t);
  if (need < 0) return bfail(b, APFC_ETOOBIG, "batch too large for one launch");
  if (need > b->part_pipe_cap) return bfail(b, APFC_EINVAL, "partial-sum buffer too small for this tile");
  BK(cudaMemcpyAsync(b->rg_dev, t.data(), sizeof(RunGeom) * b->R, cudaMemcpyHostToDevice, b->stream));
  BK(cudaStreamSynchronize(b->stream));
  b->rg = t;
  b->bl.dev = b->rg_dev;
  b->bl.host = b->rg.data();
  b->bl.R = b->R;
  b->bl.tlay = 0;
  b->bl_t = b->bl;
  b->bl_t.tlay = 1;
  drop_graphs(b);
  return APFC_OK;
}

bool set_coef(apfc_batch* b, double dt, std::string& e) {
  if (b->coef_dt == dt) return true;
  if (!make_coef(b->lat, b->par, b->gmax, b->opts.tau_mode, dt, b->coef, e)) return false;
  b->cw = cheb_weights_for(b->coef, b->gmax, b->opts.cheb_degree);
  b->coef_dt = dt;
  drop_graphs(b);  // the captured launches hold the coefficients by value
  return true;
}

OpCoef run_coef(const apfc_batch* b, int r) {
  OpCoef c = b->coef;
  c.nx = b->nx[r];
  c.ny = b->ny[r];
  c.nz = 1;
  c.pts = (long long)c.nx * c.ny;
  return c;
}

// ping-pong views of the Krylov vectors
struct Vecs {
  float2 *r[2], *p[2], *v[2], *rhat, *u, *t, *r32;
};
Vecs vecs(apfc_batch* b) {
  Vecs v;
  v.r[0] = b->blk[0];
  v.r[1] = b->blk[9];
  v.rhat = b->blk[1];
  v.p[0] = b->blk[2];
  v.p[1] = b->blk[7];
  v.v[0] = b->blk[3];
  v.v[1] = b->blk[8];
  v.u = b->blk[4];
  v.t = b->blk[5];
  v.r32 = b->blk[6];
  return v;
}

// `every` merged BiCGStab iterations over all runs, starting on side `cur`.
bool issue_block(apfc_batch* b, int cur, int every, int tile, int rows, int tile_t) {
  const Vecs x = vecs(b);
  const int m = b->opts.cheb_degree;
  cudaStream_t s = b->stream;
  for (int q = 0; q < every; ++q) {
    if (!launch_fused_merged_v<float>(m, rows, tile, b->coef, b->cw.data(), x.r[cur], x.v[cur], x.t, x.p[cur], x.u,
                                      x.r[1 - cur], x.p[1 - cur], x.v[1 - cur], x.rhat, b->rh16, b->ks, b->part_pipe, s,
                                      &b->bl))
      return false;
    launch_finalize_batch<float>(1, b->part_pipe, 0, b->bl, b->J, b->ks, OP_ALPHA, s);
    if (!launch_fused_merged_t<float>(m, rows, tile_t, b->coef, b->cw.data(), x.r[1 - cur], x.v[1 - cur], x.t,
                                      x.rhat, b->ks, b->part_pipe, s, &b->bl_t))
      return false;
    launch_finalize_batch<float>(5, b->part_pipe, 0, b->bl_t, b->J, b->ks, OP_OMEGA5, s);
    launch_final_update<float>(x.r[1 - cur], x.v[1 - cur], x.p[1 - cur], x.u, b->ks, b->coef, s, &b->bl);
    cur = 1 - cur;
  }
  return true;
}

apfc_status sync_ks(apfc_batch* b, KScal* dev, KScal* host) {
  BK(cudaGetLastError());
  BK(cudaMemcpyAsync(host, dev, sizeof(KScal) * b->R * b->J, cudaMemcpyDeviceToHost, b->stream));
  BK(cudaStreamSynchronize(b->stream));
  return APFC_OK;
}

// Start a BiCGStab solve of A P^{-1} u = r32 for every (run, amplitude); runs with
// skip[r] start converged.  fixed_tol >= 0: that relative tolerance for all; else the
// refinement's per-amplitude choice (inner_tol) from the outer residual norms.
// Leaves the scalars on the host; *any: some are active.
apfc_status krylov_init(apfc_batch* b, const std::vector<char>& skip, int max_iter, bool* any,
                        double fixed_tol = -1.0) {
  const Vecs x = vecs(b);
  cudaStream_t s = b->stream;
  const size_t bytes = sizeof(float2) * (size_t)b->elems;
  for (int r = 0; r < b->R; ++r)
    for (int j = 0; j < b->J; ++j) {
      KScal& k = b->ks_host[r * b->J + j];
      // r0 = b: a relative tolerance >= 1 stops at once; otherwise the run alone's choice
      const KScal& o = b->ks64_host[r * b->J + j];
      const double tj = skip[r]           ? 2.0
                        : fixed_tol >= 0.0 ? fixed_tol
                                           : inner_tol(b->opts.tol, b->opts.tol_inner, o.rnorm2, o.bnorm2);
      std::memset(&k, 0, sizeof(k));
      k.tolrel2 = tj * tj;
      k.max_iter = max_iter;
    }
  BK(cudaMemcpyAsync(b->ks, b->ks_host, sizeof(KScal) * b->R * b->J, cudaMemcpyHostToDevice, s));
  BK(cudaMemsetAsync(x.p[0], 0, bytes, s));
  BK(cudaMemsetAsync(x.v[0], 0, bytes, s));
  BK(cudaMemsetAsync(x.u, 0, bytes, s));
  BK(cudaMemsetAsync(x.t, 0, bytes, s));
  // r = r32 and the shadow residual rounded to bf16, as in a context alone: rho0 = (rhat, r0)
  launch_init32(x.r32, x.r[0], x.rhat, b->rh16, b->part_fix, b->coef, s, &b->bl);
  launch_finalize_batch<float>(3, b->part_fix, kDotBlocks, b->bl, b->J, b->ks, OP_INIT3, s);
  apfc_status st = sync_ks(b, b->ks, b->ks_host);
  if (st != APFC_OK) return st;
  *any = false;
  for (int i = 0; i < b->R * b->J; ++i) {
    if (b->ks_host[i].status == KS_NAN) return bfail(b, APFC_ENAN, "run " + std::to_string(i / b->J) + ": NaN/Inf");
    *any = *any || b->ks_host[i].active;
  }
  return APFC_OK;
}

// Iterate until every (run, amplitude) has stopped.
apfc_status krylov_iterate(apfc_batch* b, int max_iter, int tile, int rows, int tile_t) {
  const int every = std::max(1, b->opts.check_every);
  const bool graph = (b->flags & APFC_BATCH_GRAPH) && !profiler_on();
  int cur = 0;
  long long launched = 0, blocks = 0;
  while (true) {
    if (launched > (long long)max_iter + every) return bfail(b, APFC_ENOCONV, "Krylov iteration cap exceeded");
    launched += every;
    if (graph && blocks > 0) {
      // the first block ran eagerly (kernel attributes are set on first use)
      if (!b->gexec[cur]) {
        cudaGraph_t g = nullptr;
        BK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        const bool ok = issue_block(b, cur, every, tile, rows, tile_t);
        const cudaError_t ec = cudaStreamEndCapture(b->stream, &g);
        if (!ok) {
          if (g) cudaGraphDestroy(g);
          return bfail(b, APFC_EINVAL, "fused pipeline cannot run these options");
        }
        BK(ec);
        const cudaError_t ei = cudaGraphInstantiate(&b->gexec[cur], g, 0);
        cudaGraphDestroy(g);
        BK(ei);
      }
      BK(cudaGraphLaunch(b->gexec[cur], b->stream));
      b->graph_replays += 1;
    } else if (!issue_block(b, cur, every, tile, rows, tile_t)) {
      return bfail(b, APFC_EINVAL, "fused pipeline cannot run these options");
    }
    ++blocks;
    if (every & 1) cur = 1 - cur;
    apfc_status st = sync_ks(b, b->ks, b->ks_host);
    if (st != APFC_OK) return st;
    bool run = false;
    for (int i = 0; i < b->R * b->J; ++i) run = run || b->ks_host[i].active;
    if (!run) return APFC_OK;
  }
}

// One step of every run: FP32 Krylov solves inside FP64 iterative refinement.
apfc_status batch_step(apfc_batch* b) {
  cudaStream_t s = b->stream;
  const int tile = b->opts.tile, rows = rows_of(b->opts), tile_t = tile_t_of(b->opts);
  const Vecs x = vecs(b);
  double* part = reinterpret_cast<double*>(b->part_fix);
  bool resid_ready = false, bnorm_ready = false;
  if (b->have_prev && b->prev_dt == b->coef_dt) {
    // r0 = b - b_prev + r_prev; the new RHS goes to the other buffer
    launch_rhs_resid(b->x64, b->b64_prev, b->b64, b->r64_prev, x.r32, part, b->coef, b->nt, s, &b->bl);
    std::swap(b->b64, b->b64_prev);
    resid_ready = true;
  } else {
    // the new RHS and ||b||^2 (the same kernel as a context alone), r0 by stencil below
    launch_rhs_resid(b->x64, b->b64, nullptr, nullptr, x.r32, part, b->coef, b->nt, s, &b->bl);
    bnorm_ready = true;
  }
  b->have_prev = false;
  const double tol2 = b->opts.tol * b->opts.tol;
  std::vector<char> done(b->R, 0);
  std::vector<int> solves(b->R, 0), iters(b->R, 0);
  int sweep = 0;
  for (;; ++sweep) {
    if (resid_ready) {
      launch_finalize_batch<double>(2, part, kDotBlocks, b->bl, b->J, b->ks64, OP_NORMS, s);
    } else {
      if (sweep == 0) {
        if (bnorm_ready) {
          launch_finalize_batch<double>(2, part, kDotBlocks, b->bl, b->J, b->ks64, OP_NORMS, s);
        } else {
          DotPairs<double> d{{b->b64, nullptr, nullptr}, {b->b64, nullptr, nullptr}};
          launch_dots<double>(1, d, part, b->coef, nullptr, s, &b->bl);
          launch_finalize_batch<double>(1, part, kDotBlocks, b->bl, b->J, b->ks64, OP_BNORM, s);
        }
      }
      launch_residual_refine2d(b->b64, b->x64, x.r32, b->r64_prev, part, b->coef, s, &b->bl);
      launch_finalize_batch<double>(1, part, kDotBlocks, b->bl, b->J, b->ks64, OP_RNORM, s);
    }
    resid_ready = false;
    apfc_status st = sync_ks(b, b->ks64, b->ks64_host);
    if (st != APFC_OK) return st;
    bool all = true;
    for (int r = 0; r < b->R; ++r) {
      bool ok = true;
      for (int j = 0; j < b->J; ++j) {
        const KScal& k = b->ks64_host[r * b->J + j];
        if (!std::isfinite(k.rnorm2) || !std::isfinite(k.bnorm2))
          return bfail(b, APFC_ENAN, "run " + std::to_string(r) + ": residual norm is not finite");
        if (k.rnorm2 > tol2 * k.bnorm2) ok = false;
      }
      if (ok && !done[r]) done[r] = 1;
      all = all && done[r];
    }
    if (all) {
      // the last check of every run was a stencil residual of its final state
      b->have_prev = sweep > 0;
      b->prev_dt = b->coef_dt;
      break;
    }
    if (sweep >= b->opts.max_refine) {
      for (int r = 0; r < b->R; ++r)
        if (!done[r]) return bfail(b, APFC_ENOCONV, "run " + std::to_string(r) + ": refinement did not converge");
    }
    bool any = false;
    st = krylov_init(b, done, b->opts.max_iter, &any);
    if (st != APFC_OK) return st;
    if (any) {
      st = krylov_iterate(b, b->opts.max_iter, tile, rows, tile_t);
      if (st != APFC_OK) return st;
      // x += P^{-1} u (u = 0 for runs that did not iterate)
      if (!launch_fused_pinv_add<float>(b->opts.cheb_degree, rows, tile, b->coef, b->cw.data(), x.u, b->x64, s,
                                        &b->bl))
        return bfail(b, APFC_EINVAL, "fused pipeline cannot run these options");
    }
    for (int r = 0; r < b->R; ++r) {
      if (done[r]) continue;
      solves[r] += 1;
      int mx = 0;
      for (int j = 0; j < b->J; ++j) {
        const KScal& k = b->ks_host[r * b->J + j];
        if (k.status == KS_NAN) return bfail(b, APFC_ENAN, "run " + std::to_string(r) + ": NaN in the Krylov solve");
        mx = std::max(mx, k.iters);
      }
      iters[r] += mx;
    }
  }
  for (int r = 0; r < b->R; ++r) {
    apfc_stats_t& t = b->stats[r];
    t.steps += 1;
    t.iters_last = iters[r];
    t.iters_total += iters[r];
    t.refine_last = solves[r];
    double rr = 0.0;
    for (int j = 0; j < b->J; ++j) {
      const KScal& k = b->ks64_host[r * b->J + j];
      rr = std::max(rr, std::sqrt(k.rnorm2 / (k.bnorm2 > 0 ? k.bnorm2 : 1.0)));
    }
    t.resid_last = rr;
  }
  return APFC_OK;
}

bool valid_batch_opts(const apfc_opts& o, std::string& e) {
  if (!valid_opts(o, e)) return false;
  if (o.precision != APFC_FP32_REFINED) e = "batched runs use precision APFC_FP32_REFINED";
  else if (o.fused != 1) e = "batched runs use the fused pipeline (fused = 1)";
  else if (o.picard_iters != 1 || o.jacobian != 0) e = "batched runs take the explicit step (picard_iters 1, jacobian 0)";
  else if (o.guess != APFC_GUESS_PREV) e = "batched runs start each solve from the previous state (guess 0)";
  else if (o.cheb_degree < 1 || o.cheb_degree > fused2d_max_degree((int)sizeof(float2))) e = "cheb_degree";
  else return true;
  return false;
}

void free_batch(apfc_batch* b) {
  if (b->stream) cudaStreamSynchronize(b->stream);
  drop_graphs(b);
  cudaFree(b->rg_dev);
  cudaFree(b->x64);
  cudaFree(b->b64);
  cudaFree(b->b64_prev);
  cudaFree(b->r64_prev);
  for (auto& p : b->blk) cudaFree(p);
  cudaFree(b->rh16);
  cudaFree(b->part_pipe);
  cudaFree(b->part_fix);
  cudaFree(b->ks);
  cudaFree(b->ks64);
  cudaFree(b->epart);
  cudaFree(b->eout);
  if (b->ks_host) cudaFreeHost(b->ks_host);
  if (b->ks64_host) cudaFreeHost(b->ks64_host);
  if (b->eout_host) cudaFreeHost(b->eout_host);
  if (b->own_stream) cudaStreamDestroy(b->stream);
  delete b;
}

apfc_status check_run(apfc_batch* b, int run) {
  if (run < 0 || run >= b->R) return bfail(b, APFC_EINVAL, "run index out of range");
  return APFC_OK;
}

}  // namespace

// Why the last apfc_batch_init of this thread failed (apfc_batch_last_error(NULL)).
static thread_local std::string g_batch_init_err;

static apfc_status bfail(apfc_status s, const std::string& msg) {
  g_batch_init_err = msg;
  return s;
}

extern "C" {

apfc_status apfc_batch_init(apfc_batch** out, const apfc_lattice* lat, const apfc_params* p, int nruns, const int* nx,
                            const int* ny, double hx, double hy, const apfc_opts* opts, int flags, void* stream) {
  g_batch_init_err.clear();
  if (!out || !lat || !p || !nx || !ny) return bfail(APFC_EINVAL, "null argument");
  *out = nullptr;
  if (!valid_problem(*lat, *p) || lat->dim != 2) return bfail(APFC_EINVAL, "invalid lattice or parameters (batches are 2D)");
  if (nruns < 1 || nruns > kMaxRuns) return bfail(APFC_EINVAL, "run count out of range");
  if (!(hx > 0.0) || !(hy > 0.0) || !std::isfinite(hx) || !std::isfinite(hy))
    return bfail(APFC_EINVAL, "spacings must be positive and finite");
  if (flags & ~APFC_BATCH_GRAPH) return bfail(APFC_EINVAL, "unknown flags");
  long long total = 0;
  int mx = 0, my = 0;
  for (int r = 0; r < nruns; ++r) {
    if (nx[r] < 3 || ny[r] < 3 || nx[r] > (1 << 20) || ny[r] > (1 << 20))
      return bfail(APFC_EINVAL, "run " + std::to_string(r) + ": grid sizes must be in [3, 2^20]");
    total += (long long)nx[r] * ny[r];
    mx = std::max(mx, nx[r]);
    my = std::max(my, ny[r]);
  }
  apfc_opts o;
  apfc_default_opts(&o);
  o.precision = APFC_FP32_REFINED;
  if (opts) o = *opts;
  std::string e;
  if (!valid_batch_opts(o, e)) return bfail(APFC_EINVAL, "invalid option: " + e);
  if (total * 2LL * lat->J > (1LL << 40)) return bfail(APFC_ETOOBIG, "too many points in the batch");
  {
    int ndev = 0;
    const cudaError_t ce = cudaGetDeviceCount(&ndev);
    if (ce != cudaSuccess || ndev == 0)
      return bfail(APFC_ECUDA, std::string("no CUDA device: ") +
                                   (ce != cudaSuccess ? cudaGetErrorString(ce) : "device count 0"));
  }

  apfc_batch* b = new (std::nothrow) apfc_batch();
  if (!b) return bfail(APFC_ENOMEM, "host allocation of the batch failed");
  b->lat = *lat;
  b->par = *p;
  b->opts = o;
  b->R = nruns;
  b->J = lat->J;
  b->flags = flags;
  b->nx.assign(nx, nx + nruns);
  b->ny.assign(ny, ny + nruns);
  b->gmax.n[0] = mx;
  b->gmax.n[1] = my;
  b->gmax.n[2] = 1;
  b->gmax.h[0] = hx;
  b->gmax.h[1] = hy;
  b->gmax.h[2] = 1.0;
  b->elems = 2LL * b->J * total;
  b->has_state.assign(nruns, 0);
  b->stats.assign(nruns, apfc_stats_t{});
  auto cleanup = [&](apfc_status s) {
    if (g_batch_init_err.empty())
      g_batch_init_err = s == APFC_ENOMEM ? "device allocation failed"
                         : s == APFC_ECUDA   ? std::string("CUDA call failed: ") + cudaGetErrorString(cudaGetLastError())
                         : s == APFC_ETOOBIG ? "the batch exceeds the partial-sum table of the fused kernels"
                                             : "invalid batch";
    free_batch(b);
    return s;
  };
  if (!build_tables(*lat, *p, b->nt, b->et, e)) {
    g_batch_init_err = "nonlinear-term table: " + e;
    return cleanup(APFC_EINVAL);
  }
  b->stream = static_cast<cudaStream_t>(stream);
  if ((flags & APFC_BATCH_GRAPH) && b->stream == nullptr) {
    // graph capture needs a stream other than the legacy default one
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) return cleanup(APFC_ECUDA);
    b->own_stream = true;
  }
  // partial-sum capacity: the largest table over every tile variant and row count
  long long cap = 0;
  for (int tile = 0; tile < fused2d_tiles(); ++tile)
    for (int rows : {32, 64, 128, 256, 512, 1024, o.tile_rows}) {
      if (rows <= 0) continue;
      std::vector<RunGeom> t;
      const long long need = make_table(b, tile, rows, tile, t);
      if (need < 0) return cleanup(APFC_ETOOBIG);
      cap = std::max(cap, need);
    }
  b->part_pipe_cap = cap;
  const size_t blk64 = sizeof(double2) * (size_t)b->elems, blk32 = sizeof(float2) * (size_t)b->elems;
  const size_t nks = sizeof(KScal) * (size_t)nruns * b->J;
  if (cudaMalloc(&b->rg_dev, sizeof(RunGeom) * nruns) != cudaSuccess) return cleanup(APFC_ENOMEM);
  for (double2** q : {&b->x64, &b->b64, &b->b64_prev, &b->r64_prev})
    if (cudaMalloc(q, blk64) != cudaSuccess) return cleanup(APFC_ENOMEM);
  for (auto& q : b->blk)
    if (cudaMalloc(&q, blk32) != cudaSuccess) return cleanup(APFC_ENOMEM);
  if (cudaMalloc(&b->rh16, sizeof(uint2) * (size_t)(b->elems / 2)) != cudaSuccess) return cleanup(APFC_ENOMEM);
  if (cudaMalloc(&b->part_pipe, 16ull * (size_t)cap) != cudaSuccess) return cleanup(APFC_ENOMEM);
  if (cudaMalloc(&b->part_fix, 16ull * kDotSlots * kDotBlocks * (size_t)nruns * b->J) != cudaSuccess)
    return cleanup(APFC_ENOMEM);
  if (cudaMalloc(&b->ks, nks) != cudaSuccess || cudaMalloc(&b->ks64, nks) != cudaSuccess) return cleanup(APFC_ENOMEM);
  if (cudaMallocHost(&b->ks_host, nks) != cudaSuccess || cudaMallocHost(&b->ks64_host, nks) != cudaSuccess)
    return cleanup(APFC_ENOMEM);
  if (cudaMalloc(&b->epart, sizeof(double) * kDotBlocks) != cudaSuccess) return cleanup(APFC_ENOMEM);
  if (cudaMalloc(&b->eout, sizeof(double)) != cudaSuccess) return cleanup(APFC_ENOMEM);
  if (cudaMallocHost(&b->eout_host, sizeof(double)) != cudaSuccess) return cleanup(APFC_ENOMEM);
  std::memset(b->ks_host, 0, nks);
  std::memset(b->ks64_host, 0, nks);
  // the zeta-parts of the right-hand sides stay zero
  if (cudaMemsetAsync(b->x64, 0, blk64, b->stream) != cudaSuccess) return cleanup(APFC_ECUDA);
  if (cudaMemsetAsync(b->b64, 0, blk64, b->stream) != cudaSuccess) return cleanup(APFC_ECUDA);
  if (cudaMemsetAsync(b->b64_prev, 0, blk64, b->stream) != cudaSuccess) return cleanup(APFC_ECUDA);
  if (cudaMemsetAsync(b->ks64, 0, nks, b->stream) != cudaSuccess) return cleanup(APFC_ECUDA);
  if (use_table(b, o.tile, rows_of(o), tile_t_of(o)) != APFC_OK) return cleanup(APFC_ECUDA);
  if (!set_coef(b, 1.0, e)) return cleanup(APFC_EINVAL);
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return cleanup(APFC_ECUDA);
  *out = b;
  return APFC_OK;
}

apfc_status apfc_batch_set_opts(apfc_batch* b, const apfc_opts* opts) {
  if (!b || !opts) return APFC_EINVAL;
  std::string e;
  if (!valid_batch_opts(*opts, e)) return bfail(b, APFC_EINVAL, e);
  const bool retable = opts->tile != b->opts.tile || rows_of(*opts) != rows_of(b->opts) ||
                       tile_t_of(*opts) != tile_t_of(b->opts) || opts->cheb_degree != b->opts.cheb_degree;
  const apfc_opts old = b->opts;
  b->opts = *opts;
  if (retable) {
    std::vector<RunGeom> t;
    if (make_table(b, opts->tile, rows_of(*opts), tile_t_of(*opts), t) > b->part_pipe_cap) {
      b->opts = old;
      return bfail(b, APFC_EINVAL, "tile_rows outside the sizes the batch was created for");
    }
    apfc_status st = use_table(b, opts->tile, rows_of(*opts), tile_t_of(*opts));
    if (st != APFC_OK) return st;
  }
  const double dt = b->coef_dt;
  b->coef_dt = -1.0;  // tau_mode or the degree may have changed
  if (!set_coef(b, dt > 0 ? dt : 1.0, e)) return bfail(b, APFC_EINVAL, e);
  drop_graphs(b);
  b->have_prev = false;
  return APFC_OK;
}

apfc_status apfc_batch_set_amplitudes(apfc_batch* b, int run, const void* eta, int where) {
  if (!b || !eta || (where != APFC_HOST && where != APFC_DEVICE)) return APFC_EINVAL;
  apfc_status st = check_run(b, run);
  if (st != APFC_OK) return st;
  const RunGeom& g = b->rg[run];
  const size_t row = sizeof(double2) * (size_t)g.pts;
  const cudaMemcpyKind k = where == APFC_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  BK(cudaMemcpy2DAsync(b->x64 + g.elem_off + g.pts, 2 * row, eta, row, row, b->J, k, b->stream));
  launch_zeta(b->x64 + g.elem_off, run_coef(b, run), b->stream);
  BK(cudaGetLastError());
  BK(cudaStreamSynchronize(b->stream));
  b->has_state[run] = 1;
  b->have_prev = false;
  b->failed = false;  // as on a context: new amplitudes clear a sticky error
  b->err.clear();
  b->stats[run] = apfc_stats_t{};
  return APFC_OK;
}

apfc_status apfc_batch_get_amplitudes(apfc_batch* b, int run, void* eta, int where) {
  if (!b || !eta || (where != APFC_HOST && where != APFC_DEVICE)) return APFC_EINVAL;
  apfc_status st = check_run(b, run);
  if (st != APFC_OK) return st;
  if (!b->has_state[run]) return bfail(b, APFC_ESTATE, "no amplitudes set for this run");
  const RunGeom& g = b->rg[run];
  const size_t row = sizeof(double2) * (size_t)g.pts;
  const cudaMemcpyKind k = where == APFC_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  BK(cudaMemcpy2DAsync(eta, row, b->x64 + g.elem_off + g.pts, 2 * row, row, b->J, k, b->stream));
  BK(cudaStreamSynchronize(b->stream));
  return APFC_OK;
}

apfc_status apfc_batch_step(apfc_batch* b, double dt, int n) {
  if (!b || n < 0) return APFC_EINVAL;
  if (b->failed) return APFC_ESTATE;
  for (int r = 0; r < b->R; ++r)
    if (!b->has_state[r]) return bfail(b, APFC_ESTATE, "no amplitudes set for run " + std::to_string(r));
  std::string e;
  if (!set_coef(b, dt, e)) return bfail(b, APFC_EINVAL, e);
  for (int i = 0; i < n; ++i) {
    apfc_status st = batch_step(b);
    if (st != APFC_OK) return st;
  }
  return APFC_OK;
}

apfc_status apfc_batch_energy(apfc_batch* b, int run, double* F) {
  if (!b || !F) return APFC_EINVAL;
  apfc_status st = check_run(b, run);
  if (st != APFC_OK) return st;
  if (!b->has_state[run]) return bfail(b, APFC_ESTATE, "no amplitudes set for this run");
  launch_energy(b->x64 + b->rg[run].elem_off, b->epart, b->eout, run_coef(b, run), b->et, b->par.Bx, b->stream);
  BK(cudaGetLastError());
  BK(cudaMemcpyAsync(b->eout_host, b->eout, sizeof(double), cudaMemcpyDeviceToHost, b->stream));
  BK(cudaStreamSynchronize(b->stream));
  *F = b->gmax.h[0] * b->gmax.h[1] * b->eout_host[0];
  return APFC_OK;
}

apfc_status apfc_batch_stats(const apfc_batch* b, int run, apfc_stats_t* out) {
  if (!b || !out || run < 0 || run >= b->R) return APFC_EINVAL;
  *out = b->stats[run];
  return APFC_OK;
}

apfc_status apfc_batch_autotune(apfc_batch* b, double dt, int* tile_out, int* rows_out, double* ms_out) {
  if (!b) return APFC_EINVAL;
  if (b->failed) return APFC_ESTATE;
  for (int r = 0; r < b->R; ++r)
    if (!b->has_state[r]) return bfail(b, APFC_ESTATE, "no amplitudes set for run " + std::to_string(r));
  std::string e;
  if (!set_coef(b, dt, e)) return bfail(b, APFC_EINVAL, e);
  cudaStream_t s = b->stream;
  const Vecs x = vecs(b);
  // the first refinement residual of a step from the current state is the
  // right-hand side every candidate iterates on; the state is not changed
  double* part = reinterpret_cast<double*>(b->part_fix);
  launch_rhs(b->x64, b->b64, b->coef, b->nt, s, &b->bl);
  launch_residual_refine2d(b->b64, b->x64, x.r32, nullptr, part, b->coef, s, &b->bl);
  b->have_prev = false;
  cudaEvent_t e0, e1;
  BK(cudaEventCreate(&e0));
  BK(cudaEventCreate(&e1));
  int best_tile = b->opts.tile, best_rows = rows_of(b->opts), best_t = tile_t_of(b->opts);
  double best = 1e300;
  std::vector<char> none(b->R, 0);
  apfc_status st = APFC_OK;
  // time kTuneIters merged iterations for one (tile, rows, tile_t)
  auto time_candidate = [&](int tile, int rows, int tile_t, double* ms) -> apfc_status {
    *ms = 1e300;
    apfc_status s2 = use_table(b, tile, rows, tile_t);
    if (s2 != APFC_OK) return s2;
    for (int rep = 0; rep < 2; ++rep) {  // the first pass warms up
      bool any = false;
      // a tolerance no solve reaches within kTuneIters iterations
      if ((s2 = krylov_init(b, none, 1 << 20, &any, 1e-30)) != APFC_OK) return s2;
      BK(cudaEventRecord(e0, s));
      if (!issue_block(b, 0, kTuneIters, tile, rows, tile_t))
        return bfail(b, APFC_EINVAL, "fused pipeline cannot run these options");
      BK(cudaEventRecord(e1, s));
      BK(cudaEventSynchronize(e1));
      float f = 0.f;
      BK(cudaEventElapsedTime(&f, e0, e1));
      *ms = f;
    }
    return APFC_OK;
  };
  // pass 1: both kernels on one variant; pass 2: the t-kernel's variant with the rest fixed
  for (int tile = 0; tile < fused2d_tiles() && st == APFC_OK; ++tile)
    for (int rows : kTuneRows) {
      std::vector<RunGeom> t;
      if (make_table(b, tile, rows, tile, t) > b->part_pipe_cap) continue;
      double ms = 1e300;
      if ((st = time_candidate(tile, rows, tile, &ms)) != APFC_OK) break;
      if (ms < best) best = ms, best_tile = tile, best_rows = rows, best_t = tile;
    }
  for (int tile_t = 0; tile_t < fused2d_tiles() && st == APFC_OK; ++tile_t) {
    if (tile_t == best_t) continue;
    std::vector<RunGeom> t;
    if (make_table(b, best_tile, best_rows, tile_t, t) > b->part_pipe_cap) continue;
    double ms = 1e300;
    if ((st = time_candidate(best_tile, best_rows, tile_t, &ms)) != APFC_OK) break;
    if (ms < best) best = ms, best_t = tile_t;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != APFC_OK) return st;
  b->opts.tile = best_tile;
  b->opts.tile_rows = best_rows;
  b->opts.tile_t = best_t;
  st = use_table(b, best_tile, best_rows, best_t);
  if (st != APFC_OK) return st;
  if (tile_out) *tile_out = best_tile;
  if (rows_out) *rows_out = best_rows;
  if (ms_out) *ms_out = best / kTuneIters;
  return APFC_OK;
}

apfc_status apfc_batch_get_opts(const apfc_batch* b, apfc_opts* out) {
  if (!b || !out) return APFC_EINVAL;
  *out = b->opts;
  return APFC_OK;
}

long long apfc_batch_graph_replays(const apfc_batch* b) { return b ? b->graph_replays : -1; }

const char* apfc_batch_last_error(const apfc_batch* b) {
  if (b) return b->err.c_str();
  return g_batch_init_err.empty() ? "null batch" : g_batch_init_err.c_str();
}

void apfc_batch_destroy(apfc_batch* b) {
  if (b) free_batch(b);
}

apfc_status apfc_batch_profile_start(apfc_batch* b, int timed_id) {
  if (!b) return APFC_EINVAL;
  std::string e;
  if (!profiler_start(b->stream, timed_id, &b->coef.prof, e)) return bfail(b, APFC_EINVAL, e);
  return APFC_OK;
}

apfc_status apfc_batch_profile_read(apfc_batch* b, int id, double* ms, long long* launches, double* bytes,
                                    long long* all_launches) {
  if (!b) return APFC_EINVAL;
  std::string e;
  if (!profiler_read(b->stream, id, ms, launches, bytes, all_launches, e)) return bfail(b, APFC_EINVAL, e);
  return APFC_OK;
}

apfc_status apfc_batch_profile_stop(apfc_batch* b) {
  if (!b) return APFC_EINVAL;
  profiler_stop();
  b->coef.prof = nullptr;
  return APFC_OK;
}

}  // extern "C"
