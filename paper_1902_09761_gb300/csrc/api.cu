// C ABI of libapfc: context, validation, nonlinear-term tables, the Krylov
// driver and the time step (arXiv:1902.09761, Alg. 1 with one nonlinear
// iterate and the nonlinear term explicit; Sec. II.B for the solver).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "host_common.h"

using namespace apfc;

namespace {

constexpr int kFusedRows = 128;  // rows per block segment of the fused 2D pipeline

template <typename T>
struct Work {
  static constexpr int kBlocks = 11;  // r, rhat, p, v, u, t, z, bb, p', v', r' (ping-pong r, p, v)
  static constexpr int kFields = 5;  // f, b2p, R, Da, Db
  cplx<T>* blk[kBlocks] = {};
  cplx<T>* fld[kFields] = {};
  void* partials = nullptr;  // [J][kDotSlots][npart] x 16 bytes, npart <= npart_cap
  int npart_cap = 0;
  KScal* ks = nullptr;       // device
  KScal* ks_host = nullptr;  // pinned
  uint2* rh16 = nullptr;     // FP32: rhat as packed bf16 pairs [J][pts] (bf16pair.cuh)
  bool ready = false;
};

}  // namespace

// Process-wide measurement state (see apfc_profile_start in apfc.h).
namespace apfc {
struct Profiler {
  bool on = false;
  int timed = -1;
  cudaStream_t stream = nullptr;
  std::vector<cudaEvent_t> ev;  // begin/end pairs of the timed kernel(s)
  std::vector<int> ev_kid;      // kernel id of each pair
  size_t used = 0;
  long long launches[2 * KID_COUNT] = {};
  long long all = 0;
  unsigned long long* dev = nullptr;  // device byte counters [2 * KID_COUNT]
  bool failed = false;
};
static Profiler g_prof;

void prof_launch_begin(int kid, cudaStream_t s) {
  if (!g_prof.on) return;
  g_prof.launches[kid] += 1;
  g_prof.all += 1;
  if ((kid != g_prof.timed && g_prof.timed != -2) || g_prof.failed) return;
  if (g_prof.used + 2 > g_prof.ev.size()) {
    if (g_prof.ev.size() > 2000000) {
      g_prof.failed = true;
      return;
    }
    for (int i = 0; i < 2; ++i) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) {
        g_prof.failed = true;
        return;
      }
      g_prof.ev.push_back(e);
    }
    g_prof.ev_kid.resize(g_prof.ev.size() / 2);
  }
  g_prof.ev_kid[g_prof.used / 2] = kid;
  cudaEventRecord(g_prof.ev[g_prof.used], s);
}
void prof_launch_end(int kid, cudaStream_t s) {
  if (!g_prof.on || (kid != g_prof.timed && g_prof.timed != -2) || g_prof.failed) return;
  cudaEventRecord(g_prof.ev[g_prof.used + 1], s);
  g_prof.used += 2;
}

bool profiler_on() { return g_prof.on; }

bool profiler_start(cudaStream_t s, int timed_id, unsigned long long** dev, std::string& err) {
  if (timed_id < -2 || timed_id >= 2 * KID_COUNT) {
    err = "unknown kernel id";
    return false;
  }
  if (g_prof.on && g_prof.stream != s) {
    err = "measurement already running";
    return false;
  }
  cudaError_t e = cudaSuccess;
  if (!g_prof.dev) e = cudaMalloc(&g_prof.dev, sizeof(unsigned long long) * 2 * KID_COUNT);
  if (e == cudaSuccess) e = cudaMemsetAsync(g_prof.dev, 0, sizeof(unsigned long long) * 2 * KID_COUNT, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    err = std::string("measurement setup: ") + cudaGetErrorString(e);
    return false;
  }
  g_prof.on = true;
  g_prof.timed = timed_id;
  g_prof.stream = s;
  g_prof.used = 0;
  g_prof.failed = false;
  std::memset(g_prof.launches, 0, sizeof(g_prof.launches));
  g_prof.all = 0;
  *dev = g_prof.dev;
  return true;
}

bool profiler_read(cudaStream_t s, int id, double* ms, long long* launches, double* bytes, long long* all_launches,
                   std::string& err) {
  if (id < 0 || id >= 2 * KID_COUNT) {
    err = "unknown kernel id";
    return false;
  }
  if (!g_prof.dev) {
    err = "measurement was never started";
    return false;
  }
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    err = cudaGetErrorString(e);
    return false;
  }
  if (g_prof.failed) {
    err = "event pool exhausted";
    return false;
  }
  double total = 0.0;
  if (id == g_prof.timed || g_prof.timed == -2) {
    for (size_t i = 0; i + 1 < g_prof.used; i += 2) {
      if (g_prof.ev_kid[i / 2] != id) continue;
      float t = 0.f;
      e = cudaEventElapsedTime(&t, g_prof.ev[i], g_prof.ev[i + 1]);
      if (e != cudaSuccess) {
        err = cudaGetErrorString(e);
        return false;
      }
      total += t;
    }
  }
  unsigned long long b[2 * KID_COUNT];
  e = cudaMemcpy(b, g_prof.dev, sizeof(b), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    err = cudaGetErrorString(e);
    return false;
  }
  if (ms) *ms = total;
  if (launches) *launches = g_prof.launches[id];
  if (bytes) *bytes = (double)b[id];
  if (all_launches) *all_launches = g_prof.all;
  return true;
}

void profiler_stop() { g_prof.on = false; }
}  // namespace apfc

struct apfc_ctx {
  int sms = 152;  // multiprocessors of the context's device
  apfc_lattice lat;
  apfc_params par;
  apfc_grid grid;
  apfc_opts opts;
  cudaStream_t stream = nullptr;
  int J = 0, dim = 0;
  long long pts = 0;
  NonlinTable nt;
  EnergyTable et;
  double2* x64 = nullptr;  // state block vector (zeta, eta) per amplitude
  double2* b64 = nullptr;  // right-hand side block (0, rhs)
  // FP32-refined path: previous step's RHS and final FP64 residual (r = b - A x),
  // from which the next step's initial residual follows pointwise
  double2* b64_prev = nullptr;
  double2* r64_prev = nullptr;
  bool have_prev = false;
  double prev_dt = 0.0;
  // APFC_GUESS_EXTRAP: the state before the last completed explicit step of step size xprev_dt
  double2* x_prev = nullptr;
  bool have_xprev = false;
  double xprev_dt = 0.0;
  double* epart = nullptr;
  double* eout = nullptr;
  double* eout_host = nullptr;
  Work<double> w64;
  Work<float> w32;
  KScal* ks64 = nullptr;       // refinement norms (device)
  KScal* ks64_host = nullptr;  // pinned
  void* part64 = nullptr;      // refinement partials
  bool has_state = false;
  bool failed = false;
  std::string err;
  apfc_stats_t stats{};
  OpCoef coef{};
  double coef_dt = -1.0;
  // adjoint (allocated on first use): solve block x = (zeta', g), right-hand side
  // (0, lam), a scratch block for the energy gradient, four [J][pts] staging fields
  double2* xadj = nullptr;
  double2* badj = nullptr;
  double2* eblk = nullptr;
  double2* afld[4] = {};
  // checkpointed rollout: states every r_every steps plus the final one, and the
  // states of one segment recomputed during the backward pass
  double2* ckpt = nullptr;
  size_t ckpt_cap = 0;  // states
  double2* seg = nullptr;
  size_t seg_cap = 0;
  double r_dt = 0.0;
  int r_n = 0, r_every = 0;
  bool r_ready = false;
  // Picard iterations: eta^n, and kap_j D_j with the Jacobian
  double2* eta_step = nullptr;
  double* jd = nullptr;
  float2* jd32 = nullptr;
  // contiguous device copy of host amplitudes (one full-bandwidth host-to-device copy)
  double2* stage = nullptr;
};

namespace {

apfc_status fail(apfc_ctx* c, apfc_status s, const std::string& msg) {
  if (c) {
    c->err = msg;
    if (s == APFC_ECUDA || s == APFC_ENAN || s == APFC_ENOMEM) c->failed = true;
  }
  return s;
}

#define CK(call)                                                                              \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? APFC_ENOMEM : APFC_ECUDA,            \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                        \
  } while (0)

template <typename T>
size_t block_bytes(const apfc_ctx* c) {
  return sizeof(cplx<T>) * 2ull * (size_t)c->J * (size_t)c->pts;
}
template <typename T>
size_t field_bytes(const apfc_ctx* c) {
  return sizeof(cplx<T>) * (size_t)c->J * (size_t)c->pts;
}

template <typename T>
apfc_status alloc_work(apfc_ctx* ctx, Work<T>& w) {
  if (w.ready) return APFC_OK;
  for (auto& b : w.blk) CK(cudaMalloc(&b, block_bytes<T>(ctx)));
  for (auto& f : w.fld) CK(cudaMalloc(&f, field_bytes<T>(ctx)));
  // partial-sum slots: the unfused reductions use kDotBlocks; the fused pipeline one per block
  int cap = kDotBlocks;
  if (ctx->dim == 2) {
    OpCoef g{};
    g.nx = ctx->grid.n[0];
    g.ny = ctx->grid.n[1];
    g.nz = 1;
    g.pts = ctx->pts;
    for (int m = 1; m <= fused2d_max_degree((int)sizeof(cplx<T>)); ++m)
      for (int tile = 0; tile < fused2d_tiles(); ++tile)
        for (int rows : {32, 64, 128, 256, 512, 1024, ctx->opts.tile_rows})
          if (rows > 0) cap = std::max(cap, fused2d_npart(g, m, rows, (int)sizeof(cplx<T>), tile));
  }
  if (ctx->dim == 3) {
    OpCoef g{};
    g.nx = ctx->grid.n[0];
    g.ny = ctx->grid.n[1];
    g.nz = ctx->grid.n[2];
    g.J = ctx->J;
    cap = std::max(cap, stream3d_parts(g, (int)sizeof(cplx<T>)));
  }
  w.npart_cap = cap;
  CK(cudaMalloc(&w.partials, 16ull * kDotSlots * cap * ctx->J));
  CK(cudaMalloc(&w.ks, sizeof(KScal) * ctx->J));
  if (sizeof(T) == 4) CK(cudaMalloc(&w.rh16, sizeof(uint2) * (size_t)ctx->J * (size_t)ctx->pts));
  CK(cudaMallocHost(&w.ks_host, sizeof(KScal) * ctx->J));
  std::memset(w.ks_host, 0, sizeof(KScal) * ctx->J);
  CK(cudaMemsetAsync(w.blk[7], 0, block_bytes<T>(ctx), ctx->stream));
  w.ready = true;
  return APFC_OK;
}

template <typename T>
void free_work(Work<T>& w) {
  for (auto& b : w.blk) cudaFree(b), b = nullptr;
  for (auto& f : w.fld) cudaFree(f), f = nullptr;
  cudaFree(w.partials);
  cudaFree(w.ks);
  cudaFree(w.rh16);
  w.rh16 = nullptr;
  if (w.ks_host) cudaFreeHost(w.ks_host);
  w.partials = nullptr;
  w.ks = nullptr;
  w.ks_host = nullptr;
  w.ready = false;
}

}  // namespace

// ---------------------------------------------------------------------------
// Operator coefficients for a time step dt
// ---------------------------------------------------------------------------
const char* apfc::make_coef_into(const apfc_lattice& lat, const apfc_params& par, const apfc_grid& grid,
                                 int tau_mode, double dt, OpCoef& o) {
  if (!(dt > 0.0) || !std::isfinite(dt)) return "dt must be positive and finite";
  unsigned long long* prof = o.prof;
  std::memset(&o, 0, sizeof(o));
  o.prof = prof;
  const int dim = lat.dim;
  o.J = lat.J;
  o.dim = dim;
  o.nx = grid.n[0];
  o.ny = grid.n[1];
  o.nz = dim == 3 ? grid.n[2] : 1;
  o.pts = (long long)o.nx * o.ny * o.nz;
  double lapmax = 0.0;
  for (int d = 0; d < dim; ++d) {
    const double h = grid.h[d];
    o.ih2[d] = 1.0 / (h * h);
    o.c0 -= 2.0 / (h * h);
    lapmax += 4.0 / (h * h);
  }
  o.inv_dt = 1.0 / dt;
  for (int j = 0; j < lat.J; ++j) {
    double kap = 0.0;
    for (int d = 0; d < dim; ++d) {
      o.kh[j][d] = lat.k[j][d] / grid.h[d];
      kap += lat.k[j][d] * lat.k[j][d];
    }
    o.kap[j] = kap;
    o.kt[j] = kap * par.Bx;
    o.a[j] = 1.0 / dt + kap * par.dB;
    const double inv_tau = 1.0 / dt + (tau_mode == APFC_TAU_FOLD ? kap * par.dB : 0.0);
    if (!(o.a[j] > 0.0) || !(inv_tau > 0.0) || !(o.kt[j] > 0.0)) return "need 1/dt + |k_j|^2 dB > 0 and |k_j|^2 Bx > 0";
    o.sD[j] = std::sqrt(inv_tau);
    o.mu[j] = std::sqrt(o.kt[j]);
    o.inv_mu[j] = 1.0 / o.mu[j];
    const double lmin = o.sD[j], lmax = o.sD[j] + o.mu[j] * lapmax;
    o.inv_theta[j] = 2.0 / (lmax + lmin);
  }
  return nullptr;
}

bool apfc::make_coef(const apfc_lattice& lat, const apfc_params& par, const apfc_grid& grid, int tau_mode, double dt,
                     OpCoef& o, std::string& err) {
  const char* e = make_coef_into(lat, par, grid, tau_mode, dt, o);
  if (e) err = e;
  return e == nullptr;
}

std::vector<ChebStep> apfc::cheb_weights_for(const OpCoef& c, const apfc_grid& grid, int m) {
  std::vector<ChebStep> w(std::max(m, 1));
  cheb_weights_into(c, grid, m, w.data());
  return w;
}

double apfc::inner_tol(double tol, double tol_inner, double rnorm2, double bnorm2) {
  if (!(bnorm2 > 0.0)) return tol_inner;
  if (rnorm2 <= tol * tol * bnorm2) return 2.0;
  const double want = 0.25 * tol * std::sqrt(bnorm2 / rnorm2);
  return std::min(0.5, std::max(tol_inner, want));
}

void apfc::cheb_weights_into(const OpCoef& c, const apfc_grid& grid, int m, ChebStep* w) {
  std::memset(w, 0, sizeof(ChebStep) * std::max(m, 1));
  double lapmax = 0.0;
  for (int d = 0; d < c.dim; ++d) lapmax += 4.0 / (grid.h[d] * grid.h[d]);
  for (int j = 0; j < c.J; ++j) {
    const double lmin = c.sD[j], lmax = c.sD[j] + c.mu[j] * lapmax;
    const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin), sigma = theta / delta;
    double rho = 1.0 / sigma;
    for (int k = 0; k < m; ++k) {
      const double rn = 1.0 / (2.0 * sigma - rho);
      w[k].c1[j] = rn * rho;
      w[k].c2[j] = 2.0 * rn / delta;
      rho = rn;
    }
  }
}

namespace {

bool build_coef(apfc_ctx* c, double dt, std::string& err) {
  if (c->coef_dt == dt) return true;
  if (!make_coef(c->lat, c->par, c->grid, c->opts.tau_mode, dt, c->coef, err)) return false;
  c->coef_dt = dt;
  return true;
}

// Chebyshev recurrence weights (Saad, Sec. 12.3) for application k of D.
std::vector<ChebStep> cheb_weights(const apfc_ctx* c) { return cheb_weights_for(c->coef, c->grid, c->opts.cheb_degree); }

// ---------------------------------------------------------------------------
// Nonlinear-term tables from the resonance rule: <n^p> keeps the ordered
// p-tuples of signed modes (j, s) whose wavevectors s k_j sum to zero.
// ---------------------------------------------------------------------------
struct Mode {
  int j, s;
  bool operator<(const Mode& o) const { return j != o.j ? j < o.j : s < o.s; }
  bool operator==(const Mode& o) const { return j == o.j && s == o.s; }
};

void enumerate(const apfc_lattice& L, int p, std::map<std::vector<Mode>, int>& out) {
  const int nm = 2 * L.J;
  std::vector<int> idx(p, 0);
  while (true) {
    double v[3] = {0, 0, 0};
    for (int q = 0; q < p; ++q) {
      const int j = idx[q] >> 1, s = (idx[q] & 1) ? -1 : 1;
      for (int d = 0; d < L.dim; ++d) v[d] += s * L.k[j][d];
    }
    bool zero = true;
    for (int d = 0; d < L.dim; ++d) zero = zero && std::fabs(v[d]) < 1e-9;
    if (zero) {
      std::vector<Mode> m;
      for (int q = 0; q < p; ++q) m.push_back(Mode{idx[q] >> 1, (idx[q] & 1) ? -1 : 1});
      std::sort(m.begin(), m.end());
      out[m] += 1;
    }
    int q = p - 1;
    while (q >= 0 && ++idx[q] == nm) idx[q--] = 0;
    if (q < 0) break;
  }
}

inline int code_of(const Mode& m) { return 2 * m.j + (m.s < 0 ? 1 : 0); }

}  // namespace

bool apfc::build_tables(const apfc_lattice& L, const apfc_params& P, NonlinTable& nt, EnergyTable& et, std::string& err) {
  std::memset(&nt, 0, sizeof(nt));
  std::memset(&et, 0, sizeof(et));
  nt.t = et.t = P.t;
  nt.v = et.v = P.v;
  et.dB = P.dB;
  nt.hex = et.hex = (L.lattice == APFC_LATTICE_HEX2D) ? 1 : 0;
  if (nt.hex) return true;
  std::map<std::vector<Mode>, int> m3, m4;
  enumerate(L, 3, m3);
  enumerate(L, 4, m4);
  const double c3 = -P.t / 3.0, c4 = 0.25 * P.v;
  int n = 0;
  for (int j = 0; j < L.J; ++j) {
    nt.start[j] = n;
    for (int pass = 0; pass < 2; ++pass) {
      const auto& tab = pass == 0 ? m3 : m4;
      const double cp = pass == 0 ? c3 : c4;
      for (const auto& kv : tab) {
        const Mode target{j, -1};
        const int cnt = (int)std::count(kv.first.begin(), kv.first.end(), target);
        if (cnt == 0) continue;
        if (n >= kMaxTerms) {
          err = "nonlinear table too large for this lattice";
          return false;
        }
        std::vector<Mode> rest = kv.first;
        rest.erase(std::find(rest.begin(), rest.end(), target));
        nt.coef[n] = cp * kv.second * cnt;
        nt.nf[n] = (int)rest.size();
        for (size_t q = 0; q < rest.size(); ++q) nt.f[n][q] = code_of(rest[q]);
        ++n;
      }
    }
  }
  nt.start[L.J] = n;
  // gather the monomials |eta_m|^2 eta_j (modes (j,+1), (m,+1), (m,-1)) into weights
  int nr = 0;
  for (int j = 0; j < L.J; ++j) {
    nt.rstart[j] = nr;
    for (int q = nt.start[j]; q < nt.start[j + 1]; ++q) {
      int diag_m = -1;
      if (nt.nf[q] == 3) {
        int cj = -1;  // position of an unconjugated eta_j factor
        for (int a = 0; a < 3; ++a)
          if (nt.f[q][a] == 2 * j) cj = a;
        if (cj >= 0) {
          const int o1 = nt.f[q][(cj + 1) % 3], o2 = nt.f[q][(cj + 2) % 3];
          if ((o1 >> 1) == (o2 >> 1) && (o1 & 1) != (o2 & 1)) diag_m = o1 >> 1;
        }
      }
      if (diag_m >= 0) {
        nt.wdiag[j][diag_m] += nt.coef[q];
      } else {
        nt.ridx[nr++] = q;
      }
    }
  }
  nt.rstart[L.J] = nr;
  int ne = 0;
  for (int pass = 0; pass < 2; ++pass) {
    const auto& tab = pass == 0 ? m3 : m4;
    const double cp = pass == 0 ? c3 : c4;
    for (const auto& kv : tab) {
      if (ne >= kMaxTerms) {
        err = "energy table too large for this lattice";
        return false;
      }
      et.coef[ne] = cp * kv.second;
      et.nf[ne] = (int)kv.first.size();
      for (size_t q = 0; q < kv.first.size(); ++q) et.f[ne][q] = code_of(kv.first[q]);
      ++ne;
    }
  }
  et.ne = ne;
  return true;
}

namespace {

// chi = P^{-1} beta (four steps of Sec. II.B, M = I).
template <typename T>
void apply_pinv(apfc_ctx* ctx, Work<T>& w, const cplx<T>* beta, cplx<T>* chi, const KScal* act,
                const std::vector<ChebStep>& cw) {
  const OpCoef& c = ctx->coef;
  const long long P = c.pts;
  FieldRef<T> f{w.fld[0], P}, b2p{w.fld[1], P}, R{w.fld[2], P};
  FieldRef<T> D[2] = {{w.fld[3], P}, {w.fld[4], P}};
  FieldRef<T> chi2{chi + P, 2 * P};
  const int m = ctx->opts.cheb_degree;
  auto cheb = [&](CFieldRef<T> src, FieldRef<T> X, const PcFin<T>* fin) {
    if (m == 0) {
      launch_cheb_zero<T>(src, X, c, act, ctx->stream);
      return;
    }
    launch_cheb_first<T>(src, X, R, D[0], cw[0], m == 1, c, act, ctx->stream, fin);
    int cur = 0;
    for (int k = 1; k < m; ++k) {
      launch_cheb_sweep<T>(CFieldRef<T>{D[cur].p, P}, X, R, D[1 - cur], cw[k], k == m - 1, c, act, ctx->stream,
                           fin);
      cur = 1 - cur;
    }
  };
  launch_pc_rhs<T>(beta, f, c, act, ctx->stream);
  cheb(CFieldRef<T>{f.p, P}, b2p, nullptr);
  if (c.dim == 3 && m > 0) {
    // step 4 rides on the last pass of the second solve
    const PcFin<T> fin{CFieldRef<T>{beta, 2 * P}, CFieldRef<T>{b2p.p, P}, FieldRef<T>{chi, 2 * P}};
    cheb(CFieldRef<T>{b2p.p, P}, chi2, &fin);
    return;
  }
  cheb(CFieldRef<T>{b2p.p, P}, chi2, nullptr);
  launch_pc_final<T>(beta, CFieldRef<T>{b2p.p, P}, chi, c, act, ctx->stream);
}

// Rows per block segment of the merged iteration's fused kernels: opts.tile_rows, else the
// automatic height, the tallest of 128, 64 and 32 rows that still gives the v-kernel's
// launch about 1.5 blocks per SM (taller segments waste less on the 3S-row pipeline fill,
// but on small grids they leave SMs idle: 512^2 runs twice as fast with 32-row segments as
// with 128).  x += P^{-1} u always takes the automatic height.
int fused_rows_auto(const apfc_ctx* ctx);
int fused_rows(const apfc_ctx* ctx) {
  if (ctx->opts.tile_rows > 0) return ctx->opts.tile_rows;
  return fused_rows_auto(ctx);
}
int fused_rows_auto(const apfc_ctx* ctx) {
  const int elem = ctx->opts.precision == APFC_FP64 ? (int)sizeof(double2) : (int)sizeof(float2);
  const int m = std::max(1, ctx->opts.cheb_degree);
  for (int rows : {kFusedRows, kFusedRows / 2}) {
    int np = 0;
    fused2d_blocks(ctx->grid.n[0], ctx->grid.n[1], ctx->J, m, rows, elem, ctx->opts.tile, true, &np);
    if (2LL * np * ctx->J >= 3LL * ctx->sms) return rows;
  }
  return kFusedRows / 4;
}

bool use_fused(const apfc_ctx* ctx, int elem_bytes) {
  return ctx->dim == 2 && ctx->opts.fused != 0 && (ctx->coef.jd == nullptr || ctx->opts.cheb_degree == 1) &&
         ctx->opts.cheb_degree >= 1 &&
         ctx->opts.cheb_degree <= fused2d_max_degree(elem_bytes);
}

template <typename T>
apfc_status sync_scalars(apfc_ctx* ctx, Work<T>& w) {
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(w.ks_host, w.ks, sizeof(KScal) * ctx->J, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return APFC_OK;
}

// Right-preconditioned BiCGStab on A_j x = b for all amplitudes at once.
// The iterate is kept as x = x0 + P^{-1} u, so P^{-1} is applied to the
// search directions only inside A P^{-1} and once at the end.
// T = double: b FP64, x0 = x64 (state), restarts from the true residual.
// T = float : b FP32, x0 = 0, the correction P^{-1} u is added to x64.
// Returns the worst per-amplitude KStatus; iterations in *iters (max over j).
template <typename T>
apfc_status krylov(apfc_ctx* ctx, Work<T>& w, const cplx<T>* b, double2* x64, double tol, int max_iter, int* iters,
                   int* worst, const double* tol_amp = nullptr) {
  const OpCoef& c = ctx->coef;
  cudaStream_t s = ctx->stream;
  cplx<T>*r = w.blk[0], *rhat = w.blk[1], *p = w.blk[2], *v = w.blk[3], *u = w.blk[4], *t = w.blk[5], *z = w.blk[6];
  const auto cw = cheb_weights(ctx);
  const size_t bb = block_bytes<T>(ctx);
  const bool fp64 = sizeof(T) == 8;
  const int attempts = fp64 ? 4 : 1;
  std::vector<int> it_sum(ctx->J, 0);
  *worst = KS_CONVERGED;
  for (int attempt = 0;; ++attempt) {
    // init: r = b - A x0, rhat = r, p = v = u = 0
    for (int j = 0; j < ctx->J; ++j) {
      const double tj = tol_amp ? tol_amp[j] : tol;  // per-amplitude relative tolerance, if given
      w.ks_host[j].tolrel2 = tj * tj;
      w.ks_host[j].max_iter = max_iter;
    }
    CK(cudaMemcpyAsync(w.ks, w.ks_host, sizeof(KScal) * ctx->J, cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(p, 0, bb, s));
    CK(cudaMemsetAsync(v, 0, bb, s));
    CK(cudaMemsetAsync(u, 0, bb, s));
    if (use_fused(ctx, (int)sizeof(cplx<T>))) CK(cudaMemsetAsync(t, 0, bb, s));
    if constexpr (sizeof(T) == 4) {
      // r = b (x0 = 0) and the shadow residual rhat = b rounded to bf16 (bf16pair.cuh),
      // rho0 = (rhat, r0), in one pass
      launch_init32(reinterpret_cast<const float2*>(b), reinterpret_cast<float2*>(r), reinterpret_cast<float2*>(rhat),
                    w.rh16, w.partials, c, s);
      launch_finalize<T>(3, w.partials, w.ks, OP_INIT3, ctx->J, s);
    } else {
      launch_residual<T>(b, reinterpret_cast<const cplx<T>*>(x64), r, rhat, c, s);
      DotPairs<T> d{{r, b, nullptr}, {r, b, nullptr}};
      launch_dots<T>(2, d, w.partials, c, nullptr, s);
      launch_finalize<T>(2, w.partials, w.ks, OP_INIT, ctx->J, s);
    }
    apfc_status st = sync_scalars(ctx, w);
    if (st != APFC_OK) return st;
    bool any = false;
    *worst = KS_CONVERGED;
    for (int j = 0; j < ctx->J; ++j) {
      any = any || w.ks_host[j].active;
      *worst = std::max(*worst, w.ks_host[j].status == KS_RUNNING ? KS_CONVERGED : w.ks_host[j].status);
    }
    if (*worst == KS_NAN) break;
    if (!any) break;  // every amplitude meets tol with its true residual
    if (attempt == attempts) {
      *worst = KS_NOCONV;
      break;
    }
    // iterate
    const int every = std::max(1, ctx->opts.check_every);
    const bool fused = use_fused(ctx, (int)sizeof(cplx<T>));
    const int m = ctx->opts.cheb_degree;
    const int tile = ctx->opts.tile, rows = fused_rows(ctx);
    const int npart = fused ? fused2d_npart(c, m, rows, (int)sizeof(cplx<T>), tile) : kDotBlocks;
    // the t-kernel is latency-bound: its own tile (less look-ahead, more blocks per SM)
    const int tile_t = ctx->opts.tile_t >= 0 ? ctx->opts.tile_t : tile;
    const int npart_t = fused ? fused2d_npart(c, m, rows, (int)sizeof(cplx<T>), tile_t) : kDotBlocks;
    const int npart3 = c.dim == 3 ? stream3d_parts(c, (int)sizeof(cplx<T>)) : kDotBlocks;
    cplx<T>* pp[2] = {p, w.blk[8]};
    cplx<T>* vv[2] = {v, w.blk[9]};
    cplx<T>* rr[2] = {r, w.blk[10]};
    int cur = 0;
    long long launched = 0;  // host-side cap: every amplitude stops at max_iter on the device
    while (true) {
      if (launched > (long long)max_iter + every) {
        *worst = KS_NOCONV;
        return fail(ctx, APFC_ENOCONV, "Krylov iteration cap exceeded on the host");
      }
      launched += every;
      for (int q = 0; q < every; ++q) {
        if (fused) {
          // merged iteration: r' = r - alpha v - omega t, p' = r' + beta (p - omega v),
          // u += alpha p + omega s (the previous iteration's update), v' = A P^{-1} p'
          if (!launch_fused_merged_v<T>(m, rows, tile, c, cw.data(), rr[cur], vv[cur], t, pp[cur], u, rr[1 - cur],
                                        pp[1 - cur], vv[1 - cur], rhat, w.rh16, w.ks, w.partials, s))
            return fail(ctx, APFC_EINVAL, "the fused pipeline cannot run these options");
          launch_finalize<T>(1, w.partials, w.ks, OP_ALPHA, ctx->J, s, npart);  // alpha = rho / (rhat, v')
          // t = A P^{-1} s, s = r' - alpha v'; omega, rho', beta and ||r''||^2 from five inner products
          launch_fused_merged_t<T>(m, rows, tile_t, c, cw.data(), rr[1 - cur], vv[1 - cur], t, rhat, w.ks,
                                   w.partials, s);
          launch_finalize<T>(5, w.partials, w.ks, OP_OMEGA5, ctx->J, s, npart_t);
          // amplitudes that stopped now still owe u += alpha p' + omega s
          launch_final_update<T>(rr[1 - cur], vv[1 - cur], pp[1 - cur], u, w.ks, c, s);
          cur = 1 - cur;
          continue;
        }
        // unfused iteration; the inner products come out of the passes that produce
        // their vectors (on 3D grids also those of A P^{-1})
        launch_p_update<T>(r, p, v, c, w.ks, s);
        apply_pinv<T>(ctx, w, p, z, w.ks, cw);
        if (c.dim == 3) {
          launch_apply_A_dots<T>(z, v, rhat, 1, w.partials, c, w.ks, s);  // (rhat, v)
          launch_finalize<T>(1, w.partials, w.ks, OP_ALPHA, ctx->J, s, npart3);
        } else {
          launch_apply_A<T>(z, v, c, w.ks, s);
          DotPairs<T> d{{rhat, nullptr, nullptr}, {v, nullptr, nullptr}};
          launch_dots<T>(1, d, w.partials, c, w.ks, s);
          launch_finalize<T>(1, w.partials, w.ks, OP_ALPHA, ctx->J, s);
        }
        launch_s_update<T>(r, v, c, w.ks, s, w.partials);  // (s, s)
        launch_finalize<T>(1, w.partials, w.ks, OP_SNORM, ctx->J, s);
        apply_pinv<T>(ctx, w, r, z, w.ks, cw);
        if (c.dim == 3) {
          launch_apply_A_dots<T>(z, t, r, 2, w.partials, c, w.ks, s);  // (t, s), (t, t)
          launch_finalize<T>(2, w.partials, w.ks, OP_OMEGA, ctx->J, s, npart3);
        } else {
          launch_apply_A<T>(z, t, c, w.ks, s);
          DotPairs<T> d{{t, t, nullptr}, {r, t, nullptr}};  // (t, s), (t, t)
          launch_dots<T>(2, d, w.partials, c, w.ks, s);
          launch_finalize<T>(2, w.partials, w.ks, OP_OMEGA, ctx->J, s);
        }
        launch_r_update<T>(r, t, u, p, c, w.ks, s, rhat, w.partials);  // u += alpha p + omega s; (rhat, r), (r, r)
        launch_finalize<T>(2, w.partials, w.ks, OP_RHO, ctx->J, s);
      }
      st = sync_scalars(ctx, w);
      if (st != APFC_OK) return st;
      bool run = false;
      for (int j = 0; j < ctx->J; ++j) run = run || w.ks_host[j].active;
      if (!run) break;
    }
    // x += P^{-1} u
    // x += P^{-1} u (three stages, no partial sums) keeps the automatic height: the taller
    // segments that suit the merged iteration leave its launch with too few blocks
    if (!fused || !launch_fused_pinv_add<T>(m, fused_rows_auto(ctx), tile, c, cw.data(), u, x64, s)) {
      apply_pinv<T>(ctx, w, u, z, nullptr, cw);
      launch_add_to<T>(z, x64, c, s);
    }
    *worst = KS_CONVERGED;
    for (int j = 0; j < ctx->J; ++j) {
      it_sum[j] += w.ks_host[j].iters;
      *worst = std::max(*worst, w.ks_host[j].status == KS_RUNNING ? KS_CONVERGED : w.ks_host[j].status);
    }
    if (!fp64) break;
    if (*worst == KS_NAN) break;
  }
  *iters = 0;
  for (int j = 0; j < ctx->J; ++j) *iters = std::max(*iters, it_sum[j]);
  CK(cudaGetLastError());
  return APFC_OK;
}

double max_rel_resid(const KScal* k, int J) {
  double r = 0.0;
  for (int j = 0; j < J; ++j) {
    const double b = k[j].bnorm2 > 0 ? k[j].bnorm2 : 1.0;
    r = std::max(r, std::sqrt(k[j].rnorm2 / b));
  }
  return r;
}

apfc_status status_of(apfc_ctx* ctx, int worst) {
  if (worst == KS_NAN) {
    if (tma_timeouts() > 0) return fail(ctx, APFC_ECUDA, "a TMA tile load did not complete within its wait limit");
    return fail(ctx, APFC_ENAN, "residual norm is not finite (NaN/Inf in the state?)");
  }
  if (worst == KS_NOCONV || worst == KS_BREAKDOWN)
    return fail(ctx, APFC_ENOCONV, "Krylov solve did not reach the tolerance within max_iter");
  return APFC_OK;
}

// One step in FP64.
// APFC_GUESS_EXTRAP, after the right-hand side has been formed from the state: replace the
// state by the extrapolated guess 2 x^n - x^(n-1) (keeping x^n) when the history is that of
// a completed step of the same size; else keep x^n as the guess and start the history.
// Returns whether the guess was extrapolated.
apfc_status guess_prepare(apfc_ctx* ctx, bool* extrapolated) {
  *extrapolated = false;
  if (ctx->opts.guess != APFC_GUESS_EXTRAP) return APFC_OK;
  const size_t blk = sizeof(double2) * 2ull * ctx->J * ctx->pts;
  if (!ctx->x_prev) {
    CK(cudaMalloc(&ctx->x_prev, blk));
    ctx->have_xprev = false;
  }
  if (ctx->have_xprev && ctx->xprev_dt == ctx->coef_dt) {
    launch_extrapolate(ctx->x64, ctx->x_prev, ctx->coef, ctx->stream);
    *extrapolated = true;
  } else {
    CK(cudaMemcpyAsync(ctx->x_prev, ctx->x64, blk, cudaMemcpyDeviceToDevice, ctx->stream));
  }
  CK(cudaGetLastError());
  ctx->have_xprev = false;  // valid again once this step has converged
  return APFC_OK;
}
void guess_done(apfc_ctx* ctx, int worst) {
  if (ctx->opts.guess == APFC_GUESS_EXTRAP && worst == KS_CONVERGED) {
    ctx->have_xprev = true;
    ctx->xprev_dt = ctx->coef_dt;
  }
}

apfc_status step_fp64(apfc_ctx* ctx) {
  ctx->have_prev = false;
  apfc_status st = alloc_work<double>(ctx, ctx->w64);
  if (st != APFC_OK) return st;
  launch_rhs(ctx->x64, ctx->b64, ctx->coef, ctx->nt, ctx->stream);
  bool ex = false;
  if ((st = guess_prepare(ctx, &ex)) != APFC_OK) return st;
  int iters = 0, worst = 0;
  st = krylov<double>(ctx, ctx->w64, ctx->b64, ctx->x64, ctx->opts.tol, ctx->opts.max_iter, &iters, &worst);
  if (st != APFC_OK) return st;
  guess_done(ctx, worst);
  ctx->stats.iters_last = iters;
  ctx->stats.iters_total += iters;
  ctx->stats.refine_last = 0;
  ctx->stats.resid_last = max_rel_resid(ctx->w64.ks_host, ctx->J);
  return status_of(ctx, worst);
}

// FP32 Krylov inside FP64 iterative refinement: A x = b to opts.tol, starting
// from x.  resid_ready: the FP32 initial residual and the partials of ||r0||^2 and
// ||b||^2 are already in place (the pointwise initial residual of a step).
// r64_keep != nullptr receives the FP64 residual b - A x of every stencil
// residual sweep.  *stencil_last: the final check was such a sweep.
// bnorm_ready: the partial sums hold ||b||^2 (slot 1) from the right-hand-side kernel
apfc_status refine_solve(apfc_ctx* ctx, const double2* b, double2* x, double2* r64_keep, bool resid_ready,
                         int* total_it, int* sweeps, int* worst_out, bool* stencil_last, bool bnorm_ready = false) {
  apfc_status st = alloc_work<float>(ctx, ctx->w32);
  if (st != APFC_OK) return st;
  cudaStream_t s = ctx->stream;
  float2* r32 = ctx->w32.blk[7];
  double* part = reinterpret_cast<double*>(ctx->part64);
  int total = 0, worst = KS_CONVERGED, sweep = 0;
  bool stencil = false;
  const double tol2 = ctx->opts.tol * ctx->opts.tol;
  for (;; ++sweep) {
    if (resid_ready) {
      launch_finalize64(2, ctx->part64, ctx->ks64, OP_NORMS, ctx->J, s);  // ||r0||^2 and ||b||^2
      stencil = false;
    } else {
      if (sweep == 0) {  // ||b||^2 once per solve
        if (bnorm_ready) {
          launch_finalize64(2, ctx->part64, ctx->ks64, OP_NORMS, ctx->J, s);  // its ||r||^2 slot is 0
        } else {
          DotPairs<double> d{{b, nullptr, nullptr}, {b, nullptr, nullptr}};
          launch_dots<double>(1, d, ctx->part64, ctx->coef, nullptr, s);
          launch_finalize64(1, ctx->part64, ctx->ks64, OP_BNORM, ctx->J, s);
        }
      }
      {
        const char* terr = nullptr;
        if (!launch_residual_refine_tma(b, x, r32, r64_keep, part, ctx->coef, s, &terr))
          return fail(ctx, APFC_ECUDA, terr ? terr : "TMA residual launch failed");
        launch_finalize64(1, ctx->part64, ctx->ks64, OP_RNORM, ctx->J, s);
      }
      stencil = true;
    }
    resid_ready = false;
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(ctx->ks64_host, ctx->ks64, sizeof(KScal) * ctx->J, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    bool done = true, bad = false;
    for (int j = 0; j < ctx->J; ++j) {
      const KScal& k = ctx->ks64_host[j];
      if (!std::isfinite(k.rnorm2) || !std::isfinite(k.bnorm2)) bad = true;
      if (k.rnorm2 > tol2 * k.bnorm2) done = false;
    }
    if (bad) {
      worst = KS_NAN;
      break;
    }
    if (done) {
      worst = KS_CONVERGED;
      break;
    }
    if (sweep >= ctx->opts.max_refine) {
      worst = KS_NOCONV;
      break;
    }
    // inner tolerance per amplitude: no further than the outer tolerance needs
    double tin[kMaxJ];
    for (int j = 0; j < ctx->J; ++j)
      tin[j] = inner_tol(ctx->opts.tol, ctx->opts.tol_inner, ctx->ks64_host[j].rnorm2, ctx->ks64_host[j].bnorm2);
    int it = 0, w = 0;
    st = krylov<float>(ctx, ctx->w32, r32, x, ctx->opts.tol_inner, ctx->opts.max_iter, &it, &w, tin);
    if (st != APFC_OK) return st;
    total += it;
    if (w == KS_NAN) {
      worst = KS_NAN;
      break;
    }
  }
  *total_it = total;
  *sweeps = sweep;
  *worst_out = worst;
  *stencil_last = stencil;
  return APFC_OK;
}

// One step with FP32 Krylov inside FP64 iterative refinement.
apfc_status step_refined(apfc_ctx* ctx) {
  cudaStream_t s = ctx->stream;
  const size_t blk = sizeof(double2) * 2ull * ctx->J * ctx->pts;
  if (ctx->r64_prev == nullptr) {
    CK(cudaMalloc(&ctx->b64_prev, blk));
    CK(cudaMalloc(&ctx->r64_prev, blk));
    CK(cudaMemsetAsync(ctx->b64_prev, 0, blk, s));
    ctx->have_prev = false;
  }
  apfc_status st = alloc_work<float>(ctx, ctx->w32);
  if (st != APFC_OK) return st;
  float2* r32 = ctx->w32.blk[7];
  double* part = reinterpret_cast<double*>(ctx->part64);
  bool resid_ready = false, bnorm_ready = false;
  if (ctx->have_prev && ctx->prev_dt == ctx->coef_dt) {
    // r0 = b - b_prev + r_prev with the previous step's final residual r_prev = b_prev - A x;
    // b_prev is the RHS that residual was taken against; the new RHS goes to the other buffer
    launch_rhs_resid(ctx->x64, ctx->b64_prev, ctx->b64, ctx->r64_prev, r32, part, ctx->coef, ctx->nt, s);
    std::swap(ctx->b64, ctx->b64_prev);
    resid_ready = true;
  } else {
    // no previous residual: the new RHS and its norm, the initial residual by stencil below
    launch_rhs_resid(ctx->x64, ctx->b64, nullptr, nullptr, r32, part, ctx->coef, ctx->nt, s);
    bnorm_ready = true;
  }
  ctx->have_prev = false;
  bool ex = false;
  if ((st = guess_prepare(ctx, &ex)) != APFC_OK) return st;
  if (ex && resid_ready) {
    // the pointwise r0 belongs to x^n, not to the guess: take a stencil residual; the RHS
    // kernel's ||b||^2 (slot 1 of its partial sums) still holds
    resid_ready = false;
    bnorm_ready = true;
  }
  int total_it = 0, sweeps = 0, worst = KS_CONVERGED;
  bool stencil_last = false;
  st = refine_solve(ctx, ctx->b64, ctx->x64, ctx->r64_prev, resid_ready, &total_it, &sweeps, &worst, &stencil_last,
                    bnorm_ready);
  if (st != APFC_OK) return st;
  guess_done(ctx, worst);
  // a TMA wait that gave up leaves its kernel's results incomplete: fail the step
  if (tma_timeouts() != 0) return fail(ctx, APFC_ECUDA, "a TMA tile load did not complete within its wait limit");
  if (worst == KS_CONVERGED) {
    // after at least one sweep the last check was a stencil residual of the final
    // state, kept in r64_prev: it seeds the next step's initial residual
    ctx->have_prev = sweeps > 0 && stencil_last;
    ctx->prev_dt = ctx->coef_dt;
  }
  ctx->stats.iters_last = total_it;
  ctx->stats.iters_total += total_it;
  ctx->stats.refine_last = sweeps;
  ctx->stats.resid_last = max_rel_resid(ctx->ks64_host, ctx->J);
  return status_of(ctx, worst);
}

apfc_status copy_in_block(apfc_ctx* ctx, double2* dst_dev, const void* src, int where) {
  const cudaMemcpyKind k = where == APFC_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  CK(cudaMemcpyAsync(dst_dev, src, sizeof(double2) * 2ull * ctx->J * ctx->pts, k, ctx->stream));
  return APFC_OK;
}
apfc_status copy_out_block(apfc_ctx* ctx, void* dst, const double2* src_dev, int where) {
  const cudaMemcpyKind k = where == APFC_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  CK(cudaMemcpyAsync(dst, src_dev, sizeof(double2) * 2ull * ctx->J * ctx->pts, k, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return APFC_OK;
}

// Copy one part (0 = zeta, 1 = eta) of the state block to/from [J][pts].
apfc_status copy_part(apfc_ctx* ctx, void* plain, int where, int part, bool to_state, int dtype = APFC_C128) {
  const size_t row = sizeof(double2) * (size_t)ctx->pts;
  double2* base = ctx->x64 + (size_t)part * ctx->pts;
  if (dtype == APFC_C64) {
    // complex64: converted on the device (host buffers pass through the staging field)
    const size_t bytes = sizeof(float2) * (size_t)ctx->pts * ctx->J;
    const bool host = where == APFC_HOST;
    if (host && !ctx->stage) CK(cudaMalloc(&ctx->stage, row * ctx->J));
    float2* dev = host ? reinterpret_cast<float2*>(ctx->stage) : static_cast<float2*>(plain);
    if (to_state) {
      if (host) CK(cudaMemcpyAsync(dev, plain, bytes, cudaMemcpyHostToDevice, ctx->stream));
      launch_c64_to_part(dev, ctx->x64, ctx->pts, ctx->J, part, ctx->stream);
      CK(cudaGetLastError());
    } else {
      launch_part_to_c64(ctx->x64, dev, ctx->pts, ctx->J, part, ctx->stream);
      CK(cudaGetLastError());
      if (host) CK(cudaMemcpyAsync(plain, dev, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return APFC_OK;
  }
  cudaMemcpyKind k;
  if (to_state)
    k = where == APFC_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  else
    k = where == APFC_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (to_state && where == APFC_HOST) {
    // a strided copy from host memory runs at a fraction of the link's bandwidth:
    // one contiguous copy to the device, then the strided copy on the device
    if (!ctx->stage) CK(cudaMalloc(&ctx->stage, row * ctx->J));
    CK(cudaMemcpyAsync(ctx->stage, plain, row * ctx->J, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpy2DAsync(base, 2 * row, ctx->stage, row, row, ctx->J, cudaMemcpyDeviceToDevice, ctx->stream));
  } else if (to_state) {
    CK(cudaMemcpy2DAsync(base, 2 * row, plain, row, row, ctx->J, k, ctx->stream));
  } else if (where == APFC_HOST) {
    // the same on the way out: the strided copy on the device, then one contiguous copy
    if (!ctx->stage) CK(cudaMalloc(&ctx->stage, row * ctx->J));
    CK(cudaMemcpy2DAsync(ctx->stage, row, base, 2 * row, row, ctx->J, cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaMemcpyAsync(plain, ctx->stage, row * ctx->J, cudaMemcpyDeviceToHost, ctx->stream));
  } else {
    CK(cudaMemcpy2DAsync(plain, row, base, 2 * row, row, ctx->J, k, ctx->stream));
  }
  CK(cudaStreamSynchronize(ctx->stream));
  return APFC_OK;
}


// ---------------------------------------------------------------------------
// Adjoint of the step and checkpointed rollouts
// ---------------------------------------------------------------------------
size_t field_elems(const apfc_ctx* ctx) { return (size_t)ctx->J * (size_t)ctx->pts; }

apfc_status alloc_adjoint(apfc_ctx* ctx) {
  if (ctx->xadj) return APFC_OK;
  const size_t blk = sizeof(double2) * 2 * field_elems(ctx), fld = sizeof(double2) * field_elems(ctx);
  CK(cudaMalloc(&ctx->xadj, blk));
  CK(cudaMalloc(&ctx->badj, blk));
  CK(cudaMalloc(&ctx->eblk, blk));
  for (auto& f : ctx->afld) CK(cudaMalloc(&f, fld));
  CK(cudaMemsetAsync(ctx->xadj, 0, blk, ctx->stream));
  CK(cudaMemsetAsync(ctx->badj, 0, blk, ctx->stream));  // its zeta-parts stay zero
  return APFC_OK;
}

// [J][pts] field <-> one part (0 zeta, 1 eta) of a block vector, device to device
apfc_status field_to_block(apfc_ctx* ctx, double2* block, int part, const double2* field) {
  const size_t row = sizeof(double2) * (size_t)ctx->pts;
  CK(cudaMemcpy2DAsync(block + (size_t)part * ctx->pts, 2 * row, field, row, row, ctx->J, cudaMemcpyDeviceToDevice,
                       ctx->stream));
  return APFC_OK;
}
apfc_status block_to_field(apfc_ctx* ctx, double2* field, const double2* block, int part) {
  const size_t row = sizeof(double2) * (size_t)ctx->pts;
  CK(cudaMemcpy2DAsync(field, row, block + (size_t)part * ctx->pts, 2 * row, row, ctx->J, cudaMemcpyDeviceToDevice,
                       ctx->stream));
  return APFC_OK;
}

// state = (G_h eta, eta) from a device [J][pts] field
apfc_status load_state(apfc_ctx* ctx, const double2* eta) {
  apfc_status st = field_to_block(ctx, ctx->x64, 1, eta);
  if (st != APFC_OK) return st;
  launch_zeta(ctx->x64, ctx->coef, ctx->stream);
  CK(cudaGetLastError());
  ctx->have_prev = false;
  ctx->have_xprev = false;
  return APFC_OK;
}

// A x = b to opts.tol in the context's precision, from the given x.
apfc_status solve_block(apfc_ctx* ctx, const double2* b, double2* x, int* iters) {
  int worst = KS_CONVERGED;
  apfc_status st;
  if (ctx->opts.precision == APFC_FP64) {
    if ((st = alloc_work<double>(ctx, ctx->w64)) != APFC_OK) return st;
    st = krylov<double>(ctx, ctx->w64, b, x, ctx->opts.tol, ctx->opts.max_iter, iters, &worst);
  } else {
    int sweeps = 0;
    bool stencil = false;
    st = refine_solve(ctx, b, x, nullptr, false, iters, &sweeps, &worst, &stencil);
  }
  if (st != APFC_OK) return st;
  return status_of(ctx, worst);
}

// lam_n = adjoint of one step applied to lam_np1 (all device [J][pts] fields);
// *dB_acc += the step's derivative through S with respect to dB.  warm: start the
// adjoint solve from the previous one's solution, else from zero.
apfc_status adjoint_step_dev(apfc_ctx* ctx, const double2* eta_n, const double2* eta_np1, const double2* lam_np1,
                             double2* lam_n, double* dB_acc, bool warm) {
  apfc_status st = alloc_adjoint(ctx);
  if (st != APFC_OK) return st;
  // g = S^{-1} lam_np1: S is Hermitian, so the adjoint solve is the block solve with
  // right-hand side (0, lam_np1); g is the eta-part of its solution
  if ((st = field_to_block(ctx, ctx->badj, 1, lam_np1)) != APFC_OK) return st;
  if (!warm) CK(cudaMemsetAsync(ctx->xadj, 0, sizeof(double2) * 2 * field_elems(ctx), ctx->stream));
  int iters = 0;
  if ((st = solve_block(ctx, ctx->badj, ctx->xadj, &iters)) != APFC_OK) return st;
  ctx->stats.iters_total += iters;
  launch_adj_nonlin(eta_n, ctx->xadj, eta_np1, lam_n, ctx->epart, ctx->eout, ctx->coef, ctx->nt, ctx->stream);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(ctx->eout_host, ctx->eout, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  *dB_acc -= ctx->eout_host[0];
  return APFC_OK;
}

// Real gradient of F at eta (device fields) and dF/d dB.
apfc_status energy_grad_dev(apfc_ctx* ctx, const double2* eta, double2* grad, double* dF_ddB) {
  apfc_status st = alloc_adjoint(ctx);
  if (st != APFC_OK) return st;
  if ((st = field_to_block(ctx, ctx->eblk, 1, eta)) != APFC_OK) return st;
  launch_zeta(ctx->eblk, ctx->coef, ctx->stream);
  double vol = 1.0;
  for (int d = 0; d < ctx->dim; ++d) vol *= ctx->grid.h[d];
  launch_energy_grad(ctx->eblk, grad, 2.0 * vol, ctx->par.dB, ctx->par.Bx, ctx->epart, ctx->eout, ctx->coef, ctx->nt,
                     ctx->stream);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(ctx->eout_host, ctx->eout, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (dF_ddB) *dF_ddB = vol * ctx->eout_host[0];
  return APFC_OK;
}

apfc_status ensure_states(apfc_ctx* ctx, double2** buf, size_t* cap, size_t n) {
  if (*cap >= n) return APFC_OK;
  cudaFree(*buf);
  *buf = nullptr;
  *cap = 0;
  CK(cudaMalloc(buf, sizeof(double2) * field_elems(ctx) * n));
  *cap = n;
  return APFC_OK;
}

// One step of Alg. 1 with K = picard_iters iterations, the Jacobian optional.
apfc_status step_picard(apfc_ctx* ctx) {
  const size_t fe = field_elems(ctx);
  if (!ctx->eta_step) CK(cudaMalloc(&ctx->eta_step, sizeof(double2) * fe));
  const bool jac = ctx->opts.jacobian != 0;
  if (jac && !ctx->jd) CK(cudaMalloc(&ctx->jd, sizeof(double) * fe));
  if (jac && !ctx->jd32) CK(cudaMalloc(&ctx->jd32, sizeof(float2) * fe));
  apfc_status st = block_to_field(ctx, ctx->eta_step, ctx->x64, 1);
  if (st != APFC_OK) return st;
  ctx->have_prev = false;
  ctx->have_xprev = false;
  int total = 0;
  for (int k = 0; k < ctx->opts.picard_iters; ++k) {
    // b and kap D from eta^(k-1), the eta-parts of the state; solve from x^(k-1)
    launch_rhs_picard(ctx->x64, ctx->eta_step, ctx->b64, jac ? ctx->jd : nullptr, jac ? ctx->jd32 : nullptr,
                      ctx->coef, ctx->nt, ctx->stream);
    ctx->coef.jd = jac ? ctx->jd : nullptr;
    ctx->coef.jd32 = jac ? ctx->jd32 : nullptr;
    int it = 0;
    st = solve_block(ctx, ctx->b64, ctx->x64, &it);
    ctx->coef.jd = nullptr;
    ctx->coef.jd32 = nullptr;
    total += it;
    if (st != APFC_OK) return st;
  }
  ctx->stats.iters_last = total;
  ctx->stats.iters_total += total;
  ctx->stats.refine_last = ctx->opts.picard_iters;
  ctx->stats.resid_last = max_rel_resid(ctx->opts.precision == APFC_FP64 ? ctx->w64.ks_host : ctx->ks64_host, ctx->J);
  return APFC_OK;
}

bool explicit_step(const apfc_ctx* ctx) { return ctx->opts.picard_iters == 1 && ctx->opts.jacobian == 0; }

apfc_status one_step(apfc_ctx* ctx) {
  apfc_status st = !explicit_step(ctx)               ? step_picard(ctx)
                   : ctx->opts.precision == APFC_FP64 ? step_fp64(ctx)
                                                      : step_refined(ctx);
  if (st == APFC_OK) ctx->stats.steps += 1;
  return st;
}

}  // namespace

bool apfc::valid_opts(const apfc_opts& o, std::string& e) {
  if (o.precision != APFC_FP64 && o.precision != APFC_FP32_REFINED) e = "precision";
  else if (o.krylov != APFC_BICGSTAB) e = "krylov";
  else if (o.max_iter < 1) e = "max_iter";
  else if (o.cheb_degree < 0 || o.cheb_degree > kMaxCheb) e = "cheb_degree";
  else if (o.tau_mode != APFC_TAU_FOLD && o.tau_mode != APFC_TAU_PLAIN) e = "tau_mode";
  else if (o.max_refine < 0) e = "max_refine";
  else if (o.check_every < 1) e = "check_every";
  else if (o.fused != 0 && o.fused != 1) e = "fused";
  else if (o.tile < 0 || o.tile >= fused2d_tiles()) e = "tile";
  else if (o.tile_t < -1 || o.tile_t >= fused2d_tiles()) e = "tile_t";
  else if (o.tile_rows < 0 || o.tile_rows > 65536) e = "tile_rows";
  else if (o.picard_iters < 1 || o.picard_iters > 100) e = "picard_iters";
  else if (o.jacobian != 0 && o.jacobian != 1) e = "jacobian";
  else if (o.guess != APFC_GUESS_PREV && o.guess != APFC_GUESS_EXTRAP) e = "guess";
  else if (!(o.tol > 0.0) || !(o.tol_inner > 0.0) || !(o.tol_inner < 1.0)) e = "tol";
  else return true;
  e = "invalid option: " + e;
  return false;
}

bool apfc::valid_problem(const apfc_lattice& lat, const apfc_params& p) {
  if (lat.dim != 2 && lat.dim != 3) return false;
  if (lat.J < 1 || lat.J > kMaxJ) return false;
  if (lat.lattice != APFC_LATTICE_CUSTOM && lat.lattice != APFC_LATTICE_HEX2D && lat.lattice != APFC_LATTICE_BCC3D)
    return false;
  for (int j = 0; j < lat.J; ++j)
    for (int d = 0; d < lat.dim; ++d)
      if (!std::isfinite(lat.k[j][d])) return false;
  if (lat.lattice == APFC_LATTICE_HEX2D) {
    if (lat.J != 3 || lat.dim != 2) return false;
    for (int d = 0; d < 2; ++d)
      if (std::fabs(lat.k[0][d] + lat.k[1][d] + lat.k[2][d]) > 1e-12) return false;
  }
  if (lat.lattice == APFC_LATTICE_BCC3D && (lat.J != 6 || lat.dim != 3)) return false;
  if (!std::isfinite(p.dB) || !std::isfinite(p.t) || !std::isfinite(p.v) || !(p.Bx > 0.0)) return false;
  return true;
}

// ===========================================================================
extern "C" {

apfc_status apfc_default_opts(apfc_opts* o) {
  if (!o) return APFC_EINVAL;
  std::memset(o, 0, sizeof(*o));
  o->precision = APFC_FP64;
  o->krylov = APFC_BICGSTAB;
  o->max_iter = 500;
  o->cheb_degree = 1;
  o->tau_mode = APFC_TAU_FOLD;
  o->max_refine = 10;
  o->check_every = 4;
  o->tol = 1e-10;
  o->tol_inner = 1e-4;
  o->fused = 1;
  o->tile = 3;
  o->tile_rows = 0;
  o->picard_iters = 1;
  o->jacobian = 0;
  o->tile_t = 1;
  o->guess = APFC_GUESS_PREV;
  return APFC_OK;
}

apfc_status apfc_uniform_amplitude(const apfc_lattice* lat, const apfc_params* p, double* phi) {
  if (!lat || !p || !phi) return APFC_EINVAL;
  double disc, val;
  if (lat->lattice == APFC_LATTICE_HEX2D) {
    disc = p->t * p->t - 15.0 * p->v * p->dB;
    if (!(disc >= 0.0) || !(p->v > 0.0)) return APFC_EINVAL;
    val = (p->t + std::sqrt(disc)) / (15.0 * p->v);
  } else if (lat->lattice == APFC_LATTICE_BCC3D) {
    disc = 4.0 * p->t * p->t - 45.0 * p->v * p->dB;
    if (!(disc >= 0.0) || !(p->v > 0.0)) return APFC_EINVAL;
    val = (2.0 * p->t + std::sqrt(disc)) / (45.0 * p->v);
  } else {
    return APFC_EINVAL;
  }
  *phi = val;
  return APFC_OK;
}

// Why the last apfc_init of this thread failed (apfc_last_error(NULL)).
static thread_local std::string g_init_err;

static apfc_status init_fail(apfc_status s, const std::string& msg) {
  g_init_err = msg;
  return s;
}

apfc_status apfc_init(apfc_ctx** out, const apfc_lattice* lat, const apfc_params* p, const apfc_grid* g,
                      const apfc_opts* opts, void* stream) {
  g_init_err.clear();
  if (!out || !lat || !p || !g) return init_fail(APFC_EINVAL, "null argument");
  *out = nullptr;
  if (!valid_problem(*lat, *p)) return init_fail(APFC_EINVAL, "invalid lattice or parameters");
  for (int d = 0; d < lat->dim; ++d)
    if (g->n[d] < 3 || !(g->h[d] > 0.0) || !std::isfinite(g->h[d]))
      return init_fail(APFC_EINVAL, "grid sizes must be >= 3 and spacings positive and finite");
  if (lat->dim == 2 && g->n[2] != 1) return init_fail(APFC_EINVAL, "2D grids take n[2] = 1");
  apfc_opts o;
  apfc_default_opts(&o);
  if (opts) o = *opts;
  std::string e;
  if (!valid_opts(o, e)) return init_fail(APFC_EINVAL, "invalid option: " + e);
  {
    int ndev = 0;
    const cudaError_t ce = cudaGetDeviceCount(&ndev);
    if (ce != cudaSuccess || ndev == 0)
      return init_fail(APFC_ECUDA, std::string("no CUDA device: ") +
                                       (ce != cudaSuccess ? cudaGetErrorString(ce) : "device count 0"));
  }

  apfc_ctx* ctx = new (std::nothrow) apfc_ctx();
  if (!ctx) return init_fail(APFC_ENOMEM, "host allocation of the context failed");
  ctx->lat = *lat;
  ctx->par = *p;
  ctx->grid = *g;
  if (lat->dim == 2) ctx->grid.n[2] = 1, ctx->grid.h[2] = 1.0;
  ctx->opts = o;
  ctx->stream = static_cast<cudaStream_t>(stream);
  {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
        sms > 0)
      ctx->sms = sms;
  }
  ctx->J = lat->J;
  ctx->dim = lat->dim;
  ctx->pts = (long long)g->n[0] * g->n[1] * (lat->dim == 3 ? g->n[2] : 1);
  if (!build_tables(*lat, *p, ctx->nt, ctx->et, e)) {
    delete ctx;
    return init_fail(APFC_EINVAL, "nonlinear-term table: " + e);
  }
  // an allocation that fails for lack of memory is ENOMEM, any other CUDA failure ECUDA
  auto check = [&](cudaError_t ce, const char* what) {
    if (ce == cudaSuccess) return APFC_OK;
    g_init_err = std::string(what) + ": " + cudaGetErrorString(ce);
    apfc_destroy(ctx);
    return ce == cudaErrorMemoryAllocation ? APFC_ENOMEM : APFC_ECUDA;
  };
  const size_t blk = sizeof(double2) * 2ull * ctx->J * ctx->pts;
  apfc_status st = APFC_OK;
  if ((st = check(cudaMalloc(&ctx->x64, blk), "cudaMalloc (state)")) != APFC_OK) return st;
  if ((st = check(cudaMalloc(&ctx->b64, blk), "cudaMalloc (right-hand side)")) != APFC_OK) return st;
  if ((st = check(cudaMalloc(&ctx->epart, sizeof(double) * kDotBlocks), "cudaMalloc (energy partials)")) != APFC_OK)
    return st;
  if ((st = check(cudaMalloc(&ctx->eout, sizeof(double)), "cudaMalloc (energy)")) != APFC_OK) return st;
  if ((st = check(cudaMallocHost(&ctx->eout_host, sizeof(double)), "cudaMallocHost (energy)")) != APFC_OK) return st;
  if ((st = check(cudaMalloc(&ctx->ks64, sizeof(KScal) * ctx->J), "cudaMalloc (Krylov scalars)")) != APFC_OK)
    return st;
  if ((st = check(cudaMallocHost(&ctx->ks64_host, sizeof(KScal) * ctx->J), "cudaMallocHost (Krylov scalars)")) !=
      APFC_OK)
    return st;
  if ((st = check(cudaMalloc(&ctx->part64, 16ull * kDotSlots * kDotBlocks * ctx->J), "cudaMalloc (partials)")) !=
      APFC_OK)
    return st;
  if ((st = check(cudaMemsetAsync(ctx->b64, 0, blk, ctx->stream), "cudaMemsetAsync")) != APFC_OK) return st;
  if ((st = check(cudaMemsetAsync(ctx->ks64, 0, sizeof(KScal) * ctx->J, ctx->stream), "cudaMemsetAsync")) != APFC_OK)
    return st;
  if ((st = check(cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize")) != APFC_OK) return st;
  *out = ctx;
  return APFC_OK;
}

apfc_status apfc_set_opts(apfc_ctx* ctx, const apfc_opts* opts) {
  if (!ctx || !opts) return APFC_EINVAL;
  std::string e;
  if (!valid_opts(*opts, e)) return fail(ctx, APFC_EINVAL, e);
  ctx->opts = *opts;
  ctx->coef_dt = -1.0;  // tau_mode may have changed
  ctx->have_prev = false;
  ctx->have_xprev = false;
  return APFC_OK;
}

apfc_status apfc_set_amplitudes(apfc_ctx* ctx, const void* eta, int where, int dtype) {
  if (!ctx || !eta || (where != APFC_HOST && where != APFC_DEVICE)) return APFC_EINVAL;
  if (dtype != APFC_C128 && dtype != APFC_C64) return APFC_EINVAL;
  ctx->failed = false;
  ctx->err.clear();
  ctx->have_prev = false;
  ctx->have_xprev = false;
  apfc_status st = copy_part(ctx, const_cast<void*>(eta), where, 1, true, dtype);
  if (st != APFC_OK) return st;
  std::string e;
  if (ctx->coef_dt < 0 && !build_coef(ctx, 1.0, e)) return fail(ctx, APFC_EINVAL, e);
  launch_zeta(ctx->x64, ctx->coef, ctx->stream);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->has_state = true;
  std::memset(&ctx->stats, 0, sizeof(ctx->stats));
  return APFC_OK;
}

apfc_status apfc_get_amplitudes(apfc_ctx* ctx, void* eta, int where, int dtype) {
  if (!ctx || !eta || (where != APFC_HOST && where != APFC_DEVICE)) return APFC_EINVAL;
  if (dtype != APFC_C128 && dtype != APFC_C64) return APFC_EINVAL;
  if (!ctx->has_state) return fail(ctx, APFC_ESTATE, "no amplitudes set");
  return copy_part(ctx, eta, where, 1, false, dtype);
}

apfc_status apfc_get_zeta(apfc_ctx* ctx, void* zeta, int where) {
  if (!ctx || !zeta || (where != APFC_HOST && where != APFC_DEVICE)) return APFC_EINVAL;
  if (!ctx->has_state) return fail(ctx, APFC_ESTATE, "no amplitudes set");
  return copy_part(ctx, zeta, where, 0, false);
}

apfc_status apfc_step(apfc_ctx* ctx, double dt, int n) {
  if (!ctx || n < 0) return APFC_EINVAL;
  if (ctx->failed) return APFC_ESTATE;
  if (!ctx->has_state) return fail(ctx, APFC_ESTATE, "no amplitudes set");
  std::string e;
  if (!build_coef(ctx, dt, e)) return fail(ctx, APFC_EINVAL, e);
  for (int i = 0; i < n; ++i) {
    apfc_status st = one_step(ctx);
    if (st != APFC_OK) return st;
  }
  return APFC_OK;
}

apfc_status apfc_autotune(apfc_ctx* ctx, double dt, int* tile_rows, int* tile_t, double* ms_per_step) {
  if (!ctx) return APFC_EINVAL;
  if (ctx->failed) return APFC_ESTATE;
  if (!ctx->has_state) return fail(ctx, APFC_ESTATE, "no amplitudes set");
  std::string e;
  if (!build_coef(ctx, dt, e)) return fail(ctx, APFC_EINVAL, e);
  const bool tunable = ctx->dim == 2 && ctx->opts.precision == APFC_FP32_REFINED &&
                       use_fused(ctx, (int)sizeof(float2)) && ctx->opts.picard_iters == 1 && ctx->opts.jacobian == 0;
  if (!tunable) {
    if (tile_rows) *tile_rows = fused_rows(ctx);
    if (tile_t) *tile_t = ctx->opts.tile_t;
    if (ms_per_step) *ms_per_step = 0.0;
    return APFC_OK;
  }
  // candidate heights: the automatic one, 32, 48 and 64 rows (small grids want many blocks),
  // and every ceil(ny / s) from 96 to 256 rows
  const int ny = ctx->grid.n[1];
  const int saved_rows = ctx->opts.tile_rows, saved_tt = ctx->opts.tile_t;
  std::vector<int> cand;
  ctx->opts.tile_rows = 0;
  cand.push_back(fused_rows(ctx));
  for (int rows : {32, 48, 64})
    if (rows < ny && std::find(cand.begin(), cand.end(), rows) == cand.end()) cand.push_back(rows);
  for (int s = std::max(1, (ny + 255) / 256); s <= std::max(1, ny / 96); ++s) {
    const int rows = (ny + s - 1) / s;
    if (rows >= 32 && rows <= ny && std::find(cand.begin(), cand.end(), rows) == cand.end()) cand.push_back(rows);
  }
  const size_t blk = sizeof(double2) * 2 * (size_t)ctx->J * (size_t)ctx->pts;
  double2* saved = nullptr;
  if (cudaMalloc(&saved, blk) != cudaSuccess) {
    cudaGetLastError();
    ctx->opts.tile_rows = saved_rows;
    ctx->opts.tile_t = saved_tt;
    ctx->err = "autotune: no room for a copy of the state";  // the context stays usable
    return APFC_ENOMEM;
  }
  const apfc_stats_t stats = ctx->stats;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  apfc_status st = APFC_OK;
  int best_rows = cand[0], best_tt = saved_tt;
  double best = 1e300;
  auto restore = [&]() -> cudaError_t {
    ctx->have_prev = false;
    ctx->have_xprev = false;
    return cudaMemcpyAsync(ctx->x64, saved, blk, cudaMemcpyDeviceToDevice, ctx->stream);
  };
  if (cudaMemcpyAsync(saved, ctx->x64, blk, cudaMemcpyDeviceToDevice, ctx->stream) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    st = fail(ctx, APFC_ECUDA, "autotune: copy or event creation failed");
  // pass 1: the heights with the t-kernel variant as set; pass 2: every t-kernel variant at
  // the best height
  const int nrows = (int)cand.size(), ntt = fused2d_tiles();
  for (int i = -1; i < nrows + ntt && st == APFC_OK; ++i) {  // i = -1: untimed warm-up
    if (i >= nrows && i - nrows == (saved_tt < 0 ? ctx->opts.tile : saved_tt)) continue;  // timed in pass 1
    ctx->opts.tile_rows = i < nrows ? cand[i < 0 ? 0 : i] : best_rows;
    ctx->opts.tile_t = i < nrows ? saved_tt : i - nrows;
    if (restore() != cudaSuccess || cudaEventRecord(e0, ctx->stream) != cudaSuccess) {
      st = fail(ctx, APFC_ECUDA, "autotune: restore failed");
      break;
    }
    if ((st = one_step(ctx)) != APFC_OK) break;
    float ms = 0.f;
    if (cudaEventRecord(e1, ctx->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      st = fail(ctx, APFC_ECUDA, "autotune: timing failed");
      break;
    }
    if (i >= 0 && ms < best) best = ms, best_rows = ctx->opts.tile_rows, best_tt = ctx->opts.tile_t;
  }
  if (restore() != cudaSuccess && st == APFC_OK) st = fail(ctx, APFC_ECUDA, "autotune: restore failed");
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess && st == APFC_OK)
    st = fail(ctx, APFC_ECUDA, "autotune: synchronisation failed");
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(saved);
  ctx->stats = stats;
  ctx->opts.tile_rows = st == APFC_OK ? best_rows : saved_rows;
  ctx->opts.tile_t = st == APFC_OK ? best_tt : saved_tt;
  if (st != APFC_OK) return st;
  if (tile_rows) *tile_rows = best_rows;
  if (tile_t) *tile_t = best_tt;
  if (ms_per_step) *ms_per_step = best;
  return APFC_OK;
}

apfc_status apfc_energy(apfc_ctx* ctx, double* F) {
  if (!ctx || !F) return APFC_EINVAL;
  if (!ctx->has_state) return fail(ctx, APFC_ESTATE, "no amplitudes set");
  launch_energy(ctx->x64, ctx->epart, ctx->eout, ctx->coef, ctx->et, ctx->par.Bx, ctx->stream);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(ctx->eout_host, ctx->eout, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  double vol = 1.0;
  for (int d = 0; d < ctx->dim; ++d) vol *= ctx->grid.h[d];
  *F = vol * ctx->eout_host[0];
  return APFC_OK;
}

apfc_status apfc_stats(const apfc_ctx* ctx, apfc_stats_t* out) {
  if (!ctx || !out) return APFC_EINVAL;
  *out = ctx->stats;
  return APFC_OK;
}

const char* apfc_last_error(const apfc_ctx* ctx) {
  if (ctx) return ctx->err.c_str();
  return g_init_err.empty() ? "null context" : g_init_err.c_str();
}

void apfc_destroy(apfc_ctx* ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  cudaFree(ctx->x64);
  cudaFree(ctx->b64);
  cudaFree(ctx->b64_prev);
  cudaFree(ctx->r64_prev);
  cudaFree(ctx->x_prev);
  cudaFree(ctx->epart);
  cudaFree(ctx->eout);
  if (ctx->eout_host) cudaFreeHost(ctx->eout_host);
  cudaFree(ctx->ks64);
  if (ctx->ks64_host) cudaFreeHost(ctx->ks64_host);
  cudaFree(ctx->part64);
  free_work(ctx->w64);
  free_work(ctx->w32);
  cudaFree(ctx->xadj);
  cudaFree(ctx->badj);
  cudaFree(ctx->eblk);
  for (auto& f : ctx->afld) cudaFree(f);
  cudaFree(ctx->ckpt);
  cudaFree(ctx->seg);
  cudaFree(ctx->eta_step);
  cudaFree(ctx->jd);
  cudaFree(ctx->jd32);
  cudaFree(ctx->stage);
  delete ctx;
}

static const char* kKernelNames[KID_COUNT] = {
    "apply_A", "residual", "pc_rhs", "cheb_zero", "cheb_first", "cheb_sweep", "pc_final", "p_update", "s_update",
    "r_update", "add_to", "dots", "finalize", "rhs", "zeta", "residual_refine", "energy", "fused_apinv",
    "fused_pinv", "bicg_update", "fused_apinv_t", "adj_nonlin", "energy_grad", "rotation", "extrapolate"};

int apfc_kernel_count(void) { return 2 * KID_COUNT; }

const char* apfc_kernel_name(int id) {
  static std::string names[2 * KID_COUNT];
  if (id < 0 || id >= 2 * KID_COUNT) return "";
  if (names[id].empty()) names[id] = std::string(kKernelNames[id % KID_COUNT]) + (id < KID_COUNT ? "_f64" : "_f32");
  return names[id].c_str();
}

apfc_status apfc_profile_start(apfc_ctx* ctx, int timed_id) {
  if (!ctx) return APFC_EINVAL;
  std::string e;
  if (!profiler_start(ctx->stream, timed_id, &ctx->coef.prof, e)) return fail(ctx, APFC_EINVAL, e);
  return APFC_OK;
}

apfc_status apfc_profile_read(apfc_ctx* ctx, int id, double* ms, long long* launches, double* bytes,
                              long long* all_launches) {
  if (!ctx) return APFC_EINVAL;
  std::string e;
  if (!profiler_read(ctx->stream, id, ms, launches, bytes, all_launches, e)) return fail(ctx, APFC_EINVAL, e);
  return APFC_OK;
}

apfc_status apfc_profile_stop(apfc_ctx* ctx) {
  if (!ctx) return APFC_EINVAL;
  profiler_stop();
  ctx->coef.prof = nullptr;
  return APFC_OK;
}

apfc_status apfc_apply_operator(apfc_ctx* ctx, double dt, const void* x, void* y, int where) {
  if (!ctx || !x || !y || (where != APFC_HOST && where != APFC_DEVICE)) return APFC_EINVAL;
  std::string e;
  if (!build_coef(ctx, dt, e)) return fail(ctx, APFC_EINVAL, e);
  apfc_status st = alloc_work<double>(ctx, ctx->w64);
  if (st != APFC_OK) return st;
  double2* in = ctx->w64.blk[0];
  double2* outb = ctx->w64.blk[1];
  if (where == APFC_DEVICE) {
    in = const_cast<double2*>(static_cast<const double2*>(x));
    outb = static_cast<double2*>(y);
  } else if ((st = copy_in_block(ctx, in, x, where)) != APFC_OK) {
    return st;
  }
  launch_apply_A<double>(in, outb, ctx->coef, nullptr, ctx->stream);
  CK(cudaGetLastError());
  if (where == APFC_HOST) return copy_out_block(ctx, y, outb, where);
  CK(cudaStreamSynchronize(ctx->stream));
  return APFC_OK;
}

apfc_status apfc_apply_preconditioner(apfc_ctx* ctx, double dt, const void* b, void* x, int where) {
  if (!ctx || !b || !x || (where != APFC_HOST && where != APFC_DEVICE)) return APFC_EINVAL;
  std::string e;
  if (!build_coef(ctx, dt, e)) return fail(ctx, APFC_EINVAL, e);
  apfc_status st = alloc_work<double>(ctx, ctx->w64);
  if (st != APFC_OK) return st;
  double2* in = ctx->w64.blk[0];
  double2* outb = ctx->w64.blk[1];
  if (where == APFC_DEVICE) {
    in = const_cast<double2*>(static_cast<const double2*>(b));
    outb = static_cast<double2*>(x);
  } else if ((st = copy_in_block(ctx, in, b, where)) != APFC_OK) {
    return st;
  }
  const auto cw = cheb_weights(ctx);
  if (!use_fused(ctx, (int)sizeof(double2)) ||
      !launch_fused_pinv_store<double>(ctx->opts.cheb_degree, fused_rows(ctx), ctx->opts.tile, ctx->coef, cw.data(), in,
                                       outb,
                                       ctx->stream))
    apply_pinv<double>(ctx, ctx->w64, in, outb, nullptr, cw);
  CK(cudaGetLastError());
  if (where == APFC_HOST) return copy_out_block(ctx, x, outb, where);
  CK(cudaStreamSynchronize(ctx->stream));
  return APFC_OK;
}

apfc_status apfc_nonlinear_rhs(apfc_ctx* ctx, double dt, const void* eta, void* rhs, int where) {
  if (!ctx || !eta || !rhs || (where != APFC_HOST && where != APFC_DEVICE)) return APFC_EINVAL;
  std::string e;
  if (!build_coef(ctx, dt, e)) return fail(ctx, APFC_EINVAL, e);
  apfc_status st = alloc_work<double>(ctx, ctx->w64);
  if (st != APFC_OK) return st;
  // stage eta into the eta-parts of a scratch block, compute, copy the eta-parts out
  double2* in = ctx->w64.blk[0];
  double2* outb = ctx->w64.blk[1];
  const size_t row = sizeof(double2) * (size_t)ctx->pts;
  const cudaMemcpyKind kin = where == APFC_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  const cudaMemcpyKind kout = where == APFC_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  CK(cudaMemcpy2DAsync(in + ctx->pts, 2 * row, eta, row, row, ctx->J, kin, ctx->stream));
  launch_rhs(in, outb, ctx->coef, ctx->nt, ctx->stream);
  CK(cudaGetLastError());
  CK(cudaMemcpy2DAsync(rhs, row, outb + ctx->pts, 2 * row, row, ctx->J, kout, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return APFC_OK;
}


apfc_status apfc_set_params(apfc_ctx* ctx, const apfc_params* p) {
  if (!ctx || !p) return APFC_EINVAL;
  if (!valid_problem(ctx->lat, *p)) return fail(ctx, APFC_EINVAL, "invalid parameters");
  NonlinTable nt;
  EnergyTable et;
  std::string e;
  if (!build_tables(ctx->lat, *p, nt, et, e)) return fail(ctx, APFC_EINVAL, e);
  ctx->par = *p;
  ctx->nt = nt;
  ctx->et = et;
  ctx->coef_dt = -1.0;  // a and the preconditioner's shift depend on dB
  ctx->have_prev = false;
  ctx->have_xprev = false;
  ctx->r_ready = false;
  return APFC_OK;
}

apfc_status apfc_adjoint_step(apfc_ctx* ctx, double dt, const void* eta_n, const void* eta_np1, const void* lam_np1,
                              void* lam_n, double* dB_grad, int where) {
  if (!ctx || !eta_n || !eta_np1 || !lam_np1 || !lam_n || (where != APFC_HOST && where != APFC_DEVICE))
    return APFC_EINVAL;
  if (ctx->failed) return APFC_ESTATE;
  if (!explicit_step(ctx)) return fail(ctx, APFC_EINVAL, "the adjoint is that of the explicit step");
  std::string e;
  if (!build_coef(ctx, dt, e)) return fail(ctx, APFC_EINVAL, e);
  apfc_status st = alloc_adjoint(ctx);
  if (st != APFC_OK) return st;
  const size_t bytes = sizeof(double2) * field_elems(ctx);
  const double2 *en = static_cast<const double2*>(eta_n), *e1 = static_cast<const double2*>(eta_np1),
                *l1 = static_cast<const double2*>(lam_np1);
  double2* l0 = static_cast<double2*>(lam_n);
  if (where == APFC_HOST) {
    CK(cudaMemcpyAsync(ctx->afld[0], eta_n, bytes, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->afld[1], eta_np1, bytes, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->afld[2], lam_np1, bytes, cudaMemcpyHostToDevice, ctx->stream));
    en = ctx->afld[0];
    e1 = ctx->afld[1];
    l1 = ctx->afld[2];
    l0 = ctx->afld[3];
  }
  double dB = 0.0;
  if ((st = adjoint_step_dev(ctx, en, e1, l1, l0, &dB, false)) != APFC_OK) return st;
  if (where == APFC_HOST) CK(cudaMemcpyAsync(lam_n, l0, bytes, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (dB_grad) *dB_grad = dB;
  return APFC_OK;
}

apfc_status apfc_energy_gradient(apfc_ctx* ctx, const void* eta, void* grad, double* dF_ddB, int where) {
  if (!ctx || !eta || !grad || (where != APFC_HOST && where != APFC_DEVICE)) return APFC_EINVAL;
  std::string e;
  if (!build_coef(ctx, ctx->coef_dt > 0 ? ctx->coef_dt : 1.0, e)) return fail(ctx, APFC_EINVAL, e);
  apfc_status st = alloc_adjoint(ctx);
  if (st != APFC_OK) return st;
  const size_t bytes = sizeof(double2) * field_elems(ctx);
  const double2* in = static_cast<const double2*>(eta);
  double2* out = static_cast<double2*>(grad);
  if (where == APFC_HOST) {
    CK(cudaMemcpyAsync(ctx->afld[0], eta, bytes, cudaMemcpyHostToDevice, ctx->stream));
    in = ctx->afld[0];
    out = ctx->afld[3];
  }
  if ((st = energy_grad_dev(ctx, in, out, dF_ddB)) != APFC_OK) return st;
  if (where == APFC_HOST) CK(cudaMemcpyAsync(grad, out, bytes, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return APFC_OK;
}

apfc_status apfc_rollout_forward(apfc_ctx* ctx, double dt, int n, int every) {
  if (!ctx || n < 0 || every < 1) return APFC_EINVAL;
  if (ctx->failed) return APFC_ESTATE;
  if (!ctx->has_state) return fail(ctx, APFC_ESTATE, "no amplitudes set");
  std::string e;
  if (!build_coef(ctx, dt, e)) return fail(ctx, APFC_EINVAL, e);
  ctx->r_ready = false;
  const int nseg = (n + every - 1) / every;
  apfc_status st = ensure_states(ctx, &ctx->ckpt, &ctx->ckpt_cap, (size_t)nseg + 1);
  if (st != APFC_OK) return st;
  const size_t fe = field_elems(ctx);
  for (int i = 0; i < n; ++i) {
    if (i % every == 0) {
      // checkpoint eta^i and restart from (G_h eta^i, eta^i) without the previous
      // residual, exactly as the backward pass will when it recomputes this segment
      double2* ck = ctx->ckpt + (size_t)(i / every) * fe;
      if ((st = block_to_field(ctx, ck, ctx->x64, 1)) != APFC_OK) return st;
      if ((st = load_state(ctx, ck)) != APFC_OK) return st;
    }
    if ((st = one_step(ctx)) != APFC_OK) return st;
  }
  if ((st = block_to_field(ctx, ctx->ckpt + (size_t)nseg * fe, ctx->x64, 1)) != APFC_OK) return st;
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->r_dt = dt;
  ctx->r_n = n;
  ctx->r_every = every;
  ctx->r_ready = true;
  return APFC_OK;
}

apfc_status apfc_rollout_backward(apfc_ctx* ctx, const void* lam_n, void* lam_0, double* dB_grad, int where) {
  if (!ctx || !lam_n || !lam_0 || (where != APFC_HOST && where != APFC_DEVICE)) return APFC_EINVAL;
  if (ctx->failed) return APFC_ESTATE;
  if (!ctx->r_ready) return fail(ctx, APFC_ESTATE, "no rollout to differentiate");
  if (!explicit_step(ctx)) return fail(ctx, APFC_EINVAL, "the adjoint is that of the explicit step");
  std::string e;
  if (!build_coef(ctx, ctx->r_dt, e)) return fail(ctx, APFC_EINVAL, e);
  apfc_status st = alloc_adjoint(ctx);
  if (st != APFC_OK) return st;
  const int n = ctx->r_n, every = ctx->r_every, nseg = (n + every - 1) / every;
  if ((st = ensure_states(ctx, &ctx->seg, &ctx->seg_cap, (size_t)std::min(every, std::max(n, 1)) + 1)) != APFC_OK)
    return st;
  const size_t fe = field_elems(ctx), bytes = sizeof(double2) * fe;
  double2* lam[2] = {ctx->afld[2], ctx->afld[3]};
  CK(cudaMemcpyAsync(lam[0], lam_n, bytes, where == APFC_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                     ctx->stream));
  CK(cudaMemsetAsync(ctx->xadj, 0, 2 * bytes, ctx->stream));
  const apfc_stats_t keep = ctx->stats;  // the recomputation is not user stepping
  double dB = 0.0;
  int cur = 0;
  for (int sg = nseg - 1; sg >= 0; --sg) {
    const int s0 = sg * every, s1 = std::min(s0 + every, n);
    // recompute eta^{s0} .. eta^{s1} from the checkpoint, as the forward pass did
    const double2* ck = ctx->ckpt + (size_t)sg * fe;
    CK(cudaMemcpyAsync(ctx->seg, ck, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
    if ((st = load_state(ctx, ck)) != APFC_OK) return st;
    for (int i = s0; i < s1; ++i) {
      if ((st = one_step(ctx)) != APFC_OK) return st;
      if ((st = block_to_field(ctx, ctx->seg + (size_t)(i - s0 + 1) * fe, ctx->x64, 1)) != APFC_OK) return st;
    }
    for (int i = s1 - 1; i >= s0; --i) {
      const double2* en = ctx->seg + (size_t)(i - s0) * fe;
      const double2* e1 = ctx->seg + (size_t)(i - s0 + 1) * fe;
      if ((st = adjoint_step_dev(ctx, en, e1, lam[cur], lam[1 - cur], &dB, true)) != APFC_OK) return st;
      cur = 1 - cur;
    }
  }
  CK(cudaMemcpyAsync(lam_0, lam[cur], bytes, where == APFC_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                     ctx->stream));
  // leave the state at eta^n, as after the forward pass
  if ((st = load_state(ctx, ctx->ckpt + (size_t)nseg * fe)) != APFC_OK) return st;
  CK(cudaStreamSynchronize(ctx->stream));
  const long long adj_iters = ctx->stats.iters_total - keep.iters_total;
  ctx->stats = keep;
  ctx->stats.iters_total += adj_iters;
  if (dB_grad) *dB_grad = dB;
  return APFC_OK;
}


apfc_status apfc_rotation_field(apfc_ctx* ctx, void* omega, void* amp, void* hmap, const apfc_adapt* adapt,
                                int where) {
  if (!ctx || !omega || (where != APFC_HOST && where != APFC_DEVICE)) return APFC_EINVAL;
  if (hmap && !adapt) return APFC_EINVAL;
  if (adapt && (!(adapt->n > 0.0) || !(adapt->h_int > 0.0) || !(adapt->h_max >= adapt->h_int) ||
                !(adapt->eps >= 0.0) || !std::isfinite(adapt->A_min)))
    return fail(ctx, APFC_EINVAL, "invalid adaptivity parameters");
  if (!ctx->has_state) return fail(ctx, APFC_ESTATE, "no amplitudes set");
  std::string e;
  if (!build_coef(ctx, ctx->coef_dt > 0 ? ctx->coef_dt : 1.0, e)) return fail(ctx, APFC_EINVAL, e);
  const int dim = ctx->dim, J = ctx->J;
  // W_j = M^{-1} k_j with M = sum_j k_j k_j^T (Gauss-Jordan on [M | k_1 .. k_J])
  double Mk[3][3 + kMaxJ] = {};
  for (int a = 0; a < dim; ++a) {
    for (int b = 0; b < dim; ++b)
      for (int j = 0; j < J; ++j) Mk[a][b] += ctx->lat.k[j][a] * ctx->lat.k[j][b];
    for (int j = 0; j < J; ++j) Mk[a][dim + j] = ctx->lat.k[j][a];
  }
  for (int col = 0; col < dim; ++col) {
    int piv = col;
    for (int r = col + 1; r < dim; ++r)
      if (std::fabs(Mk[r][col]) > std::fabs(Mk[piv][col])) piv = r;
    if (std::fabs(Mk[piv][col]) < 1e-12) return fail(ctx, APFC_EINVAL, "lattice vectors do not span the space");
    for (int q = 0; q < dim + J; ++q) std::swap(Mk[col][q], Mk[piv][q]);
    const double inv = 1.0 / Mk[col][col];
    for (int q = 0; q < dim + J; ++q) Mk[col][q] *= inv;
    for (int r = 0; r < dim; ++r) {
      if (r == col) continue;
      const double f = Mk[r][col];
      for (int q = 0; q < dim + J; ++q) Mk[r][q] -= f * Mk[col][q];
    }
  }
  RotParams rp{};
  double kmax = 0.0;
  for (int j = 0; j < J; ++j) {
    double k2 = 0.0;
    for (int a = 0; a < dim; ++a) {
      rp.Wf[j][a] = (float)Mk[a][dim + j];
      k2 += ctx->lat.k[j][a] * ctx->lat.k[j][a];
    }
    kmax = std::max(kmax, std::sqrt(k2));
  }
  for (int a = 0; a < 3; ++a) {
    rp.inv2hd[a] = 1.0 / (2.0 * ctx->grid.h[a]);
    rp.inv2h[a] = (float)rp.inv2hd[a];
  }
  rp.amp_floor = 1e-12;
  if (adapt) {
    rp.pi_over_nk = M_PI / (adapt->n * kmax);
    rp.h_int = adapt->h_int;
    rp.h_max = adapt->h_max;
    rp.eps = adapt->eps;
    rp.A_min = adapt->A_min;
  }
  const int nc = dim == 2 ? 1 : 3;
  const size_t pts = (size_t)ctx->pts;
  double *om = static_cast<double*>(omega), *am = static_cast<double*>(amp), *hm = static_cast<double*>(hmap);
  double* scratch = nullptr;
  if (where == APFC_HOST) {
    CK(cudaMalloc(&scratch, sizeof(double) * pts * (nc + 2)));
    om = scratch;
    am = amp ? scratch + nc * pts : nullptr;
    hm = hmap ? scratch + (nc + 1) * pts : nullptr;
  }
  launch_rotation(ctx->x64, om, am, hm, rp, ctx->coef, ctx->stream);
  cudaError_t err = cudaGetLastError();
  if (err == cudaSuccess && where == APFC_HOST) {
    err = cudaMemcpyAsync(omega, om, sizeof(double) * pts * nc, cudaMemcpyDeviceToHost, ctx->stream);
    if (err == cudaSuccess && amp) err = cudaMemcpyAsync(amp, am, sizeof(double) * pts, cudaMemcpyDeviceToHost, ctx->stream);
    if (err == cudaSuccess && hmap) err = cudaMemcpyAsync(hmap, hm, sizeof(double) * pts, cudaMemcpyDeviceToHost, ctx->stream);
  }
  if (err == cudaSuccess) err = cudaStreamSynchronize(ctx->stream);
  cudaFree(scratch);
  if (err != cudaSuccess) return fail(ctx, APFC_ECUDA, std::string("rotation field: ") + cudaGetErrorString(err));
  return APFC_OK;
}

}  // extern "C"
