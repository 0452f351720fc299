// Preconditioner apply that allocates nothing.
//
// apfc_apply_preconditioner() keeps its intermediate fields in workspace that
// the context allocates with cudaMalloc.  Some callers cannot allocate device
// memory at the point where they want to apply the preconditioner: code that
// runs under an allocator owned by someone else (a framework memory pool that
// forbids raw cudaMalloc), code on a latency-critical path where an allocation
// would synchronise the device, or plugins that are handed device buffers and
// a stream but no right to grow the process's footprint.  For them this file
// provides apfc_apply_preconditioner_static(): the caller passes the input and
// output buffers and a stream, and the five intermediate fields live in one
// fixed, file-scope device array that every GPU holds from module load until
// process exit.
#include <cmath>
#include <cstring>
#include <mutex>

#include "apfc_internal.cuh"

using namespace apfc;

namespace {

// Intermediate fields f, beta2', R, D_a, D_b of P^{-1}, each [J][pts] complex128.
constexpr long long kStaticFields = 5;
constexpr long long kStaticMaxDof = APFC_STATIC_MAX_DOF;  // J * nx * ny * nz
static __device__ __align__(256) double2 g_pc_scratch[kStaticFields * kStaticMaxDof];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
double2* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_pc_scratch on the current device, resolved once per device.
// In host code the symbol is only a host-side stand-in, so the address must come
// from cudaGetSymbolAddress with the device current.
apfc_status scratch_on_current_device(double2** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return APFC_ECUDA;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (g_scratch_ptr[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_pc_scratch) != cudaSuccess || p == nullptr) return APFC_ECUDA;
    g_scratch_ptr[dev] = static_cast<double2*>(p);
  }
  *out = g_scratch_ptr[dev];
  return APFC_OK;
}

}  // namespace

extern "C" apfc_status apfc_apply_preconditioner_static(const apfc_lattice* lat, const apfc_params* prm,
                                                        const apfc_grid* g, int cheb_degree, int tau_mode, double dt,
                                                        const void* b, void* x, void* stream) {
  if (!lat || !prm || !g || !b || !x) return APFC_EINVAL;
  if ((lat->dim != 2 && lat->dim != 3) || lat->J < 1 || lat->J > kMaxJ) return APFC_EINVAL;
  if (cheb_degree < 0 || cheb_degree > kMaxCheb) return APFC_EINVAL;
  if (tau_mode != APFC_TAU_FOLD && tau_mode != APFC_TAU_PLAIN) return APFC_EINVAL;
  if (!(dt > 0.0) || !std::isfinite(dt) || !(prm->Bx > 0.0) || !std::isfinite(prm->dB)) return APFC_EINVAL;
  for (int d = 0; d < lat->dim; ++d)
    if (g->n[d] < 3 || !(g->h[d] > 0.0) || !std::isfinite(g->h[d])) return APFC_EINVAL;
  if (lat->dim == 2 && g->n[2] != 1) return APFC_EINVAL;
  const long long pts = (long long)g->n[0] * g->n[1] * (lat->dim == 3 ? g->n[2] : 1);
  if (pts * lat->J > kStaticMaxDof) return APFC_ETOOBIG;

  // Operator coefficients (same definitions as the context path).
  OpCoef c;
  std::memset(&c, 0, sizeof(c));
  c.J = lat->J;
  c.dim = lat->dim;
  c.nx = g->n[0];
  c.ny = g->n[1];
  c.nz = lat->dim == 3 ? g->n[2] : 1;
  c.pts = pts;
  double lapmax = 0.0;
  for (int d = 0; d < lat->dim; ++d) {
    c.ih2[d] = 1.0 / (g->h[d] * g->h[d]);
    c.c0 -= 2.0 / (g->h[d] * g->h[d]);
    lapmax += 4.0 / (g->h[d] * g->h[d]);
  }
  c.inv_dt = 1.0 / dt;
  ChebStep w[kMaxCheb > 0 ? kMaxCheb : 1];
  std::memset(w, 0, sizeof(w));
  for (int j = 0; j < lat->J; ++j) {
    double kap = 0.0;
    for (int d = 0; d < lat->dim; ++d) {
      c.kh[j][d] = lat->k[j][d] / g->h[d];
      kap += lat->k[j][d] * lat->k[j][d];
    }
    c.kap[j] = kap;
    c.kt[j] = kap * prm->Bx;
    c.a[j] = 1.0 / dt + kap * prm->dB;
    const double inv_tau = 1.0 / dt + (tau_mode == APFC_TAU_FOLD ? kap * prm->dB : 0.0);
    if (!(inv_tau > 0.0) || !(c.kt[j] > 0.0)) return APFC_EINVAL;
    c.sD[j] = std::sqrt(inv_tau);
    c.mu[j] = std::sqrt(c.kt[j]);
    c.inv_mu[j] = 1.0 / c.mu[j];
    const double lmin = c.sD[j], lmax = c.sD[j] + c.mu[j] * lapmax;
    const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin), sigma = theta / delta;
    c.inv_theta[j] = 1.0 / theta;
    double rho = 1.0 / sigma;
    for (int k = 0; k < cheb_degree; ++k) {
      const double rn = 1.0 / (2.0 * sigma - rho);
      w[k].c1[j] = rn * rho;
      w[k].c2[j] = 2.0 * rn / delta;
      rho = rn;
    }
  }

  double2* scratch = nullptr;
  apfc_status st = scratch_on_current_device(&scratch);
  if (st != APFC_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const long long F = (long long)lat->J * pts;  // one field
  FieldRef<double> f{scratch + 0 * F, pts}, b2p{scratch + 1 * F, pts}, R{scratch + 2 * F, pts};
  FieldRef<double> D[2] = {{scratch + 3 * F, pts}, {scratch + 4 * F, pts}};
  const double2* beta = static_cast<const double2*>(b);
  double2* chi = static_cast<double2*>(x);
  FieldRef<double> chi2{chi + pts, 2 * pts};
  auto cheb = [&](CFieldRef<double> src, FieldRef<double> X) {
    if (cheb_degree == 0) {
      launch_cheb_zero<double>(src, X, c, nullptr, s);
      return;
    }
    launch_cheb_first<double>(src, X, R, D[0], w[0], cheb_degree == 1, c, nullptr, s);
    int cur = 0;
    for (int k = 1; k < cheb_degree; ++k) {
      launch_cheb_sweep<double>(CFieldRef<double>{D[cur].p, pts}, X, R, D[1 - cur], w[k], k == cheb_degree - 1, c,
                                nullptr, s);
      cur = 1 - cur;
    }
  };
  launch_pc_rhs<double>(beta, f, c, nullptr, s);
  cheb(CFieldRef<double>{f.p, pts}, b2p);
  cheb(CFieldRef<double>{b2p.p, pts}, chi2);
  launch_pc_final<double>(beta, CFieldRef<double>{b2p.p, pts}, chi, c, nullptr, s);
  return cudaGetLastError() == cudaSuccess ? APFC_OK : APFC_ECUDA;
}
