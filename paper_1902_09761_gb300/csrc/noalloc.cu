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
#include "host_common.h"

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
  if (!valid_problem(*lat, *prm)) return APFC_EINVAL;
  if (cheb_degree < 0 || cheb_degree > kMaxCheb) return APFC_EINVAL;
  if (tau_mode != APFC_TAU_FOLD && tau_mode != APFC_TAU_PLAIN) return APFC_EINVAL;
  for (int d = 0; d < lat->dim; ++d)
    if (g->n[d] < 3 || !(g->h[d] > 0.0) || !std::isfinite(g->h[d])) return APFC_EINVAL;
  if (lat->dim == 2 && g->n[2] != 1) return APFC_EINVAL;
  const long long pts = (long long)g->n[0] * g->n[1] * (lat->dim == 3 ? g->n[2] : 1);
  if (pts * lat->J > kStaticMaxDof) return APFC_ETOOBIG;
  // b and x must not overlap: the last pass reads beta while it writes chi.
  const unsigned long long bytes = (unsigned long long)lat->J * 2 * pts * sizeof(double2);
  const unsigned long long pb = reinterpret_cast<unsigned long long>(b), px = reinterpret_cast<unsigned long long>(x);
  if (pb < px + bytes && px < pb + bytes) return APFC_EINVAL;

  // Operator coefficients and Chebyshev weights: the builders the context uses
  // (they write into the caller's stack and allocate nothing).
  OpCoef c;
  std::memset(&c, 0, sizeof(c));
  if (make_coef_into(*lat, *prm, *g, tau_mode, dt, c) != nullptr) return APFC_EINVAL;
  ChebStep w[kMaxCheb > 0 ? kMaxCheb : 1];
  cheb_weights_into(c, *g, cheb_degree, w);

  // A CUDA error that the caller's own work left pending is not ours to report
  // or to clear: refuse to launch rather than consume it below.
  if (cudaPeekAtLastError() != cudaSuccess) return APFC_ECUDA;
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
  // No error was pending before the launches, so whatever is pending now came
  // from them.
  return cudaGetLastError() == cudaSuccess ? APFC_OK : APFC_ECUDA;
}
