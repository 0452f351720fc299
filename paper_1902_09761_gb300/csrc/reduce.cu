// Complex inner products (u, v) = sum conj(u) v per amplitude (Sec. II.A's L2
// product, conjugate-linear in the first argument) and the per-amplitude
// BiCGStab scalar updates that consume them.
//
// FP64 fields accumulate in FP64.  FP32 fields accumulate in FP32 with
// Neumaier-compensated summation (each partial is a (sum, compensation) pair)
// through the thread, block and final stages; the fixed reduction tree makes
// every result deterministic.
#include "acc.cuh"
#include "apfc_internal.cuh"

namespace apfc {

namespace {

template <typename T, int NP>
__global__ void k_dots(DotPairs<T> pr, void* partials, OpCoef c, const KScal* act) {
  const int j = blockIdx.y;
  if (act != nullptr && act[j].active == 0) return;
  const long long n = 2LL * c.pts, o = 2LL * j * c.pts;
  if (c.prof != nullptr && blockIdx.x == 0 && threadIdx.x == 0) {
    // count each distinct array once
    const void* seen[2 * NP];
    int ns = 0;
    for (int q = 0; q < 2 * NP; ++q) {
      const void* ptr = q < NP ? (const void*)pr.u[q] : (const void*)pr.v[q - NP];
      bool dup = false;
      for (int r = 0; r < ns; ++r) dup = dup || seen[r] == ptr;
      if (!dup) seen[ns++] = ptr;
    }
    atomicAdd(c.prof + kid_of<T>(KID_DOTS), (unsigned long long)ns * n * sizeof(cplx<T>));
  }
  Acc<T> acc[NP];
#pragma unroll
  for (int q = 0; q < NP; ++q) acc[q].zero();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
#pragma unroll
    for (int q = 0; q < NP; ++q) acc[q].add(pr.u[q][o + i], pr.v[q][o + i]);
  }
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    block_reduce<T>(acc[q]);
    if (threadIdx.x == 0) acc[q].store(partials, (long long)(j * kDotSlots + q) * kDotBlocks + blockIdx.x);
  }
}

__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  const double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
__device__ __forceinline__ double2 cmul2(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ bool finite2(double2 a) { return isfinite(a.x) && isfinite(a.y); }

// Right-preconditioned BiCGStab scalar recurrences (van der Vorst 1992), one
// amplitude per block.  d[q] are the finished inner products of this op.
__device__ void scalar_update(KScal& k, int op, const double2* d) {
  switch (op) {
    case OP_INIT: {  // d0 = (r, r), d1 = (b, b); rhat = r
      k.rnorm2 = d[0].x;
      k.bnorm2 = d[1].x;
      k.tol2 = k.tolrel2 * (k.bnorm2 > 0.0 ? k.bnorm2 : k.rnorm2);
      k.rho = d[0];
      k.alpha = make_double2(0.0, 0.0);
      k.omega = make_double2(0.0, 0.0);
      k.beta = make_double2(0.0, 0.0);
      k.iters = 0;
      k.just_done = 0;
      if (!isfinite(k.rnorm2) || !isfinite(k.bnorm2)) {
        k.status = KS_NAN;
        k.active = 0;
      } else if (k.rnorm2 <= k.tol2) {
        k.status = KS_CONVERGED;
        k.active = 0;
      } else {
        k.status = KS_RUNNING;
        k.active = 1;
      }
      break;
    }
    case OP_ALPHA: {  // d0 = (rhat, v)
      if (!finite2(d[0]) || cabs2(d[0]) == 0.0) {
        k.status = finite2(d[0]) ? KS_BREAKDOWN : KS_NAN;
        k.active = 0;
      } else {
        k.alpha = cdiv(k.rho, d[0]);
      }
      break;
    }
    case OP_SNORM: {  // d0 = (s, s)
      if (!isfinite(d[0].x)) {
        k.status = KS_NAN;
        k.active = 0;
      } else if (d[0].x <= k.tol2) {
        k.rnorm2 = d[0].x;
        k.iters += 1;
        k.status = KS_CONVERGED;
        k.active = 0;
      }
      break;
    }
    case OP_OMEGA: {  // d0 = (t, s), d1 = (t, t)
      if (!finite2(d[0]) || !isfinite(d[1].x)) {
        k.status = KS_NAN;
        k.active = 0;
      } else if (d[1].x == 0.0 || cabs2(d[0]) == 0.0) {
        k.status = KS_BREAKDOWN;
        k.active = 0;
      } else {
        k.omega = make_double2(d[0].x / d[1].x, d[0].y / d[1].x);
      }
      break;
    }
    case OP_RHO: {  // d0 = (rhat, r), d1 = (r, r)
      k.iters += 1;
      k.rnorm2 = d[1].x;
      if (!isfinite(k.rnorm2) || !finite2(d[0])) {
        k.status = KS_NAN;
        k.active = 0;
      } else if (k.rnorm2 <= k.tol2) {
        k.status = KS_CONVERGED;
        k.active = 0;
      } else if (k.iters >= k.max_iter) {
        k.status = KS_NOCONV;
        k.active = 0;
      } else if (cabs2(d[0]) == 0.0) {
        k.status = KS_BREAKDOWN;
        k.active = 0;
      } else {
        k.beta = cmul2(cdiv(d[0], k.rho), cdiv(k.alpha, k.omega));
        k.rho = d[0];
      }
      break;
    }
    case OP_OMEGA3: {  // d0 = (t, s), d1 = (t, t), d2 = (s, s)
      if (!finite2(d[0]) || !isfinite(d[1].x) || !isfinite(d[2].x)) {
        k.status = KS_NAN;
        k.active = 0;
      } else if (d[2].x <= k.tol2) {
        k.omega = make_double2(0.0, 0.0);  // s already meets tol: the update sets r = s
      } else if (d[1].x == 0.0 || cabs2(d[0]) == 0.0) {
        k.status = KS_BREAKDOWN;
        k.active = 0;
      } else {
        k.omega = make_double2(d[0].x / d[1].x, d[0].y / d[1].x);
      }
      break;
    }
    case OP_BNORM: {  // d0 = (b, b)
      k.bnorm2 = d[0].x;
      break;
    }
    case OP_RNORM: {  // d0 = (r, r); ||b||^2 from an earlier OP_NORMS / OP_BNORM
      k.rnorm2 = d[0].x;
      break;
    }
    case OP_OMEGA5: {
      // merged iteration: d0 = (t, s), d1 = (t, t), d2 = (s, s), d3 = (rhat, s), d4 = (rhat, t).
      // omega = (t, s)/(t, t); by linearity r' = s - omega t has
      // (rhat, r') = (rhat, s) - omega (rhat, t) and
      // ||r'||^2 = (s, s) - 2 Re(omega conj(t, s)) + |omega|^2 (t, t).
      k.just_done = 0;
      bool fin = true;
      for (int q = 0; q < 5; ++q) fin = fin && finite2(d[q]);
      if (!fin) {
        k.status = KS_NAN;
        k.active = 0;
        break;
      }
      k.iters += 1;
      if (d[2].x <= k.tol2) {
        k.omega = make_double2(0.0, 0.0);  // s already meets tol: r' = s
        k.rnorm2 = d[2].x;
        k.status = KS_CONVERGED;
        k.active = 0;
        k.just_done = 1;
        break;
      }
      if (d[1].x == 0.0 || cabs2(d[0]) == 0.0) {
        k.status = KS_BREAKDOWN;
        k.active = 0;
        k.just_done = 1;
        break;
      }
      k.omega = make_double2(d[0].x / d[1].x, d[0].y / d[1].x);
      const double2 oc = cmul2(k.omega, make_double2(d[0].x, -d[0].y));
      double rn2 = d[2].x - 2.0 * oc.x + cabs2(k.omega) * d[1].x;
      k.rnorm2 = rn2 > 0.0 ? rn2 : 0.0;
      const double2 rho_new = make_double2(d[3].x - (k.omega.x * d[4].x - k.omega.y * d[4].y),
                                           d[3].y - (k.omega.x * d[4].y + k.omega.y * d[4].x));
      if (k.rnorm2 <= k.tol2) {
        k.status = KS_CONVERGED;
        k.active = 0;
        k.just_done = 1;
      } else if (k.iters >= k.max_iter) {
        k.status = KS_NOCONV;
        k.active = 0;
        k.just_done = 1;
      } else if (cabs2(rho_new) == 0.0) {
        k.status = KS_BREAKDOWN;
        k.active = 0;
        k.just_done = 1;
      } else {
        k.beta = cmul2(cdiv(rho_new, k.rho), cdiv(k.alpha, k.omega));
        k.rho = rho_new;
      }
      break;
    }
    case OP_NORMS: {  // d0 = (r, r), d1 = (b, b): record only
      k.rnorm2 = d[0].x;
      k.bnorm2 = d[1].x;
      break;
    }
  }
}

template <typename T, int NP>
__global__ void k_finalize(const void* partials, int npart, KScal* ks, int op) {
  const int j = blockIdx.x;
  KScal& k = ks[j];
  // a pending final update was applied after the previous OP_OMEGA5: clear the flag
  if (op == OP_ALPHA && threadIdx.x == 0) k.just_done = 0;
  if (op != OP_INIT && op != OP_NORMS && op != OP_RNORM && op != OP_BNORM && k.active == 0) return;
  __shared__ double2 res[kDotSlots];
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    Acc<T> a;
    a.zero();
    for (int b = threadIdx.x; b < npart; b += blockDim.x) {
      Acc<T> t;
      t.load(partials, (long long)(j * kDotSlots + q) * npart + b);
      a.merge(t);
    }
    block_reduce<T>(a);
    if (threadIdx.x == 0) res[q] = a.value();
  }
  if (threadIdx.x == 0) scalar_update(k, op, res);
}

}  // namespace

template <typename T>
void launch_dots(int npair, const DotPairs<T>& pr, void* partials, const OpCoef& c, const KScal* act, cudaStream_t s) {
  const dim3 g(kDotBlocks, c.J);
  ProfScope ps_(kid_of<T>(KID_DOTS), s);
  if (npair == 1)
    k_dots<T, 1><<<g, kThreads, 0, s>>>(pr, partials, c, act);
  else if (npair == 2)
    k_dots<T, 2><<<g, kThreads, 0, s>>>(pr, partials, c, act);
  else
    k_dots<T, 3><<<g, kThreads, 0, s>>>(pr, partials, c, act);
}

template <typename T>
void launch_finalize(int npair, const void* partials, KScal* k, int op, int J, cudaStream_t s, int npart) {
  ProfScope ps_(kid_of<T>(KID_FINALIZE), s);
  if (npair == 1)
    k_finalize<T, 1><<<J, kThreads, 0, s>>>(partials, npart, k, op);
  else if (npair == 2)
    k_finalize<T, 2><<<J, kThreads, 0, s>>>(partials, npart, k, op);
  else if (npair == 3)
    k_finalize<T, 3><<<J, kThreads, 0, s>>>(partials, npart, k, op);
  else
    k_finalize<T, 5><<<J, kThreads, 0, s>>>(partials, npart, k, op);
}

void launch_finalize64(int npair, const void* partials, KScal* k, int op, int J, cudaStream_t s) {
  launch_finalize<double>(npair, partials, k, op, J, s);
}

template void launch_dots<double>(int, const DotPairs<double>&, void*, const OpCoef&, const KScal*, cudaStream_t);
template void launch_dots<float>(int, const DotPairs<float>&, void*, const OpCoef&, const KScal*, cudaStream_t);
template void launch_finalize<double>(int, const void*, KScal*, int, int, cudaStream_t, int);
template void launch_finalize<float>(int, const void*, KScal*, int, int, cudaStream_t, int);

}  // namespace apfc
