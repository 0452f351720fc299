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
    if (threadIdx.x == 0) acc[q].store(partials, (long long)(j * 3 + q) * kDotBlocks + blockIdx.x);
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
      k.alpha = make_double2(1.0, 0.0);
      k.omega = make_double2(1.0, 0.0);
      k.beta = make_double2(0.0, 0.0);
      k.iters = 0;
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
  if (op != OP_INIT && op != OP_NORMS && k.active == 0) return;
  __shared__ double2 res[3];
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    Acc<T> a;
    a.zero();
    for (int b = threadIdx.x; b < npart; b += blockDim.x) {
      Acc<T> t;
      t.load(partials, (long long)(j * 3 + q) * npart + b);
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
  else
    k_finalize<T, 3><<<J, kThreads, 0, s>>>(partials, npart, k, op);
}

void launch_finalize64(int npair, const void* partials, KScal* k, int op, int J, cudaStream_t s) {
  launch_finalize<double>(npair, partials, k, op, J, s);
}

template void launch_dots<double>(int, const DotPairs<double>&, void*, const OpCoef&, const KScal*, cudaStream_t);
template void launch_dots<float>(int, const DotPairs<float>&, void*, const OpCoef&, const KScal*, cudaStream_t);
template void launch_finalize<double>(int, const void*, KScal*, int, int, cudaStream_t, int);
template void launch_finalize<float>(int, const void*, KScal*, int, int, cudaStream_t, int);

}  // namespace apfc
