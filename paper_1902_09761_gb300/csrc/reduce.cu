// Complex inner products (u, v) = sum conj(u) v per amplitude (Sec. II.A's L2
// product, conjugate-linear in the first argument) and the per-amplitude
// BiCGStab scalar updates that consume them.
//
// FP64 fields accumulate in FP64.  FP32 fields accumulate in FP32 with
// Neumaier-compensated summation (each partial is a (sum, compensation) pair)
// through the thread, block and final stages; the fixed reduction tree makes
// every result deterministic.
#include "apfc_internal.cuh"

namespace apfc {

namespace {

// ---- compensated FP32 pair arithmetic ------------------------------------
struct CF {
  float s, c;
};
__device__ __forceinline__ void cf_add(CF& a, float x) {
  const float t = a.s + x;
  if (fabsf(a.s) >= fabsf(x))
    a.c += (a.s - t) + x;
  else
    a.c += (x - t) + a.s;
  a.s = t;
}
__device__ __forceinline__ void cf_merge(CF& a, const CF& b) {
  cf_add(a, b.s);
  a.c += b.c;
}

template <typename T>
struct Acc;

template <>
struct Acc<double> {
  double re, im;
  __device__ __forceinline__ void zero() { re = im = 0.0; }
  __device__ __forceinline__ void add(double2 u, double2 v) {
    re += u.x * v.x + u.y * v.y;
    im += u.x * v.y - u.y * v.x;
  }
  __device__ __forceinline__ void shfl_merge(int o) {
    re += __shfl_xor_sync(0xffffffffu, re, o);
    im += __shfl_xor_sync(0xffffffffu, im, o);
  }
  __device__ __forceinline__ void merge(const Acc& b) {
    re += b.re;
    im += b.im;
  }
  __device__ __forceinline__ void store(void* part, long long idx) const {
    reinterpret_cast<double2*>(part)[idx] = make_double2(re, im);
  }
  __device__ __forceinline__ void load(const void* part, long long idx) {
    const double2 v = reinterpret_cast<const double2*>(part)[idx];
    re = v.x;
    im = v.y;
  }
  __device__ __forceinline__ double2 value() const { return make_double2(re, im); }
};

template <>
struct Acc<float> {
  CF re, im;
  __device__ __forceinline__ void zero() { re = CF{0.f, 0.f}; im = CF{0.f, 0.f}; }
  __device__ __forceinline__ void add(float2 u, float2 v) {
    cf_add(re, u.x * v.x + u.y * v.y);
    cf_add(im, u.x * v.y - u.y * v.x);
  }
  __device__ __forceinline__ void shfl_merge(int o) {
    CF r{__shfl_xor_sync(0xffffffffu, re.s, o), __shfl_xor_sync(0xffffffffu, re.c, o)};
    CF i{__shfl_xor_sync(0xffffffffu, im.s, o), __shfl_xor_sync(0xffffffffu, im.c, o)};
    cf_merge(re, r);
    cf_merge(im, i);
  }
  __device__ __forceinline__ void merge(const Acc& b) {
    cf_merge(re, b.re);
    cf_merge(im, b.im);
  }
  __device__ __forceinline__ void store(void* part, long long idx) const {
    reinterpret_cast<float4*>(part)[idx] = make_float4(re.s, re.c, im.s, im.c);
  }
  __device__ __forceinline__ void load(const void* part, long long idx) {
    const float4 v = reinterpret_cast<const float4*>(part)[idx];
    re = CF{v.x, v.y};
    im = CF{v.z, v.w};
  }
  __device__ __forceinline__ double2 value() const {
    return make_double2((double)re.s + (double)re.c, (double)im.s + (double)im.c);
  }
};

// Reduce an accumulator over the block; thread 0 ends with the total.
template <typename T>
__device__ __forceinline__ void block_reduce(Acc<T>& a) {
  __shared__ Acc<T> sh[kThreads / 32];
  for (int o = 16; o > 0; o >>= 1) a.shfl_merge(o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = a;
  __syncthreads();
  if (w == 0) {
    if (l < kThreads / 32)
      a = sh[l];
    else
      a.zero();
    for (int o = 16; o > 0; o >>= 1) a.shfl_merge(o);
  }
  __syncthreads();
}

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
    case OP_NORMS: {  // d0 = (r, r), d1 = (b, b): record only
      k.rnorm2 = d[0].x;
      k.bnorm2 = d[1].x;
      break;
    }
  }
}

template <typename T, int NP>
__global__ void k_finalize(const void* partials, KScal* ks, int op) {
  const int j = blockIdx.x;
  KScal& k = ks[j];
  if (op != OP_INIT && op != OP_NORMS && k.active == 0) return;
  __shared__ double2 res[3];
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    Acc<T> a;
    a.zero();
    for (int b = threadIdx.x; b < kDotBlocks; b += blockDim.x) {
      Acc<T> t;
      t.load(partials, (long long)(j * 3 + q) * kDotBlocks + b);
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
void launch_finalize(int npair, const void* partials, KScal* k, int op, int J, cudaStream_t s) {
  ProfScope ps_(kid_of<T>(KID_FINALIZE), s);
  if (npair == 1)
    k_finalize<T, 1><<<J, kThreads, 0, s>>>(partials, k, op);
  else if (npair == 2)
    k_finalize<T, 2><<<J, kThreads, 0, s>>>(partials, k, op);
  else
    k_finalize<T, 3><<<J, kThreads, 0, s>>>(partials, k, op);
}

void launch_finalize64(int npair, const void* partials, KScal* k, int op, int J, cudaStream_t s) {
  launch_finalize<double>(npair, partials, k, op, J, s);
}

template void launch_dots<double>(int, const DotPairs<double>&, void*, const OpCoef&, const KScal*, cudaStream_t);
template void launch_dots<float>(int, const DotPairs<float>&, void*, const OpCoef&, const KScal*, cudaStream_t);
template void launch_finalize<double>(int, const void*, KScal*, int, int, cudaStream_t);
template void launch_finalize<float>(int, const void*, KScal*, int, int, cudaStream_t);

}  // namespace apfc
