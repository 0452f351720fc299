// Accumulators for complex inner products (u, v) = sum conj(u) v.
//
// FP64 fields accumulate in FP64.  FP32 fields accumulate in FP32 with
// Neumaier-compensated summation: each partial is a (sum, compensation) pair
// through the thread, block and final stages, and the fixed reduction tree
// keeps every result deterministic.
#pragma once

#include "apfc_internal.cuh"
#include "dfloat.cuh"

namespace apfc {

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
  __device__ __forceinline__ void add_run(double2 u, double2 v) { add(u, v); }
  __device__ __forceinline__ void add_run_self(double2 u) { re += u.x * u.x + u.y * u.y; }  // (u, u) is real
  __device__ __forceinline__ void flush() {}
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
  // short plain FP32 runs, folded into (re, im) by flush(): packed lanes
  // rr = sum (u.x v.x, u.y v.y) and ri = sum (u.x v.y, u.y v.x), so that one product
  // term costs two packed FMAs (re = rr.x + rr.y, im = ri.x - ri.y)
  float2 rr, ri;
  __device__ __forceinline__ void zero() {
    re = CF{0.f, 0.f};
    im = CF{0.f, 0.f};
    rr = ri = make_float2(0.f, 0.f);
  }
  __device__ __forceinline__ void add(float2 u, float2 v) {
    cf_add(re, u.x * v.x + u.y * v.y);
    cf_add(im, u.x * v.y - u.y * v.x);
  }
  // Blocked compensated summation: a run of a few products is summed in plain
  // FP32 and each run total enters the compensated sum (callers flush every
  // few products and before reducing).
  __device__ __forceinline__ void add_run(float2 u, float2 v) {
    rr = p_fma(u, v, rr);
    ri = p_fma(u, make_float2(v.y, v.x), ri);
  }
  // (u, u): real, the imaginary run stays zero
  __device__ __forceinline__ void add_run_self(float2 u) { rr = p_fma(u, u, rr); }
  __device__ __forceinline__ void flush() {
    cf_add(re, rr.x + rr.y);
    cf_add(im, ri.x - ri.y);
    rr = ri = make_float2(0.f, 0.f);
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
template <typename T, int NT = kThreads>
__device__ __forceinline__ void block_reduce(Acc<T>& a) {
  __shared__ Acc<T> sh[NT / 32];
  for (int o = 16; o > 0; o >>= 1) a.shfl_merge(o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = a;
  __syncthreads();
  if (w == 0) {
    if (l < NT / 32)
      a = sh[l];
    else
      a.zero();
    for (int o = 16; o > 0; o >>= 1) a.shfl_merge(o);
  }
  __syncthreads();
}

// ---- per-amplitude BiCGStab scalar recurrences -------------------------------
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
__device__ __forceinline__ void scalar_update(KScal& k, int op, const double2* d) {
  switch (op) {
    case OP_INIT:     // d0 = (r, r), d1 = (b, b); rhat = r
    case OP_INIT3: {  // the same and d2 = (rhat, r) for a shadow residual rhat != r
      k.rnorm2 = d[0].x;
      k.bnorm2 = d[1].x;
      k.tol2 = k.tolrel2 * (k.bnorm2 > 0.0 ? k.bnorm2 : k.rnorm2);
      k.rho = op == OP_INIT3 ? d[2] : d[0];
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
    // unfused iteration: u += alpha p + omega s is one pass after OP_OMEGA, so an
    // amplitude that stops at OP_SNORM or OP_OMEGA still owes u += alpha p (just_done)
    case OP_SNORM: {  // d0 = (s, s)
      if (!isfinite(d[0].x)) {
        k.status = KS_NAN;
        k.active = 0;
        k.just_done = 1;
      } else if (d[0].x <= k.tol2) {
        k.rnorm2 = d[0].x;
        k.iters += 1;
        k.status = KS_CONVERGED;
        k.active = 0;
        k.just_done = 1;
      }
      break;
    }
    case OP_OMEGA: {  // d0 = (t, s), d1 = (t, t)
      if (!finite2(d[0]) || !isfinite(d[1].x)) {
        k.status = KS_NAN;
        k.active = 0;
        k.just_done = 1;
      } else if (d[1].x == 0.0 || cabs2(d[0]) == 0.0) {
        k.status = KS_BREAKDOWN;
        k.active = 0;
        k.just_done = 1;
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

}  // namespace apfc
