// Accumulators for complex inner products (u, v) = sum conj(u) v.
//
// FP64 fields accumulate in FP64.  FP32 fields accumulate in FP32 with
// Neumaier-compensated summation: each partial is a (sum, compensation) pair
// through the thread, block and final stages, and the fixed reduction tree
// keeps every result deterministic.
#pragma once

#include "apfc_internal.cuh"

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
  float run_re, run_im;  // short plain FP32 runs, folded into (re, im) by flush()
  __device__ __forceinline__ void zero() {
    re = CF{0.f, 0.f};
    im = CF{0.f, 0.f};
    run_re = run_im = 0.f;
  }
  __device__ __forceinline__ void add(float2 u, float2 v) {
    cf_add(re, u.x * v.x + u.y * v.y);
    cf_add(im, u.x * v.y - u.y * v.x);
  }
  // Blocked compensated summation: a run of a few products is summed in plain
  // FP32 and each run total enters the compensated sum (callers flush every
  // few products and before reducing).
  __device__ __forceinline__ void add_run(float2 u, float2 v) {
    run_re = fmaf(u.x, v.x, fmaf(u.y, v.y, run_re));
    run_im = fmaf(u.x, v.y, fmaf(-u.y, v.x, run_im));
  }
  __device__ __forceinline__ void flush() {
    cf_add(re, run_re);
    cf_add(im, run_im);
    run_re = run_im = 0.f;
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

}  // namespace apfc
