// Arithmetic-rate probe: the FMA throughput of this GPU in FP64 and FP32.
//
// The FP64 kernels of the step (outer residual, nonlinear right-hand side) are
// bound by the FP64 pipe rather than by HBM on parts whose FP64 rate is a small
// fraction of the FP32 rate, so their roofline is min(HBM bandwidth x
// intensity, FP64 rate).  The FP64 rate is measured here rather than assumed:
// every thread runs independent FMA chains (enough of them to cover the pipe
// latency) on a grid of several blocks per SM, and the rate is FMAs x 2 / time,
// timed with CUDA events on the given stream.
#include <cstdio>

#include "apfc_internal.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kProbeThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kProbeThreads) k_fma_probe(T* out, int iters, T m, T c) {
  T a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = (T)(threadIdx.x + 1) * (T)1e-3 + (T)i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int i = 0; i < kChains; ++i) {
        if constexpr (sizeof(T) == 8)
          a[i] = fma(a[i], m, c);
        else
          a[i] = fmaf(a[i], m, c);
      }
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  // never true for the chains' values; keeps the compiler from removing them
  if (s == (T)-1.2345) out[blockIdx.x] = s;
}

template <typename T>
apfc_status run_probe(cudaStream_t s, double* flops) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return APFC_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) return APFC_ECUDA;
  const int blocks = 8 * sms;
  // FP64 runs at a small fraction of the FP32 rate: fewer iterations keep both near 50 ms
  const int iters = sizeof(T) == 8 ? 512 : 16384;
  T* out = nullptr;
  if (cudaMalloc(&out, blocks * sizeof(T)) != cudaSuccess) return APFC_ENOMEM;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  apfc_status st = APFC_ECUDA;
  float best = 0.f;
  if (cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
    const T m = (T)0.999999, c = (T)1e-7;
    k_fma_probe<T><<<blocks, kProbeThreads, 0, s>>>(out, iters, m, c);  // warm-up
    st = APFC_OK;
    for (int rep = 0; rep < 3 && st == APFC_OK; ++rep) {
      cudaEventRecord(e0, s);
      k_fma_probe<T><<<blocks, kProbeThreads, 0, s>>>(out, iters, m, c);
      cudaEventRecord(e1, s);
      float ms = 0.f;
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
          cudaGetLastError() != cudaSuccess)
        st = APFC_ECUDA;
      else if (best == 0.f || ms < best)
        best = ms;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  if (st != APFC_OK || !(best > 0.f)) return APFC_ECUDA;
  const double fmas = (double)blocks * kProbeThreads * iters * 4.0 * kChains;
  *flops = 2.0 * fmas / (best * 1e-3);
  return APFC_OK;
}

}  // namespace

extern "C" apfc_status apfc_measure_fma_rate(int precision, void* stream, double* flops) {
  if (!flops || (precision != APFC_FP64 && precision != APFC_FP32_REFINED)) return APFC_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return precision == APFC_FP64 ? run_probe<double>(s, flops) : run_probe<float>(s, flops);
}
