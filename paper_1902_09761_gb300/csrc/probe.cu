// Arithmetic-rate probe: FP64 and FP32 FMA throughput and FP64 <-> FP32
// conversion throughput of this GPU.
//
// The FP64 kernels of the step (outer residual, nonlinear right-hand side) are
// bound by the FP64 pipe rather than by HBM on parts whose FP64 rate is a small
// fraction of the FP32 rate, so their roofline is min(HBM bandwidth x
// intensity, FP64 rate).  The rates are measured here rather than assumed:
// every thread runs independent chains (enough of them to cover the pipe
// latency) on a grid of several blocks per SM, timed with CUDA events on the
// given stream.
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

// FP64 -> FP32 -> FP64 round trips: two conversions per link of each chain.
__global__ void __launch_bounds__(kProbeThreads) k_cvt_probe(double* out, int iters) {
  double a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = (double)(threadIdx.x + 1) * 1e-3 + (double)i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int i = 0; i < kChains; ++i) a[i] = (double)__double2float_rn(a[i]);
  }
  double s = 0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  if (s == -1.2345) out[blockIdx.x] = s;
}

// kind 0: FP64 FMA, 1: FP32 FMA, 2: FP64 <-> FP32 conversions.  *rate: FLOP/s
// (2 per FMA) for kinds 0 and 1, conversions/s for kind 2.
template <typename T>
apfc_status run_probe(cudaStream_t s, int kind, double* rate) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return APFC_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) return APFC_ECUDA;
  const int blocks = 8 * sms;
  // FP64 runs at a small fraction of the FP32 rate: fewer iterations keep both near 50 ms
  const int iters = kind == 1 ? 16384 : 512;
  T* out = nullptr;
  if (cudaMalloc(&out, blocks * sizeof(T)) != cudaSuccess) return APFC_ENOMEM;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  apfc_status st = APFC_ECUDA;
  float best = 0.f;
  if (cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
    const T m = (T)0.999999, c = (T)1e-7;
    auto launch = [&]() {
      if constexpr (sizeof(T) == 8) {
        if (kind == 2) {
          k_cvt_probe<<<blocks, kProbeThreads, 0, s>>>(out, iters);
          return;
        }
      }
      k_fma_probe<T><<<blocks, kProbeThreads, 0, s>>>(out, iters, m, c);
    };
    launch();  // warm-up
    st = APFC_OK;
    for (int rep = 0; rep < 3 && st == APFC_OK; ++rep) {
      cudaEventRecord(e0, s);
      launch();
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
  const double ops = (double)blocks * kProbeThreads * iters * 4.0 * kChains;
  *rate = 2.0 * ops / (best * 1e-3);  // 2 FLOP per FMA, 2 conversions per link
  return APFC_OK;
}

}  // namespace

extern "C" apfc_status apfc_measure_alu_rate(int kind, void* stream, double* rate) {
  if (!rate || kind < APFC_ALU_FMA64 || kind > APFC_ALU_CVT64) return APFC_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return kind == APFC_ALU_FMA32 ? run_probe<float>(s, kind, rate) : run_probe<double>(s, kind, rate);
}
