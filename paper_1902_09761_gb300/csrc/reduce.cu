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
#include "bf16pair.cuh"

namespace apfc {

namespace {

// Batched runs (rg != nullptr): blockIdx.z selects the run; its partials start at
// slot run * J * kDotSlots * kDotBlocks.
template <typename T, int NP>
__global__ void k_dots(DotPairs<T> pr, void* partials, OpCoef c, const KScal* act, const RunGeom* rg) {
  const int j = blockIdx.y;
  long long o = 0, pbase = 0;
  if (rg != nullptr) {
    o = select_run(rg, blockIdx.z, c);
    pbase = (long long)blockIdx.z * c.J * kDotSlots * kDotBlocks;
    if (act != nullptr) act += (long long)blockIdx.z * c.J;
  }
  if (act != nullptr && act[j].active == 0) return;
  const long long n = 2LL * c.pts;
  o += 2LL * j * c.pts;
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
    if (threadIdx.x == 0) acc[q].store(partials, pbase + (long long)(j * kDotSlots + q) * kDotBlocks + blockIdx.x);
  }
}

// Reduce the partial sums of amplitude j (slots base + (j kDotSlots + q) npart + b)
// and apply the scalar update `op` to its Krylov scalars.
template <typename T, int NP>
__device__ void finalize_one(const void* partials, long long base, int npart, int j, KScal& k, int op) {
  // a pending final update was applied after the previous OP_OMEGA5: clear the flag
  if (op == OP_ALPHA && threadIdx.x == 0) k.just_done = 0;
  if (op != OP_INIT && op != OP_INIT3 && op != OP_NORMS && op != OP_RNORM && op != OP_BNORM && k.active == 0) return;
  __shared__ double2 res[kDotSlots];
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    Acc<T> a;
    a.zero();
    for (int b = threadIdx.x; b < npart; b += blockDim.x) {
      Acc<T> t;
      t.load(partials, base + (long long)(j * kDotSlots + q) * npart + b);
      a.merge(t);
    }
    block_reduce<T>(a);
    if (threadIdx.x == 0) res[q] = a.value();
  }
  if (threadIdx.x == 0) scalar_update(k, op, res);
}

// Start of an FP32 solve from x0 = 0, in one pass: r = b, rhat = b rounded to bf16 with its
// packed copy rh16 (bf16pair.cuh), and the partial sums of (r, r), (b, b) and (rhat, r) in
// slots 0-2, laid out as k_dots' (batched runs: blockIdx.z selects the run).
__global__ void __launch_bounds__(kThreads) k_init32(const float2* __restrict__ b, float2* __restrict__ r,
                                                     float2* __restrict__ rhat, uint2* __restrict__ rh16,
                                                     void* partials, OpCoef c, const RunGeom* rg) {
  const int j = blockIdx.y;
  long long o = 0, pbase = 0;
  if (rg != nullptr) {
    o = select_run(rg, blockIdx.z, c);
    pbase = (long long)blockIdx.z * c.J * kDotSlots * kDotBlocks;
  }
  const long long pts = c.pts, o1 = o + 2LL * j * pts, o2 = o1 + pts;
  uint2* q = rh16 + o / 2 + (long long)j * pts;
  if (c.prof != nullptr && blockIdx.x == 0 && threadIdx.x == 0)
    atomicAdd(c.prof + kid_of<float>(KID_DOTS), (unsigned long long)pts * (6 * sizeof(float2) + sizeof(uint2)));
  Acc<float> a0, a2;
  a0.zero();
  a2.zero();
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < pts; p += (long long)gridDim.x * blockDim.x) {
    const float2 b1 = b[o1 + p], b2 = b[o2 + p];
    r[o1 + p] = b1;
    r[o2 + p] = b2;
    const unsigned h1 = bf16_pack(b1), h2 = bf16_pack(b2);
    const float2 s1 = bf16_unpack(h1), s2 = bf16_unpack(h2);
    rhat[o1 + p] = s1;
    rhat[o2 + p] = s2;
    q[p] = make_uint2(h1, h2);
    a0.add(b1, b1);
    a0.add(b2, b2);
    a2.add(s1, b1);
    a2.add(s2, b2);
  }
  block_reduce<float>(a0);
  if (threadIdx.x == 0) {
    a0.store(partials, pbase + (long long)(j * kDotSlots + 0) * kDotBlocks + blockIdx.x);
    a0.store(partials, pbase + (long long)(j * kDotSlots + 1) * kDotBlocks + blockIdx.x);  // (b, b) = (r, r)
  }
  block_reduce<float>(a2);
  if (threadIdx.x == 0) a2.store(partials, pbase + (long long)(j * kDotSlots + 2) * kDotBlocks + blockIdx.x);
}

template <typename T, int NP>
__global__ void k_finalize(const void* partials, int npart, KScal* ks, int op) {
  finalize_one<T, NP>(partials, 0, npart, blockIdx.x, ks[blockIdx.x], op);
}

// Batched runs: block run * J + j.  npart_fixed > 0: the run's partials follow the
// fixed layout of k_dots; 0: the fused-pipeline layout of the run table (the
// t-kernel's when tlay).
template <typename T, int NP>
__global__ void k_finalize_batch(const void* partials, int npart_fixed, const RunGeom* rg, int J, KScal* ks, int op,
                                 int tlay) {
  const int run = blockIdx.x / J, j = blockIdx.x - run * J;
  long long base;
  int npart;
  if (npart_fixed > 0) {
    base = (long long)run * J * kDotSlots * npart_fixed;
    npart = npart_fixed;
  } else {
    base = tlay ? rg[run].part_off_t : rg[run].part_off;
    npart = tlay ? rg[run].npart_t : rg[run].npart;
  }
  finalize_one<T, NP>(partials, base, npart, j, ks[blockIdx.x], op);
}

}  // namespace

void launch_init32(const float2* b, float2* r, float2* rhat, uint2* rh16, void* partials, const OpCoef& c,
                   cudaStream_t s, const BatchLaunch* bl) {
  ProfScope ps_(kid_of<float>(KID_DOTS), s);
  k_init32<<<dim3(kDotBlocks, c.J, bl ? bl->R : 1), kThreads, 0, s>>>(b, r, rhat, rh16, partials, c,
                                                                        bl ? bl->dev : nullptr);
}

template <typename T>
void launch_dots(int npair, const DotPairs<T>& pr, void* partials, const OpCoef& c, const KScal* act, cudaStream_t s,
                 const BatchLaunch* bl) {
  const dim3 g(kDotBlocks, c.J, bl ? bl->R : 1);
  const RunGeom* rg = bl ? bl->dev : nullptr;
  ProfScope ps_(kid_of<T>(KID_DOTS), s);
  if (npair == 1)
    k_dots<T, 1><<<g, kThreads, 0, s>>>(pr, partials, c, act, rg);
  else if (npair == 2)
    k_dots<T, 2><<<g, kThreads, 0, s>>>(pr, partials, c, act, rg);
  else
    k_dots<T, 3><<<g, kThreads, 0, s>>>(pr, partials, c, act, rg);
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

template <typename T>
void launch_finalize_batch(int npair, const void* partials, int npart_fixed, const BatchLaunch& bl, int J, KScal* k,
                           int op, cudaStream_t s) {
  ProfScope ps_(kid_of<T>(KID_FINALIZE), s);
  const int nb = bl.R * J;
  if (npair == 1)
    k_finalize_batch<T, 1><<<nb, kThreads, 0, s>>>(partials, npart_fixed, bl.dev, J, k, op, bl.tlay);
  else if (npair == 2)
    k_finalize_batch<T, 2><<<nb, kThreads, 0, s>>>(partials, npart_fixed, bl.dev, J, k, op, bl.tlay);
  else if (npair == 3)
    k_finalize_batch<T, 3><<<nb, kThreads, 0, s>>>(partials, npart_fixed, bl.dev, J, k, op, bl.tlay);
  else
    k_finalize_batch<T, 5><<<nb, kThreads, 0, s>>>(partials, npart_fixed, bl.dev, J, k, op, bl.tlay);
}

void launch_finalize64(int npair, const void* partials, KScal* k, int op, int J, cudaStream_t s) {
  launch_finalize<double>(npair, partials, k, op, J, s);
}

template void launch_dots<double>(int, const DotPairs<double>&, void*, const OpCoef&, const KScal*, cudaStream_t,
                                  const BatchLaunch*);
template void launch_dots<float>(int, const DotPairs<float>&, void*, const OpCoef&, const KScal*, cudaStream_t,
                                 const BatchLaunch*);
template void launch_finalize_batch<double>(int, const void*, int, const BatchLaunch&, int, KScal*, int, cudaStream_t);
template void launch_finalize_batch<float>(int, const void*, int, const BatchLaunch&, int, KScal*, int, cudaStream_t);
template void launch_finalize<double>(int, const void*, KScal*, int, int, cudaStream_t, int);
template void launch_finalize<float>(int, const void*, KScal*, int, int, cudaStream_t, int);

}  // namespace apfc
