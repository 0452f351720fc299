// Fused 2D pipeline entry points: x += P^{-1} u and x = P^{-1} b (the
// pipeline without the block operator), the BiCGStab vector updates of the
// unmerged and merged iterations, and the geometry queries of the fused
// kernels.  The kernel template itself is in fused2d.cuh.
#include "fused2d.cuh"

namespace apfc {

namespace {

// BiCGStab vector update: s = r - alpha v; u += alpha p + omega s; r = s - omega t;
// partials of (rhat, r) and (r, r).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_bicg_update(cplx<T>* __restrict__ r, const cplx<T>* __restrict__ v,
                                                          const cplx<T>* __restrict__ p, cplx<T>* __restrict__ u,
                                                          const cplx<T>* __restrict__ t,
                                                          const cplx<T>* __restrict__ rhat, const KScal* ks,
                                                          long long pts, void* partials, OpCoef c) {
  const int j = blockIdx.y;
  if (ks[j].active == 0) return;
  prof_add(c, kid_of<T>(KID_BICG_UPDATE), 16ull * (unsigned long long)pts * sizeof(cplx<T>));
  const cplx<T> al = to_c<T>(ks[j].alpha), om = to_c<T>(ks[j].omega);
  const long long n = 2 * pts, o = 2LL * j * pts;
  Acc<T> a0, a1;
  a0.zero();
  a1.zero();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long q = o + i;
    const cplx<T> s = csub(r[q], cmulz(al, v[q]));
    u[q] = cadd(u[q], cadd(cmulz(al, p[q]), cmulz(om, s)));
    const cplx<T> rn = csub(s, cmulz(om, t[q]));
    r[q] = rn;
    a0.add(rhat[q], rn);
    a1.add(rn, rn);
  }
  block_reduce<T>(a0);
  if (threadIdx.x == 0) a0.store(partials, (long long)(j * kDotSlots + 0) * kDotBlocks + blockIdx.x);
  block_reduce<T>(a1);
  if (threadIdx.x == 0) a1.store(partials, (long long)(j * kDotSlots + 1) * kDotBlocks + blockIdx.x);
}

}  // namespace

int fused2d_max_degree(int elem_bytes) { return elem_bytes == 8 ? 4 : 4; }

int fused2d_npart(const OpCoef& c, int m, int Ly, int elem_bytes, int tile) {
  return geom(c, 2 * m + 2, Ly, tile_nt(elem_bytes, m, tile)).npart;
}

int fused2d_tiles() { return kTiles; }

int fused2d_blocks(int nx, int ny, int J, int m, int Ly, int elem_bytes, int tile, bool with_a, int* npart) {
  OpCoef c{};
  c.nx = nx;
  c.ny = ny;
  const PipeGeom g = geom(c, 2 * m + 1 + (with_a ? 1 : 0), Ly, tile_nt(elem_bytes, m, tile));
  if (npart) *npart = g.npart;
  return g.npart * J;
}

template <typename T>
bool launch_fused_pinv_add(int m, int Ly, int tile, const OpCoef& c, const ChebStep* w, const cplx<T>* u, double2* x64,
                           cudaStream_t s, const BatchLaunch* bl) {
  LoadPlain<T> ld{u, c.pts};
  EpAddX<T> ep{x64, c.pts};
  // reads u (2 fields); reads and writes the FP64 block x (2 FP64 fields each way)
  const int f = 2 + 4 * (int)(sizeof(double2) / sizeof(cplx<T>));
  return dispatch<T, false>(m, tile, c, w, Ly, ld, ep, nullptr, nullptr, s, kid_of<T>(KID_FUSED_PINV), f, bl);
}

template <typename T>
bool launch_fused_pinv_store(int m, int Ly, int tile, const OpCoef& c, const ChebStep* w, const cplx<T>* b, cplx<T>* x,
                             cudaStream_t s) {
  LoadPlain<T> ld{b, c.pts};
  EpStore<T> ep{x, c.pts};
  return dispatch<T, false>(m, tile, c, w, Ly, ld, ep, nullptr, nullptr, s, kid_of<T>(KID_FUSED_PINV), 4);
}

// u += alpha p + omega (r - alpha v) for amplitudes whose solve stopped in this iteration.
// Batched runs: blockIdx.z selects the run.  FP32 vectors stream as 16-byte pairs of
// complex values (each amplitude's block starts at an even element of a 256-byte
// aligned allocation, and holds an even number 2 pts of values).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_final_update(const cplx<T>* __restrict__ r,
                                                           const cplx<T>* __restrict__ v,
                                                           const cplx<T>* __restrict__ p, cplx<T>* __restrict__ u,
                                                           const KScal* ks, OpCoef c, const RunGeom* rg) {
  const int j = blockIdx.y;
  long long o = 0;
  if (rg != nullptr) {
    o = select_run(rg, blockIdx.z, c);
    ks += (long long)blockIdx.z * c.J;
  }
  if (ks[j].just_done == 0) return;
  prof_add(c, kid_of<T>(KID_BICG_UPDATE), 10ull * (unsigned long long)c.pts * sizeof(cplx<T>));
  const cplx<T> al = to_c<T>(ks[j].alpha), om = to_c<T>(ks[j].omega);
  const long long n = 2 * c.pts;
  o += 2LL * j * c.pts;
  const long long stride = (long long)gridDim.x * blockDim.x;
  if constexpr (sizeof(T) == 4) {
    const float4* r4 = reinterpret_cast<const float4*>(r + o);
    const float4* v4 = reinterpret_cast<const float4*>(v + o);
    const float4* p4 = reinterpret_cast<const float4*>(p + o);
    float4* u4 = reinterpret_cast<float4*>(u + o);
    auto upd = [&](float2 rr, float2 vv, float2 pp, float2 uu) {
      const float2 sv = csub(rr, cmulz(al, vv));
      return cadd(uu, cadd(cmulz(al, pp), cmulz(om, sv)));
    };
#pragma unroll 2
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n / 2; i += stride) {
      const float4 rr = r4[i], vv = v4[i], pp = p4[i], uu = u4[i];
      const float2 a = upd(make_float2(rr.x, rr.y), make_float2(vv.x, vv.y), make_float2(pp.x, pp.y),
                           make_float2(uu.x, uu.y));
      const float2 b = upd(make_float2(rr.z, rr.w), make_float2(vv.z, vv.w), make_float2(pp.z, pp.w),
                           make_float2(uu.z, uu.w));
      u4[i] = make_float4(a.x, a.y, b.x, b.y);
    }
  } else {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
      const long long q = o + i;
      const cplx<T> sv = csub(r[q], cmulz(al, v[q]));
      u[q] = cadd(u[q], cadd(cmulz(al, p[q]), cmulz(om, sv)));
    }
  }
}

template <typename T>
void launch_final_update(const cplx<T>* r, const cplx<T>* v, const cplx<T>* p, cplx<T>* u, const KScal* ks,
                         const OpCoef& c, cudaStream_t s, const BatchLaunch* bl) {
  ProfScope ps_(kid_of<T>(KID_BICG_UPDATE), s);
  if (bl != nullptr) {
    k_final_update<T><<<dim3(kDotBlocks, c.J, bl->R), kThreads, 0, s>>>(r, v, p, u, ks, c, bl->dev);
    return;
  }
  // usually one amplitude is done at a time: enough blocks for that one to fill the GPU
  k_final_update<T><<<dim3(4 * kDotBlocks, c.J), kThreads, 0, s>>>(r, v, p, u, ks, c, nullptr);
}

template <typename T>
void launch_bicg_update(cplx<T>* r, const cplx<T>* v, const cplx<T>* p, cplx<T>* u, const cplx<T>* t,
                        const cplx<T>* rhat, const KScal* ks, void* partials, const OpCoef& c, cudaStream_t s) {
  ProfScope ps_(kid_of<T>(KID_BICG_UPDATE), s);
  k_bicg_update<T><<<dim3(kDotBlocks, c.J), kThreads, 0, s>>>(r, v, p, u, t, rhat, ks, c.pts, partials, c);
}

#define APFC_FUSED_INST(T)                                                                                         \
  template void launch_final_update<T>(const cplx<T>*, const cplx<T>*, const cplx<T>*, cplx<T>*, const KScal*,     \
                                       const OpCoef&, cudaStream_t, const BatchLaunch*);                          \
  template bool launch_fused_pinv_add<T>(int, int, int, const OpCoef&, const ChebStep*, const cplx<T>*, double2*,   \
                                         cudaStream_t, const BatchLaunch*);                                        \
  template bool launch_fused_pinv_store<T>(int, int, int, const OpCoef&, const ChebStep*, const cplx<T>*, cplx<T>*, \
                                           cudaStream_t);                                                          \
  template void launch_bicg_update<T>(cplx<T>*, const cplx<T>*, const cplx<T>*, cplx<T>*, const cplx<T>*,          \
                                      const cplx<T>*, const KScal*, void*, const OpCoef&, cudaStream_t);

APFC_FUSED_INST(double)
APFC_FUSED_INST(float)

}  // namespace apfc
