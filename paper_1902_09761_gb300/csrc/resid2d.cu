// FP64-accurate outer residual of the FP32-refined step on one 2D grid, with its
// tiles staged by TMA.
//
// r = b - A x per amplitude, A the block operator of Eq. linear_system2 (M = I):
//   r1 = b1 - zeta + G_h eta,   r2 = b2 - kt G_h zeta - a eta.
// x and b stay FP64 in memory; the arithmetic is FP32 (split of every double
// into an FP32 pair by integer operations, one compensated sum of products per
// component: dfloat.cuh), because GB300's FP64 pipe would bound the kernel far
// below HBM speed.
//
// Each block walks the 32 x 8 point tiles of one amplitude.  Per tile one
// thread issues four TMA box loads into a two-stage shared-memory ring (zeta
// and eta with a one-point halo, b1 and b2), two tiles ahead, completing on the
// stage's mbarrier.  TMA fills boxes beyond the grid with zeros; on tiles at the
// grid's edge those cells are re-read from the periodic image with plain loads.
// The raw doubles of a tile are split once into FP32 pairs in shared memory,
// then every thread evaluates its point's residual.
#include <cstring>
#include <mutex>

#include "apfc_internal.cuh"
#include "dfloat.cuh"
#include "tma.cuh"

#include <cudaTypedefs.h>

namespace apfc {

namespace {

__device__ unsigned long long g_timeouts;

constexpr int TX = 32, TY = 8, HX = TX + 2, HY = TY + 2;
constexpr int kHalo = HX * HY;
constexpr unsigned kZBytes = kHalo * 16, kBBytes = TX * TY * 16;
constexpr unsigned kZPad = (kZBytes + 127) / 128 * 128;
// stage layout (bytes): zeta halo box, eta halo box, b1 box, b2 box
constexpr unsigned kOffE = kZPad, kOffB1 = 2 * kZPad, kOffB2 = 2 * kZPad + kBBytes;
constexpr unsigned kStageBytes = 2 * kZPad + 2 * kBBytes;
constexpr unsigned kStageTx = 2 * kZBytes + 2 * kBBytes;
constexpr int kStages = 2;
constexpr size_t kSmem = kStages * kStageBytes + 2 * kHalo * sizeof(float4) + 128;

__device__ __forceinline__ float4 pack4(PDF v) { return make_float4(v.h.x, v.l.x, v.h.y, v.l.y); }
__device__ __forceinline__ PDF unpack4(float4 v) { return PDF{make_float2(v.x, v.z), make_float2(v.y, v.w)}; }
__device__ __forceinline__ PDF swap_ri(PDF v) { return PDF{make_float2(v.h.y, v.h.x), make_float2(v.l.y, v.l.x)}; }
struct LaneC {
  float2 h, l;
};
__device__ __forceinline__ LaneC lane_c(double c, float s0, float s1) {
  const DF d = split_d(c);
  return LaneC{make_float2(s0 * d.h, s1 * d.h), make_float2(s0 * d.l, s1 * d.l)};
}

__global__ void __launch_bounds__(256) k_resid2d_tma(const __grid_constant__ CUtensorMap mx,
                                                     const __grid_constant__ CUtensorMap mb,
                                                     const double2* __restrict__ x, float2* __restrict__ r32,
                                                     double2* __restrict__ r64, double2* __restrict__ partials,
                                                     const __grid_constant__ OpCoef c) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ unsigned long long bar[kStages];
  __shared__ int s_fail;
  // TMA destinations: 128-byte aligned (the launch reserves 128 spare bytes)
  unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  float4* sz = reinterpret_cast<float4*>(smem + kStages * kStageBytes);
  float4* se = sz + kHalo;
  const int j = blockIdx.y, t = threadIdx.x;
  const int nx = c.nx, ny = c.ny;
  const long long pts = c.pts, o = 2LL * j * pts;
  if (c.prof != nullptr && blockIdx.x == 0 && t == 0)
    atomicAdd(c.prof + KID_RESID_REFINE,
              (unsigned long long)pts * (4 * sizeof(double2) + 2 * sizeof(float2) + (r64 ? 2 * sizeof(double2) : 0)));
  // G_h: c0 at the centre, 1/h_d^2 on the d-neighbours, the advection i (k_d/h_d)(u(+d) - u(-d))
  // as lane coefficients on (im, re)-swapped values; the (2,1) block carries -kt G_h
  const LaneC g0 = lane_c(c.c0, 1.f, 1.f), gx = lane_c(c.ih2[0], 1.f, 1.f), gy = lane_c(c.ih2[1], 1.f, 1.f);
  const LaneC axp = lane_c(c.kh[j][0], -1.f, 1.f), axm = lane_c(c.kh[j][0], 1.f, -1.f);
  const LaneC ayp = lane_c(c.kh[j][1], -1.f, 1.f), aym = lane_c(c.kh[j][1], 1.f, -1.f);
  const double kt = c.kt[j];
  const LaneC k0 = lane_c(kt * c.c0, -1.f, -1.f), kx = lane_c(kt * c.ih2[0], -1.f, -1.f);
  const LaneC ky = lane_c(kt * c.ih2[1], -1.f, -1.f);
  const LaneC kxp = lane_c(kt * c.kh[j][0], 1.f, -1.f), kxm = lane_c(kt * c.kh[j][0], -1.f, 1.f);
  const LaneC kyp = lane_c(kt * c.kh[j][1], 1.f, -1.f), kym = lane_c(kt * c.kh[j][1], -1.f, 1.f);
  LaneC ma = lane_c(c.a[j], -1.f, -1.f);

  const int txc = (nx + TX - 1) / TX, ntiles = txc * ((ny + TY - 1) / TY);
  auto stage = [&](int s) { return smem + s * kStageBytes; };
  auto issue = [&](int tile, int s) {  // thread 0
    const int tyi = tile / txc, x0 = (tile - tyi * txc) * TX, y0 = tyi * TY;
    unsigned char* st = stage(s);
    fence_proxy_async();
    mbar_arrive_expect_tx(&bar[s], kStageTx);
    tma_load_3d(st, &mx, &bar[s], 2 * (x0 - 1), y0 - 1, 2 * j);
    tma_load_3d(st + kOffE, &mx, &bar[s], 2 * (x0 - 1), y0 - 1, 2 * j + 1);
    tma_load_3d(st + kOffB1, &mb, &bar[s], 2 * x0, y0, 2 * j);
    tma_load_3d(st + kOffB2, &mb, &bar[s], 2 * x0, y0, 2 * j + 1);
  };
  if (t == 0) {
    tma_prefetch_map(&mx);
    tma_prefetch_map(&mb);
    for (int s = 0; s < kStages; ++s) mbar_init(&bar[s], 1);
    fence_mbar_init();
    s_fail = 0;
  }
  __syncthreads();
  if (t == 0)
    for (int s = 0; s < kStages; ++s)
      if (blockIdx.x + s * (int)gridDim.x < ntiles) issue(blockIdx.x + s * gridDim.x, s);

  const int tx = t & 31, ty = t >> 5;
  float rr = 0.f;
  int k = 0;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++k) {
    const int s = k & 1;
    const int tyi = tile / txc, x0 = (tile - tyi * txc) * TX, y0 = tyi * TY;
    if (!mbar_wait(&bar[s], (k >> 1) & 1)) s_fail = 1;
    unsigned char* st = stage(s);
    double2* rz = reinterpret_cast<double2*>(st);
    double2* re = reinterpret_cast<double2*>(st + kOffE);
    const double2 b1v = reinterpret_cast<const double2*>(st + kOffB1)[t];
    const double2 b2v = reinterpret_cast<const double2*>(st + kOffB2)[t];
    if (x0 == 0 || y0 == 0 || x0 + TX >= nx || y0 + TY >= ny) {
      // cells beyond the grid: the periodic image (TMA filled them with zeros)
      for (int i = t; i < kHalo; i += blockDim.x) {
        const int ry = i / HX, rx = i - ry * HX;
        int gxx = x0 - 1 + rx, gyy = y0 - 1 + ry;
        if (gxx >= 0 && gxx < nx && gyy >= 0 && gyy < ny) continue;
        gxx = gxx < 0 ? gxx + nx : gxx % nx;
        gyy = gyy < 0 ? gyy + ny : gyy % ny;
        const long long q = (long long)gyy * nx + gxx;
        rz[i] = x[o + q];
        re[i] = x[o + pts + q];
      }
    }
    __syncthreads();
    if (s_fail) break;
    for (int i = t; i < kHalo; i += blockDim.x) {
      sz[i] = pack4(pdf_split(rz[i]));
      se[i] = pack4(pdf_split(re[i]));
    }
    __syncthreads();
    // the stage is consumed: refill it two tiles ahead
    if (t == 0 && tile + kStages * (int)gridDim.x < ntiles) issue(tile + kStages * gridDim.x, s);
    const int xx = x0 + tx, yy = y0 + ty;
    if (xx >= nx || yy >= ny) continue;
    const long long pc = (long long)yy * nx + xx;
    const int cc = (ty + 1) * HX + tx + 1;
    const PDF zc = unpack4(sz[cc]), zl = unpack4(sz[cc - 1]), zr = unpack4(sz[cc + 1]);
    const PDF zu = unpack4(sz[cc - HX]), zd = unpack4(sz[cc + HX]);
    const PDF ec = unpack4(se[cc]), el = unpack4(se[cc - 1]), er = unpack4(se[cc + 1]);
    const PDF eu = unpack4(se[cc - HX]), ed = unpack4(se[cc + HX]);
    PAcc a1;  // r1 = b1 - zeta + G_h eta
    a1.init(pdf_split(b1v));
    a1.add(zc, -1.f);
    a1.fma(g0.h, g0.l, ec);
    a1.fma(gx.h, gx.l, el);
    a1.fma(gx.h, gx.l, er);
    a1.fma(gy.h, gy.l, eu);
    a1.fma(gy.h, gy.l, ed);
    a1.fma(axp.h, axp.l, swap_ri(er));
    a1.fma(axm.h, axm.l, swap_ri(el));
    a1.fma(ayp.h, ayp.l, swap_ri(ed));
    a1.fma(aym.h, aym.l, swap_ri(eu));
    if (c.jd != nullptr) ma = lane_c(a_at(c, j, pc), -1.f, -1.f);
    PAcc a2;  // r2 = b2 - kt G_h zeta - a eta
    a2.init(pdf_split(b2v));
    a2.fma(k0.h, k0.l, zc);
    a2.fma(kx.h, kx.l, zl);
    a2.fma(kx.h, kx.l, zr);
    a2.fma(ky.h, ky.l, zu);
    a2.fma(ky.h, ky.l, zd);
    a2.fma(kxp.h, kxp.l, swap_ri(zr));
    a2.fma(kxm.h, kxm.l, swap_ri(zl));
    a2.fma(kyp.h, kyp.l, swap_ri(zd));
    a2.fma(kym.h, kym.l, swap_ri(zu));
    a2.fma(ma.h, ma.l, ec);
    float2 f1, l1, f2, l2;
    a1.result(f1, l1);
    a2.result(f2, l2);
    r32[o + pc] = f1;
    r32[o + pts + pc] = f2;
    if (r64 != nullptr) {
      r64[o + pc] = make_double2(df_to_d(DF{f1.x, l1.x}), df_to_d(DF{f1.y, l1.y}));
      r64[o + pts + pc] = make_double2(df_to_d(DF{f2.x, l2.x}), df_to_d(DF{f2.y, l2.y}));
    }
    rr = fmaf(f1.x, f1.x, fmaf(f1.y, f1.y, fmaf(f2.x, f2.x, fmaf(f2.y, f2.y, rr))));
  }
  if (s_fail) {
    // a tile never arrived: give the copies still in flight a bounded chance to land,
    // count the timeout and make this amplitude's residual norm NaN
    if (t == 0) {
      for (int d = 0; d < kStages; ++d)
        if (blockIdx.x + (k + d) * (int)gridDim.x < ntiles) (void)mbar_wait(&bar[(k + d) & 1], ((k + d) >> 1) & 1);
      atomicAdd(&g_timeouts, 1ull);
    }
    rr = __int_as_float(0x7fc00000);
  }
  // block sum of ||r||^2 (FP64 across the block)
  double v = (double)rr;
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  __shared__ double sh[8];
  if ((t & 31) == 0) sh[t >> 5] = v;
  __syncthreads();
  if (t == 0) {
    double sum = 0.0;
    for (int w = 0; w < 8; ++w) sum += sh[w];
    partials[(j * kDotSlots + 0) * kDotBlocks + blockIdx.x] = make_double2(sum, 0.0);
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn(const char** err) {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  if (!fn && err) *err = "the driver has no cuTensorMapEncodeTiled";
  return fn;
}

}  // namespace

bool tma_encode_f64(CUtensorMap* map, const void* base, const unsigned long long dims[3],
                    const unsigned long long strides[2], const unsigned box[3], const char** err) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn(err);
  if (!fn) return false;
  const cuuint64_t gd[3] = {dims[0], dims[1], dims[2]};
  const cuuint64_t gs[2] = {strides[0], strides[1]};
  const cuuint32_t bd[3] = {box[0], box[1], box[2]};
  const cuuint32_t es[3] = {1, 1, 1};
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, const_cast<void*>(base), gd, gs, bd, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    if (err) *err = "cuTensorMapEncodeTiled rejected the tensor map";
    return false;
  }
  return true;
}

unsigned long long tma_timeouts() {
  unsigned long long v = 0;
  if (cudaMemcpyFromSymbol(&v, g_timeouts, sizeof(v)) != cudaSuccess) return 0;
  return v;
}

// x, b: block vectors [J][2][ny][nx] of complex doubles; one grid (no batch).
bool launch_residual_refine2d_tma(const double2* b, const double2* x, float2* r32, double2* r64, double* partials,
                                  const OpCoef& c, cudaStream_t s, const char** err) {
  CUtensorMap mx, mb;
  const unsigned long long dims[3] = {2ull * c.nx, (unsigned long long)c.ny, 2ull * c.J};
  const unsigned long long strides[2] = {16ull * c.nx, 16ull * c.nx * c.ny};
  const unsigned bx[3] = {2 * HX, HY, 1}, bb[3] = {2 * TX, TY, 1};
  if (!tma_encode_f64(&mx, x, dims, strides, bx, err) || !tma_encode_f64(&mb, b, dims, strides, bb, err)) return false;
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(k_resid2d_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem) != cudaSuccess) {
      if (err) *err = "cannot raise the shared memory of the residual kernel";
      return false;
    }
    attr = true;
  }
  ProfScope ps_(KID_RESID_REFINE, s);
  k_resid2d_tma<<<dim3(kDotBlocks, c.J), 256, kSmem, s>>>(mx, mb, x, r32, r64, reinterpret_cast<double2*>(partials),
                                                         c);
  return true;
}

}  // namespace apfc
