// FP64-accurate outer residual of the FP32-refined step on one 2D or 3D grid, with
// its tiles staged by TMA.
//
// r = b - A x per amplitude, A the block operator of Eq. linear_system2 (M = I):
//   r1 = b1 - zeta + G_h eta,   r2 = b2 - kt G_h zeta - a eta.
// x and b stay FP64 in memory; the arithmetic is FP32 (split of every double
// into an FP32 pair by integer operations, one compensated sum of products per
// component: dfloat.cuh), because GB300's FP64 pipe would bound the kernel far
// below HBM speed.
//
// Each block walks the 32 x 8 point tiles (of one plane, on 3D grids) of one
// amplitude.  Per tile one thread issues the TMA box loads into a two-stage
// shared-memory ring (zeta and eta with a one-point halo, b1 and b2, and on 3D
// grids the tile's own columns of zeta and eta in the planes above and below,
// whose z coordinates wrap periodically), two tiles ahead, completing on the
// stage's mbarrier.  TMA fills boxes beyond the grid with zeros; on tiles at the
// grid's edge those cells are re-read from the periodic image with plain loads.
// The raw doubles of a tile are split once into FP32 pairs in shared memory,
// then every thread evaluates its point's residual (resid_point.cuh).
#include <cstring>
#include <mutex>

#include "apfc_internal.cuh"
#include "dfloat.cuh"
#include "resid_point.cuh"
#include "tma.cuh"

#include <cudaTypedefs.h>

namespace apfc {

namespace {

__device__ unsigned long long g_timeouts;

constexpr int TX = 32, TY = 8, HX = TX + 2, HY = TY + 2;
constexpr int kHalo = HX * HY;
constexpr unsigned kZBytes = kHalo * 16, kBBytes = TX * TY * 16;
constexpr unsigned kZPad = (kZBytes + 127) / 128 * 128;
// Stage layout (bytes): zeta and eta of the tile's plane with a one-point halo, b1, b2,
// and on 3D grids the tile's own columns of zeta and eta in the planes z - 1 and z + 1.
constexpr unsigned kOffE = kZPad, kOffB1 = 2 * kZPad, kOffB2 = kOffB1 + kBBytes, kOffZN = kOffB2 + kBBytes;
template <int DIM>
struct RLay {
  static constexpr unsigned stage = kOffZN + (DIM == 3 ? 4 * kBBytes : 0);
  static constexpr unsigned tx = 2 * kZBytes + (DIM == 3 ? 6 : 2) * kBBytes;
};
constexpr int kStages = 2;
template <int DIM>
constexpr size_t resid_smem() {
  return kStages * RLay<DIM>::stage + 2 * kHalo * sizeof(float4) + 128;
}


// Grid (blocks per amplitude, J); each block walks the tiles blockIdx.x + k gridDim.x of
// its amplitude (tiles: 32 x 8 points of one plane, planes slowest).  mx: the state block
// [J][2][nz][ny][nx] as FP64 (2 nx, ny, nz, 2J) with a 34 x 10 box (x0 - 1, y0 - 1);
// mxc: the same tensor with a 32 x 8 box (3D only: planes z -+ 1); mb: the right-hand
// side block with a 32 x 8 box.
template <int DIM>
__global__ void __launch_bounds__(256, DIM == 2 ? 3 : 2) k_resid_tma(const __grid_constant__ CUtensorMap mx,
                                                   const __grid_constant__ CUtensorMap mxc,
                                                   const __grid_constant__ CUtensorMap mb,
                                                   const double2* __restrict__ x, float2* __restrict__ r32,
                                                   double2* __restrict__ r64, double2* __restrict__ partials,
                                                   const __grid_constant__ OpCoef c) {
  using LY = RLay<DIM>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ unsigned long long bar[kStages];
  __shared__ int s_fail;
  // TMA destinations: 128-byte aligned (the launch reserves 128 spare bytes)
  unsigned char* smem = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  float4* sz = reinterpret_cast<float4*>(smem + kStages * LY::stage);
  float4* se = sz + kHalo;
  const int j = blockIdx.y, t = threadIdx.x;
  const int nx = c.nx, ny = c.ny, nz = DIM == 3 ? c.nz : 1;
  const long long pts = c.pts, o = 2LL * j * pts, plane = (long long)nx * ny;
  if (c.prof != nullptr && blockIdx.x == 0 && t == 0)
    atomicAdd(c.prof + KID_RESID_REFINE,
              (unsigned long long)pts * (4 * sizeof(double2) + 2 * sizeof(float2) + (r64 ? 2 * sizeof(double2) : 0)));
  const ResidCoef<DIM> q = resid_coef<DIM>(c, j);
  LaneC ma = lane_c(c.a[j], -1.f, -1.f);

  const int txc = (nx + TX - 1) / TX, tpl = txc * ((ny + TY - 1) / TY), ntiles = tpl * nz;
  auto stage = [&](int s) { return smem + s * LY::stage; };
  auto issue = [&](int tile, int s) {  // thread 0
    const int zz = tile / tpl, rem = tile - zz * tpl, tyi = rem / txc, x0 = (rem - tyi * txc) * TX, y0 = tyi * TY;
    unsigned char* st = stage(s);
    fence_proxy_async();
    mbar_arrive_expect_tx(&bar[s], LY::tx);
    tma_load_4d(st, &mx, &bar[s], 2 * (x0 - 1), y0 - 1, zz, 2 * j);
    tma_load_4d(st + kOffE, &mx, &bar[s], 2 * (x0 - 1), y0 - 1, zz, 2 * j + 1);
    tma_load_4d(st + kOffB1, &mb, &bar[s], 2 * x0, y0, zz, 2 * j);
    tma_load_4d(st + kOffB2, &mb, &bar[s], 2 * x0, y0, zz, 2 * j + 1);
    if constexpr (DIM == 3) {
      const int zm = zz == 0 ? nz - 1 : zz - 1, zp = zz + 1 == nz ? 0 : zz + 1;
      tma_load_4d(st + kOffZN, &mxc, &bar[s], 2 * x0, y0, zm, 2 * j);
      tma_load_4d(st + kOffZN + kBBytes, &mxc, &bar[s], 2 * x0, y0, zp, 2 * j);
      tma_load_4d(st + kOffZN + 2 * kBBytes, &mxc, &bar[s], 2 * x0, y0, zm, 2 * j + 1);
      tma_load_4d(st + kOffZN + 3 * kBBytes, &mxc, &bar[s], 2 * x0, y0, zp, 2 * j + 1);
    }
  };
  if (t == 0) {
    tma_prefetch_map(&mx);
    tma_prefetch_map(&mb);
    if constexpr (DIM == 3) tma_prefetch_map(&mxc);
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
    const int zz = tile / tpl, rem = tile - zz * tpl, tyi = rem / txc, x0 = (rem - tyi * txc) * TX, y0 = tyi * TY;
    if (!mbar_wait(&bar[s], (k >> 1) & 1)) s_fail = 1;
    unsigned char* st = stage(s);
    double2* rz = reinterpret_cast<double2*>(st);
    double2* re = reinterpret_cast<double2*>(st + kOffE);
    const double2 b1v = reinterpret_cast<const double2*>(st + kOffB1)[t];
    const double2 b2v = reinterpret_cast<const double2*>(st + kOffB2)[t];
    double2 zmv, zpv, emv, epv;
    if constexpr (DIM == 3) {
      const double2* zn = reinterpret_cast<const double2*>(st + kOffZN);
      zmv = zn[t];
      zpv = zn[t + TX * TY];
      emv = zn[t + 2 * TX * TY];
      epv = zn[t + 3 * TX * TY];
    }
    if (x0 == 0 || y0 == 0 || x0 + TX >= nx || y0 + TY >= ny) {
      // cells beyond the grid in x or y: the periodic image (TMA filled them with zeros)
      for (int i = t; i < kHalo; i += blockDim.x) {
        const int ry = i / HX, rx = i - ry * HX;
        int gxx = x0 - 1 + rx, gyy = y0 - 1 + ry;
        if (gxx >= 0 && gxx < nx && gyy >= 0 && gyy < ny) continue;
        gxx = gxx < 0 ? gxx + nx : gxx % nx;
        gyy = gyy < 0 ? gyy + ny : gyy % ny;
        const long long q = zz * plane + (long long)gyy * nx + gxx;
        rz[i] = x[o + q];
        re[i] = x[o + pts + q];
      }
    }
    __syncthreads();
    if (s_fail) break;
    for (int i = t; i < kHalo; i += blockDim.x) {
      sz[i] = pdf_pack(pdf_split(rz[i]));
      se[i] = pdf_pack(pdf_split(re[i]));
    }
    __syncthreads();
    // the stage is consumed: refill it two tiles ahead
    if (t == 0 && tile + kStages * (int)gridDim.x < ntiles) issue(tile + kStages * gridDim.x, s);
    const int xx = x0 + tx, yy = y0 + ty;
    if (xx >= nx || yy >= ny) continue;
    const long long pc = zz * plane + (long long)yy * nx + xx;
    const int cc = (ty + 1) * HX + tx + 1;
    // neighbours of the point per dimension: (-, +)
    PDF zn_[DIM][2], en_[DIM][2];
    zn_[0][0] = pdf_unpack(sz[cc - 1]);
    zn_[0][1] = pdf_unpack(sz[cc + 1]);
    zn_[1][0] = pdf_unpack(sz[cc - HX]);
    zn_[1][1] = pdf_unpack(sz[cc + HX]);
    en_[0][0] = pdf_unpack(se[cc - 1]);
    en_[0][1] = pdf_unpack(se[cc + 1]);
    en_[1][0] = pdf_unpack(se[cc - HX]);
    en_[1][1] = pdf_unpack(se[cc + HX]);
    if constexpr (DIM == 3) {
      zn_[2][0] = pdf_split(zmv);
      zn_[2][1] = pdf_split(zpv);
      en_[2][0] = pdf_split(emv);
      en_[2][1] = pdf_split(epv);
    }
    if (c.jd != nullptr) ma = lane_c(a_at(c, j, pc), -1.f, -1.f);
    float2 f1, l1, f2, l2;
    resid_point<DIM>(q, ma, pdf_split(b1v), pdf_split(b2v), pdf_unpack(sz[cc]), pdf_unpack(se[cc]), zn_, en_, f1, l1,
                     f2, l2);
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
  const unsigned long long d4[4] = {dims[0], dims[1], dims[2], 1};
  const unsigned long long s4[3] = {strides[0], strides[1], strides[1] * dims[2]};
  const unsigned b4[4] = {box[0], box[1], box[2], 1};
  return tma_encode_f64_4d(map, base, d4, s4, b4, err);
}

bool tma_encode_f64_4d(CUtensorMap* map, const void* base, const unsigned long long dims[4],
                       const unsigned long long strides[3], const unsigned box[4], const char** err) {
  return tma_encode_4d(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, base, dims, strides, box, err);
}

bool tma_encode_4d(CUtensorMap* map, CUtensorMapDataType type, const void* base, const unsigned long long dims[4],
                   const unsigned long long strides[3], const unsigned box[4], const char** err) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn(err);
  if (!fn) return false;
  const cuuint64_t gd[4] = {dims[0], dims[1], dims[2], dims[3]};
  const cuuint64_t gs[3] = {strides[0], strides[1], strides[2]};
  const cuuint32_t bd[4] = {box[0], box[1], box[2], box[3]};
  const cuuint32_t es[4] = {1, 1, 1, 1};
  const CUresult r = fn(map, type, 4, const_cast<void*>(base), gd, gs, bd, es,
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
  if (cudaMemcpyFromSymbol(&v, g_timeouts, sizeof(v)) != cudaSuccess) v = 0;
  return v + stream3d_timeouts();
}

namespace {
template <int DIM>
bool launch_resid(const double2* b, const double2* x, float2* r32, double2* r64, double* partials, const OpCoef& c,
                  cudaStream_t s, const char** err) {
  const unsigned long long nz = DIM == 3 ? (unsigned long long)c.nz : 1ull;
  const unsigned long long dims[4] = {2ull * c.nx, (unsigned long long)c.ny, nz, 2ull * c.J};
  const unsigned long long row = 16ull * c.nx, pl = row * c.ny;
  const unsigned long long strides[3] = {row, pl, pl * nz};
  const unsigned bx[4] = {2 * HX, HY, 1, 1}, bb[4] = {2 * TX, TY, 1, 1};
  CUtensorMap mx, mxc, mb;
  if (!tma_encode_f64_4d(&mx, x, dims, strides, bx, err) || !tma_encode_f64_4d(&mxc, x, dims, strides, bb, err) ||
      !tma_encode_f64_4d(&mb, b, dims, strides, bb, err))
    return false;
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(k_resid_tma<DIM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)resid_smem<DIM>()) != cudaSuccess) {
      if (err) *err = "cannot raise the shared memory of the residual kernel";
      return false;
    }
    attr = true;
  }
  ProfScope ps_(KID_RESID_REFINE, s);
  k_resid_tma<DIM><<<dim3(kDotBlocks, c.J), 256, resid_smem<DIM>(), s>>>(mx, mxc, mb, x, r32, r64,
                                                                        reinterpret_cast<double2*>(partials), c);
  return true;
}
}  // namespace

// x, b: block vectors [J][2][nz][ny][nx] of complex doubles; one grid (no batch).
bool launch_residual_refine_tma(const double2* b, const double2* x, float2* r32, double2* r64, double* partials,
                                const OpCoef& c, cudaStream_t s, const char** err) {
  return c.dim == 3 ? launch_resid<3>(b, x, r32, r64, partials, c, s, err)
                    : launch_resid<2>(b, x, r32, r64, partials, c, s, err);
}

}  // namespace apfc
