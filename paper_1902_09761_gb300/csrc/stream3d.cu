// z-streaming stencil passes of the APFC step on 3D grids (arXiv:1902.09761, Sec. II):
// the block operator A_j of Eq. linear_system2 (M = I), the steps of the preconditioner of
// Eq. preconditioner (f = beta2 - kt G beta1, the Chebyshev applications of the diffusion
// solves, step 4), the outer residual r = b - A x and zeta = G eta, each one kernel that
// streams (x, y) tiles through chunks of z-planes.  The Krylov inner products of A P^{-1}
// come out of the A passes.
#include <algorithm>
#include <cstring>

#include "acc.cuh"
#include "apfc_internal.cuh"
#include "tma.cuh"

namespace apfc {

namespace {

// ---------------------------------------------------------------------------
// A block owns an (x, y) tile and streams through a chunk of kZChunk planes; the
// current plane of every stencil input sits in shared memory with a one-point halo
// (a ring of kZBuf planes, fetched kZAhead ahead with cp.async), the own-column
// z-neighbours in registers.  Each input value is read from HBM about once (the
// tile halo comes from L2).
// ---------------------------------------------------------------------------
constexpr int kZChunk = 64;
constexpr int kZBuf = 6, kZAhead = 4;  // plane buffers and planes fetched ahead
static_assert(kZBuf - kZAhead >= 2, "the passes rely on two spare plane buffers instead of a second barrier");
constexpr int kTX = 32, kHX = kTX + 2;
// FP64 passes: 32 x 8 tiles, one point per thread (k_stream3d).  FP32 passes: 64 x 8
// tiles, two adjacent points per thread (k_stream3d_pair).
template <typename T>
__host__ __device__ constexpr int tile_rows3() { return 8; }
template <typename T>
__host__ __device__ constexpr int tile_cols3() { return sizeof(T) == 4 ? 64 : 32; }

template <typename T>
struct N7 {
  cplx<T> c, xm, xp, ym, yp, zm, zp;
};

// Operator coefficients of amplitude j in the arithmetic precision T, formed once per
// block (converting the FP64 coefficients at every point kept the FP32 passes bound by
// the FP64 pipe).
template <typename T>
struct Coef7 {
  T c0, ih2[3], kh[3], kt, a, it, sD, mu, im, c1, c2;
};
template <typename T>
__device__ __forceinline__ Coef7<T> coef7(const OpCoef& c, int j) {
  Coef7<T> q;
  q.c0 = (T)c.c0;
  for (int d = 0; d < 3; ++d) {
    q.ih2[d] = (T)c.ih2[d];
    q.kh[d] = (T)c.kh[j][d];
  }
  q.kt = (T)c.kt[j];
  q.a = (T)c.a[j];
  q.it = (T)c.inv_theta[j];
  q.sD = (T)c.sD[j];
  q.mu = (T)c.mu[j];
  q.im = (T)c.inv_mu[j];
  q.c1 = q.c2 = (T)0;
  return q;
}
// (2,2) block at point p: a_j plus the Jacobian diagonal of a Picard iteration
template <typename T>
__device__ __forceinline__ T a7(const Coef7<T>& q, const OpCoef& c, int j, long long p) {
  if (c.jd == nullptr) return q.a;
  if constexpr (sizeof(T) == 4) {
    if (c.jd32 != nullptr) return q.a + c.jd32[(long long)j * c.pts + p].x;
  }
  return q.a + (T)c.jd[(long long)j * c.pts + p];
}

template <typename T>
__device__ __forceinline__ cplx<T> lap7(const N7<T>& n, const Coef7<T>& q) {
  const T c0 = q.c0, ix = q.ih2[0], iy = q.ih2[1], iz = q.ih2[2];
  return mkc<T>(c0 * n.c.x + ix * (n.xm.x + n.xp.x) + iy * (n.ym.x + n.yp.x) + iz * (n.zm.x + n.zp.x),
                c0 * n.c.y + ix * (n.xm.y + n.xp.y) + iy * (n.ym.y + n.yp.y) + iz * (n.zm.y + n.zp.y));
}
template <typename T>
__device__ __forceinline__ cplx<T> G7(const N7<T>& n, const Coef7<T>& q) {
  const cplx<T> L = lap7(n, q);
  const T kx = q.kh[0], ky = q.kh[1], kz = q.kh[2];
  const T ar = kx * (n.xp.x - n.xm.x) + ky * (n.yp.x - n.ym.x) + kz * (n.zp.x - n.zm.x);
  const T ai = kx * (n.xp.y - n.xm.y) + ky * (n.yp.y - n.ym.y) + kz * (n.zp.y - n.zm.y);
  return mkc<T>(L.x - ai, L.y + ar);
}
template <typename T>
__device__ __forceinline__ cplx<T> D7(const N7<T>& n, const Coef7<T>& q) {
  const cplx<T> L = lap7(n, q);
  return mkc<T>(q.sD * n.c.x - q.mu * L.x, q.sD * n.c.y - q.mu * L.y);
}

__device__ __forceinline__ int wrapi(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

// OP: NS stencil inputs src(k, j) (plane-major [nz][ny][nx] per amplitude) and
// apply(j, p, nbh[NS]) doing the pointwise work and the stores.
template <typename T>
__device__ __forceinline__ void cp_async_elem(cplx<T>* dst, const cplx<T>* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  if constexpr (sizeof(cplx<T>) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src));
  else
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src));
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src));
}

template <typename T, class OP>
__global__ void __launch_bounds__(256) k_stream3d(OpCoef c, OP op, const KScal* act) {
  constexpr int NS = OP::NS;
  static_assert(OP::MINB >= 1 && OP::MINB <= 8, "blocks per SM of the two-point kernel");
  constexpr int kTY = tile_rows3<T>(), kHY = kTY + 2, RPT = kTY / 8;
  // plane buffers: z (stencil), z+1 (its z+ neighbour), z+2 .. z+kZAhead (in flight)
  __shared__ cplx<T> tile[NS][kZBuf][kHY][kHX];
  const int nchunk = (c.nz + kZChunk - 1) / kZChunk;
  const int j = (int)(blockIdx.z / (unsigned)nchunk);
  if (act != nullptr && act[j].active == 0) return;
  const int chunk = (int)(blockIdx.z - (unsigned)j * nchunk);
  if (c.prof != nullptr && blockIdx.x == 0 && blockIdx.y == 0 && chunk == 0 && threadIdx.x == 0)
    atomicAdd(c.prof + op.kid, op.bytes);
  Coef7<T> q = coef7<T>(c, j);
  op.coef(q, j);
  Acc<T> acc[OP::ND > 0 ? OP::ND : 1];
#pragma unroll
  for (int d = 0; d < (OP::ND > 0 ? OP::ND : 1); ++d) acc[d].zero();
  // each thread owns column tx of rows ty (and ty + 8 in a 16-row tile)
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY;
  const int x = x0 + tx;
  const long long plane = (long long)c.nx * c.ny;
  const int z0 = chunk * kZChunk, z1 = min(c.nz, z0 + kZChunk);
  const cplx<T>* src[NS];
#pragma unroll
  for (int k = 0; k < NS; ++k) src[k] = op.src(k, j);
  // each thread copies the same (at most three) halo-tile elements of every plane
  long long qoff[3];
  int hoff[3];
  int ne = 0;
  for (int e = threadIdx.x; e < kHX * kHY; e += 256, ++ne) {
    const int hy = e / kHX, hx = e - hy * kHX;
    qoff[ne] = (long long)wrapi(y0 - 1 + hy, c.ny) * c.nx + wrapi(x0 - 1 + hx, c.nx);
    hoff[ne] = hy * kHX + hx;
  }
  auto issue_tile = [&](int buf, int z) {
    const long long zo = (long long)wrapi(z, c.nz) * plane;
    for (int i = 0; i < ne; ++i)
#pragma unroll
      for (int k = 0; k < NS; ++k) cp_async_elem<T>(&tile[k][buf][0][0] + hoff[i], src[k] + zo + qoff[i]);
    asm volatile("cp.async.commit_group;\n" ::);
  };
  bool inside[RPT];
  long long pxy[RPT];
  cplx<T> zm[RPT][NS];
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    const int y = y0 + ty + 8 * r;
    inside[r] = x < c.nx && y < c.ny;
    pxy[r] = (long long)(inside[r] ? y : 0) * c.nx + (inside[r] ? x : 0);
#pragma unroll
    for (int k = 0; k < NS; ++k) zm[r][k] = src[k][(long long)wrapi(z0 - 1, c.nz) * plane + pxy[r]];
  }
#pragma unroll
  for (int a = 0; a < kZAhead; ++a) issue_tile(a, z0 + a);
  int cb = 0;
  for (int z = z0; z < z1; ++z) {
    const int nb = cb + 1 == kZBuf ? 0 : cb + 1;
    int fb = cb + kZAhead;
    if (fb >= kZBuf) fb -= kZBuf;
    issue_tile(fb, z + kZAhead);  // into a buffer no plane in use occupies
    asm volatile("cp.async.wait_group %0;\n" ::"n"(kZAhead - 1));  // planes z and z+1 have landed
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      if (inside[r]) {
        const int ly = ty + 8 * r + 1;
        N7<T> n[NS];
#pragma unroll
        for (int k = 0; k < NS; ++k) {
          n[k].c = tile[k][cb][ly][tx + 1];
          n[k].xm = tile[k][cb][ly][tx];
          n[k].xp = tile[k][cb][ly][tx + 2];
          n[k].ym = tile[k][cb][ly - 1][tx + 1];
          n[k].yp = tile[k][cb][ly + 1][tx + 1];
          n[k].zm = zm[r][k];
          n[k].zp = tile[k][nb][ly][tx + 1];
          zm[r][k] = n[k].c;
        }
        const long long pz = (long long)z * plane + pxy[r];
        cplx<T> pv[OP::NQ > 0 ? OP::NQ : 1];
#pragma unroll
        for (int k = 0; k < OP::NQ; ++k) {
          const cplx<T>* qs = op.qsrc(k, j);
          pv[k] = qs != nullptr ? qs[pz] : cplx<T>{};
        }
        op.apply(j, pz, n, c, q, acc, pv);
      }
    }
#pragma unroll
    for (int d = 0; d < OP::ND; ++d) acc[d].flush();
    // no barrier here: the ring keeps kZBuf - kZAhead = 2 spare planes, so the buffer a thread
    // refills at plane z + 1 was last read at plane z - 1, which every thread finished before
    // the barrier of plane z that this thread has passed
    cb = nb;
  }
  asm volatile("cp.async.wait_group 0;\n" ::);
  if constexpr (OP::ND > 0) {
    const long long npart = (long long)gridDim.x * gridDim.y * nchunk;
    const long long bid = ((long long)chunk * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
#pragma unroll
    for (int d = 0; d < OP::ND; ++d) {
      block_reduce<T>(acc[d]);
      if (threadIdx.x == 0) acc[d].store(op.partials, (long long)(j * kDotSlots + d) * npart + bid);
    }
  }
}

// Pass interface of k_stream3d / k_stream3d_pair:
//   NS stencil inputs src(k, j) (read with a one-point halo), NQ pointwise inputs
//   qsrc(k, j) (their values at p arrive in pv[k]; a null qsrc is not read), ND inner
//   products accumulated in acc, MINB blocks per SM for the two-point kernel, and
//   apply(j, p, nbh[NS], c, q, acc, pv) doing the pointwise work and the stores.

// y = A x (both parts of x are stencil inputs); ND inner products of y accumulated on
// the way: ND = 1 (du, y), ND = 2 (y, du) and (y, y), with (u, v) = sum conj(u) v
template <typename T, int ND_ = 0>
struct OpA3 {
  static constexpr int NS = 2, ND = ND_, NQ = ND_ > 0 ? 2 : 0, MINB = ND_ > 0 ? 2 : 3;
  const cplx<T>* x;
  cplx<T>* y;
  long long pts;
  int kid;
  unsigned long long bytes;
  const cplx<T>* du = nullptr;
  void* partials = nullptr;
  template <typename Q>
  __device__ void coef(Q&, int) const {}
  __host__ __device__ const cplx<T>* src(int k, int j) const { return x + (2LL * j + k) * pts; }
  __host__ __device__ const cplx<T>* qsrc(int k, int j) const { return du + (2LL * j + k) * pts; }
  __device__ void apply(int j, long long p, const N7<T> (&n)[2], const OpCoef& c, const Coef7<T>& q, Acc<T>* acc,
                        const cplx<T>* pv) const {
    const cplx<T> gz = G7(n[0], q), ge = G7(n[1], q);
    const T kt = q.kt, a = a7(q, c, j, p);
    const long long o = 2LL * j * pts;
    const cplx<T> y1 = mkc<T>(n[0].c.x - ge.x, n[0].c.y - ge.y);
    const cplx<T> y2 = mkc<T>(kt * gz.x + a * n[1].c.x, kt * gz.y + a * n[1].c.y);
    y[o + p] = y1;
    y[o + pts + p] = y2;
    // plain FP32 runs, folded into the compensated sums once per plane (Acc::flush)
    if constexpr (ND == 1) {
      acc[0].add_run(pv[0], y1);
      acc[0].add_run(pv[1], y2);
    } else if constexpr (ND == 2) {
      acc[0].add_run(y1, pv[0]);
      acc[0].add_run(y2, pv[1]);
      acc[1].add_run(y1, y1);
      acc[1].add_run(y2, y2);
    }
  }
};

// r = b - A x, rhat = r
template <typename T>
struct OpRes3 {
  static constexpr int NS = 2, ND = 0, NQ = 2, MINB = 2;
  const cplx<T>* x;
  const cplx<T>* b;
  cplx<T>* r;
  cplx<T>* rhat;
  long long pts;
  int kid;
  unsigned long long bytes;
  template <typename Q>
  __device__ void coef(Q&, int) const {}
  __host__ __device__ const cplx<T>* src(int k, int j) const { return x + (2LL * j + k) * pts; }
  __host__ __device__ const cplx<T>* qsrc(int k, int j) const { return b + (2LL * j + k) * pts; }
  __device__ void apply(int j, long long p, const N7<T> (&n)[2], const OpCoef& c, const Coef7<T>& q, Acc<T>*,
                        const cplx<T>* pv) const {
    const cplx<T> gz = G7(n[0], q), ge = G7(n[1], q);
    const T kt = q.kt, a = a7(q, c, j, p);
    const long long o = 2LL * j * pts;
    const cplx<T> b1 = pv[0], b2 = pv[1];
    const cplx<T> r1 = mkc<T>(b1.x - (n[0].c.x - ge.x), b1.y - (n[0].c.y - ge.y));
    const cplx<T> r2 = mkc<T>(b2.x - (kt * gz.x + a * n[1].c.x), b2.y - (kt * gz.y + a * n[1].c.y));
    r[o + p] = r1;
    r[o + pts + p] = r2;
    rhat[o + p] = r1;
    rhat[o + pts + p] = r2;
  }
};

// f = beta2 - kt G beta1
template <typename T>
struct OpPcRhs3 {
  static constexpr int NS = 1, ND = 0, NQ = 1, MINB = 4;
  const cplx<T>* beta;
  FieldRef<T> f;
  long long pts;
  int kid;
  unsigned long long bytes;
  template <typename Q>
  __device__ void coef(Q&, int) const {}
  __host__ __device__ const cplx<T>* src(int, int j) const { return beta + 2LL * j * pts; }
  __host__ __device__ const cplx<T>* qsrc(int, int j) const { return beta + (2LL * j + 1) * pts; }
  __device__ void apply(int j, long long p, const N7<T> (&n)[1], const OpCoef& c, const Coef7<T>& q, Acc<T>*,
                        const cplx<T>* pv) const {
    const cplx<T> g = G7(n[0], q);
    const cplx<T> b2 = pv[0];
    const T kt = q.kt;
    f.at(j)[p] = mkc<T>(b2.x - kt * g.x, b2.y - kt * g.y);
  }
};

// step 4 of P^{-1} at point p: chi1 = beta1 + (beta2' - sD chi2) / mu
template <typename T>
__device__ __forceinline__ void finish_pc(const PcFin<T>& f, int j, long long p, cplx<T> b1, cplx<T> bp, cplx<T> x2,
                                          const Coef7<T>& q) {
  f.chi1.at(j)[p] = mkc<T>(b1.x + q.im * (bp.x - q.sD * x2.x), b1.y + q.im * (bp.y - q.sD * x2.y));
}

// first Chebyshev application (see k_cheb_first); pointwise input: beta1 with fin
template <typename T>
struct OpChebFirst3 {
  static constexpr int NS = 1, ND = 0, NQ = 1, MINB = 3;
  CFieldRef<T> f;
  FieldRef<T> X, R, Dn;
  ChebStep w;
  int last;
  PcFin<T> fin;  // fin.chi1.p != nullptr: also chi1 = beta1 + (beta2' - sD chi2) / mu
  int kid;
  unsigned long long bytes;
  template <typename Q>
  __device__ void coef(Q& q, int j) const {
    q.c1 = (T)w.c1[j];
    q.c2 = (T)w.c2[j];
  }
  __host__ __device__ const cplx<T>* src(int, int j) const { return f.at(j); }
  __host__ __device__ const cplx<T>* qsrc(int, int j) const { return fin.chi1.p != nullptr ? fin.b1.at(j) : nullptr; }
  __device__ void apply(int j, long long p, const N7<T> (&n)[1], const OpCoef& c, const Coef7<T>& q, Acc<T>*,
                        const cplx<T>* pv) const {
    const T it = q.it;
    const cplx<T> Df = D7(n[0], q);
    const cplx<T> d0 = mkc<T>(it * n[0].c.x, it * n[0].c.y);
    const cplx<T> r1 = mkc<T>(n[0].c.x - it * Df.x, n[0].c.y - it * Df.y);
    const T c1 = q.c1, c2 = q.c2;
    const cplx<T> d1 = mkc<T>(c1 * d0.x + c2 * r1.x, c1 * d0.y + c2 * r1.y);
    if (last) {
      const cplx<T> x2 = mkc<T>(d0.x + d1.x, d0.y + d1.y);
      X.at(j)[p] = x2;
      // the source of the second solve is beta2'
      if (fin.chi1.p != nullptr) finish_pc(fin, j, p, pv[0], n[0].c, x2, q);
    } else {
      X.at(j)[p] = d0;
      R.at(j)[p] = r1;
      Dn.at(j)[p] = d1;
    }
  }
};

// later Chebyshev application (see k_cheb_sweep); pointwise inputs X, R and, with fin,
// beta1 and beta2'
template <typename T>
struct OpChebSweep3 {
  static constexpr int NS = 1, ND = 0, NQ = 4, MINB = 3;
  CFieldRef<T> Dd;
  FieldRef<T> X, R, Dn;
  ChebStep w;
  int last;
  PcFin<T> fin;  // fin.chi1.p != nullptr: also chi1 = beta1 + (beta2' - sD chi2) / mu
  int kid;
  unsigned long long bytes;
  template <typename Q>
  __device__ void coef(Q& q, int j) const {
    q.c1 = (T)w.c1[j];
    q.c2 = (T)w.c2[j];
  }
  __host__ __device__ const cplx<T>* src(int, int j) const { return Dd.at(j); }
  __host__ __device__ const cplx<T>* qsrc(int k, int j) const {
    if (k < 2) return k == 0 ? X.at(j) : R.at(j);
    if (fin.chi1.p == nullptr) return nullptr;
    return k == 2 ? fin.b1.at(j) : fin.b2p.at(j);
  }
  __device__ void apply(int j, long long p, const N7<T> (&n)[1], const OpCoef& c, const Coef7<T>& q, Acc<T>*,
                        const cplx<T>* pv) const {
    const cplx<T> DD = D7(n[0], q);
    const cplx<T> d = n[0].c;
    const cplx<T> x = pv[0], r = pv[1];
    const cplx<T> xn = mkc<T>(x.x + d.x, x.y + d.y);
    const cplx<T> rn = mkc<T>(r.x - DD.x, r.y - DD.y);
    const T c1 = q.c1, c2 = q.c2;
    const cplx<T> dn = mkc<T>(c1 * d.x + c2 * rn.x, c1 * d.y + c2 * rn.y);
    if (last) {
      const cplx<T> x2 = mkc<T>(xn.x + dn.x, xn.y + dn.y);
      X.at(j)[p] = x2;
      if (fin.chi1.p != nullptr) finish_pc(fin, j, p, pv[2], pv[3], x2, q);
    } else {
      X.at(j)[p] = xn;
      R.at(j)[p] = rn;
      Dn.at(j)[p] = dn;
    }
  }
};

// zeta-part of the state = G_h (eta-part), FP64
struct OpZeta3 {
  static constexpr int NS = 1, ND = 0, NQ = 0, MINB = 3;
  double2* x;
  long long pts;
  int kid;
  unsigned long long bytes;
  template <typename Q>
  __device__ void coef(Q&, int) const {}
  __host__ __device__ const double2* src(int, int j) const { return x + (2LL * j + 1) * pts; }
  __host__ __device__ const double2* qsrc(int, int) const { return nullptr; }
  __device__ void apply(int j, long long p, const N7<double> (&n)[1], const OpCoef& c, const Coef7<double>& q,
                        Acc<double>*, const double2*) const {
    x[2LL * j * pts + p] = G7(n[0], q);
  }
};

// FP32 variant of k_stream3d: each thread owns two adjacent points (x, x+1) of a row of a
// 64 x 8 tile.  The plane tile (one-point halo) sits at local column x - x0 + 2, so the
// pair and its y- and z-neighbour pairs are 16-byte shared-memory loads: half the
// shared-memory instructions of one point per thread, the pipe that limited the
// single-point kernel (short-scoreboard stalls).
constexpr int kPX = 64, kPY = 8, kPW = kPX + 4;  // tile columns, rows, row stride (2 + 64 + 2)
template <class OP>
__global__ void __launch_bounds__(256, OP::MINB) k_stream3d_pair(OpCoef c, OP op, const KScal* act) {
  using T = float;
  constexpr int NS = OP::NS;
  constexpr int kHYp = kPY + 2, kNE = (kPX + 2) * kHYp;  // elements fetched per plane
  __shared__ __align__(16) float2 tile[NS][kZBuf][kHYp][kPW];
  // pointwise inputs (up to two) ride on the same copy groups: each thread fetches its own
  // pair of every plane kZAhead planes ahead into a ring of kZAhead + 1 buffers
  constexpr bool QS = OP::NQ > 0 && OP::NQ <= 2;
  constexpr int NQS = QS ? OP::NQ : 1, kQB = QS ? kZAhead + 1 : 1;
  __shared__ __align__(16) float2 qt[NQS][kQB][kPY][kPX];
  const int nchunk = (c.nz + kZChunk - 1) / kZChunk;
  const int j = (int)(blockIdx.z / (unsigned)nchunk);
  if (act != nullptr && act[j].active == 0) return;
  const int chunk = (int)(blockIdx.z - (unsigned)j * nchunk);
  if (c.prof != nullptr && blockIdx.x == 0 && blockIdx.y == 0 && chunk == 0 && threadIdx.x == 0)
    atomicAdd(c.prof + op.kid, op.bytes);
  Coef7<T> q = coef7<T>(c, j);
  op.coef(q, j);
  Acc<T> acc[OP::ND > 0 ? OP::ND : 1];
#pragma unroll
  for (int d = 0; d < (OP::ND > 0 ? OP::ND : 1); ++d) acc[d].zero();
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int x0 = blockIdx.x * kPX, y0 = blockIdx.y * kPY;
  const int xa = x0 + 2 * tx, y = y0 + ty;
  const long long plane = (long long)c.nx * c.ny;
  const int z0 = chunk * kZChunk, z1 = min(c.nz, z0 + kZChunk);
  const float2* src[NS];
#pragma unroll
  for (int k = 0; k < NS; ++k) src[k] = op.src(k, j);
  // each thread copies the same (at most three) halo-tile elements of every plane
  long long qoff[3];
  int hoff[3];
  int ne = 0;
  for (int e = threadIdx.x; e < kNE; e += 256, ++ne) {
    const int hy = e / (kPX + 2), li = e - hy * (kPX + 2);
    qoff[ne] = (long long)wrapi(y0 - 1 + hy, c.ny) * c.nx + wrapi(x0 - 1 + li, c.nx);
    hoff[ne] = hy * kPW + li + 1;
  }
  const bool in0 = xa < c.nx && y < c.ny, in1 = xa + 1 < c.nx && y < c.ny;
  const long long p0 = (long long)(in0 ? y : 0) * c.nx + (in0 ? xa : 0);
  const long long p1 = in1 ? p0 + 1 : p0;
  const float2* qs[OP::NQ > 0 ? OP::NQ : 1];
#pragma unroll
  for (int k = 0; k < OP::NQ; ++k) qs[k] = op.qsrc(k, j);
  auto issue_tile = [&](int buf, int qb, int z) {
    const long long zo = (long long)wrapi(z, c.nz) * plane;
    for (int i = 0; i < ne; ++i)
#pragma unroll
      for (int k = 0; k < NS; ++k) cp_async_elem<T>(&tile[k][buf][0][0] + hoff[i], src[k] + zo + qoff[i]);
    if constexpr (QS) {
      if (z < z1 && in0) {
#pragma unroll
        for (int k = 0; k < NQS; ++k) {
          if (qs[k] == nullptr) continue;
          const float2* g = qs[k] + zo + p0;
          float2* d = &qt[k][qb][ty][2 * tx];
          if (in1 && (reinterpret_cast<unsigned long long>(g) & 15ull) == 0) {
            cp_async16(d, g);
          } else {
            cp_async_elem<T>(d, g);
            if (in1) cp_async_elem<T>(d + 1, g + 1);
          }
        }
      }
    }
    asm volatile("cp.async.commit_group;\n" ::);
  };
  float2 zm0[NS], zm1[NS];
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    const long long zo = (long long)wrapi(z0 - 1, c.nz) * plane;
    zm0[k] = src[k][zo + p0];
    zm1[k] = src[k][zo + p1];
  }
#pragma unroll
  for (int a = 0; a < kZAhead; ++a) issue_tile(a, a, z0 + a);
  const int lc = 2 * tx + 2;  // local column of xa: even, so the pair is 16-byte aligned
  int cb = 0, qc = 0;
  for (int z = z0; z < z1; ++z) {
    const int nb = cb + 1 == kZBuf ? 0 : cb + 1;
    int fb = cb + kZAhead;
    if (fb >= kZBuf) fb -= kZBuf;
    const int qf = qc == 0 ? kQB - 1 : qc - 1;  // (qc + kZAhead) mod kQB
    issue_tile(fb, QS ? qf : 0, z + kZAhead);  // into buffers no plane in use occupies
    asm volatile("cp.async.wait_group %0;\n" ::"n"(kZAhead - 1));  // planes z and z+1 have landed
    __syncthreads();
    if (in0) {
      N7<T> n0[NS], n1[NS];
#pragma unroll
      for (int k = 0; k < NS; ++k) {
        const float4 cc = *reinterpret_cast<const float4*>(&tile[k][cb][ty + 1][lc]);
        const float4 ym = *reinterpret_cast<const float4*>(&tile[k][cb][ty][lc]);
        const float4 yp = *reinterpret_cast<const float4*>(&tile[k][cb][ty + 2][lc]);
        const float4 zp = *reinterpret_cast<const float4*>(&tile[k][nb][ty + 1][lc]);
        const float2 xm = tile[k][cb][ty + 1][lc - 1], xp = tile[k][cb][ty + 1][lc + 2];
        n0[k].c = make_float2(cc.x, cc.y);
        n0[k].xm = xm;
        n0[k].xp = make_float2(cc.z, cc.w);
        n0[k].ym = make_float2(ym.x, ym.y);
        n0[k].yp = make_float2(yp.x, yp.y);
        n0[k].zm = zm0[k];
        n0[k].zp = make_float2(zp.x, zp.y);
        n1[k].c = make_float2(cc.z, cc.w);
        n1[k].xm = make_float2(cc.x, cc.y);
        n1[k].xp = xp;
        n1[k].ym = make_float2(ym.z, ym.w);
        n1[k].yp = make_float2(yp.z, yp.w);
        n1[k].zm = zm1[k];
        n1[k].zp = make_float2(zp.z, zp.w);
        zm0[k] = n0[k].c;
        zm1[k] = n1[k].c;
      }
      const long long zo = (long long)z * plane;
      float2 pv0[OP::NQ > 0 ? OP::NQ : 1], pv1[OP::NQ > 0 ? OP::NQ : 1];
#pragma unroll
      for (int k = 0; k < OP::NQ; ++k) {
        if constexpr (QS) {
          const float4 v = *reinterpret_cast<const float4*>(&qt[k][qc][ty][2 * tx]);
          pv0[k] = make_float2(v.x, v.y);
          pv1[k] = make_float2(v.z, v.w);
        } else {
          pv0[k] = qs[k] != nullptr ? qs[k][zo + p0] : make_float2(0.f, 0.f);
          pv1[k] = qs[k] != nullptr ? qs[k][zo + p1] : make_float2(0.f, 0.f);
        }
      }
      op.apply(j, zo + p0, n0, c, q, acc, pv0);
      if (in1) op.apply(j, zo + p1, n1, c, q, acc, pv1);
#pragma unroll
      for (int d = 0; d < OP::ND; ++d) acc[d].flush();
    }
    // no barrier here: the ring keeps kZBuf - kZAhead = 2 spare planes, so the buffer a thread
    // refills at plane z + 1 was last read at plane z - 1, which every thread finished before
    // the barrier of plane z that this thread has passed
    cb = nb;
    qc = qc + 1 == kQB ? 0 : qc + 1;
  }
  asm volatile("cp.async.wait_group 0;\n" ::);
  if constexpr (OP::ND > 0) {
    const long long npart = (long long)gridDim.x * gridDim.y * nchunk;
    const long long bid = ((long long)chunk * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
#pragma unroll
    for (int d = 0; d < OP::ND; ++d) {
      block_reduce<T>(acc[d]);
      if (threadIdx.x == 0) acc[d].store(op.partials, (long long)(j * kDotSlots + d) * npart + bid);
    }
  }
}

// ---------------------------------------------------------------------------
// The FP32 passes with every plane moved by the tensor memory accelerator (grids with
// nx % 64 == 0 and ny % 8 == 0): the same 64 x 8 tiles, two points per thread and
// 64-plane z-chunks as k_stream3d_pair.  Per plane, one thread issues for every stencil
// input one box of the tile with its one-point halo (columns x0 - 2 .. x0 + 65, rows
// y0 - 1 .. y0 + 8) and for every pointwise input one box of the tile, kTAhead planes
// ahead into a ring of kTBuf planes, completing on that plane's mbarrier.  Periodic
// x and y: TMA fills halo cells beyond the grid with zeros, so tiles at the boundary
// also load the wrapped column (x = nx - 2 .. nx - 1, or 0 .. 1) or row (y = ny - 1,
// or 0) as side boxes, and the stencil takes those neighbours from there.  The z
// coordinate of every box is wrapped on issue.
// ---------------------------------------------------------------------------
constexpr int kTBuf = 4, kTAhead = 2;                 // plane buffers, planes in flight
constexpr int kTQB = kTAhead + 2;                     // pointwise-input buffers
constexpr int kMainF = 688;                           // 10 x 68 float2 (5440 B), padded to 5504 B
constexpr int kRowF = 80, kColF = 32;                 // 68 and 2 x 10 float2, padded to 640 and 256 B
constexpr int kSlotF = kMainF + 2 * kRowF + 2 * kColF;  // one plane of one stencil input (7296 B)
constexpr int kQF = kPX * kPY;                        // one plane of one pointwise input (4096 B)
struct Maps3 {
  CUtensorMap main[2], row[2], col[2], q[2];
};
template <class OP>
constexpr size_t tma3_smem() {
  constexpr bool QS = OP::NQ > 0 && OP::NQ <= 2;
  return sizeof(float2) * ((size_t)OP::NS * kTBuf * kSlotF + (QS ? (size_t)OP::NQ * kTQB * kQF : 0)) + 128;
}

__device__ unsigned long long g_timeouts3;

template <class OP>
__global__ void __launch_bounds__(256, OP::MINB) k_stream3d_tma(const __grid_constant__ OpCoef c, OP op,
                                                                const KScal* act, const __grid_constant__ Maps3 mp) {
  using T = float;
  constexpr int NS = OP::NS;
  constexpr bool QS = OP::NQ > 0 && OP::NQ <= 2;
  constexpr int NQS = QS ? OP::NQ : 1;
  extern __shared__ __align__(128) unsigned char dsm_raw[];
  __shared__ unsigned long long bar[kTBuf];
  __shared__ int s_fail;
  float2* sbase = reinterpret_cast<float2*>(dsm_raw + ((128u - (smem_u32(dsm_raw) & 127u)) & 127u));
  auto mainb = [&](int k, int b) { return sbase + (k * kTBuf + b) * kSlotF; };
  auto rowb = [&](int k, int b, int side) { return mainb(k, b) + kMainF + side * kRowF; };
  auto colb = [&](int k, int b, int side) { return mainb(k, b) + kMainF + 2 * kRowF + side * kColF; };
  float2* qbase = sbase + NS * kTBuf * kSlotF;
  auto qbuf = [&](int k, int qb) { return qbase + (k * kTQB + qb) * kQF; };

  const int nchunk = (c.nz + kZChunk - 1) / kZChunk;
  const int j = (int)(blockIdx.z / (unsigned)nchunk);
  if (act != nullptr && act[j].active == 0) return;
  const int chunk = (int)(blockIdx.z - (unsigned)j * nchunk);
  if (c.prof != nullptr && blockIdx.x == 0 && blockIdx.y == 0 && chunk == 0 && threadIdx.x == 0)
    atomicAdd(c.prof + op.kid, op.bytes);
  Coef7<T> q = coef7<T>(c, j);
  op.coef(q, j);
  Acc<T> acc[OP::ND > 0 ? OP::ND : 1];
#pragma unroll
  for (int d = 0; d < (OP::ND > 0 ? OP::ND : 1); ++d) acc[d].zero();
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int x0 = blockIdx.x * kPX, y0 = blockIdx.y * kPY;
  const int xa = x0 + 2 * tx, y = y0 + ty;
  const long long plane = (long long)c.nx * c.ny;
  const int z0 = chunk * kZChunk, z1 = min(c.nz, z0 + kZChunk);
  // sides of this tile at the periodic boundary (a one-tile-wide grid has both)
  const bool wl = x0 == 0, wr = x0 + kPX == c.nx, wt = y0 == 0, wb = y0 + kPY == c.ny;
  const float2* qs[NQS];
  int nql = 0;
#pragma unroll
  for (int k = 0; k < NQS; ++k) {
    qs[k] = QS ? op.qsrc(k, j) : nullptr;
    nql += qs[k] != nullptr ? 1 : 0;
  }
  const unsigned side_b = (wt ? 544u : 0u) + (wb ? 544u : 0u) + (wl ? 160u : 0u) + (wr ? 160u : 0u);
  auto issue = [&](int b, int qb, int z) {  // thread 0
    const int zw = wrapi(z, c.nz);
    const bool wq = QS && z < z1;
    fence_proxy_async();
    mbar_arrive_expect_tx(&bar[b], NS * (5440u + side_b) + (wq ? 4096u * nql : 0u));
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      tma_load_4d(mainb(k, b), &mp.main[k], &bar[b], 2 * (x0 - 2), y0 - 1, zw, j);
      if (wt) tma_load_4d(rowb(k, b, 0), &mp.row[k], &bar[b], 2 * (x0 - 2), c.ny - 1, zw, j);
      if (wb) tma_load_4d(rowb(k, b, 1), &mp.row[k], &bar[b], 2 * (x0 - 2), 0, zw, j);
      if (wl) tma_load_4d(colb(k, b, 0), &mp.col[k], &bar[b], 2 * (c.nx - 2), y0 - 1, zw, j);
      if (wr) tma_load_4d(colb(k, b, 1), &mp.col[k], &bar[b], 0, y0 - 1, zw, j);
    }
    if (wq) {
#pragma unroll
      for (int k = 0; k < NQS; ++k)
        if (qs[k] != nullptr) tma_load_4d(qbuf(k, qb), &mp.q[k], &bar[b], 2 * x0, y0, zw, j);
    }
  };
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NS; ++k) tma_prefetch_map(&mp.main[k]);
    for (int b = 0; b < kTBuf; ++b) mbar_init(&bar[b], 1);
    fence_mbar_init();
    s_fail = 0;
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int a = 0; a < kTAhead && z0 + a <= z1; ++a) issue(a, a, z0 + a);
  const bool in0 = xa < c.nx && y < c.ny, in1 = xa + 1 < c.nx && y < c.ny;
  const long long p0 = (long long)(in0 ? y : 0) * c.nx + (in0 ? xa : 0);
  const long long p1 = in1 ? p0 + 1 : p0;
  float2 zm0[NS], zm1[NS];
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    const float2* src = op.src(k, j);
    const long long zo = (long long)wrapi(z0 - 1, c.nz) * plane;
    zm0[k] = src[zo + p0];
    zm1[k] = src[zo + p1];
  }
  unsigned ph = 0;  // parity of the next wait of each barrier
  auto wait_buf = [&](int b) {
    const bool ok = mbar_wait(&bar[b], (ph >> b) & 1u);
    ph ^= 1u << b;
    return ok;
  };
  if (!wait_buf(0)) s_fail = 1;
  const int lc = 2 * tx + 2;  // local column of xa: even, so the pair is 16-byte aligned
  int cb = 0, qc = 0;
  int z = z0;
  for (; z < z1; ++z) {
    const int nb = cb + 1 == kTBuf ? 0 : cb + 1;
    int fb = cb + kTAhead;
    if (fb >= kTBuf) fb -= kTBuf;
    int qf = qc + kTAhead;
    if (qf >= kTQB) qf -= kTQB;
    // into buffers that held planes z - 2 (and their inputs), which every thread finished
    // before the barrier of plane z - 1 that this thread has passed
    if (threadIdx.x == 0 && z + kTAhead <= z1) issue(fb, qf, z + kTAhead);
    if (!wait_buf(nb)) s_fail = 1;  // plane z + 1 (the z+ neighbours)
    __syncthreads();
    if (s_fail) break;
    if (in0) {
      N7<T> n0[NS], n1[NS];
#pragma unroll
      for (int k = 0; k < NS; ++k) {
        const float2* m = mainb(k, cb);
        const float4 cc = *reinterpret_cast<const float4*>(m + (ty + 1) * kPW + lc);
        const float2* ymr = (ty == 0 && wt) ? rowb(k, cb, 0) + lc : m + ty * kPW + lc;
        const float2* ypr = (ty == kPY - 1 && wb) ? rowb(k, cb, 1) + lc : m + (ty + 2) * kPW + lc;
        const float4 ym = *reinterpret_cast<const float4*>(ymr);
        const float4 yp = *reinterpret_cast<const float4*>(ypr);
        const float4 zp = *reinterpret_cast<const float4*>(mainb(k, nb) + (ty + 1) * kPW + lc);
        const float2 xm = (tx == 0 && wl) ? colb(k, cb, 0)[(ty + 1) * 2 + 1] : m[(ty + 1) * kPW + lc - 1];
        const float2 xp = (tx == 31 && wr) ? colb(k, cb, 1)[(ty + 1) * 2] : m[(ty + 1) * kPW + lc + 2];
        n0[k].c = make_float2(cc.x, cc.y);
        n0[k].xm = xm;
        n0[k].xp = make_float2(cc.z, cc.w);
        n0[k].ym = make_float2(ym.x, ym.y);
        n0[k].yp = make_float2(yp.x, yp.y);
        n0[k].zm = zm0[k];
        n0[k].zp = make_float2(zp.x, zp.y);
        n1[k].c = make_float2(cc.z, cc.w);
        n1[k].xm = make_float2(cc.x, cc.y);
        n1[k].xp = xp;
        n1[k].ym = make_float2(ym.z, ym.w);
        n1[k].yp = make_float2(yp.z, yp.w);
        n1[k].zm = zm1[k];
        n1[k].zp = make_float2(zp.z, zp.w);
        zm0[k] = n0[k].c;
        zm1[k] = n1[k].c;
      }
      const long long zo = (long long)z * plane;
      float2 pv0[OP::NQ > 0 ? OP::NQ : 1], pv1[OP::NQ > 0 ? OP::NQ : 1];
#pragma unroll
      for (int k = 0; k < OP::NQ; ++k) {
        if constexpr (QS) {
          if (qs[k] != nullptr) {
            const float4 v = *reinterpret_cast<const float4*>(qbuf(k, qc) + ty * kPX + 2 * tx);
            pv0[k] = make_float2(v.x, v.y);
            pv1[k] = make_float2(v.z, v.w);
          } else {
            pv0[k] = pv1[k] = make_float2(0.f, 0.f);
          }
        } else {
          const float2* g = op.qsrc(k, j);
          pv0[k] = g != nullptr ? g[zo + p0] : make_float2(0.f, 0.f);
          pv1[k] = g != nullptr ? g[zo + p1] : make_float2(0.f, 0.f);
        }
      }
      op.apply(j, zo + p0, n0, c, q, acc, pv0);
      if (in1) op.apply(j, zo + p1, n1, c, q, acc, pv1);
#pragma unroll
      for (int d = 0; d < OP::ND; ++d) acc[d].flush();
    }
    cb = nb;
    qc = qc + 1 == kTQB ? 0 : qc + 1;
  }
  if (s_fail) {
    // a plane never arrived: bounded waits for the copies still in flight, then count the
    // timeout (the host checks the count after the solve) and make the products NaN
    if (threadIdx.x == 0) {
      for (int b = 0; b < kTBuf; ++b) (void)wait_buf(b);
      atomicAdd(&g_timeouts3, 1ull);
    }
#pragma unroll
    for (int d = 0; d < (OP::ND > 0 ? OP::ND : 1); ++d) acc[d].add(make_float2(__int_as_float(0x7fc00000), 0.f),
                                                                  make_float2(1.f, 0.f));
  }
  if constexpr (OP::ND > 0) {
    const long long npart = (long long)gridDim.x * gridDim.y * nchunk;
    const long long bid = ((long long)chunk * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
#pragma unroll
    for (int d = 0; d < OP::ND; ++d) {
      block_reduce<T>(acc[d]);
      if (threadIdx.x == 0) acc[d].store(op.partials, (long long)(j * kDotSlots + d) * npart + bid);
    }
  }
}

template <typename T>
inline dim3 grid_stream3d(const OpCoef& c) {
  return dim3((unsigned)((c.nx + tile_cols3<T>() - 1) / tile_cols3<T>()),
              (unsigned)((c.ny + tile_rows3<T>() - 1) / tile_rows3<T>()),
              (unsigned)(c.J * ((c.nz + kZChunk - 1) / kZChunk)));
}


// Tensor maps of the FP32 pass inputs for k_stream3d_tma: every input is a sequence of
// J plane-major [nz][ny][nx] fields with a constant stride between amplitudes (taken from
// src(k, 0) and src(k, 1)).  False if the grid or a buffer does not meet the TMA rules
// (the pass then takes k_stream3d_pair).
template <class OP>
bool maps3(const OpCoef& c, const OP& op, Maps3& mp) {
  if (c.nx % kPX != 0 || c.ny % kPY != 0) return false;
  auto enc = [&](CUtensorMap* m, const float2* a, const float2* b, unsigned bx, unsigned by) {
    if (a == nullptr) return true;
    if ((reinterpret_cast<unsigned long long>(a) & 15ull) != 0) return false;
    const long long ld = c.J > 1 ? (long long)(b - a) : c.pts;
    if (ld <= 0 || (ld & 1)) return false;
    const unsigned long long dims[4] = {2ull * c.nx, (unsigned long long)c.ny, (unsigned long long)c.nz,
                                        (unsigned long long)c.J};
    const unsigned long long st[3] = {8ull * c.nx, 8ull * c.nx * c.ny, 8ull * (unsigned long long)ld};
    const unsigned box[4] = {bx, by, 1, 1};
    return tma_encode_4d(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, a, dims, st, box, nullptr);
  };
  std::memset(&mp, 0, sizeof(mp));
  for (int k = 0; k < OP::NS; ++k) {
    const float2* a = op.src(k, 0);
    const float2* b = op.src(k, c.J > 1 ? 1 : 0);
    if (!enc(&mp.main[k], a, b, 2 * (kPX + 4), kPY + 2) || !enc(&mp.row[k], a, b, 2 * (kPX + 4), 1) ||
        !enc(&mp.col[k], a, b, 4, kPY + 2))
      return false;
  }
  if constexpr (OP::NQ > 0 && OP::NQ <= 2) {
    for (int k = 0; k < OP::NQ; ++k)
      if (!enc(&mp.q[k], op.qsrc(k, 0), op.qsrc(k, c.J > 1 ? 1 : 0), 2 * kPX, kPY)) return false;
  }
  return true;
}

// FP32 passes take the TMA kernel where the grid allows it, else the two-point kernel;
// FP64 passes the one-point kernel.
template <typename T, class OP>
void stream3d(const OpCoef& c, const OP& op, const KScal* act, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    Maps3 mp;
    if (maps3(c, op, mp)) {
      static bool attr = false;
      if (!attr) {
        cudaFuncSetAttribute(k_stream3d_tma<OP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tma3_smem<OP>());
        attr = true;
      }
      k_stream3d_tma<OP><<<grid_stream3d<T>(c), 256, tma3_smem<OP>(), s>>>(c, op, act, mp);
      return;
    }
    k_stream3d_pair<OP><<<grid_stream3d<T>(c), 256, 0, s>>>(c, op, act);
  } else {
    k_stream3d<T, OP><<<grid_stream3d<T>(c), 256, 0, s>>>(c, op, act);
  }
}


}  // namespace

unsigned long long stream3d_timeouts() {
  unsigned long long v = 0;
  if (cudaMemcpyFromSymbol(&v, g_timeouts3, sizeof(v)) != cudaSuccess) return 0;
  return v;
}

int stream3d_parts(const OpCoef& c, int elem_bytes) {
  const dim3 g = elem_bytes == 8 ? grid_stream3d<float>(c) : grid_stream3d<double>(c);
  return (int)(g.x * g.y * (unsigned)((c.nz + kZChunk - 1) / kZChunk));
}

template <typename T>
void launch3d_apply_A(const cplx<T>* x, cplx<T>* y, const OpCoef& c, const KScal* act, cudaStream_t s) {
  ProfScope ps3_(kid_of<T>(KID_APPLY_A), s);
  OpA3<T> op{x, y, c.pts, kid_of<T>(KID_APPLY_A), 4ull * (unsigned long long)c.pts * sizeof(cplx<T>)};
  stream3d<T, OpA3<T>>(c, op, act, s);
}
template <typename T>
void launch_apply_A_dots(const cplx<T>* x, cplx<T>* y, const cplx<T>* du, int nd, void* partials, const OpCoef& c,
                         const KScal* act, cudaStream_t s) {
  ProfScope ps3_(kid_of<T>(KID_APPLY_A), s);
  const unsigned long long b = 6ull * (unsigned long long)c.pts * sizeof(cplx<T>);
  if (nd == 1) {
    OpA3<T, 1> op{x, y, c.pts, kid_of<T>(KID_APPLY_A), b, du, partials};
    stream3d<T, OpA3<T, 1>>(c, op, act, s);
  } else {
    OpA3<T, 2> op{x, y, c.pts, kid_of<T>(KID_APPLY_A), b, du, partials};
    stream3d<T, OpA3<T, 2>>(c, op, act, s);
  }
}
template <typename T>
void launch3d_residual(const cplx<T>* b, const cplx<T>* x, cplx<T>* r, cplx<T>* rhat, const OpCoef& c,
                       cudaStream_t s) {
  ProfScope ps3_(kid_of<T>(KID_RESIDUAL), s);
  OpRes3<T> op{x, b, r, rhat, c.pts, kid_of<T>(KID_RESIDUAL), 8ull * (unsigned long long)c.pts * sizeof(cplx<T>)};
  stream3d<T, OpRes3<T>>(c, op, nullptr, s);
}
template <typename T>
void launch3d_pc_rhs(const cplx<T>* beta, FieldRef<T> f, const OpCoef& c, const KScal* act, cudaStream_t s) {
  ProfScope ps3_(kid_of<T>(KID_PC_RHS), s);
  OpPcRhs3<T> op{beta, f, c.pts, kid_of<T>(KID_PC_RHS), 3ull * (unsigned long long)c.pts * sizeof(cplx<T>)};
  stream3d<T, OpPcRhs3<T>>(c, op, act, s);
}
template <typename T>
void launch3d_cheb_first(CFieldRef<T> f, FieldRef<T> X, FieldRef<T> R, FieldRef<T> Dn, const ChebStep& w, int last,
                         const OpCoef& c, const KScal* act, cudaStream_t s, const PcFin<T>* fin) {
  ProfScope ps3_(kid_of<T>(KID_CHEB_FIRST), s);
  const bool fold = fin != nullptr;
  OpChebFirst3<T> op{f,    X,
                     R,    Dn,
                     w,    last,
                     fold ? *fin : PcFin<T>{},
                     kid_of<T>(KID_CHEB_FIRST),
                     (last ? (fold ? 4ull : 2ull) : 4ull) * (unsigned long long)c.pts * sizeof(cplx<T>)};
  stream3d<T, OpChebFirst3<T>>(c, op, act, s);
}
template <typename T>
void launch3d_cheb_sweep(CFieldRef<T> Dd, FieldRef<T> X, FieldRef<T> R, FieldRef<T> Dn, const ChebStep& w, int last,
                         const OpCoef& c, const KScal* act, cudaStream_t s, const PcFin<T>* fin) {
  ProfScope ps3_(kid_of<T>(KID_CHEB_SWEEP), s);
  const bool fold = fin != nullptr;
  OpChebSweep3<T> op{Dd,   X,
                     R,    Dn,
                     w,    last,
                     fold ? *fin : PcFin<T>{},
                     kid_of<T>(KID_CHEB_SWEEP),
                     (last ? (fold ? 7ull : 4ull) : 6ull) * (unsigned long long)c.pts * sizeof(cplx<T>)};
  stream3d<T, OpChebSweep3<T>>(c, op, act, s);
}
void launch3d_zeta(double2* x, const OpCoef& c, cudaStream_t s) {
  ProfScope ps3_(KID_ZETA, s);
  OpZeta3 op{x, c.pts, KID_ZETA, 2ull * (unsigned long long)c.pts * sizeof(double2)};
  k_stream3d<double, OpZeta3><<<grid_stream3d<double>(c), 256, 0, s>>>(c, op, nullptr);
}
#define APFC_INST3(T)                                                                                                \
  template void launch3d_apply_A<T>(const cplx<T>*, cplx<T>*, const OpCoef&, const KScal*, cudaStream_t);           \
  template void launch_apply_A_dots<T>(const cplx<T>*, cplx<T>*, const cplx<T>*, int, void*, const OpCoef&,         \
                                       const KScal*, cudaStream_t);                                                 \
  template void launch3d_residual<T>(const cplx<T>*, const cplx<T>*, cplx<T>*, cplx<T>*, const OpCoef&,             \
                                     cudaStream_t);                                                                 \
  template void launch3d_pc_rhs<T>(const cplx<T>*, FieldRef<T>, const OpCoef&, const KScal*, cudaStream_t);         \
  template void launch3d_cheb_first<T>(CFieldRef<T>, FieldRef<T>, FieldRef<T>, FieldRef<T>, const ChebStep&, int,   \
                                       const OpCoef&, const KScal*, cudaStream_t, const PcFin<T>*);                 \
  template void launch3d_cheb_sweep<T>(CFieldRef<T>, FieldRef<T>, FieldRef<T>, FieldRef<T>, const ChebStep&, int,   \
                                       const OpCoef&, const KScal*, cudaStream_t, const PcFin<T>*);

APFC_INST3(double)
APFC_INST3(float)

}  // namespace apfc
