// Stencil and pointwise kernels of the APFC step (arXiv:1902.09761, Sec. II).
//
// All operators are constant-coefficient periodic stencils:
//   L_h u  = sum_d (u(+e_d) - 2u + u(-e_d)) / h_d^2
//   G_h u  = L_h u + 2i sum_d k_d (u(+e_d) - u(-e_d)) / (2 h_d)
//   A_j (zeta, eta) = (zeta - G_h eta, kt G_h zeta + a eta)       (Eq. linear_system2, M = I)
//   D u    = sD u - mu L_h u                                      (diffusion part of Eq. preconditioner)
#include <algorithm>

#include "acc.cuh"
#include "apfc_internal.cuh"
#include "dfloat.cuh"
#include "resid_point.cuh"

namespace apfc {

namespace {

struct Nb {
  long long c, xp, xm, yp, ym, zp, zm;
};

__device__ __forceinline__ Nb neighbours(long long p, const OpCoef& c) {
  Nb n;
  n.c = p;
  const long long nx = c.nx, ny = c.ny, plane = nx * ny;
  const long long z = p / plane;
  const long long rem = p - z * plane;
  const long long y = rem / nx;
  const long long x = rem - y * nx;
  n.xp = (x + 1 == nx) ? p - x : p + 1;
  n.xm = (x == 0) ? p + nx - 1 : p - 1;
  n.yp = (y + 1 == ny) ? p - y * nx : p + nx;
  n.ym = (y == 0) ? p + (ny - 1) * nx : p - nx;
  if (c.dim == 3) {
    n.zp = (z + 1 == c.nz) ? p - z * plane : p + plane;
    n.zm = (z == 0) ? p + (long long)(c.nz - 1) * plane : p - plane;
  } else {
    n.zp = n.zm = p;
  }
  return n;
}

// G_h u at one point.
template <typename T>
__device__ __forceinline__ cplx<T> opG(const cplx<T>* __restrict__ u, const Nb& n, const OpCoef& c, int j) {
  const cplx<T> uc = u[n.c];
  T re = (T)c.c0 * uc.x, im = (T)c.c0 * uc.y;
  {
    const cplx<T> a = u[n.xp], b = u[n.xm];
    const T s = (T)c.ih2[0], k = (T)c.kh[j][0];
    re += s * (a.x + b.x) - k * (a.y - b.y);
    im += s * (a.y + b.y) + k * (a.x - b.x);
  }
  {
    const cplx<T> a = u[n.yp], b = u[n.ym];
    const T s = (T)c.ih2[1], k = (T)c.kh[j][1];
    re += s * (a.x + b.x) - k * (a.y - b.y);
    im += s * (a.y + b.y) + k * (a.x - b.x);
  }
  if (c.dim == 3) {
    const cplx<T> a = u[n.zp], b = u[n.zm];
    const T s = (T)c.ih2[2], k = (T)c.kh[j][2];
    re += s * (a.x + b.x) - k * (a.y - b.y);
    im += s * (a.y + b.y) + k * (a.x - b.x);
  }
  return mkc<T>(re, im);
}

// D u = sD u - mu L_h u at one point.
template <typename T>
__device__ __forceinline__ cplx<T> opD(const cplx<T>* __restrict__ u, const Nb& n, const OpCoef& c, int j) {
  const cplx<T> uc = u[n.c];
  T re = (T)c.c0 * uc.x, im = (T)c.c0 * uc.y;
  {
    const cplx<T> a = u[n.xp], b = u[n.xm];
    re += (T)c.ih2[0] * (a.x + b.x);
    im += (T)c.ih2[0] * (a.y + b.y);
  }
  {
    const cplx<T> a = u[n.yp], b = u[n.ym];
    re += (T)c.ih2[1] * (a.x + b.x);
    im += (T)c.ih2[1] * (a.y + b.y);
  }
  if (c.dim == 3) {
    const cplx<T> a = u[n.zp], b = u[n.zm];
    re += (T)c.ih2[2] * (a.x + b.x);
    im += (T)c.ih2[2] * (a.y + b.y);
  }
  const T sD = (T)c.sD[j], mu = (T)c.mu[j];
  return mkc<T>(sD * uc.x - mu * re, sD * uc.y - mu * im);
}

template <typename T>
__device__ __forceinline__ cplx<T> cmul(double2 s, cplx<T> v) {
  const T a = (T)s.x, b = (T)s.y;
  return mkc<T>(a * v.x - b * v.y, a * v.y + b * v.x);
}

__device__ __forceinline__ bool skip(const KScal* act, int j) { return act != nullptr && act[j].active == 0; }

// Per-pass kernels run on a 3D grid: 32 x 8 points per block in (x, y), blockIdx.z
// = z + nz * j (plane z of amplitude j).  Periodic neighbours by comparison.
__device__ __forceinline__ int amp_of(const OpCoef& c) { return (int)(blockIdx.z / (unsigned)c.nz); }

__device__ __forceinline__ Nb neighbours3(int x, int y, int z, long long p, const OpCoef& c) {
  Nb n;
  n.c = p;
  const long long nx = c.nx, plane = (long long)c.nx * c.ny;
  n.xp = (x + 1 == c.nx) ? p - x : p + 1;
  n.xm = (x == 0) ? p + nx - 1 : p - 1;
  n.yp = (y + 1 == c.ny) ? p - (long long)y * nx : p + nx;
  n.ym = (y == 0) ? p + (long long)(c.ny - 1) * nx : p - nx;
  if (c.dim == 3) {
    n.zp = (z + 1 == c.nz) ? p - (long long)z * plane : p + plane;
    n.zm = (z == 0) ? p + (long long)(c.nz - 1) * plane : p - plane;
  } else {
    n.zp = n.zm = p;
  }
  return n;
}

// algorithmic bytes, counted once per amplitude (block (0, 0, plane 0) of amplitude j)
__device__ __forceinline__ void prof_add3(const OpCoef& c, int kid, unsigned long long bytes) {
  if (c.prof != nullptr && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0 &&
      blockIdx.z % (unsigned)c.nz == 0)
    atomicAdd(c.prof + kid, bytes);
}

#define APFC_POINT_INDEX                                                               \
  const int j = amp_of(c);                                                             \
  const int zz_ = (int)(blockIdx.z - (unsigned)j * (unsigned)c.nz);                    \
  const int xx_ = blockIdx.x * 32 + (threadIdx.x & 31), yy_ = blockIdx.y * 8 + (threadIdx.x >> 5); \
  if (xx_ >= c.nx || yy_ >= c.ny) return;                                              \
  const long long p = ((long long)zz_ * c.ny + yy_) * c.nx + xx_;

#define APFC_NEIGHBOURS neighbours3(xx_, yy_, zz_, p, c)

// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_apply_A(const cplx<T>* __restrict__ x, cplx<T>* __restrict__ y, OpCoef c, const KScal* act) {
  if (skip(act, amp_of(c))) return;
  prof_add3(c, kid_of<T>(KID_APPLY_A), 4ull * (unsigned long long)c.pts * sizeof(cplx<T>));
  APFC_POINT_INDEX
  const cplx<T>* z = x + 2LL * j * c.pts;
  const cplx<T>* e = z + c.pts;
  const Nb n = APFC_NEIGHBOURS;
  const cplx<T> gz = opG<T>(z, n, c, j), ge = opG<T>(e, n, c, j);
  const cplx<T> zc = z[p], ec = e[p];
  cplx<T>* y1 = y + 2LL * j * c.pts;
  const T kt = (T)c.kt[j], a = (T)a_at(c, j, p);
  y1[p] = mkc<T>(zc.x - ge.x, zc.y - ge.y);
  y1[c.pts + p] = mkc<T>(kt * gz.x + a * ec.x, kt * gz.y + a * ec.y);
}

template <typename T>
__global__ void k_residual(const cplx<T>* __restrict__ b, const cplx<T>* __restrict__ x, cplx<T>* __restrict__ r,
                           cplx<T>* __restrict__ rhat, OpCoef c) {
  prof_add3(c, kid_of<T>(KID_RESIDUAL), 8ull * (unsigned long long)c.pts * sizeof(cplx<T>));
  APFC_POINT_INDEX
  const long long o = 2LL * j * c.pts;
  const cplx<T>* z = x + o;
  const cplx<T>* e = z + c.pts;
  const Nb n = APFC_NEIGHBOURS;
  const cplx<T> gz = opG<T>(z, n, c, j), ge = opG<T>(e, n, c, j);
  const cplx<T> zc = z[p], ec = e[p];
  const cplx<T> b1 = b[o + p], b2 = b[o + c.pts + p];
  const T kt = (T)c.kt[j], a = (T)a_at(c, j, p);
  const cplx<T> r1 = mkc<T>(b1.x - (zc.x - ge.x), b1.y - (zc.y - ge.y));
  const cplx<T> r2 = mkc<T>(b2.x - (kt * gz.x + a * ec.x), b2.y - (kt * gz.y + a * ec.y));
  r[o + p] = r1;
  r[o + c.pts + p] = r2;
  rhat[o + p] = r1;
  rhat[o + c.pts + p] = r2;
}

// Step 2 right-hand side of P^{-1}: f = beta2 - kt G_h beta1 (beta1' = beta1 since M = I).
template <typename T>
__global__ void k_pc_rhs(const cplx<T>* __restrict__ beta, FieldRef<T> f, OpCoef c, const KScal* act) {
  if (skip(act, amp_of(c))) return;
  prof_add3(c, kid_of<T>(KID_PC_RHS), 3ull * (unsigned long long)c.pts * sizeof(cplx<T>));
  APFC_POINT_INDEX
  const cplx<T>* b1 = beta + 2LL * j * c.pts;
  const cplx<T> b2 = b1[c.pts + p];
  const Nb n = APFC_NEIGHBOURS;
  const cplx<T> g = opG<T>(b1, n, c, j);
  const T kt = (T)c.kt[j];
  f.at(j)[p] = mkc<T>(b2.x - kt * g.x, b2.y - kt * g.y);
}

// Chebyshev with zero applications of D: X = f / theta.
template <typename T>
__global__ void k_cheb_zero(CFieldRef<T> f, FieldRef<T> X, OpCoef c, const KScal* act) {
  if (skip(act, amp_of(c))) return;
  prof_add3(c, kid_of<T>(KID_CHEB_ZERO), 2ull * (unsigned long long)c.pts * sizeof(cplx<T>));
  APFC_POINT_INDEX
  const T it = (T)c.inv_theta[j];
  const cplx<T> v = f.at(j)[p];
  X.at(j)[p] = mkc<T>(it * v.x, it * v.y);
}

// First Chebyshev application: d0 = f/theta, x1 = d0, r1 = f - D d0, d1 = c1 d0 + c2 r1.
// last: write x_final = x1 + d1 only.
template <typename T>
__global__ void k_cheb_first(CFieldRef<T> f, FieldRef<T> X, FieldRef<T> R, FieldRef<T> Dn, ChebStep w, int last,
                             OpCoef c, const KScal* act) {
  if (skip(act, amp_of(c))) return;
  prof_add3(c, kid_of<T>(KID_CHEB_FIRST), (last ? 2ull : 4ull) * (unsigned long long)c.pts * sizeof(cplx<T>));
  APFC_POINT_INDEX
  const cplx<T>* fj = f.at(j);

  const Nb n = APFC_NEIGHBOURS;
  const T it = (T)c.inv_theta[j];
  const cplx<T> Df = opD<T>(fj, n, c, j);
  const cplx<T> fc = fj[p];
  const cplx<T> d0 = mkc<T>(it * fc.x, it * fc.y);
  const cplx<T> r1 = mkc<T>(fc.x - it * Df.x, fc.y - it * Df.y);
  const T c1 = (T)w.c1[j], c2 = (T)w.c2[j];
  const cplx<T> d1 = mkc<T>(c1 * d0.x + c2 * r1.x, c1 * d0.y + c2 * r1.y);
  if (last) {
    X.at(j)[p] = mkc<T>(d0.x + d1.x, d0.y + d1.y);
  } else {
    X.at(j)[p] = d0;
    R.at(j)[p] = r1;
    Dn.at(j)[p] = d1;
  }
}

// Later application: x += d; r -= D d; d' = c1 d + c2 r.  last: write x + d' only.
template <typename T>
__global__ void k_cheb_sweep(CFieldRef<T> Dd, FieldRef<T> X, FieldRef<T> R, FieldRef<T> Dn, ChebStep w, int last,
                             OpCoef c, const KScal* act) {
  if (skip(act, amp_of(c))) return;
  prof_add3(c, kid_of<T>(KID_CHEB_SWEEP), (last ? 4ull : 6ull) * (unsigned long long)c.pts * sizeof(cplx<T>));
  APFC_POINT_INDEX
  const cplx<T>* dj = Dd.at(j);
  const Nb n = APFC_NEIGHBOURS;
  const cplx<T> DD = opD<T>(dj, n, c, j);
  const cplx<T> d = dj[p];
  const cplx<T> x = X.at(j)[p];
  const cplx<T> r = R.at(j)[p];
  const cplx<T> xn = mkc<T>(x.x + d.x, x.y + d.y);
  const cplx<T> rn = mkc<T>(r.x - DD.x, r.y - DD.y);
  const T c1 = (T)w.c1[j], c2 = (T)w.c2[j];
  const cplx<T> dn = mkc<T>(c1 * d.x + c2 * rn.x, c1 * d.y + c2 * rn.y);
  if (last) {
    X.at(j)[p] = mkc<T>(xn.x + dn.x, xn.y + dn.y);
  } else {
    X.at(j)[p] = xn;
    R.at(j)[p] = rn;
    Dn.at(j)[p] = dn;
  }
}

// Step 4 of P^{-1}: chi1 = beta1 + (beta2' - sD chi2) / mu; chi2 is already in place.
template <typename T>
__global__ void k_pc_final(const cplx<T>* __restrict__ beta, CFieldRef<T> b2p, cplx<T>* __restrict__ chi, OpCoef c,
                           const KScal* act) {
  if (skip(act, amp_of(c))) return;
  prof_add3(c, kid_of<T>(KID_PC_FINAL), 4ull * (unsigned long long)c.pts * sizeof(cplx<T>));
  APFC_POINT_INDEX
  const long long o = 2LL * j * c.pts;
  const cplx<T> b1 = beta[o + p];
  const cplx<T> bp = b2p.at(j)[p];
  const cplx<T> x2 = chi[o + c.pts + p];
  const T sD = (T)c.sD[j], im = (T)c.inv_mu[j];
  chi[o + p] = mkc<T>(b1.x + im * (bp.x - sD * x2.x), b1.y + im * (bp.y - sD * x2.y));
}

// BiCGStab updates on block vectors (scalars from the device KScal array).  Each
// amplitude takes kDotBlocks blocks striding over its 2 pts values, so the FP64 scalars
// are converted once per thread, and the inner products of the updated vectors come
// out of the same pass with the traversal (and so the partial sums) of k_dots.
template <typename T>
__global__ void k_p_update(const cplx<T>* __restrict__ r, cplx<T>* __restrict__ p_, const cplx<T>* __restrict__ v,
                           OpCoef c, const KScal* k) {
  const int j = blockIdx.y;
  if (!k[j].active) return;
  prof_add(c, kid_of<T>(KID_P_UPDATE), 8ull * (unsigned long long)c.pts * sizeof(cplx<T>));
  const long long n = 2LL * c.pts, o = 2LL * j * c.pts;
  const T br = (T)k[j].beta.x, bi = (T)k[j].beta.y, wr = (T)k[j].omega.x, wi = (T)k[j].omega.y;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const cplx<T> pv = p_[o + i], vv = v[o + i], rv = r[o + i];
    const T tx = pv.x - (wr * vv.x - wi * vv.y), ty = pv.y - (wr * vv.y + wi * vv.x);
    p_[o + i] = mkc<T>(rv.x + (br * tx - bi * ty), rv.y + (br * ty + bi * tx));
  }
}

// s = r - alpha v (in place in r); partials != nullptr: (s, s) in slot 0.
template <typename T>
__global__ void k_s_update(cplx<T>* __restrict__ r, const cplx<T>* __restrict__ v, OpCoef c, const KScal* k,
                           void* partials) {
  const int j = blockIdx.y;
  if (!k[j].active) return;
  prof_add(c, kid_of<T>(KID_S_UPDATE), 6ull * (unsigned long long)c.pts * sizeof(cplx<T>));
  const long long n = 2LL * c.pts, o = 2LL * j * c.pts;
  const T ar = (T)k[j].alpha.x, ai = (T)k[j].alpha.y;
  Acc<T> acc;
  acc.zero();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const cplx<T> vv = v[o + i], rv = r[o + i];
    const cplx<T> sv = mkc<T>(rv.x - (ar * vv.x - ai * vv.y), rv.y - (ar * vv.y + ai * vv.x));
    r[o + i] = sv;
    acc.add(sv, sv);
  }
  if (partials == nullptr) return;
  block_reduce<T>(acc);
  if (threadIdx.x == 0) acc.store(partials, (long long)(j * kDotSlots) * kDotBlocks + blockIdx.x);
}

// u += alpha p + omega s; r = s - omega t (s held in r); partials != nullptr: (rhat, r),
// (r, r) in slots 0 and 1.  An amplitude that stopped at the s-check or at omega (not
// active, just_done) only takes its owed u += alpha p.
template <typename T>
__global__ void k_r_update(cplx<T>* __restrict__ r, const cplx<T>* __restrict__ t, cplx<T>* __restrict__ u,
                           const cplx<T>* __restrict__ p_, const cplx<T>* __restrict__ rhat, OpCoef c,
                           const KScal* k, void* partials) {
  const int j = blockIdx.y;
  const bool act = k[j].active != 0;
  if (!act && k[j].just_done == 0) return;
  const long long n = 2LL * c.pts, o = 2LL * j * c.pts;
  const T ar = (T)k[j].alpha.x, ai = (T)k[j].alpha.y;
  const long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x, di = (long long)gridDim.x * blockDim.x;
  if (!act) {
    prof_add(c, kid_of<T>(KID_R_UPDATE), 6ull * (unsigned long long)c.pts * sizeof(cplx<T>));
    for (long long i = i0; i < n; i += di) {
      const cplx<T> pv = p_[o + i], uv = u[o + i];
      u[o + i] = mkc<T>(uv.x + (ar * pv.x - ai * pv.y), uv.y + (ar * pv.y + ai * pv.x));
    }
    return;
  }
  prof_add(c, kid_of<T>(KID_R_UPDATE),
           (partials != nullptr ? 14ull : 12ull) * (unsigned long long)c.pts * sizeof(cplx<T>));
  const T wr = (T)k[j].omega.x, wi = (T)k[j].omega.y;
  Acc<T> a0, a1;
  a0.zero();
  a1.zero();
  for (long long i = i0; i < n; i += di) {
    const cplx<T> sv = r[o + i], tv = t[o + i], uv = u[o + i], pv = p_[o + i];
    u[o + i] = mkc<T>(uv.x + (ar * pv.x - ai * pv.y) + (wr * sv.x - wi * sv.y),
                      uv.y + (ar * pv.y + ai * pv.x) + (wr * sv.y + wi * sv.x));
    const cplx<T> rn = mkc<T>(sv.x - (wr * tv.x - wi * tv.y), sv.y - (wr * tv.y + wi * tv.x));
    r[o + i] = rn;
    if (partials != nullptr) {
      a0.add(rhat[o + i], rn);
      a1.add(rn, rn);
    }
  }
  if (partials == nullptr) return;
  block_reduce<T>(a0);
  if (threadIdx.x == 0) a0.store(partials, (long long)(j * kDotSlots) * kDotBlocks + blockIdx.x);
  block_reduce<T>(a1);
  if (threadIdx.x == 0) a1.store(partials, (long long)(j * kDotSlots + 1) * kDotBlocks + blockIdx.x);
}

template <typename T>
__global__ void k_add_to(const cplx<T>* __restrict__ d, double2* __restrict__ x, long long n, OpCoef c) {
  prof_add(c, kid_of<T>(KID_ADD_TO), (unsigned long long)n * (sizeof(cplx<T>) + 2 * sizeof(double2)));
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const cplx<T> dv = d[i];
  double2 xv = x[i];
  if constexpr (sizeof(T) == 4) {  // exact widening by integer operations (no FP64 conversion)
    xv.x += f2d(dv.x);
    xv.y += f2d(dv.y);
  } else {
    xv.x += dv.x;
    xv.y += dv.y;
  }
  x[i] = xv;
}

// ---------------------------------------------------------------------------
// Explicit nonlinear right-hand side: b_eta,j = eta_j/dt - |k_j|^2 N_j(eta).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double2 cm(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }

// N_j at one point from amplitudes held in shared memory (column threadIdx.x of se, with
// |eta_m|^2 in sn): the triangular closed form, or eta_j sum_m wdiag[j][m] |eta_m|^2 plus the
// remaining table monomials.  Shared memory keeps the table's run-time amplitude indices off
// local memory; the first factor of a monomial scales its real coefficient.
__device__ __forceinline__ double2 nonlin_shared(const double2 (*se)[kThreads], const double (*sn)[kThreads], int j,
                                                 int J, double A2, const NonlinTable& nt) {
  const int t = threadIdx.x;
  const double2 ej = se[j][t];
  if (nt.hex) {
    // N_j = 3v (A^2 - |eta_j|^2) eta_j - 2t conj(eta_k eta_l)
    const int k1 = j == 2 ? 0 : j + 1, k2 = j == 0 ? 2 : j - 1;
    const double m2 = ej.x * ej.x + ej.y * ej.y;
    const double s = 3.0 * nt.v * (A2 - m2);
    const double2 pr = cconj(cm(se[k1][t], se[k2][t]));
    return make_double2(s * ej.x - 2.0 * nt.t * pr.x, s * ej.y - 2.0 * nt.t * pr.y);
  }
  double w = 0.0;
  for (int m = 0; m < J; ++m) w += nt.wdiag[j][m] * sn[m][t];
  double2 N = make_double2(w * ej.x, w * ej.y);
  for (int i = nt.rstart[j]; i < nt.rstart[j + 1]; ++i) {
    const int q = nt.ridx[i];
    const int c0 = nt.f[q][0];
    const double2 e0 = se[c0 >> 1][t];
    const double cf = nt.coef[q];
    double2 prod = make_double2(cf * e0.x, (c0 & 1) ? -cf * e0.y : cf * e0.y);
    for (int f = 1; f < nt.nf[q]; ++f) {
      const int code = nt.f[q][f];
      const double2 e = se[code >> 1][t];
      prod = cm(prod, (code & 1) ? cconj(e) : e);
    }
    N.x += prod.x;
    N.y += prod.y;
  }
  return N;
}

// Load the amplitudes of point p into shared memory (se, and |eta_m|^2 into sn); returns A^2.
__device__ __forceinline__ double load_point(const double2* __restrict__ x, long long pts, long long p, int J,
                                             double2 (*se)[kThreads], double (*sn)[kThreads]) {
  double A2 = 0.0;
  for (int j = 0; j < J; ++j) {
    const double2 e = x[(2LL * j + 1) * pts + p];
    se[j][threadIdx.x] = e;
    const double n2 = e.x * e.x + e.y * e.y;
    sn[j][threadIdx.x] = n2;
    A2 += n2;
  }
  return 2.0 * A2;
}

// Batched runs (rg != nullptr): blockIdx.y selects the run.
__global__ void k_rhs(const double2* __restrict__ x, double2* __restrict__ b, const __grid_constant__ OpCoef c,
                      const __grid_constant__ NonlinTable nt, const RunGeom* rg) {
  long long pts = c.pts;  // the run's own size when batched (c stays untouched: no local copy)
  if (rg != nullptr) {
    const RunGeom& q = rg[blockIdx.y];
    pts = q.pts;
    x += q.elem_off;
    b += q.elem_off;
  }
  if (c.prof != nullptr && blockIdx.x == 0 && threadIdx.x == 0)
    atomicAdd(c.prof + KID_RHS, 2ull * c.J * (unsigned long long)pts * sizeof(double2));
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  __shared__ double2 se[kMaxJ][kThreads];
  __shared__ double sn[kMaxJ][kThreads];
  if (p >= pts) return;
  const double A2 = load_point(x, pts, p, c.J, se, sn);
  for (int j = 0; j < c.J; ++j) {
    const double2 N = nonlin_shared(se, sn, j, c.J, A2, nt);
    const double2 ej = se[j][threadIdx.x];
    const double kap = c.kap[j];
    b[(2LL * j + 1) * pts + p] = make_double2(ej.x * c.inv_dt - kap * N.x, ej.y * c.inv_dt - kap * N.y);
  }
}

// zeta-part of the state = G_h (eta-part)
// zeta = G_h eta from the state's eta-parts, FP64-accurate without the FP64 pipe: the point
// and its neighbours split into FP32 pairs and G_h as one compensated sum of products with
// the residual's grouping (resid_point.cuh), rounded to the nearest double at the end.
template <int DIM>
__global__ void __launch_bounds__(256) k_zeta(double2* __restrict__ x, const __grid_constant__ OpCoef c) {
  prof_add3(c, KID_ZETA, 2ull * (unsigned long long)c.pts * sizeof(double2));
  APFC_POINT_INDEX
  const double2* e = x + (2LL * j + 1) * c.pts;
  const Nb n = APFC_NEIGHBOURS;
  const ResidCoef<DIM> q = resid_coef<DIM>(c, j);
  PDF en[DIM][2];
  en[0][0] = pdf_split(e[n.xm]);
  en[0][1] = pdf_split(e[n.xp]);
  en[1][0] = pdf_split(e[n.ym]);
  en[1][1] = pdf_split(e[n.yp]);
  if constexpr (DIM == 3) {
    en[2][0] = pdf_split(e[n.zm]);
    en[2][1] = pdf_split(e[n.zp]);
  }
  PAcc a;
  a.init(PDF{make_float2(0.f, 0.f), make_float2(0.f, 0.f)});
  a.fma(q.g0.h, q.g0.l, pdf_split(e[p]));
#pragma unroll
  for (int d = 0; d < DIM; ++d) a.fma(q.gl[d].h, q.gl[d].l, pdf_add(en[d][1], en[d][0]));
#pragma unroll
  for (int d = 0; d < DIM; ++d) a.fma(q.ga[d].h, q.ga[d].l, pdf_swap(pdf_sub(en[d][1], en[d][0])));
  float2 hi, lo;
  a.result(hi, lo);
  x[2LL * j * c.pts + p] = make_double2(df_to_d(DF{hi.x, lo.x}), df_to_d(DF{hi.y, lo.y}));
}

// ---------------------------------------------------------------------------
// Block sums in FP64
// ---------------------------------------------------------------------------
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV]) {
  __shared__ double sh[NV][kThreads / 32];
#pragma unroll
  for (int i = 0; i < NV; ++i)
    for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) sh[i][w] = v[i];
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      v[i] = (l < kThreads / 32) ? sh[i][l] : 0.0;
      for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
    }
  }
}

// FP64 outer residual of the refinement: r = b - A x (x, b FP64), written as FP32;
// partials: ||r||^2 and ||b||^2 per amplitude (double2 layout [J][2][kDotBlocks]).
__global__ void k_residual_refine(const double2* __restrict__ b, const double2* __restrict__ x, float2* __restrict__ r32,
                                  double2* __restrict__ partials, OpCoef c) {
  const int j = blockIdx.y;
  prof_add(c, KID_RESID_REFINE, (unsigned long long)c.pts * (4 * sizeof(double2) + 2 * sizeof(float2)));
  const long long o = 2LL * j * c.pts;
  const double2* z = x + o;
  const double2* e = z + c.pts;
  const double kt = c.kt[j], a = c.a[j];
  double acc[2] = {0.0, 0.0};
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < c.pts;
       p += (long long)gridDim.x * blockDim.x) {
    const Nb n = neighbours(p, c);
    const double2 gz = opG<double>(z, n, c, j), ge = opG<double>(e, n, c, j);
    const double2 zc = z[p], ec = e[p];
    const double2 b1 = b[o + p], b2 = b[o + c.pts + p];
    const double r1x = b1.x - (zc.x - ge.x), r1y = b1.y - (zc.y - ge.y);
    const double ap = c.jd == nullptr ? a : a_at(c, j, p);
    const double r2x = b2.x - (kt * gz.x + ap * ec.x), r2y = b2.y - (kt * gz.y + ap * ec.y);
    r32[o + p] = make_float2((float)r1x, (float)r1y);
    r32[o + c.pts + p] = make_float2((float)r2x, (float)r2y);
    acc[0] += r1x * r1x + r1y * r1y + r2x * r2x + r2y * r2y;
    acc[1] += b1.x * b1.x + b1.y * b1.y + b2.x * b2.x + b2.y * b2.y;
  }
  block_sum<2>(acc);
  if (threadIdx.x == 0) {
    partials[(j * kDotSlots + 0) * kDotBlocks + blockIdx.x] = make_double2(acc[0], 0.0);
    partials[(j * kDotSlots + 1) * kDotBlocks + blockIdx.x] = make_double2(acc[1], 0.0);
  }
}

// FP64-accurate outer residual on 2D grids, r = b - A x with x, b FP64 in memory,
// evaluated without the FP64 pipe: every input double is split into an FP32 pair
// (h, l) by integer operations and each component of r1 = b1 - zeta + G_h eta and
// r2 = b2 - kt G_h zeta - a eta is one compensated sum of products (dfloat.cuh);
// residuals to about 1e-14 of the terms' size, beneath the 1e-10 and 1e-13
// tolerances of the refinement.  Writes r as FP32 (the inner solve's right-hand
// side) and, if r64 != nullptr, as FP64 (kept as the previous residual of the
// next step).  32 x 8 point tiles whose (zeta, eta) values and one-point halo are
// split once into shared memory.  The partial ||r||^2 per amplitude is
// accumulated from the FP32-rounded residual (it only decides convergence,
// where a relative error of 1e-5 in the norm is immaterial); ||b||^2 is not
// recomputed: b is fixed within a step.
constexpr int kRTX = 32, kRTY = 8;
__global__ void __launch_bounds__(256, 3) k_residual_refine2d(const double2* __restrict__ b,
                                                           const double2* __restrict__ x, float2* __restrict__ r32,
                                                           double2* __restrict__ r64, double2* __restrict__ partials,
                                                           const __grid_constant__ OpCoef c, const RunGeom* rg) {
  const int j = blockIdx.y;
  int nx = c.nx, ny = c.ny;
  long long pts = c.pts;
  if (rg != nullptr) {  // batched runs: blockIdx.z selects the run (the Jacobian is never on here)
    const RunGeom& q = rg[blockIdx.z];
    nx = q.nx;
    ny = q.ny;
    pts = q.pts;
    b += q.elem_off;
    x += q.elem_off;
    r32 += q.elem_off;
    if (r64 != nullptr) r64 += q.elem_off;
    partials += (long long)blockIdx.z * c.J * kDotSlots * kDotBlocks;
  }
  if (c.prof != nullptr && blockIdx.x == 0 && threadIdx.x == 0)
    atomicAdd(c.prof + KID_RESID_REFINE, (unsigned long long)pts * (4 * sizeof(double2) + 2 * sizeof(float2) +
                                                                   (r64 ? 2 * sizeof(double2) : 0)));
  __shared__ float4 sz[kRTY + 2][kRTX + 2], se[kRTY + 2][kRTX + 2];
  const long long o = 2LL * j * pts;
  const double2* z = x + o;
  const double2* e = z + pts;
  const ResidCoef<2> q = resid_coef<2>(c, j);
  LaneC ma = lane_c(c.a[j], -1.f, -1.f);
  const int tx_count = (nx + kRTX - 1) / kRTX, ntiles = tx_count * ((ny + kRTY - 1) / kRTY);
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  float rr = 0.f;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int tyi = tile / tx_count;
    const int x0 = (tile - tyi * tx_count) * kRTX, y0 = tyi * kRTY;
    __syncthreads();  // the previous tile's shared values are no longer read
    for (int i = threadIdx.x; i < (kRTX + 2) * (kRTY + 2); i += 256) {
      const int ry = i / (kRTX + 2), rx = i - ry * (kRTX + 2);
      int gxx = x0 - 1 + rx, gyy = y0 - 1 + ry;
      gxx = gxx < 0 ? gxx + nx : (gxx >= nx ? gxx % nx : gxx);
      gyy = gyy < 0 ? gyy + ny : (gyy >= ny ? gyy % ny : gyy);
      const long long q = (long long)gyy * nx + gxx;
      sz[ry][rx] = pdf_pack(pdf_split(z[q]));
      se[ry][rx] = pdf_pack(pdf_split(e[q]));
    }
    __syncthreads();
    const int xx = x0 + tx, yy = y0 + ty;
    if (xx >= nx || yy >= ny) continue;
    const long long pc = (long long)yy * nx + xx;
    const PDF zn[2][2] = {{pdf_unpack(sz[ty + 1][tx]), pdf_unpack(sz[ty + 1][tx + 2])},
                          {pdf_unpack(sz[ty][tx + 1]), pdf_unpack(sz[ty + 2][tx + 1])}};
    const PDF en[2][2] = {{pdf_unpack(se[ty + 1][tx]), pdf_unpack(se[ty + 1][tx + 2])},
                          {pdf_unpack(se[ty][tx + 1]), pdf_unpack(se[ty + 2][tx + 1])}};
    if (c.jd != nullptr) ma = lane_c(a_at(c, j, pc), -1.f, -1.f);
    float2 f1, l1, f2, l2;
    resid_point<2>(q, ma, pdf_split(b[o + pc]), pdf_split(b[o + pts + pc]), pdf_unpack(sz[ty + 1][tx + 1]),
                   pdf_unpack(se[ty + 1][tx + 1]), zn, en, f1, l1, f2, l2);
    r32[o + pc] = f1;
    r32[o + pts + pc] = f2;
    if (r64 != nullptr) {
      r64[o + pc] = make_double2(df_to_d(DF{f1.x, l1.x}), df_to_d(DF{f1.y, l1.y}));
      r64[o + pts + pc] = make_double2(df_to_d(DF{f2.x, l2.x}), df_to_d(DF{f2.y, l2.y}));
    }
    rr = fmaf(f1.x, f1.x, fmaf(f1.y, f1.y, fmaf(f2.x, f2.x, fmaf(f2.y, f2.y, rr))));
  }
  double acc[1] = {(double)rr};
  block_sum<1>(acc);
  if (threadIdx.x == 0) partials[(j * kDotSlots + 0) * kDotBlocks + blockIdx.x] = make_double2(acc[0], 0.0);
}

// New right-hand side plus the initial outer residual of the step without a
// stencil: with the previous step's final residual r_prev = b_prev - A x0,
// r0 = b - A x0 = b - b_prev + r_prev (exact algebra, pointwise).  Writes b
// (eta-parts, the nearest doubles), r0 as FP32, and partials ||r0||^2, ||b||^2.
// Triangular lattice (closed-form N_j), without the FP64 pipe: amplitudes, b_prev
// and r_prev are split into FP32 pairs by integer operations and rhs_j = eta_j/dt -
// kap_j N_j(eta) and r0 are formed in double-float arithmetic (about 2^-44
// relative per operation, dfloat.cuh).
// 384 threads per block: the kernel keeps one partial-sum slot per block (kDotBlocks blocks),
// and 12 warps per block, with registers capped for two blocks per SM (80; uncapped it took
// 95 and ran 16% slower at one block), give each SM 24 resident warps to overlap its loads.
constexpr int kRhsThreads = 384;
__global__ void __launch_bounds__(kRhsThreads, 2) k_rhs_resid_hex(const double2* __restrict__ x, double2* __restrict__ b,
                                                       const double2* __restrict__ b_prev,
                                                       const double2* __restrict__ r_prev, float2* __restrict__ r32,
                                                       double2* __restrict__ partials, const __grid_constant__ OpCoef c,
                                                       const __grid_constant__ NonlinTable nt, const RunGeom* rg) {
  long long pts = c.pts;
  if (rg != nullptr) {  // batched runs: blockIdx.y selects the run
    const RunGeom& q = rg[blockIdx.y];
    pts = q.pts;
    x += q.elem_off;
    b += q.elem_off;
    if (b_prev != nullptr) {  // null: no previous step (kept null, not offset)
      b_prev += q.elem_off;
      r_prev += q.elem_off;
    }
    r32 += q.elem_off;
    partials += (long long)blockIdx.y * 3 * kDotSlots * kDotBlocks;
  }
  if (c.prof != nullptr && blockIdx.x == 0 && threadIdx.x == 0)
    atomicAdd(c.prof + KID_RHS, 3ull * pts * (b_prev ? 5 * sizeof(double2) + 2 * sizeof(float2) : 2 * sizeof(double2)));
  const DF v3 = split_d(3.0 * nt.v), t2 = split_d(2.0 * nt.t), idt = split_d(c.inv_dt);
  DF kap[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) kap[j] = split_d(c.kap[j]);
  float accf[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) accf[i] = 0.f;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < pts;
       p += (long long)gridDim.x * blockDim.x) {
    CDF eta[3];
    DF m2[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      eta[j] = cdf_split(x[(2LL * j + 1) * pts + p]);
      m2[j] = cdf_abs2(eta[j]);
    }
    const DF A2 = df_scale2(df_add(df_add(m2[0], m2[1]), m2[2]));
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      // N_j = 3v (A^2 - |eta_j|^2) eta_j - 2t conj(eta_k eta_l)
      const int k1 = j == 2 ? 0 : j + 1, k2 = j == 0 ? 2 : j - 1;
      const DF sj = df_mul(v3, df_sub(A2, m2[j]));
      const CDF N = cdf_sub(cdf_scale(sj, eta[j]), cdf_scale(t2, cdf_conj(cdf_mul(eta[k1], eta[k2]))));
      const CDF bn = cdf_sub(cdf_scale(idt, eta[j]), cdf_scale(kap[j], N));
      const long long q1 = 2LL * j * pts + p, q2 = q1 + pts;
      b[q2] = cdf_to_d(bn);
      if (b_prev != nullptr) {  // without a previous step: b and ||b||^2 only (r0 by stencil)
        const CDF r2 = cdf_add(cdf_sub(bn, cdf_split(b_prev[q2])), cdf_split(r_prev[q2]));
        const DF p1x = split_d(r_prev[q1].x), p1y = split_d(r_prev[q1].y);
        const float2 f1 = make_float2(__fadd_rn(p1x.h, p1x.l), __fadd_rn(p1y.h, p1y.l));
        const float2 f2 = make_float2(r2.x.h, r2.y.h);
        r32[q1] = f1;
        r32[q2] = f2;
        // norms only decide convergence: accumulated from FP32-rounded values
        accf[2 * j] = fmaf(f1.x, f1.x, fmaf(f1.y, f1.y, fmaf(f2.x, f2.x, fmaf(f2.y, f2.y, accf[2 * j]))));
      }
      accf[2 * j + 1] = fmaf(bn.x.h, bn.x.h, fmaf(bn.y.h, bn.y.h, accf[2 * j + 1]));
    }
  }
  __shared__ double sh[6][kRhsThreads / 32];
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    double v = (double)accf[i];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (l == 0) sh[i][w] = v;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    double v = 0.0;
    for (int k = 0; k < kRhsThreads / 32; ++k) v += sh[threadIdx.x][k];
    const int j = threadIdx.x >> 1, which = threadIdx.x & 1;
    partials[(j * kDotSlots + which) * kDotBlocks + blockIdx.x] = make_double2(v, 0.0);
  }
}

// Table lattices (bcc, custom), the same (new right-hand side and r0 = rhs - b_prev +
// r_prev) without the FP64 pipe: rhs_j = eta_j/dt -
// kap_j N_j(eta) with N_j = eta_j sum_m wdiag[j][m] |eta_m|^2 + the remaining resonance
// monomials (coefficient times a product of amplitudes and conjugates), all in
// double-float arithmetic (about 2^-44 relative per operation,
// dfloat.cuh).  The split amplitudes of a point sit in shared memory (the table indexes
// them at run time), the table's coefficients as FP32 pairs too.
__global__ void __launch_bounds__(256) k_rhs_resid_tab(const double2* __restrict__ x, double2* __restrict__ b,
                                                       const double2* __restrict__ b_prev,
                                                       const double2* __restrict__ r_prev, float2* __restrict__ r32,
                                                       double2* __restrict__ partials, const __grid_constant__ OpCoef c,
                                                       const __grid_constant__ NonlinTable nt, const RunGeom* rg) {
  long long pts = c.pts;
  if (rg != nullptr) {  // batched runs: blockIdx.y selects the run
    const RunGeom& q = rg[blockIdx.y];
    pts = q.pts;
    x += q.elem_off;
    b += q.elem_off;
    if (b_prev != nullptr) {  // null: no previous step (kept null, not offset)
      b_prev += q.elem_off;
      r_prev += q.elem_off;
    }
    r32 += q.elem_off;
    partials += (long long)blockIdx.y * c.J * kDotSlots * kDotBlocks;
  }
  const int J = c.J, t = threadIdx.x;
  if (c.prof != nullptr && blockIdx.x == 0 && t == 0)
    atomicAdd(c.prof + KID_RHS, (unsigned long long)J * pts *
                                    (b_prev ? 5 * sizeof(double2) + 2 * sizeof(float2) : 2 * sizeof(double2)));
  __shared__ float4 se4[kMaxJ][kThreads];  // split amplitudes of each thread's point (re h, re l, im h, im l)
  __shared__ float2 sn2[kMaxJ][kThreads];  // |eta_m|^2 as (h, l)
  __shared__ float2 swd[kMaxJ][kMaxJ];
  __shared__ float2 scf[kMaxTerms];
  __shared__ float2 skap[kMaxJ];
  for (int i = t; i < J * J; i += blockDim.x) {
    const DF d = split_d(nt.wdiag[i / J][i % J]);
    swd[i / J][i % J] = make_float2(d.h, d.l);
  }
  for (int i = t; i < kMaxTerms; i += blockDim.x) {
    const DF d = split_d(nt.coef[i]);
    scf[i] = make_float2(d.h, d.l);
  }
  if (t < J) {
    const DF d = split_d(c.kap[t]);
    skap[t] = make_float2(d.h, d.l);
  }
  __syncthreads();
  const DF idt = split_d(c.inv_dt);
  auto eta_of = [&](int code) {  // amplitude code >> 1, conjugated if code & 1
    const float4 v = se4[code >> 1][t];
    return (code & 1) ? CDF{DF{v.x, v.y}, DF{-v.z, -v.w}} : CDF{DF{v.x, v.y}, DF{v.z, v.w}};
  };
  float accf[2 * kMaxJ];
#pragma unroll
  for (int i = 0; i < 2 * kMaxJ; ++i) accf[i] = 0.f;
  for (long long p = (long long)blockIdx.x * blockDim.x + t; p < pts; p += (long long)gridDim.x * blockDim.x) {
    for (int m = 0; m < J; ++m) {
      const CDF e = cdf_split(x[(2LL * m + 1) * pts + p]);
      se4[m][t] = make_float4(e.x.h, e.x.l, e.y.h, e.y.l);
      const DF a = cdf_abs2(e);
      sn2[m][t] = make_float2(a.h, a.l);
    }
#pragma unroll
    for (int j = 0; j < kMaxJ; ++j) {
      if (j >= J) break;
      DF w{0.f, 0.f};
      for (int m = 0; m < J; ++m) {
        const float2 wd = swd[j][m], n2 = sn2[m][t];
        w = df_add(w, df_mul(DF{wd.x, wd.y}, DF{n2.x, n2.y}));
      }
      const CDF ej = eta_of(2 * j);
      CDF N = cdf_scale(w, ej);
      for (int i = nt.rstart[j]; i < nt.rstart[j + 1]; ++i) {
        const int q = nt.ridx[i];
        const float2 cf = scf[q];
        CDF prod = cdf_scale(DF{cf.x, cf.y}, eta_of(nt.f[q][0]));
        for (int f = 1; f < nt.nf[q]; ++f) prod = cdf_mul(prod, eta_of(nt.f[q][f]));
        N = cdf_add(N, prod);
      }
      const float2 kp = skap[j];
      const CDF bn = cdf_sub(cdf_scale(idt, ej), cdf_scale(DF{kp.x, kp.y}, N));
      const long long q1 = 2LL * j * pts + p, q2 = q1 + pts;
      b[q2] = cdf_to_d(bn);
      if (b_prev != nullptr) {  // without a previous step: b and ||b||^2 only (r0 by stencil)
        const CDF r2 = cdf_add(cdf_sub(bn, cdf_split(b_prev[q2])), cdf_split(r_prev[q2]));
        const DF p1x = split_d(r_prev[q1].x), p1y = split_d(r_prev[q1].y);
        const float2 f1 = make_float2(__fadd_rn(p1x.h, p1x.l), __fadd_rn(p1y.h, p1y.l));
        const float2 f2 = make_float2(r2.x.h, r2.y.h);
        r32[q1] = f1;
        r32[q2] = f2;
        // norms only decide convergence: accumulated from FP32-rounded values
        accf[2 * j] = fmaf(f1.x, f1.x, fmaf(f1.y, f1.y, fmaf(f2.x, f2.x, fmaf(f2.y, f2.y, accf[2 * j]))));
      }
      accf[2 * j + 1] = fmaf(bn.x.h, bn.x.h, fmaf(bn.y.h, bn.y.h, accf[2 * j + 1]));
    }
  }
  __shared__ double sh[2 * kMaxJ][kThreads / 32];
  const int w = t >> 5, l = t & 31;
  for (int i = 0; i < 2 * J; ++i) {
    double v = (double)accf[i];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (l == 0) sh[i][w] = v;
  }
  __syncthreads();
  if (t < 2 * J) {
    double v = 0.0;
    for (int k = 0; k < kThreads / 32; ++k) v += sh[t][k];
    const int j = t >> 1, which = t & 1;
    partials[(j * kDotSlots + which) * kDotBlocks + blockIdx.x] = make_double2(v, 0.0);
  }
}

// Energy density summed per block.
__global__ void k_energy(const double2* __restrict__ x, double* __restrict__ partials, OpCoef c, EnergyTable et,
                         double Bx) {
  prof_add(c, KID_ENERGY, (unsigned long long)c.J * c.pts * sizeof(double2));
  double acc[1] = {0.0};
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < c.pts;
       p += (long long)gridDim.x * blockDim.x) {
    const Nb n = neighbours(p, c);
    double2 eta[kMaxJ];
    double S2 = 0.0, S4 = 0.0, grad = 0.0;
    for (int j = 0; j < c.J; ++j) {
      const double2* e = x + (2LL * j + 1) * c.pts;
      eta[j] = e[p];
      const double m2 = eta[j].x * eta[j].x + eta[j].y * eta[j].y;
      S2 += m2;
      S4 += m2 * m2;
      const double2 g = opG<double>(e, n, c, j);
      grad += g.x * g.x + g.y * g.y;
    }
    const double A2 = 2.0 * S2;
    double f = 0.5 * et.dB * A2;
    if (et.hex) {
      const double2 cub = cm(cm(eta[0], eta[1]), eta[2]);
      f += 0.75 * et.v * A2 * A2 - 1.5 * et.v * S4 - 4.0 * et.t * cub.x;
    } else {
      for (int q = 0; q < et.ne; ++q) {
        double2 prod = make_double2(et.coef[q], 0.0);
        for (int ff = 0; ff < et.nf[q]; ++ff) {
          const int code = et.f[q][ff];
          prod = cm(prod, (code & 1) ? cconj(eta[code >> 1]) : eta[code >> 1]);
        }
        f += prod.x;
      }
    }
    acc[0] += f + Bx * grad;
  }
  block_sum<1>(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc[0];
}

__global__ void k_sum_partials(const double* __restrict__ partials, int n, double* __restrict__ out) {
  double acc[1] = {0.0};
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc[0] += partials[i];
  block_sum<1>(acc);
  if (threadIdx.x == 0) out[0] = acc[0];
}

inline dim3 grid_pts3(const OpCoef& c) {
  return dim3((unsigned)((c.nx + 31) / 32), (unsigned)((c.ny + 7) / 8), (unsigned)(c.nz * c.J));
}



// ---------------------------------------------------------------------------
// Adjoint of the step (real-gradient convention: grad = dL/dRe + i dL/dIm)
// ---------------------------------------------------------------------------

// N_j(eta) at one point (closed form on the triangular lattice, else the table).
__device__ __forceinline__ double2 nonlin_at(const double2* eta, int j, const OpCoef& c, const NonlinTable& nt) {
  if (nt.hex) {
    double A2 = 0.0;
    for (int m = 0; m < 3; ++m) A2 += eta[m].x * eta[m].x + eta[m].y * eta[m].y;
    A2 *= 2.0;
    const int k1 = (j + 1) % 3, k2 = (j + 2) % 3;
    const double m2 = eta[j].x * eta[j].x + eta[j].y * eta[j].y;
    const double s = 3.0 * nt.v * (A2 - m2);
    const double2 pr = cconj(cm(eta[k1], eta[k2]));
    return make_double2(s * eta[j].x - 2.0 * nt.t * pr.x, s * eta[j].y - 2.0 * nt.t * pr.y);
  }
  double2 N = make_double2(0.0, 0.0);
  for (int q = nt.start[j]; q < nt.start[j + 1]; ++q) {
    double2 prod = make_double2(nt.coef[q], 0.0);
    for (int f = 0; f < nt.nf[q]; ++f) {
      const int code = nt.f[q][f];
      prod = cm(prod, (code & 1) ? cconj(eta[code >> 1]) : eta[code >> 1]);
    }
    N.x += prod.x;
    N.y += prod.y;
  }
  return N;
}

__device__ __forceinline__ double2 cadd2(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub2(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

// out_k -= sum_j [w_j conj(dN_j/deta_k) + conj(w_j) dN_j/dconj(eta_k)] at one point.
__device__ __forceinline__ void nonlin_vjp_sub(const double2* eta, const double2* w, double2* out, const OpCoef& c,
                                               const NonlinTable& nt) {
  if (nt.hex) {
    double A2 = 0.0;
    for (int m = 0; m < 3; ++m) A2 += eta[m].x * eta[m].x + eta[m].y * eta[m].y;
    A2 *= 2.0;
    for (int j = 0; j < 3; ++j) {
      // dN_j/deta_j = 3v A^2 (real), dN_j/dconj(eta_j) = 3v eta_j^2
      const double a = 3.0 * nt.v * A2;
      const double2 e2 = cm(eta[j], eta[j]);
      const double2 b = make_double2(3.0 * nt.v * e2.x, 3.0 * nt.v * e2.y);
      out[j] = csub2(out[j], cadd2(make_double2(a * w[j].x, a * w[j].y), cm(cconj(w[j]), b)));
      for (int m = 0; m < 3; ++m) {
        if (m == j) continue;
        const int o = 3 - j - m;
        // dN_j/deta_m = 6v eta_j conj(eta_m); dN_j/dconj(eta_m) = 6v eta_j eta_m - 2t conj(eta_o)
        const double2 am = cm(eta[j], cconj(eta[m]));
        const double2 em = cm(eta[j], eta[m]);
        const double2 a6 = make_double2(6.0 * nt.v * am.x, 6.0 * nt.v * am.y);
        const double2 b6 = make_double2(6.0 * nt.v * em.x - 2.0 * nt.t * eta[o].x, 6.0 * nt.v * em.y + 2.0 * nt.t * eta[o].y);
        out[m] = csub2(out[m], cadd2(cm(w[j], cconj(a6)), cm(cconj(w[j]), b6)));
      }
    }
    return;
  }
  for (int j = 0; j < c.J; ++j) {
    for (int q = nt.start[j]; q < nt.start[j + 1]; ++q) {
      for (int f = 0; f < nt.nf[q]; ++f) {
        double2 d = make_double2(nt.coef[q], 0.0);  // derivative of the term by its factor f
        for (int g = 0; g < nt.nf[q]; ++g) {
          if (g == f) continue;
          const int code = nt.f[q][g];
          d = cm(d, (code & 1) ? cconj(eta[code >> 1]) : eta[code >> 1]);
        }
        const int code = nt.f[q][f], cf = code >> 1;
        out[cf] = csub2(out[cf], (code & 1) ? cm(cconj(w[j]), d) : cm(w[j], cconj(d)));
      }
    }
  }
}


// D_j = dN_j/d eta_j at one point (the Jacobian of Alg. 1 in direction eta_j): 3v A^2 on the
// triangular lattice, else the derivative of every table monomial by its unconjugated
// eta_j factors.  The exact value is real (a mixed second derivative of the real bulk
// density); the real part is returned.
__device__ __forceinline__ double jac_diag_at(const double2* eta, int j, const OpCoef& c, const NonlinTable& nt) {
  if (nt.hex) {
    double A2 = 0.0;
    for (int m = 0; m < 3; ++m) A2 += eta[m].x * eta[m].x + eta[m].y * eta[m].y;
    return 3.0 * nt.v * 2.0 * A2;
  }
  double2 D = make_double2(0.0, 0.0);
  for (int q = nt.start[j]; q < nt.start[j + 1]; ++q) {
    for (int f = 0; f < nt.nf[q]; ++f) {
      if (nt.f[q][f] != 2 * j) continue;  // an unconjugated eta_j factor
      double2 d = make_double2(nt.coef[q], 0.0);
      for (int g = 0; g < nt.nf[q]; ++g) {
        if (g == f) continue;
        const int code = nt.f[q][g];
        d = cm(d, (code & 1) ? cconj(eta[code >> 1]) : eta[code >> 1]);
      }
      D = cadd2(D, d);
    }
  }
  return D.x;
}

// Right-hand side of Picard iteration k (Alg. 1): from the previous iterate eta (the
// eta-parts of x), b_j = eta_prev_j/dt - kap_j (N_j - D_j eta_j) and jd_j = kap_j D_j
// (jd == nullptr: plain Picard, D = 0).
__global__ void k_rhs_picard(const double2* __restrict__ x, const double2* __restrict__ eta_prev,
                             double2* __restrict__ b, double* __restrict__ jd, float2* __restrict__ jd32, OpCoef c,
                             NonlinTable nt) {
  prof_add(c, KID_RHS, (unsigned long long)c.J * c.pts * (3 * sizeof(double2) + (jd ? sizeof(double) : 0)));
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < c.pts;
       p += (long long)gridDim.x * blockDim.x) {
    double2 eta[kMaxJ];
    for (int j = 0; j < c.J; ++j) eta[j] = x[(2LL * j + 1) * c.pts + p];
    for (int j = 0; j < c.J; ++j) {
      const double2 N = nonlin_at(eta, j, c, nt);
      const double D = jd != nullptr ? jac_diag_at(eta, j, c, nt) : 0.0;
      const double kap = c.kap[j];
      const double2 ep = eta_prev[j * c.pts + p];
      b[(2LL * j + 1) * c.pts + p] = make_double2(ep.x * c.inv_dt - kap * (N.x - D * eta[j].x),
                                                 ep.y * c.inv_dt - kap * (N.y - D * eta[j].y));
      if (jd != nullptr) jd[j * c.pts + p] = kap * D;
      if (jd32 != nullptr) jd32[j * c.pts + p] = make_float2((float)(kap * D), 0.f);
    }
  }
}

__global__ void k_adj_nonlin(const double2* __restrict__ eta0, const double2* __restrict__ xg,
                             const double2* __restrict__ eta1, double2* __restrict__ lam,
                             double* __restrict__ partials, OpCoef c, NonlinTable nt) {
  prof_add(c, KID_ADJ_NONLIN, 4ull * c.J * (unsigned long long)c.pts * sizeof(double2));
  double acc[1] = {0.0};
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < c.pts;
       p += (long long)gridDim.x * blockDim.x) {
    double2 e[kMaxJ], w[kMaxJ], out[kMaxJ];
    for (int j = 0; j < c.J; ++j) {
      e[j] = eta0[j * c.pts + p];
      const double2 g = xg[(2LL * j + 1) * c.pts + p];
      const double2 e1 = eta1[j * c.pts + p];
      acc[0] += c.kap[j] * (g.x * e1.x + g.y * e1.y);
      w[j] = make_double2(c.kap[j] * g.x, c.kap[j] * g.y);
      out[j] = make_double2(g.x * c.inv_dt, g.y * c.inv_dt);
    }
    nonlin_vjp_sub(e, w, out, c, nt);
    for (int j = 0; j < c.J; ++j) lam[j * c.pts + p] = out[j];
  }
  block_sum<1>(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc[0];
}

__global__ void k_energy_grad(const double2* __restrict__ x, double2* __restrict__ grad, double scale, double dB,
                              double Bx, double* __restrict__ partials, OpCoef c, NonlinTable nt) {
  prof_add(c, KID_ENERGY_GRAD, 3ull * c.J * (unsigned long long)c.pts * sizeof(double2));
  double acc[1] = {0.0};
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < c.pts;
       p += (long long)gridDim.x * blockDim.x) {
    const Nb n = neighbours(p, c);
    double2 e[kMaxJ];
    for (int j = 0; j < c.J; ++j) {
      e[j] = x[(2LL * j + 1) * c.pts + p];
      acc[0] += e[j].x * e[j].x + e[j].y * e[j].y;
    }
    for (int j = 0; j < c.J; ++j) {
      const double2 gz = opG<double>(x + 2LL * j * c.pts, n, c, j);
      const double2 N = nonlin_at(e, j, c, nt);
      grad[j * c.pts + p] = make_double2(scale * (dB * e[j].x + Bx * gz.x + N.x), scale * (dB * e[j].y + Bx * gz.y + N.y));
    }
  }
  block_sum<1>(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc[0];
}


// ---------------------------------------------------------------------------
// Rotation diagnostic and adaptivity map (Sec. II.D, Eqs. rot and hhh)
// ---------------------------------------------------------------------------
// One thread per point on a (32 x 8)-point tile grid with z in blockIdx.z.  A = sqrt(2
// sum |eta_j|^2) is formed once per point of the tile and its one-point (x, y) halo in
// shared memory (FP64: A and |grad A| decide the branches of Eq. hhh); z-neighbours
// in 3D are formed directly.  The phases go through FP32: eta converted on load, the
// product a conj(b) and atan2f in FP32 (about 1e-7 rad per difference), the weighted
// sums and omega in FP32.  The branches compare squares: |grad A|^2 >= eps^2 and
// A^2 > A_min^2.
__device__ __forceinline__ double amp_at(const double2* __restrict__ x, long long q, const OpCoef& c) {
  double s2 = 0.0;
  for (int j = 0; j < c.J; ++j) {
    const double2 e = x[(2LL * j + 1) * c.pts + q];
    s2 = fma(e.x, e.x, fma(e.y, e.y, s2));
  }
  return sqrt(2.0 * s2);
}

__global__ void __launch_bounds__(256) k_rotation(const double2* __restrict__ x, double* __restrict__ omega,
                                                  double* __restrict__ amp, double* __restrict__ hmap, RotParams rp,
                                                  OpCoef c) {
  if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0)
    prof_add(c, KID_ROTATION,
             (unsigned long long)c.pts * (c.J * sizeof(double2) + (c.dim == 2 ? 3 : 5) * sizeof(double)));
  __shared__ double sA[10][34];  // A on the tile plus a one-point (x, y) halo
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int x0 = blockIdx.x * 32, y0 = blockIdx.y * 8, zz = blockIdx.z;
  const long long plane = (long long)c.nx * c.ny, zoff = (long long)zz * plane;
  const bool want_h = hmap != nullptr;
  if (want_h || amp != nullptr) {
    for (int i = threadIdx.x; i < 10 * 34; i += 256) {
      const int ly = i / 34, lx = i - ly * 34;
      // periodic wrap (the halo of a partial tile can lie several points past a small grid)
      const int gx = ((x0 + lx - 1) % c.nx + c.nx) % c.nx, gy = ((y0 + ly - 1) % c.ny + c.ny) % c.ny;
      sA[ly][lx] = amp_at(x, zoff + (long long)gy * c.nx + gx, c);
    }
    __syncthreads();
  }
  const int xx = x0 + tx, yy = y0 + ty;
  if (xx >= c.nx || yy >= c.ny) return;
  const int dim = c.dim;
  const long long p = zoff + (long long)yy * c.nx + xx;
  long long nbp[3], nbm[3];
  nbp[0] = xx + 1 == c.nx ? p - xx : p + 1;
  nbm[0] = xx == 0 ? p + c.nx - 1 : p - 1;
  nbp[1] = yy + 1 == c.ny ? p - (long long)yy * c.nx : p + c.nx;
  nbm[1] = yy == 0 ? p + (long long)(c.ny - 1) * c.nx : p - c.nx;
  nbp[2] = zz + 1 == c.nz ? p - zoff : p + plane;
  nbm[2] = zz == 0 ? p + (long long)(c.nz - 1) * plane : p - plane;
  float du[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  bool ok = true;
  for (int j = 0; j < c.J; ++j) {
    const double2* e = x + (2LL * j + 1) * c.pts;
    const double2 ec = e[p];
    ok = ok && (ec.x * ec.x + ec.y * ec.y >= rp.amp_floor);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (d >= dim) break;
      const double2 ad = e[nbp[d]], bd = e[nbm[d]];
      const float ax = (float)ad.x, ay = (float)ad.y, bx = (float)bd.x, by = (float)bd.y;
      // arg(a conj(b)): central difference of the unwrapped phase
      const float g = atan2f(ay * bx - ax * by, ax * bx + ay * by) * rp.inv2h[d];
#pragma unroll
      for (int i = 0; i < 3; ++i)
        if (i < dim) du[i][d] += rp.Wf[j][i] * g;
    }
  }
  float om[3];
  int nc;
  if (dim == 2) {
    om[0] = 0.5f * (du[0][1] - du[1][0]);
    nc = 1;
  } else {
    om[0] = 0.5f * (du[1][2] - du[2][1]);
    om[1] = 0.5f * (du[2][0] - du[0][2]);
    om[2] = 0.5f * (du[0][1] - du[1][0]);
    nc = 3;
  }
  float wmax = 0.0f;
  for (int q = 0; q < nc; ++q) {
    if (!ok) om[q] = 0.0f;
    omega[q * c.pts + p] = (double)om[q];
    wmax = fmaxf(wmax, fabsf(om[q]));
  }
  if (!want_h && amp == nullptr) return;
  const double A = sA[ty + 1][tx + 1];
  if (amp != nullptr) amp[p] = A;
  if (want_h) {
    double gxA = (sA[ty + 1][tx + 2] - sA[ty + 1][tx]) * rp.inv2hd[0];
    double gyA = (sA[ty + 2][tx + 1] - sA[ty][tx + 1]) * rp.inv2hd[1];
    double g2 = gxA * gxA + gyA * gyA;
    if (dim == 3) {
      const double gzA = (amp_at(x, nbp[2], c) - amp_at(x, nbm[2], c)) * rp.inv2hd[2];
      g2 += gzA * gzA;
    }
    double hv;
    if (g2 >= rp.eps * rp.eps) {
      hv = rp.h_int;
    } else if (rp.A_min < 0.0 || A * A > rp.A_min * rp.A_min) {
      // theta = asin(w); sin(theta/2) = w / sqrt(2 (1 + cos(theta)))
      const float w = fminf(wmax, 1.0f);
      const float s = w / sqrtf(2.0f * (1.0f + sqrtf(1.0f - w * w)));
      const double h_amp = s > 0.0f ? rp.pi_over_nk / (double)s : INFINITY;
      hv = fmin(fmax(h_amp, rp.h_int), rp.h_max);
    } else {
      hv = rp.h_max;
    }
    hmap[p] = hv;
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// Launch wrappers
// ---------------------------------------------------------------------------
template <typename T>
void launch_apply_A(const cplx<T>* x, cplx<T>* y, const OpCoef& c, const KScal* act, cudaStream_t s) {
  if (c.dim == 3) {
    launch3d_apply_A<T>(x, y, c, act, s);
    return;
  }
  ProfScope ps_(kid_of<T>(KID_APPLY_A), s);
  k_apply_A<T><<<grid_pts3(c), kThreads, 0, s>>>(x, y, c, act);
}
template <typename T>
void launch_residual(const cplx<T>* b, const cplx<T>* x, cplx<T>* r, cplx<T>* rhat, const OpCoef& c, cudaStream_t s) {
  if (c.dim == 3) {
    launch3d_residual<T>(b, x, r, rhat, c, s);
    return;
  }
  ProfScope ps_(kid_of<T>(KID_RESIDUAL), s);
  k_residual<T><<<grid_pts3(c), kThreads, 0, s>>>(b, x, r, rhat, c);
}
template <typename T>
void launch_pc_rhs(const cplx<T>* beta, FieldRef<T> f, const OpCoef& c, const KScal* act, cudaStream_t s) {
  if (c.dim == 3) {
    launch3d_pc_rhs<T>(beta, f, c, act, s);
    return;
  }
  ProfScope ps_(kid_of<T>(KID_PC_RHS), s);
  k_pc_rhs<T><<<grid_pts3(c), kThreads, 0, s>>>(beta, f, c, act);
}
template <typename T>
void launch_cheb_zero(CFieldRef<T> f, FieldRef<T> X, const OpCoef& c, const KScal* act, cudaStream_t s) {
  ProfScope ps_(kid_of<T>(KID_CHEB_ZERO), s);
  k_cheb_zero<T><<<grid_pts3(c), kThreads, 0, s>>>(f, X, c, act);
}
template <typename T>
void launch_pc_final(const cplx<T>* beta, CFieldRef<T> b2p, cplx<T>* chi, const OpCoef& c, const KScal* act,
                     cudaStream_t s) {
  ProfScope ps_(kid_of<T>(KID_PC_FINAL), s);
  k_pc_final<T><<<grid_pts3(c), kThreads, 0, s>>>(beta, b2p, chi, c, act);
}
template <typename T>
void launch_cheb_first(CFieldRef<T> f, FieldRef<T> X, FieldRef<T> R, FieldRef<T> Dn, const ChebStep& w, int last,
                       const OpCoef& c, const KScal* act, cudaStream_t s, const PcFin<T>* fin) {
  const bool fold = fin != nullptr && last;
  if (c.dim == 3) {
    launch3d_cheb_first<T>(f, X, R, Dn, w, last, c, act, s, fold ? fin : nullptr);
    return;
  }
  {
    ProfScope ps_(kid_of<T>(KID_CHEB_FIRST), s);
    k_cheb_first<T><<<grid_pts3(c), kThreads, 0, s>>>(f, X, R, Dn, w, last, c, act);
  }
  if (fold) launch_pc_final<T>(fin->b1.p, fin->b2p, fin->chi1.p, c, act, s);
}
template <typename T>
void launch_cheb_sweep(CFieldRef<T> Dd, FieldRef<T> X, FieldRef<T> R, FieldRef<T> Dn, const ChebStep& w, int last,
                       const OpCoef& c, const KScal* act, cudaStream_t s, const PcFin<T>* fin) {
  const bool fold = fin != nullptr && last;
  if (c.dim == 3) {
    launch3d_cheb_sweep<T>(Dd, X, R, Dn, w, last, c, act, s, fold ? fin : nullptr);
    return;
  }
  {
    ProfScope ps_(kid_of<T>(KID_CHEB_SWEEP), s);
    k_cheb_sweep<T><<<grid_pts3(c), kThreads, 0, s>>>(Dd, X, R, Dn, w, last, c, act);
  }
  if (fold) launch_pc_final<T>(fin->b1.p, fin->b2p, fin->chi1.p, c, act, s);
}
template <typename T>
void launch_p_update(const cplx<T>* r, cplx<T>* p, const cplx<T>* v, const OpCoef& c, const KScal* k, cudaStream_t s) {
  ProfScope ps_(kid_of<T>(KID_P_UPDATE), s);
  k_p_update<T><<<dim3(kDotBlocks, c.J), kThreads, 0, s>>>(r, p, v, c, k);
}
template <typename T>
void launch_s_update(cplx<T>* r, const cplx<T>* v, const OpCoef& c, const KScal* k, cudaStream_t s, void* partials) {
  ProfScope ps_(kid_of<T>(KID_S_UPDATE), s);
  k_s_update<T><<<dim3(kDotBlocks, c.J), kThreads, 0, s>>>(r, v, c, k, partials);
}
template <typename T>
void launch_r_update(cplx<T>* r, const cplx<T>* t, cplx<T>* u, const cplx<T>* p, const OpCoef& c, const KScal* k,
                     cudaStream_t s, const cplx<T>* rhat, void* partials) {
  ProfScope ps_(kid_of<T>(KID_R_UPDATE), s);
  k_r_update<T><<<dim3(kDotBlocks, c.J), kThreads, 0, s>>>(r, t, u, p, rhat, c, k, partials);
}
template <typename T>
void launch_add_to(const cplx<T>* d, double2* x, const OpCoef& c, cudaStream_t s) {
  const long long n = 2LL * c.J * c.pts;
  ProfScope ps_(kid_of<T>(KID_ADD_TO), s);
  k_add_to<T><<<(unsigned)((n + kThreads - 1) / kThreads), kThreads, 0, s>>>(d, x, n, c);
}

void launch_rhs(const double2* x, double2* b, const OpCoef& c, const NonlinTable& nt, cudaStream_t s,
                const BatchLaunch* bl) {
  ProfScope ps_(KID_RHS, s);
  // batched: c.pts is the largest run's point count
  const dim3 g((unsigned)((c.pts + kThreads - 1) / kThreads), bl ? bl->R : 1);
  k_rhs<<<g, kThreads, 0, s>>>(x, b, c, nt, bl ? bl->dev : nullptr);
}
// complex64 amplitudes [J][pts] <-> part `part` of the FP64 state block [J][2][pts]
__global__ void k_c64_to_part(const float2* __restrict__ src, double2* __restrict__ x, long long pts, int J,
                              int part) {
  const long long n = (long long)J * pts;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long j = i / pts, p = i - j * pts;
    const float2 v = src[i];
    x[(2 * j + part) * pts + p] = make_double2((double)v.x, (double)v.y);
  }
}
__global__ void k_part_to_c64(const double2* __restrict__ x, float2* __restrict__ dst, long long pts, int J,
                              int part) {
  const long long n = (long long)J * pts;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long j = i / pts, p = i - j * pts;
    const double2 v = x[(2 * j + part) * pts + p];
    dst[i] = make_float2(__double2float_rn(v.x), __double2float_rn(v.y));
  }
}
void launch_c64_to_part(const float2* src, double2* x, long long pts, int J, int part, cudaStream_t s) {
  k_c64_to_part<<<4 * kDotBlocks, kThreads, 0, s>>>(src, x, pts, J, part);
}
void launch_part_to_c64(const double2* x, float2* dst, long long pts, int J, int part, cudaStream_t s) {
  k_part_to_c64<<<4 * kDotBlocks, kThreads, 0, s>>>(x, dst, pts, J, part);
}

// Linear extrapolation of the state history: x <- 2 x - xp (the next solve's initial
// guess) and xp <- x (the state it came from), elementwise over n complex values.
__global__ void k_extrapolate(double2* __restrict__ x, double2* __restrict__ xp, long long n, OpCoef c) {
  prof_add(c, KID_EXTRAP, (unsigned long long)n * 4 * sizeof(double2));
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double2 a = x[i], b = xp[i];
    xp[i] = a;
    x[i] = make_double2(fma(2.0, a.x, -b.x), fma(2.0, a.y, -b.y));
  }
}
void launch_extrapolate(double2* x, double2* xp, const OpCoef& c, cudaStream_t s) {
  ProfScope ps_(KID_EXTRAP, s);
  k_extrapolate<<<4 * kDotBlocks, kThreads, 0, s>>>(x, xp, 2LL * c.J * c.pts, c);
}

void launch_zeta(double2* x, const OpCoef& c, cudaStream_t s) {
  if (c.dim == 3) {
    launch3d_zeta(x, c, s);
    return;
  }
  ProfScope ps_(KID_ZETA, s);
  k_zeta<2><<<grid_pts3(c), kThreads, 0, s>>>(x, c);
}
void launch_residual_refine(const double2* b, const double2* x, float2* r32, double* partials, const OpCoef& c,
                            cudaStream_t s) {
  ProfScope ps_(KID_RESID_REFINE, s);
  k_residual_refine<<<dim3(kDotBlocks, c.J), kThreads, 0, s>>>(b, x, r32, reinterpret_cast<double2*>(partials), c);
}
void launch_residual_refine2d(const double2* b, const double2* x, float2* r32, double2* r64, double* partials,
                              const OpCoef& c, cudaStream_t s, const BatchLaunch* bl) {
  ProfScope ps_(KID_RESID_REFINE, s);
  k_residual_refine2d<<<dim3(kDotBlocks, c.J, bl ? bl->R : 1), 256, 0, s>>>(
      b, x, r32, r64, reinterpret_cast<double2*>(partials), c, bl ? bl->dev : nullptr);
}
void launch_rhs_resid(const double2* x, double2* b, const double2* b_prev, const double2* r_prev, float2* r32,
                      double* partials, const OpCoef& c, const NonlinTable& nt, cudaStream_t s,
                      const BatchLaunch* bl) {
  ProfScope ps_(KID_RHS, s);
  if (nt.hex) {
    k_rhs_resid_hex<<<dim3(kDotBlocks, bl ? bl->R : 1), kRhsThreads, 0, s>>>(
        x, b, b_prev, r_prev, r32, reinterpret_cast<double2*>(partials), c, nt, bl ? bl->dev : nullptr);
    return;
  }
  k_rhs_resid_tab<<<dim3(kDotBlocks, bl ? bl->R : 1), kThreads, 0, s>>>(
      x, b, b_prev, r_prev, r32, reinterpret_cast<double2*>(partials), c, nt, bl ? bl->dev : nullptr);
}
void launch_energy(const double2* x, double* partials, double* out, const OpCoef& c, const EnergyTable& et, double Bx,
                   cudaStream_t s) {
  ProfScope ps_(KID_ENERGY, s);
  k_energy<<<kDotBlocks, kThreads, 0, s>>>(x, partials, c, et, Bx);
  k_sum_partials<<<1, kThreads, 0, s>>>(partials, kDotBlocks, out);
}

void launch_adj_nonlin(const double2* eta0, const double2* xg, const double2* eta1, double2* lam, double* partials,
                       double* out, const OpCoef& c, const NonlinTable& nt, cudaStream_t s) {
  ProfScope ps_(KID_ADJ_NONLIN, s);
  k_adj_nonlin<<<kDotBlocks, kThreads, 0, s>>>(eta0, xg, eta1, lam, partials, c, nt);
  k_sum_partials<<<1, kThreads, 0, s>>>(partials, kDotBlocks, out);
}
void launch_energy_grad(const double2* x, double2* grad, double scale, double dB, double Bx, double* partials,
                        double* out, const OpCoef& c, const NonlinTable& nt, cudaStream_t s) {
  ProfScope ps_(KID_ENERGY_GRAD, s);
  k_energy_grad<<<kDotBlocks, kThreads, 0, s>>>(x, grad, scale, dB, Bx, partials, c, nt);
  k_sum_partials<<<1, kThreads, 0, s>>>(partials, kDotBlocks, out);
}

void launch_rotation(const double2* x, double* omega, double* amp, double* hmap, const RotParams& rp,
                     const OpCoef& c, cudaStream_t s) {
  ProfScope ps_(KID_ROTATION, s);
  const dim3 g((unsigned)((c.nx + 31) / 32), (unsigned)((c.ny + 7) / 8), (unsigned)(c.dim == 3 ? c.nz : 1));
  k_rotation<<<g, 256, 0, s>>>(x, omega, amp, hmap, rp, c);
}
void launch_rhs_picard(const double2* x, const double2* eta_prev, double2* b, double* jd, float2* jd32,
                       const OpCoef& c, const NonlinTable& nt, cudaStream_t s) {
  ProfScope ps_(KID_RHS, s);
  k_rhs_picard<<<(unsigned)std::min<long long>((c.pts + kThreads - 1) / kThreads, 8 * kDotBlocks), kThreads, 0, s>>>(
      x, eta_prev, b, jd, jd32, c, nt);
}
#define APFC_INST(T)                                                                                                 \
  template void launch_apply_A<T>(const cplx<T>*, cplx<T>*, const OpCoef&, const KScal*, cudaStream_t);             \
  template void launch_residual<T>(const cplx<T>*, const cplx<T>*, cplx<T>*, cplx<T>*, const OpCoef&,               \
                                   cudaStream_t);                                                                   \
  template void launch_pc_rhs<T>(const cplx<T>*, FieldRef<T>, const OpCoef&, const KScal*, cudaStream_t);           \
  template void launch_cheb_zero<T>(CFieldRef<T>, FieldRef<T>, const OpCoef&, const KScal*, cudaStream_t);          \
  template void launch_cheb_first<T>(CFieldRef<T>, FieldRef<T>, FieldRef<T>, FieldRef<T>, const ChebStep&, int,     \
                                     const OpCoef&, const KScal*, cudaStream_t, const PcFin<T>*);                   \
  template void launch_cheb_sweep<T>(CFieldRef<T>, FieldRef<T>, FieldRef<T>, FieldRef<T>, const ChebStep&, int,     \
                                     const OpCoef&, const KScal*, cudaStream_t, const PcFin<T>*);                   \
  template void launch_pc_final<T>(const cplx<T>*, CFieldRef<T>, cplx<T>*, const OpCoef&, const KScal*,             \
                                   cudaStream_t);                                                                   \
  template void launch_p_update<T>(const cplx<T>*, cplx<T>*, const cplx<T>*, const OpCoef&, const KScal*,           \
                                   cudaStream_t);                                                                   \
  template void launch_s_update<T>(cplx<T>*, const cplx<T>*, const OpCoef&, const KScal*, cudaStream_t, void*);     \
  template void launch_r_update<T>(cplx<T>*, const cplx<T>*, cplx<T>*, const cplx<T>*, const OpCoef&, const KScal*, \
                                   cudaStream_t, const cplx<T>*, void*);                                            \
  template void launch_add_to<T>(const cplx<T>*, double2*, const OpCoef&, cudaStream_t);

APFC_INST(double)
APFC_INST(float)

}  // namespace apfc
