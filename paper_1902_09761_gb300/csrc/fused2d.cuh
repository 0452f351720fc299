// Row-streaming fused application of P^{-1} (and of A P^{-1}) on 2D grids.
//
// The preconditioner of Sec. II.B (Eq. preconditioner, M = I) applied to
// beta = (beta1, beta2), followed optionally by the block operator of
// Eq. linear_system2, is a chain of radius-1 stencil stages:
//
//   stage 1         f     = beta2 - kt G_h beta1                 (step 2 right side)
//   stages 2..M+1   Chebyshev solve D beta2' = f, M applications of D
//   stages M+2..2M+1 Chebyshev solve D chi2 = beta2', M applications;
//                   the last also forms chi1 = beta1 + (beta2' - sD chi2)/mu (step 4)
//   stage 2M+2      y = A (chi1, chi2) = (chi1 - G_h chi2, kt G_h chi1 + a chi2)
//
// with D = sD I - mu L_h and the Chebyshev recurrence of Saad, Sec. 12.3
// (x += d; r -= D d; d = c1 d + c2 r).  One thread block owns a strip of
// NT columns (NT - 2S of them valid, S = number of stages) and a segment of
// rows, and streams down the rows: at local time rho, stage s works on local
// row rho - 2s.  Every stage keeps the row it produced in a shared-memory ring
// for the x- and y-neighbours of the next stage (FP32 pipelines hold the
// y-neighbours in registers and the ring for the x-neighbours); values a later stage
// needs at the same point (Chebyshev x and r, beta2, beta2') travel in register
// delay lines.  Lag 2 per stage lets all stages of one time step run without a
// barrier between them: one __syncthreads per row.  Each input row is read from
// HBM once (plus the x halo), each output row written once.
//
// Loaders form the input on the fly from Krylov vectors; epilogues store the
// result and accumulate inner products for the BiCGStab scalars.
//
// This header holds the kernel template and its launch dispatch; the entry
// points that instantiate it live in fused2d.cu (x += P^{-1} u, the BiCGStab
// vector updates), fused2d_v.cu (v = A P^{-1} p) and fused2d_t.cu
// (t = A P^{-1} s), so that the three compile in parallel.
#pragma once
#include "acc.cuh"
#include "apfc_internal.cuh"
#include "bf16pair.cuh"
#include "dfloat.cuh"

#include <algorithm>
#include <cstring>
#include <type_traits>

namespace apfc {

namespace {


// Complex helpers.  FP32 complex values use the packed f32x2 instructions of
// sm_100-class GPUs (one instruction for both components).
__device__ __forceinline__ unsigned long long pk(float2 a) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
  return r;
}
__device__ __forceinline__ float2 upk(unsigned long long r) {
  float2 a;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
  return a;
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) {
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pk(a)), "l"(pk(b)));
  return upk(r);
}
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pk(a)), "l"(pk(b)));
  return upk(r);
}
__device__ __forceinline__ float2 cscale(float s, float2 a) {
  unsigned long long r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pk(make_float2(s, s))), "l"(pk(a)));
  return upk(r);
}
__device__ __forceinline__ float2 caxpy(float s, float2 a, float2 b) {  // s a + b
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(pk(make_float2(s, s))), "l"(pk(a)), "l"(pk(b)));
  return upk(r);
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cscale(double s, double2 a) { return make_double2(s * a.x, s * a.y); }
__device__ __forceinline__ double2 caxpy(double s, double2 a, double2 b) {
  return make_double2(fma(s, a.x, b.x), fma(s, a.y, b.y));
}
template <typename C>
__device__ __forceinline__ C cmulz(C z, C a) {  // complex z a
  C r;
  r.x = z.x * a.x - z.y * a.y;
  r.y = z.x * a.y + z.y * a.x;
  return r;
}
template <typename C>
__device__ __forceinline__ C add_i(C a, C b) {  // a + i b
  C r;
  r.x = a.x - b.y;
  r.y = a.y + b.x;
  return r;
}
template <typename T>
__device__ __forceinline__ cplx<T> to_c(double2 z) {
  return mkc<T>((T)z.x, (T)z.y);
}

template <int I, int N, typename F>
__device__ __forceinline__ void static_for_rev(F&& f) {
  if constexpr (I >= N) {
    f(std::integral_constant<int, I>{});
    static_for_rev<I - 1, N>(f);
  }
}

// Per-amplitude coefficients in the field precision.
template <typename T>
struct JCoef {
  T c0, ihx, ihy, khx, khy, kt, a, sD, mu, inv_mu, it;
};

template <typename T>
__device__ __forceinline__ JCoef<T> jcoef(const OpCoef& c, int j) {
  JCoef<T> q;
  q.c0 = (T)c.c0;
  q.ihx = (T)c.ih2[0];
  q.ihy = (T)c.ih2[1];
  q.khx = (T)c.kh[j][0];
  q.khy = (T)c.kh[j][1];
  q.kt = (T)c.kt[j];
  q.a = (T)c.a[j];
  q.sD = (T)c.sD[j];
  q.mu = (T)c.mu[j];
  q.inv_mu = (T)c.inv_mu[j];
  q.it = (T)c.inv_theta[j];
  return q;
}

// 5-point neighbourhood of one point of a ring quantity.
template <typename T>
struct Nbh {
  cplx<T> c, l, r, u, d;  // centre, x-1, x+1, y-1, y+1
};

template <typename T>
__device__ __forceinline__ cplx<T> lap(const Nbh<T>& n, const JCoef<T>& q) {
  return caxpy(q.ihy, cadd(n.u, n.d), caxpy(q.ihx, cadd(n.l, n.r), cscale(q.c0, n.c)));
}
// G_h = L_h + i (k_x/h_x)(u(x+1) - u(x-1)) + i (k_y/h_y)(u(y+1) - u(y-1))
template <typename T>
__device__ __forceinline__ cplx<T> opG(const Nbh<T>& n, const JCoef<T>& q) {
  const cplx<T> adv = caxpy(q.khy, csub(n.d, n.u), cscale(q.khx, csub(n.r, n.l)));
  return add_i(lap(n, q), adv);
}
template <typename T>
__device__ __forceinline__ cplx<T> opD(const Nbh<T>& n, const JCoef<T>& q) {
  return caxpy(-q.mu, lap(n, q), cscale(q.sD, n.c));
}

struct PipeGeom {
  int nx, ny, Ly, wv, nstrips, nsegs, npart;
  long long pts;
};

// ---------------------------------------------------------------------------
// Loaders and epilogues.  Each names the global arrays ("raw values") it needs
// at a point; the kernel fetches them (asynchronously, PF rows ahead, when
// PF > 0) and hands them back to form():
//   loader raw "in": the input row          -> (beta1, beta2)
//   loader raw "re": re-forming beta1 for step 4 of P^{-1}, 2(2M+1) rows later
//   epilogue raw   : operands of the output stage (stored result, dot products)
// ---------------------------------------------------------------------------
template <typename T>
struct LoadPlain {
  static constexpr int PERIOD = 1;  // row-loop phase (see PipeShape)
  static constexpr int NIN = 2, NRE = 1;
  const cplx<T>* b;
  long long pts;
  long long off;
  // batched runs: move every array to this run's block vectors
  __device__ void rebase(long long e, long long n) {
    b += e;
    pts = n;
  }
  __device__ void setup(int j, const KScal*) { off = 2LL * j * pts; }
  __device__ const cplx<T>* in(int i) const { return b + off + i * pts; }
  __device__ const cplx<T>* re(int) const { return b + off; }
  __device__ void form_in(const cplx<T>* raw, int st, long long, bool, cplx<T>& b1, cplx<T>& b2) const {
    b1 = raw[0];
    b2 = raw[st];
  }
  __device__ cplx<T> form_re(const cplx<T>* raw, int) const { return raw[0]; }
};

// p = r + beta (p_old - omega v_old), written to p_new at the points this block owns.
template <typename T>
struct LoadP {
  static constexpr int PERIOD = 9;
  static constexpr int NIN = 6, NRE = 3;
  const cplx<T>* r;
  const cplx<T>* po;
  const cplx<T>* vo;
  cplx<T>* pn;
  long long pts;
  cplx<T> beta, omega;
  long long off;
  // batched runs: move every array to this run's block vectors
  __device__ void rebase(long long e, long long n) {
    r += e;
    po += e;
    vo += e;
    pn += e;
    pts = n;
  }
  __device__ void setup(int j, const KScal* k) {
    beta = to_c<T>(k[j].beta);
    omega = to_c<T>(k[j].omega);
    off = 2LL * j * pts;
  }
  // raw order: r1, r2, po1, po2, vo1, vo2
  __device__ const cplx<T>* in(int i) const {
    const cplx<T>* base = i < 2 ? r : (i < 4 ? po : vo);
    return base + off + (i & 1) * pts;
  }
  __device__ const cplx<T>* re(int i) const { return (i == 0 ? r : (i == 1 ? po : vo)) + off; }
  __device__ __forceinline__ cplx<T> form(cplx<T> rr, cplx<T> pp, cplx<T> vv) const {
    return cadd(rr, cmulz(beta, csub(pp, cmulz(omega, vv))));
  }
  __device__ void form_in(const cplx<T>* raw, int st, long long p, bool own, cplx<T>& b1, cplx<T>& b2) const {
    b1 = form(raw[0], raw[2 * st], raw[4 * st]);
    b2 = form(raw[st], raw[3 * st], raw[5 * st]);
    if (own) {
      pn[off + p] = b1;
      pn[off + pts + p] = b2;
    }
  }
  __device__ cplx<T> form_re(const cplx<T>* raw, int st) const { return form(raw[0], raw[st], raw[2 * st]); }
};

// s = r - alpha v.
template <typename T>
struct LoadS {
  static constexpr int PERIOD = 1;
  static constexpr int NIN = 4, NRE = 2;
  const cplx<T>* r;
  const cplx<T>* v;
  long long pts;
  cplx<T> alpha;
  long long off;
  // batched runs: move every array to this run's block vectors
  __device__ void rebase(long long e, long long n) {
    r += e;
    v += e;
    pts = n;
  }
  __device__ void setup(int j, const KScal* k) {
    alpha = to_c<T>(k[j].alpha);
    off = 2LL * j * pts;
  }
  // raw order: r1, r2, v1, v2
  __device__ const cplx<T>* in(int i) const { return (i < 2 ? r : v) + off + (i & 1) * pts; }
  __device__ const cplx<T>* re(int i) const { return (i == 0 ? r : v) + off; }
  __device__ void form_in(const cplx<T>* raw, int st, long long, bool, cplx<T>& b1, cplx<T>& b2) const {
    b1 = csub(raw[0], cmulz(alpha, raw[2 * st]));
    b2 = csub(raw[st], cmulz(alpha, raw[3 * st]));
  }
  __device__ cplx<T> form_re(const cplx<T>* raw, int st) const { return csub(raw[0], cmulz(alpha, raw[st])); }
};

// Merged BiCGStab iteration loader: from the previous iteration's r, v, t, p form
// r' = r - alpha v - omega t and p' = r' + beta (p - omega v); at owned points also
// store r', p' and apply the previous iteration's update u += alpha p + omega (r - alpha v).
template <typename T>
struct LoadPR {
  static constexpr int PERIOD = 9;
  static constexpr int NIN = 10, NRE = 4;
  const cplx<T>* r;
  const cplx<T>* v;
  const cplx<T>* t;
  const cplx<T>* p;
  cplx<T>* u;
  cplx<T>* rn;
  cplx<T>* pn;
  long long pts;
  cplx<T> al, om, be;
  long long off;
  // batched runs: move every array to this run's block vectors
  __device__ void rebase(long long e, long long n) {
    r += e;
    v += e;
    t += e;
    p += e;
    u += e;
    rn += e;
    pn += e;
    pts = n;
  }
  __device__ void setup(int j, const KScal* k) {
    al = to_c<T>(k[j].alpha);
    om = to_c<T>(k[j].omega);
    be = to_c<T>(k[j].beta);
    off = 2LL * j * pts;
  }
  // raw order: r1 r2 v1 v2 t1 t2 p1 p2 u1 u2
  __device__ const cplx<T>* in(int i) const {
    const cplx<T>* base = i < 2 ? r : (i < 4 ? v : (i < 6 ? t : (i < 8 ? p : u)));
    return base + off + (i & 1) * pts;
  }
  // raw order: r1 v1 t1 p1
  __device__ const cplx<T>* re(int i) const { return (i == 0 ? r : (i == 1 ? v : (i == 2 ? t : p))) + off; }
  __device__ __forceinline__ void form(cplx<T> rr, cplx<T> vv, cplx<T> tt, cplx<T> pp, cplx<T>& r2,
                                       cplx<T>& p2) const {
    r2 = csub(csub(rr, cmulz(al, vv)), cmulz(om, tt));
    p2 = cadd(r2, cmulz(be, csub(pp, cmulz(om, vv))));
  }
  __device__ void form_in(const cplx<T>* raw, int st, long long pnt, bool own, cplx<T>& b1, cplx<T>& b2) const {
    cplx<T> r1, r2;
    form(raw[0], raw[2 * st], raw[4 * st], raw[6 * st], r1, b1);
    form(raw[st], raw[3 * st], raw[5 * st], raw[7 * st], r2, b2);
    if (own) {
      rn[off + pnt] = r1;
      rn[off + pts + pnt] = r2;
      pn[off + pnt] = b1;
      pn[off + pts + pnt] = b2;
      // u += alpha p + omega (r - alpha v)
      const cplx<T> s1 = csub(raw[0], cmulz(al, raw[2 * st])), s2 = csub(raw[st], cmulz(al, raw[3 * st]));
      u[off + pnt] = cadd(raw[8 * st], cadd(cmulz(al, raw[6 * st]), cmulz(om, s1)));
      u[off + pts + pnt] = cadd(raw[9 * st], cadd(cmulz(al, raw[7 * st]), cmulz(om, s2)));
    }
  }
  __device__ cplx<T> form_re(const cplx<T>* raw, int st) const {
    cplx<T> r1, p1;
    form(raw[0], raw[st], raw[2 * st], raw[3 * st], r1, p1);
    return p1;
  }
};

// t = y with s = r - alpha v; (t, s), (t, t), (s, s), (rhat, s), (rhat, t).
// Epilogues: put(raw, st, p, y1, y2, k1, k2) stores the output (y1, y2) at point p; raw
// holds the operands named by ep(i) (stride st); (k1, k2) are the loader's outputs at the
// same point (beta1, beta2: s for LoadS) in FP32 pipelines, zero otherwise.
template <typename T>
struct EpT5 {
  static constexpr bool KEEP = sizeof(T) == 4;  // s = r - alpha v arrives from the loader
  static constexpr int NDOT = 5, NEP = KEEP ? 2 : 6;
  cplx<T>* t;
  const cplx<T>* r;
  const cplx<T>* v;
  const cplx<T>* rhat;
  long long pts;
  long long off;
  cplx<T> alpha;
  Acc<T> acc[5];
  // batched runs: move every array to this run's block vectors
  __device__ void rebase(long long e, long long n) {
    t += e;
    r += e;
    v += e;
    rhat += e;
    pts = n;
  }
  __device__ void setup(int j, const KScal* k) {
    off = 2LL * j * pts;
    alpha = to_c<T>(k[j].alpha);
  }
  // raw order: rhat1 rhat2 (FP32), r1 r2 v1 v2 rhat1 rhat2 (FP64)
  __device__ const cplx<T>* ep(int i) const {
    if constexpr (KEEP) return rhat + off + i * pts;
    return (i < 2 ? r : (i < 4 ? v : rhat)) + off + (i & 1) * pts;
  }
  __device__ void one(long long q, cplx<T> y, cplx<T> s, cplx<T> hh) {
    t[q] = y;
    acc[0].add_run(y, s);
    acc[1].add_run_self(y);
    acc[2].add_run_self(s);
    acc[3].add_run(hh, s);
    acc[4].add_run(hh, y);
  }
  __device__ void put(const cplx<T>* raw, int st, long long p, cplx<T> y1, cplx<T> y2, cplx<T> k1, cplx<T> k2) {
    if constexpr (KEEP) {
      one(off + p, y1, k1, raw[0]);
      one(off + pts + p, y2, k2, raw[st]);
    } else {
      one(off + p, y1, csub(raw[0], cmulz(alpha, raw[2 * st])), raw[4 * st]);
      one(off + pts + p, y2, csub(raw[st], cmulz(alpha, raw[3 * st])), raw[5 * st]);
    }
  }
};

template <typename T>
struct EpStore {  // out = y
  static constexpr int NDOT = 0, NEP = 0;
  cplx<T>* out;
  long long pts;
  long long off;
  Acc<T> acc[1];
  // batched runs: move every array to this run's block vectors
  __device__ void rebase(long long e, long long n) {
    out += e;
    pts = n;
  }
  __device__ void setup(int j, const KScal*) { off = 2LL * j * pts; }
  __device__ const cplx<T>* ep(int) const { return nullptr; }
  __device__ void put(const cplx<T>*, int, long long p, cplx<T> y1, cplx<T> y2, cplx<T>, cplx<T>) {
    out[off + p] = y1;
    out[off + pts + p] = y2;
  }
};

template <typename T>
struct EpAddX {  // x64 += y (the Krylov correction P^{-1} u)
  static constexpr int NDOT = 0, NEP = 0;
  double2* x;
  long long pts;
  long long off;
  Acc<T> acc[1];
  // batched runs: move every array to this run's block vectors
  __device__ void rebase(long long e, long long n) {
    x += e;
    pts = n;
  }
  __device__ void setup(int j, const KScal*) { off = 2LL * j * pts; }
  __device__ const cplx<T>* ep(int) const { return nullptr; }
  __device__ void put(const cplx<T>*, int, long long p, cplx<T> y1, cplx<T> y2, cplx<T>, cplx<T>) {
    double2 a = x[off + p], b = x[off + pts + p];
    if constexpr (sizeof(T) == 4) {  // exact widening by integer operations (no FP64 conversion)
      a.x += f2d(y1.x);
      a.y += f2d(y1.y);
      b.x += f2d(y2.x);
      b.y += f2d(y2.y);
    } else {
      a.x += y1.x;
      a.y += y1.y;
      b.x += y2.x;
      b.y += y2.y;
    }
    x[off + p] = a;
    x[off + pts + p] = b;
  }
};

template <typename T>
struct EpV {  // v = y; (rhat, v)
  // FP32: rhat staged as one 8-byte value per point, the bf16 pairs of its two parts
  // (rh16 [J][pts], bf16pair.cuh); FP64: both complex parts of rhat
  static constexpr bool H16 = sizeof(T) == 4;
  static constexpr int NDOT = 1, NEP = H16 ? 1 : 2;
  cplx<T>* v;
  const cplx<T>* rhat;
  const uint2* rh16;
  long long pts;
  long long off;
  Acc<T> acc[1];
  // batched runs: move every array to this run's block vectors
  __device__ void rebase(long long e, long long n) {
    v += e;
    if constexpr (H16) {
      rh16 += e / 2;
    } else {
      rhat += e;
    }
    pts = n;
  }
  __device__ void setup(int j, const KScal*) { off = 2LL * j * pts; }
  __device__ const cplx<T>* ep(int i) const {
    if constexpr (H16) return reinterpret_cast<const cplx<T>*>(rh16 + off / 2);
    return rhat + off + i * pts;
  }
  __device__ void put(const cplx<T>* raw, int st, long long p, cplx<T> y1, cplx<T> y2, cplx<T>, cplx<T>) {
    v[off + p] = y1;
    v[off + pts + p] = y2;
    if constexpr (H16) {
      const cplx<T> w = raw[0];  // the bits of the two bf16 pairs
      acc[0].add_run(bf16_unpack(__float_as_uint(w.x)), y1);
      acc[0].add_run(bf16_unpack(__float_as_uint(w.y)), y2);
    } else {
      acc[0].add_run(raw[0], y1);
      acc[0].add_run(raw[st], y2);
    }
  }
};

// Epilogue of a Picard iteration with the Jacobian on FP32 grids: the wrapped epilogue's
// operands plus kap_j D_j of the point (stored as {value, 0}), staged with them.
template <class EP, typename T>
struct EpJ : EP {
  static constexpr int NEP = EP::NEP + 1;
  const float2* jd32;
  long long jo;
  __device__ void setup(int j, const KScal* k) {
    EP::setup(j, k);
    jo = (long long)j * EP::pts;
  }
  __device__ const cplx<T>* ep(int i) const {
    return i < EP::NEP ? EP::ep(i) : reinterpret_cast<const cplx<T>*>(jd32 + jo);
  }
};

template <typename T>
struct EpT {  // t = y; (t, s), (t, t), (s, s) with s = r - alpha v
  static constexpr bool KEEP = sizeof(T) == 4;  // s arrives from the loader
  static constexpr int NDOT = 3, NEP = KEEP ? 0 : 4;
  cplx<T>* t;
  const cplx<T>* r;
  const cplx<T>* v;
  long long pts;
  long long off;
  cplx<T> alpha;
  Acc<T> acc[3];
  // batched runs: move every array to this run's block vectors
  __device__ void rebase(long long e, long long n) {
    t += e;
    r += e;
    v += e;
    pts = n;
  }
  __device__ void setup(int j, const KScal* k) {
    off = 2LL * j * pts;
    alpha = to_c<T>(k[j].alpha);
  }
  // raw order: r1, r2, v1, v2 (FP64)
  __device__ const cplx<T>* ep(int i) const { return (i < 2 ? r : v) + off + (i & 1) * pts; }
  __device__ void one(long long q, cplx<T> y, cplx<T> s) {
    t[q] = y;
    acc[0].add_run(y, s);
    acc[1].add_run_self(y);
    acc[2].add_run_self(s);
  }
  __device__ void put(const cplx<T>* raw, int st, long long p, cplx<T> y1, cplx<T> y2, cplx<T> k1, cplx<T> k2) {
    if constexpr (KEEP) {
      one(off + p, y1, k1);
      one(off + pts + p, y2, k2);
    } else {
      one(off + p, y1, csub(raw[0], cmulz(alpha, raw[2 * st])));
      one(off + pts + p, y2, csub(raw[st], cmulz(alpha, raw[3 * st])));
    }
  }
};

// ---- asynchronous global -> shared copies (one element per thread) --------
template <typename T>
__device__ __forceinline__ void cp_async(cplx<T>* dst, const cplx<T>* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  if constexpr (sizeof(cplx<T>) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src));
  else
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

// ---------------------------------------------------------------------------
// The pipeline kernel.  M = Chebyshev applications per diffusion solve;
// PF = rows of look-ahead of the asynchronous fetches (0: fetch when needed).
// ---------------------------------------------------------------------------
// Chebyshev weights of all applications: c1[k][j], c2[k][j].
struct ChebAll {
  double c1[kMaxCheb][kMaxJ];
  double c2[kMaxCheb][kMaxJ];
};

template <int N>
__host__ __device__ constexpr int pow2_at_least() {
  int p = 1;
  while (p < N) p *= 2;
  return p;
}

// Slot of row rho - D2 in a ring of depth D, given rm = rho mod D (D2 >= 0 fixed at compile time).
template <int D, int D2>
__device__ __forceinline__ int ring_slot(int rm) {
  constexpr int c = (D - D2 % D) % D;
  const int v = rm + c;
  return v >= D ? v - D : v;
}

template <typename T, int M, bool WITH_A, int PF, int NT_, class LD, class EP>
struct PipeShape {
  static constexpr int S = 2 * M + 1 + (WITH_A ? 1 : 0);  // stencil stages = halo radius
  static constexpr int NRING = 2 * M + 1 + (WITH_A ? 2 : 0);
  static constexpr int QB = M + 1;                          // ring of beta2' (deep: read again by step 4)
  // FP32 pipelines keep the y-neighbours of every stencil input in registers, so a ring
  // serves one row per step (the x-neighbours of the row two steps old): three rows are
  // live (read, next, being written).  FP64 pipelines read three rows of a ring per step
  // and write a fourth.
  static constexpr bool HIST = sizeof(T) == 4;
  static constexpr int RD = HIST ? 3 : 4;
  // beta2' is read again by step 4, 2M steps after the next stage: 2M + 1 rows live
  static constexpr int DB = HIST ? 2 * M + 1
                                 : (pow2_at_least<2 * M + 1>() < 4 ? 4 : pow2_at_least<2 * M + 1>());
  static constexpr int SCHI = 2 * M + 1;  // stage forming chi1 (step 4)
  static constexpr int SEP = S;           // stage calling the epilogue
  // FP32 pipelines keep the loader's outputs (beta1, beta2) of the last 2S + 1 rows of
  // their own column in shared memory: step 4 and the epilogue read them there instead of
  // fetching and re-forming them from the Krylov vectors again
  static constexpr bool KEEP = sizeof(T) == 4;
  static constexpr int KD = 2 * S + 1;
  static constexpr int NRE_F = KEEP ? 0 : LD::NRE;  // re-form operands fetched per row
  static constexpr int NRAW = LD::NIN + NRE_F + EP::NEP;
  // FP32 pipelines with one Chebyshev application and A run their row loop in phases of
  // PERIOD rows (the loader's choice), fully unrolled, so that the slots of every ring whose
  // depth divides PERIOD are constants in each copy of the body: no slot or address
  // arithmetic.  v-kernels take 9 rows (stage rings 3, beta2' 3, keep 9, staging 3; measured
  // 25.2 -> 24.8 ms per 4096^2 step).  The t-kernel, bound by instruction issue, loses more to
  // the longer body than it saves (9-row phases 13.9 -> 15.0 ms, 3-row phases with the
  // keep-ring slot a counter 12.9 -> 15.2 ms), so it keeps the plain loop.
  static constexpr bool PHASED = HIST && M == 1 && WITH_A && (PF == 1 || PF == 2) && LD::PERIOD > 1;
  static constexpr int PERIOD = PHASED ? LD::PERIOD : 1;
  static constexpr bool KEEP_CONST = PERIOD % KD == 0;  // keep-ring slot a constant too
  static constexpr int NSLOT = PF > 0 ? (PHASED ? 3 : PF + 1) : 0;
  static constexpr int NT = NT_;
  // ring 0 (beta1, the input of stage 1) is the keep ring's first component when KEEP
  static constexpr int R0 = KEEP ? 0 : RD;
  static constexpr size_t ring_elems = (size_t)(R0 + (NRING - 2) * RD + DB) * NT;
  static constexpr size_t keep_elems = KEEP ? (size_t)KD * 2 * NT : 0;
  static constexpr size_t smem = sizeof(cplx<T>) * (ring_elems + keep_elems + (size_t)NSLOT * NRAW * NT);
  // element offset of ring q (q >= 1 when KEEP)
  __host__ __device__ static constexpr int off(int qi) {
    return (qi == 0 ? 0 : (qi <= QB ? R0 + (qi - 1) * RD : R0 + (QB - 1) * RD + DB + (qi - QB - 1) * RD)) * NT;
  }
  __host__ __device__ static constexpr int depth(int qi) { return qi == QB ? DB : RD; }
  static_assert(!PHASED || (PERIOD % RD == 0 && PERIOD % DB == 0 && PERIOD % NSLOT == 0),
                "the phase period must be a multiple of the stage, beta2' and staging ring depths");
};

template <typename T, int NT>
__device__ __forceinline__ Nbh<T> fetch_d(const cplx<T>* ring, int mask, int row, int t) {
  const int sc = row & mask, su = (row - 1) & mask, sd = (row + 1) & mask;
  const int tl = t > 0 ? t - 1 : t, tr = t < NT - 1 ? t + 1 : t;
  Nbh<T> n;
  n.c = ring[sc * NT + t];
  n.l = ring[sc * NT + tl];
  n.r = ring[sc * NT + tr];
  n.u = ring[su * NT + t];
  n.d = ring[sd * NT + t];
  return n;
}


// Batched runs: the geometry of up to kTabRuns runs of one launch travels in
// the kernel parameters (a constant-bank table indexed by blockIdx.y), so that
// the work-item indices and grid sizes stay block-uniform values.
constexpr int kTabRuns = 64;
struct RunRec {
  long long pts, elem_off, part_off;
  int nx, ny, Ly, nstrips, nsegs, nblk, run, pad;
};
struct RunTab {
  RunRec run[kTabRuns];
};
struct NoTab {};

// ---------------------------------------------------------------------------
__device__ __forceinline__ int wrap_inc(int y, int n) { return y + 1 == n ? 0 : y + 1; }

// Grid: (nstrips, nsegs, J) for one grid (TAB = NoTab); for batched runs
// (TAB = RunTab) (blocks of the largest run, runs of the table), each block
// taking item blockIdx.x = sx + nstrips (sy + nsegs j) of run blockIdx.y.
// JAC: the (2,2) block of A carries the Jacobian diagonal c.jd of a Picard iteration.
template <typename T, int M, bool WITH_A, int PF, int NT_, class LD, class EP, class TAB, bool JAC>
__global__ void __launch_bounds__(NT_) k_pipe2d(OpCoef c, ChebAll cw, PipeGeom g, LD ld, EP ep, const KScal* act,
                                                void* partials, int kid, int fields,
                                                const __grid_constant__ TAB tab) {
  using SH = PipeShape<T, M, WITH_A, PF, NT_, LD, EP>;
  constexpr int NT = SH::NT;
  constexpr int S = SH::S;
  constexpr int NRAW = SH::NRAW;
  constexpr int OIN = 0, ORE = LD::NIN, OEP = LD::NIN + SH::NRE_F;  // raw offsets inside a slot
  extern __shared__ unsigned char smem_raw[];
  cplx<T>* sm = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* keep = sm + SH::ring_elems;  // [KD][2][NT]: loader outputs of the own column
  cplx<T>* stage_buf = keep + SH::keep_elems;

  // work item: strip sx, row segment sy, amplitude j (of run blockIdx.y when batched)
  int sx, sy, j;
  if constexpr (std::is_same<TAB, RunTab>::value) {
    const RunRec& rq = tab.run[blockIdx.y];
    const int b = blockIdx.x;
    if (b >= rq.nblk) return;
    g.nx = rq.nx;
    g.ny = rq.ny;
    g.Ly = rq.Ly;
    g.nstrips = rq.nstrips;
    g.nsegs = rq.nsegs;
    g.npart = rq.nstrips * rq.nsegs;
    g.pts = rq.pts;
    sx = b % rq.nstrips;
    sy = (b / rq.nstrips) % rq.nsegs;
    j = b / g.npart;
    ld.rebase(rq.elem_off, rq.pts);
    ep.rebase(rq.elem_off, rq.pts);
    if (act != nullptr) act += (long long)rq.run * c.J;
    if (partials != nullptr) partials = reinterpret_cast<char*>(partials) + 16ll * rq.part_off;
  } else {
    sx = blockIdx.x;
    sy = blockIdx.y;
    j = blockIdx.z;
  }
  if (act != nullptr && act[j].active == 0) return;
  const int t = threadIdx.x;
  const JCoef<T> q = jcoef<T>(c, j);
  T c1[M], c2[M];
#pragma unroll
  for (int k = 0; k < M; ++k) {
    c1[k] = (T)cw.c1[k][j];
    c2[k] = (T)cw.c2[k][j];
  }
  // M = 1: x = it f + c1 it f + c2 (f - it D f) = pa1 f + pb1 D f
  const T pa1 = (T)(c.inv_theta[j] * (1.0 + cw.c1[0][j]) + cw.c2[0][j]);
  const T pb1 = (T)(-cw.c2[0][j] * c.inv_theta[j]);
  ld.setup(j, act);
  ep.setup(j, act);
#pragma unroll
  for (int k = 0; k < EP::NDOT; ++k) ep.acc[k].zero();
  if (c.prof != nullptr && sx == 0 && sy == 0 && t == 0)
    atomicAdd(c.prof + kid, (unsigned long long)fields * (unsigned long long)g.pts * sizeof(cplx<T>));

  // zero the rings (garbage in invalid halo columns must stay finite)
  for (int i = t; i < (int)(SH::ring_elems + SH::keep_elems); i += NT) sm[i] = mkc<T>((T)0, (T)0);

  const int x_first = sx * g.wv - S;  // global column of thread 0 (unwrapped)
  int gx = (x_first + t) % g.nx;
  if (gx < 0) gx += g.nx;
  const int xo = sx * g.wv + (t - S);  // output column of this thread
  const bool col_own = (t >= S) && (t < NT - S) && (xo < g.nx);
  const int y0 = sy * g.Ly;
  const int rows_in = g.Ly + 2 * S;  // local rows 0 .. rows_in-1 = global y0-S ..
  const int steps = g.Ly + 3 * S;

  auto grow = [&](int lr) {  // only for initialising the incremental row trackers
    int y = (y0 - S + lr) % g.ny;
    return y < 0 ? y + g.ny : y;
  };
  auto row_own = [&](int lr) { return lr >= S && lr < S + g.Ly && (y0 + lr - S) < g.ny; };
  auto valid_at = [&](int s, int lr) { return lr >= s && lr < rows_in - s; };
  auto need_ep = [&](int lr) { return valid_at(SH::SEP, lr) && col_own && row_own(lr); };
  auto ptg = [&](int gy) { return (long long)gy * g.nx + gx; };

  // global rows of the points touched at this step, advanced by one row per step
  int gy_in = grow(0), gy_chi = grow(-2 * SH::SCHI), gy_ep = grow(-2 * SH::SEP);
  // rows of the next fetch, starting with the prologue's local time 0
  int fy_in = grow(0), fy_re = grow(-2 * SH::SCHI), fy_ep = grow(-2 * SH::SEP);

  // asynchronous fetch of everything local time tf will consume (rows fy_*) into staging slot ns
  auto issue = [&](int tf, int ns) {
    if constexpr (PF > 0) {
      cplx<T>* slot = stage_buf + (size_t)ns * NRAW * NT + t;
      if (tf < rows_in) {
        const long long p = ptg(fy_in);
#pragma unroll
        for (int i = 0; i < LD::NIN; ++i) cp_async<T>(slot + (OIN + i) * NT, ld.in(i) + p);
      }
      if constexpr (!SH::KEEP) {
        if (valid_at(SH::SCHI, tf - 2 * SH::SCHI)) {
          const long long p = ptg(fy_re);
#pragma unroll
          for (int i = 0; i < LD::NRE; ++i) cp_async<T>(slot + (ORE + i) * NT, ld.re(i) + p);
        }
      }
      if constexpr (EP::NEP > 0) {
        if (need_ep(tf - 2 * SH::SEP)) {
          const long long p = ptg(fy_ep);
#pragma unroll
          for (int i = 0; i < EP::NEP; ++i) cp_async<T>(slot + (OEP + i) * NT, ep.ep(i) + p);
        }
      }
      cp_commit();
      fy_in = wrap_inc(fy_in, g.ny);
      fy_re = wrap_inc(fy_re, g.ny);
      fy_ep = wrap_inc(fy_ep, g.ny);
    }
  };

  // register delay lines: beta2 (2 steps) and the Chebyshev x, r of every stage (2 steps)
  cplx<T> b2dl[2];
  cplx<T> XD[2 * M + 2][2], RD[2 * M + 2][2];
#pragma unroll
  for (int k = 0; k < 2; ++k) b2dl[k] = mkc<T>((T)0, (T)0);
#pragma unroll
  for (int s = 0; s < 2 * M + 2; ++s)
#pragma unroll
    for (int k = 0; k < 2; ++k) XD[s][k] = RD[s][k] = mkc<T>((T)0, (T)0);

  auto ring = [&](int qi) { return sm + SH::off(qi); };

  // Own-column history of every stencil input (rows newest first): FP32 pipelines keep
  // the y-neighbours in registers and read only the x-neighbours from shared memory.
  constexpr bool HIST = sizeof(T) == 4;
  cplx<T> H[HIST ? SH::NRING : 1][3];
#pragma unroll
  for (int qi = 0; qi < (HIST ? SH::NRING : 1); ++qi)
#pragma unroll
    for (int k = 0; k < 3; ++k) H[qi][k] = mkc<T>((T)0, (T)0);
  auto push = [&](int qi, cplx<T> v) {
    if constexpr (HIST) {
      H[qi][2] = H[qi][1];
      H[qi][1] = H[qi][0];
      H[qi][0] = v;
    }
  };
  // the slots of row lr = rho - 2s in the rings (sl), in the beta2' ring (sq) and in the keep ring (sk)
  auto nbh = [&](int qi, int lr, int sl, int sq, int sk) {
    if constexpr (HIST) {
      const cplx<T>* rq = ring(qi);
      int sc = qi == SH::QB ? sq : sl;
      if constexpr (SH::KEEP) {
        if (qi == 0) {  // beta1 of row lr from the keep ring (component 0 of its slot)
          rq = keep;
          sc = sk * 2;
        }
      }
      Nbh<T> n;
      n.c = H[qi][1];
      n.u = H[qi][2];
      n.d = H[qi][0];
      n.l = rq[sc * NT + (t > 0 ? t - 1 : t)];
      n.r = rq[sc * NT + (t < NT - 1 ? t + 1 : t)];
      return n;
    } else {
      return fetch_d<T, NT>(ring(qi), SH::depth(qi) - 1, lr, t);
    }
  };

  if constexpr (PF > 0) {
#pragma unroll
    for (int tf = 0; tf < PF; ++tf) issue(tf, tf % SH::NSLOT);
  }
  __syncthreads();

  // rho mod the depths of the rings, the beta2' ring and the keep ring
  int rm = 0, rq = 0, rk = 0;
  constexpr int PER = SH::PERIOD;
  // Phased pipelines: the outer loop takes PER rows at a time and the inner one is fully
  // unrolled, so rm, rq, rk and the staging slots are constants in every copy of the body.
#pragma unroll(PER == 1 && sizeof(T) == 4 ? 2 : 1)
  for (int rho0 = 0; rho0 < steps; rho0 += PER) {
#pragma unroll
  for (int ph = 0; ph < PER; ++ph) {
    const int rho = rho0 + ph;
    if (PER > 1 && rho >= steps) break;
    if constexpr (PER > 1) {
      rm = ph % SH::RD;
      rq = ph % SH::DB;
      if constexpr (SH::KEEP_CONST) rk = ph % SH::KD;
    }
    const cplx<T>* raw = nullptr;
    int st = 1;
    if constexpr (PF > 0) {
      issue(rho + PF, PER > 1 ? (ph + PF) % SH::NSLOT : (rho + PF) % SH::NSLOT);
      cp_wait<PF>();
      raw = stage_buf + (size_t)(PER > 1 ? ph % SH::NSLOT : rho % SH::NSLOT) * NRAW * NT + t;
      st = NT;
    }
    Nbh<T> nb[S + 2];
    const cplx<T> zero = mkc<T>((T)0, (T)0);
    cplx<T> b1k = zero, b2k = zero, b2p = zero;  // keep ring (beta1, beta2) and beta2' at the chi row
    cplx<T> k1e = zero, k2e = zero;              // keep ring at the row of the A stage
    // shared-memory reads of stage s (issued just before its arithmetic: reading every
    // stage's operands ahead of the step's stores raised the fused kernels' registers by
    // about 40%, cost them occupancy and made them slower)
    auto load_stage = [&](auto sc) {
      constexpr int s = decltype(sc)::value;
      const int lr = rho - 2 * s;
      if (valid_at(s, lr)) {
        const int sl = ring_slot<SH::RD, 2 * s>(rm);
        const int sq = ring_slot<SH::DB, 2 * s>(rq);
        const int sk = ring_slot<SH::KD, 2 * s>(rk);
        if constexpr (WITH_A && s == S) {
          nb[S] = nbh(2 * M + 1, lr, sl, sq, sk);
          nb[S + 1] = nbh(2 * M + 2, lr, sl, sq, sk);
          if constexpr (SH::KEEP) {
            k1e = keep[sk * 2 * NT + t];
            k2e = keep[sk * 2 * NT + NT + t];
          }
        } else {
          nb[s] = nbh(s - 1, lr, sl, sq, sk);
        }
        if constexpr (s == SH::SCHI) {
          b2p = ring(SH::QB)[sq * NT + t];
          if constexpr (SH::KEEP) {
            b1k = keep[sk * 2 * NT + t];
            if constexpr (!WITH_A) b2k = keep[sk * 2 * NT + NT + t];
          }
        }
      }
    };
    // compute and write this step's rows, latest stage first
    static_for_rev<S, 1>([&](auto sc) {
      constexpr int s = decltype(sc)::value;
      const int lr = rho - 2 * s;
      const int sl = ring_slot<SH::RD, 2 * s>(rm);
      const int sq = ring_slot<SH::DB, 2 * s>(rq);
      const bool valid = valid_at(s, lr);
      load_stage(sc);
      if constexpr (s == 1) {
        // f = beta2 - kt G beta1
        cplx<T> f = zero;
        if (valid) {
          const cplx<T> gb = opG<T>(nb[1], q);
          f = csub(b2dl[1], cscale(q.kt, gb));
          ring(1)[sl * NT + t] = f;
        }
        push(1, f);
      } else if constexpr (s <= 2 * M + 1) {
        // Chebyshev application k of solve 1 (s <= M+1) or solve 2
        constexpr bool solve1 = s <= M + 1;
        constexpr int k = solve1 ? s - 2 : s - M - 2;
        constexpr bool last = (k == M - 1);
        cplx<T> X = zero, R = zero, dn = zero, out1 = zero;
        [[maybe_unused]] cplx<T> out2 = zero;  // chi2 (WITH_A only)
        if (valid) {
          const Nbh<T>& n = nb[s];
          const cplx<T> Dd = opD<T>(n, q);
          if constexpr (M == 1) {
            // one application of D: the Chebyshev approximant of D^{-1} is the polynomial
            // pa + pb D (the recurrence below, collapsed); X holds the result, dn = 0
            X = caxpy(pb1, Dd, cscale(pa1, n.c));
          } else if constexpr (k == 0) {
            const cplx<T> d0 = cscale(q.it, n.c);
            X = d0;
            R = csub(n.c, cscale(q.it, Dd));
            dn = caxpy(c1[0], d0, cscale(c2[0], R));
          } else {
            X = cadd(XD[s - 1][1], n.c);
            R = csub(RD[s - 1][1], Dd);
            dn = caxpy(c1[k], n.c, cscale(c2[k], R));
          }
          if constexpr (!last) {
            out1 = dn;
            ring(s)[sl * NT + t] = dn;
          } else if constexpr (solve1) {
            out1 = M == 1 ? X : cadd(X, dn);  // beta2'
            ring(s)[sq * NT + t] = out1;
          } else {
            const cplx<T> chi2 = M == 1 ? X : cadd(X, dn);
            const long long p = ptg(gy_chi);
            cplx<T> b1;
            if constexpr (SH::KEEP) {
              b1 = b1k;
            } else if constexpr (PF > 0) {
              b1 = ld.form_re(raw + ORE * st, st);
            } else {
              cplx<T> rr[LD::NRE];
#pragma unroll
              for (int i = 0; i < LD::NRE; ++i) rr[i] = ld.re(i)[p];
              b1 = ld.form_re(rr, 1);
            }
            const cplx<T> chi1 = cadd(b1, cscale(q.inv_mu, csub(b2p, cscale(q.sD, chi2))));
            if constexpr (WITH_A) {
              out1 = chi1;
              out2 = chi2;
              ring(s)[sl * NT + t] = chi1;
              ring(s + 1)[sl * NT + t] = chi2;
            } else {
              if (col_own && row_own(lr)) ep.put(raw + OEP * st, st, p, chi1, chi2, b1k, b2k);
            }
          }
        }
        if constexpr (!last) {
          XD[s][1] = XD[s][0];
          XD[s][0] = X;
          RD[s][1] = RD[s][0];
          RD[s][0] = R;
        }
        if constexpr (!last || solve1) {
          push(s, out1);
        } else if constexpr (WITH_A) {
          push(s, out1);
          push(s + 1, out2);
        }
      } else {
        // y = A (chi1, chi2)
        if (valid && col_own && row_own(lr)) {
          const Nbh<T>& n1 = nb[S];
          const Nbh<T>& n2 = nb[S + 1];
          const cplx<T> g1 = opG<T>(n1, q), g2 = opG<T>(n2, q);
          const cplx<T> y1 = csub(n1.c, g2);
          const long long p = ptg(gy_ep);
          cplx<T> y2;
          if constexpr (JAC) {
            T jdv;
            if constexpr (PF > 0 && sizeof(T) == 4) {
              jdv = raw[(OEP + EP::NEP - 1) * st].x;  // staged with the epilogue operands (EpJ)
            } else {
              jdv = (T)c.jd[(long long)j * g.pts + p];
            }
            const T ap = q.a + jdv;
            y2 = caxpy(q.kt, g1, cscale(ap, n2.c));
          } else {
            y2 = caxpy(q.kt, g1, cscale(q.a, n2.c));
          }
          if constexpr (PF > 0) {
            ep.put(raw + OEP * st, st, p, y1, y2, k1e, k2e);
          } else {
            cplx<T> er[EP::NEP > 0 ? EP::NEP : 1];
#pragma unroll
            for (int i = 0; i < EP::NEP; ++i) er[i] = ep.ep(i)[p];
            ep.put(er, 1, p, y1, y2, k1e, k2e);
          }
        }
      }
    });
    // stage 0: input row rho
    {
      cplx<T> b1 = zero, b2 = zero;
      if (rho < rows_in) {
        const long long p = ptg(gy_in);
        if constexpr (PF > 0) {
          ld.form_in(raw + OIN * st, st, p, col_own && row_own(rho), b1, b2);
        } else {
          cplx<T> ri[LD::NIN];
#pragma unroll
          for (int i = 0; i < LD::NIN; ++i) ri[i] = ld.in(i)[p];
          ld.form_in(ri, 1, p, col_own && row_own(rho), b1, b2);
        }
        if constexpr (!SH::KEEP) ring(0)[rm * NT + t] = b1;
        if constexpr (SH::KEEP) {
          cplx<T>* kp = keep + rk * 2 * NT + t;
          kp[0] = b1;
          kp[NT] = b2;
        }
      }
      push(0, b1);
      b2dl[1] = b2dl[0];
      b2dl[0] = b2;
    }
    if constexpr (EP::NDOT > 0) {
      // fold the plain FP32 runs into the compensated sums every 8 rows
      if ((rho & 7) == 7) {
#pragma unroll
        for (int k = 0; k < EP::NDOT; ++k) ep.acc[k].flush();
      }
    }
    gy_in = wrap_inc(gy_in, g.ny);
    gy_chi = wrap_inc(gy_chi, g.ny);
    gy_ep = wrap_inc(gy_ep, g.ny);
    if constexpr (PER == 1) {
      rm = wrap_inc(rm, SH::RD);
      rq = wrap_inc(rq, SH::DB);
    }
    if constexpr (!SH::KEEP_CONST) rk = wrap_inc(rk, SH::KD);
    __syncthreads();
  }
  }
  if constexpr (PF > 0) cp_wait<0>();

  if constexpr (EP::NDOT > 0) {
    const int blk = sy * g.nstrips + sx;
#pragma unroll
    for (int k = 0; k < EP::NDOT; ++k) {
      ep.acc[k].flush();
      block_reduce<T, NT>(ep.acc[k]);
      if (t == 0) ep.acc[k].store(partials, (long long)(j * kDotSlots + k) * g.npart + blk);
    }
  }
}

inline PipeGeom geom(const OpCoef& c, int S, int Ly, int NT) {
  PipeGeom g;
  g.nx = c.nx;
  g.ny = c.ny;
  g.Ly = Ly < c.ny ? Ly : c.ny;
  g.wv = NT - 2 * S;
  g.nstrips = (c.nx + g.wv - 1) / g.wv;
  g.nsegs = (c.ny + g.Ly - 1) / g.Ly;
  g.npart = g.nstrips * g.nsegs;
  g.pts = c.pts;
  return g;
}

template <typename T, int M, bool WITH_A, int PF, int NT, class LD, class EP, class TAB, bool JAC>
void set_smem_attr() {
  using SH = PipeShape<T, M, WITH_A, PF, NT, LD, EP>;
  static bool done = false;
  if (!done) {
    cudaFuncSetAttribute(k_pipe2d<T, M, WITH_A, PF, NT, LD, EP, TAB, JAC>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SH::smem);
    done = true;
  }
}

template <typename T, int M, bool WITH_A, int PF, int NT, class LD, class EP, bool JAC = false>
bool launch_pipe(const OpCoef& c, const ChebStep* w, int Ly, LD ld, EP ep, const KScal* act, void* partials,
                 cudaStream_t s, int kid, int fields, const BatchLaunch* bl) {
  using SH = PipeShape<T, M, WITH_A, PF, NT, LD, EP>;
  const PipeGeom g = geom(c, SH::S, Ly, NT);
  constexpr size_t sm = SH::smem;
  ProfScope ps_(kid, s);
  ChebAll ca;
  for (int k = 0; k < kMaxCheb; ++k)
    for (int i = 0; i < kMaxJ; ++i) {
      ca.c1[k][i] = k < M ? w[k].c1[i] : 0.0;
      ca.c2[k][i] = k < M ? w[k].c2[i] : 0.0;
    }
  if (bl == nullptr) {
    set_smem_attr<T, M, WITH_A, PF, NT, LD, EP, NoTab, JAC>();
    k_pipe2d<T, M, WITH_A, PF, NT, LD, EP, NoTab, JAC>
        <<<dim3(g.nstrips, g.nsegs, c.J), NT, sm, s>>>(c, ca, g, ld, ep, act, partials, kid, fields, NoTab{});
    return true;
  }
  if constexpr (sizeof(T) == 8 || JAC) {
    return false;  // batched runs are FP32 and take the explicit step
  } else {
    set_smem_attr<T, M, WITH_A, PF, NT, LD, EP, RunTab, false>();
    // one launch per kTabRuns runs; the table holds this launch's geometry of each run
    for (int r0 = 0; r0 < bl->R; r0 += kTabRuns) {
      const int nr = std::min(kTabRuns, bl->R - r0);
      RunTab tab;
      std::memset(&tab, 0, sizeof(tab));
      int maxblk = 0;
      for (int i = 0; i < nr; ++i) {
        const RunGeom& q = bl->host[r0 + i];
        OpCoef cr = c;
        cr.nx = q.nx;
        cr.ny = q.ny;
        const PipeGeom gr = geom(cr, SH::S, Ly, NT);
        RunRec& e = tab.run[i];
        e.pts = q.pts;
        e.elem_off = q.elem_off;
        e.part_off = bl->tlay ? q.part_off_t : q.part_off;
        e.nx = q.nx;
        e.ny = q.ny;
        e.Ly = gr.Ly;
        e.nstrips = gr.nstrips;
        e.nsegs = gr.nsegs;
        e.nblk = gr.npart * c.J;
        e.run = r0 + i;
        if (WITH_A && gr.npart != (bl->tlay ? q.npart_t : q.npart)) return false;  // layout must match the table
        maxblk = std::max(maxblk, e.nblk);
      }
      k_pipe2d<T, M, WITH_A, PF, NT, LD, EP, RunTab, false>
          <<<dim3(maxblk, nr), NT, sm, s>>>(c, ca, g, ld, ep, act, partials, kid, fields, tab);
    }
    return true;
  }
}

// Tile variants of the FP32 pipeline with one Chebyshev application (the default
// degree): NT columns per block and PF rows of asynchronous look-ahead.  Other
// degrees and FP64 (arithmetic-bound, fetched on use) use one configuration each.
//   tile 0: NT 128, PF 2   1: NT 128, PF 1   2: NT 256, PF 1   3: NT 256, PF 2   4: NT 128, PF 3
//   tile 5: NT 256, PF 3
// Measured on the 4096^2 hexagonal workload with 128-row segments: the v-kernel is fastest
// with tile 3, the t-kernel (latency-bound) with tile 1.
constexpr int kTiles = 6;
inline int tile_nt(int elem_bytes, int m, int tile) {
  if (elem_bytes == 16) return 256;
  if (m != 1) return 128;
  return (tile == 2 || tile == 3 || tile == 5) ? 256 : 128;
}

// fields: algorithmic whole-field transfers per amplitude (counted in units of one
// complex field of precision T) reported to the measurement counters.
template <typename T, bool WITH_A, class LD, class EP>
bool dispatch(int m, int tile, const OpCoef& c, const ChebStep* w, int Ly, LD ld, EP ep, const KScal* act,
              void* partials, cudaStream_t s, int kid, int fields, const BatchLaunch* bl = nullptr) {
  if constexpr (WITH_A) {
    if (c.jd != nullptr) {  // Picard iteration with the Jacobian: one Chebyshev application only
      if (m != 1 || bl != nullptr) return false;
      if constexpr (sizeof(T) == 8) {
        return launch_pipe<T, 1, true, 0, 256, LD, EP, true>(c, w, Ly, ld, ep, act, partials, s, kid, fields, bl);
      } else {
        if (c.jd32 == nullptr) return false;
        EpJ<EP, T> ej{};
        static_cast<EP&>(ej) = ep;
        ej.jd32 = c.jd32;
        using EJ = EpJ<EP, T>;
        switch (tile) {
          case 1: return launch_pipe<T, 1, true, 1, 128, LD, EJ, true>(c, w, Ly, ld, ej, act, partials, s, kid, fields, bl);
          case 2: return launch_pipe<T, 1, true, 1, 256, LD, EJ, true>(c, w, Ly, ld, ej, act, partials, s, kid, fields, bl);
          case 3: return launch_pipe<T, 1, true, 2, 256, LD, EJ, true>(c, w, Ly, ld, ej, act, partials, s, kid, fields, bl);
          case 4: return launch_pipe<T, 1, true, 3, 128, LD, EJ, true>(c, w, Ly, ld, ej, act, partials, s, kid, fields, bl);
          case 5: return launch_pipe<T, 1, true, 3, 256, LD, EJ, true>(c, w, Ly, ld, ej, act, partials, s, kid, fields, bl);
          default: return launch_pipe<T, 1, true, 2, 128, LD, EJ, true>(c, w, Ly, ld, ej, act, partials, s, kid, fields, bl);
        }
      }
    }
  }
  if constexpr (sizeof(T) == 8) {
    switch (m) {
      case 1: return launch_pipe<T, 1, WITH_A, 0, 256>(c, w, Ly, ld, ep, act, partials, s, kid, fields, bl);
      case 2: return launch_pipe<T, 2, WITH_A, 0, 256>(c, w, Ly, ld, ep, act, partials, s, kid, fields, bl);
      case 3: return launch_pipe<T, 3, WITH_A, 0, 256>(c, w, Ly, ld, ep, act, partials, s, kid, fields, bl);
      case 4: return launch_pipe<T, 4, WITH_A, 0, 256>(c, w, Ly, ld, ep, act, partials, s, kid, fields, bl);
      default: return false;
    }
  } else {
    if (m == 1) {
      switch (tile) {
        case 1: return launch_pipe<T, 1, WITH_A, 1, 128>(c, w, Ly, ld, ep, act, partials, s, kid, fields, bl);
        case 2: return launch_pipe<T, 1, WITH_A, 1, 256>(c, w, Ly, ld, ep, act, partials, s, kid, fields, bl);
        case 3: return launch_pipe<T, 1, WITH_A, 2, 256>(c, w, Ly, ld, ep, act, partials, s, kid, fields, bl);
        case 4: return launch_pipe<T, 1, WITH_A, 3, 128>(c, w, Ly, ld, ep, act, partials, s, kid, fields, bl);
        case 5: return launch_pipe<T, 1, WITH_A, 3, 256>(c, w, Ly, ld, ep, act, partials, s, kid, fields, bl);
        default: return launch_pipe<T, 1, WITH_A, 2, 128>(c, w, Ly, ld, ep, act, partials, s, kid, fields, bl);
      }
    }
    switch (m) {
      case 2: return launch_pipe<T, 2, WITH_A, 2, 128>(c, w, Ly, ld, ep, act, partials, s, kid, fields, bl);
      case 3: return launch_pipe<T, 3, WITH_A, 2, 128>(c, w, Ly, ld, ep, act, partials, s, kid, fields, bl);
      case 4: return launch_pipe<T, 4, WITH_A, 2, 128>(c, w, Ly, ld, ep, act, partials, s, kid, fields, bl);
      default: return false;
    }
  }
}

}  // namespace

}  // namespace apfc
