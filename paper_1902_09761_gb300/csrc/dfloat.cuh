// FP64-accurate arithmetic without the FP64 pipe, for the outer-residual and
// right-hand-side kernels of the FP32-refined step.
//
// On GB300 the FP64 pipe (and every FP64 <-> FP32 conversion) runs at about
// 1/64 of the FP32 rate, so a kernel that evaluates a complex stencil in FP64
// is bound by that pipe long before HBM.  These helpers keep the FP64 data
// layout in memory but do the arithmetic in FP32:
//
//  * split_d: a double v becomes two floats h + l = v to within 2^-48 |v|,
//    using integer and FP32 operations only (h: sign, exponent and the top 23
//    mantissa bits; l: the remaining 29 bits rounded once to 24);
//  * f2d: the exact double of a float, by integer operations;
//  * error-free transformations (Knuth's TwoSum, the FMA TwoProd) and a
//    compensated accumulator in the manner of Ogita, Rump and Oishi's Dot2
//    ("Accurate sum and dot product", SIAM J. Sci. Comput. 26, 2005): the
//    leading parts are summed with TwoSum, every rounding error and every
//    low-order product goes to a second FP32 sum, so a sum of products
//    c_i v_i comes out as accurately as if computed in about twice the FP32
//    precision and then rounded;
//  * double-float scalars (h, l) with the usual add and multiply.
//
// The explicit __f*_rn intrinsics keep the compiler from contracting or
// reordering the error-free transformations.
#pragma once

#include <cuda_runtime.h>

namespace apfc {

struct DF {
  float h, l;
};

// Split a double into h + l (see above).  |v| < 2^-74 and zeros give (0, 0)
// (an absolute error below 1e-22, far under the precision of the sums these
// values enter); NaN, Inf and |v| >= 2^127 give (NaN, 0) so that non-finite
// states still surface as NaN residual norms.
__device__ __forceinline__ DF split_d(double v) {
  const unsigned hw = (unsigned)__double2hiint(v);
  const unsigned lw = (unsigned)__double2loint(v);
  const unsigned E = (hw >> 20) & 0x7ffu;
  const unsigned sign = hw & 0x80000000u;
  if (E < 949u) return DF{0.f, 0.f};
  if (E >= 1151u) return DF{__uint_as_float(0x7fc00000u), 0.f};
  const float h = __uint_as_float(sign | ((E - 896u) << 23) | ((hw & 0xfffffu) << 3) | (lw >> 29));
  const unsigned q = lw & 0x1fffffffu;  // low 29 mantissa bits, in units of 2^(E-1075)
  // q >> 6 and q & 63 are below 2^23: exact floats by the 2^23 magic-number trick
  const float qa = __fsub_rn(__uint_as_float(0x4B000000u | (q >> 6)), 8388608.f);
  const float qb = __fsub_rn(__uint_as_float(0x4B000000u | (q & 63u)), 8388608.f);
  const float qf = __fmaf_rn(qa, 64.f, qb);                    // q rounded to 24 bits
  const float sc = __uint_as_float(sign | ((E - 948u) << 23));  // +-2^(E-1075), a normal float
  return DF{h, __fmul_rn(qf, sc)};
}

// Exact double of a float (zero and subnormal floats give 0, Inf and NaN give NaN).
__device__ __forceinline__ double f2d(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  if (e == 0u) return 0.0;
  if (e == 255u) return __hiloint2double(0x7ff80000, 0);
  const unsigned hi = (u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7fffffu) >> 3);
  return __hiloint2double((int)hi, (int)(u << 29));
}

// The double nearest h + l (one FP64 addition of two exact conversions).
__device__ __forceinline__ double df_to_d(DF a) { return f2d(a.h) + f2d(a.l); }

// ---- scalar error-free transformations ------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {  // |a| >= |b| or a = 0
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}

// ---- double-float scalars (relative error about 2^-44 per operation) ------------
__device__ __forceinline__ DF df_norm(float s, float e) {
  DF r;
  fast_two_sum(s, e, r.h, r.l);
  return r;
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
  float s, e;
  two_sum(a.h, b.h, s, e);
  e = __fadd_rn(e, __fadd_rn(a.l, b.l));
  return df_norm(s, e);
}
__device__ __forceinline__ DF df_neg(DF a) { return DF{-a.h, -a.l}; }
__device__ __forceinline__ DF df_sub(DF a, DF b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ DF df_mul(DF a, DF b) {
  float p, e;
  two_prod(a.h, b.h, p, e);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return df_norm(p, e);
}
__device__ __forceinline__ DF df_scale2(DF a) { return DF{__fmul_rn(2.f, a.h), __fmul_rn(2.f, a.l)}; }  // exact

// Complex double-float numbers.
struct CDF {
  DF x, y;
};
__device__ __forceinline__ CDF cdf_split(double2 v) { return CDF{split_d(v.x), split_d(v.y)}; }
__device__ __forceinline__ CDF cdf_add(CDF a, CDF b) { return CDF{df_add(a.x, b.x), df_add(a.y, b.y)}; }
__device__ __forceinline__ CDF cdf_sub(CDF a, CDF b) { return CDF{df_sub(a.x, b.x), df_sub(a.y, b.y)}; }
__device__ __forceinline__ CDF cdf_scale(DF s, CDF a) { return CDF{df_mul(s, a.x), df_mul(s, a.y)}; }
__device__ __forceinline__ CDF cdf_mul(CDF a, CDF b) {
  return CDF{df_sub(df_mul(a.x, b.x), df_mul(a.y, b.y)), df_add(df_mul(a.x, b.y), df_mul(a.y, b.x))};
}
__device__ __forceinline__ CDF cdf_conj(CDF a) { return CDF{a.x, df_neg(a.y)}; }
__device__ __forceinline__ DF cdf_abs2(CDF a) { return df_add(df_mul(a.x, a.x), df_mul(a.y, a.y)); }
__device__ __forceinline__ double2 cdf_to_d(CDF a) { return make_double2(df_to_d(a.x), df_to_d(a.y)); }

// ---- compensated sum of products, both components of a complex value at once ------
// Packed FP32 pairs (re, im) through the f32x2 instructions.
__device__ __forceinline__ unsigned long long f2pk(float2 a) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
  return r;
}
__device__ __forceinline__ float2 f2upk(unsigned long long r) {
  float2 a;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
  return a;
}
__device__ __forceinline__ float2 p_add(float2 a, float2 b) {
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2pk(a)), "l"(f2pk(b)));
  return f2upk(r);
}
__device__ __forceinline__ float2 p_sub(float2 a, float2 b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2pk(a)), "l"(f2pk(b)));
  return f2upk(r);
}
__device__ __forceinline__ float2 p_mul(float2 a, float2 b) {
  unsigned long long r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2pk(a)), "l"(f2pk(b)));
  return f2upk(r);
}
__device__ __forceinline__ float2 p_fma(float2 a, float2 b, float2 c) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(f2pk(a)), "l"(f2pk(b)), "l"(f2pk(c)));
  return f2upk(r);
}

// A complex value as packed leading parts and packed low parts: value = h + l
// componentwise.
struct PDF {
  float2 h, l;
};
__device__ __forceinline__ PDF pdf_of(CDF a) { return PDF{make_float2(a.x.h, a.y.h), make_float2(a.x.l, a.y.l)}; }
__device__ __forceinline__ PDF pdf_split(double2 v) { return pdf_of(cdf_split(v)); }

// Sum of products: s holds the running leading sum, e every error term.
struct PAcc {
  float2 s, e;
  __device__ __forceinline__ void init(PDF v) {
    s = v.h;
    e = v.l;
  }
  // s + e += v (coefficient +-1: sg = +1 or -1 in both lanes)
  __device__ __forceinline__ void add(PDF v, float sg) {
    const float2 vh = make_float2(sg * v.h.x, sg * v.h.y), vl = make_float2(sg * v.l.x, sg * v.l.y);
    const float2 t = p_add(s, vh);
    const float2 bb = p_sub(t, s);
    const float2 err = p_add(p_sub(s, p_sub(t, bb)), p_sub(vh, bb));
    s = t;
    e = p_add(e, p_add(err, vl));
  }
  // s + e += c v with a per-lane coefficient c = ch + cl (double-float pair per lane)
  __device__ __forceinline__ void fma(float2 ch, float2 cl, PDF v) {
    const float2 p = p_mul(ch, v.h);
    const float2 pe = p_fma(ch, v.h, make_float2(-p.x, -p.y));
    const float2 t = p_add(s, p);
    const float2 bb = p_sub(t, s);
    const float2 err = p_add(p_sub(s, p_sub(t, bb)), p_sub(p, bb));
    s = t;
    e = p_add(e, p_add(pe, err));
    e = p_fma(ch, v.l, e);
    e = p_fma(cl, v.h, e);
  }
  // the rounded result hi = RN(s + e) and the rest lo (TwoSum: exact in either order
  // of magnitude, as s may have cancelled below e)
  __device__ __forceinline__ void result(float2& hi, float2& lo) const {
    hi = p_add(s, e);
    const float2 bb = p_sub(hi, s);
    lo = p_add(p_sub(s, p_sub(hi, bb)), p_sub(e, bb));
  }
};

}  // namespace apfc
