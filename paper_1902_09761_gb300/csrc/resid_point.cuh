// The outer residual of one grid point in FP32-pair arithmetic.
//
// r = b - A x for the block operator of Eq. linear_system2 (M = I):
//   r1 = b1 - zeta + G_h eta,   r2 = b2 - kt G_h zeta - a eta,
// G_h u = c0 u + sum_d [ (1/h_d^2)(u(+d) + u(-d)) + i (k_d/h_d)(u(+d) - u(-d)) ].
// Every operand arrives as an FP32 pair (dfloat.cuh: a double split by integer
// operations) and each component of r1, r2 is one compensated sum of products
// (PAcc).  The neighbours of a dimension enter through their sum and their
// difference, each formed once as an unnormalised pair (TwoSum of the leading
// parts, the low parts and the rounding error added), so that G_h costs 1 + 2 DIM
// products instead of 1 + 4 DIM; the pair sum's error, about 2^-47 of the
// neighbours' magnitude, stays below what the compensated sum keeps anyway.
//
// The single-grid kernel (resid2d.cu, TMA tiles) and the batched kernel
// (kernels.cu, plain loads) both evaluate points here, so that a run alone and
// in a batch round alike.
#pragma once

#include "apfc_internal.cuh"
#include "dfloat.cuh"

namespace apfc {

// Lane coefficients (s0 c, s1 c) of the double-float pair of c.
struct LaneC {
  float2 h, l;
};
__device__ __forceinline__ LaneC lane_c(double c, float s0, float s1) {
  const DF d = split_d(c);
  return LaneC{make_float2(s0 * d.h, s1 * d.h), make_float2(s0 * d.l, s1 * d.l)};
}

__device__ __forceinline__ PDF pdf_swap(PDF v) {  // (re, im) -> (im, re)
  return PDF{make_float2(v.h.y, v.h.x), make_float2(v.l.y, v.l.x)};
}
// a + b and a - b as unnormalised pairs (leading parts by TwoSum)
__device__ __forceinline__ PDF pdf_add(PDF a, PDF b) {
  const float2 s = p_add(a.h, b.h);
  const float2 bb = p_sub(s, a.h);
  const float2 err = p_add(p_sub(a.h, p_sub(s, bb)), p_sub(b.h, bb));
  return PDF{s, p_add(p_add(a.l, b.l), err)};
}
__device__ __forceinline__ PDF pdf_sub(PDF a, PDF b) {
  return pdf_add(a, PDF{make_float2(-b.h.x, -b.h.y), make_float2(-b.l.x, -b.l.y)});
}
__device__ __forceinline__ float4 pdf_pack(PDF v) { return make_float4(v.h.x, v.l.x, v.h.y, v.l.y); }
__device__ __forceinline__ PDF pdf_unpack(float4 v) { return PDF{make_float2(v.x, v.z), make_float2(v.y, v.w)}; }

// Coefficients of amplitude j: G_h (centre, neighbour sums, swapped neighbour
// differences with lane signs (-1, +1)) and -kt G_h; a is passed per point.
template <int DIM>
struct ResidCoef {
  LaneC g0, gl[DIM], ga[DIM];
  LaneC k0, kl[DIM], ka[DIM];
};
template <int DIM>
__device__ __forceinline__ ResidCoef<DIM> resid_coef(const OpCoef& c, int j) {
  ResidCoef<DIM> q;
  const double kt = c.kt[j];
  q.g0 = lane_c(c.c0, 1.f, 1.f);
  q.k0 = lane_c(kt * c.c0, -1.f, -1.f);
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    q.gl[d] = lane_c(c.ih2[d], 1.f, 1.f);
    q.ga[d] = lane_c(c.kh[j][d], -1.f, 1.f);
    q.kl[d] = lane_c(kt * c.ih2[d], -1.f, -1.f);
    q.ka[d] = lane_c(kt * c.kh[j][d], 1.f, -1.f);
  }
  return q;
}

// Residual of one point: zn[d][0], zn[d][1] (and en) are the (-, +) neighbours along
// d; ma = lane_c(a, -1, -1).  Returns r1 = f1 + l1, r2 = f2 + l2 (f the rounded value).
template <int DIM>
__device__ __forceinline__ void resid_point(const ResidCoef<DIM>& q, LaneC ma, PDF b1, PDF b2, PDF zc, PDF ec,
                                            const PDF (&zn)[DIM][2], const PDF (&en)[DIM][2], float2& f1,
                                            float2& l1, float2& f2, float2& l2) {
  // r1 = b1 - zeta + G_h eta: centre, neighbour sums, neighbour differences
  PAcc a1;
  a1.init(b1);
  a1.add(zc, -1.f);
  a1.fma(q.g0.h, q.g0.l, ec);
#pragma unroll
  for (int d = 0; d < DIM; ++d) a1.fma(q.gl[d].h, q.gl[d].l, pdf_add(en[d][1], en[d][0]));
#pragma unroll
  for (int d = 0; d < DIM; ++d) a1.fma(q.ga[d].h, q.ga[d].l, pdf_swap(pdf_sub(en[d][1], en[d][0])));
  // r2 = b2 - kt G_h zeta - a eta
  PAcc a2;
  a2.init(b2);
  a2.fma(q.k0.h, q.k0.l, zc);
#pragma unroll
  for (int d = 0; d < DIM; ++d) a2.fma(q.kl[d].h, q.kl[d].l, pdf_add(zn[d][1], zn[d][0]));
#pragma unroll
  for (int d = 0; d < DIM; ++d) a2.fma(q.ka[d].h, q.ka[d].l, pdf_swap(pdf_sub(zn[d][1], zn[d][0])));
  a2.fma(ma.h, ma.l, ec);
  a1.result(f1, l1);
  a2.result(f2, l2);
}

}  // namespace apfc
