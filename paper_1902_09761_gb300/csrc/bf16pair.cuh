// The shadow residual rhat of the FP32 BiCGStab solves, held as bf16.
//
// BiCGStab needs rhat only as a fixed vector that is not orthogonal to the
// initial residual; the classical choice rhat = r0 is kept, rounded to bf16
// (8 significant bits, FP32's exponent range).  The FP32 copy of rhat holds the
// rounded values exactly, and the fused v-kernel reads the bf16 copy instead:
// one packed 8-byte value per point (the bf16 pairs of rhat's zeta- and
// eta-parts) in place of two 8-byte complex values.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace apfc {

// (re, im) -> bf16 bits, re in the low half, rounded to nearest even
__device__ __forceinline__ unsigned bf16_pack(float2 v) {
  const unsigned lo = __bfloat16_as_ushort(__float2bfloat16_rn(v.x));
  const unsigned hi = __bfloat16_as_ushort(__float2bfloat16_rn(v.y));
  return lo | (hi << 16);
}
// bf16 bits -> the exact FP32 values
__device__ __forceinline__ float2 bf16_unpack(unsigned w) {
  return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
}

}  // namespace apfc
