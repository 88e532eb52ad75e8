// A double as an unevaluated sum of two floats, from its bits: used where FP64
// values feed FP32 arithmetic (the bf16 operand slices of the tensor-core GEMMs, the
// double-float vector combinations), so that no FP64 instruction is issued.
#pragma once

#include <cuda_runtime.h>

namespace ccsd {

// x as hi + lo in two floats, from the double's bits with 32-bit integer operations and one
// integer-to-float conversion (no FP64 instruction: the FP64 pipe issues 2 per clock per SM).
// hi keeps the top 24 significant bits of x (truncated), lo the remaining 29 bits, rounded
// once to float: |x - hi - lo| <= 2^-47 |x|.  lo is dropped for |x| < 2^-74 (relative error
// 2^-23 there), hi flushes to zero below the float normal range and saturates above it; Inf
// and NaN go to hi with lo = 0.
__device__ __forceinline__ void double_to_float2(double x, float& hi, float& lo) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned int w1 = (unsigned int)(u >> 32), w0 = (unsigned int)u;
  const unsigned int sign = w1 & 0x80000000u;
  const int E = (int)((w1 >> 20) & 0x7FFu);
  const int fe = E - 1023 + 127;
  lo = 0.0f;
  if (E == 0x7FF) {  // Inf or NaN
    hi = __uint_as_float(sign | 0x7F800000u | (((w1 & 0xFFFFFu) | w0) ? 0x400000u : 0u));
    return;
  }
  if (fe <= 0) {
    hi = __uint_as_float(sign);
    return;
  }
  if (fe >= 255) {
    hi = __uint_as_float(sign | 0x7F800000u);
    return;
  }
  hi = __uint_as_float(sign | ((unsigned int)fe << 23) | ((w1 & 0xFFFFFu) << 3) | (w0 >> 29));
  const unsigned int low = w0 & 0x1FFFFFFFu;  // the bits below hi, in units of 2^(E - 1075)
  if (low != 0u && E >= 949) {
    const float scale = __uint_as_float((unsigned int)(E - 948) << 23);  // 2^(E - 1075), a normal float
    lo = __uint_as_float(__float_as_uint(__uint2float_rn(low) * scale) | sign);
  }
}

}  // namespace ccsd
