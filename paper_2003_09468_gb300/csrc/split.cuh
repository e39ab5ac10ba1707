// fp16 hi/lo operand split shared by the tensor-core GEMM operands (tc_gemm.cuh).
//
// A matrix enters a GEMM as four fp16 planes (hi, lo of the real part, hi, lo of the
// imaginary part) of x*s, with s a power of two chosen per matrix so that the
// largest |x*s| sits near SCALE_TARGET: far from the fp16 overflow, and high enough
// that lo keeps its full 11 bits.
#pragma once

#include <cuda_fp16.h>

#include <cmath>

namespace mixed {

constexpr float SCALE_TARGET = 4096.f;

__device__ __forceinline__ float pow2_scale(double maxabs) {
  if (!(maxabs > 0.0) || !isfinite(maxabs)) return 1.f;
  int e;
  frexp((double)SCALE_TARGET / maxabs, &e);  // 2^(e-1) <= target/max < 2^e
  e -= 1;
  e = max(-100, min(100, e));
  return (float)ldexp(1.0, e);
}

// x*s split into hi = fp16(x*s) and lo = fp16(x*s - hi), in fp32 (s is a power of two, so
// x*s is exact; x*s - hi is exact in fp32).  FP64 arithmetic is avoided on purpose: the
// FP64 pipe of this GPU is about 60x slower than FP32.
__device__ __forceinline__ void split_val(float xs, __half& hi, __half& lo) {
  hi = __float2half_rn(xs);
  lo = __float2half_rn(xs - __half2float(hi));
}
__device__ __forceinline__ void put4f(__half* base, size_t plane_stride, size_t idx, float re, float im) {
  __half h, l;
  split_val(re, h, l);
  base[idx] = h;
  base[plane_stride + idx] = l;
  split_val(im, h, l);
  base[2 * plane_stride + idx] = h;
  base[3 * plane_stride + idx] = l;
}
}  // namespace mixed
