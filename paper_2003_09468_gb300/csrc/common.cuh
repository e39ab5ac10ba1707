// Shared device helpers of the k-point AFQMC library: complex arithmetic on
// interleaved (re, im) doubles and floats, launch checking.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

typedef double2 zc;   // complex128, interleaved
typedef float2 cc;    // complex64, interleaved

__host__ __device__ __forceinline__ zc zmake(double re, double im) { zc r; r.x = re; r.y = im; return r; }
__host__ __device__ __forceinline__ zc zzero() { return zmake(0.0, 0.0); }
__host__ __device__ __forceinline__ zc zadd(zc a, zc b) { return zmake(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ zc zsub(zc a, zc b) { return zmake(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ zc zscale(zc a, double s) { return zmake(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ zc zconj(zc a) { return zmake(a.x, -a.y); }
__host__ __device__ __forceinline__ zc zmul(zc a, zc b) {
  return zmake(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ zc zmulc(zc a, zc b) {   // a * conj(b)
  return zmake(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
// c + a * b with fused multiply-adds
__device__ __forceinline__ zc zfma(zc a, zc b, zc c) {
  c.x = fma(a.x, b.x, c.x);
  c.x = fma(-a.y, b.y, c.x);
  c.y = fma(a.x, b.y, c.y);
  c.y = fma(a.y, b.x, c.y);
  return c;
}
__device__ __forceinline__ double zabs2(zc a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ zc zdiv(zc a, zc b) {
  double d = b.x * b.x + b.y * b.y;
  return zmake((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
__device__ __forceinline__ zc zinv(zc b) {
  double d = b.x * b.x + b.y * b.y;
  return zmake(b.x / d, -b.y / d);
}

// Warp / block reductions -------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ zc warp_zsum(zc v) {
  v.x = warp_sum(v.x);
  v.y = warp_sum(v.y);
  return v;
}
// Sum over the whole block; every thread gets the result.  `red` needs
// blockDim.x / 32 entries.  Contains __syncthreads().
__device__ __forceinline__ zc block_zsum(zc v, zc* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_zsum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  zc t = zzero();
  for (int i = 0; i < nw; ++i) t = zadd(t, red[i]);
  return t;
}
__device__ __forceinline__ double block_dsum(double v, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double t = 0.0;
  for (int i = 0; i < nw; ++i) t += red[i];
  return t;
}

// Index helpers of the momentum grid --------------------------------------
// kminus[k * Nk + Q] = k - Q,  minus[Q] = -Q (tables in constant-size device arrays).
struct KTables {
  const int* kminus;  // [Nk][Nk]
  const int* minus;   // [Nk]
  int nk;
};
