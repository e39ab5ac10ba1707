// Auxiliary fields drawn on the device, and population control by the comb.
//
// Philox4x32-10 is the counter-based generator of Salmon, Moraes, Dror and Shaw
// ("Parallel random numbers: as easy as 1, 2, 3", SC 2011): a 128-bit counter
// (c0, c1, c2, c3) passes ten rounds of
//   (c0, c1, c2, c3) <- (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)),
// hi/lo the halves of the 64-bit product, with the 64-bit key (k0, k1) advanced by the
// Weyl increments (W0, W1) before every round after the first.  Any (counter, key) maps to
// four independent 32-bit words, so every walker and field has its own stream and a
// replayed graph only has to advance one counter.
#include <cstdint>

#include "attr.hpp"
#include "rng.hpp"

namespace rng {
namespace {

constexpr uint32_t PH_M0 = 0xD2511F53u, PH_M1 = 0xCD9E8D57u;   // round multipliers
constexpr uint32_t PH_W0 = 0x9E3779B9u, PH_W1 = 0xBB67AE85u;   // key increments

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k.x += PH_W0;
      k.y += PH_W1;
    }
    const uint32_t hi0 = __umulhi(PH_M0, c.x), lo0 = PH_M0 * c.x;
    const uint32_t hi1 = __umulhi(PH_M1, c.z), lo1 = PH_M1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// Box-Muller in fp32: two 23-bit uniforms strictly inside (0, 1) -> two normals
__device__ __forceinline__ void box_muller(uint32_t a, uint32_t b, float& z0, float& z1) {
  const float u1 = (__uint2float_rn(a >> 9) + 0.5f) * 0x1p-23f;
  const float u2 = (__uint2float_rn(b >> 9) + 0.5f) * 0x1p-23f;
  const float r = sqrtf(-2.f * logf(u1));
  float s, c;
  sincospif(2.f * u2, &s, &c);   // sin and cos of 2 pi u2
  z0 = r * c;
  z1 = r * s;
}

// x[w][f], f < F = 2 Nk G; counter (q, w, c_lo, c_hi) for the fields 4q .. 4q + 3
__global__ void fields_kernel(unsigned long long seed, const unsigned long long* counter, double* x, int W, int F) {
  const unsigned long long c = *counter;
  const uint2 key = make_uint2(static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
  const int nq = (F + 3) / 4;
  const long total = (long)W * nq;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
    const int w = (int)(e / nq), q = (int)(e % nq);
    const uint4 r = philox4x32_10(
        make_uint4(static_cast<uint32_t>(q), static_cast<uint32_t>(w), static_cast<uint32_t>(c),
                   static_cast<uint32_t>(c >> 32)),
        key);
    float z[4];
    box_muller(r.x, r.y, z[0], z[1]);
    box_muller(r.z, r.w, z[2], z[3]);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int f = 4 * q + u;
      if (f < F) x[(size_t)w * F + f] = (double)z[u];
    }
  }
}

__global__ void philox_raw_kernel(const uint4* ctr, uint2 key, uint4* out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = philox4x32_10(ctr[i], key);
}

__global__ void counter_bump_kernel(unsigned long long* counter) { *counter += 1ull; }

// Comb selection, one block: cumulative weights in walker order (one thread, so they are
// the plain running sums), u from Philox, then j_k = upper_bound(C, (k + u) C / W) per
// walker.  An invalid total keeps the identity and raises flags[3].
__global__ void comb_select_kernel(double* weight, unsigned long long seed, const unsigned long long* counter, int W,
                                   int* idx, int* flags) {
  extern __shared__ __align__(16) unsigned char cs[];
  double* C = reinterpret_cast<double*>(cs);   // [W]
  __shared__ double s_u, s_tot;
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    double acc = 0.0;
    for (int j = 0; j < W; ++j) {
      acc += weight[j];
      C[j] = acc;
    }
    s_tot = acc;
    s_ok = (acc > 0.0) && isfinite(acc);
    if (!s_ok) atomicAdd(&flags[3], 1);
    const unsigned long long c = *counter;
    const uint4 r = philox4x32_10(
        make_uint4(0u, 0xffffffffu, static_cast<uint32_t>(c), static_cast<uint32_t>(c >> 32)),
        make_uint2(static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32)));
    s_u = ((double)r.x + 0.5) * 0x1p-32;
  }
  __syncthreads();
  const double tot = s_tot, u = s_u;
  const int ok = s_ok;
  for (int k = threadIdx.x; k < W; k += blockDim.x) {
    int j = k;
    if (ok) {
      const double t = ((double)k + u) * tot / (double)W;
      int lo = 0, hi = W;   // first j with C[j] > t
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (C[mid] > t)
          hi = mid;
        else
          lo = mid + 1;
      }
      j = lo < W ? lo : W - 1;
    }
    idx[k] = j;
  }
  __syncthreads();   // every thread has read the old weights through C before they change
  if (ok)
    for (int k = threadIdx.x; k < W; k += blockDim.x) weight[k] = tot / (double)W;
}

// phi[k] = src[idx[k]], per walker `per` complex entries
__global__ void gather_kernel(const zc* src, const int* idx, zc* phi, int W, size_t per) {
  const size_t total = (size_t)W * per;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const size_t k = e / per, o = e % per;
    phi[e] = src[(size_t)idx[k] * per + o];
  }
}

}  // namespace

cudaError_t philox(const unsigned* ctr, unsigned long long seed, unsigned* out, size_t n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const size_t blocks = (n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096;
  philox_raw_kernel<<<(unsigned)blocks, 256, 0, st>>>(
      reinterpret_cast<const uint4*>(ctr), make_uint2(static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32)),
      reinterpret_cast<uint4*>(out), n);
  return cudaGetLastError();
}

cudaError_t fields(afqmc_kp* h, unsigned long long seed, unsigned long long* counter, double* x, cudaStream_t st) {
  const int F = 2 * h->nk * h->G;
  const long total = (long)h->W * ((F + 3) / 4);
  const int blocks = (int)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
  fields_kernel<<<blocks, 256, 0, st>>>(seed, counter, x, h->W, F);
  AFQMC_LAUNCHED(h);
  counter_bump_kernel<<<1, 1, 0, st>>>(counter);
  AFQMC_LAUNCHED(h);
  return cudaGetLastError();
}

size_t comb_smem_bytes(int W) { return (size_t)W * sizeof(double); }

cudaError_t comb(afqmc_kp* h, zc* phi, double* weight, unsigned long long seed, const unsigned long long* counter,
                 int* idx_out, cudaStream_t st) {
  const int W = h->W;
  const size_t per = (size_t)2 * h->NM * h->N;
  // the adjoint workspace Gam ([W][2][N][NM]) is free between calls: the gather source;
  // the index list goes into the handle's P workspace
  zc* src = h->Gam;
  int* idx = idx_out ? idx_out : reinterpret_cast<int*>(h->P);
  const size_t smem = (size_t)W * sizeof(double);
  if (smem > 48 * 1024) {
    cudaError_t e = ensure_dyn_smem(reinterpret_cast<const void*>(comb_select_kernel), smem);
    if (e != cudaSuccess) return e;
  }
  comb_select_kernel<<<1, 256, smem, st>>>(weight, seed, counter, W, idx, h->flags);
  AFQMC_LAUNCHED(h);
  cudaError_t e = cudaMemcpyAsync(src, phi, sizeof(zc) * W * per, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return e;
  const size_t total = (size_t)W * per;
  const int blocks = (int)((total + 255) / 256 < 8192 ? (total + 255) / 256 : 8192);
  gather_kernel<<<blocks, 256, 0, st>>>(src, idx, phi, W, per);
  AFQMC_LAUNCHED(h);
  return cudaGetLastError();
}

}  // namespace rng
