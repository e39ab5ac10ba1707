// FP64 path of the k-point AFQMC walker step: every contraction in complex128
// on the FP64 pipes.  It is the precision reference on the GPU and the
// baseline the tensor-core path is measured against.
//
// Paper map (arXiv:2003.09468):
//   overlap / Green's function    Sec. 2.2 Eqs. gf, gfhrot
//   Cholesky trace X, force bias  Sec. 2.2 Eq. fb; Sec. 2.3 Eq. kp_vbias
//   vHS                           Sec. 2.2 Eq. vhs; Sec. 2.3 Eq. kp_vhs
//   Taylor exp(V), one-body half  Sec. 2.1 Eq. propagator; Sec. 2.2 (Taylor series)
//   hybrid weight                 Sec. 2.1 (importance function, phase, hybrid form)
//   local energy                  Sec. 2.2 Eq. local_energy; Sec. 2.3 Eq. kp_el;
//                                 Sec. 3.2 energy steps 1-3
#include <math.h>

#include <utility>

#include "ff.cuh"
#include "handle.hpp"

namespace fp64 {

// ---------------------------------------------------------------------------
// Generic strided-batched complex GEMM:  C = alpha op(A) op(B) + beta C
// (optionally also Acc += alpha op(A) op(B)).  op: 0 = N, 1 = T, 2 = C.
// Three batch dimensions with independent strides.
// ---------------------------------------------------------------------------
struct ZGemm {
  int m, n, k;
  int opA, opB;
  const zc* A; long lda; long sA[3];
  const zc* B; long ldb; long sB[3];
  zc* C; long ldc; long sC[3];
  zc* Acc; long ldacc; long sAcc[3];
  int nb[3];
  zc alpha, beta;
};

constexpr int GBM = 32, GBN = 32, GBK = 8;

__global__ void __launch_bounds__(256) zgemm_kernel(ZGemm g) {
  __shared__ zc As[GBK][GBM + 1];
  __shared__ zc Bs[GBK][GBN + 1];
  const int t = threadIdx.x;
  const int ty = t >> 4, tx = t & 15;
  const int row0 = blockIdx.y * GBM, col0 = blockIdx.x * GBN;
  const long nbatch = (long)g.nb[0] * g.nb[1] * g.nb[2];
  for (long z = blockIdx.z; z < nbatch; z += gridDim.z) {
    const int b2 = (int)(z % g.nb[2]);
    const int b1 = (int)((z / g.nb[2]) % g.nb[1]);
    const int b0 = (int)(z / ((long)g.nb[2] * g.nb[1]));
    const zc* A = g.A + b0 * g.sA[0] + b1 * g.sA[1] + b2 * g.sA[2];
    const zc* B = g.B + b0 * g.sB[0] + b1 * g.sB[1] + b2 * g.sB[2];
    zc* C = g.C + b0 * g.sC[0] + b1 * g.sC[1] + b2 * g.sC[2];
    zc acc[2][2];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j) acc[i][j] = zzero();
    for (int p0 = 0; p0 < g.k; p0 += GBK) {
      {  // A tile: op(A)[row0 + i][p0 + p]
        int i, p;
        if (g.opA == 0) { i = t >> 3; p = t & 7; } else { p = t >> 5; i = t & 31; }
        const int gi = row0 + i, gp = p0 + p;
        zc v = zzero();
        if (gi < g.m && gp < g.k) {
          if (g.opA == 0) v = A[(long)gi * g.lda + gp];
          else { v = A[(long)gp * g.lda + gi]; if (g.opA == 2) v = zconj(v); }
        }
        As[p][i] = v;
      }
      {  // B tile: op(B)[p0 + p][col0 + j]
        int j, p;
        if (g.opB == 0) { p = t >> 5; j = t & 31; } else { j = t >> 3; p = t & 7; }
        const int gj = col0 + j, gp = p0 + p;
        zc v = zzero();
        if (gj < g.n && gp < g.k) {
          if (g.opB == 0) v = B[(long)gp * g.ldb + gj];
          else { v = B[(long)gj * g.ldb + gp]; if (g.opB == 2) v = zconj(v); }
        }
        Bs[p][j] = v;
      }
      __syncthreads();
#pragma unroll
      for (int p = 0; p < GBK; ++p) {
        zc a0 = As[p][ty * 2], a1 = As[p][ty * 2 + 1];
        zc c0 = Bs[p][tx * 2], c1 = Bs[p][tx * 2 + 1];
        acc[0][0] = zfma(a0, c0, acc[0][0]);
        acc[0][1] = zfma(a0, c1, acc[0][1]);
        acc[1][0] = zfma(a1, c0, acc[1][0]);
        acc[1][1] = zfma(a1, c1, acc[1][1]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int gi = row0 + ty * 2 + i, gj = col0 + tx * 2 + j;
        if (gi < g.m && gj < g.n) {
          zc r = zmul(g.alpha, acc[i][j]);
          zc* c = C + (long)gi * g.ldc + gj;
          if (g.beta.x != 0.0 || g.beta.y != 0.0) r = zfma(g.beta, *c, r);
          *c = r;
          if (g.Acc) {
            zc* a = g.Acc + b0 * g.sAcc[0] + b1 * g.sAcc[1] + b2 * g.sAcc[2] + (long)gi * g.ldacc + gj;
            *a = zadd(*a, zmul(g.alpha, acc[i][j]));
          }
        }
      }
  }
}

// The same GEMM in double-float arithmetic on the FP32 pipe (ff.cuh): FP64 operands are
// split into hi + lo fp32 pairs as the tiles are staged, products and sums run through the
// error-free transformations (about 48 significant bits), and the result is rounded back to
// FP64.  Tile 64 x 64, 4 x 4 outputs per thread.
constexpr int FBM = 64, FBN = 64, FBK = 8;

__device__ __forceinline__ float4 ff_load(const zc* M, long ld, int r, int c, int op, int rows, int cols) {
  // element (r, c) of op(M) as a double-float complex, zero outside rows x cols
  if (r >= rows || c >= cols) return ffa::czero();
  zc v = op == 0 ? M[(long)r * ld + c] : M[(long)c * ld + r];
  if (op == 2) v = zconj(v);
  return ffa::cfrom(v);
}

__global__ void __launch_bounds__(256) zgemm_ff_kernel(ZGemm g) {
  __shared__ float4 As[FBK][FBM];
  __shared__ float4 Bs[FBK][FBN];
  const int t = threadIdx.x;
  const int ty = t >> 4, tx = t & 15;
  const int row0 = blockIdx.y * FBM, col0 = blockIdx.x * FBN;
  const long nbatch = (long)g.nb[0] * g.nb[1] * g.nb[2];
  for (long z = blockIdx.z; z < nbatch; z += gridDim.z) {
    const int b2 = (int)(z % g.nb[2]);
    const int b1 = (int)((z / g.nb[2]) % g.nb[1]);
    const int b0 = (int)(z / ((long)g.nb[2] * g.nb[1]));
    const zc* A = g.A + b0 * g.sA[0] + b1 * g.sA[1] + b2 * g.sA[2];
    const zc* B = g.B + b0 * g.sB[0] + b1 * g.sB[1] + b2 * g.sB[2];
    zc* C = g.C + b0 * g.sC[0] + b1 * g.sC[1] + b2 * g.sC[2];
    ffa::cacc acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = ffa::cacc_from(ffa::czero());
    for (int p0 = 0; p0 < g.k; p0 += FBK) {
      __syncthreads();
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int e = t + u * 256;
        // coalesced along the operand's contiguous index
        int i, p;
        if (g.opA == 0) { i = e >> 3; p = e & 7; } else { p = e >> 6; i = e & 63; }
        As[p][i] = ff_load(A, g.lda, row0 + i, p0 + p, g.opA, g.m, g.k);
        int j, q;
        if (g.opB == 0) { q = e >> 6; j = e & 63; } else { j = e >> 3; q = e & 7; }
        // op(B)[q][j]: stored element (q, j) for N, (j, q) for T / C
        float4 bv = ffa::czero();
        if (col0 + j < g.n && p0 + q < g.k) {
          zc v = g.opB == 0 ? B[(long)(p0 + q) * g.ldb + col0 + j] : B[(long)(col0 + j) * g.ldb + p0 + q];
          if (g.opB == 2) v = zconj(v);
          bv = ffa::cfrom(v);
        }
        Bs[q][j] = bv;
      }
      __syncthreads();
#pragma unroll 2
      for (int p = 0; p < FBK; ++p) {
        float4 a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = As[p][ty * 4 + i];
#pragma unroll
        for (int j = 0; j < 4; ++j) b[j] = Bs[p][tx * 4 + j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) ffa::cacc_fma(acc[i][j], a[i], b[j]);
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int gi = row0 + ty * 4 + i, gj = col0 + tx * 4 + j;
        if (gi < g.m && gj < g.n) {
          const float4 v = ffa::cacc_get(acc[i][j]);
          const zc s = zmake(ffa::to_double(ffa::re(v)), ffa::to_double(ffa::im(v)));
          zc r = zmul(g.alpha, s);
          zc* c = C + (long)gi * g.ldc + gj;
          if (g.beta.x != 0.0 || g.beta.y != 0.0) r = zfma(g.beta, *c, r);
          *c = r;
          if (g.Acc) {
            zc* a = g.Acc + b0 * g.sAcc[0] + b1 * g.sAcc[1] + b2 * g.sAcc[2] + (long)gi * g.ldacc + gj;
            *a = zadd(*a, zmul(g.alpha, s));
          }
        }
      }
  }
}

static ZGemm gemm_init(int m, int n, int k, int opA, int opB) {
  ZGemm g;
  memset(&g, 0, sizeof(g));
  g.m = m; g.n = n; g.k = k; g.opA = opA; g.opB = opB;
  g.nb[0] = g.nb[1] = g.nb[2] = 1;
  g.alpha = zmake(1.0, 0.0);
  g.beta = zzero();
  return g;
}

static cudaError_t gemm_launch(afqmc_kp* h, const ZGemm& g, cudaStream_t st) {
  long nb = (long)g.nb[0] * g.nb[1] * g.nb[2];
  dim3 grid((g.n + GBN - 1) / GBN, (g.m + GBM - 1) / GBM, (unsigned)(nb < 65535 ? nb : 65535));
  zgemm_kernel<<<grid, 256, 0, st>>>(g);
  AFQMC_LAUNCHED(h);
  return cudaGetLastError();
}

static cudaError_t gemm_launch_ff(afqmc_kp* h, const ZGemm& g, cudaStream_t st) {
  long nb = (long)g.nb[0] * g.nb[1] * g.nb[2];
  dim3 grid((g.n + FBN - 1) / FBN, (g.m + FBM - 1) / FBM, (unsigned)(nb < 65535 ? nb : 65535));
  zgemm_ff_kernel<<<grid, 256, 0, st>>>(g);
  AFQMC_LAUNCHED(h);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Set-up kernels
// ---------------------------------------------------------------------------

// v0[k][p][q] = -1/2 sum_{Q,g,r} L[Q][k][g][p][r] conj(L[Q][k][g][q][r])
// v0[k] = -1/2 sum_{Q,g} L[Q,k,g] L[Q,k,g]^dagger in two passes: one block per (k, Q) sums
// its g's into part[k][Q] (the block reads its own slab of L once; the M x M products run
// from L1), then the Q partials are added in a fixed order.
__global__ void v0_partial_kernel(const zc* L, zc* part, int nk, int G, int M) {
  const int k = blockIdx.x, Q = blockIdx.y;
  const int MM = M * M;
  const zc* slab = L + ((size_t)Q * nk + k) * G * MM;
  zc* out = part + ((size_t)k * nk + Q) * MM;
  for (int o = threadIdx.x; o < MM; o += blockDim.x) {
    const int p = o / M, q = o % M;
    zc s = zzero();
    for (int g = 0; g < G; ++g) {
      const zc* blk = slab + (size_t)g * MM;
      for (int r = 0; r < M; ++r) s = zfma(blk[p * M + r], zconj(blk[q * M + r]), s);
    }
    out[o] = s;
  }
}
__global__ void v0_reduce_kernel(const zc* part, zc* v0, int nk, int M) {
  const int k = blockIdx.x, MM = M * M;
  for (int o = threadIdx.x; o < MM; o += blockDim.x) {
    zc s = zzero();
    for (int Q = 0; Q < nk; ++Q) s = zadd(s, part[((size_t)k * nk + Q) * MM + o]);
    v0[(size_t)k * MM + o] = zscale(s, -0.5);
  }
}

// Ehalf[k] = exp(-dt/2 (h[k] + v0[k])) by scaling, 24-term Taylor series and squaring.
// tmp: [k][3][M][M].  One block per k.
__global__ void expm_kernel(const zc* h1, const zc* v0, zc* out, zc* tmp, int M, double dt) {
  const int k = blockIdx.x;
  const long MM = (long)M * M;
  zc* Xm = tmp + (long)k * 3 * MM;
  zc* Tm = Xm + MM;
  zc* Rm = Tm + MM;
  zc* E = out + k * MM;
  __shared__ double red[32];
  __shared__ int s_sq;
  // X = -dt/2 (h + v0); 1-norm bound for scaling
  double rowmax = 0.0;
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < M; ++j) {
      zc v = zscale(zadd(h1[k * MM + i * M + j], v0[k * MM + i * M + j]), -0.5 * dt);
      Xm[i * M + j] = v;
      s += sqrt(zabs2(v));
    }
    rowmax = fmax(rowmax, s);
  }
  // block max via sum of squares is not a max; do a simple max reduction
  {
    double v = rowmax;
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double m = 0.0;
      for (int i = 0; i < (int)((blockDim.x + 31) >> 5); ++i) m = fmax(m, red[i]);
      int sq = 0;
      while (m > 0.25 && sq < 60) { m *= 0.5; ++sq; }
      s_sq = sq;
    }
    __syncthreads();
  }
  const int sq = s_sq;
  const double scl = ldexp(1.0, -sq);
  for (long e = threadIdx.x; e < MM; e += blockDim.x) {
    Xm[e] = zscale(Xm[e], scl);
    const int i = (int)(e / M), j = (int)(e % M);
    E[e] = zmake(i == j ? 1.0 : 0.0, 0.0);
    Tm[e] = E[e];
  }
  __syncthreads();
  for (int term = 1; term <= 24; ++term) {
    // Rm = Tm * Xm / term
    for (long e = threadIdx.x; e < MM; e += blockDim.x) {
      const int i = (int)(e / M), j = (int)(e % M);
      zc s = zzero();
      for (int l = 0; l < M; ++l) s = zfma(Tm[i * M + l], Xm[l * M + j], s);
      Rm[e] = zscale(s, 1.0 / term);
    }
    __syncthreads();
    for (long e = threadIdx.x; e < MM; e += blockDim.x) {
      Tm[e] = Rm[e];
      E[e] = zadd(E[e], Rm[e]);
    }
    __syncthreads();
  }
  for (int s = 0; s < sq; ++s) {
    for (long e = threadIdx.x; e < MM; e += blockDim.x) {
      const int i = (int)(e / M), j = (int)(e % M);
      zc acc = zzero();
      for (int l = 0; l < M; ++l) acc = zfma(E[i * M + l], E[l * M + j], acc);
      Rm[e] = acc;
    }
    __syncthreads();
    for (long e = threadIdx.x; e < MM; e += blockDim.x) E[e] = Rm[e];
    __syncthreads();
  }
}

static cudaError_t configure_smem(afqmc_kp* h);

cudaError_t setup_static(afqmc_kp* h, cudaStream_t st) {
  const int nk = h->nk, M = h->M, n = h->n, G = h->G;
  {
    cudaError_t e = configure_smem(h);
    if (e != cudaSuccess) return e;
  }
  // LH[Q][k][g] = A[k]^dagger L[Q][k][g]
  {
    ZGemm g = gemm_init(n, M, M, 2, 0);
    g.A = h->A; g.lda = n; g.sA[0] = 0; g.sA[1] = (long)M * n; g.sA[2] = 0;
    g.B = h->L; g.ldb = M; g.sB[0] = (long)nk * G * M * M; g.sB[1] = (long)G * M * M; g.sB[2] = (long)M * M;
    g.C = h->LH; g.ldc = M; g.sC[0] = (long)nk * G * n * M; g.sC[1] = (long)G * n * M; g.sC[2] = (long)n * M;
    g.nb[0] = nk; g.nb[1] = nk; g.nb[2] = G;
    cudaError_t e = gemm_launch(h, g, st);
    if (e != cudaSuccess) return e;
  }
  {
    // the Q partials of v0 live in a temporary buffer (create time: allocation is allowed)
    zc* part = nullptr;
    cudaError_t e = cudaMalloc(&part, sizeof(zc) * (size_t)nk * nk * M * M);
    if (e != cudaSuccess) return e;
    v0_partial_kernel<<<dim3(nk, nk), 256, 0, st>>>(h->L, part, nk, G, M);
    AFQMC_LAUNCHED(h);
    v0_reduce_kernel<<<nk, 256, 0, st>>>(part, h->v0, nk, M);
    AFQMC_LAUNCHED(h);
    e = cudaGetLastError();
    const cudaError_t e2 = cudaStreamSynchronize(st);
    cudaFree(part);
    if (e != cudaSuccess) return e;
    if (e2 != cudaSuccess) return e2;
  }
  return set_one_body(h, st);
}

cudaError_t set_one_body(afqmc_kp* h, cudaStream_t st) {
  const int nk = h->nk, M = h->M, n = h->n;
  ZGemm g = gemm_init(n, M, M, 2, 0);  // AhH[k] = A[k]^dagger h[k]
  g.A = h->A; g.lda = n; g.sA[0] = (long)M * n;
  g.B = h->h1; g.ldb = M; g.sB[0] = (long)M * M;
  g.C = h->AhH; g.ldc = M; g.sC[0] = (long)n * M;
  g.nb[0] = nk;
  cudaError_t e = gemm_launch(h, g, st);
  if (e != cudaSuccess) return e;
  expm_kernel<<<nk, 256, 0, st>>>(h->h1, h->v0, h->Ehalf, h->expm_tmp, M, h->dt);
  AFQMC_LAUNCHED(h);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Overlap, LU with partial pivoting, log det and inverse (one block per matrix)
// ---------------------------------------------------------------------------

// S[ws][(k,a)][j] = sum_p conj(A[k][p][a]) phi[ws][(k,p)][j]
// Block (ws, k); threads over j, eight rows a at a time held in registers.
constexpr int OVA = 8;
__global__ void __launch_bounds__(256) overlap_kernel(const zc* A, const zc* phi, zc* S, int nk, int M, int n,
                                                      int N) {
  const int ws = blockIdx.x, k = blockIdx.y;
  const zc* Ak = A + (size_t)k * M * n;
  const zc* ph = phi + ((size_t)ws * nk * M + (size_t)k * M) * N;
  zc* Sk = S + ((size_t)ws * N + (size_t)k * n) * N;
  for (int a0 = 0; a0 < n; a0 += OVA) {
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
      zc acc[OVA];
#pragma unroll
      for (int i = 0; i < OVA; ++i) acc[i] = zzero();
      for (int p = 0; p < M; ++p) {
        const zc v = ph[(size_t)p * N + j];
#pragma unroll
        for (int i = 0; i < OVA; ++i)
          if (a0 + i < n) acc[i] = zfma(zconj(Ak[p * n + a0 + i]), v, acc[i]);
      }
#pragma unroll
      for (int i = 0; i < OVA; ++i)
        if (a0 + i < n) Sk[(size_t)(a0 + i) * N + j] = acc[i];
    }
  }
}

static cudaError_t overlap(afqmc_kp* h, const zc* phi, cudaStream_t st) {
  overlap_kernel<<<dim3(2 * h->W, h->nk), 256, 0, st>>>(h->A, phi, h->S, h->nk, h->M, h->n, h->N);
  AFQMC_LAUNCHED(h);
  return cudaGetLastError();
}

// In-place LU of S (row pivoting), log det, optional inverse.  sing[b] = 1 if a
// pivot is zero or not finite; then Sinv = 0 and logdet = (-inf, 0).
__global__ void __launch_bounds__(256) lu_kernel(zc* S, zc* Sinv, zc* logdet, int* sing, int* flags,
                                                 int N, int want_inv, int* perm_ws) {
  const int b = blockIdx.x;
  zc* a = S + (long)b * N * N;
  int* perm = perm_ws + (long)b * N;
  __shared__ double s_val[256];
  __shared__ int s_idx[256];
  __shared__ int s_sing;
  __shared__ double s_logabs, s_arg;
  __shared__ int s_swaps;
  if (threadIdx.x == 0) { s_sing = 0; s_logabs = 0.0; s_arg = 0.0; s_swaps = 0; }
  for (int i = threadIdx.x; i < N; i += blockDim.x) perm[i] = i;
  __syncthreads();
  for (int j = 0; j < N; ++j) {
    double best = -1.0;
    int bi = j;
    for (int i = j + threadIdx.x; i < N; i += blockDim.x) {
      double v = zabs2(a[(long)i * N + j]);
      if (v > best) { best = v; bi = i; }
    }
    s_val[threadIdx.x] = best;
    s_idx[threadIdx.x] = bi;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) {
        double v2 = s_val[threadIdx.x + o];
        int i2 = s_idx[threadIdx.x + o];
        if (v2 > s_val[threadIdx.x] || (v2 == s_val[threadIdx.x] && i2 < s_idx[threadIdx.x])) {
          s_val[threadIdx.x] = v2;
          s_idx[threadIdx.x] = i2;
        }
      }
      __syncthreads();
    }
    const int p = s_idx[0];
    const double pv = s_val[0];
    if (!(pv > 0.0) || !isfinite(pv)) {
      if (threadIdx.x == 0) s_sing = 1;
      __syncthreads();
      break;
    }
    if (p != j) {
      for (int c = threadIdx.x; c < N; c += blockDim.x) {
        zc t = a[(long)j * N + c];
        a[(long)j * N + c] = a[(long)p * N + c];
        a[(long)p * N + c] = t;
      }
      if (threadIdx.x == 0) {
        int t = perm[j]; perm[j] = perm[p]; perm[p] = t;
        s_swaps++;
      }
    }
    __syncthreads();
    const zc piv = a[(long)j * N + j];
    if (threadIdx.x == 0) {
      s_logabs += 0.5 * log(zabs2(piv));
      s_arg += atan2(piv.y, piv.x);
    }
    const zc inv = zinv(piv);
    for (int i = j + 1 + threadIdx.x; i < N; i += blockDim.x) a[(long)i * N + j] = zmul(a[(long)i * N + j], inv);
    __syncthreads();
    const int rem = N - j - 1;
    for (long e = threadIdx.x; e < (long)rem * rem; e += blockDim.x) {
      const int i = j + 1 + (int)(e / rem), c = j + 1 + (int)(e % rem);
      a[(long)i * N + c] = zfma(zmake(-a[(long)i * N + j].x, -a[(long)i * N + j].y), a[(long)j * N + c],
                                a[(long)i * N + c]);
    }
    __syncthreads();
  }
  const int singular = s_sing;
  if (threadIdx.x == 0) {
    if (singular) {
      logdet[b] = zmake(-INFINITY, 0.0);
      sing[b] = 1;
      atomicAdd(&flags[0], 1);
    } else {
      double ang = s_arg + (s_swaps & 1 ? M_PI : 0.0);
      ang = remainder(ang, 2.0 * M_PI);
      logdet[b] = zmake(s_logabs, ang);
      sing[b] = 0;
    }
  }
  if (!want_inv) return;
  zc* x = Sinv + (long)b * N * N;
  if (singular) {
    for (long e = threadIdx.x; e < (long)N * N; e += blockDim.x) x[e] = zzero();
    return;
  }
  // Column c of S^-1 solves L U x = P e_c: forward (unit lower), then backward.
  for (int c = threadIdx.x; c < N; c += blockDim.x) {
    for (int i = 0; i < N; ++i) {
      zc s = zmake(perm[i] == c ? 1.0 : 0.0, 0.0);
      for (int l = 0; l < i; ++l) s = zfma(zmake(-a[(long)i * N + l].x, -a[(long)i * N + l].y), x[(long)l * N + c], s);
      x[(long)i * N + c] = s;
    }
    for (int i = N - 1; i >= 0; --i) {
      zc s = x[(long)i * N + c];
      for (int l = i + 1; l < N; ++l) s = zfma(zmake(-a[(long)i * N + l].x, -a[(long)i * N + l].y), x[(long)l * N + c], s);
      x[(long)i * N + c] = zmul(s, zinv(a[(long)i * N + i]));
    }
  }
}

// Gh[w][s] = (phi S^-1)^T = S^-T phi^T  (N x NM)
static cudaError_t green_impl(afqmc_kp* h, const zc* phi, zc* ld, int* sing, cudaStream_t st, bool ff = false) {
  cudaError_t e = overlap(h, phi, st);
  if (e != cudaSuccess) return e;
  // pivot scratch lives in the P buffer (used otherwise only by the backward pass)
  lu_kernel<<<2 * h->W, 256, 0, st>>>(h->S, h->Sinv, ld, sing, h->flags, h->N, 1, reinterpret_cast<int*>(h->P));
  AFQMC_LAUNCHED(h);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int N = h->N, NM = h->NM;
  ZGemm g = gemm_init(N, NM, N, 1, 1);
  g.A = h->Sinv; g.lda = N; g.sA[0] = (long)N * N;
  g.B = phi; g.ldb = N; g.sB[0] = (long)NM * N;
  g.C = h->Gh; g.ldc = NM; g.sC[0] = (long)N * NM;
  g.nb[0] = 2 * h->W;
  return ff ? gemm_launch_ff(h, g, st) : gemm_launch(h, g, st);
}

cudaError_t green(afqmc_kp* h, const zc* phi, cudaStream_t st) {
  prof_begin(h, AFQMC_STAGE_GREEN, st);
  cudaError_t e = green_impl(h, phi, h->ld_old, h->sing_old, st);
  prof_end(h, st);
  return e;
}

cudaError_t green_ff(afqmc_kp* h, const zc* phi, cudaStream_t st) {
  prof_begin(h, AFQMC_STAGE_GREEN, st);
  cudaError_t e = green_impl(h, phi, h->ld_old, h->sing_old, st, true);
  prof_end(h, st);
  return e;
}

// ---------------------------------------------------------------------------
// Cholesky trace X[w][Q][g] = sum_k sum_{a,r} LH[Q][k][g][a][r] (Gh_up + Gh_dn)[(k,a)][(k-Q,r)]
// Block (Q, walker chunk); one warp per g at a time, lanes over (a, r).
// ---------------------------------------------------------------------------
constexpr int XWC = 8;  // walkers per block

__global__ void __launch_bounds__(256) xtrace_kernel(const zc* LH, const zc* Gh, zc* X, const int* kminus,
                                                     int nk, int G, int M, int n, int W) {
  extern __shared__ zc sm[];  // [XWC][n*M]
  const int Q = blockIdx.x, w0 = blockIdx.y * XWC;
  const int N = nk * n, NM = nk * M, nM = n * M;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  for (int g0 = 0; g0 < G; g0 += nwarp) {
    const int g = g0 + wid;
    zc acc[XWC];
#pragma unroll
    for (int i = 0; i < XWC; ++i) acc[i] = zzero();
    for (int k = 0; k < nk; ++k) {
      const int kq = kminus[k * nk + Q];
      __syncthreads();
      for (int e = threadIdx.x; e < XWC * nM; e += blockDim.x) {
        const int wi = e / nM, ar = e % nM, a = ar / M, r = ar % M;
        const int w = w0 + wi;
        zc v = zzero();
        if (w < W) {
          const zc* g0p = Gh + ((long)(w * 2 + 0) * N + k * n + a) * NM + kq * M + r;
          const zc* g1p = Gh + ((long)(w * 2 + 1) * N + k * n + a) * NM + kq * M + r;
          v = zadd(*g0p, *g1p);
        }
        sm[e] = v;
      }
      __syncthreads();
      if (g < G) {
        const zc* lh = LH + (((long)Q * nk + k) * G + g) * nM;
        for (int ar = lane; ar < nM; ar += 32) {
          const zc l = lh[ar];
#pragma unroll
          for (int i = 0; i < XWC; ++i) acc[i] = zfma(l, sm[i * nM + ar], acc[i]);
        }
      }
    }
#pragma unroll
    for (int i = 0; i < XWC; ++i) {
      zc v = warp_zsum(acc[i]);
      if (lane == 0 && g < G && w0 + i < W) X[((long)(w0 + i) * nk + Q) * G + g] = v;
    }
  }
}

cudaError_t cholesky_trace(afqmc_kp* h, cudaStream_t st) {
  dim3 grid(h->nk, (h->W + XWC - 1) / XWC);
  size_t smem = sizeof(zc) * XWC * h->n * h->M;
  xtrace_kernel<<<grid, 256, smem, st>>>(h->LH, h->Gh, h->X, h->kminus, h->nk, h->G, h->M, h->n, h->W);
  AFQMC_LAUNCHED(h);
  return cudaGetLastError();
}

// xbar from X; y = sqrt(dt) * vHS coefficients (needs x; skipped when x == NULL).
__global__ void xbar_kernel(const zc* X, const double* x, zc* xbar, zc* y, const int* minus, int nk, int G,
                            long total, double sqdt) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
    const int g = (int)(e % G);
    const int Q = (int)((e / G) % nk);
    const long w = e / ((long)G * nk);
    const int mQ = minus[Q];
    const zc XQ = X[(w * nk + Q) * G + g], XmQ = X[(w * nk + mQ) * G + g];
    // <v+> = i (X_Q + X_-Q)/2, <v-> = -(X_Q - X_-Q)/2, xbar = -sqrt(dt) <v>
    const zc s = zadd(XQ, XmQ), d = zsub(XQ, XmQ);
    const zc xbp = zmake(0.5 * sqdt * s.y, -0.5 * sqdt * s.x);   // -sqdt * i s / 2
    const zc xbm = zscale(d, 0.5 * sqdt);                         //  sqdt * d / 2
    xbar[((w * 2 + 0) * nk + Q) * G + g] = xbp;
    xbar[((w * 2 + 1) * nk + Q) * G + g] = xbm;
    if (x) {
      // xbar at -Q: s is symmetric, d flips sign
      const zc xbp_m = xbp, xbm_m = zscale(d, -0.5 * sqdt);
      const zc tpQ = zsub(zmake(x[((w * 2 + 0) * nk + Q) * G + g], 0.0), xbp);
      const zc tmQ = zsub(zmake(x[((w * 2 + 1) * nk + Q) * G + g], 0.0), xbm);
      const zc tpM = zsub(zmake(x[((w * 2 + 0) * nk + mQ) * G + g], 0.0), xbp_m);
      const zc tmM = zsub(zmake(x[((w * 2 + 1) * nk + mQ) * G + g], 0.0), xbm_m);
      // y = (i tp_Q - tm_Q)/2 + (i tp_-Q + tm_-Q)/2
      zc v = zmake(-tpQ.y - tmQ.x - tpM.y + tmM.x, tpQ.x - tmQ.y + tpM.x + tmM.y);
      y[(w * nk + Q) * G + g] = zscale(v, 0.5 * sqdt);
    }
  }
}

cudaError_t force_bias(afqmc_kp* h, const double* x, zc* xbar_out, cudaStream_t st) {
  long total = (long)h->W * h->nk * h->G;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  xbar_kernel<<<blocks, 256, 0, st>>>(h->X, x, xbar_out, h->y, h->minus, h->nk, h->G, total, h->sqdt);
  AFQMC_LAUNCHED(h);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// vHS: V[w][(k,p)][(k-Q,r)] = sum_g L[Q][k][g][p][r] y[w][Q][g]   (y carries sqrt(dt))
// Block (Q*nk + k, walker chunk); threads over (p, r).
// ---------------------------------------------------------------------------
constexpr int VWC = 8;

__global__ void __launch_bounds__(256) vhs_kernel(const zc* L, const zc* y, zc* V, const int* kminus, int nk,
                                                  int G, int M, int W) {
  extern __shared__ zc ys[];  // [VWC][G]
  const int Q = blockIdx.x / nk, k = blockIdx.x % nk, w0 = blockIdx.y * VWC;
  const int kq = kminus[k * nk + Q];
  const int NM = nk * M, MM = M * M;
  for (int e = threadIdx.x; e < VWC * G; e += blockDim.x) {
    const int wi = e / G, g = e % G;
    ys[e] = (w0 + wi < W) ? y[((long)(w0 + wi) * nk + Q) * G + g] : zzero();
  }
  __syncthreads();
  const zc* blk = L + ((long)Q * nk + k) * G * MM;
  for (int pr = threadIdx.x; pr < MM; pr += blockDim.x) {
    zc acc[VWC];
#pragma unroll
    for (int i = 0; i < VWC; ++i) acc[i] = zzero();
    for (int g = 0; g < G; ++g) {
      const zc l = blk[(long)g * MM + pr];
#pragma unroll
      for (int i = 0; i < VWC; ++i) acc[i] = zfma(l, ys[i * G + g], acc[i]);
    }
    const int p = pr / M, r = pr % M;
#pragma unroll
    for (int i = 0; i < VWC; ++i)
      if (w0 + i < W) V[(long)(w0 + i) * NM * NM + (long)(k * M + p) * NM + kq * M + r] = acc[i];
  }
}

// ---------------------------------------------------------------------------
// Hybrid weight: one block per walker.
// ---------------------------------------------------------------------------
__global__ void weight_kernel(const double* x, const zc* xbar, const zc* ld_old, const zc* ld_new,
                              const int* sing_old, const int* sing_new, double* weight, zc* logdet_out,
                              int nf) {
  const int w = blockIdx.x;
  __shared__ zc red[32];
  zc s = zzero();
  for (int f = threadIdx.x; f < nf; f += blockDim.x) {
    const double xf = x[(long)w * nf + f];
    const zc xb = xbar[(long)w * nf + f];
    // x xbar - xbar^2 / 2
    const zc xb2 = zmul(xb, xb);
    s = zadd(s, zmake(xf * xb.x - 0.5 * xb2.x, xf * xb.y - 0.5 * xb2.y));
  }
  s = block_zsum(s, red);
  if (threadIdx.x == 0) {
    const bool dead = sing_old[2 * w] || sing_old[2 * w + 1] || sing_new[2 * w] || sing_new[2 * w + 1];
    double wn = 0.0;
    if (!dead) {
      const zc dlog = zadd(zsub(ld_new[2 * w], ld_old[2 * w]), zsub(ld_new[2 * w + 1], ld_old[2 * w + 1]));
      const double c = cos(dlog.y);
      wn = weight[w] * exp(dlog.x + s.x) * (c > 0.0 ? c : 0.0);
    }
    weight[w] = wn;
    if (logdet_out) {
      logdet_out[2 * w] = ld_new[2 * w];
      logdet_out[2 * w + 1] = ld_new[2 * w + 1];
    }
  }
}

// ---------------------------------------------------------------------------
// Householder QR of each walker spin block (NM x N), Q factor with diag(R) > 0.
// One block per (w, s); phi overwritten; Qm is NM x N scratch.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) qr_kernel(zc* phi, zc* Qm_ws, int NM, int N) {
  const int b = blockIdx.x;
  zc* a = phi + (long)b * NM * N;
  zc* Qm = Qm_ws + (long)b * NM * N;
  extern __shared__ unsigned char qsm[];
  zc* alpha = reinterpret_cast<zc*>(qsm);          // [N]  R_jj
  zc* vhead = alpha + N;                           // [N]  first entry of v_j
  double* vn2 = reinterpret_cast<double*>(vhead + N);  // [N] |v_j|^2
  __shared__ double redd[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  for (int j = 0; j < N; ++j) {
    double ss = 0.0;
    for (int i = j + threadIdx.x; i < NM; i += blockDim.x) ss += zabs2(a[(long)i * N + j]);
    ss = block_dsum(ss, redd);
    const zc x0 = a[(long)j * N + j];
    const double nx = sqrt(ss);
    const double ax0 = sqrt(zabs2(x0));
    const zc ph = ax0 > 0.0 ? zscale(x0, 1.0 / ax0) : zmake(1.0, 0.0);
    const zc al = zscale(ph, -nx);                 // alpha = -e^{i arg x0} |x|
    const zc v0 = zsub(x0, al);                    // v = x - alpha e_0
    const double v2 = ss - zabs2(x0) + zabs2(v0);  // |v|^2
    if (threadIdx.x == 0) { alpha[j] = al; vhead[j] = v0; vn2[j] = v2; }
    __syncthreads();
    // apply H = I - 2 v v^H / |v|^2 to columns c > j ; v_i = a[i][j] for i > j, v_j = v0
    for (int c = j + 1 + wid; c < N; c += nwarp) {
      zc d = zzero();
      for (int i = j + lane; i < NM; i += 32) {
        const zc vi = (i == j) ? v0 : a[(long)i * N + j];
        d = zfma(zconj(vi), a[(long)i * N + c], d);
      }
      d = warp_zsum(d);
      const zc f = v2 > 0.0 ? zscale(d, -2.0 / v2) : zzero();
      for (int i = j + lane; i < NM; i += 32) {
        const zc vi = (i == j) ? v0 : a[(long)i * N + j];
        a[(long)i * N + c] = zfma(vi, f, a[(long)i * N + c]);
      }
    }
    __syncthreads();
  }
  // Q = H_0 ... H_{N-1} [I; 0], built backwards into Qm
  for (long e = threadIdx.x; e < (long)NM * N; e += blockDim.x) {
    const int i = (int)(e / N), c = (int)(e % N);
    Qm[e] = zmake(i == c ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  for (int j = N - 1; j >= 0; --j) {
    const zc v0 = vhead[j];
    const double v2 = vn2[j];
    for (int c = wid; c < N; c += nwarp) {
      zc d = zzero();
      for (int i = j + lane; i < NM; i += 32) {
        const zc vi = (i == j) ? v0 : a[(long)i * N + j];
        d = zfma(zconj(vi), Qm[(long)i * N + c], d);
      }
      d = warp_zsum(d);
      const zc f = v2 > 0.0 ? zscale(d, -2.0 / v2) : zzero();
      for (int i = j + lane; i < NM; i += 32) {
        const zc vi = (i == j) ? v0 : a[(long)i * N + j];
        Qm[(long)i * N + c] = zfma(vi, f, Qm[(long)i * N + c]);
      }
    }
    __syncthreads();
  }
  // phi = Qm diag(alpha_j / |alpha_j|)  (makes diag(R) real positive)
  for (long e = threadIdx.x; e < (long)NM * N; e += blockDim.x) {
    const int c = (int)(e % N);
    const zc al = alpha[c];
    const double aa = sqrt(zabs2(al));
    const zc ph = aa > 0.0 ? zscale(al, 1.0 / aa) : zmake(1.0, 0.0);
    a[e] = zmul(Qm[e], ph);
  }
}

cudaError_t qr_with(afqmc_kp* h, zc* phi, zc* scratch, cudaStream_t st) {
  size_t smem = (size_t)h->N * (2 * sizeof(zc) + sizeof(double));
  qr_kernel<<<2 * h->W, 256, smem, st>>>(phi, scratch, h->NM, h->N);
  AFQMC_LAUNCHED(h);
  return cudaGetLastError();
}

// Same kernel, without a handle: nmat matrices of rows x cols, scratch of the same size.
// Launched through cudaLaunchKernel, whose return value is this launch's own status: an
// earlier, unrelated error stays pending for the code that caused it.
cudaError_t qr_launch(zc* phi, zc* scratch, int rows, int cols, int nmat, cudaStream_t st) {
  size_t smem = (size_t)cols * (2 * sizeof(zc) + sizeof(double));
  void* args[] = {&phi, &scratch, &rows, &cols};
  return cudaLaunchKernel(reinterpret_cast<const void*>(qr_kernel), dim3(nmat), dim3(256), args, smem, st);
}

static cudaError_t qr(afqmc_kp* h, zc* phi, cudaStream_t st) {
  size_t smem = (size_t)h->N * (2 * sizeof(zc) + sizeof(double));
  qr_kernel<<<2 * h->W, 256, smem, st>>>(phi, h->T1, h->NM, h->N);
  AFQMC_LAUNCHED(h);
  return cudaGetLastError();
}

// phi_out[w][s][(k,p)][j] = sum_q Ehalf[k][p][q] phi_in[w][s][(k,q)][j]
static cudaError_t one_body(afqmc_kp* h, const zc* in, zc* out, cudaStream_t st) {
  const int M = h->M, N = h->N, NM = h->NM;
  ZGemm g = gemm_init(M, N, M, 0, 0);
  g.A = h->Ehalf; g.lda = M; g.sA[0] = 0; g.sA[1] = (long)M * M;
  g.B = in; g.ldb = N; g.sB[0] = (long)NM * N; g.sB[1] = (long)M * N;
  g.C = out; g.ldc = N; g.sC[0] = (long)NM * N; g.sC[1] = (long)M * N;
  g.nb[0] = 2 * h->W; g.nb[1] = h->nk;
  return gemm_launch(h, g, st);
}

// The two halves of overlap_lu, for callers that use S before it is factorised.
cudaError_t overlap_only(afqmc_kp* h, const zc* phi, cudaStream_t st) { return overlap(h, phi, st); }
cudaError_t lu_only(afqmc_kp* h, zc* ld, int* sing, int want_inv, cudaStream_t st) {
  lu_kernel<<<2 * h->W, 256, 0, st>>>(h->S, h->Sinv, ld, sing, h->flags, h->N, want_inv,
                                      reinterpret_cast<int*>(h->P));
  AFQMC_LAUNCHED(h);
  return cudaGetLastError();
}

cudaError_t overlap_lu(afqmc_kp* h, const zc* phi, zc* ld, int* sing, int want_inv, cudaStream_t st) {
  cudaError_t e = overlap(h, phi, st);
  if (e != cudaSuccess) return e;
  lu_kernel<<<2 * h->W, 256, 0, st>>>(h->S, h->Sinv, ld, sing, h->flags, h->N, want_inv,
                                      reinterpret_cast<int*>(h->P));
  AFQMC_LAUNCHED(h);
  return cudaGetLastError();
}

static cudaError_t logdet_only(afqmc_kp* h, const zc* phi, zc* ld, int* sing, cudaStream_t st) {
  return overlap_lu(h, phi, ld, sing, 0, st);
}

#define STAGE(stage, body)          \
  do {                              \
    prof_begin(h, stage, st);       \
    cudaError_t e_ = (body);        \
    prof_end(h, st);                \
    if (e_ != cudaSuccess) return e_; \
  } while (0)

static cudaError_t vhs_build(afqmc_kp* h, cudaStream_t st) {
  dim3 grid(h->nk * h->nk, (h->W + VWC - 1) / VWC);
  vhs_kernel<<<grid, 256, sizeof(zc) * VWC * h->G, st>>>(h->L, h->y, h->V, h->kminus, h->nk, h->G, h->M, h->W);
  AFQMC_LAUNCHED(h);
  return cudaGetLastError();
}

// T0 = E phi ; acc = T0 ; T_j = V T_{j-1} / j ; acc += T_j ; phi = E acc
static cudaError_t taylor(afqmc_kp* h, zc* phi, cudaStream_t st) {
  cudaError_t e;
  const int NM = h->NM, N = h->N, W = h->W;
  if ((e = one_body(h, phi, h->T0, st)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(h->acc, h->T0, sizeof(zc) * (size_t)W * 2 * NM * N, cudaMemcpyDeviceToDevice, st)) !=
      cudaSuccess)
    return e;
  zc* cur = h->T0;
  zc* nxt = h->T1;
  for (int j = 1; j <= h->order; ++j) {
    ZGemm g = gemm_init(NM, N, NM, 0, 0);
    g.A = h->V; g.lda = NM; g.sA[0] = (long)NM * NM; g.sA[1] = 0;
    g.B = cur; g.ldb = N; g.sB[0] = 2L * NM * N; g.sB[1] = (long)NM * N;
    g.C = nxt; g.ldc = N; g.sC[0] = 2L * NM * N; g.sC[1] = (long)NM * N;
    g.Acc = h->acc; g.ldacc = N; g.sAcc[0] = 2L * NM * N; g.sAcc[1] = (long)NM * N;
    g.nb[0] = W; g.nb[1] = 2;
    g.alpha = zmake(1.0 / j, 0.0);
    if ((e = gemm_launch(h, g, st)) != cudaSuccess) return e;
    zc* t = cur; cur = nxt; nxt = t;
  }
  return one_body(h, h->acc, phi, st);
}

cudaError_t weights(afqmc_kp* h, const zc* phi, const double* x, double* w, zc* logdet, cudaStream_t st) {
  cudaError_t e;
  if ((e = logdet_only(h, phi, h->ld_new, h->sing_new, st)) != cudaSuccess) return e;
  weight_kernel<<<h->W, 256, 0, st>>>(x, h->xbar, h->ld_old, h->ld_new, h->sing_old, h->sing_new, w, logdet,
                                      2 * h->nk * h->G);
  AFQMC_LAUNCHED(h);
  return cudaGetLastError();
}

// Hybrid weight from the log dets already in ld_old / ld_new.
cudaError_t weight_only(afqmc_kp* h, const double* x, double* w, zc* logdet, cudaStream_t st) {
  weight_kernel<<<h->W, 256, 0, st>>>(x, h->xbar, h->ld_old, h->ld_new, h->sing_old, h->sing_new, w, logdet,
                                      2 * h->nk * h->G);
  AFQMC_LAUNCHED(h);
  return cudaGetLastError();
}

static cudaError_t trace_and_bias(afqmc_kp* h, const double* x, zc* xbar, cudaStream_t st) {
  cudaError_t e = cholesky_trace(h, st);
  if (e != cudaSuccess) return e;
  return force_bias(h, x, xbar, st);
}

cudaError_t propagate(afqmc_kp* h, zc* phi, const double* x, double* w, zc* logdet, int do_qr,
                      cudaStream_t st) {
  cudaError_t e;
  if ((e = green(h, phi, st)) != cudaSuccess) return e;
  STAGE(AFQMC_STAGE_FORCE_BIAS, trace_and_bias(h, x, h->xbar, st));
  STAGE(AFQMC_STAGE_VHS, vhs_build(h, st));
  STAGE(AFQMC_STAGE_TAYLOR, taylor(h, phi, st));
  STAGE(AFQMC_STAGE_WEIGHT, weights(h, phi, x, w, do_qr ? nullptr : logdet, st));
  if (do_qr) return orthonormalise(h, phi, logdet, st);
  return cudaSuccess;
}

static cudaError_t qr_and_logdet(afqmc_kp* h, zc* phi, zc* logdet, cudaStream_t st) {
  cudaError_t e = qr(h, phi, st);
  if (e != cudaSuccess) return e;
  if (logdet) return logdet_only(h, phi, logdet, h->sing_new, st);
  return cudaSuccess;
}

cudaError_t orthonormalise(afqmc_kp* h, zc* phi, zc* logdet, cudaStream_t st) {
  STAGE(AFQMC_STAGE_QR, qr_and_logdet(h, phi, logdet, st));
  return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Local energy
// ---------------------------------------------------------------------------

// E1[w] = sum_s sum_k sum_{a,q} AhH[k][a][q] Gh[w][s][(k,a)][(k,q)];  EC[w] = 1/2 sum X_Q X_-Q
__global__ void e1_ec_kernel(const zc* AhH, const zc* Gh, const zc* X, const int* minus, zc* eloc, int nk,
                             int M, int n, int G) {
  const int w = blockIdx.x;
  const int N = nk * n, NM = nk * M;
  __shared__ zc red[32];
  zc s = zzero();
  for (long e = threadIdx.x; e < 2L * nk * n * M; e += blockDim.x) {
    const int q = (int)(e % M), a = (int)((e / M) % n), k = (int)((e / ((long)M * n)) % nk);
    const int sp = (int)(e / ((long)M * n * nk));
    s = zfma(AhH[((long)k * n + a) * M + q], Gh[((long)(w * 2 + sp) * N + k * n + a) * NM + k * M + q], s);
  }
  const zc e1 = block_zsum(s, red);
  zc c = zzero();
  for (long e = threadIdx.x; e < (long)nk * G; e += blockDim.x) {
    const int g = (int)(e % G), Q = (int)(e / G);
    c = zfma(X[((long)w * nk + Q) * G + g], X[((long)w * nk + minus[Q]) * G + g], c);
  }
  const zc ec = block_zsum(c, red);
  if (threadIdx.x == 0) {
    eloc[3 * w + 0] = e1;
    eloc[3 * w + 1] = zscale(ec, 0.5);
  }
}

// Exchange partial per (w, s, Q, k): sum over k' of the canonical (Q,k,k') terms.
// The term of (Q,k,k') equals that of its partner (-Q, k'-Q, k... ) under the
// involution (Q, k, kx) -> (-Q, kx, k) with kx = k' - Q, so only the
// lexicographically smaller member of each pair is evaluated, with weight 2.
__global__ void __launch_bounds__(256) exchange_fp64_kernel(const zc* LH, const zc* Gh, const int* kminus,
                                                            const int* minus, zc* epart, int nk, int G, int M,
                                                            int n) {
  const int ws = blockIdx.x, Q = blockIdx.y, k = blockIdx.z;
  const int N = nk * n, NM = nk * M, nM = n * M;
  const int mQ = minus[Q], kq = kminus[k * nk + Q];
  extern __shared__ zc sm[];
  zc* g1 = sm;         // Gh[(kx,b)][(k-Q, r)]  n x M
  zc* g2 = sm + nM;    // Gh[(k,a)][(kx+Q, s)]  n x M
  __shared__ zc red[32];
  const zc* Gw = Gh + (long)ws * N * NM;
  zc acc = zzero();
  for (int kx = 0; kx < nk; ++kx) {
    // partner of (Q, k, kx) is (mQ, kx, k)
    const bool self = (mQ == Q) && (kx == k);
    const bool canon = (Q < mQ) || (Q == mQ && k <= kx);
    if (!canon) continue;
    const double wt = self ? 1.0 : 2.0;
    const int kxq = kminus[kx * nk + mQ];  // kx + Q
    __syncthreads();
    for (int e = threadIdx.x; e < nM; e += blockDim.x) {
      const int a = e / M, r = e % M;
      g1[e] = Gw[(long)(kx * n + a) * NM + kq * M + r];
      g2[e] = Gw[(long)(k * n + a) * NM + kxq * M + r];
    }
    __syncthreads();
    const zc* L1 = LH + ((long)Q * nk + k) * G * nM;    // LH[Q][k]
    const zc* L2 = LH + ((long)mQ * nk + kx) * G * nM;  // LH[-Q][kx]
    for (int e = threadIdx.x; e < G * n * n; e += blockDim.x) {
      const int g = e / (n * n), a = (e / n) % n, b = e % n;
      // T1[g,a,b] = sum_r LH[Q,k,g,a,r] Gh[(kx,b),(k-Q,r)]
      // T2[g,b,a] = sum_s LH[-Q,kx,g,b,s] Gh[(k,a),(kx+Q,s)]
      zc t1 = zzero(), t2 = zzero();
      const zc* l1 = L1 + ((long)g * n + a) * M;
      const zc* l2 = L2 + ((long)g * n + b) * M;
      for (int r = 0; r < M; ++r) {
        t1 = zfma(l1[r], g1[b * M + r], t1);
        t2 = zfma(l2[r], g2[a * M + r], t2);
      }
      acc = zadd(acc, zscale(zmul(t1, t2), wt));
    }
  }
  acc = block_zsum(acc, red);
  if (threadIdx.x == 0) epart[((long)ws * nk + Q) * nk + k] = zscale(acc, -0.5);
}

__global__ void ex_reduce_kernel(const zc* epart, zc* eloc, int per_walker) {
  const int w = blockIdx.x;
  __shared__ zc red[32];
  zc s = zzero();
  for (int i = threadIdx.x; i < per_walker; i += blockDim.x) s = zadd(s, epart[(long)w * per_walker + i]);
  s = block_zsum(s, red);
  if (threadIdx.x == 0) eloc[3 * w + 2] = s;
}

static cudaError_t e1_ec(afqmc_kp* h, zc* eloc, cudaStream_t st) {
  e1_ec_kernel<<<h->W, 256, 0, st>>>(h->AhH, h->Gh, h->X, h->minus, eloc, h->nk, h->M, h->n, h->G);
  AFQMC_LAUNCHED(h);
  return cudaGetLastError();
}

static cudaError_t exchange(afqmc_kp* h, cudaStream_t st) {
  dim3 grid(2 * h->W, h->nk, h->nk);
  exchange_fp64_kernel<<<grid, 256, sizeof(zc) * 2 * h->n * h->M, st>>>(h->LH, h->Gh, h->kminus, h->minus,
                                                                        h->epart, h->nk, h->G, h->M, h->n);
  AFQMC_LAUNCHED(h);
  return cudaGetLastError();
}

static cudaError_t ex_reduce(afqmc_kp* h, zc* eloc, cudaStream_t st) {
  ex_reduce_kernel<<<h->W, 256, 0, st>>>(h->epart, eloc, 2 * h->nk * h->nk);
  AFQMC_LAUNCHED(h);
  return cudaGetLastError();
}

cudaError_t local_energy(afqmc_kp* h, const zc* phi, zc* eloc, cudaStream_t st) {
  cudaError_t e;
  if ((e = green(h, phi, st)) != cudaSuccess) return e;
  STAGE(AFQMC_STAGE_FORCE_BIAS, cholesky_trace(h, st));
  STAGE(AFQMC_STAGE_ENERGY, e1_ec(h, eloc, st));
  STAGE(AFQMC_STAGE_EXCHANGE, exchange(h, st));
  STAGE(AFQMC_STAGE_ENERGY, ex_reduce(h, eloc, st));
  return cudaSuccess;
}

// One fused walker step: propagate every walker and evaluate the local energy of
// the propagated walkers.  The Green's function of the new walkers serves the
// new log det (weights), the energy, and the next step's force bias.
cudaError_t step(afqmc_kp* h, zc* phi, const double* x, double* w, zc* eloc, zc* logdet, int do_qr, int reuse,
                 cudaStream_t st) {
  cudaError_t e;
  if (!reuse) {
    STAGE(AFQMC_STAGE_GREEN, green_impl(h, phi, h->ld_old, h->sing_old, st));
    STAGE(AFQMC_STAGE_FORCE_BIAS, cholesky_trace(h, st));
  }
  STAGE(AFQMC_STAGE_FORCE_BIAS, force_bias(h, x, h->xbar, st));
  STAGE(AFQMC_STAGE_VHS, vhs_build(h, st));
  STAGE(AFQMC_STAGE_TAYLOR, taylor(h, phi, st));
  STAGE(AFQMC_STAGE_GREEN, green_impl(h, phi, h->ld_new, h->sing_new, st));
  STAGE(AFQMC_STAGE_FORCE_BIAS, cholesky_trace(h, st));
  STAGE(AFQMC_STAGE_WEIGHT, weight_only(h, x, w, do_qr ? nullptr : logdet, st));
  if (eloc) {   // NULL: a propagation-only step of a block (the energy is measured less often)
    STAGE(AFQMC_STAGE_ENERGY, e1_ec(h, eloc, st));
    STAGE(AFQMC_STAGE_EXCHANGE, exchange(h, st));
    STAGE(AFQMC_STAGE_ENERGY, ex_reduce(h, eloc, st));
  }
  if (do_qr) {
    // the Green's function is invariant under phi -> phi R^-1; only the log det moves
    STAGE(AFQMC_STAGE_QR, qr(h, phi, st));
    STAGE(AFQMC_STAGE_QR, overlap_lu(h, phi, h->ld_new, h->sing_new, 0, st));
    if (logdet &&
        (e = cudaMemcpyAsync(logdet, h->ld_new, sizeof(zc) * 2 * h->W, cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
      return e;
  }
  std::swap(h->ld_old, h->ld_new);
  std::swap(h->sing_old, h->sing_new);
  return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Adjoint of the local energy
// ---------------------------------------------------------------------------

// Gam[w][s][(k,a)][(k-Q,r)] = c2 sum_g X[w][-Q][g] LH[Q][k][g][a][r] + (Q == 0 ? c1 AhH[k][a][r] : 0)
// with c = conj(grad_e).  Every (k, k') block is written exactly once.
__global__ void gamma_init_kernel(const zc* LH, const zc* X, const zc* AhH, const zc* grad_e, zc* Gam,
                                  const int* kminus, const int* minus, int nk, int G, int M, int n) {
  const int ws = blockIdx.x, k = blockIdx.y, Q = blockIdx.z;
  const int w = ws >> 1;
  const int N = nk * n, NM = nk * M, nM = n * M;
  const int kq = kminus[k * nk + Q], mQ = minus[Q];
  const zc c1 = zconj(grad_e[3 * w + 0]), c2 = zconj(grad_e[3 * w + 1]);
  const zc* xm = X + ((long)w * nk + mQ) * G;
  const zc* lh = LH + ((long)Q * nk + k) * G * nM;
  for (int e = threadIdx.x; e < nM; e += blockDim.x) {
    zc s = zzero();
    for (int g = 0; g < G; ++g) s = zfma(xm[g], lh[(long)g * nM + e], s);
    s = zmul(c2, s);
    if (Q == 0) s = zfma(c1, AhH[(long)k * nM + e], s);
    const int a = e / M, r = e % M;
    Gam[((long)ws * N + k * n + a) * NM + kq * M + r] = s;
  }
}

// Gam[(kx,b)][(c,r)] += -c3 sum_Q sum_{g,a} T2[g,b,a] LH[Q][c+Q][g][a][r],
// T2[g,b,a] = sum_s LH[-Q][kx][g][b][s] Gh[(c+Q,a)][(kx+Q,s)].  Block (w s, kx, c).
__global__ void __launch_bounds__(256) gamma_exchange_kernel(const zc* LH, const zc* Gh, const zc* grad_e,
                                                             zc* Gam, const int* kminus, const int* minus,
                                                             int nk, int G, int M, int n) {
  const int ws = blockIdx.x, kx = blockIdx.y, c = blockIdx.z;
  const int w = ws >> 1;
  const int N = nk * n, NM = nk * M, nM = n * M;
  const zc c3 = zconj(grad_e[3 * w + 2]);
  extern __shared__ zc sm[];
  zc* gblk = sm;            // n x M : Gh[(k,a)][(kx+Q, s)]
  zc* T2 = sm + nM;         // G x n x n
  const zc* Gw = Gh + (long)ws * N * NM;
  // each thread owns outputs e = (b, r) over n*M entries
  zc outv[4];
  const int per = (nM + blockDim.x - 1) / blockDim.x;
  for (int i = 0; i < 4; ++i) outv[i] = zzero();
  for (int Q = 0; Q < nk; ++Q) {
    const int mQ = minus[Q];
    const int k = kminus[c * nk + mQ];      // k = c + Q
    const int kxq = kminus[kx * nk + mQ];   // kx + Q
    __syncthreads();
    for (int e = threadIdx.x; e < nM; e += blockDim.x) {
      const int a = e / M, s = e % M;
      gblk[e] = Gw[(long)(k * n + a) * NM + kxq * M + s];
    }
    __syncthreads();
    const zc* L2 = LH + ((long)mQ * nk + kx) * G * nM;
    for (int e = threadIdx.x; e < G * n * n; e += blockDim.x) {
      const int g = e / (n * n), b = (e / n) % n, a = e % n;
      zc t = zzero();
      const zc* l2 = L2 + ((long)g * n + b) * M;
      for (int s = 0; s < M; ++s) t = zfma(l2[s], gblk[a * M + s], t);
      T2[e] = t;
    }
    __syncthreads();
    const zc* L1 = LH + ((long)Q * nk + k) * G * nM;
    for (int i = 0; i < per && i < 4; ++i) {
      const int e = threadIdx.x + i * blockDim.x;
      if (e >= nM) break;
      const int b = e / M, r = e % M;
      zc s = outv[i];
      for (int g = 0; g < G; ++g)
        for (int a = 0; a < n; ++a) s = zfma(T2[((long)g * n + b) * n + a], L1[((long)g * n + a) * M + r], s);
      outv[i] = s;
    }
  }
  for (int i = 0; i < per && i < 4; ++i) {
    const int e = threadIdx.x + i * blockDim.x;
    if (e >= nM) break;
    const int b = e / M, r = e % M;
    zc* o = Gam + ((long)ws * N + kx * n + b) * NM + c * M + r;
    *o = zsub(*o, zmul(c3, outv[i]));
  }
}

// grad_h1[k][p][q] = sum_w g1[w] sum_s sum_a A[k][p][a] conj(Gh[w][s][(k,a)][(k,q)])
__global__ void grad_h1_kernel(const zc* A, const zc* Gh, const zc* grad_e, zc* gh1, int nk, int M, int n,
                               int W) {
  const int k = blockIdx.x;
  const int N = nk * n, NM = nk * M;
  for (int e = threadIdx.x; e < M * M; e += blockDim.x) {
    const int p = e / M, q = e % M;
    zc s = zzero();
    for (int w = 0; w < W; ++w) {
      zc t = zzero();
      for (int sp = 0; sp < 2; ++sp)
        for (int a = 0; a < n; ++a)
          t = zfma(A[((long)k * M + p) * n + a], zconj(Gh[((long)(w * 2 + sp) * N + k * n + a) * NM + k * M + q]), t);
      s = zfma(grad_e[3 * w + 0], t, s);
    }
    gh1[(long)k * M * M + e] = s;
  }
}

cudaError_t grad_h1(afqmc_kp* h, const zc* grad_e, zc* gh1, cudaStream_t st) {
  grad_h1_kernel<<<h->nk, 256, 0, st>>>(h->A, h->Gh, grad_e, gh1, h->nk, h->M, h->n, h->W);
  AFQMC_LAUNCHED(h);
  return cudaGetLastError();
}

// dE/dphi from Gam = conj(grad_e)-weighted dE/dGh: with Gh = S^-T phi^T and S = A^dag phi,
// dGh = S^-T dphi^T (I - A* Gh), so grad_phi = [S^-1 (Gam - (Gam Gh^T) A^dag)]^H in the
// conjugate convention of the binding.
cudaError_t project_gamma(afqmc_kp* h, zc* grad_phi, cudaStream_t st, bool ff) {
  cudaError_t e;
  auto launch = [&](const ZGemm& g) { return ff ? gemm_launch_ff(h, g, st) : gemm_launch(h, g, st); };
  const int nk = h->nk, M = h->M, n = h->n, N = h->N, NM = h->NM, W = h->W;
  {  // P = Gam Gh^T  (N x N)
    ZGemm g = gemm_init(N, N, NM, 0, 1);
    g.A = h->Gam; g.lda = NM; g.sA[0] = (long)N * NM;
    g.B = h->Gh; g.ldb = NM; g.sB[0] = (long)N * NM;
    g.C = h->P; g.ldc = N; g.sC[0] = (long)N * N;
    g.nb[0] = 2 * W;
    if ((e = launch(g)) != cudaSuccess) return e;
  }
  {  // Gam[:, k-block] -= P[:, k-block of n] A[k]^dagger
    ZGemm g = gemm_init(N, M, n, 0, 2);
    g.A = h->P; g.lda = N; g.sA[0] = (long)N * N; g.sA[1] = n;
    g.B = h->A; g.ldb = n; g.sB[0] = 0; g.sB[1] = (long)M * n;
    g.C = h->Gam; g.ldc = NM; g.sC[0] = (long)N * NM; g.sC[1] = M;
    g.nb[0] = 2 * W; g.nb[1] = nk;
    g.alpha = zmake(-1.0, 0.0);
    g.beta = zmake(1.0, 0.0);
    if ((e = launch(g)) != cudaSuccess) return e;
  }
  {  // grad_phi = Gam^H Sinv^H  (NM x N)
    ZGemm g = gemm_init(NM, N, N, 2, 2);
    g.A = h->Gam; g.lda = NM; g.sA[0] = (long)N * NM;
    g.B = h->Sinv; g.ldb = N; g.sB[0] = (long)N * N;
    g.C = grad_phi; g.ldc = N; g.sC[0] = (long)NM * N;
    g.nb[0] = 2 * W;
    if ((e = launch(g)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

static cudaError_t backward_impl(afqmc_kp* h, const zc* grad_e, zc* grad_phi, zc* gh1, cudaStream_t st) {
  cudaError_t e;
  const int nk = h->nk, M = h->M, n = h->n, W = h->W;
  if (gh1 && (e = grad_h1(h, grad_e, gh1, st)) != cudaSuccess) return e;
  if (!grad_phi) return cudaSuccess;
  if ((e = cholesky_trace(h, st)) != cudaSuccess) return e;
  gamma_init_kernel<<<dim3(2 * W, nk, nk), 128, 0, st>>>(h->LH, h->X, h->AhH, grad_e, h->Gam, h->kminus, h->minus,
                                                          nk, h->G, M, n);
  AFQMC_LAUNCHED(h);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  gamma_exchange_kernel<<<dim3(2 * W, nk, nk), 256, sizeof(zc) * (n * M + h->G * n * n), st>>>(
      h->LH, h->Gh, grad_e, h->Gam, h->kminus, h->minus, nk, h->G, M, n);
  AFQMC_LAUNCHED(h);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return project_gamma(h, grad_phi, st, false);
}

cudaError_t local_energy_backward(afqmc_kp* h, const zc* phi, const zc* grad_e, zc* grad_phi, zc* grad_h1,
                                  cudaStream_t st) {
  cudaError_t e;
  if ((e = green(h, phi, st)) != cudaSuccess) return e;
  STAGE(AFQMC_STAGE_BACKWARD, backward_impl(h, grad_e, grad_phi, grad_h1, st));
  return cudaSuccess;
}

static cudaError_t set_smem(const void* fn, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  if (bytes > 227 * 1024) return cudaErrorNotSupported;   // larger than one CTA may hold
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Opt in to the dynamic shared memory each kernel needs at this system size.  A tensor-core
// (mixed) handle runs none of these kernels (its own take their place), so it needs none.
static cudaError_t configure_smem(afqmc_kp* h) {
  if (h->d.prec == AFQMC_MIXED) return cudaSuccess;
  cudaError_t e = set_smem((const void*)vhs_kernel, sizeof(zc) * VWC * h->G);
  if (e == cudaSuccess)
    e = set_smem((const void*)gamma_exchange_kernel, sizeof(zc) * (h->n * h->M + (size_t)h->G * h->n * h->n));
  if (e == cudaSuccess) e = set_smem((const void*)xtrace_kernel, sizeof(zc) * XWC * h->n * h->M);
  if (e == cudaSuccess) e = set_smem((const void*)qr_kernel, (size_t)h->N * (2 * sizeof(zc) + sizeof(double)));
  if (e == cudaSuccess) e = set_smem((const void*)exchange_fp64_kernel, sizeof(zc) * 2 * h->n * h->M);
  return e;
}

}  // namespace fp64
