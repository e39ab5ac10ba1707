// Double-float dense kernels of the tensor-core path (ff.cuh): the overlap matrix,
// the trial-subspace projection of the walker, and the inverse / log-determinant
// of the overlap matrix.
//
// These are the steps of Sec. 3.2 (step 1, the Green's function of Eq. kp_gf) whose
// results need more than the 22 bits of the split GEMM: S = A^dag phi enters the
// log-determinant (the weight, Eq. hybrid) and its inverse; phi_perp = phi - B S is a
// cancelling difference.  FP64 would serve, but this GPU's FP64 pipe is two fused
// multiply-adds per clock per SM; double-float arithmetic on the FP32 pipe keeps 48
// bits at several times the speed.
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>

#include "attr.hpp"
#include "ff.cuh"
#include "ffla.hpp"
#include "split.cuh"

namespace ffla {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int OV_THREADS = 256;
constexpr int GJ_THREADS = 512;
constexpr int GJ_WARPS = GJ_THREADS / 32;
constexpr size_t OV_SMEM_TARGET = 96 * 1024;
constexpr size_t SMEM_LIMIT = 220 * 1024;
// largest N held in shared memory (N^2 float4 + per-row arrays within SMEM_LIMIT; < 128,
// which the register-held pivot row of the shared-memory variant relies on)
constexpr int GJ_SMEM_MAXN = 118;

__device__ __forceinline__ float block_max_f(float v, float* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(FULL, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  float m = 0.f;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) m = fmaxf(m, red[i]);
  return m;
}
__device__ __forceinline__ double block_sum_d(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
  return s;
}

// S[ws][(k,a)][j] = sum_p conj(A[k][p][a]) phi[ws][(k,p)][j]                       (Eq. kp_gf)
// PROJECT: phi_perp[ws][(k,p)][j] = phi[ws][(k,p)][j] - sum_a B[k][p][a] S[ws][(k,a)][j]
// (rounded to fp32) and mx[ws] = max |phi_perp| (atomic max on the bits of a
// non-negative double).  Grid (WS, nk, column chunks of JC).
template <bool PROJECT>
__global__ void __launch_bounds__(OV_THREADS)
    overlap_ff_kernel(const zc* A, const zc* phi, const zc* B, float4* Sff, float2* phi_perp,
                      unsigned long long* mx, int nk, int M, int n, int N, int JC) {
  extern __shared__ __align__(16) unsigned char ov_smem[];
  __shared__ float red[OV_THREADS / 32];
  const int ws = blockIdx.x, k = blockIdx.y, j0 = blockIdx.z * JC, tid = threadIdx.x;
  const int jc = min(JC, N - j0);
  float4* ph = reinterpret_cast<float4*>(ov_smem);   // [M][JC]
  float4* Ak = ph + (size_t)M * JC;                    // [M][n]
  float4* Bk = Ak + (size_t)M * n;                     // [M][n]
  float4* Sk = Bk + (size_t)M * n;                     // [n][JC]
  const size_t row0 = (size_t)ws * nk * M + (size_t)k * M;   // first row (k, 0) of this walker-spin
  for (int e = tid; e < M * jc; e += OV_THREADS) {
    const int p = e / jc, jj = e % jc;
    ph[p * JC + jj] = ffa::cfrom(phi[(row0 + p) * N + j0 + jj]);
  }
  for (int e = tid; e < M * n; e += OV_THREADS) {
    Ak[e] = ffa::cfrom(A[(size_t)k * M * n + e]);
    if (PROJECT) Bk[e] = ffa::cfrom(B[(size_t)k * M * n + e]);
  }
  __syncthreads();
  for (int e = tid; e < n * jc; e += OV_THREADS) {
    const int a = e / jc, jj = e % jc;
    ffa::cacc acc = ffa::cacc_from(ffa::czero());
    for (int p = 0; p < M; ++p) ffa::cacc_fma_conj(acc, Ak[p * n + a], ph[p * JC + jj]);
    const float4 v = ffa::cacc_get(acc);
    Sk[a * JC + jj] = v;
    Sff[((size_t)ws * N + (size_t)k * n + a) * N + j0 + jj] = v;
  }
  if (!PROJECT) return;
  __syncthreads();
  float m = 0.f;
  for (int e = tid; e < M * jc; e += OV_THREADS) {
    const int p = e / jc, jj = e % jc;
    ffa::cacc pa = ffa::cacc_from(ph[p * JC + jj]);
    for (int a = 0; a < n; ++a) ffa::cacc_fms(pa, Bk[p * n + a], Sk[a * JC + jj]);
    const float4 v = ffa::cacc_get(pa);
    const float2 o = make_float2(__fadd_rn(v.x, v.y), __fadd_rn(v.z, v.w));
    phi_perp[(row0 + p) * N + j0 + jj] = o;
    m = fmaxf(m, fmaxf(fabsf(o.x), fabsf(o.y)));
  }
  m = block_max_f(m, red);
  if (tid == 0) atomicMax(mx + ws, static_cast<unsigned long long>(__double_as_longlong((double)m)));
}

// Gauss-Jordan elimination with partial (row) pivoting of one N x N matrix per CTA, in
// place, in double-float.  Step j: pick the row p >= j with the largest |re| + |im| in
// column j, swap rows j and p, then
//   INV:  scale row j by 1/a_jj (a_jj itself becomes 1/a_jj) and eliminate column j
//         from every other row (a_ij becomes -a_ij / a_jj): after N steps the array
//         holds (P S)^-1, P the row permutation, so S^-1[:, perm[i]] = column i;
//   !INV: eliminate below the diagonal only (LU), for the log-determinant alone.
// Either way the pivots are the diagonal of U in P S = L U, so
//   log det S = sum_j log a_jj + i pi (number of swaps mod 2).
// A zero or non-finite pivot marks the matrix singular: logdet = (-inf, 0), sing = 1,
// flags[0] counts it, and the inverse written is zero.
// INV output: the split planes of S^-T, out[b][4][N][Np] with scale s_out[b].
template <bool SMEM, bool INV>
__global__ void __launch_bounds__(GJ_THREADS)
    gj_ff_kernel(float4* Sff, int N, zc* logdet, int* sing, int* flags, __half* out, int Np, float* s_out) {
  extern __shared__ __align__(16) unsigned char gj_smem[];
  __shared__ int s_p, s_sing, s_swaps;
  __shared__ float4 s_pv, s_ajj;
  __shared__ double s_red[GJ_WARPS];
  __shared__ float s_redf[GJ_WARPS];
  const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float4* g = Sff + (size_t)b * N * N;
  float4* a = SMEM ? reinterpret_cast<float4*>(gj_smem) : g;
  float4* f = reinterpret_cast<float4*>(gj_smem + (SMEM ? (size_t)N * N * sizeof(float4) : 0));
  double2* piv = reinterpret_cast<double2*>(f + N);
  int* perm = reinterpret_cast<int*>(piv + N);
  int* iperm = perm + N;
  if (SMEM)
    for (int e = tid; e < N * N; e += GJ_THREADS) a[e] = g[e];
  for (int i = tid; i < N; i += GJ_THREADS) perm[i] = i;
  if (tid == 0) {
    s_sing = 0;
    s_swaps = 0;
  }
  __syncthreads();
  for (int j = 0; j < N; ++j) {
    if (warp == 0) {
      float best = -1.f;
      int bi = j;
      for (int i = j + lane; i < N; i += 32) {
        const float4 v = a[(size_t)i * N + j];
        const float m = fabsf(v.x) + fabsf(v.z);
        if (m > best) {
          best = m;
          bi = i;
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const float b2 = __shfl_xor_sync(FULL, best, o);
        const int i2 = __shfl_xor_sync(FULL, bi, o);
        if (b2 > best || (b2 == best && i2 < bi)) {
          best = b2;
          bi = i2;
        }
      }
      if (lane == 0) {
        s_p = bi;
        s_pv = a[(size_t)bi * N + j];
        s_ajj = a[(size_t)j * N + j];
        if (!(best > 0.f) || !isfinite(best)) {
          s_sing = 1;
        } else if (bi != j) {
          const int t = perm[j];
          perm[j] = perm[bi];
          perm[bi] = t;
          ++s_swaps;
        }
      }
    }
    __syncthreads();
    if (s_sing) break;   // the same shared value for every thread after the barrier
    const int p = s_p;
    const float4 pv = s_pv, ajj = s_ajj;
    const float4 inv = ffa::crecip(pv);
    if (tid == 0) piv[j] = make_double2(ffa::to_double(ffa::re(pv)), ffa::to_double(ffa::im(pv)));
    // swap rows j and p (each thread owns whole columns), and, INV, scale row j
    for (int c = tid; c < N; c += GJ_THREADS) {
      const float4 tj = a[(size_t)j * N + c];
      const float4 tp = (p == j) ? tj : a[(size_t)p * N + c];
      if (INV) {
        if (c == j)
          a[(size_t)j * N + c] = inv;
        else
          a[(size_t)j * N + c] = ffa::cmul(tp, inv);
      } else {
        a[(size_t)j * N + c] = tp;
      }
      if (p != j) a[(size_t)p * N + c] = tj;
    }
    // multipliers: column j after the swap (rows j and p are the only ones moved)
    for (int i = tid; i < N; i += GJ_THREADS) {
      float4 fi;
      if (i == j)
        fi = ffa::czero();
      else
        fi = (i == p) ? ajj : a[(size_t)i * N + j];
      if (!INV) fi = ffa::cmul(fi, inv);
      f[i] = fi;
    }
    __syncthreads();
    const float4* aj = a + (size_t)j * N;
    if (SMEM) {
      // N <= GJ_SMEM_MAXN < 128: each lane owns the columns lane + 32 h, h < 4, and keeps
      // its part of row j in registers for all the rows it updates
      float4 ajr[4];
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const int c = lane + 32 * h;
        ajr[h] = (c < N) ? aj[c] : ffa::czero();
      }
      const int i0 = INV ? warp : j + 1 + warp;
      for (int i = i0; i < N; i += GJ_WARPS) {
        if (INV && i == j) continue;
        const float4 fi = f[i];
        float4* ai = a + (size_t)i * N;
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          const int c = lane + 32 * h;
          if (c >= N || (!INV && c <= j)) continue;
          if (INV && c == j)
            ai[c] = ffa::cneg(ffa::cmul(fi, inv));
          else
            ai[c] = ffa::cfms(ai[c], fi, ajr[h]);
        }
      }
    } else if (INV) {
      for (int i = warp; i < N; i += GJ_WARPS) {
        if (i == j) continue;
        const float4 fi = f[i];
        float4* ai = a + (size_t)i * N;
        for (int c = lane; c < N; c += 32) {
          if (c == j)
            ai[c] = ffa::cneg(ffa::cmul(fi, inv));
          else
            ai[c] = ffa::cfms(ai[c], fi, aj[c]);
        }
      }
    } else {
      for (int i = j + 1 + warp; i < N; i += GJ_WARPS) {
        const float4 fi = f[i];
        float4* ai = a + (size_t)i * N;
        for (int c = j + 1 + lane; c < N; c += 32) ai[c] = ffa::cfms(ai[c], fi, aj[c]);
      }
    }
    __syncthreads();
  }
  const int singular = s_sing;
  double lg = 0.0, an = 0.0;
  if (!singular)
    for (int i = tid; i < N; i += GJ_THREADS) {
      const double2 v = piv[i];
      lg += 0.5 * log(v.x * v.x + v.y * v.y);
      an += atan2(v.y, v.x);
    }
  lg = block_sum_d(lg, s_red);
  an = block_sum_d(an, s_red);
  if (tid == 0) {
    if (singular) {
      logdet[b] = make_double2(-INFINITY, 0.0);
      sing[b] = 1;
      atomicAdd(&flags[0], 1);
    } else {
      double ang = an + ((s_swaps & 1) ? M_PI : 0.0);
      ang = remainder(ang, 2.0 * M_PI);
      logdet[b] = make_double2(lg, ang);
      sing[b] = 0;
    }
  }
  if (!INV) return;
  const size_t ps = (size_t)N * Np;
  __half* o = out + (size_t)b * 4 * ps;
  if (singular) {
    for (int e = tid; e < N * N; e += GJ_THREADS) mixed::put4f(o, ps, (size_t)(e / N) * Np + e % N, 0.f, 0.f);
    if (tid == 0) s_out[b] = 1.f;
    return;
  }
  for (int c = tid; c < N; c += GJ_THREADS) iperm[perm[c]] = c;
  float m = 0.f;
  for (int e = tid; e < N * N; e += GJ_THREADS) {
    const float4 v = a[e];
    m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.z)));
  }
  m = block_max_f(m, s_redf);   // its barriers also publish iperm
  const float s = mixed::pow2_scale((double)m);
  if (tid == 0) s_out[b] = s;
  // out row i, column c = S^-T[i][c] = S^-1[c][i] = a[c][iperm[i]]
  for (int e = tid; e < N * N; e += GJ_THREADS) {
    const int i = e / N, c = e % N;
    const float4 v = a[(size_t)c * N + iperm[i]];
    mixed::put4f(o, ps, (size_t)i * Np + c, v.x * s, v.z * s);
  }
}

// Blocked form of the same Gauss-Jordan inverse, matrix in shared memory.  Pivots are taken
// in panels of GJB columns: within a panel every step updates only the panel's columns
// (all rows), so that afterwards those columns hold the panel's accumulated transform T
// (T - I has non-zeros only there); every other column c then receives the panel's row
// swaps and one rank-GJB update c <- T c = c + (T - I)[:, panel] c[panel rows].  The
// arithmetic per element is unchanged (N^3 double-float multiply-adds in all); the
// rank-GJB update reads and writes each element once per panel instead of once per pivot,
// with the panel's multipliers and rows reused from registers.
// The matrix lives in shared memory when it fits (SMEM, N <= GJB_MAXN), else in place in
// global memory (the overlap buffer, L2-resident while the CTA works on it): each panel then
// reads and writes the matrix once, where the unblocked kernel does so once per pivot.
constexpr int GJB = 8;
static_assert(GJB == 8, "the panel's index arithmetic uses shifts by 3");
constexpr int GJB_THREADS = 512;
constexpr int GJB_WARPS = GJB_THREADS / 32;
constexpr int GJB_MAXN = 112;   // N^2 + GJB N float4 + per-row arrays within SMEM_LIMIT
constexpr int GJB_GLOBAL_MAXN = 1024;   // GJB N float4 + per-row arrays within SMEM_LIMIT

// Pivot candidate key: larger |value| first, then the smaller row (m >= 0 and not NaN, so its
// bits order as the values do).
__device__ __forceinline__ unsigned long long pivot_key(float m, int i) {
  return ((unsigned long long)__float_as_uint(m) << 32) | (unsigned long long)(0xffffffffu - (unsigned)i);
}

template <bool SMEM>
__global__ void __launch_bounds__(GJB_THREADS)
    gjb_ff_kernel(float4* Sff, int N, zc* logdet, int* sing, int* flags, __half* out, int Np, float* s_out) {
  extern __shared__ __align__(16) unsigned char gj_smem[];
  __shared__ int s_swaps;
  __shared__ unsigned long long s_key[2];   // the next pivot's (|value|, row) key, two in turn
  __shared__ double s_red[GJB_WARPS];
  __shared__ float s_redf[GJB_WARPS];
  __shared__ int s_prow[GJB];
  const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float4* g = Sff + (size_t)b * N * N;
  float4* a = SMEM ? reinterpret_cast<float4*>(gj_smem) : g;   // [N][N]
  float4* tmp = reinterpret_cast<float4*>(gj_smem) + (SMEM ? (size_t)N * N : 0);   // [GJB][N] panel rows
  float4* f = tmp + (size_t)GJB * N;                      // [N] multipliers
  double2* piv = reinterpret_cast<double2*>(f + N);
  int* perm = reinterpret_cast<int*>(piv + N);
  int* iperm = perm + N;
  if (SMEM)
    for (int e = tid; e < N * N; e += GJB_THREADS) a[e] = g[e];
  for (int i = tid; i < N; i += GJB_THREADS) perm[i] = i;
  if (tid == 0) s_swaps = 0;
  __syncthreads();
  // Every thread reads the same shared pivot keys after the same barriers, so it takes the
  // singular exit at the same step as the others.
  bool singular_l = false;
  for (int j0 = 0; j0 < N && !singular_l; j0 += GJB) {
    const int jb = min(GJB, N - j0);
    // ---- panel: columns [j0, j0 + jb), every row
    // The pivot of column j is the row i >= j of largest |re.hi| + |im.hi| (the smallest i
    // among equals).  The panel's first column was last written by the rank update and is
    // searched by warp 0; every later column j + 1 is searched while the elimination of
    // column j writes it (a warp maximum of the (|value|, row) keys, then one shared atomic
    // maximum per warp), which saves the search's serial pass and a barrier per pivot.
    for (int jj = 0; jj < jb; ++jj) {
      const int j = j0 + jj;
      if (jj == 0) {
        if (warp == 0) {
          float best = -1.f;
          int bi = j;
          for (int i = j + lane; i < N; i += 32) {
            const float4 v = a[(size_t)i * N + j];
            const float m = fabsf(v.x) + fabsf(v.z);
            if (m > best) {
              best = m;
              bi = i;
            }
          }
          for (int o = 16; o > 0; o >>= 1) {
            const float b2 = __shfl_xor_sync(FULL, best, o);
            const int i2 = __shfl_xor_sync(FULL, bi, o);
            if (b2 > best || (b2 == best && i2 < bi)) {
              best = b2;
              bi = i2;
            }
          }
          if (lane == 0) s_key[0] = best >= 0.f ? pivot_key(best, bi) : 0ull;
        }
        __syncthreads();
      }
      const unsigned long long key = s_key[jj & 1];
      const float best = __uint_as_float((unsigned)(key >> 32));
      if (!(best > 0.f) || !isfinite(best)) {
        singular_l = true;
        break;
      }
      const int p = (int)(0xffffffffu - (unsigned)(key & 0xffffffffull));
      const float4 pv = a[(size_t)p * N + j], ajj = a[(size_t)j * N + j];
      const float4 inv = ffa::crecip(pv);
      if (tid == 0) {
        s_prow[jj] = p;
        if (p != j) {
          const int t = perm[j];
          perm[j] = perm[p];
          perm[p] = t;
          ++s_swaps;
        }
        piv[j] = make_double2(ffa::to_double(ffa::re(pv)), ffa::to_double(ffa::im(pv)));
        s_key[(jj + 1) & 1] = 0ull;   // read last before the previous step's barriers
      }
      // swap rows j and p and scale row j, panel columns other than j (the elimination below
      // writes column j whole: inv in row j, -f inv elsewhere)
      for (int cc = tid; cc < jb; cc += GJB_THREADS) {
        const int c = j0 + cc;
        if (c == j) continue;
        const float4 tj = a[(size_t)j * N + c];
        const float4 tp = (p == j) ? tj : a[(size_t)p * N + c];
        a[(size_t)j * N + c] = ffa::cmul(tp, inv);
        if (p != j) a[(size_t)p * N + c] = tj;
      }
      for (int i = tid; i < N; i += GJB_THREADS) {
        if (i == j)
          f[i] = ffa::czero();
        else
          f[i] = (i == p) ? ajj : a[(size_t)i * N + j];
      }
      __syncthreads();
      // eliminate column j from every other row, panel columns only: one thread per
      // (row, panel column)
      unsigned long long cand = 0ull;
      for (int e = tid; e < N * jb; e += GJB_THREADS) {
        const int i = (jb == GJB) ? (e >> 3) : e / jb, c = j0 + ((jb == GJB) ? (e & 7) : e % jb);
        if (c == j) {
          a[(size_t)i * N + c] = (i == j) ? inv : ffa::cneg(ffa::cmul(f[i], inv));
          continue;
        }
        if (i == j) continue;
        const float4 v = ffa::cfms(a[(size_t)i * N + c], f[i], a[(size_t)j * N + c]);
        a[(size_t)i * N + c] = v;
        if (c == j + 1 && i > j) {
          const float m = fabsf(v.x) + fabsf(v.z);
          if (!isnan(m)) cand = max(cand, pivot_key(m, i));
        }
      }
      if (jj + 1 < jb) {
        for (int o = 16; o > 0; o >>= 1) {
          const unsigned long long other = __shfl_xor_sync(FULL, cand, o);
          cand = other > cand ? other : cand;
        }
        if (lane == 0 && cand) atomicMax(&s_key[(jj + 1) & 1], cand);
      }
      __syncthreads();
    }
    if (singular_l) break;
    // ---- every other column: the panel's row swaps in order, a copy of the panel rows
    const int R = N - jb;   // rest column r -> c = r < j0 ? r : r + jb
    for (int r = tid; r < R; r += GJB_THREADS) {
      const int c = (r < j0) ? r : r + jb;
      for (int jj = 0; jj < jb; ++jj) {
        const int j = j0 + jj, p = s_prow[jj];
        if (p != j) {
          const float4 t = a[(size_t)j * N + c];
          a[(size_t)j * N + c] = a[(size_t)p * N + c];
          a[(size_t)p * N + c] = t;
        }
      }
      for (int jj = 0; jj < jb; ++jj) tmp[(size_t)jj * N + r] = a[(size_t)(j0 + jj) * N + c];
    }
    __syncthreads();
    // ---- rank-jb update a[i][c] += sum_l (T - I)[i][j0 + l] tmp[l][c]: a thread takes one
    // row and two rest columns r and r + H (H = ceil(R / 2)), consecutive threads consecutive
    // r, so a warp reads tmp in one conflict-free run and (mostly) one row's multipliers;
    // N H tasks spread evenly over the threads
    {
      const int H = (R + 1) / 2;
      for (int u = tid; u < N * H; u += GJB_THREADS) {
        const int i = u / H, rA = u % H, rB = rA + H;
        const bool okB = rB < R;
        const int cA = (rA < j0) ? rA : rA + jb, cB = (rB < j0) ? rB : rB + jb;
        ffa::cacc xA = ffa::cacc_from(a[(size_t)i * N + cA]);
        ffa::cacc xB = ffa::cacc_from(okB ? a[(size_t)i * N + cB] : ffa::czero());
        for (int l = 0; l < jb; ++l) {
          float4 d = a[(size_t)i * N + j0 + l];
          if (i == j0 + l) d = ffa::pack(ffa::add(ffa::re(d), ffa::make(-1.f, 0.f)), ffa::im(d));
          const float4 tA = tmp[(size_t)l * N + rA];
          const float4 tB = okB ? tmp[(size_t)l * N + rB] : ffa::czero();
          ffa::cacc_fma(xA, d, tA);
          ffa::cacc_fma(xB, d, tB);
        }
        a[(size_t)i * N + cA] = ffa::cacc_get(xA);
        if (okB) a[(size_t)i * N + cB] = ffa::cacc_get(xB);
      }
    }
    __syncthreads();
  }
  const int singular = singular_l;
  double lg = 0.0, an = 0.0;
  if (!singular)
    for (int i = tid; i < N; i += GJB_THREADS) {
      const double2 v = piv[i];
      lg += 0.5 * log(v.x * v.x + v.y * v.y);
      an += atan2(v.y, v.x);
    }
  lg = block_sum_d(lg, s_red);
  an = block_sum_d(an, s_red);
  if (tid == 0) {
    if (singular) {
      logdet[b] = make_double2(-INFINITY, 0.0);
      sing[b] = 1;
      atomicAdd(&flags[0], 1);
    } else {
      double ang = an + ((s_swaps & 1) ? M_PI : 0.0);
      ang = remainder(ang, 2.0 * M_PI);
      logdet[b] = make_double2(lg, ang);
      sing[b] = 0;
    }
  }
  const size_t ps = (size_t)N * Np;
  __half* o = out + (size_t)b * 4 * ps;
  if (singular) {
    for (int e = tid; e < N * N; e += GJB_THREADS) mixed::put4f(o, ps, (size_t)(e / N) * Np + e % N, 0.f, 0.f);
    if (tid == 0) s_out[b] = 1.f;
    return;
  }
  for (int c = tid; c < N; c += GJB_THREADS) iperm[perm[c]] = c;
  float m = 0.f;
  for (int e = tid; e < N * N; e += GJB_THREADS) {
    const float4 v = a[e];
    m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.z)));
  }
  m = block_max_f(m, s_redf);   // its barriers also publish iperm
  const float sc = mixed::pow2_scale((double)m);
  if (tid == 0) s_out[b] = sc;
  for (int e = tid; e < N * N; e += GJB_THREADS) {
    const int i = e / N, c = e % N;
    const float4 v = a[(size_t)c * N + iperm[i]];
    mixed::put4f(o, ps, (size_t)i * Np + c, v.x * sc, v.z * sc);
  }
}

template <class K>
cudaError_t set_smem(K kernel, size_t bytes) {
  return ensure_dyn_smem(reinterpret_cast<const void*>(kernel), bytes);
}

size_t gj_smem_bytes(int N, bool in_smem) {
  return (in_smem ? (size_t)N * N * sizeof(float4) : 0) + (size_t)N * (sizeof(float4) + sizeof(double2) + 2 * sizeof(int));
}

}  // namespace

size_t overlap_scratch_bytes(int WS, int N) { return (size_t)WS * N * N * sizeof(float4); }

cudaError_t overlap(const zc* A, const zc* phi, const zc* B, float4* Sff, float2* phi_perp, unsigned long long* mx,
                    int WS, int nk, int M, int n, int N, cudaStream_t st) {
  const size_t fixed = (size_t)2 * M * n * sizeof(float4);
  size_t JC = (OV_SMEM_TARGET > fixed) ? (OV_SMEM_TARGET - fixed) / ((size_t)(M + n) * sizeof(float4)) : 1;
  JC = std::max<size_t>(1, std::min<size_t>(JC, (size_t)N));
  const size_t bytes = fixed + JC * (size_t)(M + n) * sizeof(float4);
  if (bytes > SMEM_LIMIT) return cudaErrorInvalidValue;
  const dim3 grid(WS, nk, (unsigned)((N + JC - 1) / JC));
  cudaError_t e;
  if (B) {
    if ((e = set_smem(overlap_ff_kernel<true>, bytes)) != cudaSuccess) return e;
    overlap_ff_kernel<true><<<grid, OV_THREADS, bytes, st>>>(A, phi, B, Sff, phi_perp, mx, nk, M, n, N, (int)JC);
  } else {
    if ((e = set_smem(overlap_ff_kernel<false>, bytes)) != cudaSuccess) return e;
    overlap_ff_kernel<false><<<grid, OV_THREADS, bytes, st>>>(A, phi, B, Sff, phi_perp, mx, nk, M, n, N, (int)JC);
  }
  return cudaGetLastError();
}

cudaError_t invert(float4* Sff, int WS, int N, zc* logdet, int* sing, int* flags, __half* out, int Np, float* s_out,
                   cudaStream_t st) {
  cudaError_t e;
  if (out && N <= GJB_MAXN) {
    const size_t bytes = ((size_t)N * N + (size_t)GJB * N) * sizeof(float4) + gj_smem_bytes(N, false);
    if (bytes <= SMEM_LIMIT) {
      if ((e = set_smem(gjb_ff_kernel<true>, bytes)) != cudaSuccess) return e;
      gjb_ff_kernel<true><<<WS, GJB_THREADS, bytes, st>>>(Sff, N, logdet, sing, flags, out, Np, s_out);
      return cudaGetLastError();
    }
  }
  if (out && N <= GJB_GLOBAL_MAXN) {
    const size_t bytes = (size_t)GJB * N * sizeof(float4) + gj_smem_bytes(N, false);
    if (bytes <= SMEM_LIMIT) {
      if ((e = set_smem(gjb_ff_kernel<false>, bytes)) != cudaSuccess) return e;
      gjb_ff_kernel<false><<<WS, GJB_THREADS, bytes, st>>>(Sff, N, logdet, sing, flags, out, Np, s_out);
      return cudaGetLastError();
    }
  }
  const bool in_smem = N <= GJ_SMEM_MAXN && gj_smem_bytes(N, true) <= SMEM_LIMIT;
  const size_t bytes = gj_smem_bytes(N, in_smem);
#define GJ_LAUNCH(S, I)                                                                              \
  do {                                                                                               \
    if ((e = set_smem(gj_ff_kernel<S, I>, bytes)) != cudaSuccess) return e;                         \
    gj_ff_kernel<S, I><<<WS, GJ_THREADS, bytes, st>>>(Sff, N, logdet, sing, flags, out, Np, s_out); \
  } while (0)
  if (out) {
    if (in_smem) GJ_LAUNCH(true, true);
    else GJ_LAUNCH(false, true);
  } else {
    if (in_smem) GJ_LAUNCH(true, false);
    else GJ_LAUNCH(false, false);
  }
#undef GJ_LAUNCH
  return cudaGetLastError();
}

}  // namespace ffla
