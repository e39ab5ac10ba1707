// Tensor-core ("mixed") path of the k-point AFQMC walker step.
//
// Every contraction with the Cholesky vectors, the Taylor products, the
// Green's-function product and the Cholesky-QR2 Gram and apply products run as
// complex GEMMs on the tcgen05 tensor cores with an fp16 hi/lo operand split and
// fp32 accumulation (tc_gemm.cuh).  The overlap matrix, its inverse and
// log-determinant and the trial-subspace projection of the walker run in
// double-float arithmetic on the FP32 pipe (ffla.cu); the weights and every
// cross-tile energy sum stay in FP64.  The FP64 walker is the identity part of
// both one-body half steps and of the Taylor series; only the corrections pass
// through reduced precision, and they are added to it once per step.
//
// Exchange energy.  Sec. 2.2 notes that a half-rotated two-electron tensor can
// be precontracted to cut the cost of the energy by at least n_gamma, at an
// O(N^2 M^2) memory price the paper's 16 GB GPUs could not pay.  With 288 GB of
// HBM that tensor fits, so it is built once at create time, in FP64, for the
// canonical member of every pair of terms (Q, k, k') <-> (-Q, k'-Q, k) of Eq.
// kp_el (the pair contributes twice the same value):
//   Z_t[(a,s)][(b,r)] = sum_g LH[Q,k,g,a,r] LH[-Q,kx,g,b,s],   kx = k' - Q,
// and the exchange becomes, per walker-spin ws,
//   EX = -1/2 sum_t w_t sum_{(a,s)} ( sum_{(b,r)} Gh[(kx,b),(k-Q,r)] Z_t[(a,s),(b,r)] ) Gh[(k,a),(kx+Q,s)]
// i.e. one tensor-core GEMM per triple (rows = walker-spins) with a dot-product
// epilogue.  Expanding T1 and T2 of Sec. 3.2 steps 2(a)-(c) gives exactly this
// sum.
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <functional>
#include <utility>
#include <vector>

#include "mixed.hpp"
#include "attr.hpp"
#include "ffla.hpp"
#include "split.cuh"
#include "tc_gemm.cuh"

struct MixedState {
  int Np, NMp, Mp, Gp, nMp, nM, WS, T;
  // walker-dependent operands (split planes, fp16) and their scales
  __half* phi_sp = nullptr;   float* s_phi = nullptr;   // [WS][4][NM][Np]
  __half* sinvt_sp = nullptr; float* s_sinv = nullptr;  // [WS][4][N][Np]
  float2* g32 = nullptr;                                 // [Nk][Nk][WS][n][Mp]
  __half* g_sp = nullptr;     float* s_g = nullptr;     // [4][Nk][Nk][WS][n][Mp]
  __half* gsum_sp = nullptr;  float* s_gsum = nullptr;  // [4][Nk][Nk][W][n][Mp]
  __half* y_sp = nullptr;     float* s_y = nullptr;     // [4][Nk][W][Gp], s_y[Q][W]
  __half* v_sp = nullptr;                                // [W][4][NM][NMp]
  __half* t_sp[2] = {nullptr, nullptr}; float* s_t = nullptr;  // [W][4][2N][NMp]
  double2* acc = nullptr;                                // [W][2N][NM] (scratch: float4 Taylor corrections, phi_perp)
  float2* p32 = nullptr;                                 // [W][2N][NM] phi' in fp32 (Taylor series)
  double2* xpart = nullptr;                              // [T][ntile][WS]
  double2* xk = nullptr;                                 // [fb_groups][W][Nk][G] Cholesky traces per group of k blocks
  int fb_groups = 1;                                     // groups of k blocks in the force-bias GEMM
  unsigned long long* mx = nullptr;                      // max |.| bit patterns: phi[WS], sinv[WS], g[3W], acc[W]
  // static operands
  __half* lh_sp = nullptr;    float* s_lh = nullptr;    // [4][Nk][Nk][G][n][Mp], s_lh[Q][G]
  __half* lt_sp = nullptr;    float* s_l = nullptr;     // [4][Nk][Nk][M*M][Gp], s_l[Q][G]
  // Z of every triple in one array: rows 0 .. T-1 the canonical triples (exchange order),
  // rows T .. Nk^3-1 the transposes for their partners (the adjoint's operands)
  __half* z_sp = nullptr;     float* s_z = nullptr;     // [4][Nk^3][n*Mp][n*Mp], s_z[Nk^3]
  int4* tri = nullptr;                                   // [T] (Q, k, kx, weight)
  // adjoint of the exchange: the row of z_sp that holds Z of triple t = (Q nk + k) nk + kx,
  // and dEX/dGh per block
  int* zrow = nullptr;                                   // [Nk^3]
  float2* gam32 = nullptr;                               // [Nk][Nk][WS][n*Mp]
  float2* dhalf = nullptr;                               // [Nk][M][M] exp(-dt/2 H1') - I
  zc* bproj = nullptr;                                   // [Nk][M][n] A (A^dag A)^-1 per k
  float2* bproj32 = nullptr;                             // the same in fp32 (Green epilogue)
  float* inv_s_lh = nullptr;                             // 1 / s_lh
  zc* zscratch = nullptr;                                // [ZCTAS][nM*nM]
  float4* s_ff = nullptr;                                // [WS][N][N] double-float overlap matrices
  double* logr = nullptr;                                // [WS] log det R of the last Cholesky-QR2
  double2* expart = nullptr;                             // [EX_CHUNKS][WS] exchange partial sums
  // TMA ring depth of every GEMM (AFQMC_GEMM_* order), chosen at create by timing (autotune),
  // and the per-launch times measured for two and three stages (0 where not tuned)
  int ring[AFQMC_NGEMMS] = {0};
  float tune_ms[AFQMC_NGEMMS][2] = {};
  // Taylor GEMM in the CTA-pair form (chosen at create when it times faster), its B map (one
  // of the re / im halves per box) and the per-launch ms of the pair form at create
  int taylor_pair = 0;
  float taylor_pair_ms = 0.f;
  CUtensorMap m_vp;
  CUtensorMap m_sinvt, m_phi, m_gsum, m_lh, m_y, m_lt, m_t[2], m_v, m_g, m_z, m_zall;
  CUtensorMap m_phi_a, m_sinvt_b, m_t0_b;  // the same buffers boxed for the other operand slot
  std::vector<void*> allocs;
};

namespace mixed {

// Output tile width of the precise GEMM (tc_gemm.cuh): 64 columns.
constexpr int BN = tcg::BNP;
// TMA ring depth per policy: three stages by default; two where the epilogue reads global
// memory (the smaller shared-memory carve-out leaves L1 to those reads; measured faster)
constexpr int STAGES = 3;
constexpr int STAGES_LIGHT = 2;
constexpr float V_SCALE = 1024.f;   // fixed scale of vHS entries (|V| < 64 fits fp16 hi)
constexpr int ZCTAS = 304;

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
// FP64 input of moderate range: rounded once to fp32 (24 bits, of which the split keeps
// 22), then scaled (per-step operands: walkers, inverses, Green's functions)
__device__ __forceinline__ void put4(__half* base, size_t plane_stride, size_t idx, double re, double im, float s) {
  put4f(base, plane_stride, idx, (float)re * s, (float)im * s);
}
// FP64 input of any range: scaled in FP64 first (set-up data only)
__device__ __forceinline__ void put4d(__half* base, size_t plane_stride, size_t idx, double re, double im, float s) {
  put4f(base, plane_stride, idx, (float)(re * (double)s), (float)(im * (double)s));
}

__device__ __forceinline__ double block_max(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double m = 0.0;
  for (int i = 0; i < (int)((blockDim.x + 31) >> 5); ++i) m = fmax(m, red[i]);
  return m;
}
__device__ __forceinline__ double cabs_d(zc v) { return fmax(fabs(v.x), fabs(v.y)); }

template <typename T>
static cudaError_t dalloc(afqmc_kp* h, T** p, size_t count, bool zero, cudaStream_t st) {
  void* q = nullptr;
  size_t b = std::max<size_t>(count * sizeof(T), 16);
  cudaError_t e = cudaMalloc(&q, b);
  if (e != cudaSuccess) return e;
  h->mixed->allocs.push_back(q);
  h->bytes += b;
  *p = static_cast<T*>(q);
  if (zero) return cudaMemsetAsync(q, 0, b, st);
  return cudaSuccess;
}

static inline int rup(int x, int m) { return (x + m - 1) / m * m; }
static inline int cdiv(int x, int m) { return (x + m - 1) / m; }

}  // namespace mixed

// ---------------------------------------------------------------------------
// tensor maps (driver entry point fetched through the runtime)
// ---------------------------------------------------------------------------
namespace tcg {
cudaError_t make_map(CUtensorMap* map, void* base, const MapSpec& s) {
  typedef CUresult (*EncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                               const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                               CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static EncodeFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p) return cudaErrorNotSupported;
    fn = reinterpret_cast<EncodeFn>(p);
  }
  cuuint64_t dims[5], strides[4];
  cuuint32_t box[5], estr[5] = {1, 1, 1, 1, 1};
  for (int i = 0; i < 5; ++i) { dims[i] = s.dims[i]; box[i] = s.box[i]; }
  for (int i = 0; i < 4; ++i) strides[i] = s.strides[i];
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 5, base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}
}  // namespace tcg

namespace mixed {

// Build a map for an array of fp16 elements with logical dims d[0..4] (d[0]
// contiguous) and element strides e[1..4].
static cudaError_t map5(CUtensorMap* m, void* base, std::initializer_list<uint64_t> d,
                        std::initializer_list<uint64_t> estride, uint32_t rows) {
  tcg::MapSpec s;
  auto di = d.begin();
  auto ei = estride.begin();
  for (int i = 0; i < 5; ++i) s.dims[i] = di[i];
  for (int i = 0; i < 4; ++i) s.strides[i] = ei[i] * sizeof(__half);
  s.box[0] = 32;
  s.box[1] = rows;
  s.box[2] = 4;
  s.box[3] = 1;
  s.box[4] = 1;
  return tcg::make_map(m, base, s);
}

// The same for a B operand of a kPairB policy: the four planes (stride ps elements, order
// re_hi, re_lo, im_hi, im_lo in memory) are addressed as the two dimensions (re/im, hi/lo),
// so the staged box holds them as re_hi, im_hi, re_lo, im_lo; d0, d1 and the batch dimension
// keep their element strides e0 (rows) and eb.
// halves = 1: the box holds one of re / im (the CTA-pair form, each CTA staging its half).
static cudaError_t map5_pair(CUtensorMap* m, void* base, uint64_t d0, uint64_t d1, uint64_t batch, uint64_t e0,
                             uint64_t ps, uint64_t eb, uint32_t rows, uint32_t halves = 2) {
  tcg::MapSpec s;
  s.dims[0] = d0; s.dims[1] = d1; s.dims[2] = 2; s.dims[3] = 2; s.dims[4] = batch;
  s.strides[0] = e0 * sizeof(__half);
  s.strides[1] = 2 * ps * sizeof(__half);   // re -> im
  s.strides[2] = ps * sizeof(__half);       // hi -> lo
  s.strides[3] = eb * sizeof(__half);
  s.box[0] = 32; s.box[1] = rows; s.box[2] = halves; s.box[3] = 2; s.box[4] = 1;
  return tcg::make_map(m, base, s);
}

// ---------------------------------------------------------------------------
// GEMM policies
// ---------------------------------------------------------------------------

// Gh[ws] = B^T + S^-T phi_perp^T : rows i = (k1, a), cols (k2, p); written to g32 in tile
// layout.  B = A (A^dag A)^-1 and phi_perp = phi - B S (see green()).
struct GreenP {
  static constexpr bool kConjA = false;
  static constexpr bool kPairB = true;
  static constexpr int kStages = STAGES;
  int tiles, kchunks;
  int mt_n, nt_n, N, NM, n, M, Mp, nk, WS;
  const float* s_sinv;
  const float* s_phi;
  const float2* bproj32;
  float2* g32;
  __device__ void tile(int t, int& b, int& mt, int& nt) const {
    nt = t % nt_n;
    mt = (t / nt_n) % mt_n;
    b = t / (nt_n * mt_n);
  }
  __device__ tcg::Coords coords(int b, int mt, int nt, int kc) const {
    tcg::Coords c = {{kc * 32, mt * 128, 0, b, 0}, {kc * 32, nt * BN, 0, 0, b}};
    return c;
  }
  __device__ void store_tile(int b, int mt, int nt, const float2* tile, int tid, int, int) const {
    const float st = 1.f / (s_sinv[b] * s_phi[b]);
    for (int e = tid; e < 128 * BN; e += 128) {
      const int r = e / BN, c = e % BN;
      const int i = mt * 128 + r, col = nt * BN + c;
      if (i >= N || col >= NM) continue;
      const int k1 = i / n, a = i % n, k2 = col / M, p = col % M;
      const float2 v = tile[r * tcg::STAGE_LD + c];
      float gr = v.x * st, gi = v.y * st;
      if (k1 == k2) {
        const float2 bp = bproj32[((size_t)k1 * M + p) * n + a];
        gr += bp.x;
        gi += bp.y;
      }
      g32[((((size_t)k1 * nk + k2) * WS + b) * n + a) * Mp + p] = make_float2(gr, gi);
    }
  }
};

// Partial Cholesky trace of one group of k blocks:
//   Xk[grp][w][Q][g] = sum_{k in grp} sum_{a,r} LH[Q,k,g,a,r] Gsum_w[(k,a),(k-Q,r)],
// the group's k blocks running one after another along the GEMM's k loop (kcb chunks each).
// The groups (ng, dividing Nk) are as few as still give the GPU enough tiles; they are summed
// in FP64 by xsum_kernel.  Both operands carry one scale over all k (per (Q, g) and per
// walker), so the blocks of a group add in one fp32 running sum.
struct ForceBiasP {
  static constexpr bool kConjA = false;
  static constexpr bool kPairB = true;
  static constexpr int kStages = STAGES_LIGHT;
  int tiles, kchunks;
  int mt_n, nt_n, W, G, nk, ng, kg, kcb;   // ng groups of kg k blocks, kcb chunks per block
  const int* kminus;
  const float* s_gsum;
  const float* inv_s_lh;
  double2* Xk;  // [ng][W][Nk(Q)][G]
  __device__ void tile(int t, int& b, int& mt, int& nt) const {
    nt = t % nt_n;
    mt = (t / nt_n) % mt_n;
    b = t / (nt_n * mt_n);   // b = Q * ng + group
  }
  // rows = Cholesky index g of LH[Q][k] (A), columns = walkers (B = spin-summed Gh)
  __device__ tcg::Coords coords(int b, int mt, int nt, int kc) const {
    const int Q = b / ng, k = (b % ng) * kg + kc / kcb, c0 = (kc % kcb) * 32;
    tcg::Coords c = {{c0, mt * 128, 0, k, Q}, {c0, nt * BN, 0, 0, k * nk + kminus[k * nk + Q]}};
    return c;
  }
  __device__ void store_tile(int b, int mt, int nt, const float2* tile, int tid, int, int) const {
    const int Q = b / ng, grp = b % ng;
    // down the rows: consecutive threads write consecutive g of one walker
    for (int e = tid; e < 128 * BN; e += 128) {
      const int r = e % 128, c = e / 128;
      const int g = mt * 128 + r, w = nt * BN + c;
      if (w >= W || g >= G) continue;
      const float f = inv_s_lh[Q * G + g] / s_gsum[w];
      const float2 v = tile[r * tcg::STAGE_LD + c];
      Xk[(((size_t)grp * W + w) * nk + Q) * G + g] = make_double2((double)(v.x * f), (double)(v.y * f));
    }
  }
};

// X[w][Q][g] = sum over the groups of Xk[grp][w][Q][g]  (FP64, fixed order)
__global__ void xsum_kernel(const double2* Xk, zc* X, int ng, size_t per) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < per; e += (size_t)gridDim.x * blockDim.x) {
    double2 s = make_double2(0.0, 0.0);
    for (int k = 0; k < ng; ++k) {
      const double2 v = Xk[(size_t)k * per + e];
      s.x += v.x;
      s.y += v.y;
    }
    X[e] = s;
  }
}

// V[w][(k,p)][(k-Q,r)] = sum_g y[w,Q,g] L[Q,k,g,p,r]  -> split planes with a fixed scale
struct VhsP {
  static constexpr bool kConjA = false;
  static constexpr bool kPairB = true;
  static constexpr int kStages = STAGES;
  int tiles, kchunks;
  int mt_n, nt_n, W, M, nk, NM, NMp;
  const int* kminus;
  const float* s_y;  // [Q][W]
  __half* v_sp;
  int* overflow;
  __device__ void tile(int t, int& b, int& mt, int& nt) const {
    nt = t % nt_n;
    mt = (t / nt_n) % mt_n;
    b = t / (nt_n * mt_n);   // b = Q * nk + k
  }
  // rows (p, r) of L[Q][k] (A), columns = walkers (B = y[Q])
  __device__ tcg::Coords coords(int b, int mt, int nt, int kc) const {
    const int Q = b / nk, k = b % nk;
    tcg::Coords c = {{kc * 32, mt * 128, 0, k, Q}, {kc * 32, nt * BN, 0, 0, Q}};
    return c;
  }
  __device__ void store_tile(int b, int mt, int nt, const float2* tile, int tid, int, int) const {
    const int Q = b / nk, k = b % nk, kq = kminus[k * nk + Q];
    const size_t ps = (size_t)NM * NMp;
    bool bad = false;
    if ((M & 1) == 0) {
      // M even: rows 2i, 2i+1 of a tile are r, r+1 of one (p, r) run and land on one
      // 4-byte aligned pair of the output row, so each plane takes one 32-bit store
      for (int e = tid; e < 64 * BN; e += 128) {
        const int rp = e % 64, c = e / 64;
        const int pr = mt * 128 + 2 * rp, w = nt * BN + c;
        if (w >= W || pr >= M * M) continue;
        const float st = V_SCALE / s_y[Q * W + w];
        const float2 v0 = tile[(2 * rp) * tcg::STAGE_LD + c], v1 = tile[(2 * rp + 1) * tcg::STAGE_LD + c];
        const float r0 = v0.x * st, i0 = v0.y * st, r1 = v1.x * st, i1 = v1.y * st;
        bad |= !(fmaxf(fmaxf(fabsf(r0), fabsf(i0)), fmaxf(fabsf(r1), fabsf(i1))) < 60000.f);
        const int pp = pr / M, rr = pr % M;
        __half* base = v_sp + (size_t)w * 4 * ps + (size_t)(k * M + pp) * NMp + kq * M + rr;
        __half h0, l0, h1, l1;
        split_val(r0, h0, l0);
        split_val(r1, h1, l1);
        *reinterpret_cast<__half2*>(base) = __halves2half2(h0, h1);
        *reinterpret_cast<__half2*>(base + ps) = __halves2half2(l0, l1);
        split_val(i0, h0, l0);
        split_val(i1, h1, l1);
        *reinterpret_cast<__half2*>(base + 2 * ps) = __halves2half2(h0, h1);
        *reinterpret_cast<__half2*>(base + 3 * ps) = __halves2half2(l0, l1);
      }
    } else {
      // down the rows: consecutive threads write consecutive r of one (walker, p)
      for (int e = tid; e < 128 * BN; e += 128) {
        const int r = e % 128, c = e / 128;
        const int pr = mt * 128 + r, w = nt * BN + c;
        if (w >= W || pr >= M * M) continue;
        const float st = V_SCALE / s_y[Q * W + w];
        const float2 v = tile[r * tcg::STAGE_LD + c];
        const float vr = v.x * st, vi = v.y * st;
        bad |= !(fabsf(vr) < 60000.f && fabsf(vi) < 60000.f);
        const int pp = pr / M, rr = pr % M;
        put4f(v_sp + (size_t)w * 4 * ps, ps, (size_t)(k * M + pp) * NMp + kq * M + rr, vr, vi);
      }
    }
    if (bad) atomicExch(overflow, 1);
  }
};

// One Taylor term: T_j[w] = V[w] T_{j-1}[w] / j in transposed form (rows j' = (spin, column)).
// One Horner step of the Taylor series (order K): u <- phi' + V u / j, j = K .. 1, so that
// after the last step u = sum_j V^j phi' / j! (Sec. 3.2 step 3).  Rows j of R = 2N
// (spin, column), columns i of NM, D = sum_k U[j][k] V[i][k]; D carries the operand
// scales s_t (A) and V_SCALE (B), so (V u / j) * s_t = D * inv_j / V_SCALE.
//   inner steps: the new u * s_t = p32 * s_t + D * inv_j / V_SCALE goes to the split
//                planes t_next (fp32: u only ever enters a further product with V);
//   last step:   acc = phi' (FP64) + V u, the identity part exact.
struct TaylorP {
  static constexpr bool kConjA = false;
  static constexpr bool kPairB = true;
  static constexpr int kStages = STAGES;
  int tiles, kchunks;
  int mt_n, nt_n, R, NM, NMp;
  float inv_j;
  int last;
  const float* s_t;
  const float2* p32;  // [W][R][NM] phi' in fp32
  float4* corr;       // [W][R][NM] (d, .) with d = phi' - phi on entry; (phi'' - phi, phi'') after the last step
  __half* t_next;     // [W][4][R][NMp]
  __device__ void tile(int t, int& b, int& mt, int& nt) const {
    nt = t % nt_n;
    mt = (t / nt_n) % mt_n;
    b = t / (nt_n * mt_n);
  }
  __device__ tcg::Coords coords(int b, int mt, int nt, int kc) const {
    tcg::Coords c = {{kc * 32, mt * 128, 0, b, 0}, {kc * 32, nt * BN, 0, 0, b}};
    return c;
  }
  __device__ void store_tile(int b, int mt, int nt, const float2* tile, int tid, int, int) const {
    const float st = inv_j / V_SCALE, sc = s_t[b];
    // all U reads of a batch are issued before its writes, so they overlap
    if (last) {
      constexpr int U = 8;
      const float inv_s = 1.f / sc;   // power of two: exact
      float4* cb = corr + (size_t)b * R * NM;
      const float2* pb = p32 + (size_t)b * R * NM;
      for (int e0 = tid; e0 < 128 * BN; e0 += 128 * U) {
        float2 dv[U], pv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int e = e0 + 128 * u, j = mt * 128 + e / BN, i = nt * BN + e % BN;
          if (j < R && i < NM) {
            const size_t o = (size_t)j * NM + i;
            dv[u] = reinterpret_cast<const float2*>(cb)[2 * o];
            pv[u] = pb[o];
          }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int e = e0 + 128 * u, r = e / BN, c = e % BN, j = mt * 128 + r, i = nt * BN + c;
          if (j >= R || i >= NM) continue;
          const float2 v = tile[r * tcg::STAGE_LD + c];
          const float vr = v.x * st * inv_s, vi = v.y * st * inv_s;   // V u
          cb[(size_t)j * NM + i] = make_float4(dv[u].x + vr, dv[u].y + vi, pv[u].x + vr, pv[u].y + vi);
        }
      }
    } else if ((NM & 1) == 0) {
      // even NM: a thread takes two adjacent columns, one 16-byte load of phi' and one
      // 32-bit store per plane
      constexpr int U = 8;
      const size_t ps = (size_t)R * NMp;
      __half* tb = t_next + (size_t)b * 4 * ps;
      const float4* pb = reinterpret_cast<const float4*>(p32 + (size_t)b * R * NM);
      for (int e0 = tid; e0 < 128 * (BN / 2); e0 += 128 * U) {
        float4 pv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int e = e0 + 128 * u, j = mt * 128 + e / (BN / 2), i = nt * BN + 2 * (e % (BN / 2));
          if (j < R && i < NM) pv[u] = pb[((size_t)j * NM + i) / 2];
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int e = e0 + 128 * u, r = e / (BN / 2), c = 2 * (e % (BN / 2)), j = mt * 128 + r, i = nt * BN + c;
          if (j >= R || i >= NM) continue;
          const float2 v0 = tile[r * tcg::STAGE_LD + c], v1 = tile[r * tcg::STAGE_LD + c + 1];
          __half h0, l0, h1, l1;
          __half* o = tb + (size_t)j * NMp + i;
          split_val(fmaf(pv[u].x, sc, v0.x * st), h0, l0);
          split_val(fmaf(pv[u].z, sc, v1.x * st), h1, l1);
          *reinterpret_cast<__half2*>(o) = __halves2half2(h0, h1);
          *reinterpret_cast<__half2*>(o + ps) = __halves2half2(l0, l1);
          split_val(fmaf(pv[u].y, sc, v0.y * st), h0, l0);
          split_val(fmaf(pv[u].w, sc, v1.y * st), h1, l1);
          *reinterpret_cast<__half2*>(o + 2 * ps) = __halves2half2(h0, h1);
          *reinterpret_cast<__half2*>(o + 3 * ps) = __halves2half2(l0, l1);
        }
      }
    } else {
      constexpr int U = 8;
      const size_t ps = (size_t)R * NMp;
      __half* tb = t_next + (size_t)b * 4 * ps;
      const float2* pb = p32 + (size_t)b * R * NM;
      for (int e0 = tid; e0 < 128 * BN; e0 += 128 * U) {
        float2 pv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int e = e0 + 128 * u, j = mt * 128 + e / BN, i = nt * BN + e % BN;
          if (j < R && i < NM) pv[u] = pb[(size_t)j * NM + i];
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int e = e0 + 128 * u, r = e / BN, c = e % BN, j = mt * 128 + r, i = nt * BN + c;
          if (j >= R || i >= NM) continue;
          const float2 v = tile[r * tcg::STAGE_LD + c];
          put4f(tb, ps, (size_t)j * NMp + i, fmaf(pv[u].x, sc, v.x * st), fmaf(pv[u].y, sc, v.y * st));
        }
      }
    }
  }
};

// Exchange: rows = walker-spins, cols = (a, s) of Z_t in the padded order a*Mp + s, so the
// matching 64 columns of Gh[(k,a),(kx+Q,s)] are one contiguous run per walker-spin.  The
// store warps dot each staged row with that run (one thread per row), reading Gh from
// L2/HBM while the drain warps already accumulate the next tile.
struct ExchangeP {
  static constexpr bool kConjA = false;
  static constexpr bool kStreamB = true;   // Z streams through L2 once per launch when mt_n == 1
  static constexpr bool kPairB = true;
  static constexpr int kStages = STAGES_LIGHT;
  int tiles, kchunks;
  int mt_n, nt_n, WS, nk, nMp;
  const int* kminus;
  const int* minus;
  const int4* tri;
  const float* s_g;
  const float* s_z;
  const float2* g32;  // [Nk][Nk][WS][n*Mp]
  double2* xpart;     // [T][nt_n][WS]
  // with more than one row tile every Z tile is read once per row tile: keep it in L2 then
  __device__ bool stream_b() const { return mt_n == 1; }
  __device__ void tile(int t, int& b, int& mt, int& nt) const {
    nt = t % nt_n;
    mt = (t / nt_n) % mt_n;
    b = t / (nt_n * mt_n);
  }
  __device__ tcg::Coords coords(int t, int mt, int nt, int kc) const {
    const int4 q = tri[t];  // (Q, k, kx, weight)
    tcg::Coords c = {{kc * 32, mt * 128, 0, kminus[q.y * nk + q.x], q.z}, {kc * 32, nt * BN, 0, 0, t}};
    return c;
  }
  // Each store warp takes 32 rows of the tile, four at a time: eight lanes per row, each
  // reading four 16-byte pieces of the row's partner run, so that one warp load covers four
  // whole 128-byte lines.  Every load of the tile is issued before the first product.
  __device__ void store_tile(int t, int mt, int nt, const float2* tile, int tid, int, int lane) const {
    const int4 q = tri[t];
    const int kxq = kminus[q.z * nk + minus[q.x]];  // kx + Q
    const float2* gb = g32 + ((size_t)q.y * nk + kxq) * WS * nMp + nt * BN;
    // padding columns (s >= M) of Z_t are zero, so every column below n*Mp takes part
    const int pairs = min(BN, nMp - nt * BN) / 2;
    const int ri = lane >> 3, cl = lane & 7, r0 = (tid >> 5) * 32;
    constexpr int IT = 8, UJ = BN / 16;   // rows per lane, 16-byte pieces per lane and row
    float4 gv[IT][UJ];
#pragma unroll
    for (int it = 0; it < IT; ++it) {
      const int ws = mt * 128 + r0 + 4 * it + ri;
      const float4* g4 = reinterpret_cast<const float4*>(gb + (size_t)ws * nMp);
#pragma unroll
      for (int u = 0; u < UJ; ++u) {
        const int j = cl + 8 * u;
        gv[it][u] = (ws < WS && j < pairs) ? g4[j] : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    const float inv_z = 1.f / s_z[t];
#pragma unroll
    for (int it = 0; it < IT; ++it) {
      const int r = r0 + 4 * it + ri, ws = mt * 128 + r;
      float pr0 = 0.f, pi0 = 0.f, pr1 = 0.f, pi1 = 0.f;
#pragma unroll
      for (int u = 0; u < UJ; ++u) {
        const int j = cl + 8 * u;
        const float2 y0 = tile[r * tcg::STAGE_LD + 2 * j], y1 = tile[r * tcg::STAGE_LD + 2 * j + 1];
        const float4 g = gv[it][u];
        pr0 = fmaf(y0.x, g.x, fmaf(-y0.y, g.y, pr0));
        pi0 = fmaf(y0.x, g.y, fmaf(y0.y, g.x, pi0));
        pr1 = fmaf(y1.x, g.z, fmaf(-y1.y, g.w, pr1));
        pi1 = fmaf(y1.x, g.w, fmaf(y1.y, g.z, pi1));
      }
      float pr = pr0 + pr1, pi = pi0 + pi1;
#pragma unroll
      for (int o = 4; o > 0; o >>= 1) {
        pr += __shfl_xor_sync(0xffffffffu, pr, o);
        pi += __shfl_xor_sync(0xffffffffu, pi, o);
      }
      if (cl == 0 && ws < WS) {
        const float inv = inv_z / s_g[ws];   // powers of two: exact after the sum
        xpart[((size_t)t * nt_n + nt) * WS + ws] = make_double2((double)(pr * inv), (double)(pi * inv));
      }
    }
  }
};

// Adjoint of the exchange energy.  EX = -1/2 sum over all triples t = (Q, k, kx) of
// Gh_beta^T Z_t Gh_alpha with alpha = (kx, k-Q), beta = (k, kx+Q), and the partner
// (-Q, kx, k) of t swaps alpha and beta and transposes Z, so for a block beta = (k1, k2)
//   dEX/dGh_beta[ws][(a,s)] = - sum_Q sum_{(b,r)} Z_t[(a,s)][(b,r)] Gh[(kx,b),(k1-Q,r)],
//   t = (Q, k1, kx), kx = k2 - Q.
// One tile per (beta, walker-spin rows, column block); the k loop runs over Q and the
// (b, r) chunks of each triple, and every triple's own Z scale is folded in as its
// chunks are drained.  gam32 receives the sum without the minus sign.
struct AdjointP {
  static constexpr bool kConjA = false;
  static constexpr bool kStreamB = true;   // Z streams through L2 once per launch when mt_n == 1
  static constexpr bool kChunkScale = true;
  static constexpr bool kPairB = true;
  static constexpr int kStages = STAGES_LIGHT;
  int tiles, kchunks;  // kchunks = nk * kcb
  int kcb, mt_n, nt_n, WS, nk, nMp;
  const int* kminus;
  const float* s_g;
  const int* zrow;     // [Nk^3] row of z_sp holding Z of triple t
  const float* s_z;    // [Nk^3] per row
  float2* gam32;
  // with more than one row tile every Z tile is read once per row tile: keep it in L2 then
  __device__ bool stream_b() const { return mt_n == 1; }
  __device__ void tile(int t, int& b, int& mt, int& nt) const {
    nt = t % nt_n;
    mt = (t / nt_n) % mt_n;
    b = t / (nt_n * mt_n);
  }
  __device__ void split_k(int b, int kc, int& tf, int& km, int& kx, int& kk) const {
    const int Q = kc / kcb;
    kk = kc - Q * kcb;
    const int k1 = b / nk, k2 = b - k1 * nk;
    kx = kminus[k2 * nk + Q];   // k2 - Q
    km = kminus[k1 * nk + Q];   // k1 - Q
    tf = zrow[(Q * nk + k1) * nk + kx];
  }
  __device__ tcg::Coords coords(int b, int mt, int nt, int kc) const {
    int tf, km, kx, kk;
    split_k(b, kc, tf, km, kx, kk);
    tcg::Coords c = {{kk * 32, mt * 128, 0, km, kx}, {kk * 32, nt * BN, 0, 0, tf}};
    return c;
  }
  __device__ float chunk_scale(int b, int kc) const {
    int tf, km, kx, kk;
    split_k(b, kc, tf, km, kx, kk);
    return 1.f / s_z[tf];   // a power of two: exact
  }
  __device__ void store_tile(int b, int mt, int nt, const float2* tile, int tid, int, int) const {
    const int cols = min(BN, nMp - nt * BN);
    for (int e = tid; e < 128 * BN; e += 128) {
      const int r = e / BN, c = e % BN;
      const int ws = mt * 128 + r;
      if (ws >= WS || c >= cols) continue;
      const float inv = 1.f / s_g[ws];
      const float2 v = tile[r * tcg::STAGE_LD + c];
      gam32[((size_t)b * WS + ws) * nMp + nt * BN + c] = make_float2(v.x * inv, v.y * inv);
    }
  }
};

// Gram[ws] = phi_ws^dag phi_ws from the transposed split planes (rows = columns of phi).
struct GramP {
  static constexpr bool kConjA = true;
  static constexpr bool kPairB = true;
  static constexpr int kStages = STAGES;
  int tiles, kchunks;
  int mt_n, nt_n, N;
  const float* s_t;   // per walker
  float2* gram;       // [WS][N][N]
  __device__ void tile(int t, int& b, int& mt, int& nt) const {
    nt = t % nt_n;
    mt = (t / nt_n) % mt_n;
    b = t / (nt_n * mt_n);
  }
  __device__ tcg::Coords coords(int ws, int mt, int nt, int kc) const {
    const int w = ws >> 1, sp = ws & 1;
    tcg::Coords c = {{kc * 32, sp * N + mt * 128, 0, w, 0}, {kc * 32, sp * N + nt * BN, 0, 0, w}};
    return c;
  }
  __device__ void store_tile(int ws, int mt, int nt, const float2* tile, int tid, int, int) const {
    const float sc = s_t[ws >> 1];
    const float st = 1.f / (sc * sc);
    for (int e = tid; e < 128 * BN; e += 128) {
      const int r = e / BN, c = e % BN;
      const int i = mt * 128 + r, j = nt * BN + c;
      if (i >= N || j >= N) continue;
      const float2 v = tile[r * tcg::STAGE_LD + c];
      gram[((size_t)ws * N + i) * N + j] = make_float2(v.x * st, v.y * st);
    }
  }
};

// phi[ws] <- phi[ws] R^-1 : rows r = (k,p), columns j; B = (R^-1)^T split planes.
struct ApplyRP {
  static constexpr bool kConjA = false;
  static constexpr bool kPairB = true;
  static constexpr int kStages = STAGES;
  int tiles, kchunks;
  int mt_n, nt_n, NM, N;
  const float* s_phi;
  const float* s_r;
  zc* phi;
  __device__ void tile(int t, int& b, int& mt, int& nt) const {
    nt = t % nt_n;
    mt = (t / nt_n) % mt_n;
    b = t / (nt_n * mt_n);
  }
  __device__ tcg::Coords coords(int ws, int mt, int nt, int kc) const {
    tcg::Coords c = {{kc * 32, mt * 128, 0, ws, 0}, {kc * 32, nt * BN, 0, 0, ws}};
    return c;
  }
  __device__ void store_tile(int ws, int mt, int nt, const float2* tile, int tid, int, int) const {
    const float st = 1.f / (s_phi[ws] * s_r[ws]);
    for (int e = tid; e < 128 * BN; e += 128) {
      const int r = e / BN, c = e % BN;
      const int row = mt * 128 + r, j = nt * BN + c;
      if (row >= NM || j >= N) continue;
      const float2 v = tile[r * tcg::STAGE_LD + c];
      phi[((size_t)ws * NM + row) * N + j] = make_double2((double)(v.x * st), (double)(v.y * st));
    }
  }
};

// ---------------------------------------------------------------------------
// conversion kernels
// ---------------------------------------------------------------------------

// ---- two-pass splits: block-parallel max |.| (atomic max on the bit pattern of a
// non-negative double), then a block-parallel split with the resulting scale.
__device__ __forceinline__ void atomic_max_pos(unsigned long long* a, double v) {
  atomicMax(a, static_cast<unsigned long long>(__double_as_longlong(v)));
}
__device__ __forceinline__ float scale_from_bits(const unsigned long long* a) {
  return pow2_scale(__longlong_as_double(static_cast<long long>(*a)));
}

// max |.| over each of nmat contiguous arrays of `per` complex doubles; grid (nmat, chunks)
// The maximum is taken on the bit patterns of |x|: for non-negative doubles they order like
// the values (NaN patterns sort above every finite value, as the scale wants), and
// integer max keeps the FP64 pipe free.
__global__ void maxabs_kernel(const zc* src, size_t per, unsigned long long* out) {
  __shared__ unsigned long long red[32];
  const size_t chunk = (per + gridDim.y - 1) / gridDim.y;
  const size_t b = blockIdx.y * chunk, e_end = min(per, b + chunk);
  const unsigned long long* p = reinterpret_cast<const unsigned long long*>(src + (size_t)blockIdx.x * per);
  constexpr unsigned long long ABS = 0x7fffffffffffffffull;
  unsigned long long m = 0;
  for (size_t e = b + threadIdx.x; e < e_end; e += blockDim.x) {
    const unsigned long long re = p[2 * e] & ABS, im = p[2 * e + 1] & ABS;
    m = max(m, max(re, im));
  }
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) m = max(m, red[i]);
    atomicMax(out + blockIdx.x, m);
  }
}

// src[m][rows][cols] (FP64) -> dst[m][4][rows][ldd] with the per-matrix scale; grid (nmat, chunks)
__global__ void split_rows_kernel(const zc* src, int rows, int cols, int ldd, const unsigned long long* mx,
                                  float* scale, __half* dst) {
  const int mI = blockIdx.x;
  const float s = scale_from_bits(mx + mI);
  if (blockIdx.y == 0 && threadIdx.x == 0) scale[mI] = s;
  const size_t per = (size_t)rows * cols, chunk = (per + gridDim.y - 1) / gridDim.y;
  const size_t b = blockIdx.y * chunk, e_end = min(per, b + chunk);
  const zc* p = src + (size_t)mI * per;
  const size_t ps = (size_t)rows * ldd;
  __half* o = dst + (size_t)mI * 4 * ps;
  for (size_t e = b + threadIdx.x; e < e_end; e += blockDim.x) {
    const size_t i = e / cols, j = e % cols;
    put4(o, ps, i * ldd + j, p[e].x, p[e].y, s);
  }
}

// src[m][rows][cols] (fp32) -> dst[m][4][rows][ldd] with the per-matrix scale; grid (nmat, chunks)
__global__ void split_rows32_kernel(const float2* src, int rows, int cols, int ldd, const unsigned long long* mx,
                                    float* scale, __half* dst) {
  const int mI = blockIdx.x;
  const float s = scale_from_bits(mx + mI);
  if (blockIdx.y == 0 && threadIdx.x == 0) scale[mI] = s;
  const float2* p = src + (size_t)mI * rows * cols;
  const size_t ps = (size_t)rows * ldd;
  __half* o = dst + (size_t)mI * 4 * ps;
  if ((cols & 1) == 0 && (ldd & 1) == 0) {
    // column pairs: one 16-byte load and one 32-bit store per plane
    const size_t per = (size_t)rows * (cols / 2), chunk = (per + gridDim.y - 1) / gridDim.y;
    const size_t b = blockIdx.y * chunk, e_end = min(per, b + chunk);
    const float4* p4 = reinterpret_cast<const float4*>(p);
    for (size_t e = b + threadIdx.x; e < e_end; e += blockDim.x) {
      const size_t i = e / (cols / 2), j = 2 * (e % (cols / 2));
      const float4 v = p4[(i * cols + j) / 2];
      __half h0, l0, h1, l1;
      __half* q = o + i * ldd + j;
      split_val(v.x * s, h0, l0);
      split_val(v.z * s, h1, l1);
      *reinterpret_cast<__half2*>(q) = __halves2half2(h0, h1);
      *reinterpret_cast<__half2*>(q + ps) = __halves2half2(l0, l1);
      split_val(v.y * s, h0, l0);
      split_val(v.w * s, h1, l1);
      *reinterpret_cast<__half2*>(q + 2 * ps) = __halves2half2(h0, h1);
      *reinterpret_cast<__half2*>(q + 3 * ps) = __halves2half2(l0, l1);
    }
    return;
  }
  const size_t per = (size_t)rows * cols, chunk = (per + gridDim.y - 1) / gridDim.y;
  const size_t b = blockIdx.y * chunk, e_end = min(per, b + chunk);
  for (size_t e = b + threadIdx.x; e < e_end; e += blockDim.x) {
    const size_t i = e / cols, j = e % cols;
    put4f(o, ps, i * ldd + j, p[e].x * s, p[e].y * s);
  }
}

// max |.| of g32 per walker-spin and of the spin sum per walker; grid (W, chunks)
__device__ __forceinline__ float block_max_f(float v, float* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  float m = 0.f;
  for (int i = 0; i < (int)((blockDim.x + 31) >> 5); ++i) m = fmaxf(m, red[i]);
  return m;
}
__device__ __forceinline__ float cabs_inf(float2 v) { return fmaxf(fabsf(v.x), fabsf(v.y)); }

// max |.| of g32 per walker-spin and of the spin sum per walker, in fp32; grid (W, chunks)
__global__ void green_max_kernel(const float2* g32, unsigned long long* mx, int nk, int W, int nMp) {
  const int w = blockIdx.x, WS = 2 * W;
  __shared__ float red[32];
  const unsigned per = (unsigned)(nk * nk * nMp), chunk = (per + gridDim.y - 1) / gridDim.y;
  const unsigned b = blockIdx.y * chunk, e_end = min(per, b + chunk);
  float m0 = 0.f, m1 = 0.f, ms = 0.f;
  for (unsigned e = b + threadIdx.x; e < e_end; e += blockDim.x) {
    const unsigned blk = e / nMp, off = e % nMp;
    const float2 a = g32[((size_t)blk * WS + 2 * w) * nMp + off];
    const float2 c = g32[((size_t)blk * WS + 2 * w + 1) * nMp + off];
    m0 = fmaxf(m0, cabs_inf(a));
    m1 = fmaxf(m1, cabs_inf(c));
    ms = fmaxf(ms, cabs_inf(make_float2(a.x + c.x, a.y + c.y)));
  }
  m0 = block_max_f(m0, red);
  m1 = block_max_f(m1, red);
  ms = block_max_f(ms, red);
  if (threadIdx.x == 0) {
    atomic_max_pos(mx + 3 * w, (double)m0);
    atomic_max_pos(mx + 3 * w + 1, (double)m1);
    atomic_max_pos(mx + 3 * w + 2, (double)ms);
  }
}

// g32 [Nk][Nk][WS][n][Mp] -> g_sp (per walker-spin scale) and gsum_sp (spin sum, per walker scale)
__global__ void split_green_kernel(const float2* g32, const unsigned long long* mx, __half* gsp, float* s_g,
                                   __half* gsum, float* s_gsum, int nk, int W, int nMp) {
  const int w = blockIdx.x, WS = 2 * W;
  const float s0 = scale_from_bits(mx + 3 * w), s1 = scale_from_bits(mx + 3 * w + 1),
              ss = scale_from_bits(mx + 3 * w + 2);
  if (blockIdx.y == 0 && threadIdx.x == 0) {
    s_g[2 * w] = s0;
    s_g[2 * w + 1] = s1;
    s_gsum[w] = ss;
  }
  const unsigned per = (unsigned)(nk * nk * nMp), chunk = (per + gridDim.y - 1) / gridDim.y;
  const unsigned b = blockIdx.y * chunk, e_end = min(per, b + chunk);
  const size_t psg = (size_t)nk * nk * WS * nMp, pss = (size_t)nk * nk * W * nMp;
  for (unsigned e = b + threadIdx.x; e < e_end; e += blockDim.x) {
    const unsigned blk = e / nMp, off = e % nMp;
    const size_t i0 = ((size_t)blk * WS + 2 * w) * nMp + off;
    const float2 a = g32[i0];
    const float2 c = g32[i0 + nMp];
    put4f(gsp, psg, i0, a.x * s0, a.y * s0);
    put4f(gsp, psg, i0 + nMp, c.x * s1, c.y * s1);
    put4f(gsum, pss, ((size_t)blk * W + w) * nMp + off, (a.x + c.x) * ss, (a.y + c.y) * ss);
  }
}

// y [W][Nk][G] (zc, carries sqrt(dt)) -> y_sp [4][Nk][W][Gp] of y / s_l[Q][g], scale s_y[Q][W]
__global__ void split_y_kernel(const zc* y, const float* s_l, __half* out, float* s_y, int nk, int W, int G, int Gp) {
  const int Q = blockIdx.x, w = blockIdx.y;
  __shared__ double red[32];
  const zc* yp = y + ((size_t)w * nk + Q) * G;
  double m = 0.0;
  for (int g = threadIdx.x; g < G; g += blockDim.x) {
    const double f = 1.0 / (double)s_l[Q * G + g];
    m = fmax(m, cabs_d(yp[g]) * f);
  }
  m = block_max(m, red);
  const float s = pow2_scale(m);
  if (threadIdx.x == 0) s_y[Q * W + w] = s;
  const size_t ps = (size_t)nk * W * Gp;
  for (int g = threadIdx.x; g < G; g += blockDim.x) {
    const double f = 1.0 / (double)s_l[Q * G + g];
    put4(out, ps, ((size_t)Q * W + w) * Gp + g, yp[g].x * f, yp[g].y * f, s);
  }
}

// Both one-body half steps apply D = exp(-dt/2 H1') - I of one k block to 64 walker
// columns staged in shared memory (blk[q][j], j < 64, rows padded to OB_LD so that the
// transposing fill of the second half step is free of bank conflicts).  D is staged transposed,
// Dt[q][p], and a thread forms orbital p for the four columns jq, jq+16, jq+32, jq+48: the
// four products share each D element from a register.
constexpr int OB_LD = 65;
__device__ __forceinline__ void onebody_apply4(const float2* Dt, const float2* blk, int M, int p, int jq,
                                               float2 (&c)[4]) {
#pragma unroll
  for (int u = 0; u < 4; ++u) c[u] = make_float2(0.f, 0.f);
  for (int q = 0; q < M; ++q) {
    const float2 d = Dt[q * M + p];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const float2 b = blk[q * OB_LD + jq + 16 * u];
      c[u].x = fmaf(d.x, b.x, fmaf(-d.y, b.y, c[u].x));
      c[u].y = fmaf(d.x, b.y, fmaf(d.y, b.x, c[u].y));
    }
  }
}

// First one-body half step, phi' = phi + D phi (Sec. 3.2 step 3), in the transposed
// (row = (spin, column), column = orbital) layout of the Taylor series, as fp32 parts only:
// p32 = phi' (rounded) and corr.xy = D phi.  The FP64 walker itself is added back once,
// after the series (onebody_out_kernel).  mx[w] = max |p32|.
// grid (k, ws, j-chunk of 64)
__global__ void onebody_in_kernel(const zc* phi, const float2* dhalf, float4* corr, float2* p32,
                                  unsigned long long* mx, int nk, int M, int N, int NM) {
  __shared__ double red[32];
  const int k = blockIdx.x, ws = blockIdx.y, j0 = blockIdx.z * 64;
  const int w = ws >> 1, sp = ws & 1;
  const int jn = min(64, N - j0);
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* blk = reinterpret_cast<float2*>(smraw);          // [M][OB_LD]
  float2* Dt = blk + M * OB_LD;                                 // [M][M], Dt[q][p] = D[p][q]
  for (int e = threadIdx.x; e < M * M; e += blockDim.x) {
    const int p = e / M, q = e % M;
    Dt[q * M + p] = dhalf[(size_t)k * M * M + e];
  }
  const zc* src = phi + (size_t)ws * NM * N;
  for (int e = threadIdx.x; e < M * 64; e += blockDim.x) {
    const int q = e / 64, j = e % 64;
    float2 v = make_float2(0.f, 0.f);
    if (j < jn) {
      const zc x = src[(size_t)(k * M + q) * N + j0 + j];
      v = make_float2((float)x.x, (float)x.y);
    }
    blk[q * OB_LD + j] = v;
  }
  __syncthreads();
  double m = 0.0;
  for (int e = threadIdx.x; e < M * 16; e += blockDim.x) {
    const int p = e % M, jq = e / M;
    float2 c[4];
    onebody_apply4(Dt, blk, M, p, jq, c);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int j = jq + 16 * u;
      if (j >= jn) continue;
      const size_t o = ((size_t)w * 2 * N + sp * N + j0 + j) * NM + k * M + p;
      reinterpret_cast<float2*>(corr)[2 * o] = c[u];
      const float2 b = blk[p * OB_LD + j];
      const float2 v = make_float2(b.x + c[u].x, b.y + c[u].y);
      p32[o] = v;
      m = fmax(m, (double)fmaxf(fabsf(v.x), fabsf(v.y)));
    }
  }
  m = block_max(m, red);
  if (threadIdx.x == 0) atomic_max_pos(mx + w, m);
}

// Second half step: with corr.xy = d = phi'' - phi and corr.zw = phi'' (fp32) after the
// Taylor series, phi <- phi + d + D phi'' (the sum of fp32 corrections is added to the
// FP64 walker once).  grid (k, ws, j-chunk of 64).  STAGE_D: both parts of corr are staged in
// shared memory by one coalesced pass (rows j, orbitals contiguous), and the FP64 walker
// (orbital rows, columns j contiguous) is updated with sixteen consecutive threads on sixteen
// consecutive columns; without it (M too large for the second staging buffer) the threads
// run down the orbitals and read d from global memory.
template <bool STAGE_D>
__global__ void onebody_out_kernel(const float4* corr, const float2* dhalf, zc* phi, int nk, int M, int N, int NM) {
  const int k = blockIdx.x, ws = blockIdx.y, j0 = blockIdx.z * 64;
  const int w = ws >> 1, sp = ws & 1;
  const int jn = min(64, N - j0);
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* blk = reinterpret_cast<float2*>(smraw);          // [M][OB_LD] phi''
  float2* dd = blk + M * OB_LD;                                 // [M][OB_LD] d (STAGE_D)
  float2* Dt = dd + (STAGE_D ? M * OB_LD : 0);                  // [M][M]
  for (int e = threadIdx.x; e < M * M; e += blockDim.x) {
    const int p = e / M, q = e % M;
    Dt[q * M + p] = dhalf[(size_t)k * M * M + e];
  }
  const float4* src = corr + ((size_t)w * 2 * N + sp * N + j0) * NM + k * M;
  for (int e = threadIdx.x; e < M * 64; e += blockDim.x) {
    const int j = e / M, q = e % M;
    float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
    if (j < jn) x = src[(size_t)j * NM + q];
    blk[q * OB_LD + j] = make_float2(x.z, x.w);
    if (STAGE_D) dd[q * OB_LD + j] = make_float2(x.x, x.y);
  }
  __syncthreads();
  zc* dst = phi + (size_t)ws * NM * N;
  for (int e = threadIdx.x; e < M * 16; e += blockDim.x) {
    const int jq = STAGE_D ? e % 16 : e / M, p = STAGE_D ? e / 16 : e % M;
    float2 c[4];
    onebody_apply4(Dt, blk, M, p, jq, c);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int j = jq + 16 * u;
      if (j >= jn) continue;
      const float2 d = STAGE_D ? dd[p * OB_LD + j] : reinterpret_cast<const float2*>(src)[2 * ((size_t)j * NM + p)];
      zc v = dst[(size_t)(k * M + p) * N + j0 + j];
      v.x += (double)(d.x + c[u].x);
      v.y += (double)(d.y + c[u].y);
      dst[(size_t)(k * M + p) * N + j0 + j] = v;
    }
  }
}

// B[k] = A[k] (A[k]^dag A[k])^-1 by Gauss-Jordan on the Hermitian positive definite
// Gram matrix (no pivoting needed); one block per k; scratch [nk][n][2n].
__global__ void trial_projector_kernel(const zc* A, zc* B, zc* scratch, int M, int n) {
  const int k = blockIdx.x;
  const zc* Ak = A + (size_t)k * M * n;
  zc* aug = scratch + (size_t)k * n * 2 * n;  // [n][2n] = [Gram | I]
  for (int e = threadIdx.x; e < n * 2 * n; e += blockDim.x) {
    const int i = e / (2 * n), j = e % (2 * n);
    zc v = zzero();
    if (j < n) {
      for (int p = 0; p < M; ++p) v = zfma(zconj(Ak[p * n + i]), Ak[p * n + j], v);
    } else {
      v = zmake(i == j - n ? 1.0 : 0.0, 0.0);
    }
    aug[e] = v;
  }
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    const zc inv = zinv(aug[j * 2 * n + j]);
    __syncthreads();
    for (int c = threadIdx.x; c < 2 * n; c += blockDim.x) aug[j * 2 * n + c] = zmul(aug[j * 2 * n + c], inv);
    __syncthreads();
    for (int e = threadIdx.x; e < n * 2 * n; e += blockDim.x) {
      const int i = e / (2 * n), c = e % (2 * n);
      if (i != j) {
        const zc f = aug[i * 2 * n + j];
        aug[e] = zsub(aug[e], zmul(f, aug[j * 2 * n + c]));
      }
    }
    __syncthreads();
  }
  // B = A Ginv
  for (int e = threadIdx.x; e < M * n; e += blockDim.x) {
    const int p = e / n, a = e % n;
    zc v = zzero();
    for (int b = 0; b < n; ++b) v = zfma(Ak[p * n + b], aug[b * 2 * n + n + a], v);
    B[(size_t)k * M * n + e] = v;
  }
}

// phi [W][2][NM][N] (FP64) -> transposed split planes [W][4][2N][NMp] (rows = (spin, column)),
// per-walker scale; grid (W, chunks)
__global__ void split_T_kernel(const zc* phi, const unsigned long long* mx, float* scale, __half* out, int NM, int N,
                               int NMp) {
  // one 32 x 32 block (orbital rows r, columns j) of one walker-spin, transposed through
  // shared memory so that both the FP64 reads (along j) and the fp16 writes (along r)
  // are coalesced; grid (ceil(NM/32), ceil(N/32), 2W)
  __shared__ float2 t[32][33];
  const int r0 = blockIdx.x * 32, j0 = blockIdx.y * 32, w = blockIdx.z >> 1, sp = blockIdx.z & 1;
  const float s = scale_from_bits(mx + w);
  if (blockIdx.x == 0 && blockIdx.y == 0 && sp == 0 && threadIdx.x == 0) scale[w] = s;
  const zc* p = phi + ((size_t)w * 2 + sp) * NM * N;
  for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
    const int rr = e / 32, jj = e % 32, r = r0 + rr, j = j0 + jj;
    float2 v = make_float2(0.f, 0.f);
    if (r < NM && j < N) {
      const zc x = p[(size_t)r * N + j];
      v = make_float2((float)x.x * s, (float)x.y * s);
    }
    t[rr][jj] = v;
  }
  __syncthreads();
  const size_t ps = (size_t)2 * N * NMp;
  __half* o = out + (size_t)w * 4 * ps;
  for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
    const int jj = e / 32, rr = e % 32, r = r0 + rr, j = j0 + jj;
    if (r < NM && j < N) put4f(o, ps, ((size_t)sp * N + j) * NMp + r, t[rr][jj].x, t[rr][jj].y);
  }
}

// Gram = R^dag R (Cholesky, upper R in place) and X = R^-1, both in fp32 (the Gram
// comes from the split GEMM, about 22 bits, so FP64 would add nothing), then the split
// planes of X^T [WS][4][N][Np] with a per-ws scale.  One block per walker-spin, the
// matrix in shared memory when it fits (SMEM), else in place in global memory.
// R^-1 is formed by Gauss-Jordan elimination on the upper triangle: step j scales row j
// by 1/r_jj and clears column j from the rows above it, N^3/6 complex multiply-adds with
// every step fully parallel.  A Gram matrix that is not positive definite leaves X = I
// (the walker is kept) and is counted with the singular walkers.
constexpr int CI_THREADS = 512;
template <bool SMEM>
__global__ void __launch_bounds__(CI_THREADS) chol_inv_kernel(float2* gram, __half* out, float* scale, int* flags,
                                                              int N, int Np, double* logr) {
  extern __shared__ __align__(16) unsigned char ci_smem[];
  constexpr int NW = CI_THREADS / 32;
  __shared__ int s_fail;
  __shared__ float s_red[NW];
  const int ws = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float2* g = gram + (size_t)ws * N * N;
  float2* a = SMEM ? reinterpret_cast<float2*>(ci_smem) : g;
  float2* fcol = reinterpret_cast<float2*>(ci_smem + (SMEM ? (size_t)N * N * sizeof(float2) : 0));
  if (SMEM)
    for (int e = tid; e < N * N; e += CI_THREADS) a[e] = g[e];
  if (tid == 0) s_fail = 0;
  __syncthreads();
  // Cholesky, right-looking, upper triangle only
  for (int j = 0; j < N; ++j) {
    const float d = a[(size_t)j * N + j].x;
    if (!(d > 0.f) || !isfinite(d)) {   // the same value in every thread
      if (tid == 0) s_fail = 1;
      break;
    }
    const float r = sqrtf(d), ir = 1.f / r;
    __syncthreads();   // every thread has read a[j][j]
    for (int c = j + tid; c < N; c += CI_THREADS) {
      const float2 v = a[(size_t)j * N + c];
      a[(size_t)j * N + c] = (c == j) ? make_float2(r, 0.f) : make_float2(v.x * ir, v.y * ir);
    }
    __syncthreads();
    for (int i = j + 1 + warp; i < N; i += NW) {
      const float2 u = a[(size_t)j * N + i];   // conj(R[j][i]) R[j][c]
      for (int c = i + lane; c < N; c += 32) {
        const float2 v = a[(size_t)j * N + c];
        float2 t = a[(size_t)i * N + c];
        t.x -= u.x * v.x + u.y * v.y;
        t.y -= u.x * v.y - u.y * v.x;
        a[(size_t)i * N + c] = t;
      }
    }
    __syncthreads();
  }
  __syncthreads();
  const int fail = s_fail;
  if (fail && tid == 0) atomicAdd(&flags[0], 1);
  if (logr) {
    // log det R = sum_j log r_jj (real, r_jj > 0): the change of log det (A^dag phi)
    // under phi <- phi R^-1; nothing on failure (the walker is kept as it is)
    double lr = 0.0;
    if (!fail)
      for (int j = tid; j < N; j += CI_THREADS) lr += log((double)a[(size_t)j * N + j].x);
    for (int o = 16; o > 0; o >>= 1) lr += __shfl_xor_sync(0xffffffffu, lr, o);
    __shared__ double s_lr[NW];
    if (lane == 0) s_lr[warp] = lr;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < NW; ++w) t += s_lr[w];
      logr[ws] += t;
    }
    __syncthreads();
  }
  if (!fail) {
    for (int j = 0; j < N; ++j) {
      const float inv = 1.f / a[(size_t)j * N + j].x;   // r_jj is real and positive
      for (int i = tid; i < j; i += CI_THREADS) fcol[i] = a[(size_t)i * N + j];
      __syncthreads();   // every thread has read r_jj and the multipliers
      for (int c = j + tid; c < N; c += CI_THREADS) {
        const float2 v = a[(size_t)j * N + c];
        a[(size_t)j * N + c] = (c == j) ? make_float2(inv, 0.f) : make_float2(v.x * inv, v.y * inv);
      }
      __syncthreads();
      for (int i = warp; i < j; i += NW) {
        const float2 f = fcol[i];
        for (int c = j + lane; c < N; c += 32) {
          if (c == j) {
            a[(size_t)i * N + c] = make_float2(-f.x * inv, -f.y * inv);
          } else {
            const float2 v = a[(size_t)j * N + c];
            float2 t = a[(size_t)i * N + c];
            t.x -= f.x * v.x - f.y * v.y;
            t.y -= f.x * v.y + f.y * v.x;
            a[(size_t)i * N + c] = t;
          }
        }
      }
      __syncthreads();
    }
  }
  // X[i][c] (upper triangle; identity on failure); out row jr, column i = X[i][jr]
  float m = 0.f;
  for (int e = tid; e < N * N; e += CI_THREADS) {
    const int i = e / N, c = e % N;
    if (fail) {
      if (i == c) m = 1.f;
    } else if (i <= c) {
      const float2 v = a[e];
      m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
    }
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) s_red[warp] = m;
  __syncthreads();
  m = 0.f;
  for (int w = 0; w < NW; ++w) m = fmaxf(m, s_red[w]);
  const float sc = pow2_scale((double)m);
  if (tid == 0) scale[ws] = sc;
  const size_t ps = (size_t)N * Np;
  __half* o = out + (size_t)ws * 4 * ps;
  for (int e = tid; e < N * N; e += CI_THREADS) {
    const int jr = e / N, i = e % N;
    float2 v = make_float2(0.f, 0.f);
    if (fail)
      v.x = (i == jr) ? 1.f : 0.f;
    else if (i <= jr)
      v = a[(size_t)i * N + jr];
    put4f(o, ps, (size_t)jr * Np + i, v.x * sc, v.y * sc);
  }
}

// ld[ws] -= (logr[ws], 0) for every walker-spin that is not singular
__global__ void ld_shift_kernel(zc* ld, const double* logr, const int* sing, int WS) {
  const int ws = blockIdx.x * blockDim.x + threadIdx.x;
  if (ws < WS && !sing[ws]) ld[ws].x -= logr[ws];
}

__global__ void to_f32_kernel(const zc* in, float2* out, size_t n) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    out[e] = make_float2((float)in[e].x, (float)in[e].y);
}
__global__ void recip_kernel(const float* in, float* out, size_t n) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    out[e] = 1.f / in[e];
}

// dhalf = Ehalf - I in fp32
__global__ void dhalf_kernel(const zc* Ehalf, float2* d, int nk, int M) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)nk * M * M;
       e += (size_t)gridDim.x * blockDim.x) {
    const int p = (int)((e / M) % M), q = (int)(e % M);
    d[e] = make_float2((float)(Ehalf[e].x - (p == q ? 1.0 : 0.0)), (float)Ehalf[e].y);
  }
}

// E1 and EC per walker from the fp32 Green's function and the FP64 X.
__global__ void e1_ec_mixed_kernel(const zc* AhH, const float2* g32, const zc* X, const int* minus, zc* eloc, int nk,
                                   int M, int n, int Mp, int G, int WS) {
  const int w = blockIdx.x;
  __shared__ zc red[32];
  zc s = zzero();
  for (int e = threadIdx.x; e < 2 * nk * n * M; e += blockDim.x) {
    const int q = e % M, a = (e / M) % n, k = (e / (M * n)) % nk, sp = e / (M * n * nk);
    const float2 g = g32[((((size_t)k * nk + k) * WS + 2 * w + sp) * n + a) * Mp + q];
    s = zfma(AhH[((size_t)k * n + a) * M + q], zmake(g.x, g.y), s);
  }
  const zc e1 = block_zsum(s, red);
  zc c = zzero();
  for (int e = threadIdx.x; e < nk * G; e += blockDim.x) {
    const int g = e % G, Q = e / G;
    c = zfma(X[((size_t)w * nk + Q) * G + g], X[((size_t)w * nk + minus[Q]) * G + g], c);
  }
  const zc ec = block_zsum(c, red);
  if (threadIdx.x == 0) {
    eloc[3 * w + 0] = e1;
    eloc[3 * w + 1] = zscale(ec, 0.5);
  }
}

// EX[w] = -1/2 sum_t weight_t sum_nt sum_s xpart[t][nt][2w+s]
// Two passes in a fixed order (deterministic): part[c][ws] = sum over the c-th chunk of the
// (t, nt) rows of weight_t xpart[t][nt][ws], rows read whole (coalesced), four rows' loads in
// flight at a time; then per walker EX[w] = -1/2 sum_c (part[c][2w] + part[c][2w+1]) with a
// fixed-order tree over the chunks.
constexpr int EX_CHUNKS = 608;
__global__ void ex_partial_kernel(const double2* xpart, const int4* tri, double2* part, int T, int nt_n, int WS) {
  const int rows = T * nt_n, per = (rows + gridDim.x - 1) / gridDim.x;
  const int e0 = blockIdx.x * per, e1 = min(rows, e0 + per);
  for (int ws = threadIdx.x; ws < WS; ws += blockDim.x) {
    double2 s = make_double2(0.0, 0.0);
    for (int e = e0; e < e1; e += 4) {
      double2 v[4];
      double wt[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const bool in = e + u < e1;
        v[u] = in ? xpart[(size_t)(e + u) * WS + ws] : make_double2(0.0, 0.0);
        wt[u] = in ? (double)tri[(e + u) / nt_n].w : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        s.x += wt[u] * v[u].x;
        s.y += wt[u] * v[u].y;
      }
    }
    part[(size_t)blockIdx.x * WS + ws] = s;
  }
}
__global__ void ex_reduce_mixed_kernel(const double2* part, zc* eloc, int chunks, int WS) {
  const int w = blockIdx.x;
  __shared__ zc red[32];
  zc s = zzero();
  for (int c = threadIdx.x; c < chunks; c += blockDim.x) {
    const double2 a = part[(size_t)c * WS + 2 * w], b = part[(size_t)c * WS + 2 * w + 1];
    s = zadd(s, zmake(a.x + b.x, a.y + b.y));
  }
  s = block_zsum(s, red);
  if (threadIdx.x == 0) eloc[3 * w + 2] = zscale(s, -0.5);
}

// ---------------------------------------------------------------------------
// create-time kernels
// ---------------------------------------------------------------------------

// s_lh[Q][g] from max over k, a, r of |LH|; s_l[Q][g] from max over k, p, r of |L|
__global__ void static_scales_kernel(const zc* L, const zc* LH, float* s_l, float* s_lh, int nk, int G, int M, int n) {
  const int Q = blockIdx.x, g = blockIdx.y;
  __shared__ double red[32];
  double ml = 0.0, mh = 0.0;
  for (int k = 0; k < nk; ++k) {
    const zc* lp = L + (((size_t)Q * nk + k) * G + g) * M * M;
    for (int e = threadIdx.x; e < M * M; e += blockDim.x) ml = fmax(ml, cabs_d(lp[e]));
    const zc* hp = LH + (((size_t)Q * nk + k) * G + g) * n * M;
    for (int e = threadIdx.x; e < n * M; e += blockDim.x) mh = fmax(mh, cabs_d(hp[e]));
  }
  ml = block_max(ml, red);
  mh = block_max(mh, red);
  if (threadIdx.x == 0) {
    s_l[Q * G + g] = pow2_scale(ml);
    s_lh[Q * G + g] = pow2_scale(mh);
  }
}

// lh_sp[4][Q][k][g][a][Mp] and lt_sp[4][Q][k][(p,r)][Gp]; grid (Q*nk + k)
__global__ void static_split_kernel(const zc* L, const zc* LH, const float* s_l, const float* s_lh, __half* lh_sp,
                                    __half* lt_sp, int nk, int G, int Gp, int M, int Mp, int n) {
  const int b = blockIdx.x, Q = b / nk;
  const size_t lh_ps = (size_t)nk * nk * G * n * Mp, lt_ps = (size_t)nk * nk * M * M * Gp;
  const zc* hp = LH + (size_t)b * G * n * M;
  for (int e = threadIdx.x; e < G * n * M; e += blockDim.x) {
    const int g = e / (n * M), a = (e / M) % n, r = e % M;
    put4d(lh_sp, lh_ps, (((size_t)b * G + g) * n + a) * Mp + r, hp[e].x, hp[e].y, s_lh[Q * G + g]);
  }
  const zc* lp = L + (size_t)b * G * M * M;
  for (int e = threadIdx.x; e < G * M * M; e += blockDim.x) {
    const int pr = e / G, g = e % G;  // g fastest in the output
    const zc v = lp[(size_t)g * M * M + pr];
    put4d(lt_sp, lt_ps, ((size_t)b * M * M + pr) * Gp + g, v.x, v.y, s_l[Q * G + g]);
  }
}

// Z_t[(a,s)][(b,r)] = sum_g LH[Q,k,g,a,r] LH[-Q,kx,g,b,s] in FP64, split per triple.
__global__ void z_build_kernel(const zc* LH, const int4* tri, const int* minus, zc* scratch, __half* z_sp,
                               float* s_z, int T, int rows, int nk, int G, int M, int n, int Mp) {
  const int nM = n * M;
  const size_t per = (size_t)nM * nM;
  zc* buf = scratch + (size_t)blockIdx.x * per;
  __shared__ double red[32];
  const int nMp = n * Mp;
  const size_t ps = (size_t)rows * nMp * nMp;   // plane stride: z_sp holds `rows` matrices per plane
  for (int t = blockIdx.x; t < T; t += gridDim.x) {
    const int4 q = tri[t];
    const zc* L1 = LH + ((size_t)q.x * nk + q.y) * G * nM;            // LH[Q][k]
    const zc* L2 = LH + ((size_t)minus[q.x] * nk + q.z) * G * nM;     // LH[-Q][kx]
    double m = 0.0;
    for (size_t e = threadIdx.x; e < per; e += blockDim.x) {
      // e = ((a*M + s)*n + b)*M + r
      const int r = (int)(e % M), b = (int)((e / M) % n), s = (int)((e / ((size_t)M * n)) % M),
                a = (int)(e / ((size_t)M * n * M));
      zc acc = zzero();
      for (int g = 0; g < G; ++g)
        acc = zfma(L1[(size_t)g * nM + a * M + r], L2[(size_t)g * nM + b * M + s], acc);
      buf[e] = acc;
      m = fmax(m, cabs_d(acc));
    }
    m = block_max(m, red);
    const float sc = pow2_scale(m);
    if (threadIdx.x == 0) s_z[t] = sc;
    for (size_t e = threadIdx.x; e < per; e += blockDim.x) {
      const int r = (int)(e % M), b = (int)((e / M) % n), s = (int)((e / ((size_t)M * n)) % M),
                a = (int)(e / ((size_t)M * n * M));
      const size_t idx = ((size_t)t * nMp + a * Mp + s) * nMp + b * Mp + r;   // rows s >= M stay zero
      put4d(z_sp, ps, idx, buf[e].x, buf[e].y, sc);
    }
    __syncthreads();
  }
}

// The partners' rows of z_sp: row T + j holds the transpose of canonical row pmap[j].
__global__ void z_partner_kernel(__half* z_sp, float* s_z, const int* pmap, int T, int P, int rows, int nMp) {
  const size_t per = (size_t)nMp * nMp, ps = (size_t)rows * per;
  for (int j = blockIdx.x; j < P; j += gridDim.x) {
    const int i = pmap[j];
    if (threadIdx.x == 0) s_z[T + j] = s_z[i];
    for (int pl = 0; pl < 4; ++pl) {
      const __half* src = z_sp + pl * ps + (size_t)i * per;
      __half* dst = z_sp + pl * ps + (size_t)(T + j) * per;
      for (size_t e = threadIdx.x; e < per; e += blockDim.x) {
        const size_t row = e / nMp, col = e % nMp;
        dst[e] = src[col * nMp + row];
      }
    }
  }
}

// Gam[ws][(k1,a)][(k2,r)] of the adjoint, k2 = k1 - Q, in FP64 from
//   c2 sum_g X[w][-Q][g] LH[Q][k1][g][a][r]   (Coulomb; fp32 sum over g)
// + c1 AhH[k1][a][r] on the diagonal blocks  (one-body)
// - c3 gam32[k1][k2][ws][(a,r)]              (exchange, from the adjoint GEMM)
// with c = conj(grad_e) per walker.  Block (k1, Q, group of GA_W walkers).
constexpr int GA_W = 16;
__global__ void __launch_bounds__(128) gamma_assemble_kernel(const zc* LH, const zc* X, const zc* AhH,
                                                             const zc* grad_e, const float2* gam32, zc* Gam,
                                                             const int* kminus, const int* minus, int nk, int G,
                                                             int M, int n, int Mp, int W) {
  const int k1 = blockIdx.x, Q = blockIdx.y, w0 = blockIdx.z * GA_W;
  const int k2 = kminus[k1 * nk + Q], mQ = minus[Q];
  const int nw = min(GA_W, W - w0);
  const int nM = n * M, N = nk * n, NM = nk * M, WS = 2 * W, nMp = n * Mp;
  extern __shared__ float2 xs[];   // [GA_W][G]
  for (int e = threadIdx.x; e < GA_W * G; e += blockDim.x) {
    const int wi = e / G, g = e % G;
    const zc v = wi < nw ? X[((size_t)(w0 + wi) * nk + mQ) * G + g] : zzero();
    xs[e] = make_float2((float)v.x, (float)v.y);
  }
  __syncthreads();
  const zc* lh = LH + ((size_t)Q * nk + k1) * G * nM;
  for (int e = threadIdx.x; e < nM; e += blockDim.x) {
    float2 acc[GA_W];
#pragma unroll
    for (int i = 0; i < GA_W; ++i) acc[i] = make_float2(0.f, 0.f);
    for (int g = 0; g < G; ++g) {
      const zc l = lh[(size_t)g * nM + e];
      const float lr = (float)l.x, li = (float)l.y;
#pragma unroll
      for (int i = 0; i < GA_W; ++i) {
        const float2 x = xs[i * G + g];
        acc[i].x = fmaf(x.x, lr, fmaf(-x.y, li, acc[i].x));
        acc[i].y = fmaf(x.x, li, fmaf(x.y, lr, acc[i].y));
      }
    }
    const int a = e / M, r = e % M;
#pragma unroll
    for (int i = 0; i < GA_W; ++i) {
      if (i >= nw) break;
      const int w = w0 + i;
      const zc c1 = zconj(grad_e[3 * w + 0]), c2 = zconj(grad_e[3 * w + 1]), c3 = zconj(grad_e[3 * w + 2]);
      zc base = zmul(c2, zmake((double)acc[i].x, (double)acc[i].y));
      if (Q == 0) base = zfma(c1, AhH[(size_t)k1 * nM + e], base);
      for (int sp = 0; sp < 2; ++sp) {
        const int ws = 2 * w + sp;
        const float2 gx = gam32[(((size_t)k1 * nk + k2) * WS + ws) * nMp + a * Mp + r];
        Gam[((size_t)ws * N + k1 * n + a) * NM + k2 * M + r] = zsub(base, zmul(c3, zmake(gx.x, gx.y)));
      }
    }
  }
}

// ---------------------------------------------------------------------------
// host orchestration
// ---------------------------------------------------------------------------
#define MTRY(x)                         \
  do {                                  \
    cudaError_t e_ = (x);               \
    if (e_ != cudaSuccess) return e_;   \
  } while (0)

// Each policy's index in the handle's ring-depth table (AFQMC_GEMM_* of the header).
template <class P> struct GemmIdOf;
template <> struct GemmIdOf<GreenP> { static constexpr int value = AFQMC_GEMM_GREEN; };
template <> struct GemmIdOf<ForceBiasP> { static constexpr int value = AFQMC_GEMM_FORCE_BIAS; };
template <> struct GemmIdOf<VhsP> { static constexpr int value = AFQMC_GEMM_VHS; };
template <> struct GemmIdOf<TaylorP> { static constexpr int value = AFQMC_GEMM_TAYLOR; };
template <> struct GemmIdOf<ExchangeP> { static constexpr int value = AFQMC_GEMM_EXCHANGE; };
template <> struct GemmIdOf<AdjointP> { static constexpr int value = AFQMC_GEMM_ADJOINT; };
template <> struct GemmIdOf<GramP> { static constexpr int value = AFQMC_GEMM_GRAM; };
template <> struct GemmIdOf<ApplyRP> { static constexpr int value = AFQMC_GEMM_APPLY_R; };

// Launch with the handle's ring depth for this GEMM (the policy's default until tuned).  The
// depth changes only how far the TMA runs ahead: every tile's arithmetic is the same.
template <class P>
static cudaError_t run_gemm(afqmc_kp* h, const CUtensorMap& a, const CUtensorMap& b, const P& p, int* err,
                            cudaStream_t st) {
  const int r = h->mixed->ring[GemmIdOf<P>::value];
  const int depth = r ? r : P::kStages;
  return depth == 2 ? tcg::launch_precise<2>(a, b, p, err, st) : tcg::launch_precise<3>(a, b, p, err, st);
}

// The parameters of each step GEMM as the step launches it.
static GreenP green_params(const afqmc_kp* h) {
  const MixedState* m = h->mixed;
  GreenP p;
  p.mt_n = cdiv(h->N, 128);
  p.nt_n = cdiv(h->NM, BN);
  p.tiles = m->WS * p.mt_n * p.nt_n;
  p.kchunks = m->Np / 32;
  p.N = h->N; p.NM = h->NM; p.n = h->n; p.M = h->M; p.Mp = m->Mp; p.nk = h->nk; p.WS = m->WS;
  p.s_sinv = m->s_sinv; p.s_phi = m->s_phi; p.bproj32 = m->bproj32; p.g32 = m->g32;
  return p;
}
static ForceBiasP force_bias_params(const afqmc_kp* h) {
  const MixedState* m = h->mixed;
  ForceBiasP p;
  p.mt_n = cdiv(h->G, 128);
  p.nt_n = cdiv(h->W, BN);
  p.ng = m->fb_groups;
  p.kg = h->nk / p.ng;
  p.kcb = m->nMp / 32;
  p.tiles = h->nk * p.ng * p.mt_n * p.nt_n;
  p.kchunks = p.kg * p.kcb;
  p.W = h->W; p.G = h->G; p.nk = h->nk;
  p.kminus = h->kminus; p.s_gsum = m->s_gsum; p.inv_s_lh = m->inv_s_lh; p.Xk = m->xk;
  return p;
}
static VhsP vhs_params(const afqmc_kp* h) {
  const MixedState* m = h->mixed;
  VhsP p;
  p.mt_n = cdiv(h->M * h->M, 128);
  p.nt_n = cdiv(h->W, BN);
  p.tiles = h->nk * h->nk * p.mt_n * p.nt_n;
  p.kchunks = m->Gp / 32;
  p.W = h->W; p.M = h->M; p.nk = h->nk; p.NM = h->NM; p.NMp = m->NMp;
  p.kminus = h->kminus; p.s_y = m->s_y; p.v_sp = m->v_sp; p.overflow = h->flags + 2;
  return p;
}
// Taylor term j of the Horner series, writing the next iterate into t_sp[nxt]
static TaylorP taylor_params(const afqmc_kp* h, int j, int nxt) {
  const MixedState* m = h->mixed;
  const int R = 2 * h->N;
  TaylorP p;
  p.mt_n = cdiv(R, 128);
  p.nt_n = cdiv(h->NM, BN);
  p.tiles = h->W * p.mt_n * p.nt_n;
  p.kchunks = m->NMp / 32;
  p.R = R; p.NM = h->NM; p.NMp = m->NMp;
  p.inv_j = 1.f / (float)j;
  p.last = (j == 1);
  p.s_t = m->s_t; p.p32 = m->p32; p.corr = reinterpret_cast<float4*>(m->acc); p.t_next = m->t_sp[nxt];
  return p;
}
// The same term in the CTA-pair form: mt_n counts pairs of 128-row tiles.
static TaylorP taylor_params_pair(const afqmc_kp* h, int j, int nxt) {
  TaylorP p = taylor_params(h, j, nxt);
  p.mt_n = cdiv(p.mt_n, 2);
  p.tiles = h->W * p.mt_n * p.nt_n;
  return p;
}
// One Taylor-term GEMM in the form chosen at create.
static cudaError_t taylor_gemm(afqmc_kp* h, int j, int cur, int nxt, cudaStream_t st);
static ExchangeP exchange_params(const afqmc_kp* h) {
  const MixedState* m = h->mixed;
  ExchangeP p;
  p.mt_n = cdiv(m->WS, 128);
  p.nt_n = cdiv(m->nMp, BN);
  p.tiles = m->T * p.mt_n * p.nt_n;
  p.kchunks = m->nMp / 32;
  p.WS = m->WS; p.nk = h->nk; p.nMp = m->nMp;
  p.kminus = h->kminus; p.minus = h->minus; p.tri = m->tri; p.s_g = m->s_g; p.s_z = m->s_z; p.g32 = m->g32;
  p.xpart = m->xpart;
  return p;
}
static AdjointP adjoint_params(const afqmc_kp* h) {
  const MixedState* m = h->mixed;
  AdjointP p;
  p.kcb = cdiv(m->nMp, 32);
  p.kchunks = h->nk * p.kcb;
  p.mt_n = cdiv(m->WS, 128);
  p.nt_n = cdiv(m->nMp, BN);
  p.tiles = h->nk * h->nk * p.mt_n * p.nt_n;
  p.WS = m->WS; p.nk = h->nk; p.nMp = m->nMp;
  p.kminus = h->kminus; p.s_g = m->s_g; p.zrow = m->zrow; p.s_z = m->s_z; p.gam32 = m->gam32;
  return p;
}

// Autotuner: time one GEMM with a two- and a three-stage TMA ring on the handle's own
// operands (three launches each after a warm-up, CUDA events on the create stream) and keep
// the faster; the policy's default stays unless the other is faster by more than 2%.
// The operands hold whatever create left in the workspace: the timing does not depend on
// the values, and every buffer written here is scratch that the next call overwrites.
template <class P>
static cudaError_t tune_gemm(afqmc_kp* h, const CUtensorMap& a, const CUtensorMap& b, const P& p, cudaStream_t st,
                             cudaEvent_t e0, cudaEvent_t e1) {
  MixedState* m = h->mixed;
  const int id = GemmIdOf<P>::value;
  float t[2] = {0.f, 0.f};
  for (int v = 0; v < 2; ++v) {
    m->ring[id] = 2 + v;
    MTRY(run_gemm(h, a, b, p, h->flags + 1, st));
    MTRY(cudaEventRecord(e0, st));
    for (int r = 0; r < 3; ++r) MTRY(run_gemm(h, a, b, p, h->flags + 1, st));
    MTRY(cudaEventRecord(e1, st));
    MTRY(cudaEventSynchronize(e1));
    MTRY(cudaEventElapsedTime(&t[v], e0, e1));
    t[v] /= 3.f;
  }
  m->tune_ms[id][0] = t[0];
  m->tune_ms[id][1] = t[1];
  const int def = P::kStages, other = 5 - def;
  m->ring[id] = t[other - 2] < 0.98f * t[def - 2] ? other : def;
  return cudaSuccess;
}

static cudaError_t autotune(afqmc_kp* h, cudaStream_t st) {
  MixedState* m = h->mixed;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = tune_gemm(h, m->m_sinvt, m->m_phi, green_params(h), st, e0, e1);
  if (e == cudaSuccess) e = tune_gemm(h, m->m_lh, m->m_gsum, force_bias_params(h), st, e0, e1);
  if (e == cudaSuccess) e = tune_gemm(h, m->m_lt, m->m_y, vhs_params(h), st, e0, e1);
  if (e == cudaSuccess) e = tune_gemm(h, m->m_t[0], m->m_v, taylor_params(h, 2, 1), st, e0, e1);
  if (e == cudaSuccess && taylor_params(h, 2, 1).mt_n > 1) {
    // the CTA-pair form (four stages): kept when faster than the single form at its tuned ring
    // depth by more than 2%
    // (a launch the device refuses, e.g. a cluster it cannot place, leaves the single form)
    float t = 0.f;
    m->taylor_pair = 1;
    cudaError_t ep = taylor_gemm(h, 2, 0, 1, st);
    if (ep == cudaSuccess) ep = cudaEventRecord(e0, st);
    for (int r = 0; r < 3 && ep == cudaSuccess; ++r) ep = taylor_gemm(h, 2, 0, 1, st);
    if (ep == cudaSuccess) ep = cudaEventRecord(e1, st);
    if (ep == cudaSuccess) ep = cudaEventSynchronize(e1);
    if (ep == cudaSuccess) ep = cudaEventElapsedTime(&t, e0, e1);
    const int id = AFQMC_GEMM_TAYLOR;
    m->taylor_pair_ms = ep == cudaSuccess ? t / 3.f : -1.f;
    m->taylor_pair = (ep == cudaSuccess && t / 3.f < 0.98f * m->tune_ms[id][m->ring[id] - 2]) ? 1 : 0;
    if (ep == cudaErrorInvalidConfiguration || ep == cudaErrorLaunchOutOfResources ||
        ep == cudaErrorInvalidValue || ep == cudaErrorNotSupported)
      (void)cudaGetLastError();   // a refused launch: not sticky
    else
      e = ep;
  }
  if (e == cudaSuccess) e = tune_gemm(h, m->m_g, m->m_z, exchange_params(h), st, e0, e1);
  if (e == cudaSuccess) e = tune_gemm(h, m->m_g, m->m_zall, adjoint_params(h), st, e0, e1);
  // the QR GEMMs write the caller's walkers: they keep their defaults
  if (e == cudaSuccess) e = cudaMemsetAsync(h->flags, 0, sizeof(int) * 4, st);   // scratch-data flags
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return e;
}

static cudaError_t set_smem_attr(const void* fn, size_t bytes) { return ensure_dyn_smem(fn, bytes); }

static size_t onebody_smem(const afqmc_kp* h) {
  return sizeof(float2) * h->M * h->M + sizeof(float2) * h->M * OB_LD;
}
// the second half step with d staged too, where it fits
static size_t onebody_out_smem(const afqmc_kp* h) { return onebody_smem(h) + sizeof(float2) * h->M * OB_LD; }
static bool onebody_out_staged(const afqmc_kp* h) { return onebody_out_smem(h) <= 220 * 1024; }

// Free the handle's FP64 Cholesky vectors (the largest static array: Nk^2 G M^2 complex128)
// once the split operands exist.  Called with no work of the handle in flight.
static cudaError_t release_fp64_cholesky(afqmc_kp* h) {
  if (!h->L) return cudaSuccess;
  for (size_t i = 0; i < h->allocs.size(); ++i) {
    if (h->allocs[i] != static_cast<void*>(h->L)) continue;
    const size_t b = std::max<size_t>((size_t)h->nk * h->nk * h->G * h->M * h->M * sizeof(zc), 16);
    cudaError_t e = cudaFree(h->L);
    if (e != cudaSuccess) return e;
    h->allocs.erase(h->allocs.begin() + i);
    h->bytes -= b;
    h->L = nullptr;
    return cudaSuccess;
  }
  return cudaSuccess;
}

static cudaError_t create_impl(afqmc_kp* h, cudaStream_t st) {
  MixedState* m = h->mixed;
  const int nk = h->nk, M = h->M, n = h->n, G = h->G, W = h->W, N = h->N, NM = h->NM;
  m->Np = rup(N, 32);
  m->NMp = rup(NM, 32);
  m->Mp = rup(M, 32);
  m->Gp = rup(G, 32);
  m->nMp = n * m->Mp;
  m->nM = n * M;
  m->WS = 2 * W;
  const int Np = m->Np, NMp = m->NMp, Mp = m->Mp, Gp = m->Gp, nMp = m->nMp, nM = m->nM, WS = m->WS;
  // canonical triples (Q, k, kx) <-> (-Q, kx, k)
  std::vector<int4> tri;
  for (int Q = 0; Q < nk; ++Q)
    for (int k = 0; k < nk; ++k)
      for (int kx = 0; kx < nk; ++kx) {
        const int mQ = h->h_minus[Q];
        const bool self = (mQ == Q) && (kx == k);
        const bool canon = (Q < mQ) || (Q == mQ && k <= kx);
        if (canon) tri.push_back(make_int4(Q, k, kx, self ? 1 : 2));
      }
  // Order of the triples.  A triple reads two Green's-function blocks: (k - Q, kx), its
  // GEMM's A operand, and (k, kx + Q), the partner its epilogue contracts with.  Both lie on
  // the block diagonal d = k - Q - kx, so the triples are grouped by d first (the blocks a
  // group touches, 2 Nk of them, stay in L2 while the group runs) and by the A block next
  // (the triples sharing it run on neighbouring CTAs at the same time).
  std::stable_sort(tri.begin(), tri.end(), [&](const int4& a, const int4& b) {
    const int ka = h->h_kminus[(size_t)a.y * nk + a.x], kb = h->h_kminus[(size_t)b.y * nk + b.x];
    const int da = h->h_kminus[(size_t)ka * nk + a.z], db = h->h_kminus[(size_t)kb * nk + b.z];
    if (da != db) return da < db;
    return ka != kb ? ka < kb : a.z < b.z;
  });
  m->T = (int)tri.size();
  const int T = m->T;
  const int ntx = cdiv(nMp, BN);
  const int Tf = nk * nk * nk;
  // rows of the Z array: canonical triple i at row i; the partner (-Q, kx, k) of a triple
  // that is not its own partner at row T + j, j counting those triples in order
  std::vector<int> zrow_h((size_t)Tf, -1), pmap_h;
  for (int i = 0; i < T; ++i) {
    const int4 q = tri[i];
    zrow_h[((size_t)q.x * nk + q.y) * nk + q.z] = i;
    if (q.w == 2) {
      zrow_h[((size_t)h->h_minus[q.x] * nk + q.z) * nk + q.y] = T + (int)pmap_h.size();
      pmap_h.push_back(i);
    }
  }
  const int P = (int)pmap_h.size();
  if (T + P != Tf) return cudaErrorInvalidValue;
  for (int v : zrow_h)
    if (v < 0) return cudaErrorInvalidValue;   // every triple has a canonical member

  // 1. the split Cholesky operands, then the FP64 vectors are released: a mixed handle never
  //    reads them again (the half-rotated FP64 copy stays for the Z build and the adjoint)
  MTRY(dalloc(h, &m->lh_sp, (size_t)4 * nk * nk * G * nMp, true, st));
  MTRY(dalloc(h, &m->s_lh, (size_t)nk * G, true, st));
  MTRY(dalloc(h, &m->lt_sp, (size_t)4 * nk * nk * M * M * Gp, true, st));
  MTRY(dalloc(h, &m->s_l, (size_t)nk * G, true, st));
  MTRY(dalloc(h, &m->inv_s_lh, (size_t)nk * G, true, st));
  static_scales_kernel<<<dim3(nk, G), 256, 0, st>>>(h->L, h->LH, m->s_l, m->s_lh, nk, G, M, n);
  AFQMC_LAUNCHED(h);
  recip_kernel<<<64, 256, 0, st>>>(m->s_lh, m->inv_s_lh, (size_t)nk * G);
  AFQMC_LAUNCHED(h);
  static_split_kernel<<<nk * nk, 256, 0, st>>>(h->L, h->LH, m->s_l, m->s_lh, m->lh_sp, m->lt_sp, nk, G, Gp, M, Mp,
                                               n);
  AFQMC_LAUNCHED(h);
  MTRY(cudaGetLastError());
  MTRY(cudaStreamSynchronize(st));
  MTRY(release_fp64_cholesky(h));

  // 2. the precontracted exchange tensor of every triple
  MTRY(dalloc(h, &m->z_sp, (size_t)4 * Tf * nMp * nMp, true, st));
  MTRY(dalloc(h, &m->s_z, Tf, true, st));
  MTRY(dalloc(h, &m->tri, T, false, st));
  MTRY(dalloc(h, &m->zrow, Tf, false, st));
  int* pmap = nullptr;
  MTRY(dalloc(h, &pmap, std::max(P, 1), false, st));
  const int zctas = std::min(T, ZCTAS);
  MTRY(dalloc(h, &m->zscratch, std::max((size_t)zctas * nM * nM, (size_t)nk * n * 2 * n), false, st));
  MTRY(cudaMemcpyAsync(m->tri, tri.data(), sizeof(int4) * T, cudaMemcpyHostToDevice, st));
  MTRY(cudaMemcpyAsync(m->zrow, zrow_h.data(), sizeof(int) * Tf, cudaMemcpyHostToDevice, st));
  if (P) MTRY(cudaMemcpyAsync(pmap, pmap_h.data(), sizeof(int) * P, cudaMemcpyHostToDevice, st));
  z_build_kernel<<<zctas, 256, 0, st>>>(h->LH, m->tri, h->minus, m->zscratch, m->z_sp, m->s_z, T, Tf, nk, G, M, n,
                                        Mp);
  AFQMC_LAUNCHED(h);
  if (P) {
    z_partner_kernel<<<std::min(P, 4096), 256, 0, st>>>(m->z_sp, m->s_z, pmap, T, P, Tf, nMp);
    AFQMC_LAUNCHED(h);
  }
  MTRY(cudaGetLastError());
  MTRY(cudaStreamSynchronize(st));   // the host tables above are temporaries

  // 3. per-step workspace
  MTRY(dalloc(h, &m->phi_sp, (size_t)WS * 4 * NM * Np, true, st));
  MTRY(dalloc(h, &m->s_phi, WS, true, st));
  MTRY(dalloc(h, &m->sinvt_sp, (size_t)WS * 4 * N * Np, true, st));
  MTRY(dalloc(h, &m->s_sinv, WS, true, st));
  MTRY(dalloc(h, &m->g32, (size_t)nk * nk * WS * nMp, true, st));
  MTRY(dalloc(h, &m->g_sp, (size_t)4 * nk * nk * WS * nMp, true, st));
  MTRY(dalloc(h, &m->s_g, WS, true, st));
  MTRY(dalloc(h, &m->gsum_sp, (size_t)4 * nk * nk * W * nMp, true, st));
  MTRY(dalloc(h, &m->s_gsum, W, true, st));
  MTRY(dalloc(h, &m->y_sp, (size_t)4 * nk * W * Gp, true, st));
  MTRY(dalloc(h, &m->s_y, (size_t)nk * W, true, st));
  MTRY(dalloc(h, &m->v_sp, (size_t)W * 4 * NM * NMp, true, st));
  MTRY(dalloc(h, &m->t_sp[0], (size_t)W * 4 * 2 * N * NMp, true, st));
  MTRY(dalloc(h, &m->t_sp[1], (size_t)W * 4 * 2 * N * NMp, true, st));
  MTRY(dalloc(h, &m->s_t, W, true, st));
  MTRY(dalloc(h, &m->acc, (size_t)W * 2 * N * NM, true, st));
  MTRY(dalloc(h, &m->p32, (size_t)W * 2 * N * NM, true, st));
  MTRY(dalloc(h, &m->xpart, (size_t)T * ntx * WS, true, st));
  // force-bias GEMM: the fewest groups of k blocks (a divisor of Nk) that give every SM a tile
  {
    int dev = 0, sms = 0;
    MTRY(cudaGetDevice(&dev));
    MTRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int per_group = nk * cdiv(G, 128) * cdiv(W, BN);
    m->fb_groups = nk;
    for (int d = 1; d <= nk; ++d)
      if (nk % d == 0 && per_group * d >= sms) {
        m->fb_groups = d;
        break;
      }
  }
  MTRY(dalloc(h, &m->xk, (size_t)m->fb_groups * W * nk * G, true, st));
  MTRY(dalloc(h, &m->mx, (size_t)2 * WS + 3 * W + W, true, st));
  MTRY(dalloc(h, &m->gam32, (size_t)nk * nk * WS * nMp, true, st));
  MTRY(dalloc(h, &m->dhalf, (size_t)nk * M * M, true, st));
  MTRY(dalloc(h, &m->bproj, (size_t)nk * M * n, true, st));
  MTRY(dalloc(h, &m->bproj32, (size_t)nk * M * n, true, st));
  MTRY(dalloc(h, &m->s_ff, (size_t)WS * h->N * h->N, false, st));
  MTRY(dalloc(h, &m->logr, (size_t)WS, true, st));
  MTRY(dalloc(h, &m->expart, (size_t)EX_CHUNKS * WS, true, st));

  // trial projector B = A (A^dag A)^-1 (scratch: the Z build's buffer, free again in stream order)
  trial_projector_kernel<<<nk, 256, 0, st>>>(h->A, m->bproj, m->zscratch, M, n);
  AFQMC_LAUNCHED(h);
  to_f32_kernel<<<64, 256, 0, st>>>(m->bproj, m->bproj32, (size_t)nk * M * n);
  AFQMC_LAUNCHED(h);
  MTRY(cudaGetLastError());
  MTRY(set_one_body(h, st));

  // tensor maps
  MTRY(map5(&m->m_sinvt, m->sinvt_sp, {(uint64_t)Np, (uint64_t)N, 4, (uint64_t)WS, 1},
            {(uint64_t)Np, (uint64_t)N * Np, (uint64_t)4 * N * Np, (uint64_t)WS * 4 * N * Np}, 128));
  MTRY(map5_pair(&m->m_phi, m->phi_sp, (uint64_t)Np, (uint64_t)NM, (uint64_t)WS, (uint64_t)Np, (uint64_t)NM * Np,
                 (uint64_t)4 * NM * Np, BN));
  // blocks (k1, k2) of gsum addressed by the one index k1 Nk + k2 (stride W nMp)
  MTRY(map5_pair(&m->m_gsum, m->gsum_sp, (uint64_t)nMp, (uint64_t)W, (uint64_t)nk * nk, (uint64_t)nMp,
                 (uint64_t)nk * nk * W * nMp, (uint64_t)W * nMp, BN));
  MTRY(map5(&m->m_lh, m->lh_sp, {(uint64_t)nMp, (uint64_t)G, 4, (uint64_t)nk, (uint64_t)nk},
            {(uint64_t)nMp, (uint64_t)nk * nk * G * nMp, (uint64_t)G * nMp, (uint64_t)nk * G * nMp}, 128));
  MTRY(map5_pair(&m->m_y, m->y_sp, (uint64_t)Gp, (uint64_t)W, (uint64_t)nk, (uint64_t)Gp, (uint64_t)nk * W * Gp,
                 (uint64_t)W * Gp, BN));
  MTRY(map5(&m->m_lt, m->lt_sp, {(uint64_t)Gp, (uint64_t)M * M, 4, (uint64_t)nk, (uint64_t)nk},
            {(uint64_t)Gp, (uint64_t)nk * nk * M * M * Gp, (uint64_t)M * M * Gp, (uint64_t)nk * M * M * Gp}, 128));
  for (int i = 0; i < 2; ++i)
    MTRY(map5(&m->m_t[i], m->t_sp[i], {(uint64_t)NMp, (uint64_t)2 * N, 4, (uint64_t)W, 1},
              {(uint64_t)NMp, (uint64_t)2 * N * NMp, (uint64_t)4 * 2 * N * NMp, (uint64_t)W * 4 * 2 * N * NMp}, 128));
  MTRY(map5_pair(&m->m_v, m->v_sp, (uint64_t)NMp, (uint64_t)NM, (uint64_t)W, (uint64_t)NMp, (uint64_t)NM * NMp,
                 (uint64_t)4 * NM * NMp, BN));
  MTRY(map5_pair(&m->m_vp, m->v_sp, (uint64_t)NMp, (uint64_t)NM, (uint64_t)W, (uint64_t)NMp, (uint64_t)NM * NMp,
                 (uint64_t)4 * NM * NMp, BN, 1));
  MTRY(map5(&m->m_g, m->g_sp, {(uint64_t)nMp, (uint64_t)WS, 4, (uint64_t)nk, (uint64_t)nk},
            {(uint64_t)nMp, (uint64_t)nk * nk * WS * nMp, (uint64_t)WS * nMp, (uint64_t)nk * WS * nMp}, 128));
  // the exchange reads the canonical rows, the adjoint every row
  MTRY(map5_pair(&m->m_z, m->z_sp, (uint64_t)nMp, (uint64_t)nMp, (uint64_t)T, (uint64_t)nMp,
                 (uint64_t)Tf * nMp * nMp, (uint64_t)nMp * nMp, BN));
  MTRY(map5_pair(&m->m_zall, m->z_sp, (uint64_t)nMp, (uint64_t)nMp, (uint64_t)Tf, (uint64_t)nMp,
                 (uint64_t)Tf * nMp * nMp, (uint64_t)nMp * nMp, BN));
  MTRY(map5(&m->m_phi_a, m->phi_sp, {(uint64_t)Np, (uint64_t)NM, 4, (uint64_t)WS, 1},
            {(uint64_t)Np, (uint64_t)NM * Np, (uint64_t)4 * NM * Np, (uint64_t)WS * 4 * NM * Np}, 128));
  MTRY(map5_pair(&m->m_sinvt_b, m->sinvt_sp, (uint64_t)Np, (uint64_t)N, (uint64_t)WS, (uint64_t)Np, (uint64_t)N * Np,
                 (uint64_t)4 * N * Np, BN));
  MTRY(map5_pair(&m->m_t0_b, m->t_sp[0], (uint64_t)NMp, (uint64_t)2 * N, (uint64_t)W, (uint64_t)NMp,
                 (uint64_t)2 * N * NMp, (uint64_t)4 * 2 * N * NMp, BN));
  MTRY(set_smem_attr((const void*)gamma_assemble_kernel, sizeof(float2) * GA_W * G));
  MTRY(set_smem_attr((const void*)onebody_in_kernel, onebody_smem(h)));
  if (onebody_out_staged(h))
    MTRY(set_smem_attr((const void*)onebody_out_kernel<true>, onebody_out_smem(h)));
  else
    MTRY(set_smem_attr((const void*)onebody_out_kernel<false>, onebody_smem(h)));
  return autotune(h, st);
}

void gemm_tuning(const afqmc_kp* h, int* depth, double* ms2, double* ms3) {
  const MixedState* m = h->mixed;
  const int defaults[AFQMC_NGEMMS] = {GreenP::kStages, ForceBiasP::kStages, VhsP::kStages, TaylorP::kStages,
                                      ExchangeP::kStages, AdjointP::kStages, GramP::kStages, ApplyRP::kStages};
  for (int i = 0; i < AFQMC_NGEMMS; ++i) {
    depth[i] = m->ring[i] ? m->ring[i] : defaults[i];
    ms2[i] = m->tune_ms[i][0];
    ms3[i] = m->tune_ms[i][1];
  }
}

void gemm_form(const afqmc_kp* h, int gemm, int* pair, double* ms_pair) {
  const MixedState* m = h->mixed;
  const bool t = gemm == AFQMC_GEMM_TAYLOR;
  *pair = t ? m->taylor_pair : 0;
  *ms_pair = t ? m->taylor_pair_ms : 0.0;
}
bool set_gemm_form(afqmc_kp* h, int gemm, int pair) {
  if (pair && (gemm != AFQMC_GEMM_TAYLOR || taylor_params(h, 2, 1).mt_n < 2)) return false;
  if (gemm == AFQMC_GEMM_TAYLOR) h->mixed->taylor_pair = pair;
  return true;
}

afqmc_status create(afqmc_kp* h, cudaStream_t st) {
  h->mixed = new (std::nothrow) MixedState();
  if (!h->mixed) return AFQMC_ERR_OOM;
  cudaError_t e = create_impl(h, st);
  if (e == cudaErrorMemoryAllocation) return AFQMC_ERR_OOM;
  if (e == cudaErrorNotSupported) return AFQMC_ERR_UNSUPPORTED;
  return e == cudaSuccess ? AFQMC_OK : AFQMC_ERR_CUDA;
}

void destroy(afqmc_kp* h) {
  if (!h->mixed) return;
  for (void* p : h->mixed->allocs) cudaFree(p);
  delete h->mixed;
  h->mixed = nullptr;
}

cudaError_t set_one_body(afqmc_kp* h, cudaStream_t st) {
  const size_t total = (size_t)h->nk * h->M * h->M;
  dhalf_kernel<<<(int)std::min<size_t>((total + 255) / 256, 4096), 256, 0, st>>>(h->Ehalf, h->mixed->dhalf, h->nk,
                                                                                  h->M);
  AFQMC_LAUNCHED(h);
  return cudaGetLastError();
}

constexpr int SPLIT_CHUNKS = 16;  // blocks per matrix in the split kernels

// overlap + LU + inverse (FP64), split operands, Gh GEMM, split Gh
// log det (A^dag phi) of every walker-spin, double-float (ffla.cu)
static cudaError_t overlap_logdet(afqmc_kp* h, const zc* phi, zc* ld, int* sing, cudaStream_t st) {
  MixedState* m = h->mixed;
  MTRY(ffla::overlap(h->A, phi, nullptr, m->s_ff, nullptr, nullptr, m->WS, h->nk, h->M, h->n, h->N, st));
  AFQMC_LAUNCHED(h);
  MTRY(ffla::invert(m->s_ff, m->WS, h->N, ld, sing, h->flags, nullptr, m->Np, nullptr, st));
  AFQMC_LAUNCHED(h);
  return cudaSuccess;
}

// The Green's function in three parts: the double-float overlap, inverse and log det and
// the split of phi_perp (green_pre); the tensor-core GEMM; its max and split (green_post).
static cudaError_t green_pre(afqmc_kp* h, const zc* phi, zc* ld, int* sing, cudaStream_t st) {
  MixedState* m = h->mixed;
  const int WS = m->WS;
  unsigned long long* mx_phi = m->mx;
  // phi (A^dag phi)^-1 = B + phi_perp S^-1 with B = A (A^dag A)^-1 and phi_perp = phi - B S:
  // the trial-subspace part is exact, so the split GEMM never forms the large
  // cancelling partial sums of S^-1 (A^dag phi) = I.
  float2* phi_perp = reinterpret_cast<float2*>(m->acc);  // free until the Taylor series
  // S = A^dag phi, phi_perp and S^-1 / log det in double-float (ffla.cu); the inverse
  // leaves the kernel as the split planes of S^-T
  MTRY(cudaMemsetAsync(m->mx, 0, sizeof(unsigned long long) * (2 * WS + 3 * h->W), st));
  MTRY(ffla::overlap(h->A, phi, m->bproj, m->s_ff, phi_perp, mx_phi, WS, h->nk, h->M, h->n, h->N, st));
  AFQMC_LAUNCHED(h);
  MTRY(ffla::invert(m->s_ff, WS, h->N, ld, sing, h->flags, m->sinvt_sp, m->Np, m->s_sinv, st));
  AFQMC_LAUNCHED(h);
  split_rows32_kernel<<<dim3(WS, SPLIT_CHUNKS), 256, 0, st>>>(phi_perp, h->NM, h->N, m->Np, mx_phi, m->s_phi,
                                                               m->phi_sp);
  AFQMC_LAUNCHED(h);
  return cudaGetLastError();
}
static cudaError_t green_post(afqmc_kp* h, cudaStream_t st) {
  MixedState* m = h->mixed;
  unsigned long long* mx_g = m->mx + 2 * m->WS;
  green_max_kernel<<<dim3(h->W, SPLIT_CHUNKS), 256, 0, st>>>(m->g32, mx_g, h->nk, h->W, m->nMp);
  AFQMC_LAUNCHED(h);
  split_green_kernel<<<dim3(h->W, SPLIT_CHUNKS), 256, 0, st>>>(m->g32, mx_g, m->g_sp, m->s_g, m->gsum_sp, m->s_gsum,
                                                                h->nk, h->W, m->nMp);
  AFQMC_LAUNCHED(h);
  return cudaGetLastError();
}
static cudaError_t green(afqmc_kp* h, const zc* phi, zc* ld, int* sing, cudaStream_t st) {
  MixedState* m = h->mixed;
  MTRY(green_pre(h, phi, ld, sing, st));
  MTRY(run_gemm(h, m->m_sinvt, m->m_phi, green_params(h), h->flags + 1, st));
  AFQMC_LAUNCHED(h);
  return green_post(h, st);
}

static cudaError_t trace_post(afqmc_kp* h, cudaStream_t st);
static cudaError_t cholesky_trace(afqmc_kp* h, cudaStream_t st) {
  MixedState* m = h->mixed;
  const ForceBiasP p = force_bias_params(h);
  MTRY(run_gemm(h, m->m_lh, m->m_gsum, p, h->flags + 1, st));
  AFQMC_LAUNCHED(h);
  return trace_post(h, st);
}
// X from the group partials of the force-bias GEMM
static cudaError_t trace_post(afqmc_kp* h, cudaStream_t st) {
  MixedState* m = h->mixed;
  const size_t per = (size_t)h->W * h->nk * h->G;
  xsum_kernel<<<(int)std::min<size_t>((per + 255) / 256, 4096), 256, 0, st>>>(m->xk, h->X, m->fb_groups, per);
  AFQMC_LAUNCHED(h);
  return cudaGetLastError();
}

cudaError_t force_bias(afqmc_kp* h, const zc* phi, zc* xbar, cudaStream_t st) {
  prof_begin(h, AFQMC_STAGE_GREEN, st);
  cudaError_t e = green(h, phi, h->ld_old, h->sing_old, st);
  prof_end(h, st);
  if (e != cudaSuccess) return e;
  prof_begin(h, AFQMC_STAGE_FORCE_BIAS, st);
  e = cholesky_trace(h, st);
  if (e == cudaSuccess) e = fp64::force_bias(h, nullptr, xbar, st);
  prof_end(h, st);
  return e;
}

static cudaError_t vhs_pre(afqmc_kp* h, cudaStream_t st) {
  MixedState* m = h->mixed;
  split_y_kernel<<<dim3(h->nk, h->W), 256, 0, st>>>(h->y, m->s_l, m->y_sp, m->s_y, h->nk, h->W, h->G, m->Gp);
  AFQMC_LAUNCHED(h);
  return cudaGetLastError();
}
static cudaError_t vhs(afqmc_kp* h, cudaStream_t st) {
  MixedState* m = h->mixed;
  MTRY(vhs_pre(h, st));
  const VhsP p = vhs_params(h);
  MTRY(run_gemm(h, m->m_lt, m->m_y, p, h->flags + 1, st));
  AFQMC_LAUNCHED(h);
  return cudaSuccess;
}

// The Taylor series in three parts: the first one-body half step and the split of the
// series' input (taylor_pre), the Horner GEMMs, the second half step (taylor_post).
static cudaError_t taylor_pre(afqmc_kp* h, const zc* phi, cudaStream_t st) {
  MixedState* m = h->mixed;
  const int R = 2 * h->N;
  dim3 g1(h->nk, m->WS, cdiv(h->N, 64));
  unsigned long long* mx_acc = m->mx + 2 * m->WS + 3 * h->W;
  MTRY(cudaMemsetAsync(mx_acc, 0, sizeof(unsigned long long) * h->W, st));
  float4* corr = reinterpret_cast<float4*>(m->acc);
  prof_begin(h, AFQMC_STAGE_ONEBODY, st);
  onebody_in_kernel<<<g1, 256, onebody_smem(h), st>>>(phi, m->dhalf, corr, m->p32, mx_acc, h->nk, h->M, h->N,
                                                       h->NM);
  AFQMC_LAUNCHED(h);
  split_rows32_kernel<<<dim3(h->W, SPLIT_CHUNKS), 256, 0, st>>>(m->p32, R, h->NM, m->NMp, mx_acc, m->s_t, m->t_sp[0]);
  AFQMC_LAUNCHED(h);
  prof_end(h, st);
  return cudaGetLastError();
}
static cudaError_t taylor_post(afqmc_kp* h, zc* phi, cudaStream_t st) {
  MixedState* m = h->mixed;
  dim3 g1(h->nk, m->WS, cdiv(h->N, 64));
  float4* corr = reinterpret_cast<float4*>(m->acc);
  prof_begin(h, AFQMC_STAGE_ONEBODY, st);
  if (onebody_out_staged(h))
    onebody_out_kernel<true><<<g1, 256, onebody_out_smem(h), st>>>(corr, m->dhalf, phi, h->nk, h->M, h->N, h->NM);
  else
    onebody_out_kernel<false><<<g1, 256, onebody_smem(h), st>>>(corr, m->dhalf, phi, h->nk, h->M, h->N, h->NM);
  AFQMC_LAUNCHED(h);
  prof_end(h, st);
  return cudaGetLastError();
}
static cudaError_t taylor(afqmc_kp* h, zc* phi, cudaStream_t st) {
  MTRY(taylor_pre(h, phi, st));
  // Horner: u = phi'; u <- phi' + V u / j for j = order .. 1
  for (int j = h->order, step = 0; j >= 1; --j, ++step) {
    const int cur = step & 1, nxt = (step + 1) & 1;
    prof_begin(h, AFQMC_STAGE_TAYLOR, st);   // one interval per term: the GEMM launch alone
    MTRY(taylor_gemm(h, j, cur, nxt, st));
    prof_end(h, st);
    AFQMC_LAUNCHED(h);
  }
  return taylor_post(h, phi, st);
}
static cudaError_t taylor_gemm(afqmc_kp* h, int j, int cur, int nxt, cudaStream_t st) {
  MixedState* m = h->mixed;
  if (!m->taylor_pair) return run_gemm(h, m->m_t[cur], m->m_v, taylor_params(h, j, nxt), h->flags + 1, st);
  // a pair stage holds half of B (40 KB), so four stages fit beside the staged tile: the
  // deeper ring covers the cross-SM completion of each stage
  return tcg::launch_precise_pair<4>(m->m_t[cur], m->m_vp, taylor_params_pair(h, j, nxt), h->flags + 1, st);
}

cudaError_t propagate(afqmc_kp* h, zc* phi, const double* x, double* w, zc* logdet, int do_qr, cudaStream_t st) {
  cudaError_t e;
  prof_begin(h, AFQMC_STAGE_GREEN, st);
  e = green(h, phi, h->ld_old, h->sing_old, st);
  prof_end(h, st);
  if (e != cudaSuccess) return e;
  prof_begin(h, AFQMC_STAGE_FORCE_BIAS, st);
  e = cholesky_trace(h, st);
  if (e == cudaSuccess) e = fp64::force_bias(h, x, h->xbar, st);
  prof_end(h, st);
  if (e != cudaSuccess) return e;
  prof_begin(h, AFQMC_STAGE_VHS, st);
  e = vhs(h, st);
  prof_end(h, st);
  if (e != cudaSuccess) return e;
  e = taylor(h, phi, st);   // records its own ONEBODY and TAYLOR intervals
  if (e != cudaSuccess) return e;
  prof_begin(h, AFQMC_STAGE_WEIGHT, st);
  e = overlap_logdet(h, phi, h->ld_new, h->sing_new, st);
  if (e == cudaSuccess) e = fp64::weight_only(h, x, w, do_qr ? nullptr : logdet, st);
  prof_end(h, st);
  if (e != cudaSuccess) return e;
  if (do_qr) return orthonormalise(h, phi, logdet, st);
  return cudaSuccess;
}

static cudaError_t chol_inv(afqmc_kp* h, double* logr, cudaStream_t st) {
  MixedState* m = h->mixed;
  const int N = h->N;
  const size_t full = (size_t)N * N * sizeof(float2) + (size_t)N * sizeof(float2);
  const bool in_smem = full <= 220 * 1024;
  const size_t bytes = in_smem ? full : (size_t)N * sizeof(float2);
  float2* gram = reinterpret_cast<float2*>(h->P);
  if (in_smem) {
    MTRY(set_smem_attr((const void*)chol_inv_kernel<true>, bytes));
    chol_inv_kernel<true><<<m->WS, CI_THREADS, bytes, st>>>(gram, m->sinvt_sp, m->s_sinv, h->flags, N, m->Np, logr);
  } else {
    MTRY(set_smem_attr((const void*)chol_inv_kernel<false>, bytes));
    chol_inv_kernel<false><<<m->WS, CI_THREADS, bytes, st>>>(gram, m->sinvt_sp, m->s_sinv, h->flags, N, m->Np, logr);
  }
  AFQMC_LAUNCHED(h);
  return cudaGetLastError();
}

// Cholesky-QR2: twice { Gram = phi^dag phi on the tensor cores; R = chol(Gram) and R^-1 in
// fp32; phi <- phi R^-1 on the tensor cores }.  R has a real positive diagonal, so
// phi ends as the unique Q factor of the Householder QR with diag(R) > 0.
// logr != nullptr: logr[ws] receives sum_j log R_jj over both passes (R = R2 R1).
static cudaError_t cholqr2(afqmc_kp* h, zc* phi, double* logr, cudaStream_t st) {
  MixedState* m = h->mixed;
  if (logr) MTRY(cudaMemsetAsync(logr, 0, sizeof(double) * m->WS, st));
  const int WS = m->WS, N = h->N, NM = h->NM, W = h->W;
  unsigned long long* mx_phi = m->mx;
  unsigned long long* mx_w = m->mx + 2 * WS + 3 * W;
  for (int pass = 0; pass < 2; ++pass) {
    MTRY(cudaMemsetAsync(m->mx, 0, sizeof(unsigned long long) * (2 * WS + 3 * W + W), st));
    maxabs_kernel<<<dim3(W, SPLIT_CHUNKS), 256, 0, st>>>(phi, (size_t)2 * NM * N, mx_w);
    AFQMC_LAUNCHED(h);
    split_T_kernel<<<dim3(cdiv(NM, 32), cdiv(N, 32), 2 * W), 256, 0, st>>>(phi, mx_w, m->s_t, m->t_sp[0], NM, N,
                                                                          m->NMp);
    AFQMC_LAUNCHED(h);
    MTRY(cudaGetLastError());
    GramP g;
    g.mt_n = cdiv(N, 128);
    g.nt_n = cdiv(N, BN);
    g.tiles = WS * g.mt_n * g.nt_n;
    g.kchunks = m->NMp / 32;
    g.N = N; g.s_t = m->s_t; g.gram = reinterpret_cast<float2*>(h->P);
    MTRY(run_gemm(h, m->m_t[0], m->m_t0_b, g, h->flags + 1, st));
    AFQMC_LAUNCHED(h);
    MTRY(chol_inv(h, logr, st));
    maxabs_kernel<<<dim3(WS, SPLIT_CHUNKS), 256, 0, st>>>(phi, (size_t)NM * N, mx_phi);
    AFQMC_LAUNCHED(h);
    split_rows_kernel<<<dim3(WS, SPLIT_CHUNKS), 256, 0, st>>>(phi, NM, N, m->Np, mx_phi, m->s_phi, m->phi_sp);
    AFQMC_LAUNCHED(h);
    MTRY(cudaGetLastError());
    ApplyRP a;
    a.mt_n = cdiv(NM, 128);
    a.nt_n = cdiv(N, BN);
    a.tiles = WS * a.mt_n * a.nt_n;
    a.kchunks = m->Np / 32;
    a.NM = NM; a.N = N; a.s_phi = m->s_phi; a.s_r = m->s_sinv; a.phi = phi;
    MTRY(run_gemm(h, m->m_phi_a, m->m_sinvt_b, a, h->flags + 1, st));
    AFQMC_LAUNCHED(h);
  }
  return cudaSuccess;
}

cudaError_t orthonormalise(afqmc_kp* h, zc* phi, zc* logdet, cudaStream_t st) {
  prof_begin(h, AFQMC_STAGE_QR, st);
  cudaError_t e = cholqr2(h, phi, nullptr, st);
  if (e == cudaSuccess && logdet) e = overlap_logdet(h, phi, logdet, h->sing_new, st);
  prof_end(h, st);
  return e;
}

static cudaError_t e1_ec(afqmc_kp* h, zc* eloc, cudaStream_t st) {
  MixedState* m = h->mixed;
  e1_ec_mixed_kernel<<<h->W, 256, 0, st>>>(h->AhH, m->g32, h->X, h->minus, eloc, h->nk, h->M, h->n, m->Mp, h->G,
                                            m->WS);
  AFQMC_LAUNCHED(h);
  return cudaGetLastError();
}

static cudaError_t exchange(afqmc_kp* h, cudaStream_t st) {
  MixedState* m = h->mixed;
  const ExchangeP p = exchange_params(h);
  MTRY(run_gemm(h, m->m_g, m->m_z, p, h->flags + 1, st));
  AFQMC_LAUNCHED(h);
  return cudaSuccess;
}

static cudaError_t ex_reduce(afqmc_kp* h, zc* eloc, cudaStream_t st) {
  MixedState* m = h->mixed;
  ex_partial_kernel<<<EX_CHUNKS, 128, 0, st>>>(m->xpart, m->tri, m->expart, m->T, cdiv(m->nMp, BN), m->WS);
  AFQMC_LAUNCHED(h);
  ex_reduce_mixed_kernel<<<h->W, 128, 0, st>>>(m->expart, eloc, EX_CHUNKS, m->WS);
  AFQMC_LAUNCHED(h);
  return cudaGetLastError();
}

#define MSTAGE(stage, body)           \
  do {                                \
    prof_begin(h, stage, st);         \
    cudaError_t e_ = (body);          \
    prof_end(h, st);                  \
    if (e_ != cudaSuccess) return e_; \
  } while (0)

cudaError_t local_energy(afqmc_kp* h, const zc* phi, zc* eloc, cudaStream_t st) {
  MSTAGE(AFQMC_STAGE_GREEN, green(h, phi, h->ld_old, h->sing_old, st));
  MSTAGE(AFQMC_STAGE_FORCE_BIAS, cholesky_trace(h, st));
  MSTAGE(AFQMC_STAGE_ENERGY, e1_ec(h, eloc, st));
  MSTAGE(AFQMC_STAGE_EXCHANGE, exchange(h, st));
  MSTAGE(AFQMC_STAGE_ENERGY, ex_reduce(h, eloc, st));
  return cudaSuccess;
}

// One fused walker step (see fp64::step): the Green's function of the
// propagated walkers serves their log det, their energy and the next force bias.
cudaError_t step(afqmc_kp* h, zc* phi, const double* x, double* w, zc* eloc, zc* logdet, int do_qr, int reuse,
                 cudaStream_t st) {
  if (!reuse) {
    MSTAGE(AFQMC_STAGE_GREEN, green(h, phi, h->ld_old, h->sing_old, st));
    MSTAGE(AFQMC_STAGE_FORCE_BIAS, cholesky_trace(h, st));
  }
  MSTAGE(AFQMC_STAGE_FORCE_BIAS, fp64::force_bias(h, x, h->xbar, st));
  MSTAGE(AFQMC_STAGE_VHS, vhs(h, st));
  MTRY(taylor(h, phi, st));   // records its own ONEBODY and TAYLOR intervals
  MSTAGE(AFQMC_STAGE_GREEN, green(h, phi, h->ld_new, h->sing_new, st));
  MSTAGE(AFQMC_STAGE_FORCE_BIAS, cholesky_trace(h, st));
  MSTAGE(AFQMC_STAGE_WEIGHT, fp64::weight_only(h, x, w, do_qr ? nullptr : logdet, st));
  if (eloc) {   // NULL: a propagation-only step of a block (the energy is measured less often)
    MSTAGE(AFQMC_STAGE_ENERGY, e1_ec(h, eloc, st));
    MSTAGE(AFQMC_STAGE_EXCHANGE, exchange(h, st));
    MSTAGE(AFQMC_STAGE_ENERGY, ex_reduce(h, eloc, st));
  }
  if (do_qr) {
    // log det (A^dag phi R^-1) = log det (A^dag phi) - log det R, R with a real positive
    // diagonal, so only the real part of the step's new log det changes
    MixedState* m = h->mixed;
    MSTAGE(AFQMC_STAGE_QR, cholqr2(h, phi, m->logr, st));
    ld_shift_kernel<<<cdiv(m->WS, 128), 128, 0, st>>>(h->ld_new, m->logr, h->sing_new, m->WS);
    AFQMC_LAUNCHED(h);
    MTRY(cudaGetLastError());
    if (logdet)
      MTRY(cudaMemcpyAsync(logdet, h->ld_new, sizeof(zc) * 2 * h->W, cudaMemcpyDeviceToDevice, st));
  }
  std::swap(h->ld_old, h->ld_new);
  std::swap(h->sing_old, h->sing_new);
  return cudaSuccess;
}

// ---------------------------------------------------------------------------
// several handles stepped together (a group of uneven systems)
// ---------------------------------------------------------------------------
// One launch of policy P over the tiles of every listed handle (tcg::GroupP): mk(h) gives a
// handle's parameters, maps(h) its (A, B) tensor maps.  Time-outs land in the first handle's
// flags.  The TMA ring takes the depth the member with the most tiles chose at create (the
// depth changes no arithmetic).
template <class P, class MK, class MAPS>
static cudaError_t group_gemm(afqmc_kp* const* hs, int n, MK mk, MAPS maps, cudaStream_t st) {
  constexpr int NMAX = GROUP_MAX;
  if (n < 1 || n > NMAX) return cudaErrorInvalidValue;
  tcg::GroupP<P, NMAX> g{};
  g.n = n;
  g.start[0] = 0;
  for (int i = 0; i < n; ++i) {
    g.m[i] = mk(hs[i]);
    // the member's tile groups must fit the 20 bits GroupP packs them in
    if ((long long)g.m[i].tiles >= (1LL << 20) * g.m[i].mt_n * g.m[i].nt_n) return cudaErrorInvalidValue;
    const auto mp = maps(hs[i]);
    g.ma[i] = *mp.first;
    g.mb[i] = *mp.second;
    g.start[i + 1] = g.start[i] + g.m[i].tiles;
  }
  for (int i = n + 1; i <= NMAX; ++i) g.start[i] = g.start[n];
  g.tiles = g.start[n];
  g.kchunks = 0;
  int big = 0;
  for (int i = 1; i < n; ++i)
    if (g.m[i].tiles > g.m[big].tiles) big = i;
  const int r = hs[big]->mixed->ring[GemmIdOf<P>::value];
  const auto mp0 = maps(hs[0]);
  AFQMC_LAUNCHED(hs[0]);
  return (r ? r : P::kStages) == 2 ? tcg::launch_precise<2>(*mp0.first, *mp0.second, g, hs[0]->flags + 1, st)
                                   : tcg::launch_precise<3>(*mp0.first, *mp0.second, g, hs[0]->flags + 1, st);
}

// The step's tail on one member after its propagated walkers' Green's function GEMM:
// the QR where asked, the log-det bookkeeping.
static cudaError_t group_member_tail(afqmc_kp* h, zc* phi, zc* eloc, zc* logdet, int do_qr, cudaStream_t s) {
  if (eloc) MTRY(ex_reduce(h, eloc, s));
  if (do_qr) {
    MixedState* m = h->mixed;
    MTRY(cholqr2(h, phi, m->logr, s));
    ld_shift_kernel<<<cdiv(m->WS, 128), 128, 0, s>>>(h->ld_new, m->logr, h->sing_new, m->WS);
    AFQMC_LAUNCHED(h);
    MTRY(cudaGetLastError());
    if (logdet) MTRY(cudaMemcpyAsync(logdet, h->ld_new, sizeof(zc) * 2 * h->W, cudaMemcpyDeviceToDevice, s));
  }
  std::swap(h->ld_old, h->ld_new);
  std::swap(h->sing_old, h->sing_new);
  return cudaSuccess;
}

cudaError_t group_step(afqmc_kp* const* hs, int n, zc* const* phi, const double* const* x, double* const* w,
                       zc* const* eloc, zc* const* logdet, int do_qr, const int* reuse, bool all, const ForEach& each,
                       cudaStream_t st) {
  using MP = std::pair<const CUtensorMap*, const CUtensorMap*>;
  // force bias of the current walkers (their Green's function first where not reused), y
  MTRY(each([&](int i, afqmc_kp* h, cudaStream_t s) -> cudaError_t {
    if (!reuse[i]) {
      MTRY(green(h, phi[i], h->ld_old, h->sing_old, s));
      MTRY(cholesky_trace(h, s));
    }
    MTRY(fp64::force_bias(h, x[i], h->xbar, s));
    if (all) return vhs_pre(h, s);
    MTRY(vhs(h, s));
    return taylor_pre(h, phi[i], s);
  }));
  if (all) {
    MTRY(group_gemm<VhsP>(hs, n, [](const afqmc_kp* h) { return vhs_params(h); },
                          [](const afqmc_kp* h) { return MP(&h->mixed->m_lt, &h->mixed->m_y); }, st));
    MTRY(each([&](int i, afqmc_kp* h, cudaStream_t s) { return taylor_pre(h, phi[i], s); }));
  }
  const int order = hs[0]->order;
  for (int j = order, step = 0; j >= 1; --j, ++step) {
    const int cur = step & 1, nxt = (step + 1) & 1;
    MTRY(group_gemm<TaylorP>(hs, n, [&](const afqmc_kp* h) { return taylor_params(h, j, nxt); },
                             [&](const afqmc_kp* h) { return MP(&h->mixed->m_t[cur], &h->mixed->m_v); }, st));
  }
  if (!all)   // the rest of the step on each member's own launches
    return each([&](int i, afqmc_kp* h, cudaStream_t s) -> cudaError_t {
      MTRY(taylor_post(h, phi[i], s));
      MTRY(green(h, phi[i], h->ld_new, h->sing_new, s));
      MTRY(cholesky_trace(h, s));
      MTRY(fp64::weight_only(h, x[i], w[i], do_qr ? nullptr : logdet[i], s));
      if (eloc[i]) {
        MTRY(e1_ec(h, eloc[i], s));
        MTRY(exchange(h, s));
      }
      return group_member_tail(h, phi[i], eloc[i], logdet[i], do_qr, s);
    });
  // the propagated walkers' Green's function, the Cholesky trace, the weights
  MTRY(each([&](int i, afqmc_kp* h, cudaStream_t s) -> cudaError_t {
    MTRY(taylor_post(h, phi[i], s));
    return green_pre(h, phi[i], h->ld_new, h->sing_new, s);
  }));
  MTRY(group_gemm<GreenP>(hs, n, [](const afqmc_kp* h) { return green_params(h); },
                          [](const afqmc_kp* h) { return MP(&h->mixed->m_sinvt, &h->mixed->m_phi); }, st));
  MTRY(each([&](int, afqmc_kp* h, cudaStream_t s) { return green_post(h, s); }));
  MTRY(group_gemm<ForceBiasP>(hs, n, [](const afqmc_kp* h) { return force_bias_params(h); },
                              [](const afqmc_kp* h) { return MP(&h->mixed->m_lh, &h->mixed->m_gsum); }, st));
  MTRY(each([&](int i, afqmc_kp* h, cudaStream_t s) -> cudaError_t {
    MTRY(trace_post(h, s));
    MTRY(fp64::weight_only(h, x[i], w[i], do_qr ? nullptr : logdet[i], s));
    return eloc[i] ? e1_ec(h, eloc[i], s) : cudaSuccess;
  }));
  // the exchange of the members that want their energy
  std::vector<afqmc_kp*> ex;
  for (int i = 0; i < n; ++i)
    if (eloc[i]) ex.push_back(hs[i]);
  if (!ex.empty())
    MTRY(group_gemm<ExchangeP>(ex.data(), (int)ex.size(), [](const afqmc_kp* h) { return exchange_params(h); },
                               [](const afqmc_kp* h) { return MP(&h->mixed->m_g, &h->mixed->m_z); }, st));
  return each([&](int i, afqmc_kp* h, cudaStream_t s) {
    return group_member_tail(h, phi[i], eloc[i], logdet[i], do_qr, s);
  });
}

// dEX/dGh for every block (AdjointP GEMM into gam32).
static cudaError_t adjoint_exchange(afqmc_kp* h, cudaStream_t st) {
  MixedState* m = h->mixed;
  return run_gemm(h, m->m_g, m->m_zall, adjoint_params(h), h->flags + 1, st);
}

// The adjoint: Gam = conj(grad_e)-weighted dE/dGh with the exchange part from the
// tensor-core GEMM over the full precontracted tensor and the Coulomb and one-body parts in
// fp32, then the projection onto dE/dphi through S^-1 and the Green's function (FP64 LU,
// double-float products) and dE/dh.
cudaError_t local_energy_backward(afqmc_kp* h, const zc* phi, const zc* grad_e, zc* grad_phi, zc* grad_h1,
                                  cudaStream_t st) {
  MixedState* m = h->mixed;
  if (grad_phi) {
    MSTAGE(AFQMC_STAGE_GREEN, green(h, phi, h->ld_old, h->sing_old, st));
    MSTAGE(AFQMC_STAGE_FORCE_BIAS, cholesky_trace(h, st));
    MSTAGE(AFQMC_STAGE_ADJOINT_GEMM, adjoint_exchange(h, st));
    prof_begin(h, AFQMC_STAGE_BACKWARD, st);
    gamma_assemble_kernel<<<dim3(h->nk, h->nk, cdiv(h->W, GA_W)), 128, sizeof(float2) * GA_W * h->G, st>>>(
        h->LH, h->X, h->AhH, grad_e, m->gam32, h->Gam, h->kminus, h->minus, h->nk, h->G, h->M, h->n, m->Mp, h->W);
    AFQMC_LAUNCHED(h);
    prof_end(h, st);
    MTRY(cudaGetLastError());
  }
  // Green's function and inverse of the same walkers for the projection: FP64 overlap and
  // LU, the large products in double-float
  MTRY(fp64::green_ff(h, phi, st));
  if (grad_h1) MSTAGE(AFQMC_STAGE_BACKWARD, fp64::grad_h1(h, grad_e, grad_h1, st));
  if (grad_phi) MSTAGE(AFQMC_STAGE_BACKWARD, fp64::project_gamma(h, grad_phi, st, true));
  return cudaSuccess;
}

}  // namespace mixed
