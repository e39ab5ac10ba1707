// Complex GEMM on the 5th-generation tensor cores with an fp16 hi/lo split.
//
//   D[m][n] = sum_k A[m][k] * B[n][k]          (complex, no conjugation)
//
// Operands live in global memory as four fp16 "planes" of the same shape,
// K-major (k contiguous), padded to a multiple of 32 complex elements in k:
//   plane 0 = hi(Re x*s), 1 = lo(Re x*s), 2 = hi(Im x*s), 3 = lo(Im x*s)
// with hi = fp16(x*s), lo = fp16(x*s - hi) and s a power-of-two scale chosen so
// that |x*s| stays well inside the fp16 range.  Each real product is formed
// from three fp16 products (hi*hi + hi*lo + lo*hi), accumulated in fp32 in
// tensor memory, which keeps about 22 significant bits per operand.  The real
// and imaginary parts of D use two accumulators:
//   D_re = Ar Br - Ai Bi,   D_im = Ar Bi + Ai Br   (negation via the MMA's B-negate bit)
//
// Persistent kernel, one CTA per SM over a contiguous range of 128 x 64 output tiles:
// warp 0 issues TMA loads (one 5-D box per operand per 32-wide k chunk, all four planes
// at once, 64-byte swizzle) into a STAGES-deep ring; warp 1 allocates tensor memory and
// one of its threads issues the tcgen05.mma chain; warps 2-5 read the accumulators back
// with tcgen05.ld and hand the finished tile to the policy's epilogue.  Every mbarrier
// wait is bounded; on time-out the kernel records an error, drains its own copies and
// MMAs, frees tensor memory and returns.
#pragma once

#include <cuda_fp16.h>

#include "attr.hpp"
#include "tc.cuh"

namespace tcg {

constexpr int BM = 128;      // tile rows = TMEM lanes
constexpr int BK = 32;       // complex k per stage: 64-byte fp16 rows
constexpr int NPLANE = 4;
// warp 0 TMA, warp 1 MMA, warps 2-5 drain the accumulators, warps 6-9 store the drained
// tiles (so that the stores of one tile overlap the MMAs of the next)
constexpr int THREADS = 320;

struct Coords {
  int a[5];
  int b[5];
};

// Policy P provides:
//   static constexpr bool kConjA;     D = sum conj(A) B instead of sum A B
//   int tiles;                        number of output tiles
//   int kchunks;                      k chunks of BK per tile
//   __device__ void tile(int t, int& b, int& mt, int& nt) const;
//   __device__ Coords coords(int b, int mt, int nt, int kc) const;
//   __device__ void store_tile(int b, int mt, int nt, const float2* tile, int tid, int ewarp, int lane) const;
//       the finished 128 x 64 tile in shared memory, tile[r * STAGE_LD + c] = (re, im);
//       called by the 128 store threads (tid 0..127, ewarp 0..3) while the drain warps
//       already accumulate the next tile
// and optionally
//   static constexpr bool kChunkScale = true;
//   __device__ float chunk_scale(int b, int kc) const;
//       a factor applied to k chunk kc's partial sums as they are drained (operands whose
//       scale changes along k; a power of two keeps the fold exact)
template <class P, class = void>
struct ChunkScaled {
  static constexpr bool value = false;
};
template <class P>
struct ChunkScaled<P, decltype((void)P::kChunkScale)> {
  static constexpr bool value = P::kChunkScale;
};
//   static constexpr bool kPairB = true;
//       B is staged with its planes in the order (re_hi, im_hi, re_lo, im_lo) (a tensor map
//       whose plane dimensions are (re/im, hi/lo)), so that [B_re; B_im] is one 128-row
//       operand: one N = 128 MMA then gives [A_x B_re | A_x B_im], twelve MMAs per chunk
//       instead of twenty-four, and each A plane is read half as often
template <class P, class = void>
struct PairB {
  static constexpr bool value = false;
};
template <class P>
struct PairB<P, decltype((void)P::kPairB)> {
  static constexpr bool value = P::kPairB;
};

//   static constexpr int kDrainChunks = D;
//       the accumulators run over D consecutive k chunks before they are drained (default 1):
//       the drain work per MMA falls by D, each fp32 partial carries D times as many
//       truncating additions.  Not with kChunkScale (one factor per drained partial).
template <class P, class = void>
struct DrainChunks {
  static constexpr int value = 1;
};
template <class P>
struct DrainChunks<P, decltype((void)P::kDrainChunks)> {
  static constexpr int value = P::kDrainChunks;
};

//   static constexpr bool kStreamB = true;  __device__ bool stream_b() const;
//       when stream_b() is true, B is read once per launch (a large static tensor streamed
//       through, one row tile): its TMA loads carry the L2 evict-first policy, so that the
//       reused A tiles and the epilogue's operands stay in L2
template <class P, class = void>
struct StreamB {
  static constexpr bool value = false;
};
template <class P>
struct StreamB<P, decltype((void)P::kStreamB)> {
  static constexpr bool value = P::kStreamB;
};

//   static constexpr bool kGrouped = true;
//       the tiles of several problems in one launch (GroupP below): the k chunks of a tile
//       and its operands' tensor maps depend on the tile (kchunks_of(b), map_a(b), map_b(b))
template <class P, class = void>
struct Grouped {
  static constexpr bool value = false;
};
template <class P>
struct Grouped<P, decltype((void)P::kGrouped)> {
  static constexpr bool value = P::kGrouped;
};
template <class P>
__device__ __forceinline__ int kchunks_of(const P& p, int b) {
  if constexpr (Grouped<P>::value)
    return p.kchunks_of(b);
  else
    return p.kchunks;
}
template <class P>
__device__ __forceinline__ const CUtensorMap* map_a_of(const P& p, int b, const CUtensorMap* own) {
  if constexpr (Grouped<P>::value)
    return p.map_a(b);
  else
    return own;
}
template <class P>
__device__ __forceinline__ const CUtensorMap* map_b_of(const P& p, int b, const CUtensorMap* own) {
  if constexpr (Grouped<P>::value)
    return p.map_b(b);
  else
    return own;
}

template <class P>
__device__ __forceinline__ float chunk_factor(const P& p, int b, int kc) {
  if constexpr (ChunkScaled<P>::value)
    return p.chunk_scale(b, kc);
  else
    return 1.f;
}

// ---------------------------------------------------------------- precise variant
// The tensor-core accumulator adds each MMA's partial sum with truncation, so a
// long chain of MMAs into one accumulator loses accuracy in proportion to its
// length.  This variant keeps four real accumulators per k-step,
//   P_rr = Ar Br, P_ii = Ai Bi, P_ri = Ar Bi, P_ir = Ai Br   (each hi*hi + hi*lo + lo*hi),
// restarts them on every 16-wide k step (two TMEM sets in ping-pong), and the
// epilogue warps fold each step into fp32 register sums with round-to-nearest:
//   re += P_rr - P_ii,  im += P_ri + P_ir.
// Tile 128 x BNP (BNP = 64): 4 x 64 columns per set, 2 sets = all 512 TMEM columns.
constexpr int BNP = 64;

// Accumulator columns per tcgen05.ld in the drain (8 or 16): fewer round trips against more
// registers beyond the 128 running sums.
constexpr int DRAIN_COLS = 8;

// Epilogue staging: the finished 128 x 64 tile as (re, im) fp32 pairs, rows padded to 65
// entries so that row-per-thread and column-per-thread accesses both avoid bank conflicts.
constexpr int STAGE_LD = BNP + 1;

// PAIR: a stage holds one half (re or im planes) of the paired B tile.
template <int STAGES, bool PAIR = false>
struct LayoutP {
  static constexpr int A_BYTES = NPLANE * BM * 64;
  static constexpr int B_BYTES = NPLANE * BNP * 64 / (PAIR ? 2 : 1);
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr int TILE_BYTES = BM * STAGE_LD * 8;
  static constexpr int BAR_BYTES = 256;
  static constexpr int SMEM = STAGES * STAGE_BYTES + TILE_BYTES + BAR_BYTES + 1024;
  static constexpr uint32_t TMEM_COLS = 512;
};

// PAIR: the CTAs run in clusters of two and every MMA is a cta_group::2 MMA of 256 rows issued
// by the even CTA: each CTA stages its own 128 rows of A and half of the paired B (the real
// planes in the even CTA, the imaginary ones in the odd CTA, through a B map whose box holds one
// of the two), so the pair reads each B element from shared memory once where two CTAs would
// read it twice.  Tile t of the policy is then a pair of row tiles: CTA r takes row tile
// 2 mt + r.  Each CTA drains and stores its own rows as in the single form.
template <int STAGES, class P, bool PAIR = false>
__global__ void __launch_bounds__(THREADS, 1)
    cgemm_precise_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                         const __grid_constant__ P p, int* err) {
  static_assert(!PAIR || (PairB<P>::value && !Grouped<P>::value), "pair form: paired B, one problem");
  static_assert(LayoutP<STAGES, PAIR>::SMEM <= 232448, "shared memory per CTA");
  // Persistent: CTA i handles tiles i, i + grid, i + 2 grid, ...  The TMA ring and the
  // two TMEM accumulator sets run continuously across tile boundaries.  One drain per 32-wide k
  // chunk: per accumulator the four small cross products of the chunk go first, then
  // the two hi*hi products, so a drained partial carries two full-magnitude truncations.
  using Lay = LayoutP<STAGES, PAIR>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  float2* tile_buf = reinterpret_cast<float2*>(smem + STAGES * Lay::STAGE_BYTES);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * Lay::STAGE_BYTES + Lay::TILE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* accf = empty + STAGES;   // [2] MMA -> epilogue: set holds a finished chunk
  uint64_t* acce = accf + 2;         // [2] epilogue -> MMA: set drained
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acce + 2);
  volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = PAIR ? tc::cluster_ctarank() : 0u;
  const bool leader = rank == 0;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    for (int s = 0; s < 2; ++s) {
      tc::mbar_init(&accf[s], 1);
      tc::mbar_init(&acce[s], PAIR ? 8 : 4);   // the drain warps of both CTAs in the pair form
    }
    *abort = 0;
    tc::fence_mbar_init();
  }
  if (warp == 1) {
    if constexpr (PAIR) {
      tc::tmem_alloc_pair(tmem_slot, Lay::TMEM_COLS);
      tc::tmem_relinquish_pair();
    } else {
      tc::tmem_alloc(tmem_slot, Lay::TMEM_COLS);
      tc::tmem_relinquish();
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if constexpr (PAIR) tc::cluster_sync();   // the peer's barriers are initialised
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;

  // tile t runs on CTA t mod gridDim.x: the tiles in flight at any moment are
  // consecutive, so the operands they share (one walker's rows, one Cholesky block)
  // are read from HBM once and served from L2 to the others
  const int t0 = PAIR ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;
  const int tstep = PAIR ? (int)(gridDim.x >> 1) : (int)gridDim.x;
  constexpr int DC = DrainChunks<P>::value;
  static_assert(DC >= 1 && (DC == 1 || !ChunkScaled<P>::value), "one chunk factor per drained partial");

  if (warp == 0) {
    if (lane == 0) {
      if constexpr (!Grouped<P>::value) {
        tc::tma_prefetch(&tmA);
        tc::tma_prefetch(&tmB);
      }
      bool stream = false;
      if constexpr (StreamB<P>::value && !Grouped<P>::value) stream = p.stream_b();
      const uint64_t stream_pol = StreamB<P>::value ? tc::l2_evict_first_policy() : 0;
      long g = 0;
      bool failed = false;
      for (int t = t0; t < p.tiles && !failed; t += tstep) {
        int b, mt, nt;
        p.tile(t, b, mt, nt);
        const int KC = kchunks_of(p, b);
        const CUtensorMap* ma = map_a_of(p, b, &tmA);
        const CUtensorMap* mb = map_b_of(p, b, &tmB);
        if constexpr (StreamB<P>::value && Grouped<P>::value) stream = p.stream_b_of(b);   // per member
        for (int kc = 0; kc < KC; ++kc, ++g) {
          const int s = (int)(g % STAGES);
          const uint32_t ph = (uint32_t)((g / STAGES) & 1);
          if (!tc::mbar_wait(&empty[s], ph ^ 1, abort)) {
            atomicCAS(err, 0, tc::ERR_TIMEOUT_EMPTY);
            *abort = 1;
            failed = true;
            break;
          }
          uint8_t* sa = smem + s * Lay::STAGE_BYTES;
          if constexpr (PAIR) {
            // both CTAs' copies complete on the even CTA's full barrier
            if (leader) tc::mbar_arrive_expect_tx(&full[s], 2 * Lay::STAGE_BYTES);
            Coords c = p.coords(b, 2 * mt + (int)rank, nt, kc);
            c.b[2] += (int)rank;   // re planes in the even CTA, im planes in the odd one
            const uint32_t fb = tc::mapa_shared(tc::smem_u32(&full[s]), 0);
            tc::tma_load_5d_pair(sa, ma, fb, c.a[0], c.a[1], c.a[2], c.a[3], c.a[4]);
            tc::tma_load_5d_pair(sa + Lay::A_BYTES, mb, fb, c.b[0], c.b[1], c.b[2], c.b[3], c.b[4]);
            continue;
          }
          tc::mbar_arrive_expect_tx(&full[s], Lay::STAGE_BYTES);
          const Coords c = p.coords(b, mt, nt, kc);
          tc::tma_load_5d(sa, ma, &full[s], c.a[0], c.a[1], c.a[2], c.a[3], c.a[4]);
          if (stream)
            tc::tma_load_5d_hint(sa + Lay::A_BYTES, mb, &full[s], c.b[0], c.b[1], c.b[2], c.b[3], c.b[4],
                                 stream_pol);
          else
            tc::tma_load_5d(sa + Lay::A_BYTES, mb, &full[s], c.b[0], c.b[1], c.b[2], c.b[3], c.b[4]);
        }
      }
      // every issued copy must land before the CTA may exit (in the pair form the even CTA's
      // full barriers count both CTAs' copies, and the final cluster barrier holds the odd CTA)
      for (long q = (g > STAGES ? g - STAGES : 0); q < g && leader; ++q) {
        const int s = (int)(q % STAGES);
        const uint32_t ph = (uint32_t)((q / STAGES) & 1);
        int zero = 0;
        if (!tc::mbar_wait(&full[s], ph, &zero)) atomicCAS(err, 0, tc::ERR_TIMEOUT_DRAIN);
      }
    }
  } else if (warp == 1) {
    if (lane == 0 && leader) {   // the pair form's MMAs are issued by the even CTA alone
      constexpr uint32_t id = tc::idesc_f16(BM, BNP, false);
      long g = 0;   // k chunks (TMA ring)
      long a = 0;   // drained partials (accumulator sets), one per D chunks
      bool failed = false;
      for (int t = t0; t < p.tiles && !failed; t += tstep) {
        int b, mt, nt;
        p.tile(t, b, mt, nt);
        const int KC = kchunks_of(p, b);
        for (int kc = 0; kc < KC; ++kc, ++g) {
          const int s = (int)(g % STAGES);
          const uint32_t ph = (uint32_t)((g / STAGES) & 1);
          if (!tc::mbar_wait(&full[s], ph, abort)) {
            atomicCAS(err, 0, tc::ERR_TIMEOUT_FULL);
            *abort = 1;
            failed = true;
            break;
          }
          const bool open = (kc % DC) == 0;                      // first chunk of a partial
          const bool close = (kc % DC) == DC - 1 || kc == KC - 1;  // last chunk of a partial
          const int set = (int)(a & 1);
          const uint32_t use = (uint32_t)(a >> 1);
          if (open && !tc::mbar_wait(&acce[set], (use & 1) ^ 1, abort)) {
            atomicCAS(err, 0, tc::ERR_TIMEOUT_ACC);
            *abort = 1;
            failed = true;
            break;
          }
          const uint32_t acc0 = open ? 0u : 1u;   // the partial's first MMA overwrites the set
          tc::fence_after_sync();
          const uint32_t sa = tc::smem_u32(smem + s * Lay::STAGE_BYTES);
          const uint32_t sb = sa + Lay::A_BYTES;
          const uint32_t d = tmem + set * 4 * BNP;
          uint64_t A[4][2];  // [plane][k16 half]; A planes: 0 re_hi, 1 re_lo, 2 im_hi, 3 im_lo
#pragma unroll
          for (int pl = 0; pl < 4; ++pl)
#pragma unroll
            for (int kk = 0; kk < 2; ++kk) A[pl][kk] = tc::desc_kmajor_sw64(sa + pl * BM * 64 + kk * 32);
          if constexpr (PAIR) {
            // Each CTA holds [B_hi; B_lo] of its half (re in the even CTA, im in the odd one),
            // 64 rows each: the pair's B operand rows 0..127 are [Br_hi; Bi_hi] (or _lo).
            constexpr uint32_t idp = tc::idesc_f16(2 * BM, 2 * BNP, false);
            uint64_t Bh[2], Bl[2];
#pragma unroll
            for (int kk = 0; kk < 2; ++kk) {
              Bh[kk] = tc::desc_kmajor_sw64(sb + kk * 32);
              Bl[kk] = tc::desc_kmajor_sw64(sb + BNP * 64 + kk * 32);
            }
#pragma unroll
            for (int q = 0; q < 2; ++q) {
              const uint32_t dq = d + q * 2 * BNP;
              const int ah = 2 * q;
              tc::mma_f16_pair(dq, A[ah + 1][0], Bh[0], idp, acc0);
              tc::mma_f16_pair(dq, A[ah][0], Bl[0], idp, 1);
              tc::mma_f16_pair(dq, A[ah + 1][1], Bh[1], idp, 1);
              tc::mma_f16_pair(dq, A[ah][1], Bl[1], idp, 1);
              tc::mma_f16_pair(dq, A[ah][0], Bh[0], idp, 1);
              tc::mma_f16_pair(dq, A[ah][1], Bh[1], idp, 1);
            }
          } else if constexpr (PairB<P>::value) {
            // B rows 0..127 = [Br_hi; Bi_hi], rows 128..255 = [Br_lo; Bi_lo].  Accumulators:
            // Ar [Br | Bi] -> P_rr (0), P_ri (64); Ai [Br | Bi] -> P_ir (128), P_ii (192).
            constexpr uint32_t id2 = tc::idesc_f16(BM, 2 * BNP, false);
            uint64_t Bh[2], Bl[2];
#pragma unroll
            for (int kk = 0; kk < 2; ++kk) {
              Bh[kk] = tc::desc_kmajor_sw64(sb + kk * 32);
              Bl[kk] = tc::desc_kmajor_sw64(sb + 2 * BNP * 64 + kk * 32);
            }
#pragma unroll
            for (int q = 0; q < 2; ++q) {
              const uint32_t dq = d + q * 2 * BNP;
              const int ah = 2 * q;
              tc::mma_f16(dq, A[ah + 1][0], Bh[0], id2, acc0);
              tc::mma_f16(dq, A[ah][0], Bl[0], id2, 1);
              tc::mma_f16(dq, A[ah + 1][1], Bh[1], id2, 1);
              tc::mma_f16(dq, A[ah][1], Bl[1], id2, 1);
              tc::mma_f16(dq, A[ah][0], Bh[0], id2, 1);
              tc::mma_f16(dq, A[ah][1], Bh[1], id2, 1);
            }
          } else {
            uint64_t B[4][2];
#pragma unroll
            for (int pl = 0; pl < 4; ++pl)
#pragma unroll
              for (int kk = 0; kk < 2; ++kk) B[pl][kk] = tc::desc_kmajor_sw64(sb + pl * BNP * 64 + kk * 32);
            // Accumulators (column offsets):
            // P_rr = Ar Br (0), P_ii = Ai Bi (64), P_ri = Ar Bi (128), P_ir = Ai Br (192).
            const int ap[4] = {0, 2, 0, 2}, bp[4] = {0, 2, 2, 0};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const uint32_t dq = d + q * BNP;
              const int ah = ap[q], bh = bp[q];
              tc::mma_f16(dq, A[ah + 1][0], B[bh][0], id, acc0);
              tc::mma_f16(dq, A[ah][0], B[bh + 1][0], id, 1);
              tc::mma_f16(dq, A[ah + 1][1], B[bh][1], id, 1);
              tc::mma_f16(dq, A[ah][1], B[bh + 1][1], id, 1);
              tc::mma_f16(dq, A[ah][0], B[bh][0], id, 1);
              tc::mma_f16(dq, A[ah][1], B[bh][1], id, 1);
            }
          }
          if constexpr (PAIR) {
            if (close) {
              tc::mma_commit_pair(&accf[set]);
              ++a;
            }
            tc::mma_commit_pair(&empty[s]);
          } else {
            if (close) {
              tc::mma_commit(&accf[set]);
              ++a;
            }
            tc::mma_commit(&empty[s]);
          }
        }
      }
      if (a > 0) {  // our own MMAs must complete before TMEM is freed
        const long last = a - 1;
        int zero = 0;
        if (!tc::mbar_wait(&accf[last & 1], (uint32_t)((last >> 1) & 1), &zero))
          atomicCAS(err, 0, tc::ERR_TIMEOUT_DRAIN);
      }
    }
  } else if (warp < 6) {
    // Drain warps.  All four run the same sequence of named barriers for every tile, so a
    // failed (timed-out) wait never leaves a warp behind at a barrier: failure is sticky,
    // skips the work, and raises the abort flag that ends every later wait at once.
    // Hand-off to the store warps: barrier 2 ("tile staged", drain arrives, store waits)
    // and barrier 3 ("buffer free", store arrives, drain waits before the next staging
    // and once after the last tile), one phase of each per tile on both sides.
    const int q = warp & 3;
    const int r = q * 32 + lane;
    const uint32_t lane_off = static_cast<uint32_t>(q * 32) << 16;
    long g = 0;   // drained partials, in the MMA warp's order
    bool ok = true;
    int ntile = 0;
    for (int t = t0; t < p.tiles; t += tstep, ++ntile) {
      int b, mt, nt;
      p.tile(t, b, mt, nt);
      float sre[BNP], sim[BNP];
#pragma unroll
      for (int c = 0; c < BNP; ++c) { sre[c] = 0.f; sim[c] = 0.f; }
      const int KC = kchunks_of(p, b);
      for (int kc = 0; kc < KC; kc += DC, ++g) {
        const int set = (int)(g & 1);
        const uint32_t use = (uint32_t)(g >> 1);
        if (ok && !tc::mbar_wait(&accf[set], use & 1, abort)) {
          if (lane == 0) atomicCAS(err, 0, tc::ERR_TIMEOUT_ACC);
          *abort = 1;
          ok = false;
        }
        if (!ok) continue;
        tc::fence_after_sync();
        const uint32_t d = tmem + lane_off + set * 4 * BNP;
        const float cf = chunk_factor(p, b, kc);
        // column blocks of P_rr, P_ii, P_ri, P_ir in the set
        constexpr int o_ii = PairB<P>::value ? 3 : 1, o_ri = PairB<P>::value ? 1 : 2, o_ir = PairB<P>::value ? 2 : 3;
        // DRAIN_COLS columns of two accumulators per load round
#pragma unroll
        for (int gq = 0; gq < BNP / DRAIN_COLS; ++gq) {
          float x[DRAIN_COLS], y[DRAIN_COLS];
          tc::tmem_ld<DRAIN_COLS>(d + 0 * BNP + gq * DRAIN_COLS, x);      // P_rr
          tc::tmem_ld<DRAIN_COLS>(d + o_ii * BNP + gq * DRAIN_COLS, y);   // P_ii
          tc::tmem_ld_wait();
#pragma unroll
          for (int c = 0; c < DRAIN_COLS; ++c) {
            const float v = P::kConjA ? x[c] + y[c] : x[c] - y[c];
            if constexpr (ChunkScaled<P>::value)
              sre[gq * DRAIN_COLS + c] = fmaf(cf, v, sre[gq * DRAIN_COLS + c]);
            else
              sre[gq * DRAIN_COLS + c] += v;
          }
          tc::tmem_ld<DRAIN_COLS>(d + o_ri * BNP + gq * DRAIN_COLS, x);   // P_ri
          tc::tmem_ld<DRAIN_COLS>(d + o_ir * BNP + gq * DRAIN_COLS, y);   // P_ir
          tc::tmem_ld_wait();
          // conj(a) b = (ar br + ai bi) + i (ar bi - ai br)
#pragma unroll
          for (int c = 0; c < DRAIN_COLS; ++c) {
            const float v = P::kConjA ? x[c] - y[c] : x[c] + y[c];
            if constexpr (ChunkScaled<P>::value)
              sim[gq * DRAIN_COLS + c] = fmaf(cf, v, sim[gq * DRAIN_COLS + c]);
            else
              sim[gq * DRAIN_COLS + c] += v;
          }
        }
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) {
          if (PAIR && !leader)
            tc::mbar_arrive_remote(tc::mapa_shared(tc::smem_u32(&acce[set]), 0));
          else
            tc::mbar_arrive(&acce[set]);
        }
      }
      if (ntile > 0) asm volatile("bar.sync 3, 256;" ::: "memory");   // previous tile stored
#pragma unroll
      for (int c = 0; c < BNP; ++c) tile_buf[r * STAGE_LD + c] = make_float2(sre[c], sim[c]);
      __threadfence_block();
      asm volatile("bar.arrive 2, 256;" ::: "memory");
    }
    if (ntile > 0) asm volatile("bar.sync 3, 256;" ::: "memory");
  } else {
    // Store warps: write each staged tile with the policy's own (coalesced) mapping.
    const int tid = threadIdx.x - 192, ew = warp - 6;
    for (int t = t0; t < p.tiles; t += tstep) {
      int b, mt, nt;
      p.tile(t, b, mt, nt);
      asm volatile("bar.sync 2, 256;" ::: "memory");
      if (!*abort) p.store_tile(b, PAIR ? 2 * mt + (int)rank : mt, nt, tile_buf, tid, ew, lane);
      __threadfence_block();
      asm volatile("bar.arrive 3, 256;" ::: "memory");
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  // pair form: the peer's copies, MMAs and remote arrivals are all done before either CTA
  // frees its tensor memory or exits
  if constexpr (PAIR) tc::cluster_sync();
  if (warp == 1) {
    tc::fence_after_sync();
    if constexpr (PAIR)
      tc::tmem_dealloc_pair(tmem, Lay::TMEM_COLS);
    else
      tc::tmem_dealloc(tmem, Lay::TMEM_COLS);
  }
}

// ---------------------------------------------------------------- tile lists of several problems
// The tiles of up to NMAX problems of one policy kind (the same GEMM of several systems) in one
// persistent launch: tile t belongs to the member i with start[i] <= t < start[i + 1], and every
// member keeps its own parameters, k chunks and tensor maps.  A member tile computes exactly
// what it computes in its own launch.  The tile index handed to the member's policy is packed
// with the member number (b = i << 20 | member tile group).
template <class P, int NMAX = 8>
struct GroupP {
  static constexpr bool kConjA = P::kConjA;
  static constexpr bool kPairB = PairB<P>::value;
  static constexpr bool kGrouped = true;
  static constexpr bool kStreamB = StreamB<P>::value;
  static constexpr int kStages = P::kStages;
  static_assert(!ChunkScaled<P>::value && DrainChunks<P>::value == 1, "plain policies only");
  int tiles, kchunks;   // kchunks unused: per member
  int n;
  int start[NMAX + 1];
  P m[NMAX];
  CUtensorMap ma[NMAX], mb[NMAX];
  __device__ void tile(int t, int& b, int& mt, int& nt) const {
    int i = 0;
    while (i + 1 < n && t >= start[i + 1]) ++i;
    int bl;
    m[i].tile(t - start[i], bl, mt, nt);
    b = (i << 20) | bl;
  }
  __device__ Coords coords(int b, int mt, int nt, int kc) const { return m[b >> 20].coords(b & 0xFFFFF, mt, nt, kc); }
  __device__ void store_tile(int b, int mt, int nt, const float2* tile, int tid, int ew, int lane) const {
    m[b >> 20].store_tile(b & 0xFFFFF, mt, nt, tile, tid, ew, lane);
  }
  __device__ int kchunks_of(int b) const { return m[b >> 20].kchunks; }
  __device__ bool stream_b_of(int b) const {
    if constexpr (StreamB<P>::value)
      return m[b >> 20].stream_b();
    else
      return false;
  }
  __device__ const CUtensorMap* map_a(int b) const { return &ma[b >> 20]; }
  __device__ const CUtensorMap* map_b(int b) const { return &mb[b >> 20]; }
};

// ---------------------------------------------------------------- host side
// 5-D fp16 tensor map with 64-byte swizzle.  dims[0] is the contiguous k
// extent (elements), strides are byte strides of dims 1..4, box[0] = 32.
struct MapSpec {
  uint64_t dims[5];
  uint64_t strides[4];
  uint32_t box[5];
};

cudaError_t make_map(CUtensorMap* map, void* base, const MapSpec& s);

template <int STAGES, class P>
cudaError_t launch_precise(const CUtensorMap& a, const CUtensorMap& b, const P& p, int* err, cudaStream_t st) {
  using Lay = LayoutP<STAGES>;
  auto fn = cgemm_precise_kernel<STAGES, P>;
  cudaError_t e = ensure_dyn_smem(reinterpret_cast<const void*>(fn), Lay::SMEM);
  if (e != cudaSuccess) return e;
  if (p.tiles <= 0) return cudaSuccess;
  int dev = 0, sms = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if (sms <= 0) sms = 1;
  const int grid = p.tiles < sms ? p.tiles : sms;
  fn<<<grid, THREADS, Lay::SMEM, st>>>(a, b, p, err);
  return cudaGetLastError();
}

// The pair form: clusters of two CTAs, p.tiles counting pairs of row tiles, `b` the B map whose
// box holds one of the two (re, im) halves of the paired B operand.
template <int STAGES, class P>
cudaError_t launch_precise_pair(const CUtensorMap& a, const CUtensorMap& b, const P& p, int* err, cudaStream_t st) {
  using Lay = LayoutP<STAGES, true>;
  auto fn = cgemm_precise_kernel<STAGES, P, true>;
  cudaError_t e = ensure_dyn_smem(reinterpret_cast<const void*>(fn), Lay::SMEM);
  if (e != cudaSuccess) return e;
  if (p.tiles <= 0) return cudaSuccess;
  int dev = 0, sms = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const int pairs = sms / 2 > 0 ? sms / 2 : 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2 * (p.tiles < pairs ? p.tiles : pairs));
  cfg.blockDim = dim3(THREADS);
  cfg.dynamicSmemBytes = Lay::SMEM;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, fn, a, b, p, err);
}

}  // namespace tcg
