// All-pairs shared k-mer counts on the tensor cores, streamed into the rank keys.
//
// S = P P^T over the threshold planes (see rank_prep.cu) is computed tile by tile
// with tcgen05.mma of kind::mxf4nvf4: the planes are packed e2m1 values that are
// exactly 0 or 1, every block scale is 1.0, and the products are accumulated in
// f32 in TMEM. Every product is 0 or 1 and every partial sum an integer
// <= min(m_i, m_j) <= 65535 < 2^24, so the accumulators hold S exactly. Only the
// upper triangle of the stored order is visited; each accumulator tile goes
// straight into the Eq. 1 / Eq. 3 sums and is never written out:
//
//   term_ij = floor(S_ij 2^64 / D_ij), D_ij = m_j for stored i <= j (rows are in
//   decreasing length), key_i += term_ij for i <= j and key_j += term_ij for i < j.
//
// Terms are split into 24-bit limbs; the row sums of a tile stay in registers,
// the column sums are reduced across the 32 lanes of a warp with a transposing
// shuffle tree, and both are added to per-sequence 64-bit limb accumulators
// (red.global.add.u64), which a last kernel folds into the 128-bit key.
//
// When the planes are cut at a depth D, the residual sum_tau max(0, min(c_i, c_j) - D)
// of each pair arrives as a dense 128 x 256 u16 block per tile and is added to S
// before the floor, so the key is the same as with all planes.
//
// Persistent kernel, one CTA per SM, 12 warps:
//   warp 0      TMA producer: 128 B (256 plane columns) of 128 rows of A (rows I)
//               and of 256 rows of B (rows J) per stage, 128-byte swizzle, 4-stage
//               mbarrier ring
//   warp 1      MMA issuer: per stage 4 K steps of two (M=128, N=128, K=64) MMAs,
//               one per half of the tile's columns, sharing the A operand; commit
//               frees the stage. A tile's halves go to two of three 128-column TMEM
//               regions used in turn, so the next tile can start once the epilogue
//               has drained the first half of this one
//   warp 2      TMEM allocator
//   warps 4-7   also fill the scale-factor columns of TMEM with 1.0 before the
//               first MMA
//   warps 4-11  epilogue: tcgen05.ld of the accumulator halves in turn (lane
//               quadrant = warp % 4, two warps per quadrant, 64 columns each)
// The third TMEM region lets the epilogue of one tile overlap the MMAs of the next. Every wait is bounded (globaltimer); on a timeout the CTA records
// SAD_ERR_TIMEOUT, drains its copies and MMAs in flight, frees TMEM and returns.
#include "rank.cuh"

#include <cudaTypedefs.h>

namespace sad {

namespace {

constexpr int kStages = 4;
constexpr uint32_t kABytes = kRowBlock * kKChunk;
constexpr uint32_t kBBytes = kColBlock * kKChunk;
constexpr uint32_t kTxBytes = kABytes + kBBytes;
constexpr int kThreads = 384;
constexpr int kEpiThreads = 256;  // warps 4-11: two per TMEM lane quadrant
constexpr uint32_t kTmemCols = 512;
constexpr int kHalf = 128;        // columns of one MMA (N) and of one TMEM region
constexpr int kRegions = 3;       // TMEM accumulator regions, used in turn by tile halves
// TMEM columns: regions [0, 3 x 128), then the scale factors of A and B
constexpr uint32_t kSfaCol = kRegions * kHalf;
constexpr uint32_t kSfbCol = kSfaCol + 32;
constexpr uint32_t kSfCols = 64;  // filled with 1.0
static_assert(kSfaCol + kSfCols <= kTmemCols, "TMEM columns");
static_assert(kColBlock == 2 * kHalf, "a tile is two MMA halves");
constexpr int kWarpCols = kHalf / 2;  // columns of a half for one epilogue warp
constexpr uint64_t kWaitBudgetNs = 2000000000ull;

struct GemmSmem {
  uint8_t a[kStages][kABytes];
  uint8_t b[kStages][kBBytes];
  // per tile column, in three buffers (tile lt uses lt % 3): the next tile's records
  // are staged while the previous tile's residual column sums are still being added
  uint4 colrec[3][kColBlock];     // division record
  uint2 colfl[3][kColBlock];      // floor(S r / d): (r | sh1 << 16 | sh2 << 24, magic)
  int32_t colorig[3][kColBlock];  // input index (-1 = padding)
  uint32_t colres[3][kColBlock];  // residual column sums of the floor-only halves
  uint64_t full[kStages];
  uint64_t empty[kStages];
  uint64_t rfull[kRegions];   // the MMAs into a region are done
  uint64_t rempty[kRegions];  // the epilogue has read a region
  uint64_t drain;
  uint32_t tmem_base;
  int32_t abort;
  int32_t skip;
  int32_t never;  // stays 0: the abort flag of the drain waits
};

constexpr size_t kGemmSmemBytes = sizeof(GemmSmem) + 1024;

__device__ __forceinline__ void red_add_u64(unsigned long long *p, unsigned long long v) {
  asm volatile("red.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Column sums of a 32 x 16 block held one row per lane (v[i] = column i): after
// the call v[0] of lane L is the sum over all 32 lanes of column L & 15.
__device__ __forceinline__ void transpose_reduce16(uint32_t (&v)[16], uint32_t lane) {
#pragma unroll
  for (int w = 8; w >= 1; w >>= 1) {
    const bool upper = (lane & (uint32_t)w) != 0;
#pragma unroll
    for (int i = 0; i < w; ++i) {
      const uint32_t send = upper ? v[i] : v[i + w];
      const uint32_t keep = upper ? v[i + w] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, w);
    }
  }
  v[0] += __shfl_xor_sync(0xffffffffu, v[0], 16);
}

__device__ __forceinline__ void tmem_ld_32x32b_x16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
        "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}

__device__ __forceinline__ void set_abort(GemmSmem &S, WsHeader *hdr) {
  *reinterpret_cast<volatile int32_t *>(&S.abort) = 1;
  record_error(hdr, SAD_ERR_TIMEOUT, (int)blockIdx.x);
}

__global__ void __launch_bounds__(kThreads, 1)
    plane_gemm_kernel(const __grid_constant__ CUtensorMap tmA,
                      const __grid_constant__ CUtensorMap tmB, RankPtrs P) {
  extern __shared__ uint8_t smem_raw[];
  GemmSmem &S = *reinterpret_cast<GemmSmem *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  volatile int32_t *abort_flag = &S.abort;

  if (threadIdx.x == 0) {
    S.abort = 0;
    S.never = 0;
    S.skip = (P.hdr->status != 0) ? 1 : 0;
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&S.full[s], 1);
      mbar_init(&S.empty[s], 1);
    }
    for (int a = 0; a < kRegions; ++a) {
      mbar_init(&S.rfull[a], 1);
      mbar_init(&S.rempty[a], kEpiThreads);
    }
    mbar_init(&S.drain, 1);
    fence_mbar_init();
  }
  if (warp == 0 && lane == 0) {
    tma_prefetch_desc(&tmA);
    tma_prefetch_desc(&tmB);
  }
  __syncthreads();
  const bool skip = S.skip != 0;
  if (!skip && warp == 2) {
    tmem_alloc(&S.tmem_base, kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = S.tmem_base;
  if (!skip && warp >= 4 && warp < 8) {
    // every block scale of A and B is 1.0: fill their columns in this warp's lanes
    const uint32_t lanes = ((warp & 3u) * 32u) << 16;
#pragma unroll
    for (uint32_t c = 0; c < kSfCols; c += 16) tmem_st_32x32b_x16_fill(tmem + lanes + kSfaCol + c, kScaleOne4);
    tmem_st_wait();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const int32_t n_tiles = skip ? 0 : P.hdr->n_tiles;
  // counts above the plane depth come in as dense per-tile residual blocks
  const bool residual =
      !skip && P.depth_cap >= 1 && P.block_cap > 0 && P.hdr->depth < P.hdr->t_max;

  if (!skip && warp == 0 && lane == 0) {
    // ------------------------------------------------------------ producer --
    int stage = 0;
    uint32_t phase = 0, used = 0, par = 0;
    bool aborted = false;
    for (int32_t t = blockIdx.x; t < n_tiles && !aborted; t += gridDim.x) {
      const int2 tl = P.tiles[t];
      const int32_t I = tl.x & 0xFFFF, J = tl.x >> 16, nk = tl.y;
      for (int32_t kc = 0; kc < nk; ++kc) {
        if (!mbar_wait_bounded(&S.empty[stage], phase ^ 1u, abort_flag, kWaitBudgetNs)) {
          set_abort(S, P.hdr);
          aborted = true;
          break;
        }
        mbar_arrive_expect_tx(&S.full[stage], kTxBytes);
        tma_load_2d(S.a[stage], &tmA, &S.full[stage], kc * kKChunk, I * kRowBlock);
        tma_load_2d(S.b[stage], &tmB, &S.full[stage], kc * kKChunk, J * kColBlock);
        used |= 1u << stage;
        par = (par & ~(1u << stage)) | (phase << stage);
        if (++stage == kStages) {
          stage = 0;
          phase ^= 1u;
        }
      }
    }
    if (aborted || *abort_flag) {
      // let every copy this thread started land before the CTA exits
      for (int s = 0; s < kStages; ++s)
        if (used & (1u << s))
          mbar_wait_bounded(&S.full[s], (par >> s) & 1u, &S.never, kWaitBudgetNs);
    }
  } else if (!skip && warp == 1 && lane == 0) {
    // ----------------------------------------------------------------- MMA --
    // Half-tile h = 2 lt + half goes to region h % 3, for the (h / 3)-th time.
    const uint32_t idesc = idesc_f4_e2m1(kRowBlock, kHalf);
    const uint32_t sfa = tmem + kSfaCol, sfb = tmem + kSfbCol;
    int stage = 0;
    uint32_t phase = 0;
    bool aborted = false;
    int32_t lt = 0;
    for (int32_t t = blockIdx.x; t < n_tiles && !aborted; t += gridDim.x, ++lt) {
      const int32_t nk = P.tiles[t].y;
      uint32_t reg[2];
      for (int hf = 0; hf < 2; ++hf) {
        const int32_t h = 2 * lt + hf;
        reg[hf] = (uint32_t)(h % kRegions);
        if (!mbar_wait_bounded(&S.rempty[reg[hf]], ((uint32_t)(h / kRegions) & 1u) ^ 1u,
                               abort_flag, kWaitBudgetNs)) {
          set_abort(S, P.hdr);
          aborted = true;
          break;
        }
      }
      if (aborted) break;
      tc_fence_after();
      const uint32_t d0 = tmem + reg[0] * (uint32_t)kHalf, d1 = tmem + reg[1] * (uint32_t)kHalf;
      for (int32_t kc = 0; kc < nk; ++kc) {
        if (!mbar_wait_bounded(&S.full[stage], phase, abort_flag, kWaitBudgetNs)) {
          set_abort(S, P.hdr);
          aborted = true;
          break;
        }
        tc_fence_after();
        const uint64_t adesc = sdesc_kmajor_sw128(smem_u32(S.a[stage]));
        const uint64_t bdesc0 = sdesc_kmajor_sw128(smem_u32(S.b[stage]));
        // rows 128..255 of B start 128 x 128 bytes further (16-byte descriptor units)
        const uint64_t bdesc1 = bdesc0 + (uint64_t)((kHalf * kKChunk) >> 4);
        // 4 K steps of 64 values = 32 bytes per row (2 in 16-byte descriptor units)
#pragma unroll
        for (int kk = 0; kk < kKChunk / 32; ++kk) {
          const uint32_t accum = (kc | kk) != 0 ? 1u : 0u;
          mma_f4(d0, adesc + 2u * kk, bdesc0 + 2u * kk, idesc, sfa, sfb, accum);
          mma_f4(d1, adesc + 2u * kk, bdesc1 + 2u * kk, idesc, sfa, sfb, accum);
        }
        mma_commit(&S.empty[stage]);
        if (++stage == kStages) {
          stage = 0;
          phase ^= 1u;
        }
      }
      if (aborted) break;
      mma_commit(&S.rfull[reg[0]]);
      mma_commit(&S.rfull[reg[1]]);
    }
    if (aborted || *abort_flag) {
      mma_commit(&S.drain);
      mbar_wait_bounded(&S.drain, 0, &S.never, kWaitBudgetNs);
    }
  } else if (!skip && warp >= 4 && warp < 12) {
    // ------------------------------------------------------------ epilogue --
    // Warp w reads TMEM lanes 32 (w % 4).. (its quadrant) and, of each half of the
    // tile, the columns [64 v, 64 v + 64), v = (w - 4) / 4, in sub-chunks of 16.
    //
    // A half whose columns lie in a later 128-row block than the tile's rows
    // (every i < j there, D_ij = m_j) adds only the floor parts floor(S_ij r_j / d_j)
    // to both keys; the linear parts S_ij Q_j of the planes come from rank_lin.cu,
    // and those of the residual R_ij (rare) are added here: R Q_j to the row, and
    // Q_j times the residual column sum (kept in shared memory, added to the keys
    // one tile later) to the column. A half on the rows' own block adds whole
    // terms, masked to i <= j (row) and i < j (column); a half on an earlier block
    // holds only pairs j < i, visited elsewhere, and is skipped.
    const uint32_t q = warp & 3;
    const uint32_t wv = (warp - 4) >> 2;
    const uint32_t etid = threadIdx.x - 128;
    for (uint32_t c = etid; c < 3u * kColBlock; c += kEpiThreads) (&S.colres[0][0])[c] = 0;
    int32_t lt = 0;
    bool have_prev = false;  // the previous tile's residual column sums wait
    bool aborted = false;
    for (int32_t t = blockIdx.x; t < n_tiles; t += gridDim.x, ++lt) {
      const int2 tl = P.tiles[t];
      const int32_t I = tl.x & 0xFFFF, J = tl.x >> 16;
      const int buf = lt % 3;
      for (uint32_t c = etid; c < (uint32_t)kColBlock; c += kEpiThreads) {
        const int64_t jpos = (int64_t)J * kColBlock + c;
        const uint4 rec = P.rec[jpos];
        S.colrec[buf][c] = rec;
        const uint32_t d = rec.w & 0xFFFFu;
        S.colfl[buf][c] = make_uint2(((0u - rec.x * d) & 0xFFFFu) | (rec.w & 0xFFFF0000u), rec.z);
        S.colorig[buf][c] = P.perm[jpos];
      }
      const int64_t row_pos = (int64_t)I * kRowBlock + q * 32 + lane;
      const int32_t row_orig = P.perm[row_pos];
      const int32_t rblk = residual ? P.block_of[t] : -1;
      // this row's residual words in the tile's block (two u16 per word)
      const uint32_t *rrow_base =
          rblk >= 0 ? P.rblocks + (int64_t)rblk * (kResidualBlockBytes / 4) +
                          (q * 32 + lane) * (kColBlock / 2)
                    : nullptr;
      {
        const int32_t h0 = 2 * lt;
        if (!mbar_wait_bounded(&S.rfull[h0 % kRegions], (uint32_t)(h0 / kRegions) & 1u,
                               abort_flag, kWaitBudgetNs))
          set_abort(S, P.hdr);
      }
      // column records staged, previous tile done; the abort decision is the same for
      // every epilogue thread
      aborted = named_bar_sync_or(1, kEpiThreads, *abort_flag != 0);
      if (aborted) break;
      if (have_prev) {
        // residual column sums of the previous tile: Q_j times the sum
        const int pb = (lt + 2) % 3;
        for (uint32_t c = etid; c < (uint32_t)kColBlock; c += kEpiThreads) {
          const uint32_t rs = S.colres[pb][c];
          if (rs == 0) continue;
          S.colres[pb][c] = 0;
          const int32_t jorig = S.colorig[pb][c];
          if (jorig < 0) continue;
          const uint4 rec = S.colrec[pb][c];
          const uint64_t Q = ((uint64_t)rec.y << 32) | rec.x;
          const uint64_t lo = Q * rs, hi = __umul64hi(Q, (uint64_t)rs);
          unsigned long long *dst = P.acc + 3 * (int64_t)jorig;
          red_add_u64(dst + 0, lo & 0xFFFFFFull);
          red_add_u64(dst + 1, (lo >> 24) & 0xFFFFFFull);
          red_add_u64(dst + 2, (lo >> 48) | (hi << 16));
        }
      }
      have_prev = true;
      uint32_t R0 = 0, R1 = 0, R2 = 0;  // row: 24-bit limb sums of whole terms and floors
      uint64_t L0 = 0, L1 = 0, L2 = 0;  // row: residual linear part R Q_j
      for (int hf = 0; hf < 2; ++hf) {
        const int32_t h = 2 * lt + hf;
        const uint32_t region = (uint32_t)(h % kRegions);
        if (hf == 1 && !mbar_wait_bounded(&S.rfull[region], (uint32_t)(h / kRegions) & 1u,
                                          abort_flag, kWaitBudgetNs))
          set_abort(S, P.hdr);
        tc_fence_after();
        const int32_t hb = 2 * J + hf;       // 128-row block of this half's columns
        const int cbase = hf * kHalf + (int)wv * kWarpCols;
        const uint32_t taddr = tmem + ((q * 32u) << 16) + region * (uint32_t)kHalf + wv * kWarpCols;
        const uint4 *rrow = rrow_base ? reinterpret_cast<const uint4 *>(rrow_base) + cbase / 8
                                      : nullptr;
        if (hb > I) {
#pragma unroll 1
          for (int sc = 0; sc < kWarpCols / 16; ++sc) {
            const int c0 = cbase + sc * 16;
            uint32_t v[16];
            tmem_ld_32x32b_x16(taddr + (uint32_t)(sc * 16), v);
            uint4 ra = make_uint4(0, 0, 0, 0), rb = make_uint4(0, 0, 0, 0);
            if (rrow) {
              ra = __ldg(rrow + 2 * sc);
              rb = __ldg(rrow + 2 * sc + 1);
            }
            tmem_ld_wait();
            const uint32_t rw[8] = {ra.x, ra.y, ra.z, ra.w, rb.x, rb.y, rb.z, rb.w};
            uint32_t cq[16];
#pragma unroll
            for (int cc = 0; cc < 16; ++cc) {
              const uint2 fl = S.colfl[buf][c0 + cc];
              const uint32_t res = (rw[cc >> 1] >> (16 * (cc & 1))) & 0xFFFFu;
              const uint32_t sv = __float2uint_rn(__uint_as_float(v[cc])) + res;
              // floor(s r / d) by Granlund & Montgomery: s r < 2^32
              const uint32_t xq = sv * (fl.x & 0xFFFFu);
              const uint32_t t1 = __umulhi(fl.y, xq);
              const uint32_t qv = (t1 + ((xq - t1) >> ((fl.x >> 16) & 0xFFu))) >> (fl.x >> 24);
              R0 += qv;
              cq[cc] = qv;
              if (res) {
                const uint4 rec = S.colrec[buf][c0 + cc];
                const uint64_t Q = ((uint64_t)rec.y << 32) | rec.x;
                const uint64_t lo = Q * res, hi = __umul64hi(Q, (uint64_t)res);
                L0 += lo & 0xFFFFFFull;
                L1 += (lo >> 24) & 0xFFFFFFull;
                L2 += (lo >> 48) | (hi << 16);
                atomicAdd(&S.colres[buf][c0 + cc], res);
              }
            }
            transpose_reduce16(cq, lane);
            if (lane < 16) {
              const int32_t jorig = S.colorig[buf][c0 + (int)lane];
              if (jorig >= 0 && cq[0] != 0) red_add_u64(P.acc + 3 * (int64_t)jorig, cq[0]);
            }
          }
        } else if (hb == I) {
#pragma unroll 1
          for (int sc = 0; sc < kWarpCols / 16; ++sc) {
            const int c0 = cbase + sc * 16;
            uint32_t v[16];
            tmem_ld_32x32b_x16(taddr + (uint32_t)(sc * 16), v);
            uint4 ra = make_uint4(0, 0, 0, 0), rb = make_uint4(0, 0, 0, 0);
            if (rrow) {
              ra = __ldg(rrow + 2 * sc);
              rb = __ldg(rrow + 2 * sc + 1);
            }
            tmem_ld_wait();
            const uint32_t rw[8] = {ra.x, ra.y, ra.z, ra.w, rb.x, rb.y, rb.z, rb.w};
            uint32_t cs[16], cq[16];
#pragma unroll
            for (int cc = 0; cc < 16; ++cc) {
              const uint4 rec = S.colrec[buf][c0 + cc];
              const uint32_t s = __float2uint_rn(__uint_as_float(v[cc])) +
                                 ((rw[cc >> 1] >> (16 * (cc & 1))) & 0xFFFFu);
              const uint32_t d = rec.w & 0xFFFFu;
              const uint32_t sh1 = (rec.w >> 16) & 0xFFu, sh2 = rec.w >> 24;
              // floor(s * 2^64 / d) = s * Q + floor(s * r / d), r = 2^64 - Q d
              const uint32_t r = 0u - rec.x * d;
              const uint32_t xq = s * r;
              const uint32_t t1 = __umulhi(rec.z, xq);
              const uint32_t qv = (t1 + ((xq - t1) >> sh1)) >> sh2;
              const uint64_t Q = ((uint64_t)rec.y << 32) | rec.x;
              const uint64_t lo = (uint64_t)s * Q;
              const uint64_t lo2 = lo + qv;
              const uint32_t hi = lo2 < lo ? 1u : 0u;
              const uint32_t wa = (uint32_t)lo2, wb = (uint32_t)(lo2 >> 32);
              uint32_t l0 = wa & 0xFFFFFFu;
              uint32_t l1 = (wa >> 24) | ((wb & 0xFFFFu) << 8);
              uint32_t l2 = (wb >> 16) | (hi << 16);
              uint32_t scv = s, qc = qv;
              const int64_t jpos = (int64_t)J * kColBlock + c0 + cc;
              if (row_pos > jpos) { l0 = 0; l1 = 0; l2 = 0; }
              if (row_pos >= jpos) { scv = 0; qc = 0; }
              R0 += l0;
              R1 += l1;
              R2 += l2;
              cs[cc] = scv;
              cq[cc] = qc;
            }
            transpose_reduce16(cs, lane);
            transpose_reduce16(cq, lane);
            if (lane < 16) {
              const int col = c0 + (int)lane;
              const int32_t jorig = S.colorig[buf][col];
              if (jorig >= 0 && (cs[0] | cq[0]) != 0) {
                const uint4 rec = S.colrec[buf][col];
                const uint64_t Q = ((uint64_t)rec.y << 32) | rec.x;
                const unsigned __int128 sum = (unsigned __int128)Q * cs[0] + cq[0];
                unsigned long long *dst = P.acc + 3 * (int64_t)jorig;
                red_add_u64(dst + 0, (unsigned long long)(sum & 0xFFFFFFu));
                red_add_u64(dst + 1, (unsigned long long)((sum >> 24) & 0xFFFFFFu));
                red_add_u64(dst + 2, (unsigned long long)(sum >> 48));
              }
            }
          }
        }
        tc_fence_before();
        mbar_arrive(&S.rempty[region]);
      }
      if (row_orig >= 0) {
        unsigned long long *dst = P.acc + 3 * (int64_t)row_orig;
        if (R0 | L0) red_add_u64(dst + 0, (unsigned long long)R0 + L0);
        if (R1 | L1) red_add_u64(dst + 1, (unsigned long long)R1 + L1);
        if (R2 | L2) red_add_u64(dst + 2, (unsigned long long)R2 + L2);
      }
    }
    if (have_prev && !aborted) {
      // the last tile's residual column sums
      named_bar_sync(1, kEpiThreads);
      const int pb = (lt + 2) % 3;  // lt is one past the last tile here
      for (uint32_t c = etid; c < (uint32_t)kColBlock; c += kEpiThreads) {
        const uint32_t rs = S.colres[pb][c];
        const int32_t jorig = S.colorig[pb][c];
        if (rs == 0 || jorig < 0) continue;
        const uint4 rec = S.colrec[pb][c];
        const uint64_t Q = ((uint64_t)rec.y << 32) | rec.x;
        const uint64_t lo = Q * rs, hi = __umul64hi(Q, (uint64_t)rs);
        unsigned long long *dst = P.acc + 3 * (int64_t)jorig;
        red_add_u64(dst + 0, lo & 0xFFFFFFull);
        red_add_u64(dst + 1, (lo >> 24) & 0xFFFFFFull);
        red_add_u64(dst + 2, (lo >> 48) | (hi << 16));
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (!skip && warp == 2) {
    tc_fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// The planes as bytes: n_pad rows of K_cap / 2 bytes (two 4-bit values each).
int make_plane_map(CUtensorMap *map, uint8_t *planes, int64_t n_pad, int64_t k_cap, int rows) {
  auto fn = encode_fn();
  if (!fn) return SAD_ERR_CUDA;
  const cuuint64_t dims[2] = {(cuuint64_t)(k_cap / 2), (cuuint64_t)n_pad};
  const cuuint64_t strides[1] = {(cuuint64_t)(k_cap / 2)};
  const cuuint32_t box[2] = {(cuuint32_t)kKChunk, (cuuint32_t)rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, planes, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? SAD_OK : SAD_ERR_CUDA;
}

}  // namespace

int rank_gemm_launch(const RankPtrs &P, cudaStream_t st) {
  const int64_t tiles = P.tiles_total;
  if (tiles == 0) return SAD_OK;
  CUtensorMap mA, mB;
  int rc = make_plane_map(&mA, P.planes, P.n_pad, P.k_cap, kRowBlock);
  if (rc) return rc;
  rc = make_plane_map(&mB, P.planes, P.n_pad, P.k_cap, kColBlock);
  if (rc) return rc;
  static bool attr_set = false;
  if (!attr_set) {
    if (cudaFuncSetAttribute(plane_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kGemmSmemBytes) != cudaSuccess)
      return SAD_ERR_CUDA;
    attr_set = true;
  }
  const int64_t grid = tiles < num_sms() ? tiles : num_sms();
  prof_begin(st);
  plane_gemm_kernel<<<(unsigned)grid, kThreads, kGemmSmemBytes, st>>>(mA, mB, P);
  SAD_LAUNCH_CHECK();
  prof_end(st);
  return SAD_OK;
}

}  // namespace sad
