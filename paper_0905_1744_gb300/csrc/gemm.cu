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
// The row sums of a tile stay in registers, the column sums are reduced across
// the 32 lanes of a warp (redux.sync, one per column); the square modes then meet
// the two column halves' row sums and the four lane quadrants' column sums in
// shared memory, so a tile adds one sum per row and per column: 128-bit, split as
// T mod 2^32 and T >> 32 into two 64-bit accumulators per sequence (similarity),
// or one signed 64-bit value (distance form), by red.global.add.u64; a last
// kernel folds them into the key.
//
// When the planes are cut (plans of depth >= 1), the tile's column block J lists
// per column v the threshold columns (tau, t) that v counts but that the tile's K
// chunks do not cover (its remainder entries, see rank_prep.cu). They are added on
// the tensor cores as extra K chunks of the tile: entry e becomes K column e of
// a chunk whose A row u holds [c_u(tau_e) >= t_e] (the remainder bitmap's bit of
// row u) and whose B row v holds [e is an entry of column v], so the MMA adds
// sum over v's entries of [c_u(tau) >= t] to S_uv. Two builder warps write these
// chunks into the operand ring (the 128-byte-swizzled K-major layout TMA writes)
// in place of a TMA copy. Counts above the bitmap's thresholds (heavy entries,
// rare) add min(c_u, c) - T_b in the epilogue from the counts. The key is the same
// as with all planes.
//
// Persistent kernel, one CTA per SM, 12 warps:
//   warp 0      TMA producer: per stage two K chunks of 256 plane columns (128 B)
//               of A (rows I) and of B (rows J), each operand one 3-D TMA request
//               that lands as two 128-row tiles with the 128-byte swizzle; a
//               3-stage mbarrier ring (64 KB a stage: the cost of a stage is
//               mostly fixed, so fewer, larger stages run faster)
//   warp 1      MMA issuer: 8 x (M=128, N=128, K=64) per stage into one of three
//               TMEM accumulators (3 x 128 columns), commit frees the stage
//   warp 2      TMEM allocator, then with warp 3 the remainder builder
//   warps 4-7   also fill the scale-factor columns of TMEM with 1.0 before the
//               first MMA
//   warps 4-11  epilogue: tcgen05.ld of the accumulator (lane quadrant = warp % 4,
//               two warps per quadrant, each on half of the 128 columns)
// A tile's remainder chunks are issued after the next tile's plane chunks (the
// builder prepares them meanwhile); the three TMEM accumulators let the epilogue of
// one tile overlap the MMAs of the next two.
//
// Every wait is bounded (globaltimer; the budget of the main-loop waits is
// P.wait_ns, 2 s unless a test shortens it); on a timeout the CTA records
// SAD_ERR_TIMEOUT, drains its copies and MMAs in flight (waits with the full 2 s
// budget), frees TMEM and returns.
#include "rank.cuh"

#include <cudaTypedefs.h>

namespace sad {

namespace {

// A stage holds two 256-column K chunks (two 128-byte-swizzled tiles per operand,
// one 3-D TMA request each).
constexpr int kStages = 3;
constexpr int32_t kCps = 2;  // K chunks per stage
constexpr uint32_t kSubA = kRowBlock * kKChunk, kSubB = kColBlock * kKChunk;
constexpr uint32_t kABytes = kSubA * kCps;
constexpr uint32_t kBBytes = kSubB * kCps;
constexpr uint32_t kTxBytes = kABytes + kBBytes;
constexpr int kThreads = 384;
constexpr int kEpiThreads = 256;  // warps 4-11: two per TMEM lane quadrant
constexpr uint32_t kTmemCols = 512;
// three accumulators: a tile's remainder chunks run after the next tile's plane
// chunks, and the epilogue of a tile overlaps the MMAs of the two after it
constexpr int kAccs = 3;
// TMEM columns: accumulators [0, 3 kColBlock), then the scale factors of A and B
constexpr uint32_t kSfaCol = kAccs * kColBlock;
constexpr uint32_t kSfbCol = kSfaCol + 32;
constexpr uint32_t kSfCols = 64;  // filled with 1.0
static_assert(kSfaCol + kSfCols <= kTmemCols, "TMEM columns");
constexpr int kHalfCols = kColBlock / 2;  // columns of one epilogue warp
// remainder entries of a column block staged in shared memory by the builder
// (larger lists are read from global memory)
constexpr int kRemStage = 832;
static_assert(kRemBudgetDefault <= kRemStage, "the default budget fits the staging");
constexpr int kRemChunk = 2 * kKChunk;  // remainder entries per extra K chunk (one per column)
constexpr int kBuildThreads = 64;       // warps 2-3
// budget of the drain waits after an abort (the copies and MMAs in flight finish
// in microseconds)
constexpr uint64_t kDrainBudgetNs = 2000000000ull;

struct GemmSmem {
  uint8_t a[kStages][kABytes];
  uint8_t b[kStages][kBBytes];
  uint4 colrec[2][kColBlock];
  int32_t colorig[2][kColBlock];
  int64_t collb[2][kColBlock];  // distance mode: ln_q(b d) of each tile column
  // square similarity mode: the four lane quadrants' column sums (s, floor) and the
  // second column half's row sums (Rlo, Rc), added once per tile
  uint2 colpart[2][4][kColBlock];
  uint4 rowpart[2][kRowBlock];
  // the builder's tile: first remainder entry of each column (relative to its
  // column block) and, when the block's list fits, the bitmap slice (4 words: bits
  // of the tile's 128 rows) of each entry
  int32_t remoff[kColBlock + 1];
  uint4 remsl[kRemStage];
  uint32_t nib[256];  // byte b -> eight 4-bit values, 1.0 (e2m1) where b has a 1 bit
  uint64_t full[kStages];
  uint64_t empty[kStages];
  uint64_t bfree[kStages];  // the producer hands a free slot to the builder
  uint64_t tfull[kAccs];
  uint64_t tempty[kAccs];
  uint64_t drain;
  uint32_t tmem_base;
  int32_t abort;
  int32_t skip;
  int32_t never;  // stays 0: the abort flag of the drain waits
};

constexpr size_t kGemmSmemBytes = sizeof(GemmSmem) + 1024;
static_assert(kGemmSmemBytes <= 232448, "227 KB of shared memory per CTA");

__device__ __forceinline__ void red_add_u64(unsigned long long *p, unsigned long long v) {
  asm volatile("red.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// T = hi 2^64 + lo (T < 2^72) into a key's limbs: acc0 += T mod 2^32, acc1 += T >> 32.
// A key takes fewer than 2^17 such adds, so acc1 < 2^57 and acc0 < 2^49.
__device__ __forceinline__ void red_key(unsigned long long *dst, uint64_t lo, uint64_t hi) {
  red_add_u64(dst, lo & 0xFFFFFFFFull);
  red_add_u64(dst + 1, (lo >> 32) | (hi << 32));
}

__device__ __forceinline__ void named_bar_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// acc += v as a 64-bit sum with its carries counted in c.
__device__ __forceinline__ void add_carry(uint64_t &acc, uint32_t &c, uint64_t v) {
  asm("add.cc.u64 %0, %0, %2;\n\taddc.u32 %1, %1, 0;" : "+l"(acc), "+r"(c) : "l"(v));
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

// Tile t of a launch: (row block I, column block J, plane K chunks nk, remainder
// K chunks nx). Square mode: the upper-triangle list of the rank. Rectangular mode
// (every stored row against the reference rows, RectArgs): all R x C blocks,
// column block major, no remainder.
__device__ __forceinline__ void tile_at(const RankPtrs &P, const RectArgs &X, int32_t rect_nk,
                                        int32_t t, int32_t &I, int32_t &J, int32_t &nk,
                                        int32_t &nx) {
  if (X.rec_ref) {
    I = t % X.row_blocks;
    J = t / X.row_blocks;
    nk = rect_nk;
    nx = 0;
  } else {
    const int2 tl = P.tiles[t];
    I = tl.x & 0xFFFF;
    J = tl.x >> 16;
    nk = tl.y & 0xFFFF;
    nx = (int32_t)((uint32_t)tl.y >> 16);
  }
}

// 32 x 32 bit transpose across a warp: lane l holds row l (bit b = column b); on
// return lane u holds column u (bit l = row l). Recursive swap of the off-diagonal
// blocks of 16, 8, 4, 2 and 1.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x, uint32_t lane) {
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {
    const uint32_t m = s == 16 ? 0x0000FFFFu
                     : s == 8  ? 0x00FF00FFu
                     : s == 4  ? 0x0F0F0F0Fu
                     : s == 2  ? 0x33333333u
                               : 0x55555555u;
    const uint32_t y = __shfl_xor_sync(0xffffffffu, x, s);
    x = (lane & (uint32_t)s) ? ((x & ~m) | ((y >> s) & m)) : ((x & m) | ((y << s) & ~m));
  }
  return x;
}

// Bits [a, b) of a 32-bit word (clipped to [0, 32)).
__device__ __forceinline__ uint32_t bit_range(int32_t a, int32_t b) {
  a = max(a, 0);
  b = min(b, 32);
  if (a >= b) return 0u;
  const uint32_t hi = b >= 32 ? 0xFFFFFFFFu : ((1u << b) - 1u);
  const uint32_t lo = a <= 0 ? 0u : ((1u << a) - 1u);
  return hi & ~lo;
}

// One remainder K chunk x (entries [256 x, 256 x + 256) of the column block's list,
// rn entries in all) as the operand tiles a (128 rows u of the tile) and b (128
// rows v = tile columns), 128 bytes a row, 16-byte unit j of row r at unit j ^ (r & 7)
// (the 128-byte swizzle). A unit holds 32 entries of one row as 4-bit values. Row u
// of a: the bitmap bits of the tile's rows, transposed 32 x 32 at a time per warp;
// row v of b: 1.0 for the entries of column v (a contiguous range).
//
// prep_chunk_a computes this builder thread's 16 units of a into registers (before
// the ring slot is free); store_chunk writes them and the thread's 16 units of b.
// Builder warp bw takes the units j = 2 i + bw of every lane quadrant q.
template <bool kCanStage, typename SmemT>
__device__ __forceinline__ void prep_chunk_a(const RankPtrs &P, const SmemT &S, int32_t x,
                                             int32_t rn, bool staged, int64_t rbase,
                                             int64_t bm_stride, int32_t I, uint32_t bt,
                                             uint32_t lane, uint4 (&ua)[16]) {
  const uint32_t bw = bt >> 5;
  uint32_t w[16];
  bool from_smem = false;
  if constexpr (kCanStage) from_smem = staged;
  if (from_smem) {
    if constexpr (kCanStage) {
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int32_t e = x * kRemChunk + (int32_t)((2 * i + bw) * 32 + lane);
          w[4 * i + q] = e < rn ? (&S.remsl[e].x)[q] : 0u;
        }
    }
  } else {
    uint32_t col[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int32_t e = x * kRemChunk + (int32_t)((2 * i + bw) * 32 + lane);
      col[i] = e < rn ? __ldg(P.rem + rbase + e) : 0xFFFFFFFFu;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int q = 0; q < 4; ++q)
        w[4 * i + q] = col[i] != 0xFFFFFFFFu
                           ? __ldg(P.bitmap + (int64_t)col[i] * bm_stride + (int64_t)I * 4 + q)
                           : 0u;
  }
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const uint32_t m = warp_transpose32(w[k], lane);  // bit l: entry 32 j + l, row 32 q + lane
    ua[k] = make_uint4(S.nib[m & 0xFF], S.nib[(m >> 8) & 0xFF], S.nib[(m >> 16) & 0xFF],
                       S.nib[m >> 24]);
  }
}

template <typename SmemT>
__device__ __forceinline__ void store_chunk(const SmemT &S, uint8_t *a, uint8_t *b,
                                            const uint4 (&ua)[16], int32_t x, uint32_t bt,
                                            uint32_t lane) {
  const uint32_t bw = bt >> 5;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const uint32_t j = 2 * i + bw;
#pragma unroll
    for (uint32_t q = 0; q < 4; ++q) {
      const uint32_t r = q * 32 + lane;
      *reinterpret_cast<uint4 *>(a + r * 128 + ((j ^ (r & 7)) * 16)) = ua[4 * i + q];
    }
  }
  // b: rows v, two per builder thread
#pragma unroll
  for (uint32_t v = bt; v < (uint32_t)kColBlock; v += kBuildThreads) {
    const int32_t lo = S.remoff[v] - x * kRemChunk, hi = S.remoff[v + 1] - x * kRemChunk;
#pragma unroll
    for (uint32_t j = 0; j < 8; ++j) {
      const uint32_t m = bit_range(lo - (int32_t)(32 * j), hi - (int32_t)(32 * j));
      *reinterpret_cast<uint4 *>(b + v * 128 + ((j ^ (v & 7)) * 16)) =
          make_uint4(S.nib[m & 0xFF], S.nib[(m >> 8) & 0xFF], S.nib[(m >> 16) & 0xFF],
                     S.nib[m >> 24]);
    }
  }
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Square similarity epilogue over 16 columns of this lane's accumulator row.
// colrec holds (Qlo, Qhi, Wlo, Whi) per column: Q = floor((2^64 - 1) / d) and the
// floor weight W of d = m_j, so term = s Q + floor(s W / 2^63) with s = S + the
// remainder r of the column. The row keeps sum s Qlo, sum s Qhi (each below 2^54 over 64 columns)
// and the sum of the floors; cs, cq get what the columns add (s and the floor).
// On a diagonal tile the row takes j >= i only and the columns j > i only.
template <bool kDiag, bool kInt = false>
__device__ __forceinline__ void f_block16(const uint32_t (&v)[16], const uint32_t (&rr)[16],
                                          const uint4 *colrec, int64_t row_pos, int64_t jpos0,
                                          uint64_t &sql, uint64_t &sqh, uint32_t &qsum,
                                          uint32_t (&cs)[16], uint32_t (&cq)[16]) {
#pragma unroll
  for (int cc = 0; cc < 16; ++cc) {
    const uint4 rec = colrec[cc];
    // the accumulator is an integer below 2^16: + 2^23 puts it in the low mantissa bits
    // (kInt: v holds the integers already)
    const uint32_t sv =
        kInt ? v[cc] : __float_as_uint(__fadd_rn(__uint_as_float(v[cc]), 8388608.0f)) - 0x4B000000u;
    const uint32_t s = sv + rr[cc];
    const uint32_t q = (uint32_t)(((uint64_t)s * rec.w + __umulhi(s, rec.z)) >> 31);
    uint32_t sr = s, qr = q, sc = s, qc = q;
    if constexpr (kDiag) {
      const int64_t jpos = jpos0 + cc;
      if (row_pos > jpos) { sr = 0; qr = 0; }
      if (row_pos >= jpos) { sc = 0; qc = 0; }
    }
    sql += (uint64_t)sr * rec.x;
    sqh += (uint64_t)sr * rec.y;
    qsum += qr;
    cs[cc] = sc;
    cq[cc] = qc;
  }
}

// Heavy remainder of S for this lane's row and the 16 tile columns c0..c0 + 15:
// for each heavy entry (tau, c) of column v, max(0, min(c_u(tau), c) - T_b) from
// the counts (the thresholds up to T_b come through the remainder chunks).
// The heavy remainder of one tile column v (global index) for this lane's row: for
// each heavy entry (tau, c) of v, max(0, min(c_u(tau), c) - T_b). h1 is the end of
// v's entries (the next column's first, or the block's count).
__device__ __noinline__ uint32_t heavy_of_column(const RankPtrs &P, int64_t hbase, int64_t v,
                                                 int32_t h1, int32_t row_x, int32_t tbits) {
  uint32_t r = 0;
  for (int32_t h = P.rowrem[2 * v + 1]; h < h1; ++h) {
    const int2 e = __ldg(P.heavy + hbase + h);
    const int32_t cu = row_x >= 0 ? __ldg(P.counts + (int64_t)row_x * P.eps + e.x) : 0;
    const int32_t x = min(cu, e.y) - tbits;
    r += x > 0 ? (uint32_t)x : 0u;
  }
  return r;
}

// kW: columns of the tile's column block (its remainder lists' block).
template <int kW = kColBlock>
__device__ __forceinline__ void tile_heavy(const RankPtrs &P, int32_t hn, int64_t hbase,
                                           int32_t row_x, int32_t tbits, int32_t J, int c0,
                                           uint32_t (&rr)[16]) {
#pragma unroll
  for (int cc = 0; cc < 16; ++cc) rr[cc] = 0;
  if (hn > 0) {
    const int64_t v0 = (int64_t)J * kW + c0;
#pragma unroll
    for (int cc = 0; cc < 16; ++cc) {
      const int32_t h0 = P.rowrem[2 * (v0 + cc) + 1];
      const int32_t h1 = (c0 + cc + 1 < kW) ? P.rowrem[2 * (v0 + cc + 1) + 1] : hn;
      for (int32_t h = h0; h < h1; ++h) {
        const int2 e = __ldg(P.heavy + hbase + h);
        const int32_t cu = row_x >= 0 ? __ldg(P.counts + (int64_t)row_x * P.eps + e.x) : 0;
        const int32_t x = min(cu, e.y) - tbits;
        rr[cc] += x > 0 ? (uint32_t)x : 0u;
      }
    }
  }
}

template <bool kDist>
__global__ void __launch_bounds__(kThreads, 1)
    plane_gemm_kernel(const __grid_constant__ CUtensorMap tmA,
                      const __grid_constant__ CUtensorMap tmB, RankPtrs P, RectArgs X,
                      DistArgs Z) {
  pdl_enter();
  extern __shared__ uint8_t smem_raw[];
  GemmSmem &S = *reinterpret_cast<GemmSmem *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  volatile int32_t *abort_flag = &S.abort;
  const uint64_t wait_ns = P.wait_ns;  // budget of the main-loop waits

  if (threadIdx.x == 0) {
    S.abort = 0;
    S.never = 0;
    S.skip = (P.hdr->status != 0) ? 1 : 0;
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&S.full[s], 1);
      mbar_init(&S.empty[s], 1);
      mbar_init(&S.bfree[s], 1);
    }
    for (int a = 0; a < kAccs; ++a) {
      mbar_init(&S.tfull[a], 1);
      mbar_init(&S.tempty[a], kEpiThreads);
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
  const bool rect = X.rec_ref != nullptr;
  // work units: reference tiles (rectangular mode) or the rank's tiles
  const int32_t n_tiles = skip ? 0 : (rect ? X.n_tiles : P.hdr->n_tiles);
  // rectangular mode: every tile runs all K_pad columns the rank preparation wrote
  const int32_t rect_nk = (rect && !skip) ? max(1, P.hdr->k_pad / kKCols) : 0;
  // counts the planes of a tile do not cover come from the remainder lists
  const bool residual = !skip && !rect && P.depth_cap >= 1;
  const int64_t bm_stride = P.n_pad / 32;
  const int32_t tbits = t_bits_of(min(P.depth_cap, kMaxPlaneDepth));

  if (!skip && warp == 0 && lane == 0) {
    // ------------------------------------------------------------ producer --
    // Position sequence of the CTA (shared with the MMA issuer and the builder): for
    // each of its tiles in turn, the tile's plane stages, then the remainder stages
    // of the tile before (after the last tile, its remainder stages).
    int stage = 0;
    uint32_t phase = 0, used = 0, par = 0;
    bool aborted = false;
    int32_t pnx = 0;  // remainder chunks of the previous tile
    for (int32_t t = blockIdx.x; !aborted; t += gridDim.x) {
      const bool have = t < n_tiles;
      int32_t I = 0, J = 0, nk = 0, nx = 0;
      if (have) tile_at(P, X, rect_nk, t, I, J, nk, nx);
      const int32_t sk = have ? (nk + kCps - 1) / kCps : 0;
      for (int32_t kc = 0; kc < sk + pnx; ++kc) {
        if (!mbar_wait_bounded(&S.empty[stage], phase ^ 1u, abort_flag, wait_ns)) {
          set_abort(S, P.hdr);
          aborted = true;
          break;
        }
        if (kc >= sk) {
          // a remainder stage: the slot is free; the builder fills it and arrives on
          // its full barrier (slots are handed over in order, one round at a time)
          mbar_arrive(&S.bfree[stage]);
          // the copy last made into this slot has been consumed: nothing to drain
          used &= ~(1u << stage);
        } else {
          mbar_arrive_expect_tx(&S.full[stage], kTxBytes);
          tma_load_3d(S.a[stage], &tmA, &S.full[stage], 0, I * kRowBlock, kc * kCps);
          tma_load_3d(S.b[stage], &tmB, &S.full[stage], 0, J * kColBlock, kc * kCps);
          used |= 1u << stage;
          par = (par & ~(1u << stage)) | (phase << stage);
        }
        if (++stage == kStages) {
          stage = 0;
          phase ^= 1u;
        }
      }
      if (!have) break;
      pnx = nx;
    }
    // let every copy this thread started land before the CTA exits (after a normal
    // run the MMAs have consumed them all and these waits return at once)
    for (int s = 0; s < kStages; ++s)
      if (used & (1u << s)) mbar_wait_bounded(&S.full[s], (par >> s) & 1u, &S.never, kDrainBudgetNs);
  } else if (!skip && warp == 1 && lane == 0) {
    // ----------------------------------------------------------------- MMA --
    // Tile lt accumulates in TMEM accumulator lt % 3: its plane stages, then (after the
    // next tile's plane stages) its remainder stages, then the commit to tfull.
    const uint32_t idesc = idesc_f4_e2m1(kRowBlock, kColBlock);
    const uint32_t sfa = tmem + kSfaCol, sfb = tmem + kSfbCol;
    int stage = 0;
    uint32_t phase = 0;
    bool aborted = false;
    int32_t pnx = 0;
    auto issue_stage = [&](uint32_t d_tmem, int nsub, bool first) {
      for (int sub = 0; sub < nsub; ++sub) {
        const uint64_t adesc = sdesc_kmajor_sw128(smem_u32(S.a[stage] + sub * kSubA));
        const uint64_t bdesc = sdesc_kmajor_sw128(smem_u32(S.b[stage] + sub * kSubB));
        // per K chunk 4 MMAs of K = 64 values = 32 bytes per row (2 in 16-byte
        // descriptor units)
#pragma unroll
        for (int kk = 0; kk < kKChunk / 32; ++kk)
          mma_f4(d_tmem, adesc + 2u * kk, bdesc + 2u * kk, idesc, sfa, sfb,
                 (first && sub == 0 && kk == 0) ? 0u : 1u);
      }
      mma_commit(&S.empty[stage]);
      if (++stage == kStages) {
        stage = 0;
        phase ^= 1u;
      }
    };
    int32_t lt = 0;
    for (int32_t t = blockIdx.x; !aborted; t += gridDim.x, ++lt) {
      const bool have = t < n_tiles;
      int32_t nx = 0;
      if (have) {
        int32_t I, J, nk;
        tile_at(P, X, rect_nk, t, I, J, nk, nx);
        const uint32_t acc = lt % kAccs, aph = (lt / kAccs) & 1;
        if (!mbar_wait_bounded(&S.tempty[acc], aph ^ 1u, abort_flag, wait_ns)) {
          set_abort(S, P.hdr);
          aborted = true;
          break;
        }
        tc_fence_after();
        const uint32_t d_tmem = tmem + acc * (uint32_t)kColBlock;
        const int32_t sk = (nk + kCps - 1) / kCps;
        for (int32_t kc = 0; kc < sk; ++kc) {
          if (!mbar_wait_bounded(&S.full[stage], phase, abort_flag, wait_ns)) {
            set_abort(S, P.hdr);
            aborted = true;
            break;
          }
          tc_fence_after();
          // a last chunk past the tile's extent is not used
          issue_stage(d_tmem, min(kCps, nk - kc * kCps), kc == 0);
        }
        if (aborted) break;
      }
      if (lt >= 1) {
        // the previous tile: its remainder chunks, then its accumulator is complete
        const uint32_t pacc = (lt - 1) % kAccs;
        for (int32_t x = 0; x < pnx; ++x) {
          if (!mbar_wait_bounded(&S.full[stage], phase, abort_flag, wait_ns)) {
            set_abort(S, P.hdr);
            aborted = true;
            break;
          }
          tc_fence_after();
          issue_stage(tmem + pacc * (uint32_t)kColBlock, 1, false);
        }
        if (aborted) break;
        mma_commit(&S.tfull[pacc]);
      }
      if (!have) break;
      pnx = nx;
    }
    // every MMA this thread issued has completed before TMEM is freed (after an
    // abort, and also when an epilogue gave up after this loop ended normally)
    mma_commit(&S.drain);
    mbar_wait_bounded(&S.drain, 0, &S.never, kDrainBudgetNs);
  } else if (!skip && (warp == 2 || warp == 3)) {
    // -------------------------------------------------------- remainder builder --
    // Walks the same position sequence as the producer. A tile's remainder lists are
    // staged and its first chunk prepared in registers while the next tile's plane
    // stages run; each remainder stage is handed over by the producer (bfree, after
    // the slot's previous contents were consumed), written here and released to the
    // MMA on the slot's full barrier. The hand-overs of one slot complete in order,
    // so their parity is tracked per slot (bpar); no copy in flight ever leaves
    // this role.
    const uint32_t bt = threadIdx.x - 64;
    for (uint32_t i = bt; i < 256; i += kBuildThreads) {
      uint32_t v = 0;
      for (int k = 0; k < 8; ++k) v |= ((i >> k) & 1u) * (kE2M1One << (4 * k));
      S.nib[i] = v;
    }
    named_bar_sync(3, kBuildThreads);
    int stage = 0;
    uint32_t bpar = 0;
    bool aborted = false;
    // the previous tile's remainder: chunks, list base and size, staged or not,
    // row block; its first chunk's A units prepared in ua
    int32_t pnx = 0, prn = 0, pI = 0;
    int64_t prbase = 0;
    bool pstaged = true;
    uint4 ua[16];
    for (int32_t t = blockIdx.x; !aborted; t += gridDim.x) {
      const bool have = t < n_tiles;
      int32_t I = 0, J = 0, nk = 0, nx = 0;
      if (have) {
        tile_at(P, X, rect_nk, t, I, J, nk, nx);
        stage = (stage + (nk + kCps - 1) / kCps) % kStages;
      }
      for (int32_t x = 0; x < pnx; ++x) {
        bool ok = true;
        if (bt == 0) {
          ok = mbar_wait_bounded(&S.bfree[stage], (bpar >> stage) & 1u, abort_flag, wait_ns);
          if (!ok) set_abort(S, P.hdr);
        }
        bpar ^= 1u << stage;
        if (named_bar_sync_or(3, kBuildThreads, !ok || *abort_flag != 0)) {
          aborted = true;
          break;
        }
        store_chunk(S, S.a[stage], S.b[stage], ua, x, bt, lane);
        // the tensor cores read the stage through the async proxy
        fence_proxy_async_smem();
        named_bar_sync(3, kBuildThreads);
        if (bt == 0) mbar_arrive(&S.full[stage]);
        if (++stage == kStages) stage = 0;
        if (x + 1 < pnx)
          prep_chunk_a<true>(P, S, x + 1, prn, pstaged, prbase, bm_stride, pI, bt, lane, ua);
      }
      if (!have || aborted) break;
      pnx = nx;
      if (nx > 0) {
        // this tile's lists replace the previous tile's (all of whose chunks are written)
        named_bar_sync(3, kBuildThreads);
        prbase = P.blkrem[2 * J];
        prn = (int32_t)(P.blkrem[2 * J + 2] - prbase);
        pstaged = prn <= kRemStage;
        pI = I;
        for (int c = (int)bt; c <= kColBlock; c += kBuildThreads)
          S.remoff[c] = c < kColBlock ? P.rowrem[2 * ((int64_t)J * kColBlock + c)] : prn;
        if (pstaged)
          for (int e = (int)bt; e < prn; e += kBuildThreads)
            S.remsl[e] = __ldg(reinterpret_cast<const uint4 *>(
                P.bitmap + (int64_t)__ldg(P.rem + prbase + e) * bm_stride + (int64_t)pI * 4));
        named_bar_sync(3, kBuildThreads);
        prep_chunk_a<true>(P, S, 0, prn, pstaged, prbase, bm_stride, pI, bt, lane, ua);
      }
    }
  } else if (!skip && warp >= 4 && warp < 12) {
    // ------------------------------------------------------------ epilogue --
    // warp w reads TMEM lanes 32 (w % 4).. (its quadrant) and tile columns
    // [64 h, 64 h + 64), h = (w - 4) / 4, in sub-chunks of 16 columns.
    const uint32_t q = warp & 3;
    const uint32_t half = (warp - 4) >> 2;
    const uint32_t etid = threadIdx.x - 128;
    int32_t lt = 0;
    for (int32_t t = blockIdx.x; t < n_tiles; t += gridDim.x, ++lt) {
      int32_t I, J, nk, nx;
      tile_at(P, X, rect_nk, t, I, J, nk, nx);
      const bool tile_ok = true;
      const int buf = lt & 1;
      for (uint32_t c = etid; c < (uint32_t)kColBlock; c += kEpiThreads) {
        const int64_t jpos = (int64_t)J * kColBlock + c;
        if (!kDist && !rect) {
          const uint4 rc = P.rec[jpos];
          const uint2 w = P.recw[jpos];
          S.colrec[buf][c] = make_uint4(rc.x, rc.y, w.x, w.y);
        } else {
          S.colrec[buf][c] = rect ? X.rec_ref[jpos] : P.rec[jpos];
        }
        S.colorig[buf][c] = rect ? 0 : P.perm[jpos];
        if constexpr (kDist)
          S.collb[buf][c] = Z.ln_table[(int64_t)Z.b * (int64_t)(P.rec[jpos].w & 0xFFFFu)];
      }
      const int64_t row_pos = (int64_t)I * kRowBlock + q * 32 + lane;
      const int32_t row_orig = tile_ok ? P.perm[row_pos] : -1;
      const bool diag = (int64_t)I * kRowBlock + kRowBlock - 1 >= (int64_t)J * kColBlock;
      // heavy remainder entries [hbase, hbase + hn) of the column block, grouped by
      // column; they read this row's count of their word
      int64_t hbase = 0;
      int32_t hn = 0;
      if (residual) {
        hbase = P.blkrem[2 * J + 1];
        hn = (int32_t)(P.blkrem[2 * J + 3] - hbase);
      }
      const int32_t row_x = hn > 0 ? P.perm[row_pos] : -1;
      const uint32_t acc = lt % kAccs, aph = (lt / kAccs) & 1;
      const bool got = mbar_wait_bounded(&S.tfull[acc], aph, abort_flag, wait_ns);
      if (!got) set_abort(S, P.hdr);
      // column records staged; the abort decision is the same for every epilogue thread
      if (named_bar_sync_or(1, kEpiThreads, *abort_flag != 0)) break;
      tc_fence_after();
      // similarity modes: the row's sum of terms = Rc 2^64 + Rlo (every term is below
      // 2^64 but for F = 1, where it is exactly 2^64: s = d)
      uint64_t Rlo = 0;
      uint32_t Rc = 0;
      int64_t Rd = 0;  // distance mode: the row's sum of q
      if (!tile_ok) {
        // pair mode, below the diagonal: computed, counted nowhere
      } else if (kDist && rect) {
        // distance mode against reference rows: D = min(m_i, m_r) per pair, row sums only,
        // reference columns past n_ref (padding) left out
        const uint32_t dr = P.rec[row_pos].w & 0xFFFFu;
#pragma unroll 1
        for (int sc = 0; sc < kHalfCols / 16; ++sc) {
          const int c0 = (int)half * kHalfCols + sc * 16;
          uint32_t v[16];
          tmem_ld_32x32b_x16(tmem + ((q * 32u) << 16) + acc * (uint32_t)kColBlock + (uint32_t)c0,
                             v);
          tmem_ld_wait();
          int64_t ta[16], tb[16];
#pragma unroll
          for (int cc = 0; cc < 16; ++cc) {
            const uint32_t s = __float2uint_rn(__uint_as_float(v[cc]));
            const uint32_t dc = S.colrec[buf][c0 + cc].w & 0xFFFFu;
            const uint32_t d = dr < dc ? dr : dc;
            ta[cc] = __ldg(Z.ln_table + (uint32_t)Z.b * d);
            tb[cc] = __ldg(Z.ln_table + (d + (uint32_t)Z.b * s));
          }
#pragma unroll
          for (int cc = 0; cc < 16; ++cc) {
            const int64_t jpos = (int64_t)J * kColBlock + c0 + cc;
            Rd += jpos < X.n_ref ? ta[cc] - tb[cc] : 0;
          }
        }
      } else if constexpr (kDist) {
        // Eq. 2 / Eq. 3 with Delta = 1/b: q_ij = ln_q(b m_j) - ln_q(m_j + b S_ij), i <= j
        // (D_ij = m_j in the stored order); signed 64-bit sums, the column sums
        // reduced as a low 24-bit part and a signed high part
#pragma unroll 1
        for (int sc = 0; sc < kHalfCols / 16; ++sc) {
          const int c0 = (int)half * kHalfCols + sc * 16;
          uint32_t v[16];
          tmem_ld_32x32b_x16(tmem + ((q * 32u) << 16) + acc * (uint32_t)kColBlock + (uint32_t)c0,
                             v);
          uint32_t rr[16];
          tile_heavy(P, hn, hbase, row_x, tbits, J, c0, rr);
          tmem_ld_wait();
          int64_t tv[16];
#pragma unroll
          for (int cc = 0; cc < 16; ++cc) {
            const uint32_t s = __float2uint_rn(__uint_as_float(v[cc])) + rr[cc];
            const uint32_t d = S.colrec[buf][c0 + cc].w & 0xFFFFu;
            tv[cc] = __ldg(Z.ln_table + (d + (uint32_t)Z.b * s));
          }
          uint32_t cl[16], ch[16];
#pragma unroll
          for (int cc = 0; cc < 16; ++cc) {
            const int64_t qd = S.collb[buf][c0 + cc] - tv[cc];
            const int64_t jpos = (int64_t)J * kColBlock + c0 + cc;
            // padding columns (no sequence) count nowhere: unlike F, d is not 0 at S = 0
            const bool real = S.colorig[buf][c0 + cc] >= 0;
            const bool in_row = real && (!diag || row_pos <= jpos);
            const bool in_col = !diag || row_pos < jpos;
            Rd += in_row ? qd : 0;
            const int64_t cv = in_col ? qd : 0;
            cl[cc] = (uint32_t)(cv & 0xFFFFFF);
            ch[cc] = (uint32_t)(int32_t)(cv >> 24);
          }
          // column sums over the warp's 32 rows (low parts below 2^29, signed high
          // parts), one warp-wide reduction per column, met in shared memory
          uint32_t mcl = 0, mch = 0;
#pragma unroll
          for (int cc = 0; cc < 16; ++cc) {
            const uint32_t a = __reduce_add_sync(0xffffffffu, cl[cc]);
            const uint32_t b = (uint32_t)__reduce_add_sync(0xffffffffu, (int32_t)ch[cc]);
            if (lane == (uint32_t)cc) {
              mcl = a;
              mch = b;
            }
          }
          if (lane < 16) S.colpart[buf][q][c0 + (int)lane] = make_uint2(mcl, mch);
        }
      } else if (rect) {
        // every pair counts for the row only; D = min(m_i, m_r): the record of the
        // shorter of the two
        const uint4 rrec = P.rec[row_pos];
        const uint32_t dr = rrec.w & 0xFFFFu;
#pragma unroll 1
        for (int sc = 0; sc < kHalfCols / 16; ++sc) {
          const int c0 = (int)half * kHalfCols + sc * 16;
          uint32_t v[16];
          tmem_ld_32x32b_x16(tmem + ((q * 32u) << 16) + acc * (uint32_t)kColBlock + (uint32_t)c0,
                             v);
          tmem_ld_wait();
#pragma unroll
          for (int cc = 0; cc < 16; ++cc) {
            const uint4 crec = S.colrec[buf][c0 + cc];
            const uint4 rec = dr <= (crec.w & 0xFFFFu) ? rrec : crec;
            const uint32_t s = __float2uint_rn(__uint_as_float(v[cc]));
            const uint32_t d = rec.w & 0xFFFFu;
            const uint32_t sh1 = (rec.w >> 16) & 0xFFu, sh2 = rec.w >> 24;
            const uint32_t r = 0u - rec.x * d;
            const uint32_t xq = s * r;
            const uint32_t t1 = __umulhi(rec.z, xq);
            const uint32_t qv = (t1 + ((xq - t1) >> sh1)) >> sh2;
            const uint64_t Q = ((uint64_t)rec.y << 32) | rec.x;
            const uint64_t lo = (uint64_t)s * Q;
            const uint64_t lo2 = lo + qv;
            add_carry(Rlo, Rc, lo2);
            Rc += lo2 < lo ? 1u : 0u;
          }
        }
      } else {
      uint64_t sql = 0, sqh = 0;  // sum s Qlo, sum s Qhi
      uint32_t qsum = 0;          // sum floor(s W / 2^63)
#pragma unroll 1
      for (int sc = 0; sc < kHalfCols / 16; ++sc) {
        const int c0 = (int)half * kHalfCols + sc * 16;
        uint32_t v[16];
        tmem_ld_32x32b_x16(tmem + ((q * 32u) << 16) + acc * (uint32_t)kColBlock + (uint32_t)c0,
                           v);
        uint32_t rr[16];
        tile_heavy(P, hn, hbase, row_x, tbits, J, c0, rr);
        tmem_ld_wait();
        uint32_t cs[16], cq[16];
        if (diag)
          f_block16<true>(v, rr, &S.colrec[buf][c0], row_pos, (int64_t)J * kColBlock + c0, sql,
                          sqh, qsum, cs, cq);
        else
          f_block16<false>(v, rr, &S.colrec[buf][c0], row_pos, 0, sql, sqh, qsum, cs, cq);
        // column sums over the warp's 32 rows: one warp-wide reduction per column
        uint32_t mcs = 0, mcq = 0;
#pragma unroll
        for (int cc = 0; cc < 16; ++cc) {
          const uint32_t a = __reduce_add_sync(0xffffffffu, cs[cc]);
          const uint32_t b = __reduce_add_sync(0xffffffffu, cq[cc]);
          if (lane == (uint32_t)cc) {
            mcs = a;
            mcq = b;
          }
        }
        if (lane < 16) S.colpart[buf][q][c0 + (int)lane] = make_uint2(mcs, mcq);
      }
      {
        // the row's sum of terms sql + sqh 2^32 + qsum as Rc 2^64 + Rlo
        const uint64_t a = sql + (sqh << 32);
        const uint64_t b = a + qsum;
        Rlo = b;
        Rc = (uint32_t)(sqh >> 32) + (a < sql ? 1u : 0u) + (b < a ? 1u : 0u);
      }
      }
      tc_fence_before();
      mbar_arrive(&S.tempty[acc]);
      if (kDist && !rect) {
        // square distance form: as below, with one signed 64-bit sum per row and column
        if (tile_ok && half == 1)
          S.rowpart[buf][q * 32 + lane] =
              make_uint4((uint32_t)(uint64_t)Rd, (uint32_t)((uint64_t)Rd >> 32), 0u, 0u);
        named_bar_sync(2, kEpiThreads);
        if (tile_ok && half == 0) {
          if (row_orig >= 0) {
            const uint4 o = S.rowpart[buf][q * 32 + lane];
            const int64_t tot = Rd + (int64_t)(((uint64_t)o.y << 32) | o.x);
            red_add_u64(P.acc + 3 * (int64_t)row_orig, (unsigned long long)tot);
          }
        } else if (tile_ok) {
          const int c = (int)etid - kRowBlock;  // half 1: one column each
          const int32_t jorig = S.colorig[buf][c];
          int64_t tot = 0;
#pragma unroll
          for (int qq = 0; qq < 4; ++qq) {
            const uint2 v2 = S.colpart[buf][qq][c];
            tot += (int64_t)(int32_t)v2.y * (int64_t)(1 << 24) + (int64_t)v2.x;
          }
          if (jorig >= 0 && tot != 0)
            red_add_u64(P.acc + 3 * (int64_t)jorig, (unsigned long long)tot);
        }
      } else if (!kDist && !rect) {
        // square similarity: the row sums of the two column halves and the column
        // sums of the four lane quadrants meet in shared memory; then half 0 adds
        // one row each and half 1 one column each to the keys
        if (tile_ok && half == 1)
          S.rowpart[buf][q * 32 + lane] = make_uint4((uint32_t)Rlo, (uint32_t)(Rlo >> 32), Rc, 0u);
        named_bar_sync(2, kEpiThreads);
        if (tile_ok && half == 0) {
          if (row_orig >= 0) {
            const uint4 o = S.rowpart[buf][q * 32 + lane];
            const uint64_t lo = Rlo + (((uint64_t)o.y << 32) | o.x);
            const uint64_t hi = (uint64_t)Rc + o.z + (lo < Rlo ? 1u : 0u);
            red_key(P.acc + 3 * (int64_t)row_orig, lo, hi);
          }
        } else if (tile_ok) {
          const int c = (int)etid - kRowBlock;  // half 1: one column each
          const int32_t jorig = S.colorig[buf][c];
          uint32_t cs = 0, cq = 0;
#pragma unroll
          for (int qq = 0; qq < 4; ++qq) {
            const uint2 v2 = S.colpart[buf][qq][c];
            cs += v2.x;
            cq += v2.y;
          }
          if (jorig >= 0 && (cs | cq) != 0) {
            const uint4 rec = S.colrec[buf][c];
            const uint64_t Q = ((uint64_t)rec.y << 32) | rec.x;
            const unsigned __int128 sum = (unsigned __int128)Q * cs + cq;
            red_key(P.acc + 3 * (int64_t)jorig, (uint64_t)sum, (uint64_t)(sum >> 64));
          }
        }
      } else if (row_orig >= 0) {
        unsigned long long *dst = P.acc + 3 * (int64_t)row_orig;
        if constexpr (kDist)
          red_add_u64(dst, (unsigned long long)Rd);
        else
          red_key(dst, Rlo, Rc);
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

// ------------------------------------------------------------- CTA pairs ----
// 256 x 256 tiles on clusters of two CTAs (tcgen05 cta_group::2, M = 256): CTA r of
// the pair holds the 128 rows 256 I + 128 r of A and the 128 rows 256 J + 128 r of
// B, one K chunk (256 plane columns) a stage, and the lanes of its 128 rows of the
// 128 x 256 accumulator in its TMEM; the even CTA issues the MMAs for both. Per
// MMA cycle a CTA takes in half the operand bytes of a one-CTA 128 x 128 tile.
// One accumulator (256 columns; the scale factors need the rest of TMEM): the
// epilogue drains it into registers (packed 16-bit counts) and releases it before
// the arithmetic, so the next tile's MMAs wait only for the drain. A tile's
// remainder chunks go through two buffers of their own (not the operand ring), so
// the builder writes them while the tile's plane chunks run. Everything else is
// as in plane_gemm_kernel: rows in decreasing length, D_ij = m_j, the same term
// arithmetic, sums per row and column of a tile, bounded waits.
namespace pairk {

constexpr int kStages = 4;                               // one K chunk a stage
constexpr uint32_t kSub = kRowBlock * kKChunk;           // 16 KB: 128 rows x 128 bytes
constexpr uint32_t kTx = 2 * kSub;                       // A and B bytes of one CTA
constexpr int kXSlots = 2;                               // remainder chunk buffers
constexpr int kThreads = 384;
constexpr int kEpiThreads = 256;                         // warps 4-11
constexpr int kEpiWarps = kEpiThreads / 32;
constexpr int kCols = 2 * kColBlock;                     // tile columns (N = 256)
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kSfaCol = kCols, kSfbCol = kCols + 32, kSfCols = 64;
static_assert(kSfaCol + kSfCols <= kTmemCols, "TMEM columns");

struct Smem {
  uint8_t a[kStages][kSub];
  uint8_t b[kStages][kSub];
  uint8_t xa[kXSlots][kSub];
  uint8_t xb[kXSlots][kSub];
  uint4 colrec[2][kCols];
  int32_t colorig[2][kCols];
  uint2 colpart[4][kCols];  // the four lane quadrants' column sums (s, floor)
  uint4 rowpart[kRowBlock];  // the second column half's row sums
  int32_t remoff[kColBlock + 1];
  uint32_t nib[256];
  uint64_t full[kStages];    // the even CTA's count the copies of both CTAs
  uint64_t empty[kStages];
  uint64_t xfull[kXSlots];   // the even CTA's: one arrival from each CTA's builder
  uint64_t xempty[kXSlots];
  uint64_t tfull;
  uint64_t tempty;           // the even CTA's: one arrival per epilogue warp of both CTAs
  uint64_t drain;
  uint32_t tmem_base;
  int32_t abort;
  int32_t skip;
  int32_t never;
};
constexpr size_t kSmemBytes = sizeof(Smem) + 1024;
static_assert(kSmemBytes <= 232448, "227 KB of shared memory per CTA");

__device__ __forceinline__ void set_abort(Smem &S, WsHeader *hdr) {
  *reinterpret_cast<volatile int32_t *>(&S.abort) = 1;
  record_error(hdr, SAD_ERR_TIMEOUT, (int)blockIdx.x);
}

}  // namespace pairk

__global__ void __launch_bounds__(pairk::kThreads, 1)
    pair_gemm_kernel(const __grid_constant__ CUtensorMap tm, RankPtrs P) {
  pdl_enter();
  extern __shared__ uint8_t smem_raw[];
  pairk::Smem &S = *reinterpret_cast<pairk::Smem *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  volatile int32_t *abort_flag = &S.abort;
  const uint64_t wait_ns = P.wait_ns;
  const uint32_t crank = cluster_ctarank();
  const bool leader = crank == 0;
  const int32_t unit0 = (int32_t)cluster_id_x(), ustride = (int32_t)cluster_count_x();

  if (threadIdx.x == 0) {
    S.abort = 0;
    S.never = 0;
    S.skip = (P.hdr->status != 0) ? 1 : 0;
    for (int s = 0; s < pairk::kStages; ++s) {
      mbar_init(&S.full[s], 1);
      mbar_init(&S.empty[s], 1);
    }
    for (int x = 0; x < pairk::kXSlots; ++x) {
      mbar_init(&S.xfull[x], 2);
      mbar_init(&S.xempty[x], 1);
    }
    mbar_init(&S.tfull, 1);
    mbar_init(&S.tempty, 2 * pairk::kEpiWarps);
    mbar_init(&S.drain, 1);
    fence_mbar_init();
  }
  if (warp == 0 && lane == 0) tma_prefetch_desc(&tm);
  __syncthreads();
  const bool skip = S.skip != 0;
  // the allocation is a collective of both CTAs, whatever either decides
  if (warp == 2) {
    tmem_alloc_pair(&S.tmem_base, pairk::kTmemCols);
    tmem_relinquish_pair();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = S.tmem_base;
  if (warp >= 4 && warp < 8) {
    // every block scale of A and B is 1.0: fill their columns in this warp's lanes
    const uint32_t lanes = ((warp & 3u) * 32u) << 16;
#pragma unroll
    for (uint32_t c = 0; c < pairk::kSfCols; c += 16)
      tmem_st_32x32b_x16_fill(tmem + lanes + pairk::kSfaCol + c, kScaleOne4);
    tmem_st_wait();
  }
  tc_fence_before();
  __syncthreads();
  // both CTAs' barriers and TMEM are ready before either uses the other's
  cluster_sync_all();
  tc_fence_after();
  const int32_t n_tiles = skip ? 0 : P.hdr->n_tiles;
  const bool residual = !skip && P.depth_cap >= 1;
  const int64_t bm_stride = P.n_pad / 32;
  const int32_t tbits = t_bits_of(min(P.depth_cap, kMaxPlaneDepth));
  const RectArgs X{};

  if (!skip && warp == 0 && lane == 0) {
    // ------------------------------------------------------------ producer --
    // both CTAs count their copies on the even CTA's full barrier, which expects
    // the bytes of both
    int stage = 0;
    uint32_t phase = 0, used = 0, par = 0;
    bool aborted = false;
    for (int32_t p = unit0; p < n_tiles && !aborted; p += ustride) {
      int32_t I2, J2, nk, nx;
      tile_at(P, X, 0, p, I2, J2, nk, nx);
      for (int32_t kc = 0; kc < nk; ++kc) {
        if (!mbar_wait_bounded_cluster(&S.empty[stage], phase ^ 1u, abort_flag, wait_ns)) {
          pairk::set_abort(S, P.hdr);
          aborted = true;
          break;
        }
        if (leader) mbar_arrive_expect_tx(&S.full[stage], 2 * pairk::kTx);
        const uint32_t fb = mapa_shared(&S.full[stage], 0);
        tma_load_3d_pair(S.a[stage], &tm, fb, 0, (2 * I2 + (int32_t)crank) * kRowBlock, kc);
        tma_load_3d_pair(S.b[stage], &tm, fb, 0, (2 * J2 + (int32_t)crank) * kRowBlock, kc);
        used |= 1u << stage;
        par = (par & ~(1u << stage)) | (phase << stage);
        if (++stage == pairk::kStages) {
          stage = 0;
          phase ^= 1u;
        }
      }
    }
    if (aborted || *abort_flag) {
      if (leader) {
        // the even CTA's full barriers count the copies of both CTAs
        for (int s = 0; s < pairk::kStages; ++s)
          if (used & (1u << s))
            mbar_wait_bounded(&S.full[s], (par >> s) & 1u, &S.never, kDrainBudgetNs);
      } else {
        // this CTA cannot see its copies land: give them time (they take microseconds)
        const uint64_t t0 = globaltimer_ns();
        while (globaltimer_ns() - t0 < 200000ull) {
        }
      }
    }
  } else if (!skip && warp == 1 && lane == 0 && leader) {
    // ----------------------------------------------------------------- MMA --
    const uint32_t idesc = idesc_f4_e2m1(2 * kRowBlock, pairk::kCols);
    const uint32_t sfa = tmem + pairk::kSfaCol, sfb = tmem + pairk::kSfbCol;
    int stage = 0;
    uint32_t phase = 0;
    uint32_t xcount = 0;
    bool aborted = false;
    int32_t lt = 0;
    for (int32_t p = unit0; p < n_tiles && !aborted; p += ustride, ++lt) {
      int32_t I2, J2, nk, nx;
      tile_at(P, X, 0, p, I2, J2, nk, nx);
      if (!mbar_wait_bounded_cluster(&S.tempty, (lt & 1) ^ 1u, abort_flag, wait_ns)) {
        pairk::set_abort(S, P.hdr);
        aborted = true;
        break;
      }
      tc_fence_after();
      for (int32_t kc = 0; kc < nk; ++kc) {
        if (!mbar_wait_bounded_cluster(&S.full[stage], phase, abort_flag, wait_ns)) {
          pairk::set_abort(S, P.hdr);
          aborted = true;
          break;
        }
        tc_fence_after();
        const uint64_t adesc = sdesc_kmajor_sw128(smem_u32(S.a[stage]));
        const uint64_t bdesc = sdesc_kmajor_sw128(smem_u32(S.b[stage]));
#pragma unroll
        for (int kk = 0; kk < kKChunk / 32; ++kk)
          mma_f4_pair(tmem, adesc + 2u * kk, bdesc + 2u * kk, idesc, sfa, sfb,
                      (kc | kk) != 0 ? 1u : 0u);
        mma_commit_pair(&S.empty[stage], 0x3);
        if (++stage == pairk::kStages) {
          stage = 0;
          phase ^= 1u;
        }
      }
      if (aborted) break;
      for (int32_t x = 0; x < nx; ++x, ++xcount) {
        const uint32_t xs = xcount % pairk::kXSlots, xph = (xcount / pairk::kXSlots) & 1u;
        if (!mbar_wait_bounded_cluster(&S.xfull[xs], xph, abort_flag, wait_ns)) {
          pairk::set_abort(S, P.hdr);
          aborted = true;
          break;
        }
        tc_fence_after();
        const uint64_t adesc = sdesc_kmajor_sw128(smem_u32(S.xa[xs]));
        const uint64_t bdesc = sdesc_kmajor_sw128(smem_u32(S.xb[xs]));
#pragma unroll
        for (int kk = 0; kk < kKChunk / 32; ++kk)
          mma_f4_pair(tmem, adesc + 2u * kk, bdesc + 2u * kk, idesc, sfa, sfb, 1u);
        mma_commit_pair(&S.xempty[xs], 0x3);
      }
      if (aborted) break;
      mma_commit_pair(&S.tfull, 0x3);
    }
    // every MMA into either CTA's TMEM, reading either CTA's shared memory, completes
    mma_commit_pair(&S.drain, 0x1);
    mbar_wait_bounded(&S.drain, 0, &S.never, kDrainBudgetNs);
  } else if (!skip && (warp == 2 || warp == 3)) {
    // -------------------------------------------------------- remainder builder --
    // Each CTA writes its halves of a tile's remainder chunks into the chunk buffers:
    // A rows = its 128 rows, B rows = its 128 of the tile's 256 columns. A buffer is
    // written once the MMAs that read it last have completed (xempty, committed to
    // both CTAs) and released to the even CTA's MMA issuer on xfull.
    const uint32_t bt = threadIdx.x - 64;
    for (uint32_t i = bt; i < 256; i += kBuildThreads) {
      uint32_t v = 0;
      for (int k = 0; k < 8; ++k) v |= ((i >> k) & 1u) * (kE2M1One << (4 * k));
      S.nib[i] = v;
    }
    named_bar_sync(3, kBuildThreads);
    uint32_t xcount = 0;
    bool aborted = false;
    for (int32_t p = unit0; p < n_tiles && !aborted; p += ustride) {
      int32_t I2, J2, nk, nx;
      tile_at(P, X, 0, p, I2, J2, nk, nx);
      if (nx == 0) continue;
      const int64_t rbase = P.blkrem[2 * J2];
      const int32_t rn = (int32_t)(P.blkrem[2 * J2 + 2] - rbase);
      const int32_t I = 2 * I2 + (int32_t)crank;
      const int64_t v0 = (int64_t)J2 * pairk::kCols + (int64_t)crank * kColBlock;
      // first entry of each of this CTA's columns, relative to the column block
      for (int c = (int)bt; c <= kColBlock; c += kBuildThreads)
        S.remoff[c] = (crank == 0 || c < kColBlock) ? P.rowrem[2 * (v0 + c)] : rn;
      named_bar_sync(3, kBuildThreads);
      for (int32_t x = 0; x < nx; ++x, ++xcount) {
        const uint32_t xs = xcount % pairk::kXSlots, xph = (xcount / pairk::kXSlots) & 1u;
        uint4 ua[16];
        prep_chunk_a<false>(P, S, x, rn, false, rbase, bm_stride, I, bt, lane, ua);
        bool ok = true;
        if (bt == 0) {
          ok = mbar_wait_bounded_cluster(&S.xempty[xs], xph ^ 1u, abort_flag, wait_ns);
          if (!ok) pairk::set_abort(S, P.hdr);
        }
        if (named_bar_sync_or(3, kBuildThreads, !ok || *abort_flag != 0)) {
          aborted = true;
          break;
        }
        store_chunk(S, S.xa[xs], S.xb[xs], ua, x, bt, lane);
        // the tensor cores read the buffer through the async proxy
        fence_proxy_async_smem();
        named_bar_sync(3, kBuildThreads);
        if (bt == 0) {
          if (leader)
            mbar_arrive(&S.xfull[xs]);
          else
            mbar_arrive_cluster(mapa_shared(&S.xfull[xs], 0));
        }
      }
      // the next tile's offsets overwrite remoff
      named_bar_sync(3, kBuildThreads);
    }
  } else if (!skip && warp >= 4 && warp < 12) {
    // ------------------------------------------------------------ epilogue --
    // warp w: TMEM lanes 32 (w % 4).. (its quadrant of this CTA's 128 rows) and tile
    // columns [128 h, 128 h + 128), h = (w - 4) / 4: drained into 64 registers of
    // two 16-bit counts, then summed in sub-chunks of 16 columns.
    const uint32_t q = warp & 3;
    const uint32_t half = (warp - 4) >> 2;
    const uint32_t etid = threadIdx.x - 128;
    int32_t lt = 0;
    for (int32_t p = unit0; p < n_tiles; p += ustride, ++lt) {
      int32_t I2, J2, nk, nx;
      tile_at(P, X, 0, p, I2, J2, nk, nx);
      const int buf = lt & 1;
      const int32_t I = 2 * I2 + (int32_t)crank;
      for (uint32_t c = etid; c < (uint32_t)pairk::kCols; c += pairk::kEpiThreads) {
        const int64_t jpos = (int64_t)J2 * pairk::kCols + c;
        const uint4 rc = P.rec[jpos];
        const uint2 w = P.recw[jpos];
        S.colrec[buf][c] = make_uint4(rc.x, rc.y, w.x, w.y);
        S.colorig[buf][c] = P.perm[jpos];
      }
      const int64_t row_pos = (int64_t)I * kRowBlock + q * 32 + lane;
      const int32_t row_orig = P.perm[row_pos];
      const bool diag = I2 == J2;
      int64_t hbase = 0;
      int32_t hn = 0;
      if (residual) {
        hbase = P.blkrem[2 * J2 + 1];
        hn = (int32_t)(P.blkrem[2 * J2 + 3] - hbase);
      }
      const int32_t row_x = hn > 0 ? row_orig : -1;
      const bool got = mbar_wait_bounded_cluster(&S.tfull, lt & 1, abort_flag, wait_ns);
      if (!got) pairk::set_abort(S, P.hdr);
      if (named_bar_sync_or(1, pairk::kEpiThreads, *abort_flag != 0)) break;
      tc_fence_after();
      // drain this thread's 128 accumulator columns: two rounds of four loads, one wait
      // each (the next tile's MMAs wait for this drain)
      uint32_t pk[64];
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        uint32_t v[4][16];
#pragma unroll
        for (int u = 0; u < 4; ++u)
          tmem_ld_32x32b_x16(tmem + ((q * 32u) << 16) + half * 128u + (uint32_t)((4 * hh + u) * 16),
                             v[u]);
        tmem_ld_wait();
#pragma unroll
        for (int u = 0; u < 4; ++u) {
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const uint32_t a =
                __float_as_uint(__fadd_rn(__uint_as_float(v[u][2 * j]), 8388608.0f));
            const uint32_t b =
                __float_as_uint(__fadd_rn(__uint_as_float(v[u][2 * j + 1]), 8388608.0f));
            // the counts are below 2^16: the low mantissa halves of a and b
            pk[(4 * hh + u) * 8 + j] = __byte_perm(a, b, 0x5410);
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        if (leader)
          mbar_arrive(&S.tempty);
        else
          mbar_arrive_cluster(mapa_shared(&S.tempty, 0));
      }
      if (hn > 0) {
        // heavy remainder entries (rare): added to the counts (S + heavy <= min(m_i, m_j)
        // < 2^16, so each half stays within its 16 bits)
        const int64_t vb = (int64_t)J2 * pairk::kCols + half * 128;
#pragma unroll
        for (int j = 0; j < 64; ++j) {
          const int c = (int)half * 128 + 2 * j;
          const int32_t e1 = P.rowrem[2 * (vb + 2 * j + 1) + 1];
          const int32_t e2 = c + 2 < pairk::kCols ? P.rowrem[2 * (vb + 2 * j + 2) + 1] : hn;
          const uint32_t lo = heavy_of_column(P, hbase, vb + 2 * j, e1, row_x, tbits);
          const uint32_t hi = heavy_of_column(P, hbase, vb + 2 * j + 1, e2, row_x, tbits);
          pk[j] += lo | (hi << 16);
        }
      }
      uint64_t sql = 0, sqh = 0;  // sum s Qlo, sum s Qhi
      uint32_t qsum = 0;          // sum floor(s W / 2^63)
#pragma unroll
      for (int sc = 0; sc < 8; ++sc) {
        const int c0 = (int)half * 128 + sc * 16;
        uint32_t v[16];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          v[2 * j] = pk[sc * 8 + j] & 0xFFFFu;
          v[2 * j + 1] = pk[sc * 8 + j] >> 16;
        }
        uint32_t rr[16];
#pragma unroll
        for (int cc = 0; cc < 16; ++cc) rr[cc] = 0;
        uint32_t cs[16], cq[16];
        if (diag)
          f_block16<true, true>(v, rr, &S.colrec[buf][c0], row_pos, (int64_t)J2 * pairk::kCols + c0, sql,
                                sqh, qsum, cs, cq);
        else
          f_block16<false, true>(v, rr, &S.colrec[buf][c0], row_pos, 0, sql, sqh, qsum, cs, cq);
        // column sums over the warp's 32 rows: one warp-wide reduction per column
        uint32_t mcs = 0, mcq = 0;
#pragma unroll
        for (int cc = 0; cc < 16; ++cc) {
          const uint32_t a = __reduce_add_sync(0xffffffffu, cs[cc]);
          const uint32_t b = __reduce_add_sync(0xffffffffu, cq[cc]);
          if (lane == (uint32_t)cc) {
            mcs = a;
            mcq = b;
          }
        }
        if (lane < 16) S.colpart[q][c0 + (int)lane] = make_uint2(mcs, mcq);
      }
      // the row's sum of terms sql + sqh 2^32 + qsum as Rc 2^64 + Rlo
      const uint64_t ra = sql + (sqh << 32);
      const uint64_t Rlo = ra + qsum;
      const uint32_t Rc = (uint32_t)(sqh >> 32) + (ra < sql ? 1u : 0u) + (Rlo < ra ? 1u : 0u);
      if (half == 1)
        S.rowpart[q * 32 + lane] = make_uint4((uint32_t)Rlo, (uint32_t)(Rlo >> 32), Rc, 0u);
      named_bar_sync(2, pairk::kEpiThreads);
      if (half == 0 && row_orig >= 0) {
        const uint4 o = S.rowpart[q * 32 + lane];
        const uint64_t lo = Rlo + (((uint64_t)o.y << 32) | o.x);
        const uint64_t hi = (uint64_t)Rc + o.z + (lo < Rlo ? 1u : 0u);
        red_key(P.acc + 3 * (int64_t)row_orig, lo, hi);
      }
      {
        // one column of the 256 per epilogue thread: the four quadrants' sums
        const int c = (int)etid;
        const int32_t jorig = S.colorig[buf][c];
        uint32_t cs = 0, cq = 0;
#pragma unroll
        for (int qq = 0; qq < 4; ++qq) {
          const uint2 v2 = S.colpart[qq][c];
          cs += v2.x;
          cq += v2.y;
        }
        if (jorig >= 0 && (cs | cq) != 0) {
          const uint4 rec = S.colrec[buf][c];
          const uint64_t Q = ((uint64_t)rec.y << 32) | rec.x;
          const unsigned __int128 sum = (unsigned __int128)Q * cs + cq;
          red_key(P.acc + 3 * (int64_t)jorig, (uint64_t)sum, (uint64_t)(sum >> 64));
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  // every MMA into either CTA's TMEM, reading either CTA's shared memory, is done
  cluster_sync_all();
  if (warp == 2) {
    tc_fence_after();
    tmem_dealloc_pair(tmem, pairk::kTmemCols);
  }
}

}  // namespace

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
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

// The planes as bytes: n_pad rows of K_cap / 2 bytes (two 4-bit values each); a box
// is `chunks` K chunks of `rows` rows.
int make_plane_map(CUtensorMap *map, uint8_t *planes, int64_t n_pad, int64_t k_cap, int rows,
                   int chunks) {
  auto fn = encode_fn();
  if (!fn) return SAD_ERR_CUDA;
  // (byte in chunk, row, chunk): a box of kCps chunks lands as kCps row-major tiles
  const cuuint64_t dims[3] = {(cuuint64_t)kKChunk, (cuuint64_t)n_pad,
                              (cuuint64_t)(k_cap / 2 / kKChunk)};
  const cuuint64_t strides[2] = {(cuuint64_t)(k_cap / 2), (cuuint64_t)kKChunk};
  const cuuint32_t box[3] = {(cuuint32_t)kKChunk, (cuuint32_t)rows, (cuuint32_t)chunks};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, planes, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? SAD_OK : SAD_ERR_CUDA;
}

namespace {
int gemm_attr() {
  static bool attr_set = false;
  if (!attr_set) {
    if (cudaFuncSetAttribute(plane_gemm_kernel<false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kGemmSmemBytes) != cudaSuccess ||
        cudaFuncSetAttribute(plane_gemm_kernel<true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kGemmSmemBytes) != cudaSuccess)
      return SAD_ERR_CUDA;
    attr_set = true;
  }
  return SAD_OK;
}

}  // namespace

namespace {
// Largest number of co-resident clusters of two for the pair kernel (0: none).
int pair_clusters() {
  static int cached = -1;
  if (cached < 0) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)(2 * num_sms()), 1, 1);
    cfg.blockDim = dim3(pairk::kThreads, 1, 1);
    cfg.dynamicSmemBytes = pairk::kSmemBytes;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, pair_gemm_kernel, &cfg) != cudaSuccess) {
      (void)cudaGetLastError();
      n = 0;
    }
    cached = n;
  }
  return cached;
}

// One set on CTA pairs: the 256 x 256 tiles of the plan (P.tile == 256).
int rank_gemm_pair_launch(const RankPtrs &P, cudaStream_t st) {
  const int64_t tiles = P.tiles_total;
  if (tiles == 0) return SAD_OK;
  static bool attr_set = false;
  if (!attr_set) {
    if (cudaFuncSetAttribute(pair_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)pairk::kSmemBytes) != cudaSuccess)
      return SAD_ERR_CUDA;
    attr_set = true;
  }
  const int ncl = pair_clusters();
  if (ncl < 1) return SAD_ERR_UNSUPPORTED;
  CUtensorMap m;  // 128-row boxes of one K chunk: A and B rows of either CTA
  int rc = make_plane_map(&m, P.planes, P.n_pad, P.k_cap, kRowBlock, 1);
  if (rc) return rc;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  // Always every co-resident cluster, whatever the number of tiles (clusters without
  // a tile exit after setting up): the grid of this launch then never changes between
  // batches, so a CUDA graph that recorded it can be updated in place for another
  // batch (an in-place update did not grow the grid of this cluster launch beyond
  // the instantiated one, which left the extra tiles uncomputed).
  cfg.gridDim = dim3((unsigned)(2 * ncl), 1, 1);
  cfg.blockDim = dim3(pairk::kThreads, 1, 1);
  cfg.dynamicSmemBytes = pairk::kSmemBytes;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  prof_begin(st);
  if (cudaLaunchKernelEx(&cfg, pair_gemm_kernel, m, P) != cudaSuccess) {
    (void)cudaGetLastError();
    return SAD_ERR_CUDA;
  }
  note_launch();
  prof_end(st);
  return SAD_OK;
}
}  // namespace

int rank_gemm_launch(const RankPtrs &P, cudaStream_t st) {
  if (P.tile == 2 * kRowBlock) return rank_gemm_pair_launch(P, st);
  const int64_t tiles = P.tiles_total;
  if (tiles == 0) return SAD_OK;
  CUtensorMap mA, mB;
  int rc = make_plane_map(&mA, P.planes, P.n_pad, P.k_cap, kRowBlock, kCps);
  if (rc) return rc;
  rc = make_plane_map(&mB, P.planes, P.n_pad, P.k_cap, kColBlock, kCps);
  if (rc) return rc;
  if ((rc = gemm_attr())) return rc;
  const int64_t grid = tiles < num_sms() ? tiles : num_sms();
  prof_begin(st);
  pdl_launch(plane_gemm_kernel<false>, (unsigned)grid, kThreads, kGemmSmemBytes, st, mA, mB, P,
             RectArgs{}, DistArgs{});
  SAD_LAUNCH_CHECK();
  prof_end(st);
  return SAD_OK;
}

int rank_dist_gemm_launch(const RankPtrs &P, const int64_t *ln_table, int32_t b,
                          cudaStream_t st) {
  const int64_t tiles = P.tiles_total;
  if (tiles == 0) return SAD_OK;
  CUtensorMap mA, mB;
  int rc = make_plane_map(&mA, P.planes, P.n_pad, P.k_cap, kRowBlock, kCps);
  if (rc) return rc;
  rc = make_plane_map(&mB, P.planes, P.n_pad, P.k_cap, kColBlock, kCps);
  if (rc) return rc;
  if ((rc = gemm_attr())) return rc;
  DistArgs Z;
  Z.ln_table = ln_table;
  Z.b = b;
  const int64_t grid = tiles < num_sms() ? tiles : num_sms();
  pdl_launch(plane_gemm_kernel<true>, (unsigned)grid, kThreads, kGemmSmemBytes, st, mA, mB, P,
             RectArgs{}, Z);
  SAD_LAUNCH_CHECK();
  return SAD_OK;
}

int rank_rect_gemm_launch(const RankPtrs &P, uint8_t *ref_planes, const uint4 *rec_ref,
                          int64_t ref_rows, int32_t n_ref, const int64_t *ln_table, int32_t b,
                          cudaStream_t st) {
  RectArgs X;
  X.rec_ref = rec_ref;
  X.n_ref = n_ref;
  X.row_blocks = (int32_t)(P.n_pad / kRowBlock);
  const int64_t tiles = (int64_t)X.row_blocks * (ref_rows / kColBlock);
  if (tiles == 0) return SAD_OK;
  if (tiles > 0x7FFFFFFF) return SAD_ERR_UNSUPPORTED;
  X.n_tiles = (int32_t)tiles;
  CUtensorMap mA, mB;
  int rc = make_plane_map(&mA, P.planes, P.n_pad, P.k_cap, kRowBlock, kCps);
  if (rc) return rc;
  rc = make_plane_map(&mB, ref_planes, ref_rows, P.k_cap, kColBlock, kCps);
  if (rc) return rc;
  if ((rc = gemm_attr())) return rc;
  const int64_t grid = tiles < num_sms() ? tiles : num_sms();
  if (ln_table) {
    DistArgs Z;
    Z.ln_table = ln_table;
    Z.b = b;
    pdl_launch(plane_gemm_kernel<true>, (unsigned)grid, kThreads, kGemmSmemBytes, st, mA, mB, P,
               X, Z);
  } else {
    pdl_launch(plane_gemm_kernel<false>, (unsigned)grid, kThreads, kGemmSmemBytes, st, mA, mB, P,
               X, DistArgs{});
  }
  SAD_LAUNCH_CHECK();
  return SAD_OK;
}

}  // namespace sad
