// Internal definitions shared by the libsad translation units: workspace
// layouts, device-side status recording, launch bookkeeping and the inline-PTX
// wrappers for mbarrier, TMA (cp.async.bulk.tensor) and tcgen05 (5th-generation
// tensor cores with TMEM accumulators) on sm_103a.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

#include "../../include/sad.h"

namespace sad {

// ---------------------------------------------------------------- limits ----
constexpr int kMaxEps = 65536;          // words per count vector
constexpr int kMaxM = 65535;            // k-mers per sequence (L - k + 1)
constexpr int kMaxP = 4096;             // buckets
constexpr int kRowBlock = 128;          // GEMM tile rows (A operand, M)
constexpr int kColBlock = 128;          // GEMM tile columns (B operand, N)
constexpr int kColRatio = kColBlock / kRowBlock;  // row blocks per column block
constexpr int kKChunk = 128;            // K bytes of a chunk (one 128B swizzle row)
constexpr int kKCols = 2 * kKChunk;     // plane columns per K chunk: two 4-bit values a byte
constexpr int kNPad = 128;              // rows are padded to a multiple of this
// row blocks of one plane matrix: the tile list packs a tile's blocks as I | J << 16
// in an int32 and reads J back with a signed shift, so J stays below 2^15
constexpr int64_t kMaxRowBlocks = 0x7FFF;
static_assert(kColBlock % kRowBlock == 0 && kNPad % kColBlock == 0, "tile shapes");

constexpr size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// --------------------------------------------------------- workspace hdr ----
// The first 256 bytes of every workspace.
// Plane depth. A rank plan of depth D >= 1 keeps the threshold sections
// 1..min(D, t_max) (at most kMaxPlaneDepth) as planes; what the planes of a tile
// do not cover comes from the remainder lists (see rank_prep.cu).
constexpr int kMaxPlaneDepth = 8;
// thresholds above the plane depth that the remainder's bitmap still holds; counts
// beyond (kTabDepth at most) are remainder entries of their own kind (heavy)
constexpr int kBitExtra = 4;
// (threshold, word) -> column table rows
constexpr int kTabDepth = 16;
// per-row remainder profile: entries by the first depth d* that covers them
// (1..D, D + 1 = none), then the heavy entries
constexpr int kProf = kMaxPlaneDepth + 2;
// default remainder budget: entries per column block the GEMM epilogue stages
constexpr int kRemBudgetDefault = 768;

struct WsHeader {
  int32_t status;        // first recorded sad_status (0 = none)
  int32_t detail;        // optional detail of the error (e.g. offending index)
  int64_t k_eff;         // plane columns of the kept sections (kmer_rank)
  int32_t k_pad;         // k_eff rounded up to kKCols
  int32_t t_max;         // largest count of any word in any sequence
  int32_t n_tiles;       // GEMM tiles scheduled
  int32_t depth;         // threshold sections kept as planes (t_max when nothing is cut)
  unsigned long long k_chunks;  // sum over tiles of their K chunks (executed MMA work)
  int64_t list_total;    // (sequence, word) entries counted twice or more
  int64_t rem_bound;     // plan: sum over those of min(c, T_b) - 1 (remainder entries bound)
  int64_t heavy_total;   // plan: entries counted more than T_b times
  int32_t bm_cols;       // bitmap columns: (word, threshold) with 2 <= t <= T_b
  int32_t m_max;         // largest m = L - k + 1 of the set
  unsigned long long flat_count;  // entries appended by the plane kernel
  int64_t rem_entries;   // remainder entries in use (bitmap columns listed per row)
  int64_t heavy_entries; // heavy remainder entries in use
  int32_t t_bits;        // T_b: largest threshold held in the bitmap
  int32_t rem_blocks;    // column blocks whose plane depth is below their largest count
  int32_t dmin;          // smallest plane depth of any column block
  int32_t bm_lo;         // lowest plane column that can be a remainder column
  int32_t pad[36];
};
static_assert(sizeof(WsHeader) == 256, "header is 256 bytes");

__device__ __forceinline__ void record_error(WsHeader *h, int code, int detail = 0) {
  if (atomicCAS(&h->status, 0, code) == 0) h->detail = detail;
}

// Item of the partition: a rank key and its input index.
struct Item {
  uint64_t hi, lo;
  int32_t idx;
  int32_t pad;
};

__host__ __device__ __forceinline__ bool item_less(const Item &a, const Item &b) {
  if (a.hi != b.hi) return a.hi < b.hi;
  if (a.lo != b.lo) return a.lo < b.lo;
  return a.idx < b.idx;
}

// Capacities of the data-dependent regions of a rank workspace.
struct RankCaps {
  int32_t depth;         // plane depth D; 0 = all sections, no remainder
  int32_t budget;        // remainder entries per column block (0 = kRemBudgetDefault)
  int32_t tile;          // GEMM tile rows: 128 (one CTA a tile) or 256 (CTA pairs)
  int64_t k_cap;         // plane columns
  int64_t list_cap;      // entries (sequence, word) counted twice or more
  int64_t rem_cap;       // remainder entries (bitmap columns)
  int64_t heavy_cap;     // heavy remainder entries
  int64_t bm_cols;       // bitmap columns
};

// Largest threshold the remainder bitmap holds for a plan of depth D >= 1.
__host__ __device__ constexpr int32_t t_bits_of(int32_t depth) {
  return depth + kBitExtra < kTabDepth ? depth + kBitExtra : kTabDepth;
}

// One set of a (possibly batched) rank call, built on the device by rank_setup.
// Sets are consecutive in the input order; each set's stored rows are a
// contiguous range of the global plane matrix aligned to the GEMM tile (128 or
// 256 rows), so every GEMM tile stays inside one set (the batch is block-diagonal).
struct RankSet {
  int64_t seq_begin;     // first input sequence of the set
  int64_t row_base;      // first stored row (multiple of the tile rows)
  int64_t tile_base;     // first entry of the set's tiles in the tile list
  int64_t tileof_base;   // first entry of the set's (I, J) -> tile map
  int32_t n, pad;
};

// Sizes of a rank call that the host knows before launching.
struct RankShape {
  int64_t n_sets, n_total, rows_total, tiles_total, tileof_total;
};

inline int64_t n_pad_of(int64_t n, int64_t align = kNPad) {
  return (int64_t)align_up((size_t)(n > 0 ? n : 1), (size_t)align);
}

// Upper-triangle tiles of a set of n rows in square tiles of B rows.
inline int64_t tiles_of_set(int64_t n, int64_t B = kRowBlock) {
  const int64_t R = (n + B - 1) / B;
  return R * (R + 1) / 2;
}

// One more set of n sequences; with tile = 256 (CTA pairs) its rows are padded to 256
// and its tiles are the 256 x 256 tiles of its upper triangle.
inline void shape_add_set(RankShape &sh, int64_t n, int64_t tile = kRowBlock) {
  const int64_t np = n_pad_of(n, tile);
  sh.n_sets += 1;
  sh.n_total += n;
  sh.rows_total += np;
  sh.tiles_total += tiles_of_set(n, tile);
  sh.tileof_total += (np / kRowBlock) * (np / kColBlock);
}

inline RankShape shape_single(int64_t n, int64_t tile = kRowBlock) {
  RankShape sh{0, 0, 0, 0, 0};
  shape_add_set(sh, n, tile);
  return sh;
}

// Offsets of the rank workspace regions (bytes from the workspace base).
struct RankLayout {
  size_t sets, seq_set, row_set, T, secend, thist, coltab, dstar, mhist, perm, rec, recw,
      depth, bdepth, tiles, acc, prof, rowrem, blkrem, cursor, sortbuf, scanblk, colmap, flat,
      rem, heavy, planes, bitmap;
  size_t fixed_bytes;    // everything that does not depend on the capacities
  size_t bytes;          // total
  RankShape shape;
  RankCaps caps;
};

inline RankLayout rank_layout(const RankShape &sh, int64_t eps, const RankCaps &caps) {
  RankLayout L{};
  L.shape = sh;
  L.caps = caps;
  size_t o = sizeof(WsHeader);
  auto take = [&](size_t bytes) { size_t r = o; o = align_up(o + bytes, 256); return r; };
  auto nz = [](int64_t x) { return (size_t)(x > 0 ? x : 1); };
  const size_t blocks = nz(sh.rows_total / kRowBlock);
  L.sets = take(sizeof(RankSet) * nz(sh.n_sets));
  L.seq_set = take(sizeof(int32_t) * nz(sh.n_total));
  L.row_set = take(sizeof(int32_t) * nz(sh.rows_total));
  L.T = take(sizeof(int32_t) * eps);
  L.secend = take(sizeof(int32_t) * (kMaxM + 2));
  L.thist = take(sizeof(int32_t) * (kMaxM + 2));
  L.coltab = take(sizeof(int32_t) * eps * kTabDepth);
  L.mhist = take(sizeof(int32_t) * (kMaxM + 2));
  L.perm = take(sizeof(int32_t) * nz(sh.rows_total));
  L.rec = take(16 * nz(sh.rows_total));
  L.recw = take(8 * nz(sh.rows_total));
  L.depth = take(sizeof(int32_t) * blocks);
  L.bdepth = take(sizeof(int32_t) * blocks);
  L.tiles = take(2 * sizeof(int32_t) * nz(sh.tiles_total));
  L.acc = take(3 * sizeof(uint64_t) * nz(sh.n_total));
  L.prof = take(sizeof(uint32_t) * kProf * nz(sh.rows_total));
  L.rowrem = take(2 * sizeof(int32_t) * nz(sh.rows_total));
  L.blkrem = take(2 * sizeof(int64_t) * (blocks + 1));
  L.cursor = take(2 * sizeof(int32_t) * nz(sh.rows_total));
  L.sortbuf = take(sh.n_sets > 1 ? 2 * sizeof(Item) * nz(sh.n_total) : 256);
  L.scanblk = take(2 * sizeof(int64_t) * (blocks / 1024 + 2));
  L.fixed_bytes = o;
  L.colmap = take(sizeof(int32_t) * nz(caps.k_cap));
  L.dstar = take(nz(caps.k_cap));
  L.flat = take(2 * sizeof(int32_t) * nz(caps.list_cap));
  L.rem = take(sizeof(uint32_t) * nz(caps.rem_cap));
  L.heavy = take(2 * sizeof(int32_t) * nz(caps.heavy_cap));
  o = align_up(o, 1024);
  L.planes = o;  // rows_total x K_cap 4-bit values
  o = align_up(o + (size_t)sh.rows_total * (size_t)caps.k_cap / 2, 1024);
  L.bitmap = o;  // bm_cols x rows_total bits
  o += (size_t)(caps.bm_cols > 0 ? caps.bm_cols : 0) * (size_t)(sh.rows_total / 8);
  L.bytes = align_up(o, 256);
  return L;
}

// One set of a (possibly batched) partition, built on the device by part_setup.
// Sets are consecutive in the item order.
struct PartSet {
  int64_t seq_begin;     // first item of the set
  int32_t n, p;          // items, buckets
  int64_t blk_base;      // first block / bucket segment: prefix of p
  int64_t piv_base;      // prefix of p - 1
  int64_t samp_base;     // prefix of p (p - 1)
  int64_t pos_base;      // prefix of p * p
};

struct PartTotals {
  int64_t n, p, p1, pp1, pp;  // sums over sets of n, p, p - 1, p (p - 1), p^2
};

constexpr PartTotals part_totals_single(int64_t n, int64_t p) {
  return PartTotals{n, p, p - 1, p * (p - 1), p * p};
}

struct PartLayout {
  size_t sets, segoff, gbound, items, items2, samples, samples2, pos, dest, pivots;
  size_t bytes;
};

// Every region grows with n and p, so the layout at the largest (n, p) bounds all smaller ones.
constexpr PartLayout part_layout_sets(int64_t n_sets, const PartTotals &t) {
  PartLayout L{};
  size_t o = sizeof(WsHeader);
  auto take = [&](size_t bytes) { size_t r = o; o = align_up(o + bytes, 256); return r; };
  auto nz = [](int64_t x) { return (size_t)(x > 0 ? x : 1); };
  L.sets = take(sizeof(PartSet) * nz(n_sets));
  L.segoff = take(sizeof(int64_t) * (size_t)(t.p + 1));
  L.gbound = take(sizeof(int64_t) * (size_t)(t.p + 1));
  L.items = take(sizeof(Item) * nz(t.n));
  L.items2 = take(sizeof(Item) * nz(t.n));
  L.samples = take(sizeof(Item) * nz(t.pp1));
  L.samples2 = take(sizeof(Item) * nz(t.pp1));
  L.pos = take(sizeof(int32_t) * nz(t.pp));
  L.dest = take(sizeof(int32_t) * nz(t.pp));
  L.pivots = take(sizeof(Item) * nz(t.p1));
  L.bytes = o;
  return L;
}

constexpr PartLayout part_layout(int64_t n, int64_t p) {
  return part_layout_sets(1, part_totals_single(n, p));
}

// ------------------------------------------------------ host bookkeeping ----
void note_launch(int n = 1);
int num_sms();
// Budget of the plane GEMM's main-loop waits (sad_debug_wait_budget_ns; 2 s by default).
uint64_t gemm_wait_ns();
// GEMM timing hooks (no-ops unless sad_profile(1) was called)
void prof_begin(cudaStream_t st);
void prof_end(cudaStream_t st);

#define SAD_LAUNCH_CHECK()                                   \
  do {                                                       \
    ::sad::note_launch();                                    \
    if (cudaPeekAtLastError() != cudaSuccess) {              \
      cudaGetLastError();                                    \
      return SAD_ERR_CUDA;                                   \
    }                                                        \
  } while (0)

// Kernels are launched with programmatic stream serialization: a kernel's CTAs may
// be scheduled while the previous kernel on the stream is finishing, and every
// kernel's first statement, pdl_enter(), waits until that kernel has completed and
// its memory is visible (griddepcontrol.wait) before touching memory, then lets
// the next kernel be scheduled once all of this kernel's CTAs have started.
template <typename... KArgs, typename... Args>
inline void pdl_launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t st, Args &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  (void)cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);  // error: SAD_LAUNCH_CHECK
}

__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// ------------------------------------------------------------- PTX: misc ----
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31; }

__device__ __forceinline__ bool elect_lane0() { return (threadIdx.x & 31) == 0; }

// Named barrier among `count` threads (multiple of 32).
__device__ __forceinline__ void named_bar_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Named barrier that also ORs a predicate over the participating threads: every
// thread gets the same result.
__device__ __forceinline__ bool named_bar_sync_or(int id, int count, bool pred) {
  uint32_t out;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.or.pred q, %2, %3, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}\n"
      : "=r"(out)
      : "r"((uint32_t)pred), "r"(id), "r"(count)
      : "memory");
  return out != 0;
}

// --------------------------------------------------------- PTX: mbarrier ----
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Non-blocking test of the phase with the given parity.
__device__ __forceinline__ bool mbar_test_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Budgets below this are a test's: every check of the barrier is non-blocking
// and the clock is read after each, so the budget runs out even where a blocking
// try_wait would have outlasted it.
constexpr uint64_t kShortWaitNs = 1000000ull;

// Bounded wait for the phase with the given parity to complete. Gives up when
// *abort becomes non-zero or after `budget_ns` of wall time; returns false then.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                  volatile int *abort, uint64_t budget_ns) {
  if (budget_ns < kShortWaitNs) {
    const uint64_t t0 = globaltimer_ns();
    while (!mbar_test_wait(bar, parity)) {
      if (*abort) return false;
      if (globaltimer_ns() - t0 > budget_ns) return false;
    }
    return true;
  }
  if (mbar_try_wait(bar, parity)) return true;
  uint64_t t0 = globaltimer_ns();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 63) == 0) {
      if (*abort) return false;
      if (globaltimer_ns() - t0 > budget_ns) return false;
    }
  }
}

// --------------------------------------------------------------- PTX: TMA ----
// TMA box (x, y, z) into shared memory, completion counted on a local mbarrier.
__device__ __forceinline__ void tma_load_3d(void *smem_dst, const CUtensorMap *map,
                                            uint64_t *bar, int32_t x, int32_t y, int32_t z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(smem_dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
      : "memory");
}

__device__ __forceinline__ void tma_prefetch_desc(const CUtensorMap *map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// ----------------------------------------------------------- PTX: tcgen05 ----
__device__ __forceinline__ void tmem_alloc(uint32_t *dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(dst_smem)),
               "r"(ncols)
               : "memory");
}

__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// D[tmem] (+)= A[smem] * B[smem]^T, 8-bit float operands (kind::f8f6f4).
__device__ __forceinline__ void mma_f8(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc,
                                       uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Arrive on an mbarrier once all previously issued tcgen05.mma of this thread complete.
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

// 32 lanes x 32 columns of 32-bit TMEM cells -> 32 registers per thread
// (thread = lane = accumulator row, register r = column base + r).
__device__ __forceinline__ void tmem_ld_32x32b_x32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
        "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
        "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
        "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
        "=r"(v[31])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld_wait() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor for a K-major operand tile stored with the
// 128-byte swizzle (rows of 128 bytes, 8-row atoms of 1024 bytes).
__device__ __forceinline__ uint64_t sdesc_kmajor_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);   // start address, 16-byte units
  d |= (uint64_t)1 << 16;                     // leading byte offset (unused with SW128 K-major)
  d |= (uint64_t)(1024 >> 4) << 32;           // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;                     // descriptor version for tcgen05
  d |= (uint64_t)2 << 61;                     // swizzle: 128B
  return d;
}

// Block-scaled 4-bit MMA (kind::mxf4nvf4, scale_vec::4X: one UE4M3 scale per 16
// values of K), D f32 += A x B with A, B packed e2m1 from shared memory and the
// scales of A and B read from TMEM; K = 64 per instruction.
__device__ __forceinline__ void mma_f4(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc,
                                       uint32_t idesc, uint32_t sfa_tmem, uint32_t sfb_tmem,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %6, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::mxf4nvf4.block_scale.scale_vec::4X "
      "[%0], %1, %2, %3, [%4], [%5], p;\n\t}\n" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(sfa_tmem), "r"(sfb_tmem), "r"(accumulate)
      : "memory");
}

// 32 lanes (this warp's quadrant) x 16 columns of TMEM from registers, all = v.
__device__ __forceinline__ void tmem_st_32x32b_x16_fill(uint32_t taddr, uint32_t v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
      "{%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(taddr),
      "r"(v)
      : "memory");
}

__device__ __forceinline__ void tmem_st_wait() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// Instruction descriptor of the block-scaled kinds: A = B = E2M1 (format 1 of
// kind::mxf4nvf4), both K-major, scales UE4M3 (bit 23 clear), scale-factor ids 0,
// dense K = 64, shape M x N.
__host__ __device__ constexpr uint32_t idesc_f4_e2m1(int M, int N) {
  return (1u << 7) | (1u << 10)          // A, B = E2M1
         | (0u << 15) | (0u << 16)       // K-major A and B
         | ((uint32_t)(N >> 3) << 17)    // N / 8
         | (0u << 23)                    // scale type UE4M3
         | ((uint32_t)(M >> 4) << 24);   // M / 16
}

// ------------------------------------------- PTX: CTA pairs (clusters of 2) ----
// A pair runs one tcgen05.mma of M = 256: each CTA holds 128 rows of A and half of
// the N rows of B in its shared memory and 128 lanes of the accumulator in its
// TMEM; the even CTA (rank 0) issues the MMAs for both. Every tcgen05 instruction
// of such a kernel uses cta_group::2.
__device__ __forceinline__ uint32_t cluster_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ uint32_t cluster_id_x() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}

__device__ __forceinline__ uint32_t cluster_count_x() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
  return r;
}

// Shared::cluster address of the same shared variable in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t mapa_shared(const void *p, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
  return r;
}

__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait_cluster(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// mbar_wait_bounded with cluster-scope acquire (arrivals from the other CTA).
__device__ __forceinline__ bool mbar_wait_bounded_cluster(uint64_t *bar, uint32_t parity,
                                                          volatile int *abort,
                                                          uint64_t budget_ns) {
  if (mbar_try_wait_cluster(bar, parity)) return true;
  uint64_t t0 = globaltimer_ns();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try_wait_cluster(bar, parity)) return true;
    if ((it & 63) == 0) {
      if (*abort) return false;
      if (globaltimer_ns() - t0 > budget_ns) return false;
    }
  }
}

// Every thread of both CTAs; memory before it is visible to both after it.
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release;" ::: "memory");
  asm volatile("barrier.cluster.wait.acquire;" ::: "memory");
}

// TMA box into this CTA's shared memory, completion counted on an mbarrier of
// either CTA of the pair (shared::cluster address).
__device__ __forceinline__ void tma_load_3d_pair(void *smem_dst, const CUtensorMap *map,
                                                 uint32_t bar_cluster, int32_t x, int32_t y,
                                                 int32_t z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.cta_group::2.shared::cluster.global.tile.mbarrier::complete_tx::"
      "bytes [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(smem_dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar_cluster), "r"(x), "r"(y), "r"(z)
      : "memory");
}

// One warp of each CTA of the pair, together: the same columns in both TMEMs.
__device__ __forceinline__ void tmem_alloc_pair(uint32_t *dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(dst_smem)),
               "r"(ncols)
               : "memory");
}

__device__ __forceinline__ void tmem_relinquish_pair() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc_pair(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}

// mma_f4 over the pair: M = 256 (128 rows from each CTA's A), B's N rows split
// between the two CTAs' shared memory at the same offsets.
__device__ __forceinline__ void mma_f4_pair(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc,
                                            uint32_t idesc, uint32_t sfa_tmem, uint32_t sfb_tmem,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %6, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::mxf4nvf4.block_scale.scale_vec::4X "
      "[%0], %1, %2, %3, [%4], [%5], p;\n\t}\n" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(sfa_tmem), "r"(sfb_tmem), "r"(accumulate)
      : "memory");
}

// Arrive once on the mbarrier at this offset in every CTA of `mask` when all
// previously issued pair MMAs of this thread complete.
__device__ __forceinline__ void mma_commit_pair(uint64_t *bar, uint16_t mask) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
      " [%0], %1;" ::"r"(smem_u32(bar)),
      "h"(mask)
      : "memory");
}

// UE4M3 encoding of 1.0 (exponent 7 = bias, mantissa 0), four to a TMEM word.
constexpr uint32_t kScaleOne4 = 0x38383838u;
// e2m1 encoding of 1.0 (exponent 1 = bias, mantissa 0)
constexpr uint32_t kE2M1One = 0x2u;

}  // namespace sad
