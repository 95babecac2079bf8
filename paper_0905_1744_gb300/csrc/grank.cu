// Globalised k-mer rank (Sec. 3.1.1; Algorithm 2 steps 2-6) on one device.
//
//   steps 2-3  local ranks: each of the p contiguous blocks of sequences ranked
//              against its own block (the block-diagonal batched rank, blocks as
//              sets) and sorted by that rank;
//   step 4     ks samples per block, evenly spaced in the block's sorted order:
//              0-based positions floor(j w_b / (ks + 1)), j = 1..ks
//              (local_samples_launch);
//   steps 5-6  the ks x p samples are the reference set; every sequence is ranked
//              against it: key_i = sum_r floor(S_{i,r} 2^64 / D_{i,r}),
//              D = min(L_i, L_r) - k + 1, rank_i = key_i / (|R| 2^64), or in the
//              distance form of Eq. 2 key_i = sum_r q_{i,r} (see dist.cu)
//              (rank_vs_launch: the rank preparation at full plane depth, the
//              reference rows' planes gathered, then the plane GEMM in its
//              rectangular mode).
// The gather of samples to every processor and their broadcast are index steps
// here: no sequence data moves.
#include "rank.cuh"
#include "sort.cuh"

namespace sad {

namespace {

struct SamplesLayout {
  size_t segoff, items, scratch, bytes;
};

SamplesLayout samples_layout(int64_t n, int64_t p) {
  SamplesLayout L{};
  size_t o = sizeof(WsHeader);
  auto take = [&](size_t b) { size_t r = o; o = align_up(o + b, 256); return r; };
  L.segoff = take(sizeof(int64_t) * (size_t)(p + 1));
  L.items = take(sizeof(Item) * (size_t)(n > 0 ? n : 1));
  L.scratch = take(sizeof(Item) * (size_t)(n > 0 ? n : 1));
  L.bytes = o;
  return L;
}

__global__ void samples_setup_kernel(const uint64_t *__restrict__ hi, const uint64_t *__restrict__ lo,
                                     int32_t n, int32_t p, int64_t *segoff, Item *items) {
  pdl_enter();
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nt = (int64_t)gridDim.x * blockDim.x;
  for (int64_t b = tid; b <= p; b += nt) segoff[b] = b * (int64_t)n / p;
  for (int64_t x = tid; x < n; x += nt) {
    Item it;
    it.hi = hi[x];
    it.lo = lo[x];
    it.idx = (int32_t)x;
    it.pad = 0;
    items[x] = it;
  }
}

__global__ void __launch_bounds__(kSortThreads) block_sort_kernel(Item *items, Item *scratch,
                                                                   int32_t p,
                                                                   const int64_t *segoff) {
  pdl_enter();
  extern __shared__ Item sm[];
  for (int32_t b = blockIdx.x; b < p; b += gridDim.x) {
    const int64_t a = segoff[b], e = segoff[b + 1];
    cta_sort(items + a, scratch + a, e - a, sm);
  }
}

__global__ void pick_samples_kernel(const Item *items, const int64_t *segoff, int32_t p,
                                    int32_t ks, int32_t *sample_idx) {
  pdl_enter();
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)p * ks;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = t / ks, j = t % ks + 1;
    const int64_t a = segoff[b], w = segoff[b + 1] - a;
    sample_idx[t] = items[a + j * w / (ks + 1)].idx;
  }
}

// ------------------------------------------------------------- rank vs R ---

struct RefLayout {
  size_t inv, planes, rec, table, bytes;  // offsets after the rank layout
  int64_t ref_rows;
};

RefLayout ref_layout(size_t base, int64_t n_pad, int64_t n_ref, int64_t k_cap, int32_t delta_den) {
  RefLayout R{};
  R.ref_rows = (n_ref + kColBlock - 1) / kColBlock * kColBlock;
  size_t o = align_up(base, 256);
  R.inv = o;
  o = align_up(o + sizeof(int32_t) * (size_t)n_pad, 1024);
  R.planes = o;
  o = align_up(o + (size_t)R.ref_rows * (size_t)k_cap / 2, 256);
  R.rec = o;
  o = align_up(o + 16 * (size_t)R.ref_rows, 256);
  R.table = o;  // distance form: the ln_q table
  if (delta_den > 0) o = align_up(o + sizeof(int64_t) * ln_table_entries(delta_den), 256);
  R.bytes = o;
  return R;
}

__global__ void inv_perm_kernel(RankPtrs P, int32_t *inv) {
  pdl_enter();
  if (P.hdr->status != 0) return;
  for (int64_t pos = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; pos < P.n_pad;
       pos += (int64_t)gridDim.x * blockDim.x) {
    const int32_t x = P.perm[pos];
    if (x >= 0) inv[x] = (int32_t)pos;
  }
}

// Block per reference row r: its plane row (K_pad / 2 bytes) and division record;
// rows past n_ref are zero (S = 0, so their terms are 0 whatever the record).
__global__ void gather_ref_kernel(RankPtrs P, const int32_t *__restrict__ inv,
                                  const int32_t *__restrict__ ref, int32_t n_ref,
                                  int64_t ref_rows, uint8_t *ref_planes, uint4 *rec_ref) {
  pdl_enter();
  if (P.hdr->status != 0) return;
  const int64_t row_bytes = P.k_cap / 2;
  const int64_t used = P.hdr->k_pad / 2;  // multiple of 128
  for (int64_t r = blockIdx.x; r < ref_rows; r += gridDim.x) {
    uint4 *dst = reinterpret_cast<uint4 *>(ref_planes + r * row_bytes);
    int64_t pos = -1;
    if (r < n_ref) {
      const int32_t x = ref[r];
      if (x < 0 || x >= P.n_total) {
        if (threadIdx.x == 0) record_error(P.hdr, SAD_ERR_INVALID_ARGUMENT, (int)r);
      } else {
        pos = inv[x];
      }
    }
    if (pos >= 0) {
      const uint4 *src = reinterpret_cast<const uint4 *>(P.planes + pos * row_bytes);
      for (int64_t i = threadIdx.x; i < used / 16; i += blockDim.x) dst[i] = src[i];
      if (threadIdx.x == 0) rec_ref[r] = P.rec[pos];
    } else {
      for (int64_t i = threadIdx.x; i < used / 16; i += blockDim.x) dst[i] = make_uint4(0, 0, 0, 0);
      // the record of d = 1: Q = 2^64 - 1, magic 1, no shifts
      if (threadIdx.x == 0) rec_ref[r] = make_uint4(0xFFFFFFFFu, 0xFFFFFFFFu, 1u, 1u);
    }
  }
}

// key = acc0 + acc1 2^32; rank = (hi + lo 2^-64) / |R|.
__global__ void finalize_vs_kernel(RankPtrs P, int32_t n_ref, uint64_t *__restrict__ key_hi,
                                   uint64_t *__restrict__ key_lo, double *__restrict__ rank) {
  pdl_enter();
  if (P.hdr->status != 0) return;
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < P.n_total;
       x += (int64_t)gridDim.x * blockDim.x) {
    const unsigned __int128 a0 = P.acc[3 * x + 0], a1 = P.acc[3 * x + 1];
    const unsigned __int128 key = a0 + (a1 << 32);
    const uint64_t hi = (uint64_t)(key >> 64), lo = (uint64_t)key;
    key_hi[x] = hi;
    key_lo[x] = lo;
    if (rank) {
      const double whole = __ull2double_rn(hi);
      const double frac = __dmul_rn(__ull2double_rn(lo), 0x1p-64);
      rank[x] = __ddiv_rn(__dadd_rn(whole, frac), (double)n_ref);
    }
  }
}

unsigned grid_of(int64_t work, int threads) {
  int64_t g = (work + threads - 1) / threads;
  const int64_t cap = (int64_t)num_sms() * 8;
  return (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
}

}  // namespace

size_t local_samples_ws_bytes(int64_t n, int64_t p) { return samples_layout(n, p).bytes; }

int local_samples_launch(const uint64_t *key_hi, const uint64_t *key_lo, int32_t n, int32_t p,
                         int32_t ks, int32_t *sample_idx, void *ws, size_t ws_bytes,
                         cudaStream_t st) {
  const SamplesLayout L = samples_layout(n, p);
  if (ws_bytes < L.bytes) return SAD_ERR_WORKSPACE;
  uint8_t *b = static_cast<uint8_t *>(ws);
  int64_t *segoff = reinterpret_cast<int64_t *>(b + L.segoff);
  Item *items = reinterpret_cast<Item *>(b + L.items);
  Item *scratch = reinterpret_cast<Item *>(b + L.scratch);
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(block_sort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kSortSmem) != cudaSuccess)
      return SAD_ERR_CUDA;
    attr = true;
  }
  pdl_launch(samples_setup_kernel, grid_of((int64_t)n + p + 1, 256), 256, 0, st, key_hi, key_lo, n,
             p, segoff, items);
  SAD_LAUNCH_CHECK();
  pdl_launch(block_sort_kernel, (unsigned)(p < 65535 ? p : 65535), kSortThreads, kSortSmem, st,
             items, scratch, p, segoff);
  SAD_LAUNCH_CHECK();
  pdl_launch(pick_samples_kernel, grid_of((int64_t)p * ks, 256), 256, 0, st, items, segoff, p, ks,
             sample_idx);
  SAD_LAUNCH_CHECK();
  return SAD_OK;
}

size_t rank_vs_ws_bytes(int64_t n, int64_t eps, int64_t k_cap, int64_t n_ref, int32_t delta_den) {
  const RankLayout L = rank_layout(shape_single(n), eps, RankCaps{0, 0, 0, k_cap, 0, 0, 0, 0});
  return ref_layout(L.bytes, L.shape.rows_total, n_ref, k_cap, delta_den).bytes;
}

int rank_vs_launch(const int32_t *counts, const int32_t *lengths, const int32_t *word_max,
                   int32_t n, int32_t k, int64_t eps, const int32_t *ref, int32_t n_ref,
                   int64_t k_cap, int32_t delta_den, int64_t *key, uint64_t *key_hi,
                   uint64_t *key_lo, double *rank, void *ws, size_t ws_bytes, cudaStream_t st) {
  const RankLayout L = rank_layout(shape_single(n), eps, RankCaps{0, 0, 0, k_cap, 0, 0, 0, 0});
  const RefLayout R = ref_layout(L.bytes, L.shape.rows_total, n_ref, k_cap, delta_den);
  if (ws_bytes < R.bytes) return SAD_ERR_WORKSPACE;
  if (L.shape.rows_total / kRowBlock > kMaxRowBlocks) return SAD_ERR_UNSUPPORTED;
  const RankPtrs P = rank_ptrs(ws, L);
  uint8_t *b = static_cast<uint8_t *>(ws);
  int32_t *inv = reinterpret_cast<int32_t *>(b + R.inv);
  uint8_t *ref_planes = b + R.planes;
  uint4 *rec_ref = reinterpret_cast<uint4 *>(b + R.rec);
  // all planes (depth 0): no residual; the square tile list is built but not run
  int64_t *table = delta_den > 0 ? reinterpret_cast<int64_t *>(b + R.table) : nullptr;
  int rc = SAD_OK;
  if (table && (rc = ln_table_launch(table, delta_den, st))) return rc;
  rc = rank_prep_launch(P, counts, lengths, nullptr, word_max, k, (int32_t)eps, 0, st);
  if (rc) return rc;
  pdl_launch(inv_perm_kernel, grid_of(P.n_pad, 256), 256, 0, st, P, inv);
  SAD_LAUNCH_CHECK();
  pdl_launch(gather_ref_kernel, (unsigned)(R.ref_rows < 65535 ? R.ref_rows : 65535), 256, 0, st, P,
             inv, ref, n_ref, R.ref_rows, ref_planes, rec_ref);
  SAD_LAUNCH_CHECK();
  rc = rank_rect_gemm_launch(P, ref_planes, rec_ref, R.ref_rows, n_ref, table, delta_den, st);
  if (rc) return rc;
  if (table) return rank_dist_finalize_launch(P, key, key_hi, key_lo, rank, n_ref, st);
  pdl_launch(finalize_vs_kernel, grid_of(n, 256), 256, 0, st, P, n_ref, key_hi, key_lo, rank);
  SAD_LAUNCH_CHECK();
  return SAD_OK;
}

}  // namespace sad
