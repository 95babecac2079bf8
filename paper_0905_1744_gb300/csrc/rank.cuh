// Device pointers into a kmer_rank workspace and the launchers shared by the
// rank translation units.
#pragma once

#include "sad_common.cuh"

namespace sad {

// Division record for denominator d (1..65535), used by the GEMM epilogue (and the
// sparse ablation) to
// form floor(S * 2^64 / d) = S * Q + floor(S * r / d) exactly, with
// Q = floor((2^64 - 1) / d), r = 2^64 - Q d in [1, d], and floor(x / d) for
// x < 2^32 by Granlund & Montgomery (1994), "Division by invariant integers
// using multiplication", Fig. 4.1: l = ceil(log2 d),
// m' = floor(2^32 (2^l - d) / d) + 1, t1 = umulhi(m', x),
// q = (t1 + ((x - t1) >> min(l,1))) >> max(l-1, 0).
__device__ __forceinline__ uint4 division_record(uint32_t d) {
  const uint64_t Q = 0xFFFFFFFFFFFFFFFFull / d;
  const uint32_t l = 32u - (uint32_t)__clz((int)(d - 1u));
  const uint64_t magic = (((uint64_t)1 << 32) * (((uint64_t)1 << l) - d)) / d + 1u;
  const uint32_t sh1 = l < 1u ? l : 1u;
  const uint32_t sh2 = l > 0u ? l - 1u : 0u;
  return make_uint4((uint32_t)Q, (uint32_t)(Q >> 32), (uint32_t)magic,
                    d | (sh1 << 16) | (sh2 << 24));
}

// The small part of a term, floor(s r / d) with r = 2^64 - Q d in [1, d], as one
// fixed-point product: floor(s W / 2^63) with W = ceil(2^63 r / d) <= 2^63. For
// every s < 2^16 the excess s (W - 2^63 r / d) / 2^63 < 2^-47 stays below the gap
// 1/d between the fraction of s r / d and the next integer, so the floor is exact.
// W by long division in two steps (r 2^47 < 2^64, then the remainder times 2^16).
__device__ __forceinline__ uint2 floor_weight(uint32_t d) {
  const uint64_t Q = 0xFFFFFFFFFFFFFFFFull / d;
  const uint64_t r = 0ull - Q * d;
  const uint64_t n1 = r << 47;
  const uint64_t q1 = n1 / d, r1 = n1 - q1 * d;
  const uint64_t n2 = r1 << 16;
  const uint64_t q2 = n2 / d, r2 = n2 - q2 * d;
  const uint64_t W = (q1 << 16) + q2 + (r2 != 0 ? 1u : 0u);
  return make_uint2((uint32_t)W, (uint32_t)(W >> 32));
}

struct RankPtrs {
  WsHeader *hdr;
  RankSet *sets;         // [n_sets]
  int32_t *seq_set;      // [n_total] set of each input sequence (n_sets > 1 only)
  int32_t *row_set;      // [rows_total] set of each stored row (n_sets > 1 only)
  int32_t *T;            // [eps] largest count of each word over all sets
  int32_t *secend;       // [t_max + 1] end column of threshold section t
  int32_t *colmap;       // [K_cap] column -> word | threshold << 16
  int8_t *dstar;         // [K_cap] smallest plane depth d whose tiles cover the column
  int32_t *thist;        // [65537] histogram / cursor over T values
  int32_t *coltab;       // [kTabDepth][eps] column of (threshold t, word), -1 = none
  int32_t *mhist;        // [65537] histogram / cursor over m = L - k + 1 (one set)
  int32_t *perm;         // [rows_total] stored row -> input index (-1 = padding)
  int32_t *depth;        // [rows_total / 128] largest count in each 128-row block
  int32_t *bdepth;       // [rows_total / 128] plane depth of each column block (remainder)
  uint4 *rec;            // [rows_total] division record of each stored row's m
  uint2 *recw;           // [rows_total] floor_weight of each stored row's m
  int2 *tiles;           // [tiles_total] (I | J << 16, K chunks), global block indices
  unsigned long long *acc;  // [n_total][3] key = acc0 + acc1 2^32 (distance mode: acc0)
  uint8_t *planes;       // [rows_total][K_cap / 2] packed e2m1 threshold planes
  // remainder of the counts the planes of a tile do not cover (depth >= 1)
  uint32_t *prof;        // [rows_total][kProf] per-row remainder profile
  int32_t *rowrem;       // [rows_total][2] first remainder / heavy entry of the row in its block
  int64_t *blkrem;       // [blocks + 1][2] first remainder / heavy entry of each block
  int32_t *cursor;       // [rows_total][2] fill cursors
  int2 *flat;            // [list_cap] (stored row, word | count << 16), count >= 2, unordered
  uint32_t *rem;         // [rem_cap] bitmap column of each remainder entry, grouped by row
  int2 *heavy;           // [heavy_cap] (word, count) of counts above T_b, grouped by row
  uint32_t *bitmap;      // [bm_cols][rows_total / 32] bit r of column (t, word): count >= t
  Item *sortbuf;         // [2 n_total] per-set length sort (n_sets > 1 only)
  int64_t *scanblk;      // block totals of the remainder scans
  const int32_t *counts; // the rank's input counts (heavy remainder entries read them)
  int64_t n_pad;         // rows_total: stored rows over all sets
  int64_t n_total, n_sets, tiles_total, k_cap, list_cap, rem_cap, heavy_cap, bm_cols;
  int32_t depth_cap;     // 0 = all planes
  int32_t budget;        // remainder entries per column block
  int32_t tile;          // rows of a GEMM tile (and of a remainder block): 128 or 256
  int32_t eps;
  uint64_t wait_ns;      // budget of the GEMM's main-loop waits
};

RankPtrs rank_ptrs(void *ws, const RankLayout &L);
// d_n: per-set sizes on the device (n_sets > 1), or nullptr for one set of n_total.
// word_max (nullable): the largest count of every word, as kmer_count can return
// it; when given, the column-maximum pass over the counts is skipped.
int rank_prep_launch(const RankPtrs &P, const int32_t *counts, const int32_t *lengths,
                     const int32_t *d_n, const int32_t *word_max, int32_t k, int32_t eps,
                     int plan_only, cudaStream_t st);
int rank_gemm_launch(const RankPtrs &P, cudaStream_t st);

// Rectangular mode of the plane GEMM: every stored row of P against ref_rows
// reference rows (their planes in ref_planes, same K_cap, division records in
// rec_ref), the row keys only, D = min(m_i, m_r) per pair.
struct RectArgs {
  const uint4 *rec_ref = nullptr;  // nullptr: square mode
  int32_t row_blocks = 0, n_tiles = 0, n_ref = 0;
};
// ln_table != nullptr: the distance form (see DistArgs) with D = min(m_i, m_r).
int rank_rect_gemm_launch(const RankPtrs &P, uint8_t *ref_planes, const uint4 *rec_ref,
                          int64_t ref_rows, int32_t n_ref, const int64_t *ln_table, int32_t b,
                          cudaStream_t st);

// Distance mode of the plane GEMM (Eq. 2 / Eq. 3 literally, Delta = 1 / b): for
// stored i <= j, q_ij = ln_table[b m_j] - ln_table[m_j + b S_ij] (ln x times 2^32),
// the signed sums added to acc[3 x] of both sequences (the pair once).
struct DistArgs {
  const int64_t *ln_table = nullptr;  // [(b + 1) * 65535 + 1]
  int32_t b = 0;
};
int rank_dist_gemm_launch(const RankPtrs &P, const int64_t *ln_table, int32_t b,
                          cudaStream_t st);
// Distance-form rank (dist.cu).
size_t ln_table_entries(int32_t b);
int ln_table_launch(int64_t *table, int32_t b, cudaStream_t st);
int ln_q_launch(const uint64_t *x, int64_t n, int64_t *out, cudaStream_t st);
// n_div > 0: rank = key 2^-32 / n_div (a reference set); 0: the set's size.
int rank_dist_finalize_launch(const RankPtrs &P, int64_t *key, uint64_t *key_hi,
                              uint64_t *key_lo, double *rank, int64_t n_div, cudaStream_t st);
// Globalised rank (grank.cu).
size_t local_samples_ws_bytes(int64_t n, int64_t p);
int local_samples_launch(const uint64_t *key_hi, const uint64_t *key_lo, int32_t n, int32_t p,
                         int32_t ks, int32_t *sample_idx, void *ws, size_t ws_bytes,
                         cudaStream_t st);
size_t rank_vs_ws_bytes(int64_t n, int64_t eps, int64_t k_cap, int64_t n_ref, int32_t delta_den);
int rank_vs_launch(const int32_t *counts, const int32_t *lengths, const int32_t *word_max,
                   int32_t n, int32_t k, int64_t eps, const int32_t *ref, int32_t n_ref,
                   int64_t k_cap, int32_t delta_den, int64_t *key, uint64_t *key_hi,
                   uint64_t *key_lo, double *rank, void *ws, size_t ws_bytes, cudaStream_t st);

// Sparse-intersection rank on the CUDA cores (sparse.cu).
size_t sparse_ws_bytes(int64_t n, int64_t entries_cap);
int sparse_count_launch(const int32_t *counts, const int32_t *lengths, int32_t n, int32_t k,
                        int32_t eps, void *ws, size_t ws_bytes, cudaStream_t st);
int sparse_rank_launch(const int32_t *counts, const int32_t *lengths, int32_t n, int32_t k,
                       int32_t eps, int64_t entries_cap, uint64_t *key_hi, uint64_t *key_lo,
                       double *rank, void *ws, size_t ws_bytes, cudaStream_t st);

// TMA map of a plane matrix (rows x K_cap / 2 bytes, 128-byte swizzle, boxes of
// 128 bytes x box_rows rows x box_chunks K chunks).
int make_plane_map(CUtensorMap *map, uint8_t *planes, int64_t rows, int64_t k_cap, int box_rows,
                   int box_chunks);
int rank_finalize_launch(const RankPtrs &P, uint64_t *key_hi, uint64_t *key_lo, double *rank,
                         cudaStream_t st);
int64_t host_tile_count(int32_t n);

}  // namespace sad
