// Device pointers into a kmer_rank workspace and the launchers shared by the
// rank translation units.
#pragma once

#include "sad_common.cuh"

namespace sad {

struct RankPtrs {
  WsHeader *hdr;
  int32_t *T;            // [eps] largest count of each word
  int32_t *secend;       // [t_max + 1] end column of threshold section t
  int32_t *colmap;       // [K_cap] column -> word | threshold << 16
  int32_t *thist;        // [65537] histogram / cursor over T values
  int32_t *tau_sorted;   // [eps] words by decreasing T
  int32_t *mhist;        // [65537] histogram / cursor over m = L - k + 1
  int32_t *perm;         // [n_pad] stored row -> input index (-1 = padding)
  int32_t *depth;        // [n_pad / 128] largest count in each 128-row block
  uint4 *rec;            // [n_pad] division record of each stored row's m
  int2 *tiles;           // [max_tiles] (I | J << 16, K chunks)
  unsigned long long *acc;  // [n][3] 24-bit-limb accumulators of the keys
  uint8_t *planes;       // [n_pad][K_cap] fp8 threshold planes (sections 1..depth)
  // residual of the counts above the plane depth
  int32_t *cnt_gt;       // [eps] sequences whose count of the word exceeds depth
  int64_t *list_off;     // [eps + 1] start of each word's excess list
  int64_t *pair_off;     // [eps + 1] start of each word's pair range
  int32_t *cursor;       // [eps] fill cursor of the excess lists
  int2 *lists;           // [list_cap] (stored row, count - depth)
  int32_t *tile_of;      // [(n_pad/128) x (n_pad/256)] tile index of block (I, J)
  int32_t *block_of;     // [max_tiles] residual block of a tile, -1 = none
  uint32_t *rblocks;     // [block_cap][128][256] u16 residual per pair (two per word)
  int64_t n_pad, k_cap, list_cap, block_cap;
  int32_t depth_cap;     // 0 = all planes
};

RankPtrs rank_ptrs(void *ws, const RankLayout &L);
int rank_prep_launch(const RankPtrs &P, const int32_t *counts, const int32_t *lengths,
                     int32_t n, int32_t k, int32_t eps, int plan_only, cudaStream_t st);
int rank_gemm_launch(const RankPtrs &P, int32_t n, cudaStream_t st);
int rank_finalize_launch(const RankPtrs &P, int32_t n, uint64_t *key_hi, uint64_t *key_lo,
                         double *rank, cudaStream_t st);
int64_t host_tile_count(int32_t n);

}  // namespace sad
