// Regular-sampling sample sort of the rank keys into p buckets (Sec. 3.1.2 and
// Algorithm 2 steps 7-11), with the p processors as virtual buckets on one GPU:
//
//   part_init      items = (key_hi, key_lo, index)
//   seg_sort       step 7: sort each block [floor(bN/p), floor((b+1)N/p)) by
//                  (key, index), one CTA per block
//   samples        step 8-9: p-1 samples per block at floor(j w_b / p), sort the
//                  p(p-1) samples, pivots y_i = Y_{(i-1)p + floor(p/2)} (1-based)
//   subblocks      sub-block (b, i) of block b = its items in (y_{i-1}, y_i]: a
//                  binary search of every pivot in every sorted block
//   bucket_scan    bucket sizes and CSR offsets, destination of every sub-block
//                  (sub-blocks of a bucket in block order: the all-to-all step)
//   scatter        step 11: move every item to its bucket
//   seg_sort       each bucket sorted by (key, index)
//   members        output input indices
// One set with few buckets takes a faster route (chunk sorts and rank merges,
// below) to the same result.
//
// Sorting inside one CTA: a bitonic network in shared memory for up to 4096
// items; longer ranges sort 4096-item chunks that way and then merge runs of
// doubling width in global memory, each item finding its place by a binary
// search in the other run (all items differ, the index breaking ties).
#include "sort.cuh"

namespace sad {

namespace {

__device__ __forceinline__ int64_t block_lo(int64_t b, int64_t n, int64_t p) { return b * n / p; }

// Set holding global item x: last s with sets[s].seq_begin <= x.
__device__ __forceinline__ int32_t set_of(const PartSet *sets, int32_t n_sets, int64_t x) {
  int lo = 0, hi = n_sets - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (sets[mid].seq_begin <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// One block: the set table from per-set sizes (d_n, d_p; or the single set n1, p1)
// and the block boundaries segoff[blk_base + b] = seq_begin + floor(b n / p).
__global__ void __launch_bounds__(1024) part_setup_kernel(const int32_t *d_n, const int32_t *d_p,
                                                          int32_t n_sets, int32_t n1, int32_t p1,
                                                          PartSet *sets, int64_t *segoff) {
  pdl_enter();
  __shared__ int64_t s_warp[32];
  __shared__ int64_t s_c[5];
  const int tid = threadIdx.x;
  if (tid < 5) s_c[tid] = 0;
  __syncthreads();
  for (int base = 0; base < n_sets; base += blockDim.x) {
    const int s = base + tid;
    const int64_t n = s < n_sets ? (d_n ? d_n[s] : n1) : 0;
    const int64_t p = s < n_sets ? (d_p ? d_p[s] : p1) : 0;
    const int64_t v[5] = {n, p, p > 0 ? p - 1 : 0, p * (p > 0 ? p - 1 : 0), p * p};
    int64_t ex[5];
#pragma unroll
    for (int f = 0; f < 5; ++f) {
      int64_t x = v[f];
      for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if ((tid & 31) >= o) x += y;
      }
      if ((tid & 31) == 31) s_warp[tid >> 5] = x;
      __syncthreads();
      if (tid < 32) {
        int64_t w = s_warp[tid];
        for (int o = 1; o < 32; o <<= 1) {
          const int64_t y = __shfl_up_sync(0xffffffffu, w, o);
          if (tid >= o) w += y;
        }
        s_warp[tid] = w;
      }
      __syncthreads();
      const int64_t incl = x + ((tid >> 5) > 0 ? s_warp[(tid >> 5) - 1] : 0);
      ex[f] = s_c[f] + incl - v[f];
      __syncthreads();
      if (tid == (int)blockDim.x - 1) s_c[f] += incl;
      __syncthreads();
    }
    if (s < n_sets) {
      PartSet e;
      e.seq_begin = ex[0];
      e.n = (int32_t)n;
      e.p = (int32_t)p;
      e.blk_base = ex[1];
      e.piv_base = ex[2];
      e.samp_base = ex[3];
      e.pos_base = ex[4];
      sets[s] = e;
      for (int64_t b = 0; b <= p; ++b) segoff[e.blk_base + b] = e.seq_begin + block_lo(b, n, p);
    }
  }
}

// One set with its size on the host: the set table (every base 0), the block
// offsets floor(b n / p) and the items, in one launch.
__global__ void part_init_single_kernel(const uint64_t *__restrict__ hi,
                                        const uint64_t *__restrict__ lo, int64_t n, int64_t p,
                                        PartSet *sets, int64_t *segoff, Item *items) {
  pdl_enter();
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nt = (int64_t)gridDim.x * blockDim.x;
  if (tid == 0) {
    PartSet e;
    e.seq_begin = 0;
    e.n = (int32_t)n;
    e.p = (int32_t)p;
    e.blk_base = 0;
    e.piv_base = 0;
    e.samp_base = 0;
    e.pos_base = 0;
    sets[0] = e;
  }
  for (int64_t b = tid; b <= p; b += nt) segoff[b] = block_lo(b, n, p);
  for (int64_t x = tid; x < n; x += nt) {
    Item it;
    it.hi = hi[x];
    it.lo = lo[x];
    it.idx = (int32_t)x;
    it.pad = 0;
    items[x] = it;
  }
}

__global__ void part_init_kernel(const uint64_t *__restrict__ hi, const uint64_t *__restrict__ lo,
                                 int64_t n, const PartSet *sets, int32_t n_sets, Item *items) {
  pdl_enter();
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
       x += (int64_t)gridDim.x * blockDim.x) {
    Item it;
    it.hi = hi[x];
    it.lo = lo[x];
    it.idx = (int32_t)(x - sets[set_of(sets, n_sets, x)].seq_begin);
    it.pad = 0;
    items[x] = it;
  }
}

// Segment s = items [offs[s], offs[s+1]), one block per segment.
__global__ void __launch_bounds__(kSortThreads) seg_sort_kernel(Item *items, Item *scratch,
                                                                 int64_t n_seg,
                                                                 const int64_t *offs) {
  pdl_enter();
  extern __shared__ Item sm[];
  for (int64_t s = blockIdx.x; s < n_seg; s += gridDim.x) {
    const int64_t lo = offs[s], hi = offs[s + 1];
    cta_sort(items + lo, scratch + lo, hi - lo, sm);
  }
}

// One block per set: regular samples of the sorted blocks, sorted; pivots.
__global__ void __launch_bounds__(kSortThreads) samples_kernel(const Item *items, Item *Y_all,
                                                                Item *Y2_all, Item *piv_all,
                                                                int32_t *pivot_idx,
                                                                const PartSet *sets,
                                                                int32_t n_sets) {
  pdl_enter();
  extern __shared__ Item sm[];
  for (int32_t si = blockIdx.x; si < n_sets; si += gridDim.x) {
    const PartSet S = sets[si];
    const int64_t n = S.n, p = S.p;
    if (p <= 1) continue;
    Item *Y = Y_all + S.samp_base, *Y2 = Y2_all + S.samp_base, *piv = piv_all + S.piv_base;
    const Item *it = items + S.seq_begin;
    const int64_t ns = p * (p - 1);
    if (ns <= (int64_t)blockDim.x) {
      // few samples: each thread ranks one against all of them in shared memory
      // (a sample taken twice, w_b < p, is ordered by its sample number) and the
      // samples at the pivot ranks are the pivots
      for (int64_t e = threadIdx.x; e < ns; e += blockDim.x) {
        const int64_t b = e / (p - 1), j = e % (p - 1) + 1;
        const int64_t lo = block_lo(b, n, p), w = block_lo(b + 1, n, p) - lo;
        sm[e] = it[lo + j * w / p];
      }
      __syncthreads();
      // a group of g threads (a power of two, within a warp) ranks one sample
      int g = 1;
      while (g < 32 && (int64_t)(2 * g) * ns <= (int64_t)blockDim.x) g *= 2;
      const int64_t e = threadIdx.x / g;
      const int u = (int)(threadIdx.x % g);
      int32_t r = 0;
      Item y{};
      if (e < ns) {
        y = sm[e];
        for (int64_t f = u; f < ns; f += g) {
          const Item z = sm[f];
          r += (item_less(z, y) || (f < e && !item_less(y, z))) ? 1 : 0;
        }
      }
      for (int o = 1; o < g; o <<= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
      if (e < ns && u == 0) {
        const int64_t off = r - (p / 2 - 1);  // rank (i)p + floor(p/2) - 1, 0-based
        if (off >= 0 && off % p == 0 && off / p < p - 1) {
          piv[off / p] = y;
          if (pivot_idx) pivot_idx[S.piv_base + off / p] = y.idx;
        }
      }
      __syncthreads();
      continue;
    }
    for (int64_t e = threadIdx.x; e < ns; e += blockDim.x) {
      const int64_t b = e / (p - 1), j = e % (p - 1) + 1;
      const int64_t lo = block_lo(b, n, p), w = block_lo(b + 1, n, p) - lo;
      Y[e] = it[lo + j * w / p];
    }
    __syncthreads();
    cta_sort(Y, Y2, ns, sm);
    for (int64_t i = threadIdx.x; i < p - 1; i += blockDim.x) {
      const Item y = Y[i * p + p / 2 - 1];  // Y_{(i)p + floor(p/2)}, 1-based
      piv[i] = y;
      if (pivot_idx) pivot_idx[S.piv_base + i] = y.idx;
    }
    __syncthreads();
  }
}

// pos[b][i] = items of sorted block b that are <= y_i (i < p-1); pos[b][p-1] = w_b.
// blockIdx.y = set.
__global__ void subblocks_kernel(const Item *items, const Item *piv_all, int32_t *pos_all,
                                 const PartSet *sets) {
  pdl_enter();
  const PartSet S = sets[blockIdx.y];
  const int64_t n = S.n, p = S.p, total = p * p;
  const Item *it = items + S.seq_begin;
  const Item *piv = piv_all + S.piv_base;
  int32_t *pos = pos_all + S.pos_base;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = e / p, i = e % p;
    const int64_t lo = block_lo(b, n, p), w = block_lo(b + 1, n, p) - lo;
    pos[e] = (int32_t)(i == p - 1 ? w : count_not_greater(it + lo, w, piv[i]));
  }
}

// One block per set: bucket sizes, CSR offsets (local, written at blk_base + set),
// the global start of every bucket (gbound) and of every sub-block (dest).
__global__ void __launch_bounds__(1024) bucket_scan_kernel(const int32_t *pos_all,
                                                           int32_t *dest_all,
                                                           int32_t *bucket_offsets,
                                                           int64_t *gbound,
                                                           const PartSet *sets,
                                                           int32_t n_sets) {
  pdl_enter();
  __shared__ int32_t s_warp[32];
  __shared__ int32_t s_carry;
  const int tid = threadIdx.x;
  for (int32_t si = blockIdx.x; si < n_sets; si += gridDim.x) {
    const PartSet S = sets[si];
    const int p = S.p;
    const int32_t *pos = pos_all + S.pos_base;
    int32_t *dest = dest_all + S.pos_base;
    int32_t *boff = bucket_offsets + S.blk_base + si;
    if (tid == 0) s_carry = 0;
    __syncthreads();
    for (int base = 0; base < p; base += blockDim.x) {
      const int i = base + tid;
      int32_t size = 0;
      if (i < p)
        for (int b = 0; b < p; ++b)
          size += pos[(int64_t)b * p + i] - (i > 0 ? pos[(int64_t)b * p + i - 1] : 0);
      int32_t x = size;
      for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if ((tid & 31) >= o) x += y;
      }
      if ((tid & 31) == 31) s_warp[tid >> 5] = x;
      __syncthreads();
      if (tid < 32) {
        int32_t w = s_warp[tid];
        for (int o = 1; o < 32; o <<= 1) {
          const int32_t y = __shfl_up_sync(0xffffffffu, w, o);
          if (tid >= o) w += y;
        }
        s_warp[tid] = w;
      }
      __syncthreads();
      const int32_t incl = x + ((tid >> 5) > 0 ? s_warp[(tid >> 5) - 1] : 0) + s_carry;
      if (i < p) {
        int32_t at = incl - size;
        boff[i] = at;
        gbound[S.blk_base + i] = S.seq_begin + at;
        for (int b = 0; b < p; ++b) {
          dest[(int64_t)b * p + i] = (int32_t)(S.seq_begin + at);
          at += pos[(int64_t)b * p + i] - (i > 0 ? pos[(int64_t)b * p + i - 1] : 0);
        }
      }
      __syncthreads();
      if (tid == blockDim.x - 1) s_carry = incl;
      __syncthreads();
    }
    if (tid == 0) {
      boff[p] = S.n;
      gbound[S.blk_base + p] = S.seq_begin + S.n;
    }
    __syncthreads();
  }
}

__global__ void scatter_kernel(const Item *items, Item *out, const int32_t *pos_all,
                               const int32_t *dest_all, int64_t n_total, const PartSet *sets,
                               int32_t n_sets) {
  pdl_enter();
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n_total;
       x += (int64_t)gridDim.x * blockDim.x) {
    const PartSet S = sets[set_of(sets, n_sets, x)];
    const int64_t n = S.n, p = S.p, xl = x - S.seq_begin;
    int64_t b = xl * p / n;
    while (b + 1 < p && block_lo(b + 1, n, p) <= xl) ++b;
    while (b > 0 && block_lo(b, n, p) > xl) --b;
    const int64_t e = xl - block_lo(b, n, p);
    const int32_t *pb = pos_all + S.pos_base + b * p;
    int lo = 0, hi = (int)p - 1;  // first i with e < pos[b][i]
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (e < pb[mid]) hi = mid; else lo = mid + 1;
    }
    const int64_t start = lo > 0 ? pb[lo - 1] : 0;
    out[dest_all[S.pos_base + b * p + lo] + (e - start)] = items[x];
  }
}

// ---------------------------------------------------------------------------
// One set with p <= kFastP and blocks of at most kFastChunks chunks: more CTAs and
// no second sort. Each block's chunks of kChunk items are sorted by one CTA each,
// and an item's place in its sorted block is its place in its chunk plus the
// number of smaller items in each other chunk (binary searches; all items differ).
// After the pivots, the items of bucket i arrive as p sorted runs (its sub-block
// of every block), so an item's place in its bucket is, the same way, its place
// in its run plus the smaller items of the other runs; members are written there.
constexpr int kChunk = 256;
constexpr int kFastChunks = 64;
constexpr int kFastP = 64;

// (blockIdx.y = block b, blockIdx.x = chunk of the block): sort it in place.
__global__ void __launch_bounds__(128) chunk_sort_kernel(Item *items, const int64_t *segoff) {
  pdl_enter();
  __shared__ Item sm[kChunk];
  const int64_t a = segoff[blockIdx.y], e = segoff[blockIdx.y + 1];
  const int64_t lo = a + (int64_t)blockIdx.x * kChunk;
  if (lo >= e) return;
  cta_sort_small(items + lo, (int)min((int64_t)kChunk, e - lo), sm);
}

__device__ __forceinline__ int64_t block_of_item(int64_t x, int64_t n, int64_t p) {
  int64_t b = x * p / n;
  while (b + 1 < p && block_lo(b + 1, n, p) <= x) ++b;
  while (b > 0 && block_lo(b, n, p) > x) --b;
  return b;
}

// Thread per item: its place in its chunk plus the smaller items of the block's
// other chunks (a few binary searches).
__global__ void chunk_merge_kernel(const Item *__restrict__ in, Item *__restrict__ out,
                                   int64_t n, int64_t p) {
  pdl_enter();
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
       x += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = block_of_item(x, n, p);
    const int64_t lo = block_lo(b, n, p), e = block_lo(b + 1, n, p);
    const int64_t c = (x - lo) / kChunk;
    const Item it = in[x];
    int64_t rank = x - (lo + c * kChunk);
    for (int64_t c2 = 0; lo + c2 * kChunk < e; ++c2) {
      if (c2 == c) continue;
      const int64_t a = lo + c2 * kChunk;
      rank += count_less(in + a, min((int64_t)kChunk, e - a), it);
    }
    out[lo + rank] = it;
  }
}

// Warp per item of the sorted blocks: its bucket, then the lanes count the smaller
// items of the bucket's other runs; members in bucket order (offsets in boff).
__global__ void bucket_place_kernel(const Item *__restrict__ sorted, const int32_t *pos,
                                    const int32_t *boff, int32_t *members, int64_t n,
                                    int64_t p) {
  pdl_enter();
  const int lane = threadIdx.x & 31;
  for (int64_t x = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; x < n;
       x += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int64_t b = block_of_item(x, n, p);
    const int64_t e = x - block_lo(b, n, p);
    const int32_t *pb = pos + b * p;
    int lo = 0, hi = (int)p - 1;  // bucket: first i with e < pos[b][i]
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (e < pb[mid]) hi = mid; else lo = mid + 1;
    }
    const int i = lo;
    const Item it = sorted[x];
    int64_t rank = 0;
    for (int64_t b2 = lane; b2 < p; b2 += 32) {
      if (b2 == b) continue;
      const int32_t *q = pos + b2 * p;
      const int64_t a = block_lo(b2, n, p) + (i > 0 ? q[i - 1] : 0);
      rank += count_less(sorted + a, q[i] - (i > 0 ? q[i - 1] : 0), it);
    }
    for (int o = 16; o > 0; o >>= 1) rank += __shfl_xor_sync(0xffffffffu, rank, o);
    if (lane == 0) members[boff[i] + rank + e - (i > 0 ? pb[i - 1] : 0)] = it.idx;
  }
}

__global__ void members_kernel(const Item *items, int32_t *members, int64_t n) {
  pdl_enter();
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
       x += (int64_t)gridDim.x * blockDim.x)
    members[x] = items[x].idx;
}

inline unsigned grid_for(int64_t work, int threads) {
  int64_t g = (work + threads - 1) / threads;
  const int64_t cap = (int64_t)num_sms() * 8;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (unsigned)g;
}

bool g_sort_attr = false;

}  // namespace

// Partition of n_sets consecutive sets (sizes d_n / p per set d_p on the device; or
// one set of n_single items into p_single buckets when d_n == nullptr). Outputs per
// set s: bucket_offsets[blk_base_s + s ..] (p_s + 1 local offsets), members (local
// indices, in the sets' item ranges), pivot_idx[piv_base_s ..] (p_s - 1).
int partition_sets_launch(const uint64_t *key_hi, const uint64_t *key_lo, int32_t n_sets,
                          const int32_t *d_n, const int32_t *d_p, int32_t n_single,
                          int32_t p_single, const PartTotals &tot, int32_t max_p,
                          int32_t *bucket_offsets, int32_t *members, int32_t *pivot_idx,
                          void *ws, cudaStream_t st) {
  const PartLayout L = part_layout_sets(n_sets, tot);
  uint8_t *b = static_cast<uint8_t *>(ws);
  PartSet *sets = reinterpret_cast<PartSet *>(b + L.sets);
  int64_t *segoff = reinterpret_cast<int64_t *>(b + L.segoff);
  int64_t *gbound = reinterpret_cast<int64_t *>(b + L.gbound);
  Item *items = reinterpret_cast<Item *>(b + L.items);
  Item *items2 = reinterpret_cast<Item *>(b + L.items2);
  Item *Y = reinterpret_cast<Item *>(b + L.samples);
  Item *Y2 = reinterpret_cast<Item *>(b + L.samples2);
  int32_t *pos = reinterpret_cast<int32_t *>(b + L.pos);
  int32_t *dest = reinterpret_cast<int32_t *>(b + L.dest);
  Item *piv = reinterpret_cast<Item *>(b + L.pivots);
  if (!g_sort_attr) {
    if (cudaFuncSetAttribute(seg_sort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kSortSmem) != cudaSuccess ||
        cudaFuncSetAttribute(samples_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kSortSmem) != cudaSuccess)
      return SAD_ERR_CUDA;
    g_sort_attr = true;
  }
  const int64_t n = tot.n;
  const unsigned gsets = (unsigned)(n_sets < 65535 ? n_sets : 65535);
  const unsigned gseg = (unsigned)(tot.p < 65535 * 4 ? tot.p : 65535 * 4);
  if (n_sets == 1 && !d_n && !d_p) {
    pdl_launch(part_init_single_kernel, grid_for(n, 256), 256, 0, st, key_hi, key_lo, n,
               (int64_t)p_single, sets, segoff, items);
    SAD_LAUNCH_CHECK();
  } else {
    pdl_launch(part_setup_kernel, 1, 1024, 0, st, d_n, d_p, n_sets, n_single, p_single, sets,
               segoff);
    SAD_LAUNCH_CHECK();
    pdl_launch(part_init_kernel, grid_for(n, 256), 256, 0, st, key_hi, key_lo, n, sets, n_sets,
               items);
    SAD_LAUNCH_CHECK();
  }
  // one set of small blocks and few buckets: chunk sorts and rank merges
  const int64_t w_max = d_n || p_single < 1 ? 0 : ((int64_t)n_single + p_single - 1) / p_single;
  if (!d_n && n_single > 0 && p_single <= kFastP && w_max <= (int64_t)kFastChunks * kChunk) {
    dim3 gc((unsigned)((w_max + kChunk - 1) / kChunk), (unsigned)p_single);
    pdl_launch(chunk_sort_kernel, gc, 128, 0, st, items, segoff);
    SAD_LAUNCH_CHECK();
    pdl_launch(chunk_merge_kernel, grid_for(n, 128), 128, 0, st, items, items2, n, p_single);
    SAD_LAUNCH_CHECK();
    if (max_p > 1) {
      pdl_launch(samples_kernel, gsets, kSortThreads, kSortSmem, st, items2, Y, Y2, piv, pivot_idx,
                 sets, n_sets);
      SAD_LAUNCH_CHECK();
    }
    {
      const int64_t pp = (int64_t)max_p * max_p;
      dim3 g((unsigned)((pp + 255) / 256 < 1024 ? (pp + 255) / 256 : 1024), (unsigned)n_sets);
      pdl_launch(subblocks_kernel, g, 256, 0, st, items2, piv, pos, sets);
      SAD_LAUNCH_CHECK();
    }
    pdl_launch(bucket_scan_kernel, gsets, 1024, 0, st, pos, dest, bucket_offsets, gbound, sets,
               n_sets);
    SAD_LAUNCH_CHECK();
    // a warp per item, all resident at once
    pdl_launch(bucket_place_kernel,
               (unsigned)((n * 32 + 255) / 256 < 65535 * 16 ? (n * 32 + 255) / 256 : 65535 * 16),
               256, 0, st, items2, pos, bucket_offsets, members, n, p_single);
    SAD_LAUNCH_CHECK();
    return SAD_OK;
  }
  pdl_launch(seg_sort_kernel, gseg, kSortThreads, kSortSmem, st, items, items2, tot.p, segoff);
  SAD_LAUNCH_CHECK();
  if (max_p > 1) {
    pdl_launch(samples_kernel, gsets, kSortThreads, kSortSmem, st, items, Y, Y2, piv, pivot_idx,
               sets, n_sets);
    SAD_LAUNCH_CHECK();
  }
  {
    const int64_t pp = (int64_t)max_p * max_p;
    dim3 g((unsigned)((pp + 255) / 256 < 1024 ? (pp + 255) / 256 : 1024), (unsigned)n_sets);
    pdl_launch(subblocks_kernel, g, 256, 0, st, items, piv, pos, sets);
    SAD_LAUNCH_CHECK();
  }
  pdl_launch(bucket_scan_kernel, gsets, 1024, 0, st, pos, dest, bucket_offsets, gbound, sets,
             n_sets);
  SAD_LAUNCH_CHECK();
  pdl_launch(scatter_kernel, grid_for(n, 256), 256, 0, st, items, items2, pos, dest, n, sets,
             n_sets);
  SAD_LAUNCH_CHECK();
  pdl_launch(seg_sort_kernel, gseg, kSortThreads, kSortSmem, st, items2, items, tot.p, gbound);
  SAD_LAUNCH_CHECK();
  pdl_launch(members_kernel, grid_for(n, 256), 256, 0, st, items2, members, n);
  SAD_LAUNCH_CHECK();
  return SAD_OK;
}

int partition_launch(const uint64_t *key_hi, const uint64_t *key_lo, int32_t n, int32_t p,
                     int32_t *bucket_offsets, int32_t *members, int32_t *pivot_idx, void *ws,
                     cudaStream_t st) {
  return partition_sets_launch(key_hi, key_lo, 1, nullptr, nullptr, n, p,
                               part_totals_single(n, p), p, bucket_offsets, members, pivot_idx,
                               ws, st);
}

}  // namespace sad
