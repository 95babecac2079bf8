// Preparation of the threshold-plane GEMM behind kmer_rank.
//
// Eq. 1's numerator S(X,Y) = sum_tau min(c^X_tau, c^Y_tau) is rewritten with the
// exact identity min(a, b) = sum_{t>=1} [a >= t][b >= t]: with one 0/1 column
// per (word tau, threshold t), t = 1..T_tau, T_tau = max_x c^x_tau, the matrix
// P[x][(tau,t)] = [c^x_tau >= t] satisfies S = P P^T. The columns are laid out
// threshold-major: section t holds the words with T_tau >= t, so the first
// sections are the dense ones and a tile whose rows never count any word more
// than d times only needs the first d sections (its K extent).
//
// Depth cap. Only the sections t = 1..D may be kept as planes (D = the plan's
// depth; 0 keeps all). What the planes miss is exact too:
//   min(a, b) = sum_{t=1..D} [a >= t][b >= t] + max(0, min(a, b) - D),
// and the second term is nonzero only for words both sequences hold more than
// D times. Each such (set, word) gets a list of (stored row, count - D); every
// pair in a list adds min of the two excesses to that pair's residual, which is
// summed into a dense 128 x 128 u16 block of its GEMM tile and added to the
// tile's accumulator in the epilogue, before the floor.
//
// Sets. A call ranks one or more independent sets (a batch). Each set's rows are
// stored contiguously (128-aligned) and its tiles only pair rows of that set, so
// the GEMM is block-diagonal; the column layout is shared (T over all sets).
// Within a set, rows are stored in order of decreasing length (the order of
// equal lengths is free: it changes no result), so that for every stored pair
// i <= j the Eq. 1 denominator is min(L_i, L_j) - k + 1 = m_j, the column's own.
//
// Kernels, in launch order:
//   rank_setup     the set table (row, tile and tile-map bases per set)
//   rank_setmaps   set index of every sequence and stored row (batches only)
//   rank_init      zero the scratch regions of the workspace
//   lengths        m = L - k + 1, validation, histogram of m (one set)
//   colmax         T_tau = max_x c^x_tau, count validation, #{x : c^x_tau > D}
//   colmap         t_max, section ends, K_eff at depth D, the column map
//   list_scan_*    offsets of the excess lists and of their pair ranges
//   lensort_*      stored row of every sequence, per-row division records
//   planes         P rows as packed e2m1 (2 = 1.0, 0 = 0.0), block depths,
//                  excess-list entries
//   tiles          per set, the upper-triangle tile list with per-tile K extent
//   residual_*     give residual blocks to tiles, zero them, add every pair
#include "rank.cuh"
#include "sort.cuh"

namespace sad {

RankPtrs rank_ptrs(void *ws, const RankLayout &L) {
  uint8_t *b = static_cast<uint8_t *>(ws);
  RankPtrs P;
  P.hdr = reinterpret_cast<WsHeader *>(b);
  P.sets = reinterpret_cast<RankSet *>(b + L.sets);
  P.seq_set = reinterpret_cast<int32_t *>(b + L.seq_set);
  P.row_set = reinterpret_cast<int32_t *>(b + L.row_set);
  P.T = reinterpret_cast<int32_t *>(b + L.T);
  P.secend = reinterpret_cast<int32_t *>(b + L.secend);
  P.colmap = reinterpret_cast<int32_t *>(b + L.colmap);
  P.thist = reinterpret_cast<int32_t *>(b + L.thist);
  P.coltab = reinterpret_cast<int32_t *>(b + L.coltab);
  P.promcol = reinterpret_cast<int32_t *>(b + L.promcol);
  P.weight = reinterpret_cast<int64_t *>(b + L.weight);
  P.mhist = reinterpret_cast<int32_t *>(b + L.mhist);
  P.perm = reinterpret_cast<int32_t *>(b + L.perm);
  P.rec = reinterpret_cast<uint4 *>(b + L.rec);
  P.recw = reinterpret_cast<uint2 *>(b + L.recw);
  P.depth = reinterpret_cast<int32_t *>(b + L.depth);
  P.tiles = reinterpret_cast<int2 *>(b + L.tiles);
  P.acc = reinterpret_cast<unsigned long long *>(b + L.acc);
  P.planes = b + L.planes;
  P.cnt_gt = reinterpret_cast<int32_t *>(b + L.cnt_gt);
  P.list_off = reinterpret_cast<int64_t *>(b + L.list_off);
  P.item_off = reinterpret_cast<int64_t *>(b + L.item_off);
  P.cursor = reinterpret_cast<int32_t *>(b + L.cursor);
  P.lists = reinterpret_cast<int2 *>(b + L.lists);
  P.flat = reinterpret_cast<int2 *>(b + L.flat);
  P.tile_of = reinterpret_cast<int32_t *>(b + L.tile_of);
  P.block_of = reinterpret_cast<int32_t *>(b + L.block_of);
  P.rblocks = reinterpret_cast<uint32_t *>(b + L.rblocks);
  P.sortbuf = reinterpret_cast<Item *>(b + L.sortbuf);
  P.scanblk = reinterpret_cast<int64_t *>(b + L.scanblk);
  P.n_pad = L.shape.rows_total;
  P.n_total = L.shape.n_total;
  P.n_sets = L.shape.n_sets;
  P.tiles_total = L.shape.tiles_total;
  P.k_cap = L.caps.k_cap;
  P.list_cap = L.caps.list_cap;
  P.block_cap = L.caps.block_cap;
  P.depth_cap = L.caps.depth;
  P.wait_ns = gemm_wait_ns();
  return P;
}

namespace {

template <typename T>
__device__ __forceinline__ void zero_range(T *p, int64_t count, int64_t tid, int64_t nthreads) {
  for (int64_t i = tid; i < count; i += nthreads) p[i] = T(0);
}

// Inclusive prefix sum of x over the block's threads in thread order; every
// thread must call it. s_warp: 32 slots of shared memory. Returns the prefix and
// writes the block total to *total.
template <typename V>
__device__ __forceinline__ V block_scan_incl(V x, V *s_warp, V *total) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  for (int o = 1; o < 32; o <<= 1) {
    const V y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[wid] = x;
  __syncthreads();
  if (wid == 0) {
    V w = lane < nw ? s_warp[lane] : V(0);
    for (int o = 1; o < 32; o <<= 1) {
      const V y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    s_warp[lane] = w;
  }
  __syncthreads();
  const V r = x + (wid > 0 ? s_warp[wid - 1] : V(0));
  *total = s_warp[nw - 1];
  __syncthreads();
  return r;
}

__device__ __forceinline__ int64_t dev_n_pad(int64_t n) {
  return ((n > 0 ? n : 1) + kNPad - 1) / kNPad * kNPad;
}

__device__ __forceinline__ int64_t dev_tiles_of_set(int64_t n) {
  const int64_t R = (n + kRowBlock - 1) / kRowBlock, C = (n + kColBlock - 1) / kColBlock;
  int64_t total = 0;  // sum over I < R of max(0, C - floor(I / kColRatio))
  for (int64_t I = 0; I < R; ++I) {
    const int64_t j0 = I / kColRatio;
    if (j0 < C) total += C - j0;
  }
  return total;
}

__device__ __forceinline__ int32_t set_of_seq(const RankPtrs &P, int64_t x) {
  return P.n_sets > 1 ? P.seq_set[x] : 0;
}

__device__ __forceinline__ int32_t set_of_row(const RankPtrs &P, int64_t r) {
  return P.n_sets > 1 ? P.row_set[r] : 0;
}

// One block: the set table (prefix sums of n, padded rows, tiles, tile-map size).
__global__ void __launch_bounds__(1024) rank_setup_kernel(const int32_t *d_n, int32_t n1,
                                                          RankPtrs P) {
  pdl_enter();
  __shared__ int64_t s_warp[32];
  __shared__ int64_t s_c[4];
  const int tid = threadIdx.x;
  const int32_t S = (int32_t)P.n_sets;
  if (tid < 4) s_c[tid] = 0;
  __syncthreads();
  for (int base = 0; base < S; base += blockDim.x) {
    const int s = base + tid;
    const int64_t n = s < S ? (d_n ? d_n[s] : n1) : 0;
    const int64_t np = s < S ? dev_n_pad(n) : 0;
    const int64_t v[4] = {n, np, s < S ? dev_tiles_of_set(n) : 0,
                          (np / kRowBlock) * (np / kColBlock)};
    int64_t ex[4];
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      int64_t tot;
      const int64_t incl = block_scan_incl<int64_t>(v[f], s_warp, &tot);
      ex[f] = s_c[f] + incl - v[f];
      __syncthreads();
      if (tid == 0) s_c[f] += tot;
      __syncthreads();
    }
    if (s < S) {
      RankSet e;
      e.seq_begin = ex[0];
      e.row_base = ex[1];
      e.tile_base = ex[2];
      e.tileof_base = ex[3];
      e.n = (int32_t)n;
      e.pad = 0;
      P.sets[s] = e;
    }
  }
}

// Set index of every input sequence and every stored row (batches only).
__global__ void rank_setmaps_kernel(RankPtrs P) {
  pdl_enter();
  for (int32_t s = blockIdx.x; s < (int32_t)P.n_sets; s += gridDim.x) {
    const RankSet e = P.sets[s];
    for (int64_t i = threadIdx.x; i < e.n; i += blockDim.x) P.seq_set[e.seq_begin + i] = s;
    const int64_t np = dev_n_pad(e.n);
    for (int64_t i = threadIdx.x; i < np; i += blockDim.x) P.row_set[e.row_base + i] = s;
  }
}

__global__ void rank_init_kernel(RankPtrs P, int32_t eps, int with_keys) {
  pdl_enter();
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nt = (int64_t)gridDim.x * blockDim.x;
  const int64_t we = P.n_sets * (int64_t)eps;
  zero_range(P.T, eps, tid, nt);
  zero_range(P.thist, kMaxM + 2, tid, nt);
  zero_range(P.mhist, kMaxM + 2, tid, nt);
  zero_range(P.secend, kMaxM + 2, tid, nt);
  zero_range(P.cnt_gt, we, tid, nt);
  zero_range(P.cursor, we, tid, nt);
  if (with_keys) {
    zero_range(P.depth, P.n_pad / kRowBlock, tid, nt);
    zero_range(P.acc, 3 * P.n_total, tid, nt);
  }
  if (tid == 0) {
    P.hdr->k_eff = 0;
    P.hdr->k_pad = 0;
    P.hdr->t_max = 0;
    P.hdr->n_tiles = 0;
    P.hdr->k_chunks = 0;
    P.hdr->depth = 0;
    P.hdr->list_total = 0;
    P.hdr->pairs_total = 0;
    P.hdr->n_blocks = 0;
    P.hdr->m_max = 0;
    P.hdr->n_promoted = 0;
    P.hdr->k_ext = 0;
    P.hdr->flat_count = 0;
  }
}

__global__ void lengths_kernel(const int32_t *__restrict__ lengths, int32_t k, RankPtrs P) {
  pdl_enter();
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < P.n_total;
       x += (int64_t)gridDim.x * blockDim.x) {
    const int32_t m = lengths[x] - k + 1;
    if (m < 1) {
      record_error(P.hdr, SAD_ERR_BAD_INPUT, (int)x);
    } else if (m > kMaxM) {
      record_error(P.hdr, SAD_ERR_UNSUPPORTED, (int)x);
    } else {
      if (P.n_sets == 1) atomicAdd(&P.mhist[m], 1);
      atomicMax(&P.hdr->m_max, m);
    }
  }
}

// T_tau = max over rows of counts[x][tau] and (D >= 1) the number of rows of each
// set whose count exceeds D. Block (256 words) x (row slice).
__global__ void colmax_kernel(const int32_t *__restrict__ counts, int32_t eps, RankPtrs P,
                              int count_gt) {
  pdl_enter();
  const int32_t tau = blockIdx.x * blockDim.x + threadIdx.x;
  if (tau >= eps) return;
  const int32_t D = count_gt ? P.depth_cap : 0;
  const int64_t n = P.n_total;
  const int64_t per = (n + gridDim.y - 1) / gridDim.y;
  const int64_t r0 = (int64_t)blockIdx.y * per;
  const int64_t r1 = r0 + per < n ? r0 + per : n;
  int32_t mx = 0, mn = 0, gt = 0;
  int32_t cur = r0 < r1 ? set_of_seq(P, r0) : 0;
  int64_t r = r0;
  if (P.n_sets == 1) {
    for (; r + 4 <= r1; r += 4) {
      const int32_t a = __ldg(counts + (r + 0) * eps + tau);
      const int32_t b = __ldg(counts + (r + 1) * eps + tau);
      const int32_t c = __ldg(counts + (r + 2) * eps + tau);
      const int32_t d = __ldg(counts + (r + 3) * eps + tau);
      mx = max(mx, max(max(a, b), max(c, d)));
      mn = min(mn, min(min(a, b), min(c, d)));
      gt += (a > D) + (b > D) + (c > D) + (d > D);
    }
  } else {
    for (; r + 4 <= r1; r += 4) {
      int32_t v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = __ldg(counts + (r + u) * eps + tau);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        mx = max(mx, v[u]);
        mn = min(mn, v[u]);
        const int32_t s = P.seq_set[r + u];
        if (s != cur) {
          if (D >= 1 && gt) atomicAdd(&P.cnt_gt[(int64_t)cur * eps + tau], gt);
          gt = 0;
          cur = s;
        }
        gt += v[u] > D;
      }
    }
  }
  for (; r < r1; ++r) {
    const int32_t a = __ldg(counts + r * eps + tau);
    mx = max(mx, a);
    mn = min(mn, a);
    const int32_t s = set_of_seq(P, r);
    if (s != cur) {
      if (D >= 1 && gt) atomicAdd(&P.cnt_gt[(int64_t)cur * eps + tau], gt);
      gt = 0;
      cur = s;
    }
    gt += a > D;
  }
  if (mn < 0) record_error(P.hdr, SAD_ERR_BAD_INPUT, tau);
  if (mx > kMaxM) record_error(P.hdr, SAD_ERR_UNSUPPORTED, tau);
  if (mx > 0) atomicMax(&P.T[tau], mx);
  if (D >= 1 && gt) atomicAdd(&P.cnt_gt[(int64_t)cur * eps + tau], gt);
}

// T_tau taken from a per-word maximum computed while counting.
__global__ void copy_word_max_kernel(const int32_t *__restrict__ word_max, int32_t eps,
                                     RankPtrs P) {
  pdl_enter();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < eps; i += gridDim.x * blockDim.x) {
    const int32_t t = word_max[i];
    if (t < 0) record_error(P.hdr, SAD_ERR_BAD_INPUT, i);
    if (t > kMaxM) record_error(P.hdr, SAD_ERR_UNSUPPORTED, i);
    P.T[i] = t;
  }
}

// One block of 1024 threads: histogram of T, t_max, section ends secend[t] =
// sum_{t'<=t} #{tau : T_tau >= t'}, K_eff at the depth cap and (unless plan_only)
// the column map colmap[col] = tau | t << 16.
__global__ void __launch_bounds__(1024) colmap_kernel(RankPtrs P, int32_t eps, int plan_only) {
  pdl_enter();
  __shared__ int32_t s_tmax;
  __shared__ int32_t s_warp[32];
  __shared__ int32_t s_carry;
  const int tid = threadIdx.x;
  if (tid == 0) s_tmax = 0;
  __syncthreads();
  int32_t local_max = 0;
  for (int tau = tid; tau < eps; tau += blockDim.x) {
    const int32_t t = min(P.T[tau], kMaxM);
    local_max = max(local_max, t);
    // most words share a few values of T: one atomic per value per warp
    const unsigned same = __match_any_sync(__activemask(), t);
    if ((tid & 31) == __ffs(same) - 1) atomicAdd(&P.thist[t], __popc(same));
  }
  atomicMax(&s_tmax, local_max);
  __syncthreads();
  const int32_t tmax = s_tmax;
  // n_t = #{tau : T_tau >= t} = suffix sum of thist (into secend[t]), then the
  // prefix sums of n_t over t = 1..tmax (into secend[t]).
  if (tid == 0) s_carry = 0;
  __syncthreads();
  for (int base = tmax; base >= 1; base -= blockDim.x) {
    const int t = base - tid;
    int32_t tot;
    const int32_t incl = block_scan_incl<int32_t>(t >= 1 ? P.thist[t] : 0, s_warp, &tot);
    if (t >= 1) P.secend[t] = s_carry + incl;  // n_t
    __syncthreads();
    if (tid == 0) s_carry += tot;
    __syncthreads();
  }
  if (tid == 0) s_carry = 0;
  __syncthreads();
  for (int base = 1; base <= tmax; base += blockDim.x) {
    const int t = base + tid;
    int32_t tot;
    const int32_t incl = block_scan_incl<int32_t>(t <= tmax ? P.secend[t] : 0, s_warp, &tot);
    if (t <= tmax) P.secend[t] = s_carry + incl;
    __syncthreads();
    if (tid == 0) s_carry += tot;
    __syncthreads();
  }
  if (tid == 0) P.secend[0] = 0;
  __syncthreads();
  // planes kept: sections 1..dkeep; a residual exists when some count exceeds it
  const int32_t dkeep = P.depth_cap >= 1 ? min(P.depth_cap, tmax) : tmax;
  const int64_t k_eff = dkeep >= 1 ? (int64_t)P.secend[dkeep] : 0;
  int64_t k_pad = (k_eff + kKCols - 1) / kKCols * kKCols;
  if (k_pad < kKCols) k_pad = kKCols;
  if (tid == 0) {
    P.hdr->t_max = tmax;
    P.hdr->depth = dkeep;
    P.hdr->k_eff = k_eff;
    P.hdr->k_pad = (int32_t)k_pad;
  }
  if (plan_only) return;
  if (k_pad > P.k_cap) {
    if (tid == 0) record_error(P.hdr, SAD_ERR_WORKSPACE, (int)k_pad);
    return;
  }
  // Column map, sections in ascending word order: section 1 = the words with
  // T >= 1; section t + 1 = the words of section t with T >= t + 1 (a stable
  // compaction of the previous section, so the work is linear in K_eff). Columns
  // next to each other then look up nearby words when the planes are written.
  for (int t = 1; t <= dkeep; ++t) {
    if (t == 1 && P.secend[1] == eps) {
      // every word occurs somewhere: section 1 is the identity
      for (int c = tid; c < eps; c += blockDim.x) P.colmap[c] = c | (1 << 16);
      __syncthreads();
      continue;
    }
    const int32_t src_lo = t == 1 ? 0 : P.secend[t - 2];
    const int32_t src_n = t == 1 ? eps : P.secend[t - 1] - P.secend[t - 2];
    const int32_t dst_lo = P.secend[t - 1];
    if (src_n <= 32) {
      // short sections: one warp
      if (tid < 32) {
        const int32_t tau = tid < src_n ? (t == 1 ? tid : (P.colmap[src_lo + tid] & 0xFFFF)) : 0;
        const bool keep = tid < src_n && P.T[tau] >= t;
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        if (keep) P.colmap[dst_lo + __popc(m & ((1u << tid) - 1u))] = tau | (t << 16);
      }
    } else {
      if (tid == 0) s_carry = 0;
      __syncthreads();
      for (int base = 0; base < src_n; base += blockDim.x) {
        const int i = base + tid;
        int32_t tau = 0;
        if (i < src_n) tau = t == 1 ? i : (P.colmap[src_lo + i] & 0xFFFF);
        const int32_t keep = (i < src_n && P.T[tau] >= t) ? 1 : 0;
        int32_t tot;
        const int32_t incl = block_scan_incl<int32_t>(keep, s_warp, &tot);
        if (keep) P.colmap[dst_lo + s_carry + incl - 1] = tau | (t << 16);
        __syncthreads();
        if (tid == 0) s_carry += tot;
        __syncthreads();
      }
    }
    __syncthreads();
  }
  if (P.depth_cap >= 1 && P.depth_cap <= kTabDepth) {
    // the inverse map for the streaming plane writer: column of (t, word)
    for (int i = tid; i < dkeep * eps; i += blockDim.x) P.coltab[i] = -1;
    __syncthreads();
    for (int c = tid; c < k_eff; c += blockDim.x) {
      const int32_t e = P.colmap[c];
      P.coltab[(int64_t)((e >> 16) - 1) * eps + (e & 0xFFFF)] = c;
    }
  }
}

// Offsets of the excess lists over all (set, word) entries w: list_off[w] =
// prefix of c_w and item_off[w] = prefix of items(c_w), c_w = cnt_gt[w] (0 when
// nothing is cut), where items(c) counts the pairs of kPairChunk-entry chunks of
// a list of c entries (the residual's units of work). Three passes: per-block
// totals, a scan of the block totals, per-block scans with the block's carry.
// The number of residual pairs, sum c_w (c_w + 1) / 2, is added up on the side.
constexpr int kScanChunk = kScanChunkWords;
constexpr int kPairChunk = 128;

__host__ __device__ __forceinline__ int64_t items_of(int64_t c) {
  const int64_t n = (c + kPairChunk - 1) / kPairChunk;
  return n * (n + 1) / 2;
}

__device__ __forceinline__ bool residual_needed(const RankPtrs &P) {
  return P.hdr->depth < P.hdr->t_max;
}

__global__ void __launch_bounds__(256) list_scan_reduce_kernel(RankPtrs P, int64_t we) {
  pdl_enter();
  __shared__ int64_t s_warp[32];
  const bool on = residual_needed(P);
  const int64_t b0 = (int64_t)blockIdx.x * kScanChunk;
  int64_t sl = 0, sp = 0, sq = 0;
  for (int64_t w = b0 + threadIdx.x; w < b0 + kScanChunk && w < we; w += blockDim.x) {
    const int64_t c = on ? P.cnt_gt[w] : 0;
    sl += c;
    sp += items_of(c);
    sq += c * (c + 1) / 2;
  }
  int64_t tl, tp, tq;
  block_scan_incl<int64_t>(sl, s_warp, &tl);
  block_scan_incl<int64_t>(sp, s_warp, &tp);
  block_scan_incl<int64_t>(sq, s_warp, &tq);
  if (threadIdx.x == 0) {
    P.scanblk[2 * blockIdx.x] = tl;
    P.scanblk[2 * blockIdx.x + 1] = tp;
    if (tq) atomicAdd(reinterpret_cast<unsigned long long *>(&P.hdr->pairs_total),
                      (unsigned long long)tq);
  }
}

__global__ void __launch_bounds__(1024) list_scan_top_kernel(RankPtrs P, int64_t nblk) {
  pdl_enter();
  __shared__ int64_t s_warp[32];
  __shared__ int64_t s_l, s_p;
  if (threadIdx.x == 0) {
    s_l = 0;
    s_p = 0;
  }
  __syncthreads();
  for (int64_t base = 0; base < nblk; base += blockDim.x) {
    const int64_t b = base + threadIdx.x;
    const int64_t vl = b < nblk ? P.scanblk[2 * b] : 0;
    const int64_t vp = b < nblk ? P.scanblk[2 * b + 1] : 0;
    int64_t tl, tp;
    const int64_t il = block_scan_incl<int64_t>(vl, s_warp, &tl);
    const int64_t ip = block_scan_incl<int64_t>(vp, s_warp, &tp);
    if (b < nblk) {
      P.scanblk[2 * b] = s_l + il - vl;  // exclusive carry of block b
      P.scanblk[2 * b + 1] = s_p + ip - vp;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      s_l += tl;
      s_p += tp;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    P.hdr->list_total = s_l;
    P.hdr->items_total = s_p;
  }
}

__global__ void __launch_bounds__(256) list_scan_down_kernel(RankPtrs P, int64_t we,
                                                             int plan_only) {
  pdl_enter();
  __shared__ int64_t s_warp[32];
  __shared__ int64_t s_l, s_p;
  const bool on = residual_needed(P);
  const int64_t b0 = (int64_t)blockIdx.x * kScanChunk;
  if (threadIdx.x == 0) {
    s_l = P.scanblk[2 * blockIdx.x];
    s_p = P.scanblk[2 * blockIdx.x + 1];
  }
  __syncthreads();
  for (int64_t base = b0; base < b0 + kScanChunk && base < we; base += blockDim.x) {
    const int64_t w = base + threadIdx.x;
    const int64_t c = (on && w < we) ? P.cnt_gt[w] : 0;
    const int64_t pc = items_of(c);
    int64_t tl, tp;
    const int64_t il = block_scan_incl<int64_t>(c, s_warp, &tl);
    const int64_t ip = block_scan_incl<int64_t>(pc, s_warp, &tp);
    if (w < we) {
      P.list_off[w] = s_l + il - c;
      P.item_off[w] = s_p + ip - pc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      s_l += tl;
      s_p += tp;
    }
    __syncthreads();
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
    P.list_off[we] = P.hdr->list_total;
    P.item_off[we] = P.hdr->items_total;
    if (!plan_only && (P.hdr->list_total > P.list_cap || (on && P.block_cap <= 0)))
      record_error(P.hdr, SAD_ERR_WORKSPACE, -1);
  }
}

// Planes in the K padding. K_eff is padded to a whole number of K chunks, so the
// GEMM multiplies K_pad - K_eff zero columns anyway; they are given the plane of
// threshold depth + 1 of the words with the most residual pairs (weight = sum over
// sets of cnt_gt^2, ties by word), at no cost in the GEMM. Their excess entries
// lose one (the new plane holds it) and leave the residual when nothing remains.
__global__ void promote_weight_kernel(RankPtrs P, int32_t eps) {
  pdl_enter();
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < eps;
       t += (int64_t)gridDim.x * blockDim.x) {
    int64_t w = 0;
    if (P.hdr->status == 0 && residual_needed(P))
      for (int64_t s = 0; s < P.n_sets; ++s) {
        const int64_t c = P.cnt_gt[s * eps + t];
        w += c * c;
      }
    P.weight[t] = w;
    P.promcol[t] = -1;
  }
}

// One block: the words with weight >= w*, w* the smallest threshold that selects at
// most K_pad - K_eff words (and only words with two or more excess sequences),
// numbered in word order after K_eff. w* is one above the (n_free + 1)-th largest
// weight, found by a radix select (8-bit digits from the top: a histogram of the
// candidates' digit, then the digit where the count from the top reaches the rank).
__global__ void __launch_bounds__(1024) promote_select_kernel(RankPtrs P, int32_t eps,
                                                              int staged) {
  pdl_enter();
  extern __shared__ int64_t s_w[];  // [eps] when staged
  __shared__ int32_t s_warp[32];
  __shared__ int32_t s_hist[257];  // + a bin for words that are not candidates
  __shared__ unsigned long long s_max, s_prefix;
  __shared__ int32_t s_rank, s_found;
  if (P.hdr->status != 0 || !residual_needed(P)) return;
  const int32_t k_eff = (int32_t)P.hdr->k_eff, n_free = P.hdr->k_pad - k_eff;
  if (n_free <= 0) return;
  const int tid = threadIdx.x;
  const uint64_t *w = reinterpret_cast<const uint64_t *>(staged ? s_w : P.weight);
  if (tid == 0) {
    s_max = 0;
    s_prefix = 0;
    s_rank = n_free + 1;
    s_found = 1;
  }
  if (staged)
    for (int t = tid; t < eps; t += blockDim.x) s_w[t] = P.weight[t];
  __syncthreads();
  {
    uint64_t mx = 0;
    for (int t = tid; t < eps; t += blockDim.x) mx = max(mx, w[t]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((tid & 31) == 0) atomicMax(&s_max, (unsigned long long)mx);
  }
  __syncthreads();
  int top = 0;
  while (top < 64 && (s_max >> top) > 255) top += 8;
  uint64_t mask = 0;
  for (int shift = top; shift >= 0; shift -= 8) {
    if (tid < 257) s_hist[tid] = 0;
    __syncthreads();
    const uint64_t prefix = s_prefix;
    // lanes with the same digit add together (most weights share the low digits)
    for (int base = 0; base < eps; base += blockDim.x) {
      const int t = base + tid;
      const bool cand = t < eps && (w[t] & mask) == prefix;
      const int d = cand ? (int)((w[t] >> shift) & 255) : 256;
      const unsigned same = __match_any_sync(0xffffffffu, d);
      if (cand && (tid & 31) == __ffs(same) - 1) atomicAdd(&s_hist[d], __popc(same));
    }
    __syncthreads();
    if (tid < 32) {
      // warp 0 walks the bins from the top: lane l holds bins 255-8l .. 248-8l
      const int32_t need = s_rank;
      int32_t mine = 0;
#pragma unroll
      for (int j = 0; j < 8; ++j) mine += s_hist[255 - 8 * tid - j];
      int32_t incl = mine;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (tid >= o) incl += v;
      }
      const unsigned hit = __ballot_sync(0xffffffffu, incl >= need);
      if (hit == 0) {  // fewer candidates than the rank: every weight is selectable
        if (tid == 0) {
          s_found = 0;
          s_prefix = prefix;
        }
      } else if (tid == __ffs(hit) - 1) {
        int32_t cum = incl - mine, d = 255 - 8 * tid;
        while (cum + s_hist[d] < need) cum += s_hist[d--];
        s_rank = need - cum;
        s_prefix = prefix | ((unsigned long long)d << shift);
      }
    }
    mask |= (uint64_t)255 << shift;
    __syncthreads();
    if (!s_found) break;
  }
  // the (n_free + 1)-th largest weight is s_prefix (when there are that many words)
  const uint64_t wstar = max((uint64_t)4, s_found ? (uint64_t)s_prefix + 1 : (uint64_t)0);
  // number the selected words in word order: each thread takes consecutive words
  const int per = (eps + blockDim.x - 1) / blockDim.x;
  const int t0 = tid * per;
  int32_t mine = 0;
  for (int t = t0; t < t0 + per && t < eps; ++t) mine += w[t] >= wstar ? 1 : 0;
  int32_t tot;
  const int32_t incl = block_scan_incl<int32_t>(mine, s_warp, &tot);
  int32_t next = k_eff + incl - mine;
  for (int t = t0; t < t0 + per && t < eps; ++t)
    if (w[t] >= wstar) P.promcol[t] = next++;
  if (tid == 0) {
    P.hdr->n_promoted = tot;
    P.hdr->k_ext = k_eff + tot;
    P.hdr->k_eff = k_eff + tot;
  }
}

// Excess entries of promoted words: the plane value at the word's new column, one
// less excess; entries left with none are dropped (row -1) and uncounted.
__global__ void promote_apply_kernel(RankPtrs P, int32_t eps) {
  pdl_enter();
  if (P.hdr->status != 0 || !residual_needed(P) || P.hdr->n_promoted == 0) return;
  const int64_t total = min((int64_t)P.hdr->flat_count, P.list_cap);
  const int64_t row_words = P.k_cap / 8;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int2 e = P.flat[i];
    const int32_t tau = e.y & 0xFFFF, ex = (int32_t)((uint32_t)e.y >> 16);
    const int32_t col = P.promcol[tau];
    if (col < 0) continue;
    atomicOr(reinterpret_cast<unsigned int *>(P.planes) + (int64_t)e.x * row_words + (col >> 3),
             kE2M1One << (4 * (col & 7)));
    if (ex > 1) {
      P.flat[i] = make_int2(e.x, tau | ((ex - 1) << 16));
    } else {
      atomicSub(&P.cnt_gt[(int64_t)set_of_row(P, e.x) * eps + tau], 1);
      P.flat[i] = make_int2(-1, e.y);
    }
  }
}

// Excess entries from the unordered append into their (set, word) lists.
__global__ void group_lists_kernel(RankPtrs P, int32_t eps) {
  pdl_enter();
  if (P.hdr->status != 0 || !residual_needed(P)) return;
  const int64_t total = (int64_t)P.hdr->flat_count;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int2 e = P.flat[i];
    if (e.x < 0) continue;  // all of its excess went into a promoted plane
    const int32_t tau = e.y & 0xFFFF, ex = (int32_t)((uint32_t)e.y >> 16);
    const int64_t w = (int64_t)set_of_row(P, e.x) * eps + tau;
    const int32_t slot = atomicAdd(&P.cursor[w], 1);
    P.lists[P.list_off[w] + slot] = make_int2(e.x, ex);
  }
}

// One set: exclusive prefix over m in decreasing order, mhist[m] := #{x : m_x > m},
// for m = m_max down to 1, 1024 consecutive values per step.
__global__ void __launch_bounds__(1024) lensort_scan_kernel(RankPtrs P) {
  pdl_enter();
  __shared__ int32_t s_warp[32];
  __shared__ int32_t s_carry;
  const int tid = threadIdx.x;
  const int32_t m_max = P.hdr->m_max;
  if (tid == 0) s_carry = 0;
  __syncthreads();
  for (int base = m_max; base >= 1; base -= blockDim.x) {
    const int m = base - tid;
    const int32_t v = m >= 1 ? P.mhist[m] : 0;
    int32_t tot;
    const int32_t incl = block_scan_incl<int32_t>(v, s_warp, &tot);
    if (m >= 1) P.mhist[m] = s_carry + incl - v;
    __syncthreads();
    if (tid == 0) s_carry += tot;
    __syncthreads();
  }
}

// One set: stored row of every sequence from the counting sort over m.
__global__ void lensort_place_kernel(const int32_t *__restrict__ lengths, int32_t k,
                                     RankPtrs P) {
  pdl_enter();
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < P.n_pad;
       x += (int64_t)gridDim.x * blockDim.x) {
    if (x < P.n_total) {
      const int32_t m = lengths[x] - k + 1;
      if (m < 1 || m > kMaxM) continue;  // already recorded as an error
      const int32_t pos = atomicAdd(&P.mhist[m], 1);
      P.perm[pos] = (int32_t)x;
      P.rec[pos] = division_record((uint32_t)m);
      P.recw[pos] = floor_weight((uint32_t)m);
    } else {
      P.perm[x] = -1;
      P.rec[x] = division_record(1u);  // padding rows: S = 0, term = 0
      P.recw[x] = floor_weight(1u);
    }
  }
}

// Batches: one block per set sorts the set's sequences by (decreasing m, index)
// and places them (and the set's padding rows) at the set's rows.
__global__ void __launch_bounds__(kSortThreads) lensort_sets_kernel(
    const int32_t *__restrict__ lengths, int32_t k, RankPtrs P) {
  pdl_enter();
  extern __shared__ Item sm[];
  Item *buf = P.sortbuf, *scratch = P.sortbuf + P.n_total;
  for (int32_t s = blockIdx.x; s < (int32_t)P.n_sets; s += gridDim.x) {
    const RankSet e = P.sets[s];
    for (int64_t i = threadIdx.x; i < e.n; i += blockDim.x) {
      const int32_t m = lengths[e.seq_begin + i] - k + 1;
      Item it;
      it.hi = (uint64_t)(kMaxM - min(max(m, 1), kMaxM));
      it.lo = 0;
      it.idx = (int32_t)i;
      it.pad = 0;
      buf[e.seq_begin + i] = it;
    }
    __syncthreads();
    cta_sort(buf + e.seq_begin, scratch + e.seq_begin, e.n, sm);
    const int64_t np = dev_n_pad(e.n);
    for (int64_t i = threadIdx.x; i < np; i += blockDim.x) {
      const int64_t row = e.row_base + i;
      if (i < e.n) {
        const int32_t x = buf[e.seq_begin + i].idx;
        const int32_t m = lengths[e.seq_begin + x] - k + 1;
        P.perm[row] = (int32_t)(e.seq_begin + x);
        P.rec[row] = division_record((uint32_t)min(max(m, 1), kMaxM));
        P.recw[row] = floor_weight((uint32_t)min(max(m, 1), kMaxM));
      } else {
        P.perm[row] = -1;
        P.rec[row] = division_record(1u);
        P.recw[row] = floor_weight(1u);
      }
    }
    __syncthreads();
  }
}

// Plane rows, kPlaneRows stored rows per block iteration: stage the rows' counts
// (as 16-bit) in shared memory with 16-byte loads, write their K_pad plane bytes
// 16 at a time (the column map of a chunk is read once for all the rows), raise
// the depth of each row's 128-row block to the row's largest count, check that
// the row's counts add up to its number of windows m, and append its excess
// entries (counts above the depth) to the (set, word) lists.
constexpr int kPlaneRows = 2;

// counts 4q..4q+3 of a row into its shared u16 copy (one 8-byte store), clamped to
// [0, 65535] (larger counts do not occur: windows per sequence are at most 65535)
__device__ __forceinline__ void stage4(uint16_t *sc, int q, int4 v) {
  const uint32_t a = (uint32_t)min(max(v.x, 0), 0xFFFF) | (uint32_t)min(max(v.y, 0), 0xFFFF) << 16;
  const uint32_t b = (uint32_t)min(max(v.z, 0), 0xFFFF) | (uint32_t)min(max(v.w, 0), 0xFFFF) << 16;
  reinterpret_cast<uint2 *>(sc)[q] = make_uint2(a, b);
}

__global__ void __launch_bounds__(256) planes_kernel(const int32_t *__restrict__ counts,
                                                     int32_t eps, RankPtrs P) {
  pdl_enter();
  extern __shared__ uint16_t s_cnt[];  // [kPlaneRows][eps]
  __shared__ int32_t s_max[kPlaneRows], s_sum[kPlaneRows];
  __shared__ int32_t s_scan[32];
  __shared__ unsigned long long s_first;
  if (P.hdr->status != 0) return;
  const int32_t k_eff = (int32_t)P.hdr->k_eff;
  const int32_t k_pad = P.hdr->k_pad;
  const int32_t dkeep = P.hdr->depth;
  const bool residual = dkeep < P.hdr->t_max;
  const bool vec = (eps & 3) == 0 && (reinterpret_cast<uintptr_t>(counts) & 15) == 0;
  const int64_t groups = P.n_pad / kPlaneRows;
  for (int64_t g = blockIdx.x; g < groups; g += gridDim.x) {
    int32_t xs[kPlaneRows];
#pragma unroll
    for (int r = 0; r < kPlaneRows; ++r) xs[r] = P.perm[g * kPlaneRows + r];
    if (threadIdx.x < kPlaneRows) {
      s_max[threadIdx.x] = 0;
      s_sum[threadIdx.x] = 0;
    }
#pragma unroll
    for (int r = 0; r < kPlaneRows; ++r) {
      uint16_t *sc = s_cnt + r * eps;
      int32_t mx = 0, sum = 0;
      if (xs[r] >= 0) {
        const int32_t *row = counts + (int64_t)xs[r] * eps;
        if (vec) {
          const int4 *row4 = reinterpret_cast<const int4 *>(row);
          const int q4 = eps >> 2;
          int q = threadIdx.x;
          for (; q + 3 * 256 < q4; q += 4 * 256) {
            int4 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = __ldg(row4 + q + u * 256);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              stage4(sc, q + u * 256, v[u]);
              mx = max(mx, max(max(v[u].x, v[u].y), max(v[u].z, v[u].w)));
              sum += v[u].x + v[u].y + v[u].z + v[u].w;
            }
          }
          for (; q < q4; q += 256) {
            const int4 v = __ldg(row4 + q);
            stage4(sc, q, v);
            mx = max(mx, max(max(v.x, v.y), max(v.z, v.w)));
            sum += v.x + v.y + v.z + v.w;
          }
        } else {
          for (int t = threadIdx.x; t < eps; t += blockDim.x) {
            const int32_t c = __ldg(row + t);
            sc[t] = (uint16_t)min(max(c, 0), 0xFFFF);
            mx = max(mx, c);
            sum += c;
          }
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        sum += __shfl_xor_sync(0xffffffffu, sum, o);
      }
      __syncthreads();  // s_max/s_sum reset visible (first row); s_cnt complete below
      if ((threadIdx.x & 31) == 0) {
        atomicMax(&s_max[r], mx);
        atomicAdd(&s_sum[r], sum);
      }
    }
    __syncthreads();
    if (residual) {
      // excess entries of the rows, appended unordered: (stored row, word | excess << 16);
      // the per-(set, word) sizes are counted for the grouping that follows. The
      // block counts its entries first and reserves their slots with one atomic.
      int32_t mine = 0;
#pragma unroll
      for (int r = 0; r < kPlaneRows; ++r)
        if (xs[r] >= 0)
          for (int tau = threadIdx.x; tau < eps; tau += blockDim.x)
            mine += s_cnt[r * eps + tau] > dkeep;
      int32_t total;
      const int32_t incl = block_scan_incl<int32_t>(mine, s_scan, &total);
      if (threadIdx.x == 0)
        s_first = total ? atomicAdd(&P.hdr->flat_count, (unsigned long long)total) : 0ull;
      __syncthreads();
      unsigned long long slot = s_first + (unsigned long long)(incl - mine);
#pragma unroll
      for (int r = 0; r < kPlaneRows; ++r) {
        if (xs[r] < 0 || mine == 0) continue;
        const int64_t pos = g * kPlaneRows + r;
        const int64_t wbase = (int64_t)set_of_row(P, pos) * eps;
        for (int tau = threadIdx.x; tau < eps; tau += blockDim.x) {
          const int32_t c = s_cnt[r * eps + tau];
          if (c > dkeep) {
            atomicAdd(&P.cnt_gt[wbase + tau], 1);
            if (slot < (unsigned long long)P.list_cap)
              P.flat[slot] = make_int2((int32_t)pos, tau | ((c - dkeep) << 16));
            ++slot;
          }
        }
      }
    }
    // plane values: thread writes 8 consecutive columns (one 32-bit store of eight
    // 4-bit values per row); neighbouring lanes look up neighbouring words of the
    // same section
    uint32_t *dst[kPlaneRows];
#pragma unroll
    for (int r = 0; r < kPlaneRows; ++r)
      dst[r] = reinterpret_cast<uint32_t *>(P.planes + (g * kPlaneRows + r) * (P.k_cap / 2));
    for (int c = threadIdx.x; c < k_pad / 8; c += blockDim.x) {
      uint32_t w[kPlaneRows] = {};
      const int32_t c0 = c * 8;
      if (c0 + 8 <= k_eff) {
        const int4 e4a = __ldg(reinterpret_cast<const int4 *>(P.colmap + c0));
        const int4 e4b = __ldg(reinterpret_cast<const int4 *>(P.colmap + c0 + 4));
        const int32_t ev[8] = {e4a.x, e4a.y, e4a.z, e4a.w, e4b.x, e4b.y, e4b.z, e4b.w};
#pragma unroll
        for (int b = 0; b < 8; ++b) {
          const uint32_t tau = (uint32_t)ev[b] & 0xFFFFu, t = (uint32_t)ev[b] >> 16;
#pragma unroll
          for (int r = 0; r < kPlaneRows; ++r)
            if ((uint32_t)s_cnt[r * eps + tau] >= t) w[r] |= kE2M1One << (4 * b);
        }
      } else {
        for (int b = 0; b < 8; ++b) {
          if (c0 + b < k_eff) {
            const int32_t e = __ldg(P.colmap + c0 + b);
            const uint32_t tau = (uint32_t)e & 0xFFFFu, t = (uint32_t)e >> 16;
#pragma unroll
            for (int r = 0; r < kPlaneRows; ++r)
              if ((uint32_t)s_cnt[r * eps + tau] >= t) w[r] |= kE2M1One << (4 * b);
          }
        }
      }
#pragma unroll
      for (int r = 0; r < kPlaneRows; ++r) dst[r][c] = xs[r] >= 0 ? w[r] : 0u;
    }
    if (threadIdx.x < kPlaneRows && xs[threadIdx.x] >= 0) {
      const int64_t pos = g * kPlaneRows + threadIdx.x;
      atomicMax(&P.depth[pos / kRowBlock], s_max[threadIdx.x]);
      // the counts of a row must add up to its number of windows, m
      if (s_sum[threadIdx.x] != (int32_t)(P.rec[pos].w & 0xFFFFu))
        record_error(P.hdr, SAD_ERR_BAD_INPUT, xs[threadIdx.x]);
    }
    __syncthreads();
  }
}

// Plane rows for depths D <= kTabDepth, streamed: one warp per stored row reads the
// row's counts once (16 bytes per lane, four loads in flight). A plane value is
// the 4-bit e2m1 [c >= t] (1.0 or 0), two columns to a byte. When every word
// occurs somewhere, section 1 is the identity map and a lane writes its four words
// as one 2-byte store; the columns past section 1 are zero-filled with 16-byte
// stores first, and only the words counted twice or more then set their values in
// sections 2..min(c, D) (atomic OR: neighbouring columns share bytes). Otherwise
// the whole row is zero-filled and every 1 is set that way. Counts above D go to a
// per-warp buffer and are appended to the flat excess list with one atomic per
// row; a row with more than kExCap of them is scanned again for the append.
constexpr int kExCap = 64;
constexpr int kStreamUnroll = 4;

__device__ __forceinline__ uint32_t plane_val(int32_t c, int32_t t) { return c >= t ? kE2M1One : 0u; }

// Set plane column col of a row to 1.0 (the row bytes are zero there beforehand).
__device__ __forceinline__ void plane_set(uint8_t *prow, int32_t col) {
  atomicOr(reinterpret_cast<unsigned int *>(prow) + (col >> 3), kE2M1One << (4 * (col & 7)));
}

__global__ void __launch_bounds__(256) planes_stream_kernel(const int32_t *__restrict__ counts,
                                                            int32_t eps, RankPtrs P) {
  pdl_enter();
  __shared__ int2 s_ex[8][kExCap];
  __shared__ int32_t s_exn[8];
  if (P.hdr->status != 0) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int32_t k_pad = P.hdr->k_pad;
  const int32_t dkeep = P.hdr->depth;
  const bool residual = dkeep < P.hdr->t_max;
  const int q4 = eps >> 2;
  const int32_t s1 = P.secend[1];  // end of section 1
  const bool ident = s1 == eps;    // section 1 = every word, in order
  const int32_t kb = k_pad / 2;    // row bytes in use
  // bytes zero-filled before the ones are set: past section 1, or all of the row
  const int32_t z0 = ident ? s1 / 2 : 0;
  const int32_t z16 = min((z0 + 15) & ~15, kb);
  if (lane == 0) s_exn[warp] = 0;
  __syncwarp();
  for (int64_t pos = (int64_t)blockIdx.x * 8 + warp; pos < P.n_pad;
       pos += (int64_t)gridDim.x * 8) {
    const int32_t x = P.perm[pos];
    uint8_t *prow = P.planes + pos * (P.k_cap / 2);
    if (x < 0) {  // padding row: all zero
      for (int c = 16 * lane; c < kb; c += 512)
        *reinterpret_cast<uint4 *>(prow + c) = make_uint4(0, 0, 0, 0);
      continue;
    }
    for (int c = z0 + lane; c < z16; c += 32) prow[c] = 0;
    for (int c = z16 + 16 * lane; c < kb; c += 512)
      *reinterpret_cast<uint4 *>(prow + c) = make_uint4(0, 0, 0, 0);
    __syncwarp();
    const int4 *row4 = reinterpret_cast<const int4 *>(counts + (int64_t)x * eps);
    const int64_t wbase = (int64_t)set_of_row(P, pos) * eps;
    int32_t mx = 0, sum = 0;
    for (int base = 0; base < q4; base += 32 * kStreamUnroll) {
      int4 v[kStreamUnroll];
#pragma unroll
      for (int u = 0; u < kStreamUnroll; ++u) {
        const int q = base + 32 * u + lane;
        v[u] = q < q4 ? __ldg(row4 + q) : make_int4(0, 0, 0, 0);
      }
#pragma unroll
      for (int u = 0; u < kStreamUnroll; ++u) {
        const int q = base + 32 * u + lane;
        if (q >= q4) continue;
        const int32_t c[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
        mx = max(mx, max(max(c[0], c[1]), max(c[2], c[3])));
        sum += c[0] + c[1] + c[2] + c[3];
        if (ident) {
          // columns 4q..4q+3 = bytes 2q, 2q+1
          *reinterpret_cast<uint16_t *>(prow + 2 * q) =
              (uint16_t)(plane_val(c[0], 1) | plane_val(c[1], 1) << 4 | plane_val(c[2], 1) << 8 |
                         plane_val(c[3], 1) << 12);
        } else {
          const int4 col = __ldg(reinterpret_cast<const int4 *>(P.coltab) + q);
          const int32_t cc[4] = {col.x, col.y, col.z, col.w};
#pragma unroll
          for (int b = 0; b < 4; ++b)
            if (cc[b] >= 0 && c[b] >= 1) plane_set(prow, cc[b]);
        }
        if (dkeep >= 2) {
          // a word counted c >= 2 times is in sections 2..T >= c: its values there are 1
#pragma unroll
          for (int b = 0; b < 4; ++b)
            for (int t = 2; t <= min(c[b], dkeep); ++t)
              plane_set(prow, P.coltab[(int64_t)(t - 1) * eps + 4 * q + b]);
        }
        if (residual) {
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            if (c[b] > dkeep) {
              const int slot = atomicAdd(&s_exn[warp], 1);
              if (slot < kExCap)
                s_ex[warp][slot] = make_int2((int32_t)pos, (4 * q + b) | ((c[b] - dkeep) << 16));
            }
          }
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      sum += __shfl_xor_sync(0xffffffffu, sum, o);
    }
    if (lane == 0) {
      atomicMax(&P.depth[pos / kRowBlock], mx);
      // the counts of a row must add up to its number of windows, m
      if (sum != (int32_t)(P.rec[pos].w & 0xFFFFu)) record_error(P.hdr, SAD_ERR_BAD_INPUT, x);
    }
    if (residual) {
      __syncwarp();
      const int32_t n_ex = s_exn[warp];
      if (n_ex > 0) {
        unsigned long long first = 0;
        if (lane == 0) first = atomicAdd(&P.hdr->flat_count, (unsigned long long)n_ex);
        first = __shfl_sync(0xffffffffu, first, 0);
        if (n_ex <= kExCap) {
          for (int i = lane; i < n_ex; i += 32) {
            const int2 e = s_ex[warp][i];
            atomicAdd(&P.cnt_gt[wbase + (e.y & 0xFFFF)], 1);
            if (first + i < (unsigned long long)P.list_cap) P.flat[first + i] = e;
          }
        } else {
          // the buffer overflowed: scan the row again and append every entry
          __syncwarp();
          if (lane == 0) s_exn[warp] = 0;
          __syncwarp();
          for (int q = lane; q < q4; q += 32) {
            const int4 v = __ldg(row4 + q);
            const int32_t c[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int b = 0; b < 4; ++b) {
              if (c[b] > dkeep) {
                const unsigned long long slot = first + (unsigned)atomicAdd(&s_exn[warp], 1);
                atomicAdd(&P.cnt_gt[wbase + 4 * q + b], 1);
                if (slot < (unsigned long long)P.list_cap)
                  P.flat[slot] = make_int2((int32_t)pos, (4 * q + b) | ((c[b] - dkeep) << 16));
              }
            }
          }
        }
      }
      __syncwarp();
      if (lane == 0) s_exn[warp] = 0;
      __syncwarp();
    }
  }
}

// Upper-triangle tile list of every set (blocks per set and column group). Tile (I, J) of a
// set covers its stored rows [128 I, 128 I + 128) and columns [128 J, 128 J + 128)
// (set-local, kColBlock = 128); it is needed when some pair i <= j lies in it
// (I <= J) and both ranges hold real rows. Tiles are grouped by kGroupCols column blocks,
// rows ascending inside a group, so that the tiles running at the same time share
// their operand panels in L2. Each entry is (I | J << 16, K chunks) with global
// block indices, the K extent being the end of section min(depth(I), depth(J), D).
constexpr int kGroupCols = 8;

// Tiles of column group g of a set: rows I with J in [8g, 8g + 8) and J >= I / kColRatio.
__device__ __forceinline__ int32_t group_row_tiles(int32_t g, int32_t I, int32_t C) {
  const int32_t j0 = max(g * kGroupCols, I / kColRatio);
  const int32_t j1 = min((g + 1) * kGroupCols, C);
  return max(0, j1 - j0);
}

// (blockIdx.y: sets in a grid stride; blockIdx.x: column groups in a grid stride)
__global__ void __launch_bounds__(256) tiles_kernel(RankPtrs P) {
  pdl_enter();
  __shared__ int32_t s_warp[32];
  __shared__ int32_t s_carry;
  const int tid = threadIdx.x;
  const int32_t nblk = (int32_t)(P.n_pad / kRowBlock);
  const int32_t dkeep = P.hdr->depth;
  for (int32_t si = blockIdx.y; si < (int32_t)P.n_sets; si += gridDim.y) {
    const RankSet e = P.sets[si];
    const int32_t n = e.n;
    const int32_t R = (n + kRowBlock - 1) / kRowBlock;
    const int32_t C = (n + kColBlock - 1) / kColBlock;
    const int64_t cfull = dev_n_pad(n) / kColBlock;
    const int32_t I0 = (int32_t)(e.row_base / kRowBlock), J0 = (int32_t)(e.row_base / kColBlock);
    const int32_t groups = (C + kGroupCols - 1) / kGroupCols;
    for (int32_t g = blockIdx.x; g < groups; g += gridDim.x) {
      // tiles of the groups before g come first
      int32_t before = 0;
      for (int64_t gi = tid; gi < (int64_t)g * R; gi += blockDim.x)
        before += group_row_tiles((int32_t)(gi / R), (int32_t)(gi % R), C);
      int32_t tot;
      block_scan_incl<int32_t>(before, s_warp, &tot);
      if (tid == 0) s_carry = tot;
      __syncthreads();
      unsigned long long chunks = 0;
      int32_t group_tiles = 0;
      for (int32_t base = 0; base < R; base += blockDim.x) {
        const int32_t I = base + tid;
        const int32_t cnt = I < R ? group_row_tiles(g, I, C) : 0;
        const int32_t incl = block_scan_incl<int32_t>(cnt, s_warp, &tot);
        int64_t out = e.tile_base + s_carry + incl - cnt;
        if (cnt > 0) {
          const int32_t dI = P.depth[I0 + I];
          const int32_t j0 = max(g * kGroupCols, I / kColRatio);
          for (int32_t J = j0; J < j0 + cnt; ++J) {
            // the column block spans row blocks kColRatio (J0 + J) .. + kColRatio - 1
            int32_t dJ = 0;
            for (int32_t b = kColRatio * (J0 + J); b < kColRatio * (J0 + J + 1) && b < nblk; ++b)
              dJ = max(dJ, P.depth[b]);
            const int32_t d = min(min(dI, dJ), dkeep);
            // the promoted planes of depth + 1 sit right after K_eff of the sections
            const int32_t kend =
                (P.hdr->n_promoted > 0 && min(dI, dJ) > dkeep) ? P.hdr->k_ext : P.secend[max(d, 0)];
            const int32_t nk = max(1, (kend + kKCols - 1) / kKCols);
            P.tile_of[e.tileof_base + (int64_t)I * cfull + J] = (int32_t)out;
            P.block_of[out] = 0;
            P.tiles[out++] = make_int2((I0 + I) | ((J0 + J) << 16), nk);
            chunks += (unsigned long long)nk;
          }
        }
        __syncthreads();
        if (tid == 0) s_carry += tot;
        group_tiles += tot;
        __syncthreads();
      }
      if (chunks) atomicAdd(&P.hdr->k_chunks, chunks);
      if (tid == 0) atomicAdd(&P.hdr->n_tiles, group_tiles);
      __syncthreads();
    }
  }
}

// ------------------------------------------------------------- residual ----
// The pairs (u, v), u <= v, of each (set, word) excess list (stored row,
// count - D) are cut into work items: pairs of kPairChunk-entry chunks (cu, cv),
// cu <= cv, numbered cv-major within the list after the items of the lists
// before it (item_off). Blocks take items in a grid stride, so that the pairs of
// a long list are spread over many blocks. A block stages the two chunks in
// shared memory sorted by row (neighbouring pairs then land in neighbouring
// columns of the same tile row) and its threads walk the chunk pair. fn(tile,
// row in tile, column in tile, value) is called once per pair with value = min
// of the two excesses; u == v is the sequence's own pair.

// Ascending bitonic sort by .x of s[0, n), n <= kPairChunk, padded with INT_MAX.
__device__ __forceinline__ void block_sort_by_row(int2 *s, int n) {
  int p2 = 1;
  while (p2 < n) p2 <<= 1;
  for (int i = n + threadIdx.x; i < p2; i += blockDim.x) s[i] = make_int2(0x7FFFFFFF, 0);
  __syncthreads();
  for (int size = 2; size <= p2; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < (p2 >> 1); i += blockDim.x) {
        const int a = ((i & ~(stride - 1)) << 1) | (i & (stride - 1)), b = a + stride;
        const bool asc = (a & size) == 0;
        const int2 x = s[a], y = s[b];
        if (asc ? (y.x < x.x) : (x.x < y.x)) {
          s[a] = y;
          s[b] = x;
        }
      }
      __syncthreads();
    }
  }
}

template <typename Fn>
__device__ __forceinline__ void for_each_residual_pair(const RankPtrs &P, int32_t eps, Fn fn) {
  __shared__ int2 s_u[kPairChunk], s_v[kPairChunk];
  __shared__ int64_t s_w;
  const int64_t we = P.n_sets * (int64_t)eps;
  const int64_t total = P.hdr->items_total;
  for (int64_t it = blockIdx.x; it < total; it += gridDim.x) {
    __syncthreads();  // the previous item's chunks are no longer read
    if (threadIdx.x == 0) {
      // the list holding item it: item_off[w] <= it < item_off[w + 1]
      int64_t lo = 0, hi = we;
      while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (P.item_off[mid] <= it) lo = mid;
        else hi = mid;
      }
      s_w = lo;
    }
    __syncthreads();
    const int64_t w = s_w;
    const int64_t base = P.list_off[w];
    const int64_t len = P.list_off[w + 1] - base;
    const int64_t j = it - P.item_off[w];
    int64_t cv = (int64_t)((sqrt(8.0 * (double)j + 1.0) - 1.0) * 0.5);
    while (cv * (cv + 1) / 2 > j) --cv;
    while ((cv + 1) * (cv + 2) / 2 <= j) ++cv;
    const int64_t cu = j - cv * (cv + 1) / 2;
    const RankSet e = P.sets[w / eps];
    const int64_t cfull = dev_n_pad(e.n) / kColBlock;
    const int nv = (int)min((int64_t)kPairChunk, len - cv * kPairChunk);
    const int nu = (int)min((int64_t)kPairChunk, len - cu * kPairChunk);
    const bool same = cu == cv;
    for (int i = threadIdx.x; i < nv; i += blockDim.x) s_v[i] = P.lists[base + cv * kPairChunk + i];
    if (!same)
      for (int i = threadIdx.x; i < nu; i += blockDim.x) s_u[i] = P.lists[base + cu * kPairChunk + i];
    block_sort_by_row(s_v, nv);
    if (!same) block_sort_by_row(s_u, nu);
    const int npairs = nu * nv;  // <= kPairChunk^2
    for (int q = threadIdx.x; q < npairs; q += blockDim.x) {
      const int iu = q / nv, iv = q - iu * nv;
      if (same && iu > iv) continue;
      const int2 eu = same ? s_v[iu] : s_u[iu];
      const int2 ev = s_v[iv];
      const int32_t a = min(eu.x, ev.x), b = max(eu.x, ev.x);
      const int64_t al = a - e.row_base, bl = b - e.row_base;
      const int32_t t = P.tile_of[e.tileof_base + (al / kRowBlock) * cfull + bl / kColBlock];
      fn(t, (int32_t)(al % kRowBlock), (int32_t)(bl % kColBlock), (uint32_t)min(eu.y, ev.y));
    }
  }
}

__device__ __forceinline__ bool residual_on(const RankPtrs &P) {
  return P.hdr->status == 0 && P.hdr->depth < P.hdr->t_max;
}

// Only needed when fewer residual blocks than tiles are reserved: mark the
// tiles that some pair touches.
__global__ void __launch_bounds__(256) residual_mark_kernel(RankPtrs P, int32_t eps) {
  pdl_enter();
  if (!residual_on(P)) return;
  for_each_residual_pair(P, eps, [&](int32_t t, int32_t, int32_t, uint32_t) {
    if (P.block_of[t] != 1) P.block_of[t] = 1;
  });
}

// block_of[t] := index of tile t's residual block, -1 if none. With a block for
// every tile (identity) nothing needs marking.
__global__ void __launch_bounds__(1024) residual_scan_kernel(RankPtrs P, int identity) {
  pdl_enter();
  __shared__ int32_t s_warp[32];
  __shared__ int32_t s_carry;
  const int32_t nt = P.hdr->n_tiles;
  const bool on = residual_on(P);
  if (identity) {
    // a block per tile: no scan
    for (int32_t t = threadIdx.x; t < nt; t += blockDim.x) P.block_of[t] = on ? t : -1;
    if (threadIdx.x == 0) {
      P.hdr->n_blocks = on ? nt : 0;
      if (on && nt > P.block_cap) record_error(P.hdr, SAD_ERR_WORKSPACE, nt);
    }
    return;
  }
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (int32_t base = 0; base < nt; base += blockDim.x) {
    const int32_t t = base + threadIdx.x;
    const int32_t f = (on && t < nt && (identity || P.block_of[t] == 1)) ? 1 : 0;
    int32_t tot;
    const int32_t incl = block_scan_incl<int32_t>(f, s_warp, &tot);
    if (t < nt) P.block_of[t] = f ? s_carry + incl - 1 : -1;
    __syncthreads();
    if (threadIdx.x == 0) s_carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    P.hdr->n_blocks = s_carry;
    if (s_carry > P.block_cap) record_error(P.hdr, SAD_ERR_WORKSPACE, s_carry);
  }
}

__global__ void residual_zero_kernel(RankPtrs P) {
  pdl_enter();
  if (P.hdr->status != 0) return;
  const int64_t words4 = (int64_t)P.hdr->n_blocks * (int64_t)(kResidualBlockBytes / 16);
  uint4 *p = reinterpret_cast<uint4 *>(P.rblocks);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words4;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = make_uint4(0, 0, 0, 0);
}

__global__ void __launch_bounds__(256) residual_add_kernel(RankPtrs P, int32_t eps) {
  pdl_enter();
  if (!residual_on(P)) return;
  for_each_residual_pair(P, eps, [&](int32_t t, int32_t row, int32_t col, uint32_t val) {
    const int64_t blk = P.block_of[t];
    // two u16 per word; a pair's residual never exceeds 65535, so no carry crosses
    atomicAdd(&P.rblocks[blk * (kResidualBlockBytes / 4) + row * (kColBlock / 2) + (col >> 1)],
              val << (16 * (col & 1)));
  });
}

// key = acc0 + acc1 2^32 (128-bit); rank = (hi + lo 2^-64) / N of the set.
__global__ void finalize_kernel(RankPtrs P, uint64_t *__restrict__ key_hi,
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
      const double n = (double)P.sets[set_of_seq(P, x)].n;
      const double whole = __ull2double_rn(hi);
      const double frac = __dmul_rn(__ull2double_rn(lo), 0x1p-64);
      rank[x] = __ddiv_rn(__dadd_rn(whole, frac), n);
    }
  }
}

inline unsigned grid_for(int64_t work, int threads, int cap_per_sm = 8) {
  int64_t g = (work + threads - 1) / threads;
  const int64_t cap = (int64_t)num_sms() * cap_per_sm;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (unsigned)g;
}

bool g_attr_sort = false;

}  // namespace

int rank_prep_launch(const RankPtrs &P, const int32_t *counts, const int32_t *lengths,
                     const int32_t *d_n, const int32_t *word_max, int32_t k, int32_t eps,
                     int plan_only, cudaStream_t st) {
  const int64_t n = P.n_total;
  const unsigned gsets = (unsigned)(P.n_sets < 4096 ? P.n_sets : 4096);
  const int64_t we = P.n_sets * (int64_t)eps;
  const int64_t nblk = (we + kScanChunk - 1) / kScanChunk;
  auto list_scan = [&]() -> int {
    pdl_launch(list_scan_reduce_kernel, (unsigned)nblk, 256, 0, st, P, we);
    SAD_LAUNCH_CHECK();
    pdl_launch(list_scan_top_kernel, 1, 1024, 0, st, P, nblk);
    SAD_LAUNCH_CHECK();
    pdl_launch(list_scan_down_kernel, (unsigned)nblk, 256, 0, st, P, we, plan_only);
    SAD_LAUNCH_CHECK();
    return SAD_OK;
  };
  pdl_launch(rank_setup_kernel, 1, 1024, 0, st, d_n, (int32_t)n, P);
  SAD_LAUNCH_CHECK();
  if (P.n_sets > 1) {
    pdl_launch(rank_setmaps_kernel, gsets, 256, 0, st, P);
    SAD_LAUNCH_CHECK();
  }
  pdl_launch(rank_init_kernel, grid_for(we + kMaxM, 256), 256, 0, st, P, eps, !plan_only);
  SAD_LAUNCH_CHECK();
  if (!plan_only) {
    pdl_launch(lengths_kernel, grid_for(n, 256), 256, 0, st, lengths, k, P);
    SAD_LAUNCH_CHECK();
  }
  if (word_max && !plan_only) {
    pdl_launch(copy_word_max_kernel, grid_for(eps, 256), 256, 0, st, word_max, eps, P);
    SAD_LAUNCH_CHECK();
  } else {
    dim3 g((eps + 255) / 256, 1);
    int64_t slices = ((int64_t)num_sms() * 8 + g.x - 1) / g.x;
    if (slices > (n + 63) / 64) slices = (n + 63) / 64;
    if (slices < 1) slices = 1;
    g.y = (unsigned)slices;
    // the plan counts the excess entries here; a run counts them in the plane kernel
    pdl_launch(colmax_kernel, g, 256, 0, st, counts, eps, P, plan_only);
    SAD_LAUNCH_CHECK();
  }
  pdl_launch(colmap_kernel, 1, 1024, 0, st, P, eps, plan_only);
  SAD_LAUNCH_CHECK();
  if (plan_only) return list_scan();
  if (P.n_sets == 1) {
    pdl_launch(lensort_scan_kernel, 1, 1024, 0, st, P);
    SAD_LAUNCH_CHECK();
    pdl_launch(lensort_place_kernel, grid_for(P.n_pad, 256), 256, 0, st, lengths, k, P);
    SAD_LAUNCH_CHECK();
  } else {
    if (!g_attr_sort) {
      if (cudaFuncSetAttribute(lensort_sets_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)kSortSmem) != cudaSuccess)
        return SAD_ERR_CUDA;
      g_attr_sort = true;
    }
    pdl_launch(lensort_sets_kernel, gsets, kSortThreads, kSortSmem, st, lengths, k, P);
    SAD_LAUNCH_CHECK();
  }
  if (P.depth_cap >= 1 && P.depth_cap <= kTabDepth && (eps & 3) == 0 &&
      (reinterpret_cast<uintptr_t>(counts) & 15) == 0 && (P.k_cap & 31) == 0) {
    const int64_t warps = P.n_pad;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, planes_stream_kernel, 256, 0) !=
        cudaSuccess)
      return SAD_ERR_CUDA;
    const int64_t cap = (int64_t)num_sms() * (per_sm > 0 ? per_sm : 1);
    const int64_t want = (warps + 7) / 8;
    pdl_launch(planes_stream_kernel, (unsigned)(want < cap ? want : cap), 256, 0, st, counts, eps,
               P);
    SAD_LAUNCH_CHECK();
  } else {
    const size_t smem = sizeof(uint16_t) * (size_t)eps * kPlaneRows;
    if (cudaFuncSetAttribute(planes_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
      return SAD_ERR_CUDA;
    // every block resident at once: the grid stride then splits the rows evenly
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, planes_kernel, 256, smem) !=
        cudaSuccess)
      return SAD_ERR_CUDA;
    const int64_t groups = P.n_pad / kPlaneRows;
    const int64_t cap = (int64_t)num_sms() * (per_sm > 0 ? per_sm : 1);
    pdl_launch(planes_kernel, (unsigned)(groups < cap ? groups : cap), 256, smem, st, counts, eps,
               P);
    SAD_LAUNCH_CHECK();
  }
  if (P.depth_cap >= 1 && P.list_cap > 0) {
    pdl_launch(promote_weight_kernel, grid_for(eps, 256), 256, 0, st, P, eps);
    SAD_LAUNCH_CHECK();
    const int staged = eps <= 16384 ? 1 : 0;
    const size_t smem = staged ? sizeof(int64_t) * (size_t)eps : 0;
    if (staged && cudaFuncSetAttribute(promote_select_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem) != cudaSuccess)
      return SAD_ERR_CUDA;
    pdl_launch(promote_select_kernel, 1, 1024, smem, st, P, eps, staged);
    SAD_LAUNCH_CHECK();
    pdl_launch(promote_apply_kernel, grid_for(P.list_cap, 256), 256, 0, st, P, eps);
    SAD_LAUNCH_CHECK();
  }
  int rc = list_scan();
  if (rc) return rc;
  if (P.depth_cap >= 1 && P.list_cap > 0) {
    pdl_launch(group_lists_kernel, grid_for(P.list_cap, 256), 256, 0, st, P, eps);
    SAD_LAUNCH_CHECK();
  }
  {
    // one set: a CTA per column group; batches: a few per set
    const int64_t groups1 = ((n + kColBlock - 1) / kColBlock + kGroupCols - 1) / kGroupCols;
    dim3 g((unsigned)(P.n_sets == 1 ? (groups1 > 0 ? groups1 : 1) : 4), gsets);
    pdl_launch(tiles_kernel, g, 256, 0, st, P);
  }
  SAD_LAUNCH_CHECK();
  if (P.depth_cap >= 1 && P.block_cap > 0) {
    // the residual only exists when the planes are cut below the largest count
    const int identity = P.block_cap >= P.tiles_total ? 1 : 0;
    const unsigned gw = (unsigned)(we < num_sms() * 8 ? we : num_sms() * 8);
    if (!identity) {
      pdl_launch(residual_mark_kernel, gw, 256, 0, st, P, eps);
      SAD_LAUNCH_CHECK();
    }
    pdl_launch(residual_scan_kernel, 1, 1024, 0, st, P, identity);
    SAD_LAUNCH_CHECK();
    pdl_launch(residual_zero_kernel, (unsigned)num_sms() * 8, 256, 0, st, P);
    SAD_LAUNCH_CHECK();
    pdl_launch(residual_add_kernel, gw, 256, 0, st, P, eps);
    SAD_LAUNCH_CHECK();
  }
  return SAD_OK;
}

int rank_finalize_launch(const RankPtrs &P, uint64_t *key_hi, uint64_t *key_lo, double *rank,
                         cudaStream_t st) {
  pdl_launch(finalize_kernel, grid_for(P.n_total, 256), 256, 0, st, P, key_hi, key_lo, rank);
  SAD_LAUNCH_CHECK();
  return SAD_OK;
}

int64_t host_tile_count(int32_t n) { return tiles_of_set(n); }

}  // namespace sad
