// Preparation of the threshold-plane GEMM behind kmer_rank.
//
// Eq. 1's numerator S(X,Y) = sum_tau min(c^X_tau, c^Y_tau) is rewritten with the
// exact identity min(a, b) = sum_{t>=1} [a >= t][b >= t]: with one 0/1 column
// per (word tau, threshold t), t = 1..T_tau, T_tau = max_x c^x_tau, the matrix
// P[x][(tau,t)] = [c^x_tau >= t] satisfies S = P P^T. The columns are laid out
// threshold-major: section t holds the words with T_tau >= t (in word order), so
// the first sections are the dense ones and a tile whose rows never count any
// word more than d times only needs the columns up to the end of section d.
//
// Plane depth and remainder (plans of depth D >= 1). Only the sections 1..D'
// (D' = min(D, t_max, 8)) are kept as planes. Each column block J of 128 stored
// rows gets its own plane depth d_J <= D': the tiles of column J run the GEMM over
// the plane columns [0, K_end(d_J)), K_end(d) = the end of section d rounded up
// to the 256-column K chunk, and every threshold column (tau, t) that a row v of
// block J counts (c_v(tau) >= t, t >= 2) but that lies at or past K_end(d_J) -- or
// above the planes -- is a remainder entry of row v. For a pair (u, v) of such a
// tile the planes give the identity's sum over the covered columns, and
//   S_uv = (plane columns < K_end) + sum over v's remainder entries (tau, t) of
//          [c_u(tau) >= t],
// which the GEMM epilogue evaluates from a bitmap of the columns (bit u of
// column (tau, t) = [c_u(tau) >= t]) before the floor, so every key is exact for
// every choice of depths. (When a tile's extent is cut lower by its row blocks'
// largest counts, the columns between are zero for the block that cuts it.)
// d_J is the smallest depth whose remainder entries fit the plan's budget per
// block. Thresholds above T_b = min(D' + 4, 16) are not in the bitmap: a count
// c > T_b of row v adds a heavy entry (tau, c), worth max(0, min(c_u, c) - T_b)
// for row u, which the epilogue reads from the counts.
//
// Sets. A call ranks one or more independent sets (a batch). Each set's rows are
// stored contiguously (aligned to the GEMM tile) and its tiles only pair rows of that set, so
// the GEMM is block-diagonal; the column layout is shared (T over all sets).
// Within a set, rows are stored in order of decreasing length (the order of
// equal lengths is free: it changes no result), so that for every stored pair
// i <= j the Eq. 1 denominator is min(L_i, L_j) - k + 1 = m_j, the column's own.
//
// Kernels, in launch order:
//   rank_setup     the set table (row and tile bases per set)
//   rank_setmaps   set index of every sequence and stored row (batches only)
//   rank_init      zero the scratch regions of the workspace
//   lengths        m = L - k + 1, validation, histogram of m (one set)
//   colmax         T_tau = max_x c^x_tau, count validation (and, for a plan, the
//                  sizes of the remainder lists)
//   colmap         t_max, section ends, K_eff, the column maps, the covering depth
//                  of every plane column
//   lensort_*      stored row of every sequence, per-row division records
//   planes         P rows as packed e2m1 (2 = 1.0, 0 = 0.0), block largest counts;
//                  depth >= 1: per-row remainder profile, the (row, word,
//                  count >= 2) entries
//   rem_depth      per column block: plane depth d_J, per-row entry offsets; the
//                  smallest depth of a block with remainder entries
//   rem_scan       block offsets of the remainder lists; the lowest column a
//                  remainder entry can name
//   bitmap_zero    clear the remainder bitmap from that column on
//   rem_scatter    the remainder lists, grouped by row, and the bitmap bits
//   tiles          per set, the upper-triangle tile list with per-tile K extent
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
  P.dstar = reinterpret_cast<int8_t *>(b + L.dstar);
  P.thist = reinterpret_cast<int32_t *>(b + L.thist);
  P.coltab = reinterpret_cast<int32_t *>(b + L.coltab);
  P.mhist = reinterpret_cast<int32_t *>(b + L.mhist);
  P.perm = reinterpret_cast<int32_t *>(b + L.perm);
  P.rec = reinterpret_cast<uint4 *>(b + L.rec);
  P.recw = reinterpret_cast<uint2 *>(b + L.recw);
  P.depth = reinterpret_cast<int32_t *>(b + L.depth);
  P.bdepth = reinterpret_cast<int32_t *>(b + L.bdepth);
  P.tiles = reinterpret_cast<int2 *>(b + L.tiles);
  P.acc = reinterpret_cast<unsigned long long *>(b + L.acc);
  P.planes = b + L.planes;
  P.prof = reinterpret_cast<uint32_t *>(b + L.prof);
  P.rowrem = reinterpret_cast<int32_t *>(b + L.rowrem);
  P.blkrem = reinterpret_cast<int64_t *>(b + L.blkrem);
  P.cursor = reinterpret_cast<int32_t *>(b + L.cursor);
  P.flat = reinterpret_cast<int2 *>(b + L.flat);
  P.rem = reinterpret_cast<uint32_t *>(b + L.rem);
  P.heavy = reinterpret_cast<int2 *>(b + L.heavy);
  P.bitmap = reinterpret_cast<uint32_t *>(b + L.bitmap);
  P.sortbuf = reinterpret_cast<Item *>(b + L.sortbuf);
  P.scanblk = reinterpret_cast<int64_t *>(b + L.scanblk);
  P.counts = nullptr;
  P.n_pad = L.shape.rows_total;
  P.n_total = L.shape.n_total;
  P.n_sets = L.shape.n_sets;
  P.tiles_total = L.shape.tiles_total;
  P.k_cap = L.caps.k_cap;
  P.list_cap = L.caps.list_cap;
  P.rem_cap = L.caps.rem_cap;
  P.heavy_cap = L.caps.heavy_cap;
  P.bm_cols = L.caps.bm_cols;
  P.depth_cap = L.caps.depth;
  P.budget = L.caps.budget > 0 ? L.caps.budget : kRemBudgetDefault;
  P.tile = L.caps.tile == 2 * kRowBlock ? 2 * kRowBlock : kRowBlock;
  P.eps = 0;
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

// Stored rows of a set of n sequences: padded to the GEMM tile rows B.
__device__ __forceinline__ int64_t dev_n_pad(int64_t n, int64_t B) {
  return ((n > 0 ? n : 1) + B - 1) / B * B;
}

// Upper-triangle tiles of a set of n rows in square tiles of B rows.
__device__ __forceinline__ int64_t dev_tiles_of_set(int64_t n, int64_t B) {
  const int64_t R = (n + B - 1) / B;
  return R * (R + 1) / 2;
}

__device__ __forceinline__ int32_t set_of_seq(const RankPtrs &P, int64_t x) {
  return P.n_sets > 1 ? P.seq_set[x] : 0;
}


// Plane depth kept by a plan (0 = every section).
__device__ __forceinline__ int32_t kept_depth(const RankPtrs &P, int32_t tmax) {
  return P.depth_cap >= 1 ? min(min(P.depth_cap, kMaxPlaneDepth), tmax) : tmax;
}

// Largest threshold of the remainder bitmap (counts above it are heavy entries).
__device__ __forceinline__ int32_t bit_depth(const RankPtrs &P) {
  return t_bits_of(min(P.depth_cap, kMaxPlaneDepth));
}

__device__ __forceinline__ bool remainder_mode(const RankPtrs &P) { return P.depth_cap >= 1; }

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
    const int64_t np = s < S ? dev_n_pad(n, P.tile) : 0;
    const int64_t v[4] = {n, np, s < S ? dev_tiles_of_set(n, P.tile) : 0,
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
    const int64_t np = dev_n_pad(e.n, P.tile);
    for (int64_t i = threadIdx.x; i < np; i += blockDim.x) P.row_set[e.row_base + i] = s;
  }
}

__global__ void rank_init_kernel(RankPtrs P, int32_t eps, int with_keys) {
  pdl_enter();
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nt = (int64_t)gridDim.x * blockDim.x;
  zero_range(P.T, eps, tid, nt);
  zero_range(P.thist, kMaxM + 2, tid, nt);
  zero_range(P.mhist, kMaxM + 2, tid, nt);
  zero_range(P.secend, kMaxM + 2, tid, nt);
  if (with_keys) {
    zero_range(P.depth, P.n_pad / kRowBlock, tid, nt);
    zero_range(P.acc, 3 * P.n_total, tid, nt);
    if (remainder_mode(P)) zero_range(P.cursor, 2 * P.n_pad, tid, nt);
  }
  if (tid == 0) {
    P.hdr->k_eff = 0;
    P.hdr->k_pad = 0;
    P.hdr->t_max = 0;
    P.hdr->n_tiles = 0;
    P.hdr->k_chunks = 0;
    P.hdr->depth = 0;
    P.hdr->list_total = 0;
    P.hdr->rem_bound = 0;
    P.hdr->heavy_total = 0;
    P.hdr->bm_cols = 0;
    P.hdr->m_max = 0;
    P.hdr->flat_count = 0;
    P.hdr->rem_entries = 0;
    P.hdr->heavy_entries = 0;
    P.hdr->t_bits = 0;
    P.hdr->rem_blocks = 0;
    P.hdr->dmin = 0x7FFFFFFF;
    P.hdr->bm_lo = 0;
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

// T_tau = max over rows of counts[x][tau]. For a plan of depth >= 1 also the sizes of
// the remainder: entries (x, tau) with a count c >= 2, the sum of min(c, T_b) - 1
// over them (the remainder entries there can be) and the entries with c > T_b.
// Block (256 words) x (row slice).
__global__ void colmax_kernel(const int32_t *__restrict__ counts, int32_t eps, RankPtrs P,
                              int count_lists) {
  pdl_enter();
  const int32_t tau = blockIdx.x * blockDim.x + threadIdx.x;
  if (tau >= eps) return;
  const bool lists = count_lists && remainder_mode(P);
  const int32_t tb = bit_depth(P);
  const int64_t n = P.n_total;
  const int64_t per = (n + gridDim.y - 1) / gridDim.y;
  const int64_t r0 = (int64_t)blockIdx.y * per;
  const int64_t r1 = r0 + per < n ? r0 + per : n;
  int32_t mx = 0, mn = 0;
  long long nl = 0, nr = 0, nh = 0;
  for (int64_t r = r0; r < r1; ++r) {
    const int32_t a = __ldg(counts + r * eps + tau);
    mx = max(mx, a);
    mn = min(mn, a);
    if (lists && a >= 2) {
      nl += 1;
      nr += min(a, tb) - 1;
      nh += a > tb ? 1 : 0;
    }
  }
  if (mn < 0) record_error(P.hdr, SAD_ERR_BAD_INPUT, tau);
  if (mx > kMaxM) record_error(P.hdr, SAD_ERR_UNSUPPORTED, tau);
  if (mx > 0) atomicMax(&P.T[tau], mx);
  if (nl) {
    atomicAdd(reinterpret_cast<unsigned long long *>(&P.hdr->list_total),
              (unsigned long long)nl);
    atomicAdd(reinterpret_cast<unsigned long long *>(&P.hdr->rem_bound),
              (unsigned long long)nr);
    if (nh)
      atomicAdd(reinterpret_cast<unsigned long long *>(&P.hdr->heavy_total),
                (unsigned long long)nh);
  }
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
// sum_{t'<=t} #{tau : T_tau >= t'}, K_eff at the kept depth, the bitmap columns
// and (unless plan_only) the column map colmap[col] = tau | t << 16, the column
// table coltab[t - 1][tau] (thresholds up to the bitmap's, depth >= 1) and the
// covering depth dstar[col] of every plane column: the smallest d whose K extent,
// the end of section d rounded up to a K chunk, lies past the column.
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
  // planes kept: sections 1..dkeep; the bitmap holds thresholds 2..tb
  const int32_t dkeep = kept_depth(P, tmax);
  const int64_t k_eff = dkeep >= 1 ? (int64_t)P.secend[dkeep] : 0;
  int64_t k_pad = (k_eff + kKCols - 1) / kKCols * kKCols;
  if (k_pad < kKCols) k_pad = kKCols;
  const bool rem = remainder_mode(P);
  const int32_t tb = rem ? min(bit_depth(P), tmax) : 0;
  const int32_t bm_cols = tb >= 2 ? P.secend[tb] - P.secend[1] : 0;
  if (tid == 0) {
    P.hdr->t_max = tmax;
    P.hdr->depth = dkeep;
    P.hdr->k_eff = k_eff;
    P.hdr->k_pad = (int32_t)k_pad;
    P.hdr->t_bits = tb;
    P.hdr->bm_cols = bm_cols;
  }
  if (plan_only) return;
  if (k_pad > P.k_cap || (int64_t)bm_cols > P.bm_cols) {
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
  if (rem) {
    // the inverse map: column of (t, word) for t <= max(dkeep, tb) (-1 = none); the
    // kept sections from the column map, the bitmap's further sections by a scan
    const int32_t ttab = max(dkeep, tb);
    for (int i = tid; i < ttab * eps; i += blockDim.x) P.coltab[i] = -1;
    __syncthreads();
    for (int c = tid; c < k_eff; c += blockDim.x) {
      const int32_t e = P.colmap[c];
      P.coltab[(int64_t)((e >> 16) - 1) * eps + (e & 0xFFFF)] = c;
    }
    for (int t = dkeep + 1; t <= tb; ++t) {
      if (tid == 0) s_carry = 0;
      __syncthreads();
      for (int base = 0; base < eps; base += blockDim.x) {
        const int tau = base + tid;
        const int32_t keep = (tau < eps && P.T[tau] >= t) ? 1 : 0;
        int32_t tot;
        const int32_t incl = block_scan_incl<int32_t>(keep, s_warp, &tot);
        if (keep) P.coltab[(int64_t)(t - 1) * eps + tau] = P.secend[t - 1] + s_carry + incl - 1;
        __syncthreads();
        if (tid == 0) s_carry += tot;
        __syncthreads();
      }
    }
    // covering depth of each plane column (columns past K_eff: padding, never a
    // remainder entry)
    for (int64_t c = tid; c < k_pad; c += blockDim.x) {
      int32_t d = 1;
      while (d < dkeep &&
             min((int64_t)(P.secend[d] + kKCols - 1) / kKCols * kKCols, k_pad) <= c)
        ++d;
      P.dstar[c] = (int8_t)d;
    }
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
    const int64_t np = dev_n_pad(e.n, P.tile);
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

// Remainder bookkeeping of a count c >= 2 of word tau in stored row pos (plans of
// depth >= 1): the row's profile, each threshold 2..min(c, tb) counted under the
// first plane depth that covers its column (dkeep + 1 when it is above the planes),
// and the row's heavy count (c > tb). ru[d] = the K extent of depth d (the end of
// section d rounded up to a K chunk, at most K_pad), d = 1..dkeep: the covering
// depth of a column is the smallest d whose extent lies past it. (The remainder
// bitmap is filled later, from the flat entries, once the block depths are known.)
__device__ __forceinline__ void note_count(const RankPtrs &P, int32_t tau, int32_t c, int32_t dkeep,
                                        int32_t tb, const int32_t *ru, uint32_t *s_prof) {
  const int32_t top = min(c, tb);
  for (int32_t t = 2; t <= top; ++t) {
    int32_t ds = dkeep + 1;
    if (t <= dkeep) {
      const int32_t col = P.coltab[(int64_t)(t - 1) * P.eps + tau];
      ds = 1;
      while (ds < dkeep && ru[ds] <= col) ++ds;
    }
    atomicAdd(&s_prof[ds - 1], 1u);
  }
  if (c > tb) atomicAdd(&s_prof[kProf - 1], 1u);
}

// K extents of the kept depths into ru[1..dkeep] (shared; the calling block then
// synchronises).
__device__ __forceinline__ void fill_extents(const RankPtrs &P, int32_t dkeep, int32_t k_pad,
                                             int32_t *ru) {
  for (int d = threadIdx.x; d <= kMaxPlaneDepth; d += blockDim.x)
    ru[d] = d >= 1 && d <= dkeep ? min((P.secend[d] + kKCols - 1) / kKCols * kKCols, k_pad) : 0;
}

__global__ void bitmap_zero_kernel(RankPtrs P) {
  pdl_enter();
  if (P.hdr->status != 0) return;
  // the columns from bm_lo on (the only ones a remainder entry can name)
  const int64_t c0 = max(P.hdr->bm_lo - P.secend[1], 0);
  const int64_t words4 = max((int64_t)P.hdr->bm_cols - c0, (int64_t)0) * (P.n_pad / 128);
  uint4 *p = reinterpret_cast<uint4 *>(P.bitmap) + c0 * (P.n_pad / 128);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words4;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = make_uint4(0, 0, 0, 0);
}

// Plane rows, kPlaneRows stored rows per block iteration: stage the rows' counts
// (as 16-bit) in shared memory with 16-byte loads, write their K_pad plane bytes
// 16 at a time (the column map of a chunk is read once for all the rows), raise
// the largest count of each row's 128-row block, check that the row's counts add
// up to its number of windows m, and (depth >= 1) note its counts >= 2 for the
// remainder and append them to the flat entry list.
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
  __shared__ uint32_t s_prof[kPlaneRows][kProf];
  __shared__ int32_t s_ru[kMaxPlaneDepth + 1];
  // the K extents first: every thread reaches the barrier
  fill_extents(P, P.hdr->depth, P.hdr->k_pad, s_ru);
  __syncthreads();
  if (P.hdr->status != 0) return;
  const int32_t k_eff = (int32_t)P.hdr->k_eff;
  const int32_t k_pad = P.hdr->k_pad;
  const int32_t dkeep = P.hdr->depth;
  const bool residual = remainder_mode(P);
  const int32_t tb = bit_depth(P);
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
    if (threadIdx.x < kPlaneRows * kProf) (&s_prof[0][0])[threadIdx.x] = 0u;
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
      // counts >= 2 of the rows, appended unordered: (stored row, word | count << 16).
      // The block counts its entries first and reserves their slots with one atomic.
      int32_t mine = 0;
#pragma unroll
      for (int r = 0; r < kPlaneRows; ++r)
        if (xs[r] >= 0)
          for (int tau = threadIdx.x; tau < eps; tau += blockDim.x)
            mine += s_cnt[r * eps + tau] >= 2;
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
        for (int tau = threadIdx.x; tau < eps; tau += blockDim.x) {
          const int32_t c = s_cnt[r * eps + tau];
          if (c >= 2) {
            note_count(P, tau, c, dkeep, tb, s_ru, s_prof[r]);
            if (slot < (unsigned long long)P.list_cap)
              P.flat[slot] = make_int2((int32_t)pos, tau | (c << 16));
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
    __syncthreads();  // the rows' profiles are complete
    if (threadIdx.x < kPlaneRows && xs[threadIdx.x] >= 0) {
      const int64_t pos = g * kPlaneRows + threadIdx.x;
      atomicMax(&P.depth[pos / kRowBlock], s_max[threadIdx.x]);
      // the counts of a row must add up to its number of windows, m
      if (s_sum[threadIdx.x] != (int32_t)(P.rec[pos].w & 0xFFFFu))
        record_error(P.hdr, SAD_ERR_BAD_INPUT, xs[threadIdx.x]);
    }
    if (residual && threadIdx.x < kPlaneRows * kProf) {
      const int r = threadIdx.x / kProf, j = threadIdx.x % kProf;
      P.prof[(g * kPlaneRows + r) * kProf + j] = s_prof[r][j];
    }
    __syncthreads();
  }
}

// Plane rows for plans of depth >= 1 (the streaming writer below). A plane value is
// the 4-bit e2m1 [c >= t] (1.0 or 0), two columns to a byte. Counts >= 2 also set
// their remainder bitmap bits and the row's profile, and go to a per-warp buffer
// that is appended to the flat entry list with one atomic per row; a row with more
// than kExCap of them is scanned again for the append.
constexpr int kExCap = 64;
constexpr int kStreamUnroll = 4;

__device__ __forceinline__ uint32_t plane_val(int32_t c, int32_t t) { return c >= t ? kE2M1One : 0u; }

// The streaming plane writer: a warp per stored row, two passes over the row.
// Pass 1 streams the row's counts once (16 bytes per lane, four loads in flight):
// the row's largest count and sum, the remainder bookkeeping of every count >= 2,
// section 1 written directly when it is the identity map (four words to one 2-byte
// store), and the counts kept in the warp's shared memory as 4-bit values
// saturated at 15 (every plane threshold is <= 8). Pass 2 writes every other
// 32-bit word of the row (eight columns) once, in order: for each column its word
// and threshold from the column map, its value [count >= t] from the shared 4-bit
// counts. No global atomics, no zero fill: each byte is written once.
constexpr int kStreamWarps = 8;
constexpr int kStreamThreads = 32 * kStreamWarps;

__global__ void __launch_bounds__(kStreamThreads, 4) planes_stream_kernel(
    const int32_t *__restrict__ counts, int32_t eps, RankPtrs P) {
  pdl_enter();
  extern __shared__ uint4 s_nib4[];
  __shared__ int2 s_ex[kStreamWarps][kExCap];
  __shared__ int32_t s_exn[kStreamWarps];
  __shared__ uint32_t s_prof[kStreamWarps][kProf];
  __shared__ int32_t s_ru[kMaxPlaneDepth + 1];
  // the K extents first: every thread reaches the barrier
  fill_extents(P, P.hdr->depth, P.hdr->k_pad, s_ru);
  __syncthreads();
  if (P.hdr->status != 0) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wa = blockDim.x >> 5;
  const int32_t k_pad = P.hdr->k_pad;
  const int32_t k_eff = (int32_t)P.hdr->k_eff;
  const int32_t dkeep = P.hdr->depth;
  const bool residual = remainder_mode(P);
  const int32_t tb = bit_depth(P);
  const int q4 = eps >> 2;
  const int32_t s1 = P.secend[1];  // end of section 1
  const bool ident = s1 == eps;    // section 1 = every word, in order
  const int32_t kw = k_pad / 8;    // 32-bit words of the row in use
  // words [0, w1) hold section-1 columns only and are written in pass 1
  const int32_t w1 = ident ? s1 / 8 : 0;
  // the warp's 4-bit counts: eps / 2 bytes rounded up to 16
  const int32_t nib_words = ((eps / 2 + 15) & ~15) / 4;
  uint32_t *nib = reinterpret_cast<uint32_t *>(s_nib4) + (size_t)warp * nib_words;
  uint16_t *nib16 = reinterpret_cast<uint16_t *>(nib);
  if (lane == 0) s_exn[warp] = 0;
  if (lane < kProf) s_prof[warp][lane] = 0u;
  __syncwarp();
  for (int64_t pos = (int64_t)blockIdx.x * wa + warp; pos < P.n_pad;
       pos += (int64_t)gridDim.x * wa) {
    const int32_t x = P.perm[pos];
    uint8_t *prow = P.planes + pos * (P.k_cap / 2);
    if (x < 0) {  // padding row: all zero
      for (int c = 16 * lane; c < k_pad / 2; c += 512)
        *reinterpret_cast<uint4 *>(prow + c) = make_uint4(0, 0, 0, 0);
      if (residual && lane < kProf) P.prof[pos * kProf + lane] = 0u;
      continue;
    }
    const int4 *row4 = reinterpret_cast<const int4 *>(counts + (int64_t)x * eps);
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
        nib16[q] = (uint16_t)(min(c[0], 15) | min(c[1], 15) << 4 | min(c[2], 15) << 8 |
                              min(c[3], 15) << 12);
        if (ident && q < 2 * w1) {
          // columns 4q..4q+3 = bytes 2q, 2q+1
          *reinterpret_cast<uint16_t *>(prow + 2 * q) =
              (uint16_t)(plane_val(c[0], 1) | plane_val(c[1], 1) << 4 | plane_val(c[2], 1) << 8 |
                         plane_val(c[3], 1) << 12);
        }
        if (residual) {
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            if (c[b] >= 2) {
              note_count(P, 4 * q + b, c[b], dkeep, tb, s_ru, s_prof[warp]);
              const int slot = atomicAdd(&s_exn[warp], 1);
              if (slot < kExCap) s_ex[warp][slot] = make_int2((int32_t)pos, (4 * q + b) | (c[b] << 16));
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
    // pass 2: the row's words from w1 on, eight columns each, gathered from the
    // column map and the 4-bit counts (columns past K_eff are 0). A section above the
    // row's largest count holds no 1 of the row: the gather stops at the end of
    // section min(largest count, D) and the words past it are zero.
    __syncwarp();
    uint32_t *prow32 = reinterpret_cast<uint32_t *>(prow);
    const int32_t top = min(mx, dkeep);
    const int32_t wg = top >= 1 ? min((P.secend[top] + 7) / 8, kw) : w1;
    for (int32_t w = max(wg, w1) + lane; w < kw; w += 32) prow32[w] = 0u;
    for (int32_t w = w1 + lane; w < wg; w += 32) {
      const int32_t c0 = 8 * w;
      uint32_t val = 0;
      if (c0 + 8 <= k_eff) {
        const int4 e4a = __ldg(reinterpret_cast<const int4 *>(P.colmap + c0));
        const int4 e4b = __ldg(reinterpret_cast<const int4 *>(P.colmap + c0 + 4));
        const int32_t ev[8] = {e4a.x, e4a.y, e4a.z, e4a.w, e4b.x, e4b.y, e4b.z, e4b.w};
#pragma unroll
        for (int b = 0; b < 8; ++b) {
          const uint32_t tau = (uint32_t)ev[b] & 0xFFFFu, t = (uint32_t)ev[b] >> 16;
          if (((nib[tau >> 3] >> (4 * (tau & 7))) & 15u) >= t) val |= kE2M1One << (4 * b);
        }
      } else {
        for (int b = 0; b < 8 && c0 + b < k_eff; ++b) {
          const int32_t e = __ldg(P.colmap + c0 + b);
          const uint32_t tau = (uint32_t)e & 0xFFFFu, t = (uint32_t)e >> 16;
          if (((nib[tau >> 3] >> (4 * (tau & 7))) & 15u) >= t) val |= kE2M1One << (4 * b);
        }
      }
      prow32[w] = val;
    }
    __syncwarp();  // the next row's pass 1 rewrites the 4-bit counts
    if (lane == 0) {
      atomicMax(&P.depth[pos / kRowBlock], mx);
      // the counts of a row must add up to its number of windows, m
      if (sum != (int32_t)(P.rec[pos].w & 0xFFFFu)) record_error(P.hdr, SAD_ERR_BAD_INPUT, x);
    }
    if (residual) {
      __syncwarp();
      if (lane < kProf) {
        P.prof[pos * kProf + lane] = s_prof[warp][lane];
        s_prof[warp][lane] = 0u;
      }
      const int32_t n_ex = s_exn[warp];
      if (n_ex > 0) {
        unsigned long long first = 0;
        if (lane == 0) first = atomicAdd(&P.hdr->flat_count, (unsigned long long)n_ex);
        first = __shfl_sync(0xffffffffu, first, 0);
        if (n_ex <= kExCap) {
          for (int i = lane; i < n_ex; i += 32) {
            if (first + i < (unsigned long long)P.list_cap) P.flat[first + i] = s_ex[warp][i];
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
              if (c[b] >= 2) {
                const unsigned long long slot = first + (unsigned)atomicAdd(&s_exn[warp], 1);
                if (slot < (unsigned long long)P.list_cap)
                  P.flat[slot] = make_int2((int32_t)pos, (4 * q + b) | (c[b] << 16));
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

// ------------------------------------------------------------ remainder ----
// Per column block b (B = P.tile stored rows, one thread each): N_b(d) = the block's
// remainder entries at plane depth d (its rows' thresholds whose covering depth is
// above d), for d = 1..min(dkeep, largest count); the block's depth d_b is the
// smallest d with N_b(d) <= budget (else the largest). Each row's entries at d_b
// (and its heavy entries) get offsets inside the block; the block totals go to
// blkrem for the scan. Profile slot j of a row counts the thresholds whose
// covering depth is j + 1 (slot dkeep: above the planes); at depth d the slots
// j >= d are uncovered.
constexpr int kRemThreads = 2 * kColBlock;  // largest block (CTA-pair tiles)

__global__ void __launch_bounds__(kRemThreads) rem_depth_kernel(RankPtrs P) {
  pdl_enter();
  __shared__ uint32_t s_n[kMaxPlaneDepth + 1];
  __shared__ int32_t s_d;
  __shared__ int32_t s_warp[32];
  if (P.hdr->status != 0) return;
  const int32_t dkeep = P.hdr->depth;
  const int64_t B = P.tile;  // == blockDim.x
  const int64_t nblk = P.n_pad / B;
  for (int64_t b = blockIdx.x; b < nblk; b += gridDim.x) {
    const int64_t v = b * B + threadIdx.x;
    uint32_t pr[kProf];
#pragma unroll
    for (int j = 0; j < kProf; ++j) pr[j] = P.prof[v * kProf + j];
    if (threadIdx.x <= kMaxPlaneDepth) s_n[threadIdx.x] = 0u;
    __syncthreads();
    uint32_t tail = 0;
#pragma unroll
    for (int d = kMaxPlaneDepth; d >= 1; --d) {
      if (d <= dkeep) {
        tail += pr[d];
        uint32_t w = tail;
        for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(&s_n[d], w);
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int32_t bmax = 0;
      for (int64_t b1 = b * (B / kRowBlock); b1 < (b + 1) * (B / kRowBlock); ++b1)
        bmax = max(bmax, P.depth[b1]);
      const int32_t dcap = max(1, min(dkeep, bmax));
      int32_t d = dcap;
      for (int32_t dd = 1; dd < dcap; ++dd)
        if (s_n[dd] <= (uint32_t)P.budget) {
          d = dd;
          break;
        }
      s_d = d;
      for (int64_t b1 = b * (B / kRowBlock); b1 < (b + 1) * (B / kRowBlock); ++b1) P.bdepth[b1] = d;
      if (d < bmax) atomicAdd(&P.hdr->rem_blocks, 1);
    }
    __syncthreads();
    const int32_t d = s_d;
    uint32_t e = 0;
#pragma unroll
    for (int j = 1; j <= kMaxPlaneDepth; ++j)
      if (j >= d && j <= dkeep) e += pr[j];
    const uint32_t h = pr[kProf - 1];
    int32_t tot_e, tot_h;
    const int32_t incl_e = block_scan_incl<int32_t>((int32_t)e, s_warp, &tot_e);
    const int32_t incl_h = block_scan_incl<int32_t>((int32_t)h, s_warp, &tot_h);
    P.rowrem[2 * v] = incl_e - (int32_t)e;
    P.rowrem[2 * v + 1] = incl_h - (int32_t)h;
    if (threadIdx.x == 0) {
      P.blkrem[2 * b] = tot_e;
      P.blkrem[2 * b + 1] = tot_h;
      // the smallest depth of a block that has remainder entries: no column covered at
      // that depth is ever a remainder column
      if (tot_e > 0) atomicMin(&P.hdr->dmin, d);
    }
    __syncthreads();
  }
}

// One block: exclusive scan of the block totals (in place), the grand totals at
// index nblk, and the capacity checks.
__global__ void __launch_bounds__(1024) rem_scan_kernel(RankPtrs P) {
  pdl_enter();
  __shared__ int64_t s_warp[32];
  __shared__ int64_t s_carry[2];
  if (P.hdr->status != 0) return;
  const int64_t nblk = P.n_pad / P.tile;
  if (threadIdx.x < 2) s_carry[threadIdx.x] = 0;
  __syncthreads();
  for (int64_t base = 0; base < nblk; base += blockDim.x) {
    const int64_t b = base + threadIdx.x;
#pragma unroll
    for (int f = 0; f < 2; ++f) {
      const int64_t x = b < nblk ? P.blkrem[2 * b + f] : 0;
      int64_t tot;
      const int64_t incl = block_scan_incl<int64_t>(x, s_warp, &tot);
      if (b < nblk) P.blkrem[2 * b + f] = s_carry[f] + incl - x;
      __syncthreads();
      if (threadIdx.x == 0) s_carry[f] += tot;
      __syncthreads();
    }
  }
  if (threadIdx.x == 0) {
    // lowest remainder column: past the planes (t > dkeep), or past the K extent of
    // the smallest block depth; none when no block has remainder entries
    const int32_t dkeep = P.hdr->depth, dmin = P.hdr->dmin;
    int32_t lo = P.secend[dkeep];
    if (dmin < dkeep)
      lo = min(lo, min((P.secend[dmin] + kKCols - 1) / kKCols * kKCols, P.hdr->k_pad));
    P.hdr->bm_lo = dmin == 0x7FFFFFFF ? P.secend[1] + P.hdr->bm_cols : lo;
    P.blkrem[2 * nblk] = s_carry[0];
    P.blkrem[2 * nblk + 1] = s_carry[1];
    P.hdr->rem_entries = s_carry[0];
    P.hdr->heavy_entries = s_carry[1];
    if (P.hdr->flat_count > (unsigned long long)P.list_cap)
      record_error(P.hdr, SAD_ERR_WORKSPACE, 1);
    else if (s_carry[0] > P.rem_cap)
      record_error(P.hdr, SAD_ERR_WORKSPACE, 2);
    else if (s_carry[1] > P.heavy_cap)
      record_error(P.hdr, SAD_ERR_WORKSPACE, 3);
  }
}

// Every flat entry (row, word, count): the thresholds that the plane depth of the
// row's block does not cover become remainder entries of the row (their bitmap
// columns), and a count above T_b one heavy entry. The order inside a row is free.
__global__ void __launch_bounds__(256) rem_scatter_kernel(RankPtrs P) {
  pdl_enter();
  if (P.hdr->status != 0) return;
  const int32_t dkeep = P.hdr->depth;
  const int32_t tb = bit_depth(P);
  const int32_t n1 = P.secend[1];
  const int32_t bm_lo = P.hdr->bm_lo;
  const int64_t bm_stride = P.n_pad / 32;
  const int64_t nf = (int64_t)min(P.hdr->flat_count, (unsigned long long)P.list_cap);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nf;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int2 f = P.flat[i];
    const int64_t pos = f.x;
    const int32_t tau = f.y & 0xFFFF;
    const int32_t c = (int32_t)((uint32_t)f.y >> 16);
    const int64_t b = pos / P.tile;
    const int32_t d = P.bdepth[pos / kRowBlock];
    const int64_t base = P.blkrem[2 * b] + P.rowrem[2 * pos];
    const int32_t top = min(c, tb);
    for (int32_t t = 2; t <= top; ++t) {
      const int32_t col = P.coltab[(int64_t)(t - 1) * P.eps + tau];
      // the row's bit in the remainder bitmap (columns a remainder entry can name)
      if (col >= bm_lo)
        atomicOr(&P.bitmap[(int64_t)(col - n1) * bm_stride + (pos >> 5)], 1u << (pos & 31));
      const bool covered = t <= dkeep && (int32_t)P.dstar[col] <= d;
      if (!covered) {
        const int32_t slot = atomicAdd(&P.cursor[2 * pos], 1);
        P.rem[base + slot] = (uint32_t)(col - n1);
      }
    }
    if (c > tb) {
      const int32_t slot = atomicAdd(&P.cursor[2 * pos + 1], 1);
      P.heavy[P.blkrem[2 * b + 1] + P.rowrem[2 * pos + 1] + slot] = make_int2(tau, c);
    }
  }
}

// Upper-triangle tile list of every set (blocks per set and column group). Tile (I, J) of a
// set covers its stored rows [B I, B I + B) and columns [B J, B J + B), B = P.tile
// (set-local; 128, or 256 for CTA pairs); it is needed when some pair i <= j lies in it
// (I <= J) and both ranges hold real rows. Tiles are grouped by G column blocks,
// rows ascending inside a group, so that the tiles running at the same time share
// their operand panels in L2: a group's G column panels stay in L2 while the row
// panels stream past them once per group, so G is as large as an L2 budget allows
// for the panel size (group_cols). Each entry is (I | J << 16, nk | nx << 16) with global
// block indices: nk plane K chunks, up to the end of section e = min(largest count
// of I, largest count of J, plane depth of J) (the kept depth when nothing is cut),
// and nx remainder K chunks of 256 entries of column block J.
// Column blocks per tile group: G panels of `rows` rows x K_cap / 2 bytes within
// kGroupL2Bytes, between 8 and 64.
constexpr int64_t kGroupL2Bytes = 40ll << 20;
inline int32_t group_cols(int64_t k_cap, int64_t rows) {
  const int64_t panel = rows * (k_cap > 0 ? k_cap : kKCols) / 2;
  const int64_t g = kGroupL2Bytes / panel;
  return (int32_t)(g < 8 ? 8 : (g > 64 ? 64 : g));
}
// remainder entries per extra K chunk of a tile: one K column each
constexpr int kRemChunkCols = kKCols;

// Tiles of column group g of a set: rows I with J in [G g, G g + G) and J >= I.
__device__ __forceinline__ int32_t group_row_tiles(int32_t g, int32_t I, int32_t C, int32_t G) {
  const int32_t j0 = max(g * G, I);
  const int32_t j1 = min((g + 1) * G, C);
  return max(0, j1 - j0);
}

// (blockIdx.y: sets in a grid stride; blockIdx.x: column groups in a grid stride)
__global__ void __launch_bounds__(256) tiles_kernel(RankPtrs P, int32_t G) {
  pdl_enter();
  __shared__ int32_t s_warp[32];
  __shared__ int32_t s_carry;
  const int tid = threadIdx.x;
  const int32_t nblk = (int32_t)(P.n_pad / kRowBlock);
  const int32_t dkeep = P.hdr->depth;
  const bool rem = remainder_mode(P);
  const int32_t B = P.tile, sub = P.tile / kRowBlock;  // tile rows, 128-row blocks in one
  for (int32_t si = blockIdx.y; si < (int32_t)P.n_sets; si += gridDim.y) {
    const RankSet e = P.sets[si];
    const int32_t n = e.n;
    const int32_t R = (n + B - 1) / B;
    const int32_t C = R;
    const int32_t I0 = (int32_t)(e.row_base / B), J0 = (int32_t)(e.row_base / B);
    const int32_t groups = (C + G - 1) / G;
    for (int32_t g = blockIdx.x; g < groups; g += gridDim.x) {
      // tiles of the groups before g come first
      int32_t before = 0;
      for (int64_t gi = tid; gi < (int64_t)g * R; gi += blockDim.x)
        before += group_row_tiles((int32_t)(gi / R), (int32_t)(gi % R), C, G);
      int32_t tot;
      block_scan_incl<int32_t>(before, s_warp, &tot);
      if (tid == 0) s_carry = tot;
      __syncthreads();
      unsigned long long chunks = 0;
      int32_t group_tiles = 0;
      for (int32_t base = 0; base < R; base += blockDim.x) {
        const int32_t I = base + tid;
        const int32_t cnt = I < R ? group_row_tiles(g, I, C, G) : 0;
        const int32_t incl = block_scan_incl<int32_t>(cnt, s_warp, &tot);
        int64_t out = e.tile_base + s_carry + incl - cnt;
        if (cnt > 0) {
          // largest counts of the tile's row and column blocks (sub 128-row blocks each)
          int32_t dI = 0;
          for (int32_t b = sub * (I0 + I); b < sub * (I0 + I + 1) && b < nblk; ++b)
            dI = max(dI, P.depth[b]);
          const int32_t j0 = max(g * G, I);
          for (int32_t J = j0; J < j0 + cnt; ++J) {
            int32_t dJ = 0;
            for (int32_t b = sub * (J0 + J); b < sub * (J0 + J + 1) && b < nblk; ++b)
              dJ = max(dJ, P.depth[b]);
            const int32_t cut = rem ? P.bdepth[sub * (J0 + J)] : dkeep;
            const int32_t d = min(min(dI, dJ), cut);
            const int32_t kend = P.secend[max(d, 0)];
            const int32_t nk = max(1, (kend + kKCols - 1) / kKCols);
            // remainder chunks of the column block (one K column per entry)
            int32_t nx = 0;
            if (rem) {
              const int64_t ne = P.blkrem[2 * (J0 + J) + 2] - P.blkrem[2 * (J0 + J)];
              const int64_t x = (ne + kRemChunkCols - 1) / kRemChunkCols;
              if (x > 0x7FFF) record_error(P.hdr, SAD_ERR_UNSUPPORTED, J0 + J);
              nx = (int32_t)min(x, (int64_t)0x7FFF);
            }
            P.tiles[out++] = make_int2((I0 + I) | ((J0 + J) << 16), nk | (nx << 16));
            chunks += (unsigned long long)(nk + nx);
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
  const bool rem = P.depth_cap >= 1;
  RankPtrs Q = P;
  Q.eps = eps;
  Q.counts = counts;
  pdl_launch(rank_setup_kernel, 1, 1024, 0, st, d_n, (int32_t)n, Q);
  SAD_LAUNCH_CHECK();
  if (Q.n_sets > 1) {
    pdl_launch(rank_setmaps_kernel, gsets, 256, 0, st, Q);
    SAD_LAUNCH_CHECK();
  }
  pdl_launch(rank_init_kernel, grid_for(2 * Q.n_pad + kMaxM, 256), 256, 0, st, Q, eps,
             !plan_only);
  SAD_LAUNCH_CHECK();
  if (!plan_only) {
    pdl_launch(lengths_kernel, grid_for(n, 256), 256, 0, st, lengths, k, Q);
    SAD_LAUNCH_CHECK();
  }
  if (word_max && !plan_only) {
    pdl_launch(copy_word_max_kernel, grid_for(eps, 256), 256, 0, st, word_max, eps, Q);
    SAD_LAUNCH_CHECK();
  } else {
    dim3 g((eps + 255) / 256, 1);
    int64_t slices = ((int64_t)num_sms() * 8 + g.x - 1) / g.x;
    if (slices > (n + 63) / 64) slices = (n + 63) / 64;
    if (slices < 1) slices = 1;
    g.y = (unsigned)slices;
    // the plan counts the remainder's sizes here; a run counts its entries in the plane kernel
    pdl_launch(colmax_kernel, g, 256, 0, st, counts, eps, Q, plan_only);
    SAD_LAUNCH_CHECK();
  }
  pdl_launch(colmap_kernel, 1, 1024, 0, st, Q, eps, plan_only);
  SAD_LAUNCH_CHECK();
  if (plan_only) return SAD_OK;
  if (Q.n_sets == 1) {
    pdl_launch(lensort_scan_kernel, 1, 1024, 0, st, Q);
    SAD_LAUNCH_CHECK();
    pdl_launch(lensort_place_kernel, grid_for(Q.n_pad, 256), 256, 0, st, lengths, k, Q);
    SAD_LAUNCH_CHECK();
  } else {
    if (!g_attr_sort) {
      if (cudaFuncSetAttribute(lensort_sets_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)kSortSmem) != cudaSuccess)
        return SAD_ERR_CUDA;
      g_attr_sort = true;
    }
    pdl_launch(lensort_sets_kernel, gsets, kSortThreads, kSortSmem, st, lengths, k, Q);
    SAD_LAUNCH_CHECK();
  }
  if (rem && (eps & 3) == 0 && (reinterpret_cast<uintptr_t>(counts) & 15) == 0 &&
      (Q.k_cap & 31) == 0) {
    // 4-bit counts of a row per warp: eps / 2 bytes rounded up to 16; as many warps a
    // block as fit in 96 KB (eight for eps <= 24000)
    const int64_t nib_bytes = ((eps / 2 + 15) & ~15);
    const int64_t fit = (96 << 10) / nib_bytes;
    const int warps = (int)std::max<int64_t>(1, std::min<int64_t>(kStreamWarps, fit));
    const int dyn = (int)(warps * nib_bytes);
    static bool attr_set = false;
    if (!attr_set) {
      if (cudaFuncSetAttribute(planes_stream_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               96 << 10) != cudaSuccess)
        return SAD_ERR_CUDA;
      attr_set = true;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, planes_stream_kernel, 32 * warps,
                                                      dyn) != cudaSuccess)
      return SAD_ERR_CUDA;
    const int64_t cap = (int64_t)num_sms() * (per_sm > 0 ? per_sm : 1);
    const int64_t want = (Q.n_pad + warps - 1) / warps;
    pdl_launch(planes_stream_kernel, (unsigned)(want < cap ? want : cap), 32 * warps, (size_t)dyn,
               st, counts, eps, Q);
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
    const int64_t groups = Q.n_pad / kPlaneRows;
    const int64_t cap = (int64_t)num_sms() * (per_sm > 0 ? per_sm : 1);
    pdl_launch(planes_kernel, (unsigned)(groups < cap ? groups : cap), 256, smem, st, counts, eps,
               Q);
    SAD_LAUNCH_CHECK();
  }
  if (rem) {
    const int64_t nblk = Q.n_pad / Q.tile;
    pdl_launch(rem_depth_kernel, (unsigned)(nblk < 65535 ? nblk : 65535), (unsigned)Q.tile, 0, st,
               Q);
    SAD_LAUNCH_CHECK();
    pdl_launch(rem_scan_kernel, 1, 1024, 0, st, Q);
    SAD_LAUNCH_CHECK();
    if (Q.bm_cols > 0) {
      pdl_launch(bitmap_zero_kernel, (unsigned)num_sms() * 8, 256, 0, st, Q);
      SAD_LAUNCH_CHECK();
    }
    pdl_launch(rem_scatter_kernel, grid_for(Q.list_cap, 256), 256, 0, st, Q);
    SAD_LAUNCH_CHECK();
  }
  {
    // one set: a CTA per column group; batches: a few per set
    const int32_t G = group_cols(Q.k_cap, Q.tile);
    const int64_t groups1 = ((n + Q.tile - 1) / Q.tile + G - 1) / G;
    dim3 g((unsigned)(Q.n_sets == 1 ? (groups1 > 0 ? groups1 : 1) : 4), gsets);
    pdl_launch(tiles_kernel, g, 256, 0, st, Q, G);
  }
  SAD_LAUNCH_CHECK();
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
