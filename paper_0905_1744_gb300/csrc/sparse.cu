// The k-mer rank by sparse intersection on the CUDA cores: the per-pair cost of
// Table 2 (O(L) per pair: the common counts of Eq. 1 found by walking one
// sequence's list of occurring words), as a comparison point for the
// threshold-plane GEMM. Same keys as kmer_rank, bit for bit:
//     key_i = sum_j floor(S_ij 2^64 / D_ij),  D_ij = min(L_i, L_j) - k + 1.
//
//   sparse_nnz / scan / fill  each sequence's occurring words as a sorted list of
//                             (word << 16 | count), from the dense counts
//   sparse_rank               one CTA per sequence i: its counts in a shared u16
//                             histogram; warps take sequences j, lanes walk j's
//                             list and add min(c_i(word), c_j(word)); the term
//                             S Q + floor(S r / d) (division record of the shorter
//                             sequence) is summed in 128 bits. Every ordered pair
//                             is evaluated (each unordered pair twice), so no atomics.
#include "rank.cuh"

namespace sad {

namespace {

struct SparseLayout {
  size_t nnz, off, rec, entries, bytes;
};

SparseLayout sparse_layout(int64_t n, int64_t entries_cap) {
  SparseLayout L{};
  size_t o = sizeof(WsHeader);
  auto take = [&](size_t b) { size_t r = o; o = align_up(o + b, 256); return r; };
  L.nnz = take(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  L.off = take(sizeof(int64_t) * (size_t)(n + 1));
  L.rec = take(16 * (size_t)(n > 0 ? n : 1));
  L.entries = take(sizeof(uint32_t) * (size_t)(entries_cap > 0 ? entries_cap : 1));
  L.bytes = o;
  return L;
}

// Warp per sequence: words with a nonzero count; the division record of m = L - k + 1.
__global__ void sparse_nnz_kernel(const int32_t *__restrict__ counts, const int32_t *lengths,
                                  int32_t n, int32_t eps, int32_t k, int32_t *nnz, uint4 *rec,
                                  WsHeader *hdr) {
  pdl_enter();
  const int lane = threadIdx.x & 31;
  for (int64_t x = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; x < n;
       x += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int32_t *row = counts + x * (int64_t)eps;
    int32_t c = 0;
    for (int t = lane; t < eps; t += 32) c += row[t] != 0;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) {
      nnz[x] = c;
      const int32_t m = lengths[x] - k + 1;
      if (m < 1 || m > kMaxM) record_error(hdr, m < 1 ? SAD_ERR_BAD_INPUT : SAD_ERR_UNSUPPORTED,
                                           (int)x);
      rec[x] = division_record((uint32_t)min(max(m, 1), kMaxM));
      atomicAdd(reinterpret_cast<unsigned long long *>(&hdr->list_total),
                (unsigned long long)c);
    }
  }
}

// One block: exclusive prefix of the per-sequence list sizes.
__global__ void __launch_bounds__(1024) sparse_scan_kernel(const int32_t *nnz, int32_t n,
                                                           int64_t *off, int64_t cap,
                                                           WsHeader *hdr) {
  pdl_enter();
  __shared__ int64_t s_warp[32];
  __shared__ int64_t s_carry;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int64_t base = 0; base < n; base += blockDim.x) {
    const int64_t x = base + threadIdx.x;
    int64_t v = x < n ? nnz[x] : 0, incl = v;
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      int64_t w = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      s_warp[lane] = w;
    }
    __syncthreads();
    const int64_t before = s_carry + (wid > 0 ? s_warp[wid - 1] : 0) + incl - v;
    if (x < n) off[x] = before;
    __syncthreads();
    if (threadIdx.x == 0) s_carry += s_warp[(blockDim.x >> 5) - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    off[n] = s_carry;
    if (s_carry > cap) record_error(hdr, SAD_ERR_WORKSPACE, -1);
  }
}

// Warp per sequence: the list in ascending word order (ballot compaction).
__global__ void sparse_fill_kernel(const int32_t *__restrict__ counts, int32_t n, int32_t eps,
                                   const int64_t *off, uint32_t *entries, WsHeader *hdr) {
  pdl_enter();
  if (hdr->status != 0) return;
  const int lane = threadIdx.x & 31;
  for (int64_t x = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; x < n;
       x += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int32_t *row = counts + x * (int64_t)eps;
    int64_t out = off[x];
    for (int base = 0; base < eps; base += 32) {
      const int t = base + lane;
      const int32_t c = t < eps ? row[t] : 0;
      const unsigned m = __ballot_sync(0xffffffffu, c != 0);
      if (c != 0)
        entries[out + __popc(m & ((1u << lane) - 1u))] =
            ((uint32_t)t << 16) | (uint32_t)min(c, 0xFFFF);
      out += __popc(m);
    }
  }
}

__device__ __forceinline__ void add128(uint64_t &hi, uint64_t &lo, uint64_t ahi, uint64_t alo) {
  lo += alo;
  hi += ahi + (lo < alo ? 1u : 0u);
}

// floor(S 2^64 / d) as (hi, lo) from the division record of d (S <= 65535).
__device__ __forceinline__ void term128(uint32_t s, uint4 rec, uint64_t &hi, uint64_t &lo) {
  const uint32_t d = rec.w & 0xFFFFu;
  const uint32_t sh1 = (rec.w >> 16) & 0xFFu, sh2 = rec.w >> 24;
  const uint32_t r = 0u - rec.x * d;
  const uint32_t xq = s * r;
  const uint32_t t1 = __umulhi(rec.z, xq);
  const uint32_t qv = (t1 + ((xq - t1) >> sh1)) >> sh2;
  const uint64_t Q = ((uint64_t)rec.y << 32) | rec.x;
  lo = (uint64_t)s * Q;
  hi = __umul64hi((uint64_t)s, Q);
  const uint64_t l2 = lo + qv;
  hi += l2 < lo ? 1u : 0u;
  lo = l2;
}

constexpr int kSparseWarps = 8;

__global__ void __launch_bounds__(kSparseWarps * 32)
    sparse_rank_kernel(const int32_t *__restrict__ counts, int32_t n, int32_t eps,
                       const int64_t *__restrict__ off, const uint32_t *__restrict__ entries,
                       const uint4 *__restrict__ rec, uint64_t *key_hi, uint64_t *key_lo,
                       double *rank, WsHeader *hdr) {
  pdl_enter();
  extern __shared__ uint16_t s_hist[];  // [eps]
  __shared__ uint64_t s_hi[kSparseWarps], s_lo[kSparseWarps];
  if (hdr->status != 0) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
    __syncthreads();
    const int32_t *row = counts + i * (int64_t)eps;
    for (int t = threadIdx.x; t < eps; t += blockDim.x)
      s_hist[t] = (uint16_t)min(max(row[t], 0), 0xFFFF);
    __syncthreads();
    const uint4 rec_i = rec[i];
    const uint32_t m_i = rec_i.w & 0xFFFFu;
    uint64_t acc_hi = 0, acc_lo = 0;  // lane 0 of each warp
    for (int64_t j = warp; j < n; j += kSparseWarps) {
      const int64_t a = off[j], e = off[j + 1];
      uint32_t s = 0;
      for (int64_t p = a + lane; p < e; p += 32) {
        const uint32_t v = entries[p];
        s += min((uint32_t)s_hist[v >> 16], v & 0xFFFFu);
      }
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) {
        const uint4 rec_j = rec[j];
        uint64_t th, tl;
        term128(s, m_i <= (rec_j.w & 0xFFFFu) ? rec_i : rec_j, th, tl);
        add128(acc_hi, acc_lo, th, tl);
      }
    }
    if (lane == 0) {
      s_hi[warp] = acc_hi;
      s_lo[warp] = acc_lo;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      uint64_t hi = 0, lo = 0;
      for (int w = 0; w < kSparseWarps; ++w) add128(hi, lo, s_hi[w], s_lo[w]);
      key_hi[i] = hi;
      key_lo[i] = lo;
      if (rank) {
        const double whole = __ull2double_rn(hi);
        const double frac = __dmul_rn(__ull2double_rn(lo), 0x1p-64);
        rank[i] = __ddiv_rn(__dadd_rn(whole, frac), (double)n);
      }
    }
  }
}

unsigned grid_of(int64_t work, int threads) {
  int64_t g = (work + threads - 1) / threads;
  const int64_t cap = (int64_t)num_sms() * 8;
  return (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
}

}  // namespace

size_t sparse_ws_bytes(int64_t n, int64_t entries_cap) {
  return sparse_layout(n, entries_cap).bytes;
}

int sparse_count_launch(const int32_t *counts, const int32_t *lengths, int32_t n, int32_t k,
                        int32_t eps, void *ws, size_t ws_bytes, cudaStream_t st) {
  const SparseLayout L = sparse_layout(n, 0);
  if (ws_bytes < L.bytes) return SAD_ERR_WORKSPACE;
  uint8_t *b = static_cast<uint8_t *>(ws);
  WsHeader *hdr = reinterpret_cast<WsHeader *>(b);
  if (cudaMemsetAsync(hdr, 0, sizeof(WsHeader), st) != cudaSuccess) return SAD_ERR_CUDA;
  pdl_launch(sparse_nnz_kernel, grid_of((int64_t)n * 32, 256), 256, 0, st, counts, lengths, n, eps,
             k, reinterpret_cast<int32_t *>(b + L.nnz), reinterpret_cast<uint4 *>(b + L.rec), hdr);
  SAD_LAUNCH_CHECK();
  return SAD_OK;
}

int sparse_rank_launch(const int32_t *counts, const int32_t *lengths, int32_t n, int32_t k,
                       int32_t eps, int64_t entries_cap, uint64_t *key_hi, uint64_t *key_lo,
                       double *rank, void *ws, size_t ws_bytes, cudaStream_t st) {
  const SparseLayout L = sparse_layout(n, entries_cap);
  if (ws_bytes < L.bytes) return SAD_ERR_WORKSPACE;
  const size_t smem = sizeof(uint16_t) * (size_t)eps;
  if (smem > 200 * 1024) return SAD_ERR_UNSUPPORTED;
  int rc = sparse_count_launch(counts, lengths, n, k, eps, ws, ws_bytes, st);
  if (rc) return rc;
  uint8_t *b = static_cast<uint8_t *>(ws);
  WsHeader *hdr = reinterpret_cast<WsHeader *>(b);
  int64_t *off = reinterpret_cast<int64_t *>(b + L.off);
  uint32_t *entries = reinterpret_cast<uint32_t *>(b + L.entries);
  const uint4 *rec = reinterpret_cast<const uint4 *>(b + L.rec);
  pdl_launch(sparse_scan_kernel, 1, 1024, 0, st, reinterpret_cast<const int32_t *>(b + L.nnz), n,
             off, entries_cap, hdr);
  SAD_LAUNCH_CHECK();
  pdl_launch(sparse_fill_kernel, grid_of((int64_t)n * 32, 256), 256, 0, st, counts, n, eps, off,
             entries, hdr);
  SAD_LAUNCH_CHECK();
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(sparse_rank_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             200 * 1024) != cudaSuccess)
      return SAD_ERR_CUDA;
    attr = true;
  }
  const int64_t grid = n < (int64_t)num_sms() * 4 ? n : (int64_t)num_sms() * 4;
  // plain stream order: launched early, its CTAs (4 a SM, rows in a static stride)
  // would be placed unevenly while the previous kernel still holds SMs (measured 2x
  // slower); its pdl_enter() is then a no-op
  sparse_rank_kernel<<<(unsigned)(grid > 0 ? grid : 1), kSparseWarps * 32, smem, st>>>(
      counts, n, eps, off, entries, rec, key_hi, key_lo, rank, hdr);
  SAD_LAUNCH_CHECK();
  return SAD_OK;
}

}  // namespace sad
