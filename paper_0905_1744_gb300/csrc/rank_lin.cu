// Linear part of the rank keys (Eq. 1 / Eq. 3) for pairs of rows in different
// 128-row blocks, in O(N K) instead of per pair.
//
// The key of a stored row i is sum_j floor(S_ij 2^64 / D_ij) with D_ij = m_j for
// i <= j (rows in decreasing length), and floor(S 2^64 / d) = S Q + floor(S r / d)
// with Q = floor((2^64 - 1) / d), r = 2^64 - Q d. The GEMM epilogue adds the floor
// parts of every pair, and the whole term for pairs inside one 128-row block (the
// diagonal tiles). What remains is sum over i < j in different blocks of S_ij Q_j,
// added to key_i and to key_j. With S_ij = sum_k P_ik P_jk over the plane columns k:
//
//   for i in block b:  sum_{j in later blocks} S_ij Q_j = sum_k P_ik V_k(b),
//                      V_k(b) = sum over rows j of the set's blocks after b of P_jk Q_j
//   for j in block b:  Q_j sum_{i in earlier blocks} S_ij = Q_j sum_k P_jk U_k(b),
//                      U_k(b) = number of rows i of the set's blocks before b with P_ik = 1
//
// Three passes: per block and column the count and Q sum of its rows (lin_cols),
// exclusive prefix / suffix over the blocks of each set (lin_scan), and per row
// the two dot products with its own plane row, added to the key limbs (lin_rows).
// Counts above the plane depth are not in the planes: their share of the linear
// part is added by the GEMM epilogue, where the residual is.
#include "rank.cuh"

namespace sad {

namespace {

__device__ __forceinline__ void red_add_u64(unsigned long long *p, unsigned long long v) {
  asm volatile("red.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// (blockIdx.y = 128-row block b, thread = one 32-bit word = 8 plane columns)
__global__ void __launch_bounds__(256) lin_cols_kernel(RankPtrs P) {
  if (P.hdr->status != 0) return;
  const int64_t words = P.hdr->k_pad / 8;
  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= words) return;
  const int64_t b = blockIdx.y;
  const int64_t row_words = P.k_cap / 8;
  const uint32_t *col = reinterpret_cast<const uint32_t *>(P.planes) + b * kRowBlock * row_words + w;
  uint32_t cnt[8] = {};
  uint64_t qlo[8] = {}, qhi[8] = {};
  constexpr int kBatch = 16;  // rows loaded before any is used
  for (int r0 = 0; r0 < kRowBlock; r0 += kBatch) {
    uint32_t v[kBatch];
#pragma unroll
    for (int r = 0; r < kBatch; ++r) v[r] = __ldg(col + (r0 + r) * row_words);
#pragma unroll
    for (int r = 0; r < kBatch; ++r) {
      if (v[r] == 0) continue;
      const uint4 rec = __ldg(P.rec + b * kRowBlock + r0 + r);
      const uint64_t Q = (uint64_t)rec.x | ((uint64_t)rec.y << 32);
#pragma unroll
      for (int n = 0; n < 8; ++n) {
        if ((v[r] >> (4 * n)) & 0xFu) {
          cnt[n] += 1;
          qlo[n] += Q;
          qhi[n] += qlo[n] < Q ? 1u : 0u;
        }
      }
    }
  }
  const int64_t o = b * P.k_cap + 8 * w;
#pragma unroll
  for (int n = 0; n < 8; ++n) {
    P.lin_cnt[o + n] = cnt[n];
    P.lin_q[o + n] = make_ulonglong2(qlo[n], qhi[n]);
  }
}

// (thread = one plane column of one set): U exclusive prefix of the counts, V
// exclusive suffix of the Q sums, over the set's blocks.
__global__ void __launch_bounds__(256) lin_scan_kernel(RankPtrs P) {
  if (P.hdr->status != 0) return;
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= P.hdr->k_pad) return;
  for (int64_t si = blockIdx.y; si < P.n_sets; si += gridDim.y) {
    const RankSet e = P.sets[si];
    const int64_t b0 = e.row_base / kRowBlock;
    const int64_t nb = ((e.n > 0 ? e.n : 1) + kNPad - 1) / kNPad * kNPad / kRowBlock;
    if (nb <= 1) continue;  // one block: every pair is in its diagonal tile
    // batches of kBatch blocks: all loads of a batch before its stores
    constexpr int kBatch = 16;
    uint32_t run = 0;
    for (int64_t bb = 0; bb < nb; bb += kBatch) {
      uint32_t c[kBatch];
#pragma unroll
      for (int i = 0; i < kBatch; ++i)
        c[i] = bb + i < nb ? P.lin_cnt[(b0 + bb + i) * P.k_cap + k] : 0u;
#pragma unroll
      for (int i = 0; i < kBatch; ++i) {
        if (bb + i < nb) P.lin_cnt[(b0 + bb + i) * P.k_cap + k] = run;
        run += c[i];
      }
    }
    uint64_t vlo = 0, vhi = 0;
    for (int64_t bb = 0; bb < nb; bb += kBatch) {  // blocks from the last one down
      ulonglong2 q[kBatch];
#pragma unroll
      for (int i = 0; i < kBatch; ++i)
        q[i] = bb + i < nb ? P.lin_q[(b0 + nb - 1 - bb - i) * P.k_cap + k] : make_ulonglong2(0, 0);
#pragma unroll
      for (int i = 0; i < kBatch; ++i) {
        if (bb + i < nb) P.lin_q[(b0 + nb - 1 - bb - i) * P.k_cap + k] = make_ulonglong2(vlo, vhi);
        vlo += q[i].x;
        vhi += q[i].y + (vlo < q[i].x ? 1u : 0u);
      }
    }
  }
}

// (warp = one stored row x in block b): key += sum_k P_xk V_k(b) + Q_x sum_k P_xk U_k(b)
__global__ void __launch_bounds__(256) lin_rows_kernel(RankPtrs P) {
  if (P.hdr->status != 0) return;
  const int lane = threadIdx.x & 31;
  const int64_t words = P.hdr->k_pad / 8;
  const int64_t row_words = P.k_cap / 8;
  for (int64_t x = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; x < P.n_pad;
       x += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int32_t orig = P.perm[x];
    if (orig < 0) continue;
    const int64_t b = x / kRowBlock;
    const RankSet e = P.sets[P.n_sets > 1 ? P.row_set[x] : 0];
    if (((e.n > 0 ? e.n : 1) + kNPad - 1) / kNPad * kNPad <= kRowBlock) continue;
    const uint32_t *row = reinterpret_cast<const uint32_t *>(P.planes) + x * row_words;
    const uint32_t *U = P.lin_cnt + b * P.k_cap;
    const ulonglong2 *V = P.lin_q + b * P.k_cap;
    uint64_t u = 0, s0 = 0, s1 = 0, s2 = 0;
    for (int64_t w0 = 4 * lane; w0 < words; w0 += 128) {
      // four words (32 columns) per lane: 16-byte load (rows are 16-byte aligned)
      const uint4 v4 = __ldg(reinterpret_cast<const uint4 *>(row + w0));
      const uint32_t vw[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        uint32_t v = vw[i];
        while (v) {
          const int n = (__ffs((int)v) - 1) >> 2;  // nibble holding the lowest set bit
          v &= ~(0xFu << (4 * n));
          const int64_t k = 8 * (w0 + i) + n;
          u += __ldg(U + k);
          const ulonglong2 q = __ldg(V + k);
          s0 += q.x & 0xFFFFFFull;
          s1 += (q.x >> 24) & 0xFFFFFFull;
          s2 += (q.x >> 48) | (q.y << 16);
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      u += __shfl_xor_sync(0xffffffffu, u, o);
      s0 += __shfl_xor_sync(0xffffffffu, s0, o);
      s1 += __shfl_xor_sync(0xffffffffu, s1, o);
      s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if (lane == 0) {
      const uint4 rec = P.rec[x];
      const uint64_t Q = (uint64_t)rec.x | ((uint64_t)rec.y << 32);
      const uint64_t lo = Q * u, hi = __umul64hi(Q, u);
      unsigned long long *dst = P.acc + 3 * (int64_t)orig;
      red_add_u64(dst + 0, s0 + (lo & 0xFFFFFFull));
      red_add_u64(dst + 1, s1 + ((lo >> 24) & 0xFFFFFFull));
      red_add_u64(dst + 2, s2 + ((lo >> 48) | (hi << 16)));
    }
  }
}

}  // namespace

int rank_linear_launch(const RankPtrs &P, cudaStream_t st) {
  const int64_t nblk = P.n_pad / kRowBlock;
  if (nblk <= 1 || P.k_cap <= 0) return SAD_OK;
  {
    const int64_t words = P.k_cap / 8;
    dim3 g((unsigned)((words + 255) / 256), (unsigned)nblk);
    lin_cols_kernel<<<g, 256, 0, st>>>(P);
    SAD_LAUNCH_CHECK();
  }
  {
    const int64_t sets = P.n_sets < 65535 ? P.n_sets : 65535;
    dim3 g((unsigned)((P.k_cap + 255) / 256), (unsigned)sets);
    lin_scan_kernel<<<g, 256, 0, st>>>(P);
    SAD_LAUNCH_CHECK();
  }
  {
    int64_t blocks = (P.n_pad * 32 + 255) / 256;
    const int64_t cap = (int64_t)num_sms() * 8;
    if (blocks > cap) blocks = cap;
    lin_rows_kernel<<<(unsigned)blocks, 256, 0, st>>>(P);
    SAD_LAUNCH_CHECK();
  }
  return SAD_OK;
}

}  // namespace sad
