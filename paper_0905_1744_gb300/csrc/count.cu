// k-mer count vectors (Sec. 3, "k-mer Rank"): c^X_tau = number of windows of X
// whose k letters spell word tau = sum_r a_r * alphabet^(k-1-r).
//
// One warp owns one sequence at a time. The warp reads the sequence 512 bytes
// per step as 16-byte vectors (lane l: bytes 16l..16l+15 of the step); the k-1
// bytes a lane's last windows run into come from the next lane by shuffle, and
// lane 31 loads them itself. Each window's word is counted in the warp's
// private shared-memory histogram (two 16-bit bins per 32-bit word), which is
// then streamed out as the dense int32 row and cleared in the same pass. If asked,
// the same pass keeps which words occurred (a bit each, in a bitmap private to the
// lane that writes the word: a lane always owns the same columns) and, per block,
// the largest count of the words seen twice or more (a byte each, counts above
// 255 going straight to global memory), and merges both into the per-word maximum
// over all sequences when the block is done.
#include "sad_common.cuh"

namespace sad {

namespace {

__device__ __forceinline__ uint4 load16_guarded(const uint8_t *codes, int64_t pos, int64_t end) {
  // 16 bytes at pos (16-aligned); bytes at or past `end` read as zero.
  if (pos + 16 <= end) return __ldg(reinterpret_cast<const uint4 *>(codes + pos));
  uint32_t w[4] = {0, 0, 0, 0};
  for (int b = 0; b < 16; ++b)
    if (pos + b < end) w[b >> 2] |= (uint32_t)__ldg(codes + pos + b) << (8 * (b & 3));
  return make_uint4(w[0], w[1], w[2], w[3]);
}

__device__ __forceinline__ uint32_t byte_of(const uint32_t (&w)[8], int b) {
  return (w[b >> 2] >> (8 * (b & 3))) & 0xFFu;
}

__device__ __forceinline__ uint32_t byte_of3(const uint32_t (&w)[3], int b) {
  return (w[b >> 2] >> (8 * (b & 3))) & 0xFFu;
}

// Word t has count c >= 2 in one sequence: raise its byte maximum (compare-and-swap
// on the containing word), counts above 255 go to the global maximum directly.
__device__ __forceinline__ void note_repeat(uint32_t *max8, int32_t *word_max, int t, int32_t c) {
  if (c < 2) return;
  if (c > 255) {
    atomicMax(word_max + t, c);
    return;
  }
  const uint32_t sh = 8u * (uint32_t)(t & 3);
  uint32_t old = max8[t >> 2];
  while ((int32_t)((old >> sh) & 0xFFu) < c) {
    const uint32_t upd = (old & ~(0xFFu << sh)) | ((uint32_t)c << sh);
    const uint32_t seen = atomicCAS(&max8[t >> 2], old, upd);
    if (seen == old) break;
    old = seen;
  }
}

// Words of one warp's presence bitmap: 32 lanes x one word per 4 passes of column
// octets (eps divisible by 8) or per 32 passes of single columns.
__host__ __device__ __forceinline__ int pres_words_of(int32_t eps) {
  if ((eps & 7) == 0) {
    const int passes = ((eps >> 3) + 31) / 32;
    return 32 * ((passes + 3) / 4);
  }
  const int passes = (eps + 31) / 32;
  return 32 * ((passes + 31) / 32);
}

template <int K>
__global__ void __launch_bounds__(128) kmer_count_kernel(const uint8_t *__restrict__ codes,
                                                        const int64_t *__restrict__ offsets,
                                                        int32_t n, int32_t alphabet, int32_t eps,
                                                        int32_t *__restrict__ counts,
                                                        int32_t *__restrict__ word_max,
                                                        WsHeader *hdr) {
  pdl_enter();
  extern __shared__ uint32_t smem[];
  const int warps = blockDim.x >> 5;
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int words = (eps + 1) >> 1;
  uint32_t *hist = smem + (size_t)wid * words;
  // word maxima: per warp a presence bitmap ([pass / 4][lane] words holding the 8
  // bits of the lane's column octet for 4 passes); per block byte maxima
  const int pres_words = pres_words_of(eps);
  uint32_t *present = smem + (size_t)warps * words + (size_t)wid * pres_words;
  uint32_t *max8 = smem + (size_t)warps * (words + pres_words);  // [ceil(eps / 4)]
  for (int i = lane; i < words; i += 32) hist[i] = 0;
  if (word_max) {
    for (int i = lane; i < pres_words; i += 32) present[i] = 0;
    for (int i = threadIdx.x; i < ((eps + 3) >> 2); i += blockDim.x) max8[i] = 0;
  }
  __syncthreads();
  const int64_t codes_end = offsets[n];
  const bool octets = (eps & 7) == 0 && (reinterpret_cast<uintptr_t>(counts) & 15) == 0;

  for (int64_t x = (int64_t)blockIdx.x * warps + wid; x < n; x += (int64_t)gridDim.x * warps) {
    const int64_t s = offsets[x], e = offsets[x + 1];
    if (s < 0 || e > codes_end || e < s) {
      // malformed offsets: nothing is read from codes
      if (lane == 0) record_error(hdr, SAD_ERR_INVALID_ARGUMENT, (int)x);
    } else if (e - s < K) {
      if (lane == 0) record_error(hdr, SAD_ERR_BAD_INPUT, (int)x);
    } else if (e - s - K + 1 > kMaxM) {
      // 16-bit bins: longer sequences are outside what the library handles.
      if (lane == 0) record_error(hdr, SAD_ERR_UNSUPPORTED, (int)x);
    } else {
      bool bad = false;
      for (int64_t c = s & ~(int64_t)15; c < e; c += 512) {
        const int64_t my = c + 16 * lane;
        uint4 v = my < e ? load16_guarded(codes, my, codes_end) : make_uint4(0, 0, 0, 0);
        uint4 nx;
        nx.x = __shfl_down_sync(0xffffffffu, v.x, 1);
        nx.y = __shfl_down_sync(0xffffffffu, v.y, 1);
        nx.z = __shfl_down_sync(0xffffffffu, v.z, 1);
        nx.w = __shfl_down_sync(0xffffffffu, v.w, 1);
        if (lane == 31 && K > 1)
          nx = (my + 16 < e) ? load16_guarded(codes, my + 16, codes_end) : make_uint4(0, 0, 0, 0);
        if (my >= e) continue;
        const uint32_t w[8] = {v.x, v.y, v.z, v.w, nx.x, nx.y, nx.z, nx.w};
        if (my >= s && my + 16 + K - 1 <= e) {
          // all 16 windows of the lane lie inside the sequence: no bounds checks
          if (alphabet < 256) {
            const uint32_t lim = 0x01010101u * (uint32_t)alphabet;
            bad |= (__vcmpgeu4(v.x, lim) | __vcmpgeu4(v.y, lim) | __vcmpgeu4(v.z, lim) |
                    __vcmpgeu4(v.w, lim)) != 0u;
          }
#pragma unroll
          for (int b = 0; b < 16; ++b) {
            uint32_t tau = 0;
#pragma unroll
            for (int r = 0; r < K; ++r) tau = tau * (uint32_t)alphabet + byte_of(w, b + r);
            if (tau < (uint32_t)eps) atomicAdd(&hist[tau >> 1], 1u << (16 * (tau & 1)));
          }
          continue;
        }
#pragma unroll
        for (int b = 0; b < 16; ++b) {
          const int64_t pos = my + b;
          if (pos >= s && pos < e && byte_of(w, b) >= (uint32_t)alphabet) bad = true;
          if (pos >= s && pos + K <= e) {
            uint32_t tau = 0;
#pragma unroll
            for (int r = 0; r < K; ++r) tau = tau * (uint32_t)alphabet + byte_of(w, b + r);
            if (tau < (uint32_t)eps) atomicAdd(&hist[tau >> 1], 1u << (16 * (tau & 1)));
          }
        }
      }
      if (__any_sync(0xffffffffu, bad) && lane == 0) record_error(hdr, SAD_ERR_BAD_INPUT, (int)x);
    }
    __syncwarp();
    int32_t *row = counts + x * (int64_t)eps;
    if (octets) {
      // lane writes octets of columns o = lane + 32 pass: one 16-byte shared load
      // (and clear) and two 16-byte stores of the row
      uint4 *h4 = reinterpret_cast<uint4 *>(hist);
      int4 *row4 = reinterpret_cast<int4 *>(row);
      int pass = 0;
      for (int o = lane; o < (eps >> 3); o += 32, ++pass) {
        const uint4 h = h4[o];
        h4[o] = make_uint4(0, 0, 0, 0);
        row4[2 * o] = make_int4((int)(h.x & 0xFFFFu), (int)(h.x >> 16), (int)(h.y & 0xFFFFu),
                                (int)(h.y >> 16));
        row4[2 * o + 1] = make_int4((int)(h.z & 0xFFFFu), (int)(h.z >> 16),
                                    (int)(h.w & 0xFFFFu), (int)(h.w >> 16));
        if (word_max) {
          const uint32_t any = h.x | h.y | h.z | h.w;
          if (any) {
            const uint32_t hw[4] = {h.x, h.y, h.z, h.w};
            uint32_t nz = 0;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const uint32_t m = __vcmpne2(hw[u], 0u);  // 0xFFFF per nonzero half
              nz |= ((m & 1u) | ((m >> 15) & 2u)) << (2 * u);
            }
            present[(pass >> 2) * 32 + lane] |= nz << (8 * (pass & 3));
            if (any & 0xFFFEFFFEu) {  // some count >= 2
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                note_repeat(max8, word_max, 8 * o + 2 * u, (int32_t)(hw[u] & 0xFFFFu));
                note_repeat(max8, word_max, 8 * o + 2 * u + 1, (int32_t)(hw[u] >> 16));
              }
            }
          }
        }
      }
    } else {
      int pass = 0;
      for (int t = lane; t < eps; t += 32, ++pass) {
        const int c = (int)((hist[t >> 1] >> (16 * (t & 1))) & 0xFFFFu);
        row[t] = c;
        if (word_max && c > 0) {
          present[(pass >> 5) * 32 + lane] |= 1u << (pass & 31);
          note_repeat(max8, word_max, t, c);
        }
      }
      __syncwarp();
      for (int i = lane; i < words; i += 32) hist[i] = 0;
    }
    __syncwarp();
  }
  if (word_max) {
    // blocks start at different words and skip words whose maximum already
    // covers theirs, so that the atomics do not queue on the same addresses
    __syncthreads();
    const int off = (int)(((int64_t)blockIdx.x * 1024) % eps);
    const uint32_t *pres0 = smem + (size_t)warps * words;
    for (int i = threadIdx.x; i < eps; i += blockDim.x) {
      const int t = i + off < eps ? i + off : i + off - eps;
      // the bit of word t: column octet o = t / 8 (or column t) is owned by lane
      // o % 32 in pass o / 32
      int idx, bit;
      if (octets) {
        const int o = t >> 3, pass = o >> 5;
        idx = (pass >> 2) * 32 + (o & 31);
        bit = 8 * (pass & 3) + (t & 7);
      } else {
        const int pass = t >> 5;
        idx = (pass >> 5) * 32 + (t & 31);
        bit = pass & 31;
      }
      uint32_t any = 0;
      for (int w = 0; w < warps; ++w) any |= pres0[(size_t)w * pres_words + idx];
      const int32_t m8 = (int32_t)((max8[t >> 2] >> (8 * (t & 3))) & 0xFFu);
      const int32_t v = m8 > 0 ? m8 : (int32_t)((any >> bit) & 1u);
      if (v && v > *(volatile int32_t *)(word_max + t)) atomicMax(word_max + t, v);
    }
  }
}

template <int K>
int launch_count_warp(const uint8_t *codes, const int64_t *offsets, int32_t n, int32_t alphabet,
                      int32_t eps, int32_t *counts, int32_t *word_max, WsHeader *hdr,
                      cudaStream_t st) {
  const size_t per_warp = sizeof(uint32_t) * (size_t)((eps + 1) / 2);
  int warps = (int)((96 * 1024) / per_warp);
  warps = warps < 1 ? 1 : (warps > 4 ? 4 : warps);
  const size_t max_bytes =
      word_max ? sizeof(uint32_t) * ((size_t)warps * pres_words_of(eps) + ((eps + 3) >> 2)) : 0;
  const size_t smem = per_warp * warps + max_bytes;
  if (word_max) {
    if (cudaMemsetAsync(word_max, 0, sizeof(int32_t) * (size_t)eps, st) != cudaSuccess)
      return SAD_ERR_CUDA;
  }
  if (smem > 227 * 1024) return SAD_ERR_UNSUPPORTED;
  auto kern = kmer_count_kernel<K>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return SAD_ERR_CUDA;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, warps * 32, smem) !=
      cudaSuccess)
    return SAD_ERR_CUDA;
  int64_t blocks = (int64_t)num_sms() * (per_sm > 0 ? per_sm : 1);
  const int64_t need = (n + warps - 1) / warps;
  if (blocks > need) blocks = need;
  if (blocks < 1) blocks = 1;
  pdl_launch(kern, (unsigned)blocks, warps * 32, smem, st, codes, offsets, n, alphabet, eps, counts,
             word_max, hdr);
  SAD_LAUNCH_CHECK();
  return SAD_OK;
}

// CTA per sequence (eps divisible by 8, eps <= 8 * kCtaThreads * 4, 16-byte aligned
// rows): the 8 warps share a shared histogram, double-buffered: while the CTA writes
// one sequence's row out of one buffer, the threads holding the next sequence's
// bytes count it into the other, so a sequence costs one barrier and its counting
// hides behind the previous row's stores. Thread t always writes the column quads
// o = t + kCtaThreads * pass (16 bytes each, so a warp store covers 512 contiguous
// bytes), and the words it has seen occur fit one 32-bit register (4 bits per
// pass); counts >= 2 go to per-CTA byte maxima as in the warp kernel.
constexpr int kCtaThreads = 256;

template <int K>
__device__ __forceinline__ bool cta_count_sequence(const uint8_t *__restrict__ codes,
                                                   int64_t codes_end, int64_t s, int64_t e,
                                                   int32_t alphabet, int32_t eps,
                                                   uint32_t *hist) {
  bool bad = false;
  // eight threads per 16-byte chunk, two windows each (a sequence of a few hundred
  // codes spreads over half of the CTA); the chunk and the k - 1 bytes past it come
  // from two 16-byte loads, shared through L1
  const int part = (int)(threadIdx.x & 7u);
  for (int64_t c = (s & ~(int64_t)15) + 16 * (threadIdx.x >> 3); c < e;
       c += 16 * (kCtaThreads / 8)) {
    const uint4 v = load16_guarded(codes, c, codes_end);
    const uint4 nx = (K > 1 && c + 16 < e) ? load16_guarded(codes, c + 16, codes_end)
                                           : make_uint4(0, 0, 0, 0);
    // bytes 2 part .. 2 part + 9 of the two loads: the words from 4 (part / 2) on,
    // shifted right by 2 (part & 1) bytes
    const int q = part >> 1;
    const uint32_t a0 = q == 0 ? v.x : q == 1 ? v.y : q == 2 ? v.z : v.w;
    const uint32_t a1 = q == 0 ? v.y : q == 1 ? v.z : q == 2 ? v.w : nx.x;
    const uint32_t a2 = q == 0 ? v.z : q == 1 ? v.w : q == 2 ? nx.x : nx.y;
    const uint32_t a3 = q == 0 ? v.w : q == 1 ? nx.x : q == 2 ? nx.y : nx.z;
    const uint32_t sh = 16u * (uint32_t)(part & 1);
    const uint32_t w[3] = {__funnelshift_r(a0, a1, sh), __funnelshift_r(a1, a2, sh),
                           __funnelshift_r(a2, a3, sh)};
    const int64_t c2 = c + 2 * part;
    if (c2 >= s && c2 + 2 + K - 1 <= e) {
      if (alphabet < 256)
        bad |= (__vcmpgeu4(w[0], 0x01010101u * (uint32_t)alphabet) & 0xFFFFu) != 0u;
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        uint32_t tau = 0;
#pragma unroll
        for (int r = 0; r < K; ++r) tau = tau * (uint32_t)alphabet + byte_of3(w, b + r);
        if (tau < (uint32_t)eps) atomicAdd(&hist[tau >> 1], 1u << (16 * (tau & 1)));
      }
    } else {
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        const int64_t pos = c2 + b;
        if (pos >= s && pos < e && byte_of3(w, b) >= (uint32_t)alphabet) bad = true;
        if (pos >= s && pos + K <= e) {
          uint32_t tau = 0;
#pragma unroll
          for (int r = 0; r < K; ++r) tau = tau * (uint32_t)alphabet + byte_of3(w, b + r);
          if (tau < (uint32_t)eps) atomicAdd(&hist[tau >> 1], 1u << (16 * (tau & 1)));
        }
      }
    }
  }
  return bad;
}

// Validates sequence x and counts it into hist; returns the thread's bad-code flag.
template <int K>
__device__ __forceinline__ bool cta_take_sequence(const uint8_t *__restrict__ codes,
                                                  const int64_t *__restrict__ offsets,
                                                  int64_t codes_end, int64_t x, int32_t alphabet,
                                                  int32_t eps, uint32_t *hist, WsHeader *hdr) {
  const int64_t s = offsets[x], e = offsets[x + 1];
  int err = 0;
  if (s < 0 || e > codes_end || e < s) err = SAD_ERR_INVALID_ARGUMENT;
  else if (e - s < K) err = SAD_ERR_BAD_INPUT;
  else if (e - s - K + 1 > kMaxM) err = SAD_ERR_UNSUPPORTED;
  if (err) {
    if (threadIdx.x == 0) record_error(hdr, err, (int)x);
    return false;
  }
  return cta_count_sequence<K>(codes, codes_end, s, e, alphabet, eps, hist);
}

template <int K>
__global__ void __launch_bounds__(kCtaThreads) kmer_count_cta_kernel(
    const uint8_t *__restrict__ codes, const int64_t *__restrict__ offsets, int32_t n,
    int32_t alphabet, int32_t eps, int32_t *__restrict__ counts, int32_t *__restrict__ word_max,
    WsHeader *hdr) {
  pdl_enter();
  extern __shared__ uint32_t smem[];
  uint32_t *histbuf = smem;                   // 2 x [eps / 2]
  uint32_t *max8 = smem + eps;                // [eps / 4]
  const int tid = threadIdx.x;
  for (int i = tid; i < eps; i += kCtaThreads) histbuf[i] = 0;
  if (word_max)
    for (int i = tid; i < (eps >> 2); i += kCtaThreads) max8[i] = 0;
  uint32_t present = 0;
  __syncthreads();
  const int64_t codes_end = offsets[n];
  const int quads = eps >> 2;  // at most 8 kCtaThreads: 4 presence bits a pass fit `present`
  int64_t x = blockIdx.x;
  if (x < n) {
    const bool bad = cta_take_sequence<K>(codes, offsets, codes_end, x, alphabet, eps, histbuf, hdr);
    if (__syncthreads_or(bad) && tid == 0) record_error(hdr, SAD_ERR_BAD_INPUT, (int)x);
  }
  for (int it = 0; x < n; ++it, x += gridDim.x) {
    uint32_t *cur = histbuf + (it & 1) * (eps >> 1);
    uint32_t *nxt = histbuf + ((it + 1) & 1) * (eps >> 1);
    const int64_t xn = x + gridDim.x;
    bool badn = false;
    if (xn < n) badn = cta_take_sequence<K>(codes, offsets, codes_end, xn, alphabet, eps, nxt, hdr);
    // the row of x: quad o = tid + kCtaThreads pass (4 counts), one 8-byte shared
    // load (and clear) and one 16-byte store, so a warp writes 512 contiguous bytes
    uint2 *h2 = reinterpret_cast<uint2 *>(cur);
    int4 *row4 = reinterpret_cast<int4 *>(counts + x * (int64_t)eps);
    int pass = 0;
    for (int o = tid; o < quads; o += kCtaThreads, ++pass) {
      const uint2 h = h2[o];
      h2[o] = make_uint2(0, 0);
      row4[o] = make_int4((int)(h.x & 0xFFFFu), (int)(h.x >> 16), (int)(h.y & 0xFFFFu),
                          (int)(h.y >> 16));
      if (word_max) {
        const uint32_t any = h.x | h.y;
        if (any) {
          const uint32_t m0 = __vcmpne2(h.x, 0u), m1 = __vcmpne2(h.y, 0u);
          const uint32_t nz = (m0 & 1u) | ((m0 >> 15) & 2u) | ((m1 & 1u) << 2) | ((m1 >> 13) & 8u);
          present |= nz << (4 * pass);
          if (any & 0xFFFEFFFEu) {
            note_repeat(max8, word_max, 4 * o + 0, (int32_t)(h.x & 0xFFFFu));
            note_repeat(max8, word_max, 4 * o + 1, (int32_t)(h.x >> 16));
            note_repeat(max8, word_max, 4 * o + 2, (int32_t)(h.y & 0xFFFFu));
            note_repeat(max8, word_max, 4 * o + 3, (int32_t)(h.y >> 16));
          }
        }
      }
    }
    // the next sequence is counted and this row's buffer is clear for the one after
    if (__syncthreads_or(badn) && tid == 0) record_error(hdr, SAD_ERR_BAD_INPUT, (int)xn);
  }
  if (word_max) {
    __syncthreads();
    int pass = 0;
    for (int o = tid; o < quads; o += kCtaThreads, ++pass) {
      for (int u = 0; u < 4; ++u) {
        const int t = 4 * o + u;
        const int32_t m8 = (int32_t)((max8[o] >> (8 * u)) & 0xFFu);
        const int32_t v = m8 > 0 ? m8 : (int32_t)((present >> (4 * pass + u)) & 1u);
        if (v && v > *(volatile int32_t *)(word_max + t)) atomicMax(word_max + t, v);
      }
    }
  }
}

template <int K>
int launch_count(const uint8_t *codes, const int64_t *offsets, int32_t n, int32_t alphabet,
                 int32_t eps, int32_t *counts, int32_t *word_max, WsHeader *hdr,
                 cudaStream_t st) {
  if ((eps & 7) == 0 && eps <= 8 * kCtaThreads * 4 &&
      (reinterpret_cast<uintptr_t>(counts) & 15) == 0) {
    const size_t smem = sizeof(uint32_t) * (size_t)(eps + (word_max ? (eps >> 2) : 0));
    if (word_max && cudaMemsetAsync(word_max, 0, sizeof(int32_t) * (size_t)eps, st) != cudaSuccess)
      return SAD_ERR_CUDA;
    auto kern = kmer_count_cta_kernel<K>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return SAD_ERR_CUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kCtaThreads, smem) !=
        cudaSuccess)
      return SAD_ERR_CUDA;
    int64_t blocks = (int64_t)num_sms() * (per_sm > 0 ? per_sm : 1);
    if (blocks > n) blocks = n;
    if (blocks < 1) blocks = 1;
    pdl_launch(kern, (unsigned)blocks, kCtaThreads, smem, st, codes, offsets, n, alphabet, eps,
               counts, word_max, hdr);
    SAD_LAUNCH_CHECK();
    return SAD_OK;
  }
  return launch_count_warp<K>(codes, offsets, n, alphabet, eps, counts, word_max, hdr, st);
}

}  // namespace

int count_launch(const uint8_t *codes, const int64_t *offsets, int32_t n, int32_t k,
                 int32_t alphabet, int32_t eps, int32_t *counts, int32_t *word_max,
                 WsHeader *hdr, cudaStream_t st) {
  switch (k) {
#define SAD_COUNT_CASE(KK) \
  case KK: return launch_count<KK>(codes, offsets, n, alphabet, eps, counts, word_max, hdr, st);
    SAD_COUNT_CASE(1) SAD_COUNT_CASE(2) SAD_COUNT_CASE(3) SAD_COUNT_CASE(4)
    SAD_COUNT_CASE(5) SAD_COUNT_CASE(6) SAD_COUNT_CASE(7) SAD_COUNT_CASE(8)
#undef SAD_COUNT_CASE
    default: return SAD_ERR_UNSUPPORTED;
  }
}

}  // namespace sad
