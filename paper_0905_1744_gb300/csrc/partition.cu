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
//
// Sorting inside one CTA: a bitonic network in shared memory for up to 4096
// items; longer ranges sort 4096-item chunks that way and then merge runs of
// doubling width in global memory, each item finding its place by a binary
// search in the other run (all items differ, the index breaking ties).
#include "sad_common.cuh"

namespace sad {

namespace {

constexpr int kSortThreads = 1024;
constexpr int kSmemItems = 4096;
constexpr size_t kSortSmem = sizeof(Item) * kSmemItems;

__device__ __forceinline__ Item item_inf() {
  Item x;
  x.hi = ~0ull;
  x.lo = ~0ull;
  x.idx = 0x7FFFFFFF;
  x.pad = 0;
  return x;
}

// Ascending bitonic sort of data[0, cnt), cnt <= kSmemItems, by the whole CTA.
__device__ void cta_sort_small(Item *data, int cnt, Item *sm) {
  int p2 = 1;
  while (p2 < cnt) p2 <<= 1;
  for (int i = threadIdx.x; i < p2; i += blockDim.x) sm[i] = i < cnt ? data[i] : item_inf();
  __syncthreads();
  for (int size = 2; size <= p2; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < (p2 >> 1); i += blockDim.x) {
        const int a = 2 * stride * (i / stride) + (i % stride);
        const int b = a + stride;
        const bool asc = (a & size) == 0;
        const Item x = sm[a], y = sm[b];
        if (asc ? item_less(y, x) : item_less(x, y)) {
          sm[a] = y;
          sm[b] = x;
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) data[i] = sm[i];
  __syncthreads();
}

// Number of items of run[0, len) that are less than x.
__device__ __forceinline__ int64_t count_less(const Item *run, int64_t len, const Item &x) {
  int64_t lo = 0, hi = len;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (item_less(run[mid], x)) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Number of items of run[0, len) that are not greater than x.
__device__ __forceinline__ int64_t count_not_greater(const Item *run, int64_t len, const Item &x) {
  int64_t lo = 0, hi = len;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (!item_less(x, run[mid])) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Ascending sort of data[0, cnt) by one CTA; scratch holds cnt items.
__device__ void cta_sort(Item *data, Item *scratch, int64_t cnt, Item *sm) {
  if (cnt <= 1) return;
  if (cnt <= kSmemItems) {
    cta_sort_small(data, (int)cnt, sm);
    return;
  }
  for (int64_t c0 = 0; c0 < cnt; c0 += kSmemItems)
    cta_sort_small(data + c0, (int)(cnt - c0 < kSmemItems ? cnt - c0 : kSmemItems), sm);
  Item *src = data, *dst = scratch;
  for (int64_t w = kSmemItems; w < cnt; w <<= 1) {
    for (int64_t i = threadIdx.x; i < cnt; i += blockDim.x) {
      const int64_t a0 = i / (2 * w) * (2 * w);
      const int64_t a1 = a0 + w < cnt ? a0 + w : cnt;
      const int64_t b1 = a0 + 2 * w < cnt ? a0 + 2 * w : cnt;
      const Item x = src[i];
      if (i < a1)
        dst[i + count_less(src + a1, b1 - a1, x)] = x;
      else
        dst[a0 + (i - a1) + count_less(src + a0, a1 - a0, x)] = x;
    }
    __syncthreads();
    Item *t = src;
    src = dst;
    dst = t;
  }
  if (src != data) {
    for (int64_t i = threadIdx.x; i < cnt; i += blockDim.x) data[i] = src[i];
    __syncthreads();
  }
}

__device__ __forceinline__ int64_t block_lo(int64_t b, int64_t n, int64_t p) { return b * n / p; }

__global__ void part_init_kernel(const uint64_t *__restrict__ hi, const uint64_t *__restrict__ lo,
                                 int64_t n, Item *items) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
       x += (int64_t)gridDim.x * blockDim.x) {
    Item it;
    it.hi = hi[x];
    it.lo = lo[x];
    it.idx = (int32_t)x;
    it.pad = 0;
    items[x] = it;
  }
}

// Segment s = [offs[s], offs[s+1]) if offs, else the floor block of s.
__global__ void __launch_bounds__(kSortThreads) seg_sort_kernel(Item *items, Item *scratch,
                                                                 int64_t n, int32_t p,
                                                                 const int32_t *offs) {
  extern __shared__ Item sm[];
  for (int32_t s = blockIdx.x; s < p; s += gridDim.x) {
    const int64_t lo = offs ? (int64_t)offs[s] : block_lo(s, n, p);
    const int64_t hi = offs ? (int64_t)offs[s + 1] : block_lo(s + 1, n, p);
    cta_sort(items + lo, scratch + lo, hi - lo, sm);
  }
}

__global__ void __launch_bounds__(kSortThreads) samples_kernel(const Item *items, Item *Y,
                                                                Item *Y2, Item *piv,
                                                                int32_t *pivot_idx, int64_t n,
                                                                int32_t p) {
  extern __shared__ Item sm[];
  const int64_t ns = (int64_t)p * (p - 1);
  for (int64_t e = threadIdx.x; e < ns; e += blockDim.x) {
    const int64_t b = e / (p - 1), j = e % (p - 1) + 1;
    const int64_t lo = block_lo(b, n, p), w = block_lo(b + 1, n, p) - lo;
    Y[e] = items[lo + j * w / p];
  }
  __syncthreads();
  cta_sort(Y, Y2, ns, sm);
  for (int64_t i = threadIdx.x; i < p - 1; i += blockDim.x) {
    const Item y = Y[i * p + p / 2 - 1];  // Y_{(i)p + floor(p/2)}, 1-based
    piv[i] = y;
    if (pivot_idx) pivot_idx[i] = y.idx;
  }
}

// pos[b][i] = items of sorted block b that are <= y_i (i < p-1); pos[b][p-1] = w_b.
__global__ void subblocks_kernel(const Item *items, const Item *piv, int32_t *pos, int64_t n,
                                 int32_t p) {
  const int64_t total = (int64_t)p * p;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = e / p, i = e % p;
    const int64_t lo = block_lo(b, n, p), w = block_lo(b + 1, n, p) - lo;
    pos[e] = (int32_t)(i == p - 1 ? w : count_not_greater(items + lo, w, piv[i]));
  }
}

__global__ void __launch_bounds__(1024) bucket_scan_kernel(const int32_t *pos, int32_t *dest,
                                                           int32_t *bucket_offsets, int32_t n,
                                                           int32_t p) {
  __shared__ int32_t s_warp[32];
  __shared__ int32_t s_carry;
  const int tid = threadIdx.x;
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
      bucket_offsets[i] = at;
      for (int b = 0; b < p; ++b) {
        dest[(int64_t)b * p + i] = at;
        at += pos[(int64_t)b * p + i] - (i > 0 ? pos[(int64_t)b * p + i - 1] : 0);
      }
    }
    __syncthreads();
    if (tid == blockDim.x - 1) s_carry = incl;
    __syncthreads();
  }
  if (tid == 0) bucket_offsets[p] = n;
}

__global__ void scatter_kernel(const Item *items, Item *out, const int32_t *pos,
                               const int32_t *dest, int64_t n, int32_t p) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
       x += (int64_t)gridDim.x * blockDim.x) {
    int64_t b = x * p / n;
    while (b + 1 < p && block_lo(b + 1, n, p) <= x) ++b;
    while (b > 0 && block_lo(b, n, p) > x) --b;
    const int64_t e = x - block_lo(b, n, p);
    const int32_t *pb = pos + b * p;
    int lo = 0, hi = p - 1;  // first i with e < pos[b][i]
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (e < pb[mid]) hi = mid; else lo = mid + 1;
    }
    const int64_t start = lo > 0 ? pb[lo - 1] : 0;
    out[dest[b * p + lo] + (e - start)] = items[x];
  }
}

__global__ void members_kernel(const Item *items, int32_t *members, int64_t n) {
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

int partition_launch(const uint64_t *key_hi, const uint64_t *key_lo, int32_t n, int32_t p,
                     int32_t *bucket_offsets, int32_t *members, int32_t *pivot_idx, void *ws,
                     cudaStream_t st) {
  const PartLayout L = part_layout(n, p);
  uint8_t *b = static_cast<uint8_t *>(ws);
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
  part_init_kernel<<<grid_for(n, 256), 256, 0, st>>>(key_hi, key_lo, n, items);
  SAD_LAUNCH_CHECK();
  seg_sort_kernel<<<(unsigned)p, kSortThreads, kSortSmem, st>>>(items, items2, n, p, nullptr);
  SAD_LAUNCH_CHECK();
  if (p > 1) {
    samples_kernel<<<1, kSortThreads, kSortSmem, st>>>(items, Y, Y2, piv, pivot_idx, n, p);
    SAD_LAUNCH_CHECK();
  }
  subblocks_kernel<<<grid_for((int64_t)p * p, 256), 256, 0, st>>>(items, piv, pos, n, p);
  SAD_LAUNCH_CHECK();
  bucket_scan_kernel<<<1, 1024, 0, st>>>(pos, dest, bucket_offsets, n, p);
  SAD_LAUNCH_CHECK();
  scatter_kernel<<<grid_for(n, 256), 256, 0, st>>>(items, items2, pos, dest, n, p);
  SAD_LAUNCH_CHECK();
  seg_sort_kernel<<<(unsigned)p, kSortThreads, kSortSmem, st>>>(items2, items, n, p,
                                                                  bucket_offsets);
  SAD_LAUNCH_CHECK();
  members_kernel<<<grid_for(n, 256), 256, 0, st>>>(items2, members, n);
  SAD_LAUNCH_CHECK();
  return SAD_OK;
}

}  // namespace sad
