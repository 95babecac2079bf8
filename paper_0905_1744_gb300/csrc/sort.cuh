// In-block sorting of (key, index) items, shared by the partition and the
// per-set length sort of batched rank calls.
//
// A bitonic network in shared memory sorts up to 4096 items; longer ranges sort
// 4096-item chunks that way and then merge runs of doubling width in global
// memory, each item finding its place by a binary search in the other run (all
// items differ, the index breaking ties).
#pragma once

#include "sad_common.cuh"

namespace sad {

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
__device__ inline void cta_sort_small(Item *data, int cnt, Item *sm) {
  int p2 = 1;
  while (p2 < cnt) p2 <<= 1;
  for (int i = threadIdx.x; i < p2; i += blockDim.x) sm[i] = i < cnt ? data[i] : item_inf();
  __syncthreads();
  for (int size = 2; size <= p2; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < (p2 >> 1); i += blockDim.x) {
        // pair i of the stage: i with a zero bit inserted at the stride's position
        const int a = ((i & ~(stride - 1)) << 1) | (i & (stride - 1));
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
__device__ inline void cta_sort(Item *data, Item *scratch, int64_t cnt, Item *sm) {
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

}  // namespace sad
