// partition_noalloc: the regular-sampling partition for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code that runs inside a pool or
// arena that owns every device byte, plug-ins and embedders whose host
// application forbids allocation after start-up, or a hot path that must never
// hit the allocator's latency or failure modes. For them this entry point
// keeps its scratch in a fixed array in this library's device image, so the
// call needs nothing but the caller's inputs and outputs.
//
// The scratch array is file-scope device memory: every GPU that loads the
// library holds it (kNoAllocScratchBytes) until the process exits. Its size
// bounds the problem: N <= kNoAllocMaxN sequences and p <= kNoAllocMaxP
// buckets; larger calls are rejected with SAD_ERR_UNSUPPORTED before anything
// is launched.
//
// Host code cannot use the array's name as a device address (there it is only
// a host-side stand-in), so the first call on each device looks the address up
// with cudaGetSymbolAddress while that device is current and caches it. That
// first call should therefore come before any stream capture.
//
// Every call shares the one array and leaves its contents behind; nothing in it
// has to start at zero, because each call's kernels write every region before
// they read it (the partition records no status in the header). Calls whose GPU work
// overlaps (on different streams, or from different threads without ordering)
// race on the array: serialise them on one stream.
#include <mutex>

#include "sad_common.cuh"

namespace sad {

int partition_launch(const uint64_t *key_hi, const uint64_t *key_lo, int32_t n, int32_t p,
                     int32_t *bucket_offsets, int32_t *members, int32_t *pivot_idx, void *ws,
                     cudaStream_t st);

namespace {

constexpr int32_t kNoAllocMaxN = 32768;
constexpr int32_t kNoAllocMaxP = 64;
// The partition's workspace at the largest accepted (N, p): every region of the
// layout grows with N and p, so this holds every accepted call (about 2.1 MiB).
constexpr size_t kNoAllocScratchBytes = part_layout(kNoAllocMaxN, kNoAllocMaxP).bytes;
static_assert(kNoAllocScratchBytes <= ((size_t)3 << 20), "scratch stays modest");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (looked up once).
int noalloc_scratch(void **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return SAD_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return SAD_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> g(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return SAD_ERR_CUDA;
    }
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return SAD_OK;
}

}  // namespace
}  // namespace sad

using namespace sad;

extern "C" int partition_noalloc(const uint64_t *d_key_hi, const uint64_t *d_key_lo,
                                 int32_t n_seq, int32_t p, int32_t *d_bucket_offsets,
                                 int32_t *d_members, int32_t *d_pivot_idx, void *stream) {
  if (n_seq < 0 || p < 1) return SAD_ERR_INVALID_ARGUMENT;
  if (n_seq > 0 && p > n_seq) return SAD_ERR_INVALID_ARGUMENT;
  if (n_seq > kNoAllocMaxN || p > kNoAllocMaxP) return SAD_ERR_UNSUPPORTED;
  if (!d_bucket_offsets) return SAD_ERR_INVALID_ARGUMENT;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (n_seq == 0) {
    if (cudaMemsetAsync(d_bucket_offsets, 0, sizeof(int32_t) * (size_t)(p + 1), st) !=
        cudaSuccess) {
      cudaGetLastError();
      return SAD_ERR_CUDA;
    }
    return SAD_OK;
  }
  if (!d_key_hi || !d_key_lo || !d_members) return SAD_ERR_INVALID_ARGUMENT;
  void *scratch = nullptr;
  int rc = noalloc_scratch(&scratch);
  if (rc) return rc;
  // every region the partition kernels read is written by an earlier kernel of the
  // same call, so nothing needs clearing between calls
  return partition_launch(d_key_hi, d_key_lo, n_seq, p, d_bucket_offsets, d_members,
                          d_pivot_idx, scratch, st);
}
