// Distance-form k-mer rank (Eq. 2 and Eq. 3 as written): d(i, j) = -ln(Delta + F(i, j)),
// R_i = (1/N) sum_j d(i, j), with Delta = 1/b.
//
// With F = S / D, Delta + F = (D + b S) / (b D), so d = ln(b D) - ln(D + b S): a
// difference of natural logarithms of integers below (b + 1) 65536. Both are taken
// from one table of ln_q(x) = ln(x) 2^32 as a deterministic fixed-point value, so
// every per-pair value and every sum is an exact integer, the same on any device:
//
//   ln_q(x): x = 2^e m with m in [1, 2) held as a 64-bit mantissa; 40 fraction
//   bits of log2 m by repeated squaring (the square of m in [1, 2) lies in [1, 4):
//   when it reaches 2 the next bit is 1 and it is halved; Turner, "A fast binary
//   logarithm algorithm", IEEE Signal Processing Magazine, 2010, describes the
//   method); log2 x = e + fraction; ln_q = floor(log2 x 2^40 floor(ln 2 2^64) 2^-72).
//
// key_i = sum_j q_ij (signed 64-bit, j = i included), rank_i = key_i 2^-32 / N.
// The GEMM epilogue forms q_ij per pair (gemm.cu, distance mode).
#include "rank.cuh"

namespace sad {

namespace {

// floor(ln 2 * 2^64), from the decimal expansion ln 2 = 0.693147180559945309417...
constexpr uint64_t kLn2Q64 = 0xB17217F7D1CF79ABull;

__device__ __forceinline__ int64_t ln_q_dev(uint64_t x) {
  if (x == 0) return 0;
  const int e = 63 - __clzll((long long)x);
  uint64_t y = x << (63 - e);  // m = y / 2^63
  uint64_t f = 0;
  for (int i = 1; i <= 40; ++i) {
    const uint64_t lo = y * y, hi = __umul64hi(y, y);  // m^2 = (hi:lo) / 2^126
    if (hi >> 63) {               // m^2 >= 2: next bit 1, halve
      y = hi;
      f |= 1ull << (40 - i);
    } else {
      y = (hi << 1) | (lo >> 63);
    }
  }
  const uint64_t l2 = ((uint64_t)e << 40) | f;  // log2 x, 40 fraction bits
  return (int64_t)(__umul64hi(l2, kLn2Q64) >> 8);
}

__global__ void ln_table_kernel(int64_t *table, int64_t n) {
  pdl_enter();
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
       x += (int64_t)gridDim.x * blockDim.x)
    table[x] = ln_q_dev((uint64_t)x);
}

__global__ void ln_q_kernel(const uint64_t *x, int64_t n, int64_t *out) {
  pdl_enter();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = ln_q_dev(x[i]);
}

// key = acc0 as a signed 64-bit sum; the unsigned (hi, lo) view keeps the order
// (offset binary: hi = 0, lo = key xor 2^63); rank = key 2^-32 / N of the set.
__global__ void dist_finalize_kernel(RankPtrs P, int64_t *key, uint64_t *__restrict__ key_hi,
                                     uint64_t *__restrict__ key_lo, double *__restrict__ rank,
                                     int64_t n_div) {
  pdl_enter();
  if (P.hdr->status != 0) return;
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < P.n_total;
       x += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = (int64_t)P.acc[3 * x];
    if (key) key[x] = k;
    key_hi[x] = 0;
    key_lo[x] = (uint64_t)k ^ (1ull << 63);
    if (rank) {
      const double n = n_div > 0 ? (double)n_div : (double)P.sets[P.n_sets > 1 ? P.seq_set[x] : 0].n;
      rank[x] = __ddiv_rn(__dmul_rn(__ll2double_rn(k), 0x1p-32), n);
    }
  }
}

unsigned grid_of(int64_t work, int threads) {
  int64_t g = (work + threads - 1) / threads;
  const int64_t cap = (int64_t)num_sms() * 8;
  return (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
}

}  // namespace

size_t ln_table_entries(int32_t b) { return (size_t)(b + 1) * (size_t)kMaxM + 1; }

int ln_table_launch(int64_t *table, int32_t b, cudaStream_t st) {
  const int64_t n = (int64_t)ln_table_entries(b);
  pdl_launch(ln_table_kernel, grid_of(n, 256), 256, 0, st, table, n);
  SAD_LAUNCH_CHECK();
  return SAD_OK;
}

int ln_q_launch(const uint64_t *x, int64_t n, int64_t *out, cudaStream_t st) {
  if (n <= 0) return SAD_OK;
  pdl_launch(ln_q_kernel, grid_of(n, 256), 256, 0, st, x, n, out);
  SAD_LAUNCH_CHECK();
  return SAD_OK;
}

int rank_dist_finalize_launch(const RankPtrs &P, int64_t *key, uint64_t *key_hi,
                              uint64_t *key_lo, double *rank, int64_t n_div, cudaStream_t st) {
  pdl_launch(dist_finalize_kernel, grid_of(P.n_total, 256), 256, 0, st, P, key, key_hi, key_lo,
             rank, n_div);
  SAD_LAUNCH_CHECK();
  return SAD_OK;
}

}  // namespace sad
