// C-ABI entry points of libsad (declared in include/sad.h): argument checks,
// workspace layout, launch sequencing, device status readback.
#include <atomic>
#include <cstring>
#include <mutex>
#include <vector>

#include "rank.cuh"

namespace sad {

int count_launch(const uint8_t *codes, const int64_t *offsets, int32_t n, int32_t k,
                 int32_t alphabet, int32_t eps, int32_t *counts, int32_t *word_max,
                 WsHeader *hdr, cudaStream_t st);
int partition_launch(const uint64_t *key_hi, const uint64_t *key_lo, int32_t n, int32_t p,
                     int32_t *bucket_offsets, int32_t *members, int32_t *pivot_idx, void *ws,
                     cudaStream_t st);
int partition_sets_launch(const uint64_t *key_hi, const uint64_t *key_lo, int32_t n_sets,
                          const int32_t *d_n, const int32_t *d_p, int32_t n_single,
                          int32_t p_single, const PartTotals &tot, int32_t max_p,
                          int32_t *bucket_offsets, int32_t *members, int32_t *pivot_idx,
                          void *ws, cudaStream_t st);

namespace {
std::atomic<uint64_t> g_launches{0};

int64_t eps_of(int32_t k, int32_t alphabet) {
  if (k < 1 || k > 8 || alphabet < 2 || alphabet > 256) return -1;
  int64_t e = 1;
  for (int i = 0; i < k; ++i) {
    e *= alphabet;
    if (e > kMaxEps) return -1;
  }
  return e;
}

bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

RankCaps planes_only(int64_t k_cap) { return RankCaps{0, 0, kRowBlock, k_cap, 0, 0, 0, 0}; }

// GEMM tile rows of a plan: 0 means 128 (one CTA a tile); 256 runs CTA pairs.
int32_t tile_of(const sad_rank_plan *plan) { return plan->tile == 2 * kRowBlock ? 2 * kRowBlock : kRowBlock; }

RankCaps caps_of(const sad_rank_plan *plan) {
  return RankCaps{plan->depth, plan->budget, tile_of(plan), plan->k_cap, plan->list_cap,
                  plan->rem_cap, plan->heavy_cap, plan->bm_cols};
}

// Largest K_cap (multiple of kKCols) whose planes-only rank layout fits in ws_bytes.
int64_t k_cap_for(const RankShape &sh, int64_t eps, size_t ws_bytes) {
  const RankLayout base = rank_layout(sh, eps, planes_only(0));
  if (ws_bytes <= base.fixed_bytes) return 0;
  // upper bound (the layout only grows with K_cap), then step down until it fits
  // (two plane columns per byte)
  int64_t k = (int64_t)(2 * ((ws_bytes - base.fixed_bytes) / (size_t)sh.rows_total));
  k = k / kKCols * kKCols;
  while (k > 0 && rank_layout(sh, eps, planes_only(k)).bytes > ws_bytes) k -= kKCols;
  return k;
}

int check_cuda(cudaError_t e) {
  if (e == cudaSuccess) return SAD_OK;
  cudaGetLastError();
  return SAD_ERR_CUDA;
}
}  // namespace

void note_launch(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }

namespace {
constexpr uint64_t kDefaultWaitNs = 2000000000ull;
std::atomic<uint64_t> g_wait_ns{kDefaultWaitNs};
}  // namespace

uint64_t gemm_wait_ns() { return g_wait_ns.load(std::memory_order_relaxed); }

namespace {
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<cudaEvent_t> g_prof_pool;                       // reusable events
std::vector<std::pair<cudaEvent_t, cudaEvent_t>> g_prof_open;  // recorded pairs
cudaEvent_t g_prof_pending = nullptr;

cudaEvent_t prof_event() {
  if (!g_prof_pool.empty()) {
    cudaEvent_t e = g_prof_pool.back();
    g_prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}
}  // namespace

void prof_begin(cudaStream_t st) {
  std::lock_guard<std::mutex> g(g_prof_mu);
  if (!g_prof_on) return;
  g_prof_pending = prof_event();
  if (g_prof_pending) cudaEventRecord(g_prof_pending, st);
}

void prof_end(cudaStream_t st) {
  std::lock_guard<std::mutex> g(g_prof_mu);
  if (!g_prof_on || !g_prof_pending) return;
  cudaEvent_t e = prof_event();
  if (!e) return;
  cudaEventRecord(e, st);
  g_prof_open.emplace_back(g_prof_pending, e);
  g_prof_pending = nullptr;
}

int num_sms() {
  static int cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (dev < 0 || dev >= 64) dev = 0;
  if (cached[dev] == 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1)
      v = 1;
    cached[dev] = v;
  }
  return cached[dev];
}

}  // namespace sad

using namespace sad;

extern "C" {

int sad_debug_wait_budget_ns(uint64_t ns) {
  g_wait_ns.store(ns == 0 ? kDefaultWaitNs : ns, std::memory_order_relaxed);
  return SAD_OK;
}

const char *sad_status_string(int status) {
  switch (status) {
    case SAD_OK: return "ok";
    case SAD_ERR_INVALID_ARGUMENT: return "invalid argument";
    case SAD_ERR_WORKSPACE: return "workspace too small for the data";
    case SAD_ERR_CUDA: return "CUDA runtime error";
    case SAD_ERR_TIMEOUT: return "bounded device wait timed out";
    case SAD_ERR_UNSUPPORTED: return "unsupported parameters";
    case SAD_ERR_BAD_INPUT: return "bad input data (letter code >= alphabet, length < k, or "
                                   "counts inconsistent with lengths)";
    default: return "unknown status";
  }
}

int sad_abi_version(void) { return SAD_ABI_VERSION; }

uint64_t sad_launch_count(void) { return g_launches.load(); }

size_t sad_workspace_bytes(int32_t op, int32_t n_seq, int32_t k, int32_t alphabet, int32_t p,
                           int32_t depth) {
  if (n_seq < 0) return 0;
  const int64_t eps = eps_of(k, alphabet);
  switch (op) {
    case SAD_OP_COUNT:
      return eps < 0 ? 0 : sizeof(WsHeader);
    case SAD_OP_RANK: {
      if (eps < 0) return 0;
      const RankShape sh = shape_single(n_seq);
      if (depth <= 0) return rank_layout(sh, eps, planes_only(0)).fixed_bytes;
      const int64_t k_cap =
          (int64_t)align_up((size_t)eps * (size_t)depth, (size_t)kKCols);
      return rank_layout(sh, eps, planes_only(k_cap)).bytes;
    }
    case SAD_OP_PARTITION:
      if (p < 1 || p > kMaxP) return 0;
      return part_layout(n_seq, p).bytes;
    default:
      return 0;
  }
}

int kmer_count(const uint8_t *d_codes, const int64_t *d_offsets, int32_t n_seq, int32_t k,
               int32_t alphabet, int32_t *d_counts, int32_t *d_word_max, void *d_ws,
               size_t ws_bytes, void *stream) {
  const int64_t eps = eps_of(k, alphabet);
  if (n_seq < 0 || eps < 0) return eps < 0 && n_seq >= 0 ? SAD_ERR_UNSUPPORTED
                                                           : SAD_ERR_INVALID_ARGUMENT;
  if (!d_ws || !aligned(d_ws, 256) || ws_bytes < sizeof(WsHeader)) return SAD_ERR_INVALID_ARGUMENT;
  if (n_seq == 0) return SAD_OK;
  if (!d_codes || !d_offsets || !d_counts || !aligned(d_counts, 16) || !aligned(d_offsets, 8))
    return SAD_ERR_INVALID_ARGUMENT;
  return count_launch(d_codes, d_offsets, n_seq, k, alphabet, (int32_t)eps, d_counts,
                      d_word_max, static_cast<WsHeader *>(d_ws),
                      static_cast<cudaStream_t>(stream));
}

}  // extern "C"

namespace {

// Plan for `sh` (one set, or a batch with per-set sizes d_n on the device).
int rank_plan_impl(const int32_t *d_counts, const RankShape &sh, const int32_t *d_n,
                   int64_t eps, int32_t k, sad_rank_plan *plan, void *d_ws, size_t ws_bytes,
                   cudaStream_t st) {
  RankCaps c0 = planes_only(0);
  c0.depth = plan->depth;
  const RankLayout L0 = rank_layout(sh, eps, c0);
  if (ws_bytes < L0.fixed_bytes) {
    plan->ws_bytes = L0.fixed_bytes;
    return SAD_ERR_WORKSPACE;
  }
  WsHeader h{};
  if (sh.n_total > 0) {
    if (!d_counts) return SAD_ERR_INVALID_ARGUMENT;
    const RankPtrs P = rank_ptrs(d_ws, L0);
    int rc = rank_prep_launch(P, d_counts, nullptr, d_n, nullptr, k, (int32_t)eps, 1, st);
    if (rc) return rc;
    rc = check_cuda(cudaMemcpyAsync(&h, d_ws, sizeof(h), cudaMemcpyDeviceToHost, st));
    if (rc) return rc;
    rc = check_cuda(cudaStreamSynchronize(st));
    if (rc) return rc;
    if (h.status != 0) return h.status;
  }
  int64_t k_pad = (int64_t)align_up((size_t)h.k_eff, kKCols);
  if (k_pad < kKCols) k_pad = kKCols;
  const bool rem = plan->depth >= 1 && sh.n_total > 0;
  plan->t_max = h.t_max;
  plan->t_bits = h.t_bits;
  plan->k_eff = h.k_eff;
  plan->list_entries = h.list_total;
  plan->rem_bound = h.rem_bound;
  plan->heavy_entries = h.heavy_total;
  plan->k_cap = k_pad;
  plan->list_cap = rem ? h.list_total : 0;
  plan->rem_cap = rem ? h.rem_bound : 0;
  plan->heavy_cap = rem ? h.heavy_total : 0;
  plan->bm_cols = rem ? h.bm_cols : 0;
  plan->ws_bytes = rank_layout(sh, eps, caps_of(plan)).bytes;
  return SAD_OK;
}

bool plan_valid(const sad_rank_plan *plan) {
  return plan->depth >= 0 && plan->budget >= 0 &&
         (plan->tile == 0 || plan->tile == kRowBlock || plan->tile == 2 * kRowBlock) &&
         plan->k_cap >= kKCols &&
         plan->k_cap % kKCols == 0 && plan->list_cap >= 0 && plan->rem_cap >= 0 &&
         plan->heavy_cap >= 0 && plan->bm_cols >= 0;
}

int rank_run_impl(const int32_t *d_counts, const int32_t *d_lengths, const int32_t *word_max,
                  const RankShape &sh, const int32_t *d_n, int64_t eps, int32_t k,
                  const sad_rank_plan *plan,
                  uint64_t *d_key_hi, uint64_t *d_key_lo, double *d_rank, void *d_ws,
                  size_t ws_bytes, cudaStream_t st) {
  if (sh.rows_total / kRowBlock > kMaxRowBlocks) return SAD_ERR_UNSUPPORTED;  // packed tile ids
  RankCaps caps = planes_only(0);
  if (plan) {
    if (!plan_valid(plan)) return SAD_ERR_INVALID_ARGUMENT;
    caps = caps_of(plan);
    if (rank_layout(sh, eps, caps).bytes > ws_bytes) return SAD_ERR_WORKSPACE;
  } else {
    caps.k_cap = k_cap_for(sh, eps, ws_bytes);
    if (caps.k_cap < kKCols) return SAD_ERR_WORKSPACE;
  }
  const RankLayout L = rank_layout(sh, eps, caps);
  RankPtrs P = rank_ptrs(d_ws, L);
  P.eps = (int32_t)eps;
  P.counts = d_counts;
  int rc = rank_prep_launch(P, d_counts, d_lengths, d_n, word_max, k, (int32_t)eps, 0, st);
  if (rc) return rc;
  rc = rank_gemm_launch(P, st);
  if (rc) return rc;
  return rank_finalize_launch(P, d_key_hi, d_key_lo, d_rank, st);
}

// Host-side shape of a batch; validates the per-set sizes.
int batch_shape(const int32_t *h_n, const int32_t *h_p, int32_t n_sets, int64_t tile,
                RankShape *sh, PartTotals *pt, int32_t *max_p) {
  if (n_sets < 1 || !h_n) return SAD_ERR_INVALID_ARGUMENT;
  *sh = RankShape{0, 0, 0, 0, 0};
  *pt = PartTotals{0, 0, 0, 0, 0};
  *max_p = 1;
  for (int32_t s = 0; s < n_sets; ++s) {
    if (h_n[s] < 1) return SAD_ERR_INVALID_ARGUMENT;
    shape_add_set(*sh, h_n[s], tile);
    if (h_p) {
      const int64_t p = h_p[s];
      if (p < 1 || p > kMaxP || p > h_n[s]) return SAD_ERR_INVALID_ARGUMENT;
      pt->n += h_n[s];
      pt->p += p;
      pt->p1 += p - 1;
      pt->pp1 += p * (p - 1);
      pt->pp += p * p;
      if (p > *max_p) *max_p = (int32_t)p;
    }
  }
  if (sh->n_total > 0x7FFFFFFF) return SAD_ERR_UNSUPPORTED;
  return SAD_OK;
}

// Capacities of a plan from host-side bounds alone (no look at the counts): shape
// sh, total_len residues in all its sequences. Section 3.1.2's counts give
// K_eff = sum over words of min(T, d) <= eps d; every remainder entry, heavy entry
// and bitmap column belongs to a k-mer window (total_len - n (k - 1) of them).
int plan_bound_caps(const RankShape &sh, int64_t total_len, int32_t k, int64_t eps,
                    sad_rank_plan *plan) {
  if (sh.rows_total / kRowBlock > kMaxRowBlocks) return SAD_ERR_UNSUPPORTED;
  const int64_t d = plan->depth < kMaxPlaneDepth ? plan->depth : kMaxPlaneDepth;
  const int64_t tb = t_bits_of((int32_t)d);
  int64_t k_cap = (int64_t)align_up((size_t)(eps * d), kKCols);
  if (k_cap < kKCols) k_cap = kKCols;
  const int64_t n_seq = sh.n_total;
  const int64_t windows = total_len - n_seq * (k - 1);
  int64_t bm = 0;
  for (int64_t t = 2; t <= tb && windows > 0; ++t) bm += windows / t < eps ? windows / t : eps;
  plan->t_max = -1;
  plan->t_bits = -1;
  plan->k_eff = -1;
  plan->list_entries = -1;
  plan->rem_bound = -1;
  plan->heavy_entries = -1;
  plan->k_cap = k_cap;
  plan->list_cap = windows > 0 ? windows / 2 : 0;
  plan->rem_cap = windows > n_seq ? windows - n_seq : 0;
  plan->heavy_cap = windows > 0 ? windows / (tb + 1) : 0;
  plan->bm_cols = bm;
  plan->ws_bytes = rank_layout(sh, eps, caps_of(plan)).bytes;
  return SAD_OK;
}

}  // namespace

extern "C" {

int kmer_rank_plan(const int32_t *d_counts, int32_t n_seq, int32_t k, int32_t alphabet,
                   sad_rank_plan *plan, void *d_ws, size_t ws_bytes, void *stream) {
  const int64_t eps = eps_of(k, alphabet);
  if (eps < 0) return SAD_ERR_UNSUPPORTED;
  if (n_seq < 0 || !plan || !d_ws || !aligned(d_ws, 256) || plan->depth < 0 ||
      !(plan->tile == 0 || plan->tile == kRowBlock || plan->tile == 2 * kRowBlock))
    return SAD_ERR_INVALID_ARGUMENT;
  return rank_plan_impl(d_counts, shape_single(n_seq, tile_of(plan)), nullptr, eps, k, plan,
                        d_ws, ws_bytes, static_cast<cudaStream_t>(stream));
}

int kmer_rank_plan_bound(int32_t n_seq, int64_t total_len, int32_t k, int32_t alphabet,
                         sad_rank_plan *plan) {
  const int64_t eps = eps_of(k, alphabet);
  if (eps < 0) return SAD_ERR_UNSUPPORTED;
  if (n_seq < 0 || total_len < 0 || !plan || plan->depth < 1 ||
      !(plan->tile == 0 || plan->tile == kRowBlock || plan->tile == 2 * kRowBlock))
    return SAD_ERR_INVALID_ARGUMENT;
  return plan_bound_caps(shape_single(n_seq, tile_of(plan)), total_len, k, eps, plan);
}

int kmer_rank(const int32_t *d_counts, const int32_t *d_lengths, const int32_t *d_word_max,
              int32_t n_seq, int32_t k, int32_t alphabet, const sad_rank_plan *plan,
              uint64_t *d_key_hi, uint64_t *d_key_lo, double *d_rank, void *d_ws,
              size_t ws_bytes, void *stream) {
  const int64_t eps = eps_of(k, alphabet);
  if (eps < 0) return SAD_ERR_UNSUPPORTED;
  if (n_seq < 0 || !d_ws || !aligned(d_ws, 256)) return SAD_ERR_INVALID_ARGUMENT;
  if (n_seq == 0) return SAD_OK;
  if (!d_counts || !d_lengths || !d_key_hi || !d_key_lo) return SAD_ERR_INVALID_ARGUMENT;
  return rank_run_impl(d_counts, d_lengths, d_word_max,
                       shape_single(n_seq, plan ? tile_of(plan) : kRowBlock), nullptr, eps, k,
                       plan,
                       d_key_hi, d_key_lo, d_rank, d_ws, ws_bytes,
                       static_cast<cudaStream_t>(stream));
}

size_t sad_local_samples_workspace_bytes(int32_t n_seq, int32_t p) {
  if (n_seq < 1 || p < 1 || p > n_seq) return 0;
  return local_samples_ws_bytes(n_seq, p);
}

int sad_local_samples(const uint64_t *d_key_hi, const uint64_t *d_key_lo, int32_t n_seq,
                      int32_t p, int32_t ks, int32_t *d_sample_idx, void *d_ws,
                      size_t ws_bytes, void *stream) {
  if (n_seq < 1 || p < 1 || p > n_seq || ks < 1 || (int64_t)ks * p > 0x7FFFFFFF)
    return SAD_ERR_INVALID_ARGUMENT;
  if (!d_key_hi || !d_key_lo || !d_sample_idx || !d_ws || !aligned(d_ws, 256))
    return SAD_ERR_INVALID_ARGUMENT;
  return local_samples_launch(d_key_hi, d_key_lo, n_seq, p, ks, d_sample_idx, d_ws, ws_bytes,
                              static_cast<cudaStream_t>(stream));
}

size_t kmer_rank_vs_workspace_bytes(const sad_rank_plan *plan, int32_t n_seq, int32_t k,
                                    int32_t alphabet, int32_t n_ref, int32_t delta_den) {
  const int64_t eps = eps_of(k, alphabet);
  if (eps < 0 || !plan || n_seq < 1 || n_ref < 1 || plan->k_cap < kKCols || delta_den < 0 ||
      delta_den > 1024)
    return 0;
  return rank_vs_ws_bytes(n_seq, eps, plan->k_cap, n_ref, delta_den);
}

int kmer_rank_vs(const int32_t *d_counts, const int32_t *d_lengths, const int32_t *d_word_max,
                 int32_t n_seq, int32_t k, int32_t alphabet, const int32_t *d_ref,
                 int32_t n_ref, int32_t delta_den, const sad_rank_plan *plan, int64_t *d_key,
                 uint64_t *d_key_hi, uint64_t *d_key_lo, double *d_rank, void *d_ws,
                 size_t ws_bytes, void *stream) {
  const int64_t eps = eps_of(k, alphabet);
  if (eps < 0) return SAD_ERR_UNSUPPORTED;
  if (n_seq < 1 || n_ref < 1 || !plan || !d_counts || !d_lengths || !d_ref || !d_key_hi ||
      !d_key_lo || !d_ws || !aligned(d_ws, 256) || delta_den < 0 || delta_den > 1024)
    return SAD_ERR_INVALID_ARGUMENT;
  if (plan->depth != 0 || plan->k_cap < kKCols || plan->k_cap % kKCols != 0)
    return SAD_ERR_INVALID_ARGUMENT;
  return rank_vs_launch(d_counts, d_lengths, d_word_max, n_seq, k, eps, d_ref, n_ref,
                        plan->k_cap, delta_den, d_key, d_key_hi, d_key_lo, d_rank, d_ws,
                        ws_bytes, static_cast<cudaStream_t>(stream));
}

size_t kmer_rank_dist_workspace_bytes(const sad_rank_plan *plan, int32_t n_seq, int32_t k,
                                      int32_t alphabet, int32_t delta_den) {
  const int64_t eps = eps_of(k, alphabet);
  if (eps < 0 || !plan || n_seq < 1 || delta_den < 1 || delta_den > 1024) return 0;
  const size_t base = rank_layout(shape_single(n_seq), eps, caps_of(plan)).bytes;
  return align_up(base, 256) + sizeof(int64_t) * ln_table_entries(delta_den);
}

int kmer_rank_dist(const int32_t *d_counts, const int32_t *d_lengths, const int32_t *d_word_max,
                   int32_t n_seq, int32_t k, int32_t alphabet, int32_t delta_den,
                   const sad_rank_plan *plan, int64_t *d_key, uint64_t *d_key_hi,
                   uint64_t *d_key_lo, double *d_rank, void *d_ws, size_t ws_bytes,
                   void *stream) {
  const int64_t eps = eps_of(k, alphabet);
  if (eps < 0) return SAD_ERR_UNSUPPORTED;
  if (n_seq < 1 || !plan || !d_counts || !d_lengths || !d_key_hi || !d_key_lo || !d_ws ||
      !aligned(d_ws, 256) || delta_den < 1 || delta_den > 1024)
    return SAD_ERR_INVALID_ARGUMENT;
  // the distance form runs one CTA per tile
  if (!plan_valid(plan) || tile_of(plan) != kRowBlock) return SAD_ERR_INVALID_ARGUMENT;
  const RankShape sh = shape_single(n_seq);
  if (sh.rows_total / kRowBlock > kMaxRowBlocks) return SAD_ERR_UNSUPPORTED;
  const RankLayout L = rank_layout(sh, eps, caps_of(plan));
  const size_t table_off = align_up(L.bytes, 256);
  if (table_off + sizeof(int64_t) * ln_table_entries(delta_den) > ws_bytes)
    return SAD_ERR_WORKSPACE;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  int64_t *table = reinterpret_cast<int64_t *>(static_cast<uint8_t *>(d_ws) + table_off);
  RankPtrs P = rank_ptrs(d_ws, L);
  P.eps = (int32_t)eps;
  P.counts = d_counts;
  int rc = ln_table_launch(table, delta_den, st);
  if (rc) return rc;
  rc = rank_prep_launch(P, d_counts, d_lengths, nullptr, d_word_max, k, (int32_t)eps, 0, st);
  if (rc) return rc;
  rc = rank_dist_gemm_launch(P, table, delta_den, st);
  if (rc) return rc;
  return rank_dist_finalize_launch(P, d_key, d_key_hi, d_key_lo, d_rank, 0, st);
}

size_t kmer_rank_sparse_workspace_bytes(int32_t n_seq, int64_t entries_cap) {
  if (n_seq < 1 || entries_cap < 0) return 0;
  return sparse_ws_bytes(n_seq, entries_cap);
}

int kmer_rank_sparse_entries(const int32_t *d_counts, const int32_t *d_lengths, int32_t n_seq,
                             int32_t k, int32_t alphabet, int64_t *entries, void *d_ws,
                             size_t ws_bytes, void *stream) {
  const int64_t eps = eps_of(k, alphabet);
  if (eps < 0) return SAD_ERR_UNSUPPORTED;
  if (n_seq < 1 || !d_counts || !d_lengths || !entries || !d_ws || !aligned(d_ws, 256))
    return SAD_ERR_INVALID_ARGUMENT;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  int rc = sparse_count_launch(d_counts, d_lengths, n_seq, k, (int32_t)eps, d_ws, ws_bytes, st);
  if (rc) return rc;
  WsHeader h;
  rc = check_cuda(cudaMemcpyAsync(&h, d_ws, sizeof(h), cudaMemcpyDeviceToHost, st));
  if (rc) return rc;
  rc = check_cuda(cudaStreamSynchronize(st));
  if (rc) return rc;
  if (h.status != 0) return h.status;
  *entries = h.list_total;
  return SAD_OK;
}

int kmer_rank_sparse(const int32_t *d_counts, const int32_t *d_lengths, int32_t n_seq,
                     int32_t k, int32_t alphabet, int64_t entries_cap, uint64_t *d_key_hi,
                     uint64_t *d_key_lo, double *d_rank, void *d_ws, size_t ws_bytes,
                     void *stream) {
  const int64_t eps = eps_of(k, alphabet);
  if (eps < 0) return SAD_ERR_UNSUPPORTED;
  if (n_seq < 1 || entries_cap < 0 || !d_counts || !d_lengths || !d_key_hi || !d_key_lo ||
      !d_ws || !aligned(d_ws, 256))
    return SAD_ERR_INVALID_ARGUMENT;
  return sparse_rank_launch(d_counts, d_lengths, n_seq, k, (int32_t)eps, entries_cap, d_key_hi,
                            d_key_lo, d_rank, d_ws, ws_bytes, static_cast<cudaStream_t>(stream));
}

int sad_ln_q(const uint64_t *d_x, int64_t n, int64_t *d_out, void *stream) {
  if (n < 0 || (n > 0 && (!d_x || !d_out))) return SAD_ERR_INVALID_ARGUMENT;
  return ln_q_launch(d_x, n, d_out, static_cast<cudaStream_t>(stream));
}

}  // extern "C"

namespace {

// The host-known part of a batch plan (set totals, partition sizes) from the
// per-set sizes; the shape for its rank.
int batch_plan_shape(const int32_t *h_n, const int32_t *h_p, int32_t n_sets,
                     sad_batch_plan *plan, RankShape *sh) {
  PartTotals pt;
  int32_t max_p;
  int rc = batch_shape(h_n, h_p, n_sets, tile_of(&plan->rank), sh, &pt, &max_p);
  if (rc) return rc;
  plan->n_sets = n_sets;
  plan->max_p = max_p;
  plan->n_total = sh->n_total;
  plan->rows_total = sh->rows_total;
  plan->tiles_total = sh->tiles_total;
  plan->tileof_total = sh->tileof_total;
  plan->sum_p = pt.p;
  plan->sum_p1 = pt.p1;
  plan->sum_pp1 = pt.pp1;
  plan->sum_pp = pt.pp;
  plan->part_ws_bytes = part_layout_sets(n_sets, pt).bytes;
  return SAD_OK;
}

bool tile_valid(const sad_rank_plan *plan) {
  return plan->tile == 0 || plan->tile == kRowBlock || plan->tile == 2 * kRowBlock;
}

}  // namespace

extern "C" {

int sad_batch_plan_make(const int32_t *d_counts, const int32_t *h_n, const int32_t *h_p,
                        const int32_t *d_n, int32_t n_sets, int32_t k, int32_t alphabet,
                        sad_batch_plan *plan, void *d_ws, size_t ws_bytes, void *stream) {
  const int64_t eps = eps_of(k, alphabet);
  if (eps < 0) return SAD_ERR_UNSUPPORTED;
  if (!plan || !h_p || !d_n || !d_ws || !aligned(d_ws, 256) || plan->rank.depth < 0 ||
      !tile_valid(&plan->rank))
    return SAD_ERR_INVALID_ARGUMENT;
  RankShape sh;
  int rc = batch_plan_shape(h_n, h_p, n_sets, plan, &sh);
  if (rc) return rc;
  return rank_plan_impl(d_counts, sh, d_n, eps, k, &plan->rank, d_ws, ws_bytes,
                        static_cast<cudaStream_t>(stream));
}

int sad_batch_plan_bound(const int32_t *h_n, const int32_t *h_p, int32_t n_sets,
                         int64_t total_len, int32_t k, int32_t alphabet, sad_batch_plan *plan) {
  const int64_t eps = eps_of(k, alphabet);
  if (eps < 0) return SAD_ERR_UNSUPPORTED;
  if (!plan || !h_p || total_len < 0 || plan->rank.depth < 1 || !tile_valid(&plan->rank))
    return SAD_ERR_INVALID_ARGUMENT;
  RankShape sh;
  int rc = batch_plan_shape(h_n, h_p, n_sets, plan, &sh);
  if (rc) return rc;
  return plan_bound_caps(sh, total_len, k, eps, &plan->rank);
}

int sad_batch_rank(const int32_t *d_counts, const int32_t *d_lengths, const int32_t *d_word_max,
                   const int32_t *d_n, int32_t k, int32_t alphabet, const sad_batch_plan *plan,
                   uint64_t *d_key_hi, uint64_t *d_key_lo, double *d_rank, void *d_ws,
                   size_t ws_bytes, void *stream) {
  const int64_t eps = eps_of(k, alphabet);
  if (eps < 0) return SAD_ERR_UNSUPPORTED;
  if (!plan || plan->n_sets < 1 || !d_n || !d_counts || !d_lengths || !d_key_hi || !d_key_lo ||
      !d_ws || !aligned(d_ws, 256))
    return SAD_ERR_INVALID_ARGUMENT;
  const RankShape sh{plan->n_sets, plan->n_total, plan->rows_total, plan->tiles_total,
                     plan->tileof_total};
  return rank_run_impl(d_counts, d_lengths, d_word_max, sh, plan->n_sets > 1 ? d_n : nullptr,
                       eps, k,
                       &plan->rank, d_key_hi, d_key_lo, d_rank, d_ws, ws_bytes,
                       static_cast<cudaStream_t>(stream));
}

int sad_batch_partition(const uint64_t *d_key_hi, const uint64_t *d_key_lo, const int32_t *d_n,
                        const int32_t *d_p, const sad_batch_plan *plan,
                        int32_t *d_bucket_offsets, int32_t *d_members, int32_t *d_pivot_idx,
                        void *d_ws, size_t ws_bytes, void *stream) {
  if (!plan || plan->n_sets < 1 || !d_n || !d_p || !d_key_hi || !d_key_lo ||
      !d_bucket_offsets || !d_members || !d_ws || !aligned(d_ws, 256))
    return SAD_ERR_INVALID_ARGUMENT;
  if (ws_bytes < plan->part_ws_bytes) return SAD_ERR_WORKSPACE;
  const PartTotals pt{plan->n_total, plan->sum_p, plan->sum_p1, plan->sum_pp1, plan->sum_pp};
  if (plan->n_sets == 1) {
    // one set: its sizes are the plan's, so the single-set route (chunk sorts and rank
    // merges for few buckets) applies; same outputs, same workspace layout
    return partition_sets_launch(d_key_hi, d_key_lo, 1, nullptr, nullptr,
                                 (int32_t)plan->n_total, (int32_t)plan->sum_p, pt, plan->max_p,
                                 d_bucket_offsets, d_members, d_pivot_idx, d_ws,
                                 static_cast<cudaStream_t>(stream));
  }
  return partition_sets_launch(d_key_hi, d_key_lo, plan->n_sets, d_n, d_p, 0, 0, pt,
                               plan->max_p, d_bucket_offsets, d_members, d_pivot_idx, d_ws,
                               static_cast<cudaStream_t>(stream));
}

int partition(const uint64_t *d_key_hi, const uint64_t *d_key_lo, int32_t n_seq, int32_t p,
              int32_t *d_bucket_offsets, int32_t *d_members, int32_t *d_pivot_idx, void *d_ws,
              size_t ws_bytes, void *stream) {
  if (n_seq < 0 || p < 1 || p > kMaxP) return SAD_ERR_INVALID_ARGUMENT;
  if (n_seq > 0 && p > n_seq) return SAD_ERR_INVALID_ARGUMENT;
  if (!d_ws || !aligned(d_ws, 256) || !d_bucket_offsets) return SAD_ERR_INVALID_ARGUMENT;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (n_seq == 0) {
    return check_cuda(
        cudaMemsetAsync(d_bucket_offsets, 0, sizeof(int32_t) * (size_t)(p + 1), st));
  }
  if (!d_key_hi || !d_key_lo || !d_members) return SAD_ERR_INVALID_ARGUMENT;
  if (ws_bytes < part_layout(n_seq, p).bytes) return SAD_ERR_WORKSPACE;
  return partition_launch(d_key_hi, d_key_lo, n_seq, p, d_bucket_offsets, d_members,
                          d_pivot_idx, d_ws, st);
}

int sad_rank_info(void *d_ws, int64_t *info, void *stream) {
  if (!d_ws || !info) return SAD_ERR_INVALID_ARGUMENT;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  WsHeader h;
  int rc = check_cuda(cudaMemcpyAsync(&h, d_ws, sizeof(h), cudaMemcpyDeviceToHost, st));
  if (rc) return rc;
  rc = check_cuda(cudaStreamSynchronize(st));
  if (rc) return rc;
  info[0] = h.status;
  info[1] = h.k_eff;
  info[2] = h.k_pad;
  info[3] = h.t_max;
  info[4] = h.n_tiles;
  info[5] = (int64_t)h.k_chunks;
  info[6] = h.depth;
  info[7] = h.rem_entries;
  info[8] = h.rem_blocks;
  info[9] = h.heavy_entries;
  info[10] = h.bm_cols;
  return SAD_OK;
}

int sad_profile(int32_t enable) {
  std::lock_guard<std::mutex> g(g_prof_mu);
  g_prof_on = enable != 0;
  return SAD_OK;
}

int sad_profile_read(double *gemm_ms, int64_t *gemm_launches) {
  std::lock_guard<std::mutex> g(g_prof_mu);
  double total = 0.0;
  int64_t count = 0;
  for (auto &pr : g_prof_open) {
    float ms = 0.f;
    if (cudaEventSynchronize(pr.second) == cudaSuccess &&
        cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess) {
      total += ms;
      ++count;
    } else {
      cudaGetLastError();
    }
    g_prof_pool.push_back(pr.first);
    g_prof_pool.push_back(pr.second);
  }
  g_prof_open.clear();
  if (gemm_ms) *gemm_ms = total;
  if (gemm_launches) *gemm_launches = count;
  return SAD_OK;
}

int sad_status_read(void *d_ws, int32_t clear, void *stream) {
  if (!d_ws) return SAD_ERR_INVALID_ARGUMENT;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int32_t h[2] = {0, 0};
  int rc = check_cuda(cudaMemcpyAsync(h, d_ws, sizeof(h), cudaMemcpyDeviceToHost, st));
  if (rc) return rc;
  rc = check_cuda(cudaStreamSynchronize(st));
  if (rc) return rc;
  if (clear && h[0] != 0) {
    const int32_t z[2] = {0, 0};
    rc = check_cuda(cudaMemcpyAsync(d_ws, z, sizeof(z), cudaMemcpyHostToDevice, st));
    if (rc) return rc;
    rc = check_cuda(cudaStreamSynchronize(st));
    if (rc) return rc;
  }
  return h[0];
}

}  // extern "C"
