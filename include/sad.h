/*
 * sad.h - C-ABI of libsad, the GB300 (sm_103a) implementation of the
 * data-decomposition step of Sample-Align-D (Saeed & Khokhar, arXiv 0905.1744):
 * per-sequence k-mer count vectors, the k-mer rank of every sequence against the
 * whole set, and the regular-sampling partition of the rank-ordered set into p
 * buckets.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Pointers named d_* are device pointers (global memory of the current CUDA
 *   device). The caller owns every buffer; the library allocates no device
 *   memory. Scratch space comes from the caller as a workspace (d_ws, ws_bytes),
 *   256-byte aligned, sized with the query functions below.
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *   Every call is asynchronous on that stream unless it says otherwise.
 * - Return value: a sad_status. Argument errors that the host can see are
 *   returned at once and nothing is launched. Errors found in the data on the
 *   device (a letter code >= alphabet, a sequence shorter than k, a workspace
 *   too small for the data) are recorded in the workspace's status word and
 *   reported by sad_status_read(); kernels that see a recorded error skip their
 *   work, so outputs are then undefined. A recorded status stays until
 *   sad_status_read(..., clear = 1) resets it.
 * - Indices are 0-based positions in the input order. All results are
 *   deterministic integers (floating outputs are derived views).
 * - Layouts are row-major and densely packed.
 */
#ifndef SAD_H
#define SAD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SAD_ABI_VERSION 7

typedef enum sad_status {
  SAD_OK = 0,
  SAD_ERR_INVALID_ARGUMENT = 1, /* bad size, null pointer, misaligned buffer   */
  SAD_ERR_WORKSPACE = 2,        /* workspace smaller than the data requires    */
  SAD_ERR_CUDA = 3,             /* a CUDA runtime call failed                  */
  SAD_ERR_TIMEOUT = 4,          /* a bounded device-side wait gave up          */
  SAD_ERR_UNSUPPORTED = 5,      /* parameters outside what the library handles */
  SAD_ERR_BAD_INPUT = 6         /* code >= alphabet, length < k, counts that do
                                   not add up to L - k + 1                     */
} sad_status;

typedef enum sad_op {
  SAD_OP_COUNT = 0,
  SAD_OP_RANK = 1,
  SAD_OP_PARTITION = 2
} sad_op;

/* Human-readable name of a status code. Never NULL. */
const char *sad_status_string(int status);

/* SAD_ABI_VERSION of the loaded library. */
int sad_abi_version(void);

/*
 * Workspace bytes an entry point needs.
 *   op        SAD_OP_COUNT, SAD_OP_RANK or SAD_OP_PARTITION.
 *   n_seq     number of sequences N.
 *   k, alphabet  word length and alphabet size (eps = alphabet^k words).
 *   p         number of buckets (SAD_OP_PARTITION only).
 *   depth     SAD_OP_RANK only: the threshold-plane columns to reserve, as a
 *             multiple of eps (K_cap = eps * depth rounded up to 256), with no
 *             residual capacity: enough for kmer_rank without a plan when
 *             K_eff = sum over words of the largest count <= K_cap.
 *             kmer_rank_plan() gives exact sizes for any depth. depth <= 0 gives
 *             the fixed part only, which is what kmer_rank_plan() needs.
 * Returns 0 for arguments outside the supported range.
 */
size_t sad_workspace_bytes(int32_t op, int32_t n_seq, int32_t k, int32_t alphabet,
                           int32_t p, int32_t depth);

/*
 * kmer_count - per-sequence k-mer count vectors (Sec. 3, "k-mer Rank": the
 * vector c^X = (c^X_1, ..., c^X_eps) of occurrences of each of the eps = c^k
 * words in X).
 *   d_codes    uint8 letter codes of all sequences, concatenated; a code must be
 *              < alphabet (SAD_ERR_BAD_INPUT otherwise).
 *   d_offsets  int64 [n_seq + 1], sequence x is d_codes[off[x] .. off[x+1]);
 *              non-decreasing, off[0] >= 0. Every length must be >= k.
 *   k          1..8; alphabet 2..256; eps = alphabet^k <= 65536; every
 *              L - k + 1 must be <= 65535 (SAD_ERR_UNSUPPORTED otherwise).
 *   Malformed offsets (negative, decreasing, past off[n_seq]) are reported as
 *   SAD_ERR_INVALID_ARGUMENT and no code byte outside [off[0], off[n_seq]) is read.
 *   d_counts   int32 [n_seq][eps] output; word index
 *              tau = sum_r a_r * alphabet^(k-1-r) (first letter most significant).
 *   d_word_max (nullable) int32 [eps] output: the largest count of every word
 *              over the n_seq sequences; passing it to kmer_rank saves that call
 *              a pass over the counts.
 *   d_ws       workspace of sad_workspace_bytes(SAD_OP_COUNT, ...) bytes.
 */
int kmer_count(const uint8_t *d_codes, const int64_t *d_offsets, int32_t n_seq,
               int32_t k, int32_t alphabet, int32_t *d_counts, int32_t *d_word_max,
               void *d_ws, size_t ws_bytes, void *stream);

/*
 * Plan of a kmer_rank call. `depth` and `budget` are chosen by the caller (an
 * autotuner, or 0); kmer_rank_plan fills in the rest from the counts.
 *   depth        threshold sections kept as planes on the tensor cores: 0 keeps
 *                them all (no remainder); D >= 1 keeps min(D, 8). Each column
 *                block of 128 stored rows then runs its tiles over its own first
 *                d_J <= D sections (d_J: the smallest depth whose remainder fits
 *                the budget), and every threshold of min(a, b) = sum_t [a >= t]
 *                [b >= t] that those columns leave out is added back exactly in
 *                the epilogue from per-row remainder lists, so the keys are
 *                identical for every depth and budget.
 *   budget       remainder entries per column block (0 = the default, 768).
 *   tile         rows of a GEMM tile: 0 or 128 runs one CTA per 128 x 128 tile;
 *                256 runs pairs of CTAs (tcgen05 cta_group::2) on 256 x 256
 *                tiles, for one set (kmer_rank, not the batched or distance
 *                forms), its rows padded to 256 and the plane depths chosen per
 *                256-row column block. The keys are the same for either.
 *   t_max        largest count of any word in any sequence.
 *   t_bits       largest threshold of the remainder bitmap, min(D + 4, 16);
 *                counts above it are heavy entries, read from the counts.
 *   k_eff        plane columns of the kept sections.
 *   list_entries (sequence, word) entries counted twice or more.
 *   rem_bound    remainder entries there can be: sum over those entries of
 *                min(count, t_bits) - 1.
 *   heavy_entries entries counted more than t_bits times.
 *   k_cap, list_cap, rem_cap, heavy_cap, bm_cols  capacities kmer_rank lays
 *                the workspace out with (plane columns, entries counted twice or
 *                more, remainder entries, heavy entries, bitmap columns of
 *                rows_total bits); kmer_rank_plan sets them to what the data needs.
 *   ws_bytes     workspace bytes kmer_rank needs with this plan.
 */
typedef struct sad_rank_plan {
  int32_t depth;
  int32_t budget;
  int32_t tile;
  int32_t t_max;
  int32_t t_bits;
  int32_t reserved;
  int64_t k_eff;
  int64_t list_entries;
  int64_t rem_bound;
  int64_t heavy_entries;
  int64_t k_cap;
  int64_t list_cap;
  int64_t rem_cap;
  int64_t heavy_cap;
  int64_t bm_cols;
  size_t ws_bytes;
} sad_rank_plan;

/*
 * kmer_rank_plan - SYNCHRONOUS helper: reads the counts on the device and fills
 * `plan` (plan->depth is the input) with the sizes kmer_rank will need. Blocks
 * until `stream` is idle.
 *   d_counts   int32 [n_seq][eps], as written by kmer_count.
 *   d_ws       a workspace of at least sad_workspace_bytes(SAD_OP_RANK, n_seq,
 *              k, alphabet, 0, 0) bytes (the fixed part). A smaller one returns
 *              SAD_ERR_WORKSPACE at once with plan->ws_bytes set to that size.
 */
int kmer_rank_plan(const int32_t *d_counts, int32_t n_seq, int32_t k, int32_t alphabet,
                   sad_rank_plan *plan, void *d_ws, size_t ws_bytes, void *stream);

/*
 * kmer_rank_plan_bound - host only (no device access, no synchronisation): fills
 * `plan` (plan->depth >= 1 and plan->budget are the input) with capacities that
 * hold for ANY counts of n_seq sequences of total length total_len residues, so
 * kmer_rank can run right after kmer_count without the synchronous
 * kmer_rank_plan. With W = total_len - n_seq (k - 1) windows, D = min(depth, 8)
 * and T_b = min(D + 4, 16) (the threshold identity of Sec. 3 Eq. 1):
 *   k_cap      = eps * D rounded up to 256 (K_eff = sum_tau min(T_tau, D)),
 *   list_cap   = W / 2 (a sequence of m windows has at most m / 2 words counted
 *                twice or more),
 *   rem_cap    = W - n_seq (a sequence's counts c >= 2 add at most m - 1
 *                thresholds above the first),
 *   heavy_cap  = W / (T_b + 1),
 *   bm_cols    = sum over t = 2..T_b of min(eps, W / t) (section t holds the
 *                words some sequence counts t times).
 * t_max, t_bits, k_eff, list_entries, rem_bound and heavy_entries are set to -1
 * (not known).
 * Returns SAD_ERR_INVALID_ARGUMENT for depth < 1 (all planes need the word
 * maxima) or negative sizes, SAD_ERR_UNSUPPORTED for unsupported k / alphabet
 * or more than 32767 row blocks of 128 (n_seq > 4194176).
 */
int kmer_rank_plan_bound(int32_t n_seq, int64_t total_len, int32_t k, int32_t alphabet,
                         sad_rank_plan *plan);

/*
 * kmer_rank - the k-mer rank of every sequence against the whole set.
 * Eq. 1: F(X,Y) = sum_i min(c^X_i, c^Y_i) / (min(n, m) - k + 1); Eq. 3:
 * R_i = (1/N) sum_{j=1..N} F(i, j), j = i included, taken on F itself (the mean
 * similarity) rather than on the distance of Eq. 2.
 * The rank is carried exactly as a 128-bit fixed-point key
 *     key_i = sum_j floor(S_ij * 2^64 / D_ij),
 * S_ij = sum_i min(...) and D_ij = min(L_i, L_j) - k + 1, split into
 * key = key_hi * 2^64 + key_lo; the float view is
 *     rank_i = (key_hi + key_lo * 2^-64) / N   (each step rounded to nearest).
 * Internally min(a, b) = sum_t [a >= t][b >= t] turns all pairs into one
 * threshold-plane GEMM on the tensor cores; the N x N matrix is never stored.
 *   d_counts   int32 [n_seq][eps] from kmer_count (16-byte aligned for the
 *              vector path); n_seq (or, batched, the rows of all sets, each set
 *              padded to a multiple of 128) at most 32767 x 128 = 4194176
 *              (SAD_ERR_UNSUPPORTED otherwise).
 *   d_lengths  int32 [n_seq] sequence lengths L (residues); every
 *              L - k + 1 must be in 1..65535 (SAD_ERR_UNSUPPORTED otherwise)
 *              and equal to the sum of the sequence's counts (SAD_ERR_BAD_INPUT).
 *   d_word_max (nullable) int32 [eps], the largest count of every word, as
 *              kmer_count returns it for these counts.
 *   plan       (nullable) a plan from kmer_rank_plan for these counts; NULL keeps
 *              all planes and takes the plane capacity from ws_bytes.
 *   d_key_hi, d_key_lo  uint64 [n_seq] outputs.
 *   d_rank     (nullable) float64 [n_seq] output.
 *   d_ws       workspace of at least plan->ws_bytes (or, without a plan,
 *              sad_workspace_bytes(SAD_OP_RANK, ..., depth) with
 *              depth * eps >= K_eff). Data that need more than the capacities
 *              record SAD_ERR_WORKSPACE and write no keys.
 */
int kmer_rank(const int32_t *d_counts, const int32_t *d_lengths, const int32_t *d_word_max,
              int32_t n_seq, int32_t k, int32_t alphabet, const sad_rank_plan *plan,
              uint64_t *d_key_hi, uint64_t *d_key_lo, double *d_rank, void *d_ws,
              size_t ws_bytes, void *stream);

/*
 * partition - regular-sampling sample sort of the keys into p buckets
 * (Sec. 3.1.2 and Algorithm 2 steps 7-11, the p processors being virtual
 * buckets on one device):
 *   block b = input positions [floor(bN/p), floor((b+1)N/p)) is sorted by
 *   (key, index); p-1 samples are taken per block at 0-based positions
 *   floor(j w_b / p), j = 1..p-1; the p(p-1) samples are sorted and the pivots
 *   are y_i = Y_{(i-1)p + floor(p/2)} (1-based), i = 1..p-1; bucket i (1-based)
 *   receives the keys in (y_{i-1}, y_i] (Sec. 3.3.2), ties ordered by index.
 *   d_key_hi, d_key_lo  uint64 [n_seq] keys (as from kmer_rank).
 *   p          1 <= p <= n_seq (or n_seq == 0), p <= 4096.
 *   d_bucket_offsets  int32 [p + 1] output (CSR offsets).
 *   d_members  int32 [n_seq] output: input indices, bucket by bucket, each bucket
 *              in ascending (key, index) order.
 *   d_pivot_idx  (nullable) int32 [p - 1] output: input index of each pivot.
 *   d_ws       workspace of sad_workspace_bytes(SAD_OP_PARTITION, ...) bytes.
 */
int partition(const uint64_t *d_key_hi, const uint64_t *d_key_lo, int32_t n_seq,
              int32_t p, int32_t *d_bucket_offsets, int32_t *d_members,
              int32_t *d_pivot_idx, void *d_ws, size_t ws_bytes, void *stream);

/*
 * partition_noalloc - the same partition as partition(), for callers that
 * cannot allocate device memory (an arena or pool that owns every device byte,
 * a host application that forbids allocation after start-up, a hot path that
 * must not touch the allocator). The paper has no counterpart: this is an
 * interface convenience of this library.
 *   Its scratch is a fixed array inside the library's device image, sized for
 *   the largest accepted call (about 2.1 MiB), held by every GPU that loads the
 *   library until the process exits. Limits: n_seq <= 32768 and p <= 64, in
 *   any combination; larger calls return SAD_ERR_UNSUPPORTED and launch
 *   nothing. Other arguments and outputs are those of partition().
 *   The first call on a device looks up the array's device address (with that
 *   device current); make that first call before any stream capture.
 *   All calls share the one array and it keeps the last call's contents;
 *   nothing in it needs clearing, since each call writes every region before
 *   reading it. Calls whose GPU work overlaps race on the array: keep them
 *   ordered on one stream.
 */
int partition_noalloc(const uint64_t *d_key_hi, const uint64_t *d_key_lo, int32_t n_seq,
                      int32_t p, int32_t *d_bucket_offsets, int32_t *d_members,
                      int32_t *d_pivot_idx, void *stream);

/*
 * Batched forms: n_sets independent sequence sets processed together, the
 * batching workload of the paper's many-set setting. The sets are laid out one
 * after the other in every per-sequence array (set s holds the sequences
 * [seq_begin_s, seq_begin_s + n_s), seq_begin the prefix sum of n). kmer_count
 * already takes all sets at once (one offsets array over every sequence).
 * The rank is block-diagonal: one persistent GEMM launch covers every set's
 * tiles, and a set's keys depend only on its own sequences (Eq. 3 with N = n_s).
 * The partition cuts every set into its own p_s buckets (Sec. 3.1.2 per set).
 * After sad_batch_plan_make the two calls launch no synchronising operation, so
 * the whole batch can be captured in a CUDA graph and replayed.
 *
 *   rank            depth, budget and tile in (see sad_rank_plan); sizes and
 *                   capacities out, for all sets together (rank.ws_bytes:
 *                   sad_batch_rank's workspace).
 *   n_sets, max_p   sets and the largest p_s.
 *   n_total, rows_total, tiles_total, tileof_total  sums over sets of n_s,
 *                   stored rows (n_s rounded up to the plan's tile rows, 128
 *                   or 256), GEMM tiles and tile-map entries.
 *   sum_p, sum_p1, sum_pp1, sum_pp  sums of p_s, p_s - 1, p_s (p_s - 1), p_s^2.
 *   part_ws_bytes   workspace bytes of sad_batch_partition.
 */
typedef struct sad_batch_plan {
  sad_rank_plan rank;
  int32_t n_sets;
  int32_t max_p;
  int64_t n_total;
  int64_t rows_total;
  int64_t tiles_total;
  int64_t tileof_total;
  int64_t sum_p, sum_p1, sum_pp1, sum_pp;
  size_t part_ws_bytes;
} sad_batch_plan;

/*
 * sad_batch_plan_make - SYNCHRONOUS: the plan of a batch.
 *   d_counts   int32 [n_total][eps] counts of all sets (from one kmer_count).
 *   h_n, h_p   host int32 [n_sets]: sequences and buckets per set
 *              (1 <= p_s <= min(n_s, 4096)).
 *   d_n        device copy of h_n.
 *   plan       plan->rank.depth, budget and tile in; the rest out.
 *   d_ws       rank workspace; if smaller than the fixed part, returns
 *              SAD_ERR_WORKSPACE with plan->rank.ws_bytes = the bytes needed.
 */
int sad_batch_plan_make(const int32_t *d_counts, const int32_t *h_n, const int32_t *h_p,
                        const int32_t *d_n, int32_t n_sets, int32_t k, int32_t alphabet,
                        sad_batch_plan *plan, void *d_ws, size_t ws_bytes, void *stream);

/*
 * sad_batch_rank - kmer_rank of every set of the batch (Eq. 1, Eq. 3 per set).
 *   d_counts, d_lengths  all sets' counts and lengths, set after set.
 *   d_word_max (nullable) largest count of every word over the whole batch.
 *   d_n        device int32 [n_sets] set sizes (as given to the plan).
 *   d_key_hi, d_key_lo, d_rank  per-sequence outputs, set after set.
 *   d_ws       at least plan->rank.ws_bytes.
 */
int sad_batch_rank(const int32_t *d_counts, const int32_t *d_lengths, const int32_t *d_word_max,
                   const int32_t *d_n, int32_t k, int32_t alphabet, const sad_batch_plan *plan,
                   uint64_t *d_key_hi, uint64_t *d_key_lo, double *d_rank, void *d_ws,
                   size_t ws_bytes, void *stream);

/*
 * sad_batch_partition - partition() of every set of the batch.
 *   d_n, d_p   device int32 [n_sets] set sizes and bucket counts.
 *   d_bucket_offsets  int32 [sum over sets of (p_s + 1)]: set s's CSR offsets
 *              (local, 0..n_s) start at entry sum_{s'<s} (p_s' + 1).
 *   d_members  int32 [n_total]: set s's members (local indices) fill
 *              [seq_begin_s, seq_begin_s + n_s).
 *   d_pivot_idx (nullable) int32 [sum_p1]: set s's p_s - 1 pivots (local
 *              indices) start at sum_{s'<s} (p_s' - 1).
 *   d_ws       at least plan->part_ws_bytes.
 */
int sad_batch_partition(const uint64_t *d_key_hi, const uint64_t *d_key_lo, const int32_t *d_n,
                        const int32_t *d_p, const sad_batch_plan *plan,
                        int32_t *d_bucket_offsets, int32_t *d_members, int32_t *d_pivot_idx,
                        void *d_ws, size_t ws_bytes, void *stream);

/*
 * sad_batch_plan_bound - the plan of a batch from host-side bounds alone: no
 * device work, no synchronisation, no look at the counts (the batched form of
 * kmer_rank_plan_bound, whose capacity rules it applies to the whole batch).
 *   h_n, h_p   host int32 [n_sets] as for sad_batch_plan_make.
 *   total_len  residues of all sequences of the batch (off[n_total] - off[0]).
 *   plan       plan->rank.depth (>= 1), budget and tile in; the rest out
 *              (rank.t_max, t_bits, k_eff, list_entries, rem_bound and
 *              heavy_entries are -1: unknown without the counts).
 * Returns SAD_ERR_INVALID_ARGUMENT for depth < 1, a tile other than 0, 128,
 * 256, or sizes outside those of sad_batch_plan_make. Batches of the same
 * per-set sizes and total length get the same plan, so a CUDA graph captured
 * for one of them (sad_graph_*) can be updated to the next without any device
 * synchronisation.
 */
int sad_batch_plan_bound(const int32_t *h_n, const int32_t *h_p, int32_t n_sets,
                         int64_t total_len, int32_t k, int32_t alphabet, sad_batch_plan *plan);

/*
 * sad_seq_lengths - d_lengths[i] = off[i + 1] - off[i] for the n_seq sequences
 * of an offsets array (the L of Sec. 2's F denominator, as kmer_rank takes it).
 *   d_offsets  device int64 [n_seq + 1].
 *   d_lengths  device int32 [n_seq] output.
 *   d_ws       (nullable) a workspace whose header records SAD_ERR_BAD_INPUT
 *              for a negative or too long length (that entry is written 0).
 * Launches one kernel on `stream`; no synchronisation.
 */
int sad_seq_lengths(const int64_t *d_offsets, int32_t n_seq, int32_t *d_lengths, void *d_ws,
                    void *stream);

/*
 * Reusable CUDA graphs. sad_graph_begin starts stream capture on `stream`
 * (thread-local mode); the caller then makes asynchronous library calls on it
 * (for example sad_batch_rank and sad_batch_partition on a bound plan);
 * sad_graph_end ends the capture. On the first end (*g == NULL) the captured
 * graph is instantiated into a new handle; on later ends with the same handle
 * it replaces the instantiated graph's parameters in place when the launch
 * sequence has the same topology (a new batch of the same plan shape: new
 * buffers and sizes, no re-instantiation), and is instantiated afresh
 * otherwise. sad_graph_launch runs the current graph on `stream`.
 * sad_graph_stats: updates and instantiations so far, kernel nodes of the
 * current graph. sad_graph_destroy frees the handle (NULL is accepted).
 * No call made between begin and end may synchronise (the capture fails and
 * sad_graph_end returns SAD_ERR_CUDA, leaving the handle's graph as it was).
 * The library's own launches inside a capture are recorded, not run.
 */
typedef struct sad_graph_s *sad_graph;
int sad_graph_begin(void *stream);
int sad_graph_end(void *stream, sad_graph *g);
int sad_graph_launch(sad_graph g, void *stream);
int sad_graph_stats(sad_graph g, int64_t *updates, int64_t *instantiations, int32_t *kernels);
int sad_graph_destroy(sad_graph g);

/*
 * sad_status_read - SYNCHRONOUS: waits for `stream`, then returns the status
 * recorded in the workspace by the device (SAD_OK if none). With clear != 0 the
 * recorded status is reset to SAD_OK. d_ws must be a workspace previously passed
 * to one of the entry points above (its first 256 bytes are the header).
 */
int sad_status_read(void *d_ws, int32_t clear, void *stream);

/*
 * Globalised k-mer rank (Sec. 3.1.1, Algorithm 2 steps 2-6). Each of p
 * "processors" holds the contiguous block [floor(bN/p), floor((b+1)N/p)) of the
 * sequences (input order). Step 2 ranks every block against itself: use the
 * batched rank (sad_batch_plan_make / sad_batch_rank) with the blocks as sets.
 * Steps 3-5 are sad_local_samples, step 6 is kmer_rank_vs with the samples as
 * the reference set; partition on its keys then gives the buckets (steps 7-11).
 *
 * sad_local_samples - sorts every block by its key (ties by input index) and
 *   takes ks evenly spaced samples of it, at the 0-based positions
 *   floor(j w_b / (ks + 1)), j = 1..ks, of the sorted block of w_b sequences
 *   (the spacing of the regular sampling of Sec. 3.1.2; a position may repeat
 *   when w_b <= ks).
 *   d_key_hi, d_key_lo  uint64 [n_seq] local keys (input order).
 *   p          blocks, 1 <= p <= n_seq; ks >= 1, ks * p < 2^31.
 *   d_sample_idx  int32 [p * ks] output: input indices, block-major.
 *   d_ws       workspace of sad_local_samples_workspace_bytes(n_seq, p) bytes.
 *   Asynchronous on `stream`; argument errors return SAD_ERR_INVALID_ARGUMENT.
 */
size_t sad_local_samples_workspace_bytes(int32_t n_seq, int32_t p);
int sad_local_samples(const uint64_t *d_key_hi, const uint64_t *d_key_lo, int32_t n_seq,
                      int32_t p, int32_t ks, int32_t *d_sample_idx, void *d_ws,
                      size_t ws_bytes, void *stream);

/*
 * kmer_rank_vs - the k-mer rank of every sequence against a reference multiset R
 * of sequences of the same set (Algorithm 2 step 6):
 *     key_i = sum_{r in R} floor(S_ir * 2^64 / D_ir),   D_ir = min(L_i, L_r) - k + 1,
 *     rank_i = (key_hi + key_lo * 2^-64) / |R|,
 * an index listed twice in R counting twice. With R = every sequence once this is
 * the kmer_rank key. With delta_den = b > 0 the rank is the distance form of
 * kmer_rank_dist instead: key_i = sum_r (ln_q(b D_ir) - ln_q(D_ir + b S_ir)),
 * rank_i = key_i 2^-32 / |R|, signed keys in d_key (nullable), the order-keeping
 * unsigned view in (d_key_hi, d_key_lo). Runs the rank preparation at full plane
 * depth, gathers the reference rows' planes and runs the plane GEMM over
 * (all rows) x (R).
 *   d_counts, d_lengths, d_word_max   as for kmer_rank.
 *   d_ref      int32 [n_ref] input indices of R (0 <= d_ref[r] < n_seq, checked on
 *              the device: SAD_ERR_INVALID_ARGUMENT).
 *   delta_den  0: the similarity form; b in 1..1024: the distance form, Delta = 1/b.
 *   plan       (required) a plan from kmer_rank_plan with depth 0 for these
 *              counts (it fixes the plane capacity k_cap).
 *   d_ws       workspace of kmer_rank_vs_workspace_bytes(plan, n_seq, k,
 *              alphabet, n_ref, delta_den) bytes.
 *   d_key      (nullable) int64 [n_seq], the signed keys of the distance form.
 *   d_key_hi, d_key_lo  uint64 [n_seq]; d_rank (nullable) float64 [n_seq].
 */
size_t kmer_rank_vs_workspace_bytes(const sad_rank_plan *plan, int32_t n_seq, int32_t k,
                                    int32_t alphabet, int32_t n_ref, int32_t delta_den);
int kmer_rank_vs(const int32_t *d_counts, const int32_t *d_lengths, const int32_t *d_word_max,
                 int32_t n_seq, int32_t k, int32_t alphabet, const int32_t *d_ref,
                 int32_t n_ref, int32_t delta_den, const sad_rank_plan *plan, int64_t *d_key,
                 uint64_t *d_key_hi, uint64_t *d_key_lo, double *d_rank, void *d_ws,
                 size_t ws_bytes, void *stream);

/*
 * kmer_rank_dist - the k-mer rank of Eq. 2 and Eq. 3 as written: the mean over
 * the set of the distance d(i, j) = -ln(Delta + F(i, j)), Delta = 1 / delta_den.
 * With F = S / D, d = ln(b D) - ln(D + b S) (b = delta_den), and both logarithms
 * are the deterministic fixed-point values ln_q(x) = ln(x) * 2^32 of sad_ln_q (a
 * repeated-squaring binary logarithm with 40 fraction bits times ln 2; within
 * 2^-32 of ln x), so every per-pair value q_ij = ln_q(b D) - ln_q(D + b S) is an
 * integer and the key
 *     key_i = sum_j q_ij   (signed, j = i included)
 * is exact. rank_i = key_i * 2^-32 / N (each step rounded to nearest), in nats;
 * a smaller rank is a more similar sequence. d_key_hi = 0 and d_key_lo = key_i xor
 * 2^63 order the keys as unsigned values, for partition.
 *   delta_den  b, 1..1024.
 *   plan       (required) a plan from kmer_rank_plan for these counts (any depth).
 *   d_key      (nullable) int64 [n_seq]: the signed keys.
 *   d_ws       workspace of kmer_rank_dist_workspace_bytes(plan, n_seq, k, alphabet,
 *              delta_den) bytes (the rank workspace plus the ln_q table).
 * Other arguments as for kmer_rank.
 */
size_t kmer_rank_dist_workspace_bytes(const sad_rank_plan *plan, int32_t n_seq, int32_t k,
                                      int32_t alphabet, int32_t delta_den);
int kmer_rank_dist(const int32_t *d_counts, const int32_t *d_lengths, const int32_t *d_word_max,
                   int32_t n_seq, int32_t k, int32_t alphabet, int32_t delta_den,
                   const sad_rank_plan *plan, int64_t *d_key, uint64_t *d_key_hi,
                   uint64_t *d_key_lo, double *d_rank, void *d_ws, size_t ws_bytes,
                   void *stream);

/*
 * sad_ln_q - ln_q(x) = ln(x) * 2^32 as the fixed-point value the distance-form
 * rank uses (0 for x = 0), for n values d_x on the device into d_out (int64).
 */
int sad_ln_q(const uint64_t *d_x, int64_t n, int64_t *d_out, void *stream);

/*
 * kmer_rank_sparse - the kmer_rank keys (same definition, bit for bit) computed by
 * sparse intersection on the CUDA cores instead of the threshold-plane GEMM: the
 * per-pair cost of Table 2, O(L) per pair (one sequence's list of occurring words
 * against the other's counts), every ordered pair evaluated. A comparison point
 * for the tensor-core path, not a faster one.
 * kmer_rank_sparse_entries - SYNCHRONOUS: the total number of (sequence, word)
 *   entries with a nonzero count, the capacity kmer_rank_sparse needs; its
 *   workspace must hold kmer_rank_sparse_workspace_bytes(n_seq, 0) bytes.
 *   entries_cap  at least that total (SAD_ERR_WORKSPACE recorded otherwise).
 *   d_ws       kmer_rank_sparse_workspace_bytes(n_seq, entries_cap) bytes.
 *   eps = alphabet^k up to 65536 (a 16-bit shared histogram of eps bins per CTA).
 * Other arguments as for kmer_rank.
 */
size_t kmer_rank_sparse_workspace_bytes(int32_t n_seq, int64_t entries_cap);
int kmer_rank_sparse_entries(const int32_t *d_counts, const int32_t *d_lengths, int32_t n_seq,
                             int32_t k, int32_t alphabet, int64_t *entries, void *d_ws,
                             size_t ws_bytes, void *stream);
int kmer_rank_sparse(const int32_t *d_counts, const int32_t *d_lengths, int32_t n_seq,
                     int32_t k, int32_t alphabet, int64_t entries_cap, uint64_t *d_key_hi,
                     uint64_t *d_key_lo, double *d_rank, void *d_ws, size_t ws_bytes,
                     void *stream);

/* Number of kernels this library has launched in this process. */
uint64_t sad_launch_count(void);

/*
 * Diagnostics.
 * sad_rank_info - SYNCHRONOUS: after kmer_rank on `stream`, copies the plan the
 *   device chose into info[0..10]: {status, K_eff, K_pad, t_max, tiles,
 *   executed K chunks (sum over tiles of plane chunks + remainder chunks, 256
 *   K columns each), planes kept per word (the plan's depth), remainder
 *   entries, column blocks with remainder entries, heavy entries (counts above
 *   the remainder bitmap), remainder bitmap columns}; info must hold 16 entries.
 * sad_profile - enable != 0 starts recording a CUDA event pair around every
 *   launch of the GEMM kernel (one CTA or CTA-pair form, on its own stream);
 *   0 stops.
 * sad_profile_read - SYNCHRONOUS: waits for the recorded events, returns the
 *   summed GEMM time in milliseconds and the number of launches, and clears them.
 */
int sad_rank_info(void *d_ws, int64_t *info, void *stream);
int sad_profile(int32_t enable);
int sad_profile_read(double *gemm_ms, int64_t *gemm_launches);

/*
 * sad_debug_wait_budget_ns - failure detection test hook (the paper has no
 *   counterpart). Every wait of the plane GEMM (a TMA copy landing, an MMA
 *   freeing a pipeline stage, an accumulator filling or draining) is a bounded
 *   spin on %globaltimer; on running out the CTA records SAD_ERR_TIMEOUT in the
 *   workspace status, waits for its own copies and MMAs in flight (with a fixed
 *   2 s budget), frees its tensor memory and returns, so the context stays
 *   usable. This sets the budget of those main-loop waits for every later launch
 *   in the process: ns = 0 restores the default of 2 s. A budget of a few
 *   nanoseconds makes the first wait that does not succeed at once give up,
 *   which is how the tests drive the timeout path without a hang.
 *   Returns SAD_OK.
 */
int sad_debug_wait_budget_ns(uint64_t ns);

#ifdef __cplusplus
}
#endif

#endif /* SAD_H */
