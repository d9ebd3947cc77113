/*
 * sogrand.h -- C ABI of libsogrand: soft-output GRAND (SOGRAND) decoding of
 * short even linear codes and block-turbo decoding of product codes on one
 * NVIDIA GB300 (sm_103a).
 *
 * Method: P. Yuan, M. Medard, K. Galligan, K. R. Duffy, "Soft-output (SO)
 * GRAND and iterative decoding to outperform LDPCs", arXiv 2310.10737.
 *
 * Conventions shared by every call
 *   - LLR = log p(r | bit 0) / p(r | bit 1) (Sec. V-B); a negative LLR is a
 *     hard 1, an LLR of exactly 0 is a hard 0.
 *   - The SISO input of a word is lambda = fl32(L_Ch + L_A), one FP32
 *     rounding; every decision (hard bits, reliability ranks, the 1-line
 *     parameter) is taken on that value.
 *   - Query order: 1-line ORBGRAND (the paper's choice, Sec. VI): patterns by
 *     increasing cost = (sum of reliability ranks) + c * (Hamming weight),
 *     ties by weight then lexicographic rank vector; ranks by |lambda|
 *     ascending with ties to the lower bit index; c is the rounded
 *     intercept/slope of the exact least-squares line through the sorted
 *     |lambda| quantised to 1/256 (saturating at 4096), clamped to [0, n].
 *   - Even codes (Sec. III-B): only noise patterns with the parity of the
 *     hard decision are queried, and the soft output is conditioned on that
 *     parity class: phi = (2^k - 1)/(2^(n-1) - 1) in the Corollary of Sec. IV.
 *   - Device pointers are CUDA device (or managed) memory of the current
 *     device; `stream` is a cudaStream_t (NULL = legacy default stream).
 *     Calls are asynchronous on `stream` unless stated; results are valid
 *     once the stream has reached the call.  The caller owns every buffer.
 *   - Every call returns SOGRAND_OK or one of the error codes below and
 *     writes nothing on an argument error.  sogrand_strerror() names them.
 */
#ifndef SOGRAND_H
#define SOGRAND_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SOGRAND_OK 0
#define SOGRAND_EINVAL 1       /* invalid argument (sizes, pointers, code) */
#define SOGRAND_ENOMEM 2       /* device or host allocation failed */
#define SOGRAND_ECUDA 3        /* a CUDA runtime call failed */
#define SOGRAND_ETIMEOUT 4     /* a bounded device wait gave up */
#define SOGRAND_EUNSUPPORTED 5 /* valid but not implemented (e.g. row and column codes of different kernel classes) */

/* Opaque code object: parity-check matrix, its device copy and the query-order
 * tables.  Immutable after creation apart from table growth (see
 * sogrand_code_reserve); may be shared by threads and streams. */
typedef struct sogrand_code sogrand_code;

/*
 * Create a code from its (n-k) x n parity-check matrix H (Sec. III-B:
 * x is a codeword iff H x = 0).
 *   n      2 <= n <= 128
 *   k      1 <= k < n, n - k <= 64
 *   H      HOST pointer, (n-k) x n row-major, entries 0 or 1
 *   even   1: the code is even (all-ones vector in the row space of H) and
 *          the search is restricted to the parity class of the hard
 *          decision (Sec. III-B); EINVAL if the code is not even.
 *          0: all patterns are queried, phi = (2^k-1)/(2^n-1).
 *   out    receives the object (NULL on error)
 * Builds the query-order tables for query caps up to 10^4 and copies them to
 * the current device (synchronous).  Errors: EINVAL, ENOMEM, ECUDA.
 */
int sogrand_code_create(int n, int k, const uint8_t *H, int even, sogrand_code **out);

/* Release a code and its device memory.  No decode using it may be in
 * flight.  NULL is ignored. */
void sogrand_code_destroy(sogrand_code *code);

/*
 * Make the query-order tables cover query caps up to max_query_cap
 * (synchronous; reallocates the tables, so no decode using `code` may be in
 * flight).  Decodes with a larger cap call this themselves.
 * Errors: EINVAL (max_query_cap < 1 or > 2^24), ENOMEM, ECUDA.
 */
int sogrand_code_reserve(sogrand_code *code, int64_t max_query_cap);

/* Length n and dimension k of a code (either pointer may be NULL). */
int sogrand_code_info(const sogrand_code *code, int *n, int *k);

/* The query-order tables of a code: the query cap they cover and their
 * device memory in bytes (either pointer may be NULL).  Errors: EINVAL. */
int sogrand_code_tables(const sogrand_code *code, int64_t *query_cap, int64_t *bytes);

/*
 * Limits of the bounded device-side waits (process-wide; read when a decode
 * is launched, so set them while no decode is being launched).  The paper has
 * no counterpart: these bound the GPU decoders' own synchronisation.
 *   queue_wait_us  microseconds of accumulated back-off that a warp of a
 *                  batched (persistent) launch waits for work before the
 *                  launch stops and returns SOGRAND_ETIMEOUT (default
 *                  2,000,000; 0 gives up at the first wait)
 *   lock_polls     polls of its block's remaining-mass lock after which a
 *                  warp gives up on the lock (default 2^22); the batched forms
 *                  then stop and return SOGRAND_ETIMEOUT
 *   lock_preheld   1: every block starts with its remaining-mass lock taken,
 *                  as if a warp held it and never released it (tests of the
 *                  bound; decoding results are then invalid); 0: normal
 * A negative value keeps the current setting.  Errors: EINVAL (a value above
 * 2^31 - 1, lock_preheld > 1).
 */
int sogrand_set_wait_limits(int64_t queue_wait_us, int64_t lock_polls, int lock_preheld);

/*
 * SOGRAND soft-input soft-output decoding of n_words independent words
 * (Fig. siso; Sec. IV Corollary; Sec. V-B eq. LLRi).  One warp per word.
 *   llr_ch     device [n_words][n] channel LLRs L_Ch
 *   llr_a      device [n_words][n] a-priori LLRs L_A, or NULL for zeros
 *   L          list size, 1 <= L <= 16: the search stops at the L-th codeword
 *   query_cap  1 <= cap <= 2^24: the search also stops after this many queries
 *   thr        0 disables; else the search also stops as soon as the predicted
 *              probability that the list misses the transmitted codeword
 *              (eq. app_approxlist) drops below thr (checked at each new word)
 *   outputs (device, each may be NULL):
 *   hard       [n_words][n] u8: 1 where L_APP < 0
 *   llr_app    [n_words][n] L_APP (eq. LLRi)
 *   llr_ext    [n_words][n] L_E = L_APP - lambda (0 when the list is empty)
 *   p_miss     [n_words] probability that the codeword is not in the list
 *   queries    [n_words] codebook queries made; -1 marks a word with a
 *              non-finite input LLR (its outputs: L_APP = lambda, L_E = 0,
 *              p_miss = 1, empty list)
 *   list_words [n_words][L][ceil(n/64)] u64: the listed codewords in query
 *              order, bit i of the word = bit (i mod 64) of u64 (i / 64);
 *              unused slots are 0
 *   list_app   [n_words][L] APP of each listed codeword (eq. app_approx_correct)
 *   list_count [n_words] number of listed codewords
 * With an empty list (cap reached before any codeword) L_APP = lambda.
 * May grow the tables (synchronous) if query_cap exceeds the reserved cap.
 * Errors: EINVAL, ENOMEM, ECUDA.
 */
int sogrand_decode(sogrand_code *code, int64_t n_words, const float *llr_ch, const float *llr_a, int L,
                   int64_t query_cap, float thr, uint8_t *hard, float *llr_app, float *llr_ext, float *p_miss,
                   int64_t *queries, uint64_t *list_words, float *list_app, int32_t *list_count, void *stream);

/*
 * The same SISO decoding with Forney's approximation of the soft output
 * (Sec. IV, eq. missingterm): the APPs are normalised over the list alone, the
 * mass of the codewords outside the list being taken as 0.  The paper uses it
 * as the comparison for SOGRAND's soft output (Fig. list_BLER: Forney's
 * predicted list-BLER for the first L' words of an (L'+1)-word list is the
 * last word's APP).  Outputs as sogrand_decode, with p_miss = 0 and
 * L_APP = +-infinity for bits on which every listed word agrees; an empty list
 * gives L_APP = lambda and p_miss = 1.  There is no threshold rule (its
 * prediction would always be 0).  Errors: EINVAL, ENOMEM, ECUDA.
 */
int sogrand_decode_forney(sogrand_code *code, int64_t n_words, const float *llr_ch, const float *llr_a, int L,
                          int64_t query_cap, uint8_t *hard, float *llr_app, float *llr_ext, float *p_miss,
                          int64_t *queries, uint64_t *list_words, float *list_app, int32_t *list_count, void *stream);

/*
 * Block turbo decoding of n_frames product codes (Sec. VI, Fig. turboDec):
 * L_A = 0; each half iteration decodes every row (odd halves) or column (even
 * halves) of every running frame with SOGRAND (lambda = L_Ch + fl32(alpha L_E)
 * of the previous half), takes the hard decision of L_APP and stops a frame
 * as soon as every row and column is a codeword; at most 2 * max_iter halves.
 *   row_code, col_code  the component codes: every row of a frame is a word
 *              of the row code (n_row = its n), every column a word of the
 *              column code (n_col = its n).  They may be the same object (a
 *              square product code) or two codes of one kernel class: both n
 *              in 1..32, in 33..64 or in 65..128, and both n - k <= 32 or both
 *              above (EUNSUPPORTED otherwise).  Below, n x n reads n_col x n_row.
 *   llr_ch     device [n_frames][n_col][n_row] channel LLRs, row-major (bit
 *              (i, j) is row i, column j)
 *   L, query_cap, thr   as for sogrand_decode (query_cap < 2^(n-1) for both
 *              codes, so the search never exhausts a parity class)
 *   alpha      extrinsic scaling, > 0 (the paper uses 0.5)
 *   max_iter   1 <= max_iter <= 1000 full (row + column) iterations
 *   outputs (device):
 *   bits       [n_frames][ceil(n_col*n_row/8)] u8: the final hard decision,
 *              bit p = i*n_row + j at byte p/8, bit p%8 (required)
 *   half_iters [n_frames] half iterations run (may be NULL)
 *   status     [n_frames] 0 decoded (all rows and columns codewords), 1 max
 *              iterations reached, 2 non-finite input (may be NULL)
 *   queries    [n_frames] total codebook queries (may be NULL)
 * Allocates its scratch (about 4 n^2 + 8 n ceil(n/64) + 16 bytes per frame)
 * stream-ordered on `stream` and reads a device flag between halves to stop
 * early, so the call returns when the decode has finished.
 * Errors: EINVAL, EUNSUPPORTED, ENOMEM, ECUDA.
 */
int product_decode(sogrand_code *row_code, const sogrand_code *col_code, int64_t n_frames, const float *llr_ch,
                   int L, int64_t query_cap, float thr, float alpha, int max_iter, uint8_t *bits,
                   int32_t *half_iters, uint8_t *status, int64_t *queries, void *stream);

/* Optional extra outputs and measurements of product_decode_ex.  Every
 * member may be NULL. */
typedef struct {
  int64_t *par_queries;  /* device [n_frames]: "parallelized" queries, the sum
                            over half iterations of the largest per-word query
                            count (Sec. VI) */
  uint64_t *weight_sum;  /* device [1]: incremented by the summed Hamming
                            weights of every queried noise pattern */
  int32_t *xf_words;     /* device [1]: incremented once per component decoding
                            whose remaining-mass sum needed the extended-range
                            arithmetic (all FP32-scaled terms underflowed) */
  float *timing_ms;      /* HOST [2]: device time of the half-iteration kernels
                            and of the frame-check kernels, from CUDA events on
                            `stream` around each launch */
  int32_t *launches;     /* HOST [1]: kernels launched by the call */
  /* Teacher-forcing traces of the plain form (product_decode_ex only; the
     batched forms ignore them).  Entry h-1 describes half iteration h; a
     frame's entries past its last half are not written. */
  float *le_trace;       /* device [2 max_iter][n_frames][n_col][n_row]: the
                            extrinsic state L_E = L_APP - lambda after half h,
                            row-major positions (Sec. V-B); the SISO input of
                            half h+1 is lambda = fl32(L_Ch + fl32(alpha L_E)) */
  int32_t *word_queries; /* device [2 max_iter][n_frames][max(n_row, n_col)]:
                            queries of each word decoded in half h (rows in odd
                            halves, columns in even ones; -1 for a non-finite
                            input) */
} product_decode_stats;

/*
 * product_decode with optional statistics and per-half traces (stats may be
 * NULL; same errors).  With traces the call also copies the L_E state after
 * every half (4 n^2 bytes a frame per half).
 */
int product_decode_ex(sogrand_code *row_code, const sogrand_code *col_code, int64_t n_frames, const float *llr_ch,
                      int L, int64_t query_cap, float thr, float alpha, int max_iter, uint8_t *bits,
                      int32_t *half_iters, uint8_t *status, int64_t *queries, product_decode_stats *stats,
                      void *stream);

/*
 * Batched form of product_decode_ex: the whole batch is decoded by one
 * persistent kernel (Sec. VI decoding, same arithmetic, same results as
 * product_decode_ex).  Frames wait in a device-side queue; warps take word
 * tickets from the frame at its head, and the warp that completes a frame's
 * last word of a half runs that frame's row/column check and either finishes
 * the frame or queues it for its next half.  No per-half launches and no
 * host round trips; every frame advances at its own pace.  Waits inside the
 * kernel are bounded (sogrand_set_wait_limits): if a warp finds no work for
 * 2 s of accumulated back-off while frames are unfinished, or cannot take its
 * block's remaining-mass lock, the kernel stops and the call returns
 * SOGRAND_ETIMEOUT.  stats->timing_ms[0] is the kernel's device time;
 * launches counts 2 (queue set-up and the decoder).  Scratch, allocated
 * stream-ordered from the library's pool (see sogrand_release_cached): about
 * 4 n^2 + 8 n ceil(n/64) + 8 max_iter + 37 bytes per frame.  The
 * call synchronises `stream` at its end to read the kernel's status.
 * Errors: as product_decode_ex, plus ETIMEOUT; EINVAL also if
 * n_frames * 2 * max_iter >= 2^31.
 */
int product_decode_persistent(sogrand_code *row_code, const sogrand_code *col_code, int64_t n_frames,
                              const float *llr_ch, int L, int64_t query_cap, float thr, float alpha, int max_iter,
                              uint8_t *bits, int32_t *half_iters, uint8_t *status, int64_t *queries,
                              product_decode_stats *stats, void *stream);

/*
 * Iterative decoding of the (n^2, n^2 - 2n(n-k)) QC-GLDPC code built on a
 * component code (Sec. VI, from Lentmaier et al.): the n^2 bits, as an n x n
 * array X[r][j], form n row words (bit j = X[r][j]) and n wrapped diagonal
 * words (bit j = X[(d + j) mod n][j]), each a codeword of `code`.  Decoding
 * is the batched form of product decoding with diagonals in place of
 * columns: rows in odd halves, diagonals in even halves, L_A = fl32(alpha L_E)
 * of the other set, a frame stopping once every row and diagonal is a
 * codeword.  Arguments and outputs as product_decode_persistent with
 * llr_ch device [n_frames][n][n] (X row-major) and bits the decided array.
 * The paper decodes this code with alpha = 0.6.  Errors: as
 * product_decode_persistent.
 */
int gldpc_decode(sogrand_code *code, int64_t n_frames, const float *llr_ch, int L, int64_t query_cap, float thr,
                 float alpha, int max_iter, uint8_t *bits, int32_t *half_iters, uint8_t *status, int64_t *queries,
                 product_decode_stats *stats, void *stream);

/*
 * Schedule of a code's decoding kernels: the number of resident blocks per SM
 * (128 threads each) they are compiled for, 8 (64 registers a thread) or 12
 * (40 registers).  Which is faster depends on the code (register pressure of
 * its syndrome width and list against the latency the extra warps hide) and
 * is measured by sogrand_code_tune.  The default until tuned: 12 for
 * n <= 64, else 8.
 *   minb     0 (query only), 8 or 12
 *   current  HOST out (may be NULL): the schedule in force
 * Not to be changed while a decode of this code is in flight.  Errors: EINVAL.
 */
int sogrand_code_schedule(sogrand_code *code, int minb, int *current);

/*
 * Where the batched forms keep each block's remaining-mass area (the exact
 * positive-sum fallback of Sec. IV's remaining mass, used by about 1% of
 * component decodings or fewer): 0 in shared memory, 1 in global memory,
 * which leaves the SM's on-chip memory to L1 (faster for long codes and codes
 * with many checks).  The default until tuned: shared for n <= 64 and
 * n - k <= 8, else global; sogrand_code_tune measures both.
 *   where    -1 (query only), 0 or 1
 *   current  HOST out (may be NULL): the placement in force
 * Not to be changed while a decode of this code is in flight.  Errors: EINVAL.
 */
int sogrand_code_dp_area(sogrand_code *code, int where, int *current);

/*
 * Where the query loop takes its patterns (1-line ORBGRAND order, Sec. III-B:
 * increasing cost = sum of reliability ranks + c * Hamming weight, the
 * patterns of one cost and weight being the partitions of that rank sum into
 * distinct parts <= n):
 *   0  read from the code's precomputed order table (one 16-byte entry per
 *      query, copied ahead into shared memory; the default, and the faster);
 *   1  enumerated by the lanes themselves: lane j of a chunk of 32 queries
 *      finds the (cost, weight) group of its query from the order's group
 *      list and unranks its partition with a table of subset counts.
 * Both give the same query order, hence identical results.  Source 1 applies
 * to sogrand_decode and to the batched form of square product codes
 * (product_decode_persistent, product_decode_mixed, product_decode_host, the
 * server) when thr = 0; every other case reads the table, and the
 * remaining-mass computation reads it either way.  Source 1 runs kernels of
 * their own, so the table path's kernels are unaffected by it.
 *   source   -1 (query only), 0 or 1
 *   current  HOST out (may be NULL): the source in force
 * Not to be changed while a decode of this code is in flight.  Errors: EINVAL.
 */
int sogrand_code_order_source(sogrand_code *code, int source, int *current);

/*
 * Autotuner: decodes a sample of frames (device [n_frames][n][n] LLRs, with
 * the decode parameters of the intended workload) with the batched form
 * under each schedule (8 or 12 blocks per SM, each with the remaining-mass
 * area in shared and in global memory), twice each (the first run warms
 * caches), and keeps the fastest for this code.  Synchronous on `stream`;
 * writes no caller buffer but `chosen` (HOST, may be NULL: 8 or 12) and ms_out
 * (HOST [2] or NULL: the better timed run for 8 and for 12 blocks per SM); the
 * chosen placement is read with sogrand_code_dp_area.  Errors: as
 * product_decode_persistent; EINVAL also for n_frames < 1.
 */
int sogrand_code_tune(sogrand_code *code, int64_t n_frames, const float *llr_ch, int L, int64_t query_cap, float thr,
                      float alpha, int max_iter, int *chosen, float *ms_out, void *stream);

/*
 * One group of frames of the mixed form: square product frames of one code.
 * All pointers are device memory of the current device.
 */
#define SOGRAND_MIX_MAX_GROUPS 16
typedef struct {
  sogrand_code *code;   /* row and column code of the group's frames */
  int64_t n_frames;     /* >= 0 */
  const float *llr_ch;  /* [n_frames][n][n] channel LLRs, row-major */
  uint8_t *bits;        /* [n_frames][ceil(n*n/8)] out (required when n_frames > 0) */
  int32_t *half_iters;  /* [n_frames] out, or NULL */
  uint8_t *status;      /* [n_frames] out, or NULL */
  int64_t *queries;     /* [n_frames] out, or NULL */
} sogrand_frame_group;

/*
 * Mixed form of product decoding (Sec. VI turbo decoding of each frame, as
 * product_decode_persistent): frames of up to SOGRAND_MIX_MAX_GROUPS codes of
 * different lengths decoded by ONE launch of a CUDA graph that holds the
 * list set-up of every group and then the batched (persistent) decoder of
 * every group, each with its own frame-half list, chained by programmatic
 * dependent launches.  Each decoder has a full grid; as its work runs out
 * its surplus warps leave, and the next group's decoder starts on the SMs
 * they free, so one code's tail overlaps the next code's decoding (the paper
 * decodes one code at a time; this is a batching form of the same
 * computation).  Every frame's results equal those of
 * product_decode_persistent on that frame alone.  L, query_cap, thr, alpha
 * and max_iter apply to every group.
 *   groups   HOST [n_groups] (read during the call)
 *   stats    optional: weight_sum, xf_words, timing_ms[0] (the graph
 *            launch), launches (1: the graph launch; par_queries is ignored)
 * Synchronous on `stream` (reads the kernels' status).  Errors: EINVAL (as
 * product_decode_persistent for any group, n_groups outside
 * 1..SOGRAND_MIX_MAX_GROUPS), ENOMEM, ECUDA, ETIMEOUT.
 */
int product_decode_mixed(int n_groups, const sogrand_frame_group *groups, int L, int64_t query_cap, float thr,
                         float alpha, int max_iter, product_decode_stats *stats, void *stream);

/*
 * product_decode on HOST buffers: copies llr_ch to the device, decodes with
 * the batched form (product_decode_persistent) and copies the results back
 * before returning.  The batch is split into chunks of 2048 frames, then
 * twice as many each time up to a quarter of the batch (7 chunks for 100,000
 * frames), whose host-to-device copy, decoding (two internal streams, chunks
 * in turn) and device-to-host copy overlap; the internal streams start after the
 * work already queued on `stream`, and `stream` is synchronised before the
 * call returns.  Device buffers come from the library's memory pool and are
 * freed before return.  Pinned host memory makes the copies asynchronous DMA
 * (and lets them overlap decoding); pageable memory works too.
 *   llr_ch     HOST [n_frames][n][n]
 *   bits       HOST [n_frames][ceil(n*n/8)] (required)
 *   half_iters, status, queries  HOST [n_frames] (each may be NULL)
 * Errors: as product_decode_persistent.
 */
int product_decode_host(sogrand_code *row_code, const sogrand_code *col_code, int64_t n_frames,
                        const float *llr_ch, int L, int64_t query_cap, float thr, float alpha, int max_iter,
                        uint8_t *bits, int32_t *half_iters, uint8_t *status, int64_t *queries, void *stream);

/* Size of the fixed device array behind product_decode_noalloc. */
#define SOGRAND_NOALLOC_SCRATCH_BYTES (32u << 20)

/*
 * product_decode for callers that cannot allocate device memory.  The paper
 * has no counterpart: this is a deployment variant.  Some callers may not
 * call cudaMalloc or a stream-ordered allocator: code that runs with a
 * fixed, pre-reserved memory budget (a real-time receiver pipeline, an
 * embedded deployment), or code that must not add allocations, and with them
 * implicit synchronisation, to a stream other work depends on.
 * product_decode_noalloc takes its scratch (extrinsic state, hard decisions,
 * frame flags, about 4 n^2 + 8 n ceil(n/64) + 16 bytes per frame) from one
 * fixed device array of SOGRAND_NOALLOC_SCRATCH_BYTES, which every GPU that
 * loads the library holds until the process exits.  The call allocates
 * nothing: no cudaMalloc, cudaFree or allocating library routine.
 *   arguments and results as for product_decode, except that half_iters,
 *   status and queries are required; every output is device memory.
 *   Only square product codes of one code are accepted: row_code must be
 *   col_code (any other pair returns SOGRAND_EUNSUPPORTED).
 *   The call is asynchronous on `stream` and always launches all 2 *
 *   max_iter half iterations (frames that finished are skipped).
 *   The first call on a device looks up the array's device address on that
 *   device (cudaGetSymbolAddress); make that first call before any stream
 *   capture.  The query-order tables of the code must already cover
 *   query_cap (sogrand_code_create covers 10^4; larger caps need
 *   sogrand_code_reserve first), because growing them allocates.
 *   All calls share the array and it keeps the last call's contents; every
 *   call clears what must start at zero.  Calls that overlap on the GPU (on
 *   different streams, or from different threads) race on the array and
 *   produce wrong results; serialise them.
 * Errors: EUNSUPPORTED when row_code != col_code; EINVAL also when n_frames
 * needs more scratch than the array holds
 * (the bound is 4 n^2 F + 8 n ceil(n/64) F + 16 F bytes plus up to 1280
 * bytes of alignment, within SOGRAND_NOALLOC_SCRATCH_BYTES; for n = 64 about
 * 1980 frames) or when the tables do not cover query_cap; EUNSUPPORTED,
 * ECUDA as for product_decode.  Nothing is written on an argument error.
 */
int product_decode_noalloc(sogrand_code *row_code, const sogrand_code *col_code, int64_t n_frames,
                           const float *llr_ch, int L, int64_t query_cap, float thr, float alpha, int max_iter,
                           uint8_t *bits, int32_t *half_iters, uint8_t *status, int64_t *queries, void *stream);

/*
 * Test hook: the device's canonical query order for one word, from the
 * order table or, with sogrand_code_order_source(code, 1), as the lanes
 * enumerate it.
 *   llr          HOST [n] lambda values
 *   max_q        number of queries to list, >= 1
 *   patterns_out HOST [max_q][ceil(n/64)] u64 noise patterns in RANK space:
 *                bit r-1 set = the bit of reliability rank r is flipped
 *   n_out        HOST: number written (fewer than max_q if the class ends)
 *   c_out        HOST: the 1-line parameter used (may be NULL)
 * Synchronous.  Errors: EINVAL, ENOMEM, ECUDA.
 */
int sogrand_trace_patterns(sogrand_code *code, const float *llr, int64_t max_q, uint64_t *patterns_out,
                           int64_t *n_out, int32_t *c_out);

/*
 * Serving loop: continuous batching of product-decode requests (the turbo
 * decoder of Sec. VI as a service; the paper has no serving system).
 *
 * A server owns, per registered code, a device pool of `slots[i]` frame slots
 * (channel LLRs, L_E state, hard decisions and counters of a frame stay
 * resident there across half iterations: about 8 n^2 + 8 n ceil(n/64) +
 * n^2/8 + 16 max_iter + 60 bytes a slot, allocated at creation: the memory
 * budget).  A worker thread drives each pool: when its previous launch has
 * finished it retires the frames that stopped, completes requests whose last
 * frame stopped (copying their outputs to the caller's host buffers), admits
 * waiting requests of that code in arrival order while free slots last
 * (copying their LLRs in), and launches the batched decoder over every
 * resident frame for at most `epoch_halves` half iterations; frames that need
 * more stay parked in their slots.  Pools launch on their own streams, so
 * requests of different codes decode concurrently, and a request that arrives
 * while others are decoding joins at its pool's next epoch.  Every frame runs
 * the arithmetic of product_decode_persistent, so its results are the same
 * alone and in any mix.  Decode parameters are the server's.
 *
 *   codes[n_codes]   registered codes (1..16; each is the row and column code
 *                    of its requests); slots[n_codes] frames each pool holds
 *   epoch_halves     1 .. 2 max_iter
 * Errors: EINVAL, ENOMEM (a pool does not fit), ECUDA.
 */
typedef struct sogrand_server sogrand_server;
int sogrand_server_create(int n_codes, sogrand_code *const *codes, const int64_t *slots, int L, int64_t query_cap,
                          float thr, float alpha, int max_iter, int epoch_halves, sogrand_server **out);

/*
 * Queue a request of n_frames frames of registered code `code_index`.
 *   llr        HOST [n_frames][n][n] channel LLRs (pinned memory recommended);
 *              read when the request is admitted: keep it until completion
 *   bits       HOST [n_frames][ceil(n*n/8)] out (required)
 *   half_iters, status, queries  HOST [n_frames] out, or NULL
 *   ticket     HOST out: identifies the request for sogrand_server_wait
 * Outputs are written before the request is reported done.  Errors: EINVAL
 * (bad arguments, n_frames above the pool's slots, server stopping), the
 * server's error if it has failed.
 */
int sogrand_server_submit(sogrand_server *server, int code_index, int64_t n_frames, const float *llr, uint8_t *bits,
                          int32_t *half_iters, uint8_t *status, int64_t *queries, int64_t *ticket);

/*
 * Wait up to timeout_ms (<= 0: do not wait) for a request.  *done = 1 when it
 * has completed; then *latency_ms (may be NULL) is the time from submission to
 * completion (outputs in host memory) and the request's record is released
 * (a ticket is reported done once).  Returns the request's status once done
 * (SOGRAND_OK, ETIMEOUT if its launch hit the bounded-wait limit, ECUDA),
 * else SOGRAND_OK.  Errors: EINVAL (unknown or already reported ticket).
 */
int sogrand_server_wait(sogrand_server *server, int64_t ticket, int timeout_ms, int *done, double *latency_ms);

/* Counters (each may be NULL).  Returns the server's error state. */
int sogrand_server_stats(sogrand_server *server, int64_t *launches, int64_t *frames_done, int64_t *requests_done,
                         int64_t *frames_resident, int64_t *requests_waiting);

/* Finish every submitted request, stop the worker and free the pools.
 * Returns the server's error state. */
int sogrand_server_destroy(sogrand_server *server);

/*
 * Device scratch of the decoders (the per-frame L_E state and counters) comes
 * from one stream-ordered memory pool per device that the library creates on
 * first use and that keeps freed memory for the next call.  This returns the
 * idle memory of every such pool to the device.  Call it once the streams
 * that used the library are synchronised (memory whose stream-ordered free
 * has not yet run stays in the pool).  Errors: ECUDA.
 */
int sogrand_release_cached(void);

/*
 * Integer-pipe throughput of the current device: 32-bit LOP3 (three-input
 * logic) and IADD instructions retired per second by every SM at full
 * occupancy, from a timed kernel of independent dependency chains
 * (trips x 128 such instructions per thread).  The decoders' ceiling: their
 * work is integer and logic instructions.  Synchronous on `stream`.
 *   trips      loop trips, 1 .. 2^30 (about 1.5e5 runs for tens of ms)
 *   ops_per_s  HOST out: lane-operations per second
 *   ms_out     HOST out (may be NULL): the timed kernel's duration
 * Errors: EINVAL, ECUDA.
 */
int sogrand_int_peak(int64_t trips, double *ops_per_s, double *ms_out, void *stream);

/* Static text for an error code. */
const char *sogrand_strerror(int err);

#ifdef __cplusplus
}
#endif

#endif /* SOGRAND_H */
