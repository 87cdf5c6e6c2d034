/*
 * perm_f3.h -- C ABI of the GB300 library for permanents over F3
 * (D. Scheinerman, "Fast computation of permanents over F3 via F2
 * arithmetic", arXiv 2407.20205).
 *
 * perm(A) for A in F3^{n x n}, n <= 64, by Ryser's formula (Eq. (2)) walked in
 * reflected-binary Gray-code order (Sec. 3), each row-subset sum held as the
 * paper's bit-sliced (mag, sgn) pair (Sec. 2, Definition 2.1), one launch per
 * call on the current CUDA device.
 *
 * Conventions shared by every entry point:
 *   - A matrix is n*n bytes, row-major, entries in {0,1,2} where 2 stands for
 *     -1 (the paper's alphabet is {-1,0,1}, Sec. 3).  An entry above 2 is an
 *     error (PF3_EDOMAIN); the paper's packing routine asserts the same
 *     (appendix, conversion to the bipedal pair).
 *   - Results are perm(A) mod 3 in {0,1,2} (-1 is returned as 2).
 *   - Counts: for Gray index i (subset gray(i) = i ^ (i >> 1), Sec. 3.1
 *     footnote) the Ryser term is (-1)^{|S|} * prod(subset sum) in {-1,0,1}.
 *     "plus" counts the indices whose term is +1, "minus" those whose term is
 *     -1; perm(A) = (-1)^n (plus - minus) mod 3.  Counts are exact 64-bit
 *     integers.  The subsets are ROW subsets, as in the paper's code (Sec. 3),
 *     which equals Eq. (2)'s column form because perm(A) = perm(A^T).
 *   - n = 0: perm is 1 (the empty product; the paper is silent) and A may be
 *     NULL.
 *   - Host-pointer entry points (perm_f3, perm_f3_counts, perm_f3_range_counts,
 *     perm_f3_batch) copy their inputs before returning, are synchronous, and
 *     leave outputs untouched on error.  The library owns its device scratch;
 *     calls are serialised per device.
 *   - Device-pointer entry points (suffix _async) are stream-ordered on the
 *     given cudaStream_t (NULL = legacy default stream); they return once the
 *     work is enqueued.  The caller owns every pointer passed in.  They share
 *     the device's scratch with each other and with the host-pointer calls;
 *     the library orders every use of it after the previous one (an event
 *     recorded after each launch, waited for by the next, on whatever
 *     stream), so calls on different streams are correct but do not run
 *     concurrently.  Inside a stream capture that ordering is left out and
 *     the capturing caller must order the calls itself.
 *   - Return value: >= 0 on success, a negative PF3_E* code on failure.
 */
#ifndef PERM_F3_H
#define PERM_F3_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PF3_OK 0
#define PF3_PENDING 1        /* perm_f3_poll: job not finished yet */
#define PF3_EINVAL (-1)      /* null pointer, n outside 0..64, first > last, bad size */
#define PF3_EDOMAIN (-2)     /* a matrix entry outside {0,1,2} */
#define PF3_ECUDA (-3)       /* a CUDA runtime call failed (no device, launch error) */
#define PF3_ENOMEM (-4)      /* device or pinned host allocation failed */
#define PF3_ETIMEDOUT (-5)   /* perm_f3_wait: the deadline passed */
#define PF3_ECANCELED (-6)   /* the job or context was cancelled */
#define PF3_EBUSY (-7)       /* perm_f3_submit: the request queue is full */
#define PF3_ETOOBIG (-8)     /* request larger than a fixed buffer: no-allocation scratch, output array */

#define PF3_MAX_N 64
/* Widest merged matrix counted by column-sum vector (pf3_class_counts): its
 * table holds 2 * 3^8 counters. */
#define PF3_CLASS_MAX_COLS 8
/* Most matrices in one batch call (work items index matrices with 32-bit
 * integers); larger counts are rejected with PF3_EINVAL. */
#define PF3_MAX_BATCH 2147483583LL

/* Human-readable text for a return code (static storage). */
const char* pf3_strerror(int code);

/* Library version string (static storage). */
const char* pf3_version(void);

/* ------------------------------------------------------------ one matrix */

/* perm(A) mod 3 (Eq. (2), Sec. 3).  A: host, n*n bytes.  Returns 0, 1 or 2,
 * or a negative PF3_E* code. */
int perm_f3(const uint8_t* A, int n);

/* The final map of Eq. (2) (with the closing cmod3 of Sec. 3): perm(A) =
 * (-1)^n (plus - minus) mod 3, returned in {0,1,2}, for the exact term counts
 * of an n x n matrix (sums of perm_f3_range_counts over disjoint ranges, e.g.
 * from several processes).  Counts are unsigned 64-bit: each is reduced mod 3
 * on its own, so counts of 2^63 and above (n = 64) are exact.  Host only; no
 * device is touched.  PF3_EINVAL when n is outside 0..64. */
int pf3_perm_from_counts(int n, uint64_t plus, uint64_t minus);

/* Term counts over all 2^n Gray indices (the exact sum behind perm_f3).
 * plus/minus: host outputs.  For n = 0, plus = 1 and minus = 0. */
int perm_f3_counts(const uint8_t* A, int n, uint64_t* plus, uint64_t* minus);

/* Term counts over the Gray indices first..last inclusive (0 <= first <= last
 * <= 2^n - 1; for n = 64 last may be UINT64_MAX).  This is the per-job block
 * sum of Sec. 3.1: disjoint ranges add up to perm_f3_counts.  n >= 1. */
int perm_f3_range_counts(const uint8_t* A, int n, uint64_t first, uint64_t last, uint64_t* plus,
                         uint64_t* minus);

/* Device-pointer form of perm_f3_range_counts (and, with first = 0 and
 * last = 2^n - 1, of perm_f3).  dA: device, n*n bytes.  d_out: device,
 * 3 x uint64: plus, minus, and perm mod 3 in {0,1,2} -- or UINT64_MAX there
 * when an entry of dA is outside {0,1,2} (then plus = minus = 0).  n >= 1.
 * stream: a cudaStream_t. */
int perm_f3_range_counts_async(const uint8_t* dA, int n, uint64_t first, uint64_t last, uint64_t* d_out,
                               void* stream);

/* No-allocation form of perm_f3_range_counts_async, for callers that must not
 * let a library allocate device memory -- for instance a process whose memory
 * manager reserves the whole GPU up front and forbids allocations it did not
 * make, or a latency-sensitive caller that cannot afford cudaMalloc/cudaFree,
 * which may synchronise the whole device.  (The paper has no counterpart: this
 * is a library-interface concern.)  Same arguments, results and stream
 * ordering as perm_f3_range_counts_async; the caller owns dA and d_out.  The
 * kernel's scratch lives in a fixed device array inside the library
 * (PF3_NOALLOC_MAX_CTAS * 16 + 256 bytes, held by every GPU that loads the
 * library until the process exits), so this entry point never calls
 * cudaMalloc or cudaFree.  ctas: CTAs to launch, 0 = one resident wave;
 * values above PF3_NOALLOC_MAX_CTAS are rejected with PF3_ETOOBIG.  The first
 * call on each device looks up the array's device address and the kernel's
 * occupancy; make that first call before any stream capture.  That address
 * is kept for the life of the process: after a cudaDeviceReset by the caller
 * it is stale, so a process that resets a device must not call this entry
 * point on it again.  All calls on a device share the array (each call clears
 * its flags first): calls that overlap on the GPU race and must be ordered by
 * the caller. */
#define PF3_NOALLOC_MAX_CTAS 1024
int perm_f3_range_counts_noalloc(const uint8_t* dA, int n, uint64_t first, uint64_t last, uint64_t* d_out,
                                 int ctas, void* stream);

/* Long walks in bounded launches (Sec. 3.1's split of the Gray range into
 * jobs, here consecutive launches of at most 2^chunk_log2 indices each,
 * 10 <= chunk_log2 <= PF3_LONGRUN_MAX_CHUNK_LOG2, so that one launch lasts
 * seconds at most and cancellation and max_seconds are seen often).  The
 * device is held for one launch at a time: other calls on it interleave.
 * After every launch the exact counts and the next Gray index are written to
 * checkpoint_path (temporary file + rename; NULL = no checkpoint).  If the
 * file already holds a checkpoint of the same matrix, the walk resumes from
 * it; one of another matrix is refused (PF3_EINVAL).  Stops between launches
 * when max_seconds (> 0) of wall time have passed (PF3_ETIMEDOUT; checked
 * after each launch, so every call makes at least one launch of progress) or
 * when pf3_longrun_cancel(1) was called (PF3_ECANCELED; checked before each
 * launch); the counts so far are returned and saved either way.  *finished = 1 once the whole range is done;
 * *next_index is the first index not yet walked (0 when finished).  result
 * (may be NULL): perm(A) mod 3 in {0,1,2} once finished, untouched before.
 * A fresh run (no checkpoint to resume) of a matrix whose equal columns merge
 * into at most pf3_get_class_limit() columns (n > 32) is counted by column-sum
 * vector (pf3_class_counts) in one launch instead. */
#define PF3_LONGRUN_MAX_CHUNK_LOG2 44
int pf3_longrun(const uint8_t* A, int n, int chunk_log2, const char* checkpoint_path, double max_seconds,
                uint64_t* plus, uint64_t* minus, uint64_t* next_index, int* finished, int* result);

/* Set (1) or clear (0) the flag that makes pf3_longrun stop at its next
 * launch boundary; callable from any thread. */
void pf3_longrun_cancel(int on);

/* ------------------------------------------------------------ batches */

/* perm mod 3 of `count` matrices in one call.  As: host, the matrices back to
 * back, matrix k (size ns[k] x ns[k]) starting at byte sum_{j<k} ns[j]^2.
 * results: host, count bytes.  hist: optional host uint64[3], the number of
 * results equal to 0, 1 and 2 (the Monte Carlo statistic of Sec. 4).  Matrices
 * of different n may be mixed.  0 <= count <= PF3_MAX_BATCH.  Returns 0 or a
 * negative code. */
int perm_f3_batch(const uint8_t* As, const int32_t* ns, int64_t count, uint8_t* results, uint64_t* hist);

/* Device-pointer batch: dAs, d_results (count bytes) and d_hist (3 x uint64,
 * overwritten) on the device; ns and the matrix offsets are read from the HOST
 * array ns (the library builds its work plan from them).  Stream-ordered on
 * `stream`; an entry outside {0,1,2} gives result 255 for that matrix.  The
 * launch sequence (item-table upload, counter resets, one persistent kernel
 * per plane width) is captured as a CUDA graph; a later call with the same ns,
 * pointers and tuning replays the graph without re-planning, reading the
 * current contents of dAs.  0 <= count <= PF3_MAX_BATCH. */
int perm_f3_batch_async(const uint8_t* dAs, const int32_t* ns, int64_t count, uint8_t* d_results,
                        uint64_t* d_hist, void* stream);

/* Table 2 (Sec. 4): perm mod 3 of every one of the 3^(n^2) matrices in
 * F3^{n x n}, n in 1..5, counted by value: counts[v] = #{A : perm(A) = v}
 * (counts[0] = z(n)).  Matrices are generated on the device from their
 * index; runs in bounded launches (n = 5: 8.47e11 matrices). */
int pf3_count_exhaustive(int n, uint64_t* counts);

/* ------------------------------------------------------------ serving */

/* A request loop for streams of permanents (the Monte Carlo use of Sec. 4):
 * requests are admitted as device slots free up, each request's Gray range is
 * cut into work items of 2^chunk_log2 indices (Sec. 3.1 blocks), and every
 * launch of the batch kernel runs items of many requests under a work budget:
 * first every request whose remaining work is at most 2^small_work_log2 Gray
 * indices (least remaining first), then the others in arrival order.
 * Matrices and partial counts stay on the device until a request finishes.
 * A context is driven by its own host thread; all calls are thread-safe. */
typedef struct pf3_config {
    int32_t max_jobs;        /* device slots (requests resident at once); default 4096 */
    int32_t queue_depth;     /* requests waiting for a slot before PF3_EBUSY; default 2^20 */
    int32_t chunk_log2;      /* Gray indices per work item (log2); default 22 */
    int32_t launch_items;    /* work items per launch at most; default 16384 */
    int32_t max_admit;       /* requests admitted per launch at most; default 1024 */
    int32_t small_work_log2; /* requests with at most 2^small_work_log2 Gray indices left
                                are served first, least remaining first; the others
                                in arrival order (0..64); default 33 */
    uint64_t launch_budget;  /* Gray indices per launch (soft cap); default 2^33 */
    int32_t class_max_cols;  /* a request whose merged matrix (n > 32) has at most this
                                many columns is counted by column-sum vector
                                (pf3_class_counts) in the launch that admits it, not
                                walked; 0..PF3_CLASS_MAX_COLS, default PF3_CLASS_MAX_COLS */
} pf3_config;

typedef struct pf3_ctx pf3_ctx;

/* Fill cfg with the defaults above. */
void pf3_config_default(pf3_config* cfg);

/* Create a serving context on the current device (cfg NULL = defaults). */
int pf3_create(pf3_ctx** ctx, const pf3_config* cfg);

/* Finish admitted requests, cancel queued ones (PF3_ECANCELED), free all.
 * No other thread may use ctx during or after this call. */
void pf3_destroy(pf3_ctx* ctx);

/* Cancel every request still waiting for a slot (they report PF3_ECANCELED);
 * admitted requests run to completion.  Returns how many were cancelled. */
int pf3_cancel_queued(pf3_ctx* ctx);

/* Queue perm(A) mod 3; A (host, n*n bytes) is copied.  Returns a ticket >= 0,
 * or PF3_EBUSY when queue_depth requests are already waiting, PF3_EDOMAIN /
 * PF3_EINVAL on bad input. */
int64_t perm_f3_submit(pf3_ctx* ctx, const uint8_t* A, int n);

/* PF3_OK with *result set, PF3_PENDING, or the request's error code. */
int perm_f3_poll(pf3_ctx* ctx, int64_t ticket, uint8_t* result);

/* Block until the request finishes or timeout_us passes (negative: no
 * limit).  PF3_OK, PF3_ETIMEDOUT or the request's error code. */
int perm_f3_wait(pf3_ctx* ctx, int64_t ticket, uint8_t* result, int64_t timeout_us);

/* Host steady-clock times (ns) of submission and of the result becoming
 * visible; PF3_PENDING while unfinished. */
int pf3_job_times(pf3_ctx* ctx, int64_t ticket, uint64_t* submit_ns, uint64_t* done_ns);

/* Launches issued, work items run and requests finished so far. */
int pf3_serve_stats(pf3_ctx* ctx, uint64_t* launches, uint64_t* items, uint64_t* jobs_done);

/* The serving loop's choice of work items on the host alone (no device is
 * touched): requests of ns[k] rows and ms[k] columns (ms NULL: ms = ns; fewer
 * columns stand for a request whose equal columns were merged), all admitted
 * in index order, planned under cfg (NULL = defaults) with Gray blocks of
 * 2^U[0] indices for one plane word and 2^U[1] for two, for `launches`
 * consecutive launches (fewer when every item has been issued).  items (host,
 * capacity entries; NULL to ask for the count only) receive the items in the
 * order each launch issues them: request index, launch, class (0 one word, 1
 * two), first block and number of blocks (0 blocks: the whole request by one
 * lane), block_log2, and last = 1 on a request's final item.  *num_items
 * receives their number.  PF3_EINVAL on a bad argument, PF3_ETOOBIG when
 * capacity is too small (nothing written to items). */
typedef struct {
    int64_t request;
    int32_t launch;
    int32_t cls;
    uint64_t first_block;
    uint64_t num_blocks;
    int32_t block_log2;
    int32_t last;
} pf3_serve_item;
int pf3_serve_plan(const int32_t* ns, const int32_t* ms, int64_t count, const pf3_config* cfg, const int* U,
                   int launches, pf3_serve_item* items, int64_t capacity, int64_t* num_items);

/* The steady clock the serving times use (ns). */
uint64_t pf3_now_ns(void);

/* ------------------------------------------------------------ bipedal vectors */

/* Elementwise operations on bipedal vectors (Sec. 2, Theorem 2.1): `count`
 * vectors of length n.  A vector takes w = ceil(n / 64) host words per plane
 * (the footnote of Sec. 3 on rows longer than a machine word): vector k is
 * words k*w .. k*w + w - 1 of m1/s1 (and of m2/s2), column j in bit j % 64 of
 * its word j / 64.  The result (m3, s3), same layout, is a bipedal
 * representation of the sum, difference, pointwise product or pointwise
 * quotient (quotient: meaningful where the divisor is nonzero).  Inputs may
 * use either representation of 0; bits at and above n are cleared in the
 * results.  1 <= n <= PF3_VEC_MAX_N and count * w <= PF3_VEC_MAX_WORDS,
 * else PF3_EINVAL.  Off the permanent's path. */
#define PF3_OP_ADD 0
#define PF3_OP_SUB 1
#define PF3_OP_MUL 2
#define PF3_OP_DIV 3
#define PF3_VEC_MAX_N (1 << 24)
#define PF3_VEC_MAX_WORDS (1LL << 31)
int pf3_vec_op(int op, int n, int64_t count, const uint64_t* m1, const uint64_t* s1, const uint64_t* m2,
               const uint64_t* s2, uint64_t* m3, uint64_t* s3);

/* psi of Sec. 2: vectors (mag, sgn) in the layout above back to entries
 * {0,1,2} (2 == -1).  out: host, count * n bytes, vector k's entries at
 * out[k*n .. k*n + n). */
int pf3_vec_unpack(int n, int64_t count, const uint64_t* mag, const uint64_t* sgn, uint8_t* out);

/* phi of Sec. 2: count vectors of n entries in {0,1,2} (host, count * n
 * bytes, vector k at in[k*n ..]) to (mag, sgn) in the layout above (host,
 * count * ceil(n / 64) words each; bits at and above n are 0).  An entry
 * above 2 gives PF3_EDOMAIN and leaves mag and sgn untouched. */
int pf3_vec_pack(int n, int64_t count, const uint8_t* in, uint64_t* mag, uint64_t* sgn);

/* ------------------------------------------------------------ diagnostics */

/* The row step on every case: for state s in 0..3 ((mag, sgn) = (s>>1, s&1)),
 * constant c in {0,1,2} and direction d (0 add, 1 subtract), writes
 * out[((s*3 + c)*2 + d)*2 + {0,1}] = (mag', sgn'), 48 host uint32 (Sec. 2,
 * Theorem 2.1 / Table 1 semantics). */
int pf3_step_table(uint32_t* out);

/* The bit planes of A as the kernels pack them (phi of Sec. 2): column j is
 * bit j, least significant first.  mag, sgn: host, n uint64 each. */
int pf3_pack(const uint8_t* A, int n, uint64_t* mag, uint64_t* sgn);

/* The column merge the host-pointer single-matrix calls (perm_f3,
 * perm_f3_counts, perm_f3_range_counts, pf3_longrun) apply before walking:
 * columns equal up to a factor -1 are one class; a class of odd multiplicity
 * is kept once and one of even multiplicity twice (in F3, x^mult is x or x^2),
 * each as its canonical vector (first nonzero entry 1).  Every Ryser term of
 * the merged n x m matrix B (n rows, the same row subsets) equals A's times
 * the product of the factors, (-1)^negate, so the +1/-1 counts are A's,
 * swapped when negate is 1.  The library merges when n > 32 and m <= 32 (one
 * plane word instead of two: matrices with many equal columns are those whose
 * terms are mostly nonzero).  A: host, n*n bytes; B: host, room for n*32
 * bytes, row-major n x m.  Returns 1 and fills B, m and negate when it merges,
 * 0 when it does not (nothing written), or a negative code.  Host only; no
 * device is touched.  (Not in the paper: an exact rewriting of Eq. (2).) */
int pf3_column_merge(const uint8_t* A, int n, uint8_t* B, int* m, int* negate);

/* Ryser counts (plus, minus as above) of A by column-sum vector.  A term
 * depends on its row subset S only through the column sums over S (a point
 * of F3^m) and the parity of |S|; the number of subsets on each of those
 * 2 * 3^m pairs follows row by row, and the counts are read off the pairs
 * whose sums are all nonzero.  Exactly the walk's counts, in n * 3^m steps
 * instead of 2^n.  A's columns are first merged as by pf3_column_merge (here
 * for any n); when the merged matrix has at most PF3_CLASS_MAX_COLS columns
 * the counts are computed on the device (one CTA) and 1 is returned, else 0
 * and nothing is written.  A: host, n*n bytes, 1 <= n <= 64.  perm_f3,
 * perm_f3_counts, pf3_longrun (a fresh run) and the serving contexts take
 * this route for n > 32 when the merged width is at most the limit set by
 * pf3_set_class_limit (perm_f3 and the long run) or pf3_config.class_max_cols
 * (serving).  (Not in the paper: an exact regrouping of Eq. (2)'s sum.) */
int pf3_class_counts(const uint8_t* A, int n, uint64_t* plus, uint64_t* minus);

/* Widest merged matrix (0..PF3_CLASS_MAX_COLS) that perm_f3, perm_f3_counts
 * and a fresh pf3_longrun count by column-sum vector instead of walking, on
 * the current device; 0 walks every matrix.  Default PF3_CLASS_MAX_COLS.
 * pf3_get_class_limit returns the current value or a negative code. */
int pf3_set_class_limit(int max_cols);
int pf3_get_class_limit(void);

/* Integer-pipe microbenchmark (the roofline denominator of the walk).  kind:
 * 0 LOP3, 1 IMAD, 2 IADD, 3 LOP3+IMAD, 4 full row step (3 LOP3 + compare),
 * 5 POPC, 6 MAX(+IMAD), 7 2 LOP3 + MAX, 8 probe (2 LOP3 + compare),
 * 9 row step + IMAD, 10 2 LOP3 + IADD, 11 probe with inverted gate tested
 * against zero, 12 probe tested against all ones, 13 inverted probe with an AND
 * chain of "nonzero" (2 LOP3 + compare each).
 * Runs `ctas_per_sm` CTAs of `threads` threads per SM for `iters` rounds and
 * reports instructions per clock per SM (thread instructions, i.e. lanes),
 * thread instructions per second over the whole GPU, and the SM clock in MHz
 * the CTAs saw.  Any output pointer may be NULL. */
int pf3_intpipe_bench(int kind, int ctas_per_sm, int threads, int iters, double* inst_per_clk_per_sm,
                      double* inst_per_s, double* sm_mhz);

/* Device facts the roofline uses: SM count and the current device index. */
int pf3_device_info(int* sm_count, int* device);

/* ------------------------------------------------------------ tuning */

/* Kernel variants (probe group and unrolled block lengths, register budget,
 * CTA size).  which: 0 = single-matrix kernel, 1 = batch kernel, 2 =
 * single-matrix kernel for launches of fewer than 2^28 Gray indices (their
 * own size class: there the fixed costs of a launch decide), 3 = single-matrix
 * kernel for long launches of a matrix whose equal columns were merged (see
 * pf3_column_merge; W = 1 only: such matrices have mostly nonzero terms).
 * W: words per plane (1 for up to 32 columns, 2 for up to 64).
 * pf3_set_variant(0, W, v) sets both single-matrix size classes; (2, W, v)
 * only the short one; (3, 1, v) the merged class; pf3_get_variant(0, W)
 * reads the long class.  Results never depend on the variant, only speed
 * does. */
int pf3_variant_count(int which);
int pf3_set_variant(int which, int W, int v);
int pf3_get_variant(int which, int W);

/* Shape of variant v: unrolled block 2^U Gray indices, probe group 2^G
 * indices per carried base state, minimum resident CTAs per SM. */
int pf3_variant_info(int which, int v, int* U, int* G, int* min_ctas);

/* Threads per CTA of variant v (which as above), or PF3_EINVAL. */
int pf3_variant_threads(int which, int v);

/* Batch work split: matrices with n > cutoff are cut into work items of
 * 2^chunk_log2 Gray indices (Sec. 3.1 blocks); others are one item each.
 * chunk_log2 in 12..62, or 0 for the automatic split (see
 * pf3_set_batch_tuning; cutoff is then unused).  PF3_EINVAL otherwise. */
int pf3_set_batch_split(int cutoff, int chunk_log2);

/* All batch planning parameters (the autotuner sets tiny_cutoff and
 * items_per_warp and selects the automatic split):
 *   tiny_cutoff     0..PF3_TINY_MAX_N: matrices with n <= tiny_cutoff are
 *                   packed 32 to a warp and walked one per lane (the packing
 *                   cutoff); larger ones get at least a whole warp;
 *   split_cutoff    0..64, chunk_log2 12..62: fixed split, as
 *                   pf3_set_batch_split;
 *   chunk_log2 = 0  guided split: per plane width, the non-packed matrices
 *                   are taken largest first (2^n Gray indices each) and each
 *                   is cut into items (Sec. 3.1 blocks) no longer than the
 *                   work from that matrix to the end of the order divided by
 *                   (warps of the persistent grid x items_per_warp), rounded
 *                   down to a power of two and at least 2^20 indices, so the
 *                   last items handed out are short and the warps finish
 *                   together;
 *   items_per_warp  1..1024, the divisor of the guided split.
 * Results never depend on these, only speed does.  PF3_EINVAL on a value out
 * of range. */
#define PF3_TINY_MAX_N 16
int pf3_set_batch_tuning(int tiny_cutoff, int split_cutoff, int chunk_log2, int items_per_warp);
int pf3_get_batch_tuning(int* tiny_cutoff, int* split_cutoff, int* chunk_log2, int* items_per_warp);

/* One work item of a batch plan (diagnostic view).  kind: 0 = a whole matrix
 * walked by one warp, 1 = one piece of a split matrix, 2 = a packed group of
 * num_blocks consecutive matrices (index mat, mat + 1, ...) of the same n
 * walked one per lane, 3 = a matrix with n <= block_log2 walked by one lane.
 * Kinds 0 and 1 cover Gray indices [first_block, first_block + num_blocks) x
 * 2^block_log2 of matrix mat; cls is 0 for n <= 32 (one word per plane), 1
 * otherwise. */
typedef struct {
    int64_t mat;
    int32_t n;
    int32_t kind;
    uint64_t first_block;
    uint64_t num_blocks;
    int32_t block_log2;
    int32_t cls;
} pf3_plan_item;

/* The batch planner on the host alone (no device is touched): the work items
 * perm_f3_batch would launch for sizes ns[count] under the given tuning
 * (tiny_cutoff, split_cutoff, chunk_log2, items_per_warp as
 * pf3_set_batch_tuning), batch kernel variants variant[2] and persistent grids
 * of warps[2] warps, in launch order per class (class 1 first, each sorted
 * largest first).  items (host, capacity entries) may be NULL to ask for the
 * count only; *num_items receives the number of items; auto_chunk_log2[2]
 * (may be NULL) receives, per class, log2 of the longest item of its largest
 * matrix (0 for a class without such matrices).  PF3_EINVAL on a bad argument, PF3_ETOOBIG when
 * capacity < *num_items (nothing written to items). */
int pf3_batch_plan(const int32_t* ns, int64_t count, int tiny_cutoff, int split_cutoff, int chunk_log2,
                   int items_per_warp, const int* variant, const int* warps, pf3_plan_item* items, int64_t capacity,
                   int64_t* num_items, int* auto_chunk_log2);

/* The single-matrix launch plan on the host alone (no device is touched):
 * how Gray indices [first, last] of an n x n matrix are cut for variant
 * `variant` of the single-matrix kernel on `grid` CTAs (Sec. 3.1's blocks of
 * consecutive Gray states).  info (host, 12 uint64) receives: has_head,
 * head_first, head_last (indices walked one by one before the first whole
 * block), has_tail, tail_first, tail_last (after the last one), mid_B0,
 * mid_NB (the whole blocks of 2^U indices in between), dynamic (1: warps take
 * chunks of blocks from an atomic cursor; 0: each thread walks one contiguous
 * share), U, threads per CTA, nchunks.  When dynamic, chunk_first/chunk_len
 * (host, capacity entries each; both NULL to ask for the count only) receive
 * each chunk's first block (relative to mid_B0) and length in blocks, in the
 * order warps take them; *num_chunks receives their number (0 when not
 * dynamic).  PF3_EINVAL on a bad argument, PF3_ETOOBIG when capacity is too
 * small. */
int pf3_range_plan(int n, uint64_t first, uint64_t last, int variant, int grid, uint64_t* info,
                   uint64_t* chunk_first, uint64_t* chunk_len, int64_t capacity, int64_t* num_chunks);

/* Time every variant on the current device and keep the fastest per W (a
 * variant replaces the current choice, variant 0 first, only when it is at
 * least 1 % faster) (single-matrix kernel: n = 32 over 2^31 Gray indices for W = 1, n = 40 over
 * 2^36 for W = 2, for the short-launch class n = 24 over 2^24 and n = 36
 * over 2^27, and for the merged class J_36 merged to 36 x 2 over 2^33; batch
 * kernel: 8192 matrices of n = 24 and 32 of n = 33 under the guided split),
 * then pick the batch packing cutoff and split granularity
 * (pf3_autotune_ex).
 * single_ms (pf3_variant_count(0) * 2 doubles) and batch_ms
 * (pf3_variant_count(1) * 2 doubles) receive the variant timings, W = 1
 * first; either may be NULL.  Takes a few seconds.  When the environment
 * variable PF3_TUNE_CACHE names a file, the choice is stored there under the
 * GPU's name and SM count, and later processes load it when they first use
 * the device. */
int pf3_autotune(double* single_ms, double* batch_ms);

/* pf3_autotune with the timings of all its stages.  single_short_ms
 * (pf3_variant_count(2) * 2 doubles, may be NULL): the short-launch class, per
 * variant, W = 1 first.  The batch planning stages:
 * pack_ms (2 * (PF3_TINY_MAX_N + 1) doubles, may be NULL): [n] the packed
 * walk and [PF3_TINY_MAX_N + 1 + n] the warp walk of a full grid of n x n
 * matrices, for n from the W = 1 batch variant's U + 1 up to the first n at
 * which the warp walk is as fast (0 where not timed); the packing cutoff is
 * the last n at which the packed walk was faster (at least min(U, 16)).
 * split_ms (PF3_SPLIT_CANDIDATES doubles, may be NULL): three batches
 * (3000 x n = 26; 300 x 28 + 600 x 26 + 1200 x 24; 20 x 33 + 6 x 34) under
 * the guided split with items_per_warp 1, 2, 4, 8, 16; the fastest total is
 * kept, ties within 1 % going to fewer items.  Takes a few seconds. */
#define PF3_SPLIT_CANDIDATES 5
int pf3_autotune_ex(double* single_ms, double* single_short_ms, double* batch_ms, double* pack_ms,
                    double* split_ms);

#ifdef __cplusplus
}
#endif

#endif /* PERM_F3_H */
