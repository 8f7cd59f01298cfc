/*
 * messi.h -- C ABI of the GB300 exact k-NN engine over an in-memory iSAX
 * index (MESSI, arXiv 2110.07519).
 *
 * Problem (Sec. 2.1, "Similarity Search"): given a collection of N series of
 * length len and a query series of the same length, return the k series with
 * the smallest Euclidean distance (ED) or Dynamic Time Warping distance under
 * a Sakoe-Chiba window (DTW, Sec. 3.4).  The answer is exact: ids and
 * distances equal a brute-force scan (Theorem 2, Sec. 4), with ties between
 * equal distances broken by the lowest original id.
 *
 * Conventions for every call:
 *   - Returns a messi_status; nothing throws.  On failure messi_last_error()
 *     gives a thread-local message.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Device work is stream-ordered; a call returns once its work
 *     is queued, except where its comment says it synchronises.
 *   - Pointers named "device or host" may point to either; host pointers
 *     are detected with cudaPointerGetAttributes and staged through device
 *     buffers inside the call, which then synchronises `stream` before it
 *     returns so the host outputs are valid.
 *   - Series are row-major float32 [n][len].  Output ids are int64 original
 *     0-based row indices; dists are float32 distances (square roots).
 *   - Device-side faults of a kernel (a bounded wait that ran out, an
 *     invalid query value) are recorded in a status word of the index and
 *     reported by messi_check().
 *
 * Limits: 1 <= len <= 4096 with len % segments == 0 and m = len / segments
 * a power of two >= 4; 1 <= segments <= 16; cardinality a power of two in
 * [2, 256]; 1 <= n < 2^32 - 1; 1 <= k <= min(n, 1024); window < len.
 */
#ifndef MESSI_H
#define MESSI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct messi_index messi_index;
typedef struct messi_server messi_server;
typedef void *messi_stream; /* cudaStream_t */

typedef enum { MESSI_ED = 0, MESSI_DTW = 1 } messi_dist;

typedef enum {
    MESSI_OK = 0,
    MESSI_EINVAL = 1,   /* an argument is outside the documented limits       */
    MESSI_ENOMEM = 2,   /* device or pinned-host allocation failed            */
    MESSI_ECUDA = 3,    /* a CUDA runtime call failed                         */
    MESSI_ETIMEOUT = 4, /* a device-side bounded wait ran out                 */
    MESSI_EBUSY = 5,    /* result not ready yet (server poll) / queue full    */
    MESSI_ETIES = 6     /* accepted near-ties were dropped (a full log)       */
} messi_status;

/* Build options.  Zero-initialised fields take their defaults. */
typedef struct {
    uint32_t leaf_capacity; /* max series per leaf before it splits; default
                               2000 (Sec. 5.2, "Parameter Tuning") */
    uint32_t reserved[7];
} messi_config;

/* Counters of the most recent messi_query / messi_query_batched call. */
typedef struct {
    uint64_t queries;
    uint64_t lb_evaluated;    /* series whose iSAX lower bound was computed   */
    uint64_t lb_survivors;    /* series that passed the iSAX lower bound      */
    uint64_t lbk_survivors;   /* DTW: series that passed LB_Keogh             */
    uint64_t seeded;          /* series refined unconditionally in seed leaves */
    uint64_t refined;         /* real distances computed to the end           */
    uint64_t abandoned;       /* real distances abandoned early               */
    uint64_t bsf_updates;     /* improvements of the k-th best distance       */
    uint64_t tie_rechecks;    /* FP64 recomputations of near-tied candidates  */
    uint64_t kernel_launches; /* kernels this call queued                     */
    uint64_t scan_launches;   /* lower-bound scan launches (profiling mode)   */
    double scan_ms;           /* summed scan durations, CUDA events (profiling) */
    double query_ms_p50;      /* per-query device latency (profiling mode)    */
    double query_ms_p99;
    uint64_t leaves_live;     /* leaves whose symbol box did not prune them   */
    uint64_t screened_queries; /* batched screen: queries over all its passes
                                  (a query screened again counts again)      */
    uint64_t row_bytes;       /* ED refinement: bytes of raw rows read (whole
                                  256-point chunks up to an early abandon)   */
    uint64_t dtw_cells;       /* DTW: band cells computed, (2r + 1) per row of
                                  the recurrence evaluated (up to an abandon) */
    double refine_ms;         /* summed durations of the final refinement
                                  kernel (ED refine / banded DTW), CUDA events
                                  (profiling level >= 1, per-query path)      */
    uint64_t refine_launches;
} messi_stats;

typedef struct {
    uint64_t n_series;
    uint32_t len, segments, cardinality, leaf_capacity;
    uint64_t n_leaves;
    uint64_t max_leaf_size;
    uint64_t device_bytes;    /* bytes of device memory the index holds       */
    double build_ms;          /* device time of the last build                */
} messi_index_info;

/* ---------------------------------------------------------------- build --
 * Index construction (Sec. 3.2, Algorithms 1-4): every series is summarised
 * by PAA and SAX (Sec. 2.2), the interleaved iSAX words are radix-sorted, and
 * the sorted run is cut into leaves of at most leaf_capacity series by
 * splitting on one iSAX bit at a time (the root has one child per value of
 * the first bit of each segment).  The raw series are copied into leaf order.
 *
 * series      device or host, n*len float32; copied, so the caller may free it
 *             after the call returns.  Must be finite.
 * cfg         may be NULL.
 * out         receives the index; release with messi_free.
 * Synchronises `stream`.  Returns EINVAL for invalid sizes or non-finite
 * values, ENOMEM when the device cannot hold the index. */
messi_status messi_build(const float *series, uint64_t n, uint32_t len, uint32_t segments,
                         uint32_t cardinality, const messi_config *cfg, messi_stream stream,
                         messi_index **out);

/* Release every device allocation of the index.  NULL is a no-op. */
void messi_free(messi_index *ix);

/* Sizes of a built index (collection shape, leaf count and largest leaf,
 * device bytes held, build time).  Host-side only; out must not be NULL. */
messi_status messi_index_get_info(const messi_index *ix, messi_index_info *out);

/* Sliding-window subsequences of one long series, the collection MESSI
 * indexes for streaming series and for subsequence matching (Sec. 2: a
 * streaming series is cut into subsequences of length n by a sliding window
 * and those are indexed; Sec. 6: subsequence matching slides a window of the
 * query's length over the long series and indexes every subsequence).
 * Window i (0 <= i < count, count = (length - n) / stride + 1) is
 * series[i*stride .. i*stride + n) and becomes row i of out, so a k-NN id
 * over an index built from out is a window number: start = id * stride.
 * With znorm != 0 each window is z-normalised (mean 0, standard deviation 1,
 * Sec. 2) by these steps in FP64, round-to-nearest, no contraction:
 *   mean = (x_0 + ... + x_{n-1}, summed in order) / n
 *   var  = ((x_0 - mean)^2 + ... + (x_{n-1} - mean)^2, in order) / n
 *   inv  = 1 / sqrt(var), or 0 when var == 0 (a constant window -> zeros)
 *   out_j = (float)((x_j - mean) * inv)
 * so every other implementation of these steps yields the same bits; with
 * znorm == 0 the windows are copied unchanged.
 *
 * series  device pointer, length float32 values.
 * n       window length, 1..65536; stride >= 1; length >= n.
 * out     device pointer, count * n float32 (caller-allocated, row-major).
 * count   may be NULL; receives the number of windows written.
 * Asynchronous on `stream` (nothing is allocated).  Returns EINVAL for null
 * or host pointers and invalid sizes; ECUDA if the launch fails. */
messi_status messi_windows(const float *series, uint64_t length, uint32_t n, uint32_t stride,
                           int32_t znorm, float *out, uint64_t *count, messi_stream stream);

/* ---------------------------------------------------------------- query --
 * Exact k-NN (Algorithm 5 for ED, Sec. 3.4 for DTW; k-NN as a sorted array
 * of the k best, Sec. 5.4), one query after another as in the paper's
 * protocol (Sec. 5.1).  Per query: summarise the query (its PAA, or the PAA
 * of its LB_Keogh envelope for DTW), seed the best-so-far from the query's
 * own leaf (approxSearch, Sec. 3.1), prune whole leaves by the symbol box of
 * their words (the subtree pruning of Sec. 3), stream the iSAX words of the
 * remaining leaves through the lower bound, compact the survivors, refine
 * them in increasing bound order (the priority-queue order of Sec. 3) with ED
 * (Algorithm 9) or LB_Keogh / LB_Improved-filtered DTW (Algorithm 10), and
 * resolve near-ties in FP64.
 *
 * queries     device or host, nq*len float32.
 * window      DTW Sakoe-Chiba reach r in points (ignored for ED); r < len.
 * ids, dists  device or host, nq*k each, row q sorted by (dist, id).
 * A query holding a non-finite value yields ids -1 and dists NaN for its row
 * and a MESSI_EINVAL status in messi_check(). */
messi_status messi_query(const messi_index *ix, const float *queries, uint32_t nq, uint32_t k,
                         messi_dist dist, uint32_t window, int64_t *ids, float *dists,
                         messi_stream stream);

/* Batched form (no counterpart in the paper, which answers queries one at a
 * time): up to `batch` queries per launch.  Same arguments and results as
 * messi_query; batch = 0 picks the tuned default.  Two modes, chosen with
 * messi_set_batch_mode:
 *   MESSI_BATCH_TC_SCREEN (default): every (series, query) squared distance is
 *     estimated as |x|^2 + |q|^2 - 2 q.x with f16 tensor-core MMAs (FP32
 *     accumulation), widened by a rigorous per-pair error bound; pairs whose
 *     lower end stays within the query's k-th best bound are recomputed
 *     exactly in FP32.  Needs len % 16 == 0, len <= 2048 and |values| <= 65000
 *     (an f16 copy of the rows, 2*len bytes per series, is built on first
 *     use); otherwise, or for DTW, the call takes the other kernels.
 *   MESSI_BATCH_LB_REFINE: a persistent fused lower-bound-then-refine kernel
 *     where the queries of a batch share each pass over the iSAX words; every
 *     full batch of a call replays one captured CUDA graph.
 * A query a batch cannot settle exactly (a screen that keeps overflowing, or
 * more accepted near-ties than a batch slot logs) is answered again by the
 * per-query kernels, so results equal messi_query's.  Both modes synchronise
 * `stream` (they read per-batch outcomes on the host).
 * DTW (either mode): the queries' per-query kernel sequences run side by side
 * on up to 4 streams of the library, each with its own workspace (24 bytes
 * per series each), so the small grids of one query share the GPU with the
 * others'; the call waits for them on `stream` and synchronises it. */
messi_status messi_query_batched(const messi_index *ix, const float *queries, uint32_t nq,
                                 uint32_t k, messi_dist dist, uint32_t window, uint32_t batch,
                                 int64_t *ids, float *dists, messi_stream stream);

/* Lower bounds of one query against every series, in original id order:
 * lb2[i] = squared iSAX mindist (ED, Property 1 in Sec. 4) or squared
 * envelope mindist (DTW, Sec. 3.4) as the query kernels use it (each term
 * rounded down, so lb2[i] never exceeds the exact bound).
 * query device or host len floats; lb2 device or host n floats. */
messi_status messi_lower_bounds(const messi_index *ix, const float *query, messi_dist dist,
                                uint32_t window, float *lb2, messi_stream stream);

/* Lower bounds like messi_lower_bounds, for callers that may not allocate
 * device memory while they run: an embedding that owns a fixed device-memory
 * budget and gives the library only its input and output buffers, or a
 * latency-critical loop that must not stall in cudaMalloc / cudaFree (which
 * can synchronise the device).  The paper has no counterpart; this is an
 * interface of this library.
 *
 * Allocates nothing: query and lb2 must be device pointers (EINVAL for host
 * buffers, which would need staging memory) on the device the index was
 * built on, and that device must be current (EINVAL otherwise).  The scratch
 * -- query state, lower-bound table, query and envelope rows -- lives in one
 * fixed array of 41,216 bytes that every GPU loading the library holds until
 * the process exits.  That array bounds the series length: an index with
 * len > 2048 is rejected with EINVAL (use messi_lower_bounds).  Every call
 * shares the array, so calls whose work overlaps on the GPU (on different
 * streams, or from several threads) race and must be serialised by the
 * caller; each call clears the query state it needs before use.  The first
 * call on each device looks up the array's device address
 * (cudaGetSymbolAddress) and should come before any stream capture.  A query
 * holding a non-finite value leaves lb2 unwritten (its previous contents
 * stay) and messi_check() then reports MESSI_EINVAL.  Results equal
 * messi_lower_bounds bit for bit. */
messi_status messi_lower_bounds_noalloc(const messi_index *ix, const float *query, messi_dist dist,
                                        uint32_t window, float *lb2, messi_stream stream);

/* Counters of the last query call.  Synchronises the index's last stream. */
messi_status messi_query_stats(const messi_index *ix, messi_stats *out);

/* Kernels messi_query_batched uses for ED (see there); EINVAL for other modes.
 * Not thread-safe against concurrent batched calls on the same index. */
enum { MESSI_BATCH_LB_REFINE = 0, MESSI_BATCH_TC_SCREEN = 1 };
messi_status messi_set_batch_mode(messi_index *ix, int mode);

/* Shapes of the batched forms.  The paper has no counterpart: it answers one
 * query at a time (Sec. 5.1); batching is this library's addition. */
typedef struct {
    uint32_t batch;         /* queries per batch when messi_query_batched gets batch = 0 */
    uint32_t chunk_tiles;   /* lower-bound form: scan tiles a CTA claims at a time      */
    uint32_t ctas_per_sm;   /* lower-bound form: resident CTAs per SM (1 or 2)         */
    uint32_t mode;          /* MESSI_BATCH_LB_REFINE or MESSI_BATCH_TC_SCREEN          */
    double ms_per_query;    /* device time per query of the chosen shape (autotune)    */
    uint32_t reserved[4];
} messi_tuning;

/* Time the index's current batch mode on `queries` (device pointer, nq rows,
 * nq >= 32) for a set of shapes -- lower-bound form: batch 32..256, chunk
 * tiles 16/32/64, 1 or 2 CTAs per SM; screened form: batch 128..1024 -- with
 * CUDA events on `stream`, one warm-up batch and one timed batch per shape,
 * and keep the fastest per query.  Writes the choice to *out (may be NULL).
 * Synchronises `stream`.  EINVAL for host queries or nq < 32. */
messi_status messi_autotune(messi_index *ix, const float *queries, uint32_t nq, uint32_t k, messi_stream stream,
                            messi_tuning *out);

/* Apply shapes (for instance a cached autotune result); mode is ignored.
 * EINVAL for batch 0 or > 65535, chunk_tiles 0 or > 1024, ctas_per_sm not 1 or 2. */
messi_status messi_set_tuning(messi_index *ix, const messi_tuning *t);

/* Diagnostic of the tensor-core operand layout used by the screen: one
 * 128 x n x k f16 GEMM tile, D = A * B^T with FP32 accumulation, through the
 * same tcgen05 instructions.  a_tile (128 x k) and b_tile (n x k) are f16 bit
 * patterns already in the operand layout (8-row x 16-byte core matrices, see
 * paper_2110_07519_gb300/csrc/tc.cuh); lbo / sbo are the descriptor's
 * leading and stride byte offsets; d receives 128 x n floats, row-major.
 * Host pointers; synchronises the device.  k a multiple of 16 <= 256, n a
 * multiple of 32 <= 256.  The paper has no counterpart. */
messi_status messi_debug_tc_gemm(const uint16_t *a_tile, const uint16_t *b_tile, uint32_t k, uint32_t n,
                                 uint32_t lbo, uint32_t sbo, float *d);

/* Test hook for the failure path of the k > 1 result array (no counterpart
 * in the paper).  The array of the k best is updated under a lock taken with
 * a bounded spin; a thread that gives up after spin_limit tries drops its
 * candidate and sets the timeout bit of the index's status word, which the
 * next messi_check() reports as MESSI_ETIMEOUT (the answer of that call is
 * then not exact).  With hold_lock != 0 every query of messi_query starts
 * with that lock held, so its first k > 1 insertion gives up.  Defaults:
 * spin_limit 4,194,304, hold_lock 0 (restore them with those values).  No
 * wait of the kernels on memory copies is affected. */
messi_status messi_debug_set_lock_fault(messi_index *ix, uint32_t spin_limit, int hold_lock);

/* Profiling level, reported by messi_query_stats.  0 (default): off.
 * 1: CUDA events around every lower-bound scan group (per-query path), every
 * screen launch (screened batch) and every fused launch (lower-bound batch
 * form) -- scan_ms / scan_launches -- and around every final refinement
 * kernel of the per-query path (also for batched DTW) -- refine_ms /
 * refine_launches.  2: also around every query (per-query
 * path) or batch (batched forms) -- query_ms_p50 / p99.  Events are recorded
 * on the call's stream.  Any level above 0 turns off the graph replay of the
 * lower-bound batch form.  EINVAL for other levels. */
messi_status messi_set_profiling(messi_index *ix, int enable);

/* Synchronise `stream` and report (then clear) the device status word. */
messi_status messi_check(const messi_index *ix, messi_stream stream);

/* ------------------------------------------------------- summaries -------
 * PAA + SAX of n series (Sec. 2.2; ConvertToiSAX in Algorithm 3) without
 * building an index.  words receives n*16 bytes: byte s of word i is the
 * symbol of segment s (0 = lowest region) for s < segments, 0 beyond.
 * series, words: device or host. */
messi_status messi_summarize(const float *series, uint64_t n, uint32_t len, uint32_t segments,
                             uint32_t cardinality, uint8_t *words, messi_stream stream);

/* Leaf layout of an index (for inspection and tests).  order: n uint32
 * original ids in leaf order; leaf_off: n_leaves+1 uint64; leaf_depth:
 * n_leaves uint8 (key prefix bits of each leaf).  Host pointers; any may be
 * NULL.  Synchronises. */
messi_status messi_index_layout(const messi_index *ix, uint32_t *order, uint64_t *leaf_off,
                                uint8_t *leaf_depth);

/* The FP64 breakpoints the library uses (Sec. 2.2: N(0,1) quantiles j/c,
 * j = 1..c-1).  Host only, no GPU needed.  out: cardinality-1 doubles. */
messi_status messi_breakpoints(uint32_t cardinality, double *out);

/* ------------------------------------------------------------ serving ----
 * A request loop over a resident index (the paper answers queries one after
 * another and has no counterpart).  Requests enter an arrival queue; worker
 * threads, one per CUDA stream, admit them into device batches in arrival
 * order while the device memory charged to unfinished requests stays within
 * mem_budget (a request is admitted beyond it only when nothing else is in
 * flight), run each batch through messi_query_batched's forms with k = the
 * largest k of the batch, and give every
 * request the first k of its row.  Batches on different streams overlap on
 * the device.  A request's result does not depend on what else is in flight:
 * the answer is exact and a k-NN answer is a prefix of any larger k.
 */
typedef struct {
    uint32_t max_batch;     /* queries per device batch; default 1024            */
    uint32_t max_k;         /* largest k a request may ask for; default 64       */
    uint32_t streams;       /* worker streams (batches in flight); default 2     */
    uint32_t max_queued;    /* arrival-queue cap (0 = unbounded); submit returns
                               EBUSY beyond it                                   */
    uint64_t mem_budget;    /* device bytes charged to admitted unfinished
                               requests (0 = streams * max_batch requests)       */
    uint64_t reserved[4];
} messi_server_config;

typedef struct {
    uint64_t submitted, completed, rejected, batches, inflight_peak;
    double p50_ms, p99_ms, mean_ms;   /* submit-to-result latency of completed requests */
    uint64_t budget_waits;            /* times a worker found queued requests but had to
                                         wait for admitted ones to free their memory */
    uint64_t reserved[3];
} messi_server_stats;

/* Start a server on `ix` (which must outlive it); cfg may be NULL.  Builds
 * the screening copy of the index if needed and allocates per-stream
 * buffers.  Synchronises the device. */
messi_status messi_server_create(messi_index *ix, const messi_server_config *cfg, messi_server **out);

/* Queue one query (host pointer, len floats; copied before return).  Returns
 * a ticket.  EINVAL for bad k / window, EBUSY when the queue is full. */
messi_status messi_server_submit(messi_server *srv, const float *query, uint32_t k, messi_dist dist,
                                 uint32_t window, uint64_t *ticket);

/* Collect a finished request: ids / dists are host arrays of its k entries,
 * latency_ms (may be NULL) the time from submit to result.  Waits up to
 * wait_us microseconds; EBUSY when not finished yet, EINVAL for an unknown or
 * already collected ticket. */
messi_status messi_server_poll(messi_server *srv, uint64_t ticket, int64_t *ids, float *dists,
                               double *latency_ms, uint64_t wait_us);

/* Counters of a server since creation: requests submitted / completed /
 * rejected, batches run, the largest number in flight, and submit-to-result
 * latency percentiles (ms) over completed requests. */
messi_status messi_server_get_stats(messi_server *srv, messi_server_stats *out);

/* Hold (paused != 0) or resume admission.  While held, workers finish the
 * batches they have but admit nothing new; submit keeps queueing (up to
 * max_queued).  For draining a server before the index changes, and for
 * bringing the queue to a known state. */
messi_status messi_server_pause(messi_server *srv, int paused);

/* Stop the workers after the queued requests and release everything. */
void messi_server_destroy(messi_server *srv);

/* Thread-local description of the last failure ("" when none). */
const char *messi_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* MESSI_H */
