// messi_internal.cuh -- shared declarations of the GB300 iSAX k-NN library.
//
// Data layout in HBM (one index, positions are leaf order):
//   raw        float [N][len]   series copied into leaf order (Sec. 3.2: a
//                               leaf points at its raw series; here the rows
//                               of a leaf are contiguous)
//   sax        uint4 [N]        iSAX word, byte s = symbol of segment s
//   ids        u32   [N]        original row id of each position
//   pos_of_id  u32   [N]        inverse permutation
//   leaf_off   u64   [L+1]      first position of each leaf
//   leaf_key   uint4 [L]        interleaved key of each leaf's first series
//   leaf_depth u8    [L]        key prefix bits of each leaf
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <atomic>
#include <vector>

#include <cuda_fp16.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/messi.h"

namespace messi {

// ------------------------------------------------------------ constants
constexpr int kMaxSegments = 16;
constexpr int kMaxCard = 256;
constexpr int kMaxLen = 4096;
constexpr int kMaxK = 1024;
constexpr int kLogCap = 8192;        // candidates the final step resolves at once (shared memory)
constexpr int kBatchLogCap = 20480;  // log entries of a batched query slot
constexpr int kScanTileWordsHost = 1024;   // words per lower-bound scan tile (see query.cu)
constexpr int kOrderBuckets = 4096;  // survivors bucketed by the top 12 bits of their FP32 bound
constexpr int kSeedMax = 4096;       // series of the seed leaf refined up front
constexpr unsigned long long kEmpty = ~0ull;   // packed "no candidate"
constexpr int kMaxScanGrid = 2048;   // scan CTAs (each owns one survivor region)

// device status word bits
constexpr unsigned kStTimeout = 1u;
constexpr unsigned kStInvalidQuery = 2u;
constexpr unsigned kStTieOverflow = 4u;

// spin limits of bounded waits (iterations; each sleeps a few hundred ns)
constexpr unsigned kSpinLimit = 1u << 22;

// ------------------------------------------------------- per-query state
struct QueryCounters {
    unsigned long long lb_evaluated, lb_survivors, lbk_survivors, seeded, refined, abandoned,
        bsf_updates, tie_rechecks, leaves_live, row_bytes, dtw_cells;
};

struct QueryState {
    unsigned long long thr;     // packed (d2 bits << 32 | id) of the current k-th best
    unsigned int lock;          // k > 1 insertion lock
    unsigned int kcount;        // entries in karr
    unsigned int surv_count;    // lower-bound survivors
    unsigned int surv2_count;   // LB_Keogh survivors (DTW)
    unsigned int log_count;     // accepted / near-tie candidates logged
    unsigned int seed_lo, seed_hi;
    unsigned int seed_count;    // distances written by the seed phase
    unsigned int invalid;       // non-finite query value seen
    unsigned int scan_grid;     // CTAs of the last scan: survivor regions
    unsigned int region_words;  // words (and survivor slots) per scan CTA
    unsigned int ord_count;     // survivors in the bound-ordered list
    unsigned int live_tiles;    // scan tiles holding a leaf that its box did not prune
    uint4 qsym;                 // per segment (byte s) a symbol where the table is 0
    uint4 qkey;                 // interleaved key of the query word
    QueryCounters c;
};

// Arrays belonging to one query slot (device pointers).
struct QuerySlot {
    QueryState *st;
    float *lut;                 // [16][256] squared-distance table, rounded down
    float *q;                   // [len] query
    float *U, *L;               // [len] LB_Keogh envelope (DTW)
    unsigned long long *karr;   // [kMaxK] sorted k best (k > 1)
    unsigned long long *log;    // [log_cap] accepted / near-tie candidates
    unsigned long long *seedbuf;// [kSeedMax]
    unsigned int *surv_pos;     // [N] (plain path only), region of scan CTA c
    float *surv_lb;             // [N]    starts at c * region_words
    unsigned int *region_count; // [kMaxScanGrid] survivors found by each scan CTA
    unsigned int *surv2;        // [N] compact LB_Keogh survivors, or the bound-ordered ED survivors
    float *surv2_lb;            // [N] their lower bounds
    unsigned int *bucket;       // [2][kOrderBuckets] bucket counts, then write cursors
    unsigned int *tile_epoch;   // [scan tiles] last query epoch that found the tile live
    unsigned int *live_list;    // [scan tiles] live tiles of the current query
    double *dtw64;              // [32 warps][3][len] FP64 DTW diagonals (finalize)
    QueryCounters *acc;         // per-call counter accumulator
    unsigned log_cap;           // entries of `log`
};

// Parameters every query kernel needs, passed by value.
struct IndexView {
    const float *raw;
    const uint4 *sax;
    const unsigned int *ids;
    const unsigned int *pos_of_id;
    const unsigned long long *leaf_off;
    const uint4 *leaf_key;
    const uint4 *leaf_box;      // [L][2]: per segment (byte s) the smallest, then the largest symbol
    const double *beta64;       // [card-1] breakpoints
    unsigned long long N;
    unsigned long long L;
    int len, w, card, bits, m;
    unsigned int *status;       // device status word
};

struct QueryParams {
    int k;
    int dist;                   // 0 ED, 1 DTW
    int r;                      // DTW window
    float F;                    // near-tie band factor (>= (1+gamma)^2)
    unsigned lock_spin;         // tries of the k-array lock before a timeout (kSpinLimit)
};

}  // namespace messi

namespace messi {
// Mutable per-call state of the query paths.  The index owns one; a server
// owns one per stream so that batches in flight on different streams never
// share scratch memory.
// One batch of a graph-replayed call: where its query rows are read and its
// results written (device pointers).
struct BatchArgs {
    const float *queries;
    long long *ids;
    float *dists;
    unsigned *redo;     // per query: 1 when the batch could not answer it exactly
};

struct Workspace {
    // plain path: one query slot with survivor arrays of N entries
    void *ws_block = nullptr;
    size_t ws_bytes = 0;
    QuerySlot slot{};
    // staging of host queries / outputs
    void *stage_block = nullptr;
    size_t stage_bytes = 0;
    // batched path
    void *bws_block = nullptr;
    size_t bws_bytes = 0;
    int bws_slots = 0;
    QuerySlot *bslots_dev = nullptr;
    unsigned *bcounter = nullptr;
    QueryCounters *bacc = nullptr;
    bool last_batched = false;
    // tensor-core screen, per batch
    void *tcws_block = nullptr;
    size_t tcws_bytes = 0;
    unsigned tcws_B = 0;
    // statistics of the last call
    messi_stats last{};
    cudaStream_t last_stream = nullptr;
    unsigned epoch = 0;               // per-query stamp of the live-tile marks
    // graph of one fused lower-bound batch, replayed once per batch of a call
    cudaGraphExec_t graph = nullptr;
    unsigned long long graph_key[4] = {0, 0, 0, 0};
    BatchArgs *gargs_dev = nullptr, *gargs_host = nullptr;   // argument table (device, pinned staging)
    unsigned *redo_dev = nullptr, *redo_host = nullptr;       // per-query redo flags of a batched call
    size_t redo_cap = 0;
    unsigned *gcursor = nullptr;
    size_t gargs_cap = 0;
    unsigned long long graph_replays = 0;
    cudaEvent_t gargs_done = nullptr;     // the staging table's last copy
    cudaStream_t capture_stream = nullptr;
    unsigned long long tile_count = 0;   // scan tiles of the plain slot's stamp array
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, int>> scan_ev, query_ev, refine_ev;   // pairs of event indices
    unsigned long long launches = 0;
    // batched DTW: per-query pipelines overlapped on several streams, each
    // with a workspace of its own
    std::vector<Workspace *> sub;
    std::vector<cudaStream_t> sub_streams;
    std::vector<cudaEvent_t> sub_done;
    cudaEvent_t fork = nullptr;
};
void free_workspace(Workspace &w);
}  // namespace messi

struct messi_index;
namespace messi {
// query paths on an explicit workspace (api.cu)
// Builds the f16 screening copy of the rows if the index has none yet
// (screen_state 0); leaves screen_state -1 where the rows cannot use it.
messi_status ensure_screen_copy(messi_index *ix, cudaStream_t s);
// Survivors of the scan (src 0: per-CTA regions of surv_pos / surv_lb) or of
// LB_Keogh (src 1: surv2 / surv2_lb) written to dst_pos / dst_lb in
// increasing order of lower-bound bucket; st->ord_count receives their number.
void launch_order(const QueryParams &qp, const QuerySlot &slot, int src, unsigned *dst_pos, float *dst_lb,
                  cudaStream_t s);
messi_status run_plain(messi_index *ix, Workspace *ws, const float *queries, uint32_t nq, uint32_t k,
                       messi_dist dist, uint32_t window, int64_t *ids, float *dists, messi_stream stream);
messi_status run_batched(messi_index *ix, Workspace *ws, const float *queries, uint32_t nq, uint32_t k,
                         messi_dist dist, uint32_t window, uint32_t batch, int64_t *ids, float *dists,
                         messi_stream stream);
}  // namespace messi

struct messi_index {
    int device = 0;
    unsigned long long N = 0;
    int len = 0, w = 0, card = 0, bits = 0, m = 0;
    unsigned cap = 2000;
    unsigned long long L = 0, max_leaf = 0;
    // device arrays
    float *raw = nullptr;
    uint4 *sax = nullptr;
    unsigned int *ids = nullptr;
    unsigned int *pos_of_id = nullptr;
    unsigned long long *leaf_off = nullptr;
    uint4 *leaf_key = nullptr;
    unsigned char *leaf_depth = nullptr;
    uint4 *leaf_box = nullptr;
    double *beta64 = nullptr;
    unsigned int *status = nullptr;
    double beta_host[256] = {0};
    // default workspace of messi_query / messi_query_batched
    messi::Workspace ws;
    // bookkeeping
    std::atomic<size_t> device_bytes{0};   // workspaces of server workers grow it concurrently
    double build_ms = 0.0;
    int profiling = 0;                  // 1: events around the scan / screen launches; 2: and every query
    unsigned long long launches = 0;
    // tuned shapes of the batched path
    unsigned tune_batch = 64, tune_chunk_tiles = 32, tune_ctas_per_sm = 2;
    int batch_mode = 1;                 // 0: lower bound + FP32 refine, 1: tensor-core screen
    // test hook (messi_debug_set_lock_fault): tries of the k-array lock, and
    // whether the per-query path starts every query with that lock held
    unsigned lock_spin = messi::kSpinLimit;
    bool hold_lock = false;
    // tensor-core screen: f16 tile copy of the rows and their norms
    __half *screen16 = nullptr;
    float *xn = nullptr, *xnorm = nullptr;
    int screen_state = 0;               // 0 not built, 1 ready, -1 unavailable (values outside f16 range)
};

namespace messi {

// ------------------------------------------------------------ host helpers
// NVTX range over a host scope (build phases, a call, the stages of a query
// as they are enqueued), for profilers that read NVTX; a no-op otherwise.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

void set_error(const std::string &msg);
messi_status fail(messi_status st, const std::string &msg);
bool cuda_ok(cudaError_t e, const char *what);
#define MESSI_CUDA(call)                                  \
    do {                                                  \
        if (!::messi::cuda_ok((call), #call)) return MESSI_ECUDA; \
    } while (0)

int num_sms();
void compute_breakpoints(int card, double *beta);
// device or managed memory (false for host memory and unknown pointers)
bool is_device_ptr(const void *p);
// EINVAL unless the current device is the one the index lives on, and every
// non-null device pointer in ptrs (host pointers are skipped) is memory of
// that device (managed memory is accepted on any device)
messi_status check_device(const messi_index *ix, const void *const *ptrs, int n, const char *where);
IndexView view_of(const messi_index *ix);
// query parameters of one call: k, distance, window, near-tie band and the
// index's k-array lock spin limit
QueryParams make_params(const messi_index *ix, uint32_t k, int dist, uint32_t window);

// ------------------------------------------------------------- launchers
// summarize.cu
void launch_summarize(const float *series, unsigned long long n, int len, int w, int card,
                      const double *beta64, const float *beta32, uint4 *sax_out, uint4 *key_out,
                      unsigned int *id_out, unsigned int *status, cudaStream_t s);
// radix_sort.cu
size_t radix_sort_temp_bytes(unsigned long long n);
void radix_sort_keys(uint4 *keys, unsigned int *vals, uint4 *keys_alt, unsigned int *vals_alt,
                     unsigned long long n, int key_bits, void *temp, cudaStream_t s,
                     unsigned long long *launches);
size_t scan_temp_bytes(unsigned long long n);
void exclusive_scan_u32(const unsigned int *in, unsigned int *out, unsigned long long n,
                        void *temp, cudaStream_t s, unsigned long long *launches);
// leaves.cu
messi_status build_leaves(messi_index *ix, const uint4 *sorted_keys, const uint4 *sax_unsorted,
                          const float *series, cudaStream_t s);
// query.cu
void launch_prep(const IndexView &iv, const QueryParams &qp, QuerySlot slot, const float *query,
                 cudaStream_t s);
void launch_seed(const IndexView &iv, const QueryParams &qp, QuerySlot slot, cudaStream_t s,
                 unsigned long long *launches);
// Leaf boxes against the query's table (live tiles stamped with `epoch`,
// which must differ from every earlier query's on this slot), then the
// lower-bound scan of the live tiles.
void launch_scan(const IndexView &iv, const QueryParams &qp, QuerySlot slot, unsigned epoch, cudaStream_t s);
// ev0 / ev1 (may be null): recorded around the final refinement kernel
// (k_refine_ed for ED, the banded DTW for DTW)
void launch_refine(const IndexView &iv, const QueryParams &qp, QuerySlot slot, cudaStream_t s,
                   unsigned long long *launches, cudaEvent_t ev0 = nullptr, cudaEvent_t ev1 = nullptr);
void launch_finalize(const IndexView &iv, const QueryParams &qp, QuerySlot slot, long long *ids,
                     float *dists, cudaStream_t s);
void launch_lower_bounds(const IndexView &iv, QuerySlot slot, float *lb2_by_id, cudaStream_t s);
void init_kernel_attributes();
// screen.cu
constexpr unsigned kTcCap = 16384;   // candidates per query per screening pass
constexpr unsigned kTcMaxLenHost = 2048;  // longest series the screen takes
size_t screen_smem_bytes(int len);
void init_screen_attributes();
void launch_make_screen_copy(const float *raw, unsigned long long N, int len, __half *tiles, float *xn, float *xnorm,
                             unsigned *bad, cudaStream_t s);
constexpr unsigned kTcTopKHost = 16;   // longest per-query top-k list of the screen
void launch_tc_qprep(const QuerySlot *slots, unsigned B, int len, const QueryParams &qp, __half *qtiles,
                     float *qconst, unsigned *Ubits, unsigned *cand_count, unsigned *flags, unsigned *active,
                     float *tkinit, unsigned *glock, uint2 *srange, cudaStream_t s);
void launch_tc_next_pass(const QuerySlot *slots, unsigned B, const QueryParams &qp, unsigned cap, unsigned *Ubits,
                         unsigned *cand_count, unsigned *active, unsigned *n_active, const __half *qtiles,
                         __half *qtiles2, unsigned *qmap, int len, cudaStream_t s);
void launch_tc_screen(const __half *rtiles, const float *xn, const float *xnorm, const __half *qtiles,
                      const float *qconst, unsigned *Ubits, unsigned *cand_count, unsigned *cand_pos,
                      const unsigned *active, const unsigned *qmap, float *topk, unsigned *glock, int lists,
                      const uint2 *srange, unsigned cap, unsigned long long N, int len, unsigned B, int k,
                      unsigned *status, cudaStream_t s);
void launch_tc_recheck(const IndexView &iv, const QueryParams &qp, const QuerySlot *slots, unsigned B,
                       const unsigned *cand_count, const unsigned *cand_pos, unsigned cap, const unsigned *active,
                       cudaStream_t s);
void launch_batch_args(const IndexView &iv, const QueryParams &qp, const QuerySlot *slots_dev, unsigned B,
                       const BatchArgs *args, unsigned *cursor, unsigned chunk_tiles, unsigned ctas_per_sm,
                       unsigned *counter, cudaStream_t s);
void launch_batch_seed(const IndexView &iv, const QueryParams &qp, const QuerySlot *slots_dev, unsigned B,
                       const float *queries, cudaStream_t s, unsigned long long *launches);
void launch_batch_finalize(const IndexView &iv, const QueryParams &qp, const QuerySlot *slots_dev, unsigned B,
                           long long *ids, float *dists, unsigned *redo, cudaStream_t s, unsigned long long *launches);
void launch_batch(const IndexView &iv, const QueryParams &qp, const QuerySlot *slots_dev, unsigned B,
                  const float *queries, long long *ids, float *dists, unsigned *redo, unsigned chunk_tiles,
                  unsigned ctas_per_sm, unsigned *counter, cudaStream_t s, unsigned long long *launches,
                  cudaEvent_t ev0, cudaEvent_t ev1);
void launch_reset_state(QuerySlot slot, cudaStream_t s);
// dst[0] += src[0] + ... + src[n-1] (counter accumulators of several slots)
void launch_add_counters(QueryCounters *dst, const QueryCounters *const *src, int n, cudaStream_t s);
constexpr int kDtwStreams = 4;       // streams of the batched DTW form
float band_factor(int dist, int len);

}  // namespace messi
