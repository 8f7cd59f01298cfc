// api.cu -- the C ABI declared in include/messi.h: argument checks, device
// allocation, host<->device staging and the per-query kernel sequence.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "messi_internal.cuh"

namespace messi {

namespace {
thread_local std::string g_last_error;

bool is_pow2(unsigned v) { return v && !(v & (v - 1)); }

std::mutex g_attr_mu;
std::vector<int> g_attr_done;

void ensure_attributes()
{
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_attr_mu);
    if (std::find(g_attr_done.begin(), g_attr_done.end(), dev) != g_attr_done.end()) return;
    init_kernel_attributes();
    g_attr_done.push_back(dev);
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Growable device buffer owned by the index (host staging of inputs/outputs).
bool ensure_stage(Workspace *ws, size_t bytes)
{
    if (ws->stage_bytes >= bytes) return true;
    if (ws->stage_block) cudaFree(ws->stage_block);
    ws->stage_block = nullptr;
    ws->stage_bytes = 0;
    if (cudaMalloc(&ws->stage_block, bytes) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    ws->stage_bytes = bytes;
    return true;
}

// Stamp for the next query's live-tile marks on this workspace.  Stamps only
// need to differ from every earlier one on the same array; after 2^32 - 1
// queries the array is cleared and the stamps start again.
unsigned next_epoch(Workspace *ws, cudaStream_t s)
{
    if (++ws->epoch == 0u) {
        const unsigned long long n = ws->tile_count;
        cudaMemsetAsync(ws->slot.tile_epoch, 0, n * 4, s);
        ws->epoch = 1u;
    }
    return ws->epoch;
}

// Plain-path workspace: one query slot with survivor arrays of N entries.
messi_status ensure_workspace(messi_index *ix, Workspace *ws)
{
    if (ws->ws_block) return MESSI_OK;
    const size_t N = ix->N, len = ix->len;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    const size_t o_st = take(sizeof(QueryState));
    const size_t o_lut = take(kMaxSegments * kMaxCard * 4);
    const size_t o_q = take(len * 4), o_u = take(len * 4), o_l = take(len * 4);
    // every position is offered at most once on this path: a log of N + seed
    // entries cannot overflow
    const size_t log_cap = N + kSeedMax;
    const size_t o_karr = take(kMaxK * 8), o_log = take(log_cap * 8), o_seed = take(kSeedMax * 8);
    // scan survivors: CTA c writes region c of ceil(live tiles / grid) tiles,
    // so the arrays hold ntiles + kMaxScanGrid tiles of words
    const size_t ntiles = (N + kScanTileWordsHost - 1) / kScanTileWordsHost;
    const size_t nsurv = (ntiles + kMaxScanGrid) * kScanTileWordsHost;
    const size_t o_sp = take(nsurv * 4), o_sl = take(nsurv * 4), o_s2 = take(N * 4), o_s2l = take(N * 4);
    const size_t o_bk = take(2 * kOrderBuckets * 4);
    const size_t o_te = take(ntiles * 4), o_ll = take(ntiles * 4);
    const size_t o_dtw = take(32 * 3 * len * 8);
    const size_t o_rc = take(kMaxScanGrid * 4);
    const size_t o_acc = take(sizeof(QueryCounters));
    char *base = nullptr;
    if (cudaMalloc(&base, off) != cudaSuccess) {
        cudaGetLastError();
        return fail(MESSI_ENOMEM, "messi_query: cannot allocate the query workspace");
    }
    ws->ws_block = base;
    ws->ws_bytes = off;
    ix->device_bytes += off;
    QuerySlot &s = ws->slot;
    s.st = reinterpret_cast<QueryState *>(base + o_st);
    s.lut = reinterpret_cast<float *>(base + o_lut);
    s.q = reinterpret_cast<float *>(base + o_q);
    s.U = reinterpret_cast<float *>(base + o_u);
    s.L = reinterpret_cast<float *>(base + o_l);
    s.karr = reinterpret_cast<unsigned long long *>(base + o_karr);
    s.log = reinterpret_cast<unsigned long long *>(base + o_log);
    s.seedbuf = reinterpret_cast<unsigned long long *>(base + o_seed);
    s.surv_pos = reinterpret_cast<unsigned *>(base + o_sp);
    s.surv_lb = reinterpret_cast<float *>(base + o_sl);
    s.surv2 = reinterpret_cast<unsigned *>(base + o_s2);
    s.surv2_lb = reinterpret_cast<float *>(base + o_s2l);
    s.bucket = reinterpret_cast<unsigned *>(base + o_bk);
    s.tile_epoch = reinterpret_cast<unsigned *>(base + o_te);
    s.live_list = reinterpret_cast<unsigned *>(base + o_ll);
    s.dtw64 = reinterpret_cast<double *>(base + o_dtw);
    s.region_count = reinterpret_cast<unsigned *>(base + o_rc);
    s.acc = reinterpret_cast<QueryCounters *>(base + o_acc);
    s.log_cap = (unsigned)std::min<size_t>(log_cap, 0xffffffffu);
    // bucket counts start at zero; every ordering step leaves them cleared
    if (!cuda_ok(cudaMemset(s.bucket, 0, kOrderBuckets * 4), "messi_query: clear the bound buckets") ||
        !cuda_ok(cudaMemset(s.tile_epoch, 0, ntiles * 4), "messi_query: clear the tile stamps"))
        return MESSI_ECUDA;
    ws->epoch = 0;
    ws->tile_count = ntiles;
    return MESSI_OK;
}

// Batched workspace: B query slots (no survivor arrays: the fused kernel keeps
// survivors in shared memory), their device-side descriptor array, the work
// counter and the call's counter accumulator.
messi_status ensure_batch_workspace(messi_index *ix, Workspace *ws, unsigned B)
{
    if (ws->bws_block && (unsigned)ws->bws_slots >= B) return MESSI_OK;
    if (ws->bws_block) {
        cudaFree(ws->bws_block);
        ix->device_bytes -= ws->bws_bytes;
        ws->bws_block = nullptr;
        ws->bws_slots = 0;
    }
    const size_t len = ix->len;
    const size_t per = align256(sizeof(QueryState)) + align256(kMaxSegments * kMaxCard * 4) + 3 * align256(len * 4) +
                       align256(kMaxK * 8) + align256(kBatchLogCap * 8) + align256(kSeedMax * 8);
    const size_t head = align256(B * sizeof(QuerySlot)) + align256(64) + align256(sizeof(QueryCounters));
    char *base = nullptr;
    if (cudaMalloc(&base, head + per * B) != cudaSuccess) {
        cudaGetLastError();
        return fail(MESSI_ENOMEM, "messi_query_batched: cannot allocate the batch workspace");
    }
    ws->bws_block = base;
    ws->bws_bytes = head + per * B;
    ws->bws_slots = (int)B;
    ix->device_bytes += ws->bws_bytes;
    ws->bslots_dev = reinterpret_cast<QuerySlot *>(base);
    ws->bcounter = reinterpret_cast<unsigned *>(base + align256(B * sizeof(QuerySlot)));
    ws->bacc = reinterpret_cast<QueryCounters *>(base + align256(B * sizeof(QuerySlot)) + align256(64));
    std::vector<QuerySlot> host(B);
    char *p = base + head;
    for (unsigned b = 0; b < B; ++b) {
        QuerySlot &q = host[b];
        q = QuerySlot{};
        q.st = reinterpret_cast<QueryState *>(p); p += align256(sizeof(QueryState));
        q.lut = reinterpret_cast<float *>(p); p += align256(kMaxSegments * kMaxCard * 4);
        q.q = reinterpret_cast<float *>(p); p += align256(len * 4);
        q.U = reinterpret_cast<float *>(p); p += align256(len * 4);
        q.L = reinterpret_cast<float *>(p); p += align256(len * 4);
        q.karr = reinterpret_cast<unsigned long long *>(p); p += align256(kMaxK * 8);
        q.log = reinterpret_cast<unsigned long long *>(p); p += align256(kBatchLogCap * 8);
        q.log_cap = kBatchLogCap;
        q.seedbuf = reinterpret_cast<unsigned long long *>(p); p += align256(kSeedMax * 8);
        q.acc = ws->bacc;
    }
    if (!cuda_ok(cudaMemcpy(ws->bslots_dev, host.data(), B * sizeof(QuerySlot), cudaMemcpyHostToDevice),
                 "messi_query_batched: slot table upload"))
        return MESSI_ECUDA;
    return MESSI_OK;
}

}  // namespace

// f16 tile copy of the rows for the tensor-core screen (built on first use).
messi_status ensure_screen_copy(messi_index *ix, cudaStream_t s)
{
    if (ix->screen_state != 0) return MESSI_OK;
    if (ix->len % 16 || ix->len > (int)kTcMaxLenHost) {
        ix->screen_state = -1;
        return MESSI_OK;
    }
    const unsigned long long rows = (ix->N + 127) / 128 * 128;
    char *p = nullptr;
    const size_t b16 = align256(rows * ix->len * 2), bn = align256(rows * 4);
    if (cudaMalloc(&p, b16 + 2 * bn + 256) != cudaSuccess) {
        cudaGetLastError();
        ix->screen_state = -1;   // no room: the batched path uses the lower-bound kernels
        return MESSI_OK;
    }
    ix->screen16 = reinterpret_cast<__half *>(p);
    ix->xn = reinterpret_cast<float *>(p + b16);
    ix->xnorm = reinterpret_cast<float *>(p + b16 + bn);
    unsigned *bad = reinterpret_cast<unsigned *>(p + b16 + 2 * bn);
    MESSI_CUDA(cudaMemsetAsync(bad, 0, 4, s));
    launch_make_screen_copy(ix->raw, ix->N, ix->len, ix->screen16, ix->xn, ix->xnorm, bad, s);
    ++ix->launches;
    unsigned hbad = 0;
    MESSI_CUDA(cudaMemcpyAsync(&hbad, bad, 4, cudaMemcpyDeviceToHost, s));
    MESSI_CUDA(cudaStreamSynchronize(s));
    if (hbad) {
        cudaFree(p);
        ix->screen16 = nullptr;
        ix->screen_state = -1;
        return MESSI_OK;
    }
    ix->device_bytes += b16 + 2 * bn + 256;
    ix->screen_state = 1;
    return MESSI_OK;
}

namespace {

struct TcWs {
    __half *qtiles, *qtiles2;       // the batch's query tiles; those screened again, gathered
    float *qconst;
    unsigned *Ubits, *cand_count, *flags, *active, *cand_pos, *n_active, *qmap;
    float *tkinit;                  // per query: its k smallest upper ends (from the seed leaf's k best)
    unsigned *glock;                // per query: the lock of that list
    uint2 *srange;                  // per query: the seed leaf's positions
};

TcWs tc_ws_view(messi_index *ix, Workspace *ws)
{
    const unsigned P = (ws->tcws_B + 127) / 128 * 128;
    char *p = static_cast<char *>(ws->tcws_block);
    TcWs w;
    w.qtiles = reinterpret_cast<__half *>(p); p += align256((size_t)P * ix->len * 2);
    w.qconst = reinterpret_cast<float *>(p); p += align256((size_t)P * 16);
    w.Ubits = reinterpret_cast<unsigned *>(p); p += align256((size_t)P * 4);
    w.cand_count = reinterpret_cast<unsigned *>(p); p += align256((size_t)P * 4);
    w.flags = reinterpret_cast<unsigned *>(p); p += align256((size_t)P * 4);
    w.active = reinterpret_cast<unsigned *>(p); p += align256((size_t)P * 4);
    w.n_active = reinterpret_cast<unsigned *>(p); p += 256;
    w.qtiles2 = reinterpret_cast<__half *>(p); p += align256((size_t)P * ix->len * 2);
    w.qmap = reinterpret_cast<unsigned *>(p); p += align256((size_t)P * 4);
    w.tkinit = reinterpret_cast<float *>(p); p += align256((size_t)P * kTcTopKHost * 4);
    w.glock = reinterpret_cast<unsigned *>(p); p += align256((size_t)P * 4);
    w.srange = reinterpret_cast<uint2 *>(p); p += align256((size_t)P * 8);
    w.cand_pos = reinterpret_cast<unsigned *>(p);
    return w;
}

messi_status ensure_tc_workspace(messi_index *ix, Workspace *ws, unsigned B)
{
    if (ws->tcws_block && ws->tcws_B >= B) return MESSI_OK;
    if (ws->tcws_block) {
        cudaFree(ws->tcws_block);
        ix->device_bytes -= ws->tcws_bytes;
        ws->tcws_block = nullptr;
    }
    const size_t P = (B + 127) / 128 * 128;
    const size_t bytes = 2 * align256(P * ix->len * 2) + align256(P * 16) + 6 * align256(P * 4) + 256 +
                         align256(P * kTcTopKHost * 4) + align256(P * 8) + P * kTcCap * 4;
    if (cudaMalloc(&ws->tcws_block, bytes) != cudaSuccess) {
        cudaGetLastError();
        ws->tcws_block = nullptr;
        return fail(MESSI_ENOMEM, "messi_query_batched: cannot allocate the screening workspace");
    }
    ws->tcws_bytes = bytes;
    ws->tcws_B = B;
    ix->device_bytes += bytes;
    return MESSI_OK;
}

cudaEvent_t pool_event(Workspace *ws, size_t i)
{
    while (ws->ev_pool.size() <= i) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        ws->ev_pool.push_back(e);
    }
    return ws->ev_pool[i];
}

messi_status check_sizes(uint64_t n, uint32_t len, uint32_t segments, uint32_t card)
{
    if (n == 0 || n >= 0xffffffffull) return fail(MESSI_EINVAL, "n must be in [1, 2^32-1)");
    if (segments == 0 || segments > (unsigned)kMaxSegments)
        return fail(MESSI_EINVAL, "segments must be in [1, 16]");
    if (len == 0 || len > (unsigned)kMaxLen || len % segments)
        return fail(MESSI_EINVAL, "len must be a multiple of segments and at most 4096");
    const unsigned m = len / segments;
    if (m < 4 || !is_pow2(m)) return fail(MESSI_EINVAL, "len/segments must be a power of two >= 4");
    if (!is_pow2(card) || card < 2 || card > (unsigned)kMaxCard)
        return fail(MESSI_EINVAL, "cardinality must be a power of two in [2, 256]");
    return MESSI_OK;
}

}  // namespace

IndexView view_of(const messi_index *ix)
{
    IndexView v;
    v.raw = ix->raw;
    v.sax = ix->sax;
    v.ids = ix->ids;
    v.pos_of_id = ix->pos_of_id;
    v.leaf_off = ix->leaf_off;
    v.leaf_key = ix->leaf_key;
    v.leaf_box = ix->leaf_box;
    v.beta64 = ix->beta64;
    v.N = ix->N;
    v.L = ix->L;
    v.len = ix->len;
    v.w = ix->w;
    v.card = ix->card;
    v.bits = ix->bits;
    v.m = ix->m;
    v.status = ix->status;
    return v;
}

bool is_device_ptr(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

messi_status check_device(const messi_index *ix, const void *const *ptrs, int n, const char *where)
{
    int dev = 0;
    if (!cuda_ok(cudaGetDevice(&dev), where)) return MESSI_ECUDA;
    if (dev != ix->device)
        return fail(MESSI_EINVAL, std::string(where) + ": the index lives on device " + std::to_string(ix->device) +
                                      " but device " + std::to_string(dev) + " is current");
    for (int i = 0; i < n; ++i) {
        if (!ptrs[i]) continue;
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, ptrs[i]) != cudaSuccess) {
            cudaGetLastError();
            continue;   // not CUDA memory: a host pointer
        }
        if (a.type == cudaMemoryTypeDevice && a.device != dev)
            return fail(MESSI_EINVAL, std::string(where) + ": a buffer lives on device " + std::to_string(a.device) +
                                          ", not on the index's device " + std::to_string(dev));
    }
    return MESSI_OK;
}

QueryParams make_params(const messi_index *ix, uint32_t k, int dist, uint32_t window)
{
    QueryParams qp;
    qp.k = (int)k;
    qp.dist = dist;
    qp.r = dist == MESSI_DTW ? (int)window : 0;
    qp.F = band_factor(dist, ix->len);
    qp.lock_spin = ix->lock_spin;
    return qp;
}

void set_error(const std::string &msg) { g_last_error = msg; }

messi_status fail(messi_status st, const std::string &msg)
{
    g_last_error = msg;
    return st;
}

bool cuda_ok(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return true;
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    cudaGetLastError();
    return false;
}

void free_workspace(Workspace &w)
{
    void *ptrs[] = {w.ws_block, w.stage_block, w.bws_block, w.tcws_block, w.gargs_dev, w.gcursor, w.redo_dev};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (w.gargs_host) cudaFreeHost(w.gargs_host);
    if (w.redo_host) cudaFreeHost(w.redo_host);
    if (w.graph) cudaGraphExecDestroy(w.graph);
    if (w.gargs_done) cudaEventDestroy(w.gargs_done);
    if (w.capture_stream) cudaStreamDestroy(w.capture_stream);
    for (cudaEvent_t e : w.ev_pool) cudaEventDestroy(e);
    for (Workspace *sw : w.sub) {
        if (!sw) continue;
        free_workspace(*sw);
        delete sw;
    }
    for (cudaStream_t t : w.sub_streams) cudaStreamDestroy(t);
    for (cudaEvent_t e : w.sub_done) cudaEventDestroy(e);
    if (w.fork) cudaEventDestroy(w.fork);
    w = Workspace{};
}

int num_sms()
{
    static int cached[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (!cached[dev]) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        cached[dev] = v > 0 ? v : 1;
    }
    return cached[dev];
}

}  // namespace messi

using namespace messi;

extern "C" {

const char *messi_last_error(void) { return g_last_error.c_str(); }

messi_status messi_breakpoints(uint32_t cardinality, double *out)
{
    if (!out || !is_pow2(cardinality) || cardinality < 2 || cardinality > (unsigned)kMaxCard)
        return fail(MESSI_EINVAL, "messi_breakpoints: cardinality must be a power of two in [2, 256]");
    compute_breakpoints((int)cardinality, out);
    return MESSI_OK;
}

void messi_free(messi_index *ix)
{
    if (!ix) return;
    void *ptrs[] = {ix->raw,      ix->sax,        ix->ids,    ix->pos_of_id, ix->leaf_off,
                    ix->leaf_key, ix->leaf_depth, ix->beta64, ix->status,    ix->screen16,
                    ix->leaf_box};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    free_workspace(ix->ws);
    delete ix;
}

messi_status messi_index_get_info(const messi_index *ix, messi_index_info *out)
{
    if (!ix || !out) return fail(MESSI_EINVAL, "messi_index_get_info: null argument");
    out->n_series = ix->N;
    out->len = ix->len;
    out->segments = ix->w;
    out->cardinality = ix->card;
    out->leaf_capacity = ix->cap;
    out->n_leaves = ix->L;
    out->max_leaf_size = ix->max_leaf;
    out->device_bytes = ix->device_bytes.load();
    out->build_ms = ix->build_ms;
    return MESSI_OK;
}

messi_status messi_build(const float *series, uint64_t n, uint32_t len, uint32_t segments,
                         uint32_t cardinality, const messi_config *cfg, messi_stream stream,
                         messi_index **out)
{
    if (!series || !out) return fail(MESSI_EINVAL, "messi_build: null argument");
    *out = nullptr;
    messi_status chk = check_sizes(n, len, segments, cardinality);
    if (chk != MESSI_OK) return chk;
    const unsigned cap = (cfg && cfg->leaf_capacity) ? cfg->leaf_capacity : 2000u;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    ensure_attributes();
    {
        // what the finished index holds at least (rows in leaf order, words,
        // ids both ways), plus the staging copy of host series: more than the
        // device has free is refused before anything is allocated or read
        const bool host_series = !is_device_ptr(series);
        const double need = (double)n * len * 4.0 * (host_series ? 2.0 : 1.0) + (double)n * 24.0;
        size_t free_b = 0, total_b = 0;
        if (!cuda_ok(cudaMemGetInfo(&free_b, &total_b), "messi_build: cudaMemGetInfo")) return MESSI_ECUDA;
        if (need > (double)free_b)
            return fail(MESSI_ENOMEM, "messi_build: the index needs at least " + std::to_string((long long)(need / 1e6)) +
                                          " MB of device memory, " + std::to_string(free_b / 1000000) + " MB are free");
    }

    messi_index *ix = new messi_index();
    cudaGetDevice(&ix->device);
    ix->N = n;
    ix->len = (int)len;
    ix->w = (int)segments;
    ix->card = (int)cardinality;
    while ((1 << ix->bits) < ix->card) ++ix->bits;
    ix->m = ix->len / ix->w;
    ix->cap = cap;
    compute_breakpoints(ix->card, ix->beta_host);

    std::vector<void *> tmp;
    auto bail = [&](messi_status st, const std::string &msg) {
        for (void *p : tmp) cudaFree(p);
        messi_free(ix);
        cudaGetLastError();
        return fail(st, msg);
    };
    auto talloc = [&](void **p, size_t bytes) {
        if (cudaMalloc(p, std::max<size_t>(bytes, 1)) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        tmp.push_back(*p);
        return true;
    };

    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);

    if (cudaMalloc(&ix->beta64, kMaxCard * 8) != cudaSuccess || cudaMalloc(&ix->status, 256) != cudaSuccess)
        return bail(MESSI_ENOMEM, "messi_build: cannot allocate breakpoint tables");
    float beta32_h[kMaxCard];
    for (int j = 0; j < ix->card - 1; ++j) beta32_h[j] = (float)ix->beta_host[j];
    float *beta32 = nullptr;
    if (!talloc((void **)&beta32, kMaxCard * 4)) return bail(MESSI_ENOMEM, "messi_build: out of device memory");
    if (cudaMemcpyAsync(ix->beta64, ix->beta_host, (ix->card - 1) * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(beta32, beta32_h, (ix->card - 1) * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(ix->status, 0, 256, s) != cudaSuccess)
        return bail(MESSI_ECUDA, "messi_build: cannot upload breakpoints");

    const float *dseries = series;
    const size_t raw_bytes = (size_t)n * len * 4;
    if (!is_device_ptr(series)) {
        float *d = nullptr;
        if (!talloc((void **)&d, raw_bytes)) return bail(MESSI_ENOMEM, "messi_build: cannot stage host series");
        if (cudaMemcpyAsync(d, series, raw_bytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
            return bail(MESSI_ECUDA, "messi_build: host-to-device copy failed");
        dseries = d;
    }

    uint4 *keys = nullptr, *keys_alt = nullptr, *sax_tmp = nullptr;
    unsigned *vals_alt = nullptr;
    void *sort_tmp = nullptr;
    if (!talloc((void **)&keys, n * 16) || !talloc((void **)&keys_alt, n * 16) ||
        !talloc((void **)&sax_tmp, n * 16) || !talloc((void **)&vals_alt, n * 4) ||
        !talloc(&sort_tmp, radix_sort_temp_bytes(n)))
        return bail(MESSI_ENOMEM, "messi_build: cannot allocate sort buffers");
    if (cudaMalloc(&ix->ids, n * 4) != cudaSuccess) return bail(MESSI_ENOMEM, "messi_build: out of device memory");

    NvtxRange r_build("messi:build");
    // a non-finite value makes its segment sum non-finite; the kernel flags it
    // in the status word, read once the build has finished
    launch_summarize(dseries, n, ix->len, ix->w, ix->card, ix->beta64, beta32, sax_tmp, keys, ix->ids,
                     ix->status, s);
    ++ix->launches;
    radix_sort_keys(keys, ix->ids, keys_alt, vals_alt, n, ix->w * ix->bits, sort_tmp, s, &ix->launches);
    if (!cuda_ok(cudaStreamSynchronize(s), "messi_build: summarise/sort")) return bail(MESSI_ECUDA, g_last_error);
    cudaFree(keys_alt);
    cudaFree(vals_alt);
    cudaFree(sort_tmp);
    tmp.erase(std::remove_if(tmp.begin(), tmp.end(),
                             [&](void *p) { return p == keys_alt || p == vals_alt || p == sort_tmp; }),
              tmp.end());

    if (cudaMalloc(&ix->raw, raw_bytes) != cudaSuccess || cudaMalloc(&ix->sax, n * 16) != cudaSuccess ||
        cudaMalloc(&ix->pos_of_id, n * 4) != cudaSuccess)
        return bail(MESSI_ENOMEM, "messi_build: cannot allocate the index arrays");
    ix->device_bytes = raw_bytes + n * 16 + n * 8 + kMaxCard * 8 + 256;

    messi_status st = build_leaves(ix, keys, sax_tmp, dseries, s);
    if (st != MESSI_OK) return bail(st, g_last_error);
    cudaEventRecord(e1, s);
    if (!cuda_ok(cudaEventSynchronize(e1), "messi_build")) return bail(MESSI_ECUDA, g_last_error);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    ix->build_ms = ms;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (void *p : tmp) cudaFree(p);
    tmp.clear();

    unsigned status = 0;
    cudaMemcpy(&status, ix->status, 4, cudaMemcpyDeviceToHost);
    if (status & kStInvalidQuery) {
        messi_free(ix);
        return fail(MESSI_EINVAL, "messi_build: the series hold a non-finite value");
    }
    ix->ws.last_stream = s;
    *out = ix;
    return MESSI_OK;
}

}  // extern "C"

namespace messi {
static messi_status query_args(const messi_index *ix, const float *queries, uint32_t nq, uint32_t k,
                               messi_dist dist, uint32_t window, const int64_t *ids, const float *dists)
{
    if (!ix || !queries || !ids || !dists) return fail(MESSI_EINVAL, "messi_query: null argument");
    if (nq == 0) return fail(MESSI_EINVAL, "messi_query: nq must be >= 1");
    if (k == 0 || k > (uint32_t)kMaxK || k > ix->N) return fail(MESSI_EINVAL, "messi_query: k must be in [1, min(n, 1024)]");
    if (dist != MESSI_ED && dist != MESSI_DTW) return fail(MESSI_EINVAL, "messi_query: unknown distance");
    if (dist == MESSI_DTW && window >= (uint32_t)ix->len) return fail(MESSI_EINVAL, "messi_query: window must be < len");
    const void *ptrs[3] = {queries, ids, dists};
    return check_device(ix, ptrs, 3, "messi_query");
}

// The per-query kernel sequence of one query on stream s and slot workspace
// qws; profiling events (ix->profiling) are recorded on s and registered in
// ews, the workspace whose statistics the call reports.
static cudaError_t enqueue_query(messi_index *ix, Workspace *qws, Workspace *ews, const IndexView &iv,
                                 const QueryParams &qp, const float *q, long long *ids, float *dists, cudaStream_t s,
                                 size_t &evn)
{
    const QuerySlot slot = qws->slot;
    NvtxRange r_query("messi:query");
    int eq0 = -1, es0 = -1;
    if (ix->profiling >= 2) {
        eq0 = (int)evn;
        cudaEventRecord(pool_event(ews, evn++), s);
    }
    nvtxRangePushA("messi:prep+seed");
    launch_prep(iv, qp, slot, q, s);
    if (ix->hold_lock) {   // test hook: the k-array lock starts out held
        const cudaError_t e = cudaMemsetAsync(&slot.st->lock, 0xff, sizeof(unsigned), s);
        if (e != cudaSuccess) return e;
    }
    launch_seed(iv, qp, slot, s, &ews->launches);
    nvtxRangePop();
    if (ix->profiling) {
        es0 = (int)evn;
        cudaEventRecord(pool_event(ews, evn++), s);
    }
    nvtxRangePushA("messi:scan");
    launch_scan(iv, qp, slot, next_epoch(qws, s), s);
    nvtxRangePop();
    if (ix->profiling) {
        cudaEventRecord(pool_event(ews, evn++), s);
        ews->scan_ev.push_back({es0, es0 + 1});
    }
    cudaEvent_t r0 = nullptr, r1 = nullptr;
    if (ix->profiling) {
        ews->refine_ev.push_back({(int)evn, (int)evn + 1});
        r0 = pool_event(ews, evn++);
        r1 = pool_event(ews, evn++);
    }
    nvtxRangePushA("messi:refine+finalize");
    launch_refine(iv, qp, slot, s, &ews->launches, r0, r1);
    launch_finalize(iv, qp, slot, ids, dists, s);
    nvtxRangePop();
    ews->launches += 3;
    if (ix->profiling >= 2) {
        cudaEventRecord(pool_event(ews, evn++), s);
        ews->query_ev.push_back({eq0, (int)evn - 1});
    }
    return cudaGetLastError();
}

messi_status run_plain(messi_index *ix, Workspace *ws, const float *queries, uint32_t nq, uint32_t k,
                       messi_dist dist, uint32_t window, int64_t *ids, float *dists, messi_stream stream)
{
    messi_status chk = query_args(ix, queries, nq, k, dist, window, ids, dists);
    if (chk != MESSI_OK) return chk;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    ensure_attributes();
    if ((chk = ensure_workspace(ix, ws)) != MESSI_OK) return chk;

    const bool hq = !is_device_ptr(queries), hi = !is_device_ptr(ids), hd = !is_device_ptr(dists);
    const size_t qbytes = (size_t)nq * ix->len * 4, ibytes = (size_t)nq * k * 8, dbytes = (size_t)nq * k * 4;
    const size_t need = (hq ? align256(qbytes) : 0) + (hi ? align256(ibytes) : 0) + (hd ? align256(dbytes) : 0);
    if (need && !ensure_stage(ws, need)) return fail(MESSI_ENOMEM, "messi_query: cannot allocate staging buffers");
    char *stage = static_cast<char *>(ws->stage_block);
    const float *dq = queries;
    long long *did = reinterpret_cast<long long *>(ids);
    float *ddist = dists;
    size_t so = 0;
    if (hq) {
        dq = reinterpret_cast<const float *>(stage + so);
        MESSI_CUDA(cudaMemcpyAsync(stage + so, queries, qbytes, cudaMemcpyHostToDevice, s));
        so += align256(qbytes);
    }
    if (hi) { did = reinterpret_cast<long long *>(stage + so); so += align256(ibytes); }
    if (hd) { ddist = reinterpret_cast<float *>(stage + so); so += align256(dbytes); }

    const IndexView iv = view_of(ix);
    const QueryParams qp = make_params(ix, k, (int)dist, window);
    const QuerySlot slot = ws->slot;
    MESSI_CUDA(cudaMemsetAsync(slot.acc, 0, sizeof(QueryCounters), s));
    const unsigned long long launches0 = ws->launches;
    ws->scan_ev.clear();
    ws->query_ev.clear();
    ws->refine_ev.clear();
    size_t evn = 0;
    for (uint32_t qi = 0; qi < nq; ++qi)
        MESSI_CUDA(enqueue_query(ix, ws, ws, iv, qp, dq + (size_t)qi * ix->len, did + (size_t)qi * k,
                                 ddist + (size_t)qi * k, s, evn));
    MESSI_CUDA(cudaGetLastError());
    ws->last = messi_stats{};
    ws->last.queries = nq;
    ws->last.kernel_launches = ws->launches - launches0;
    ws->last_stream = s;
    ws->last_batched = false;
    if (hi) MESSI_CUDA(cudaMemcpyAsync(ids, did, ibytes, cudaMemcpyDeviceToHost, s));
    if (hd) MESSI_CUDA(cudaMemcpyAsync(dists, ddist, dbytes, cudaMemcpyDeviceToHost, s));
    if (hq || hi || hd) MESSI_CUDA(cudaStreamSynchronize(s));
    return MESSI_OK;
}

// One query on the per-query kernels (the plain slot), for queries a batch
// could not settle.
static messi_status answer_one(messi_index *ix, Workspace *ws, const IndexView &iv, const QueryParams &qp,
                               const float *q, long long *ids, float *dists, cudaStream_t s)
{
    messi_status chk = ensure_workspace(ix, ws);
    if (chk != MESSI_OK) return chk;
    const QuerySlot one = ws->slot;
    MESSI_CUDA(cudaMemsetAsync(one.acc, 0, sizeof(QueryCounters), s));
    launch_prep(iv, qp, one, q, s);
    launch_seed(iv, qp, one, s, &ws->launches);
    launch_scan(iv, qp, one, next_epoch(ws, s), s);
    launch_refine(iv, qp, one, s, &ws->launches);
    launch_finalize(iv, qp, one, ids, dists, s);
    ws->launches += 3;
    return MESSI_OK;
}

// Per-query redo flags of a batched call (device, pinned host copy).
static messi_status ensure_redo(Workspace *ws, size_t nq)
{
    if (ws->redo_cap >= nq) return MESSI_OK;
    if (ws->redo_dev) cudaFree(ws->redo_dev);
    if (ws->redo_host) cudaFreeHost(ws->redo_host);
    ws->redo_dev = nullptr;
    ws->redo_host = nullptr;
    ws->redo_cap = 0;
    if (cudaMalloc(&ws->redo_dev, nq * 4) != cudaSuccess || cudaMallocHost(&ws->redo_host, nq * 4) != cudaSuccess) {
        cudaGetLastError();
        return fail(MESSI_ENOMEM, "messi_query_batched: cannot allocate the redo flags");
    }
    ws->redo_cap = nq;
    return MESSI_OK;
}

// The lower-bound batch form as a CUDA graph: one batch (prep, seed, fused
// scan-and-refine, finalize, cursor advance) is captured once per shape on a
// private stream, with its query rows and result rows read from an argument
// table; every full batch of a call is then one graph launch on the caller's
// stream, the table advancing by one entry per replay.
static messi_status replay_lb_batches(messi_index *ix, Workspace *ws, const IndexView &iv, const QueryParams &qp,
                                      unsigned B, unsigned nfull, const float *dq, long long *did, float *ddist,
                                      unsigned *redo, cudaStream_t s)
{
    if (!ws->capture_stream && !cuda_ok(cudaStreamCreateWithFlags(&ws->capture_stream, cudaStreamNonBlocking),
                                        "messi_query_batched: capture stream"))
        return MESSI_ECUDA;
    if (!ws->gargs_done && !cuda_ok(cudaEventCreateWithFlags(&ws->gargs_done, cudaEventDisableTiming),
                                    "messi_query_batched: event"))
        return MESSI_ECUDA;
    if (ws->gargs_cap < nfull) {
        if (ws->gargs_dev) cudaFree(ws->gargs_dev);
        if (ws->gargs_host) cudaFreeHost(ws->gargs_host);
        ws->gargs_dev = nullptr;
        ws->gargs_host = nullptr;
        ws->gargs_cap = 0;
        if (cudaMalloc(&ws->gargs_dev, nfull * sizeof(BatchArgs)) != cudaSuccess ||
            cudaMallocHost(&ws->gargs_host, nfull * sizeof(BatchArgs)) != cudaSuccess) {
            cudaGetLastError();
            return fail(MESSI_ENOMEM, "messi_query_batched: cannot allocate the batch argument table");
        }
        ws->gargs_cap = nfull;
    }
    if (!ws->gcursor && cudaMalloc(&ws->gcursor, 4) != cudaSuccess) {
        cudaGetLastError();
        return fail(MESSI_ENOMEM, "messi_query_batched: cannot allocate the batch cursor");
    }
    const unsigned long long key[4] = {B, (unsigned long long)qp.k,
                                       ((unsigned long long)ix->tune_chunk_tiles << 8) | ix->tune_ctas_per_sm,
                                       (unsigned long long)(uintptr_t)ws->bslots_dev};
    if (!ws->graph || std::memcmp(key, ws->graph_key, sizeof(key)) != 0) {
        if (ws->graph) cudaGraphExecDestroy(ws->graph);
        ws->graph = nullptr;
        cudaGraph_t graph = nullptr;
        MESSI_CUDA(cudaStreamBeginCapture(ws->capture_stream, cudaStreamCaptureModeThreadLocal));
        launch_batch_args(iv, qp, ws->bslots_dev, B, ws->gargs_dev, ws->gcursor, ix->tune_chunk_tiles,
                          ix->tune_ctas_per_sm, ws->bcounter, ws->capture_stream);
        MESSI_CUDA(cudaStreamEndCapture(ws->capture_stream, &graph));
        const cudaError_t e = cudaGraphInstantiate(&ws->graph, graph, 0);
        cudaGraphDestroy(graph);
        if (!cuda_ok(e, "messi_query_batched: graph instantiation")) {
            ws->graph = nullptr;
            return MESSI_ECUDA;
        }
        std::memcpy(ws->graph_key, key, sizeof(key));
    }
    // the staging table may still feed the previous call's copy
    MESSI_CUDA(cudaEventSynchronize(ws->gargs_done));
    for (unsigned b = 0; b < nfull; ++b)
        ws->gargs_host[b] = BatchArgs{dq + (size_t)b * B * ix->len, did + (size_t)b * B * qp.k,
                                      ddist + (size_t)b * B * qp.k, redo + (size_t)b * B};
    MESSI_CUDA(cudaMemcpyAsync(ws->gargs_dev, ws->gargs_host, nfull * sizeof(BatchArgs), cudaMemcpyHostToDevice, s));
    MESSI_CUDA(cudaEventRecord(ws->gargs_done, s));
    MESSI_CUDA(cudaMemsetAsync(ws->gcursor, 0, 4, s));
    for (unsigned b = 0; b < nfull; ++b) MESSI_CUDA(cudaGraphLaunch(ws->graph, s));
    ws->launches += 7ull * nfull;
    ws->graph_replays += nfull;
    return MESSI_OK;
}

// Batched DTW: the queries' per-query kernel sequences run side by side on up
// to kDtwStreams streams, each with a workspace of its own, so that the small
// grids of one query (its seed leaf, the DTW of few candidates) share the GPU
// with the others' work.  The streams start after the caller's stream reaches
// this call and the caller's stream continues once all of them are done.
static messi_status run_dtw_batched(messi_index *ix, Workspace *ws, const float *dq, uint32_t nq, uint32_t k,
                                    const QueryParams &qp, long long *did, float *ddist, cudaStream_t s)
{
    const unsigned want = std::min<unsigned>(kDtwStreams, nq);
    while (ws->sub.size() < want) {
        Workspace *sw = new Workspace();
        cudaStream_t t = nullptr;
        cudaEvent_t e = nullptr;
        if (ensure_workspace(ix, sw) != MESSI_OK ||
            cudaStreamCreateWithFlags(&t, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            if (t) cudaStreamDestroy(t);
            free_workspace(*sw);
            delete sw;
            break;   // run on the streams there is memory for
        }
        ws->sub.push_back(sw);
        ws->sub_streams.push_back(t);
        ws->sub_done.push_back(e);
    }
    if (!ws->fork && !cuda_ok(cudaEventCreateWithFlags(&ws->fork, cudaEventDisableTiming), "messi_query_batched: event"))
        return MESSI_ECUDA;
    const unsigned S = std::min<unsigned>(want, (unsigned)ws->sub.size());
    if (S == 0) return fail(MESSI_ENOMEM, "messi_query_batched: cannot allocate a DTW stream workspace");
    const IndexView iv = view_of(ix);
    MESSI_CUDA(cudaEventRecord(ws->fork, s));
    for (unsigned j = 0; j < S; ++j) {
        MESSI_CUDA(cudaStreamWaitEvent(ws->sub_streams[j], ws->fork, 0));
        MESSI_CUDA(cudaMemsetAsync(ws->sub[j]->slot.acc, 0, sizeof(QueryCounters), ws->sub_streams[j]));
    }
    size_t evn = 0;
    for (uint32_t qi = 0; qi < nq; ++qi) {
        const unsigned j = qi % S;
        MESSI_CUDA(enqueue_query(ix, ws->sub[j], ws, iv, qp, dq + (size_t)qi * ix->len, did + (size_t)qi * k,
                                 ddist + (size_t)qi * k, ws->sub_streams[j], evn));
    }
    const QueryCounters *accs[kDtwStreams];
    for (unsigned j = 0; j < S; ++j) {
        MESSI_CUDA(cudaEventRecord(ws->sub_done[j], ws->sub_streams[j]));
        MESSI_CUDA(cudaStreamWaitEvent(s, ws->sub_done[j], 0));
        accs[j] = ws->sub[j]->slot.acc;
    }
    launch_add_counters(ws->slot.acc, accs, (int)S, s);
    ++ws->launches;
    return MESSI_OK;
}

messi_status run_batched(messi_index *ix, Workspace *ws, const float *queries, uint32_t nq, uint32_t k,
                         messi_dist dist, uint32_t window, uint32_t batch, int64_t *ids, float *dists,
                         messi_stream stream)
{
    messi_status chk = query_args(ix, queries, nq, k, dist, window, ids, dists);
    if (chk != MESSI_OK) return chk;
    if (dist == MESSI_DTW) {
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        ensure_attributes();
        if ((chk = ensure_workspace(ix, ws)) != MESSI_OK) return chk;
        const bool hq = !is_device_ptr(queries), hi = !is_device_ptr(ids), hd = !is_device_ptr(dists);
        const size_t qbytes = (size_t)nq * ix->len * 4, ibytes = (size_t)nq * k * 8, dbytes = (size_t)nq * k * 4;
        const size_t need = (hq ? align256(qbytes) : 0) + (hi ? align256(ibytes) : 0) + (hd ? align256(dbytes) : 0);
        if (need && !ensure_stage(ws, need)) return fail(MESSI_ENOMEM, "messi_query_batched: cannot allocate staging buffers");
        char *stage = static_cast<char *>(ws->stage_block);
        const float *dq = queries;
        long long *did = reinterpret_cast<long long *>(ids);
        float *ddist = dists;
        size_t so = 0;
        if (hq) {
            dq = reinterpret_cast<const float *>(stage + so);
            MESSI_CUDA(cudaMemcpyAsync(stage + so, queries, qbytes, cudaMemcpyHostToDevice, s));
            so += align256(qbytes);
        }
        if (hi) { did = reinterpret_cast<long long *>(stage + so); so += align256(ibytes); }
        if (hd) { ddist = reinterpret_cast<float *>(stage + so); so += align256(dbytes); }
        const unsigned long long launches0 = ws->launches;
        ws->scan_ev.clear();
        ws->query_ev.clear();
        ws->refine_ev.clear();
        const QueryParams qp = make_params(ix, k, (int)dist, window);
        if ((chk = run_dtw_batched(ix, ws, dq, nq, k, qp, did, ddist, s)) != MESSI_OK) return chk;
        MESSI_CUDA(cudaGetLastError());
        ws->last = messi_stats{};
        ws->last.queries = nq;
        ws->last.kernel_launches = ws->launches - launches0;
        ws->last_stream = s;
        ws->last_batched = false;
        if (hi) MESSI_CUDA(cudaMemcpyAsync(ids, did, ibytes, cudaMemcpyDeviceToHost, s));
        if (hd) MESSI_CUDA(cudaMemcpyAsync(dists, ddist, dbytes, cudaMemcpyDeviceToHost, s));
        // the call synchronises, as the other batched forms do
        MESSI_CUDA(cudaStreamSynchronize(s));
        return MESSI_OK;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    ensure_attributes();
    const unsigned B = std::min<unsigned>(batch ? batch : ix->tune_batch, nq);
    if ((chk = ensure_batch_workspace(ix, ws, B)) != MESSI_OK) return chk;

    const bool hq = !is_device_ptr(queries), hi = !is_device_ptr(ids), hd = !is_device_ptr(dists);
    const size_t qbytes = (size_t)nq * ix->len * 4, ibytes = (size_t)nq * k * 8, dbytes = (size_t)nq * k * 4;
    const size_t need = (hq ? align256(qbytes) : 0) + (hi ? align256(ibytes) : 0) + (hd ? align256(dbytes) : 0);
    if (need && !ensure_stage(ws, need)) return fail(MESSI_ENOMEM, "messi_query_batched: cannot allocate staging buffers");
    char *stage = static_cast<char *>(ws->stage_block);
    const float *dq = queries;
    long long *did = reinterpret_cast<long long *>(ids);
    float *ddist = dists;
    size_t so = 0;
    if (hq) {
        dq = reinterpret_cast<const float *>(stage + so);
        MESSI_CUDA(cudaMemcpyAsync(stage + so, queries, qbytes, cudaMemcpyHostToDevice, s));
        so += align256(qbytes);
    }
    if (hi) { did = reinterpret_cast<long long *>(stage + so); so += align256(ibytes); }
    if (hd) { ddist = reinterpret_cast<float *>(stage + so); so += align256(dbytes); }

    const IndexView iv = view_of(ix);
    const QueryParams qp = make_params(ix, k, MESSI_ED, 0);
    MESSI_CUDA(cudaMemsetAsync(ws->bacc, 0, sizeof(QueryCounters), s));
    const unsigned long long launches0 = ws->launches;
    ws->scan_ev.clear();
    ws->query_ev.clear();
    ws->refine_ev.clear();
    size_t evn = 0;
    unsigned long long screened = 0;
    bool use_tc = ix->batch_mode == 1;
    if (use_tc && (chk = ensure_screen_copy(ix, s)) != MESSI_OK) return chk;
    use_tc = use_tc && ix->screen_state == 1;
    if (use_tc && (chk = ensure_tc_workspace(ix, ws, B)) != MESSI_OK) return chk;
    if ((chk = ensure_redo(ws, nq)) != MESSI_OK) return chk;
    for (uint32_t g = 0; g < nq && use_tc; g += B) {
        const unsigned nb = std::min<unsigned>(B, nq - g);
        int eq0 = -1, es0 = -1;
        if (ix->profiling >= 2) {
            eq0 = (int)evn;
            cudaEventRecord(pool_event(ws, evn++), s);
        }
        NvtxRange r_batch("messi:screened batch");
        const TcWs w = tc_ws_view(ix, ws);
        launch_batch_seed(iv, qp, ws->bslots_dev, nb, dq + (size_t)g * ix->len, s, &ws->launches);
        launch_tc_qprep(ws->bslots_dev, nb, ix->len, qp, w.qtiles, w.qconst, w.Ubits, w.cand_count, w.flags,
                        w.active, w.tkinit, w.glock, w.srange, s);
        ++ws->launches;
        // pass 0 screens the batch; later passes only the queries whose
        // candidate lists overflowed, gathered into the first query tiles
        unsigned more = 1, count = nb;
        const __half *qt = w.qtiles;
        const unsigned *qm = nullptr;
        const size_t qtiles_bytes = (size_t)(ws->tcws_B + 127) / 128 * 128 * ix->len * 2;
        for (int pass = 0; pass < 3 && more; ++pass) {
            if (ix->profiling) {
                es0 = (int)evn;
                cudaEventRecord(pool_event(ws, evn++), s);
            }
            launch_tc_screen(ix->screen16, ix->xn, ix->xnorm, qt, w.qconst, w.Ubits, w.cand_count, w.cand_pos,
                             w.active, qm, w.tkinit, w.glock, pass == 0 ? 1 : 0, w.srange, kTcCap, ix->N, ix->len,
                             count, (int)k, ix->status, s);
            screened += count;
            if (ix->profiling) {
                cudaEventRecord(pool_event(ws, evn++), s);
                ws->scan_ev.push_back({es0, es0 + 1});
            }
            launch_tc_recheck(iv, qp, ws->bslots_dev, nb, w.cand_count, w.cand_pos, kTcCap, w.active, s);
            MESSI_CUDA(cudaMemsetAsync(w.n_active, 0, 4, s));
            // rows past the gathered queries stay zero
            MESSI_CUDA(cudaMemsetAsync(w.qtiles2, 0, qtiles_bytes, s));
            launch_tc_next_pass(ws->bslots_dev, nb, qp, kTcCap, w.Ubits, w.cand_count, w.active, w.n_active, w.qtiles,
                                w.qtiles2, w.qmap, ix->len, s);
            ws->launches += 3;
            MESSI_CUDA(cudaMemcpyAsync(&more, w.n_active, 4, cudaMemcpyDeviceToHost, s));
            MESSI_CUDA(cudaStreamSynchronize(s));
            count = more;
            qt = w.qtiles2;
            qm = w.qmap;
        }
        launch_batch_finalize(iv, qp, ws->bslots_dev, nb, did + (size_t)g * k, ddist + (size_t)g * k,
                              ws->redo_dev + g, s, &ws->launches);
        // queries the screen could not settle (values outside f16 range, still
        // overflowing after three passes, or a near-tie log that overflowed):
        // the per-query kernels
        std::vector<unsigned> hflags(nb), hact(nb), hredo(nb);
        MESSI_CUDA(cudaMemcpyAsync(hflags.data(), w.flags, nb * 4, cudaMemcpyDeviceToHost, s));
        MESSI_CUDA(cudaMemcpyAsync(hact.data(), w.active, nb * 4, cudaMemcpyDeviceToHost, s));
        MESSI_CUDA(cudaMemcpyAsync(hredo.data(), ws->redo_dev + g, nb * 4, cudaMemcpyDeviceToHost, s));
        MESSI_CUDA(cudaStreamSynchronize(s));
        for (unsigned b = 0; b < nb; ++b)
            if ((hflags[b] & 4u) || hact[b] || hredo[b])
                if ((chk = answer_one(ix, ws, iv, qp, dq + (size_t)(g + b) * ix->len, did + (size_t)(g + b) * k,
                                      ddist + (size_t)(g + b) * k, s)) != MESSI_OK)
                    return chk;
        if (ix->profiling >= 2) {
            cudaEventRecord(pool_event(ws, evn++), s);
            for (unsigned r = 0; r < nb; ++r) ws->query_ev.push_back({eq0, (int)evn - 1});
        }
    }
    // full batches of the lower-bound form replay one captured graph
    uint32_t g_first = 0;
    if (!use_tc && !ix->profiling && nq / B >= 2) {
        chk = replay_lb_batches(ix, ws, iv, qp, B, nq / B, dq, did, ddist, ws->redo_dev, s);
        if (chk != MESSI_OK) return chk;
        g_first = (nq / B) * B;
    }
    for (uint32_t g = g_first; g < nq && !use_tc; g += B) {
        const unsigned nb = std::min<unsigned>(B, nq - g);
        int eq0 = -1, es0 = -1;
        cudaEvent_t f0 = nullptr, f1 = nullptr;
        if (ix->profiling) {
            if (ix->profiling >= 2) {
                eq0 = (int)evn;
                cudaEventRecord(pool_event(ws, evn++), s);
            }
            es0 = (int)evn;
            f0 = pool_event(ws, evn++);
            f1 = pool_event(ws, evn++);
        }
        launch_batch(iv, qp, ws->bslots_dev, nb, dq + (size_t)g * ix->len, did + (size_t)g * k, ddist + (size_t)g * k,
                     ws->redo_dev + g, ix->tune_chunk_tiles, ix->tune_ctas_per_sm, ws->bcounter, s, &ws->launches,
                     f0, f1);
        if (ix->profiling) ws->scan_ev.push_back({es0, es0 + 1});
        if (ix->profiling >= 2) {
            cudaEventRecord(pool_event(ws, evn++), s);
            for (unsigned r = 0; r < nb; ++r) ws->query_ev.push_back({eq0, (int)evn - 1});
        }
    }
    if (!use_tc) {
        // the lower-bound form runs without host decisions; queries whose
        // near-tie log overflowed (a mass tie) are answered again here
        MESSI_CUDA(cudaMemcpyAsync(ws->redo_host, ws->redo_dev, (size_t)nq * 4, cudaMemcpyDeviceToHost, s));
        MESSI_CUDA(cudaStreamSynchronize(s));
        for (uint32_t i = 0; i < nq; ++i)
            if (ws->redo_host[i])
                if ((chk = answer_one(ix, ws, iv, qp, dq + (size_t)i * ix->len, did + (size_t)i * k,
                                      ddist + (size_t)i * k, s)) != MESSI_OK)
                    return chk;
    }
    MESSI_CUDA(cudaGetLastError());
    ws->last = messi_stats{};
    ws->last.queries = nq;
    ws->last.kernel_launches = ws->launches - launches0;
    ws->last.screened_queries = screened;
    ws->last_stream = s;
    ws->last_batched = true;
    if (hi) MESSI_CUDA(cudaMemcpyAsync(ids, did, ibytes, cudaMemcpyDeviceToHost, s));
    if (hd) MESSI_CUDA(cudaMemcpyAsync(dists, ddist, dbytes, cudaMemcpyDeviceToHost, s));
    if (hq || hi || hd) MESSI_CUDA(cudaStreamSynchronize(s));
    return MESSI_OK;
}

}  // namespace messi

extern "C" {

messi_status messi_query(const messi_index *cix, const float *queries, uint32_t nq, uint32_t k,
                         messi_dist dist, uint32_t window, int64_t *ids, float *dists, messi_stream stream)
{
    if (!cix) return fail(MESSI_EINVAL, "messi_query: null index");
    messi_index *ix = const_cast<messi_index *>(cix);
    return run_plain(ix, &ix->ws, queries, nq, k, dist, window, ids, dists, stream);
}

messi_status messi_query_batched(const messi_index *cix, const float *queries, uint32_t nq, uint32_t k,
                                 messi_dist dist, uint32_t window, uint32_t batch, int64_t *ids, float *dists,
                                 messi_stream stream)
{
    if (!cix) return fail(MESSI_EINVAL, "messi_query_batched: null index");
    messi_index *ix = const_cast<messi_index *>(cix);
    return run_batched(ix, &ix->ws, queries, nq, k, dist, window, batch, ids, dists, stream);
}

messi_status messi_query_stats(const messi_index *cix, messi_stats *out)
{
    if (!cix || !out) return fail(MESSI_EINVAL, "messi_query_stats: null argument");
    messi_index *ix = const_cast<messi_index *>(cix);
    Workspace *ws = &ix->ws;
    *out = ws->last;
    const QueryCounters *acc = ws->last_batched ? ws->bacc : ws->slot.acc;
    if (!acc) return MESSI_OK;
    MESSI_CUDA(cudaStreamSynchronize(ws->last_stream));
    QueryCounters c{};
    MESSI_CUDA(cudaMemcpy(&c, acc, sizeof(c), cudaMemcpyDeviceToHost));
    out->lb_evaluated = c.lb_evaluated;
    out->lb_survivors = c.lb_survivors;
    out->lbk_survivors = c.lbk_survivors;
    out->seeded = c.seeded;
    out->refined = c.refined;
    out->abandoned = c.abandoned;
    out->bsf_updates = c.bsf_updates;
    out->tie_rechecks = c.tie_rechecks;
    out->leaves_live = c.leaves_live;
    out->row_bytes = c.row_bytes;
    out->dtw_cells = c.dtw_cells;
    if (ix->profiling) {
        double sum = 0.0;
        for (auto &pr : ws->scan_ev) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ws->ev_pool[pr.first], ws->ev_pool[pr.second]);
            sum += ms;
        }
        out->scan_ms = sum;
        out->scan_launches = ws->scan_ev.size();
        double rsum = 0.0;
        for (auto &pr : ws->refine_ev) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ws->ev_pool[pr.first], ws->ev_pool[pr.second]);
            rsum += ms;
        }
        out->refine_ms = rsum;
        out->refine_launches = ws->refine_ev.size();
        std::vector<double> lat;
        for (auto &pr : ws->query_ev) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ws->ev_pool[pr.first], ws->ev_pool[pr.second]);
            lat.push_back(ms);
        }
        if (!lat.empty()) {
            std::sort(lat.begin(), lat.end());
            auto pct = [&](double p) {
                size_t i = (size_t)std::ceil(p * lat.size()) - 1;
                return lat[std::min(i, lat.size() - 1)];
            };
            out->query_ms_p50 = pct(0.50);
            out->query_ms_p99 = pct(0.99);
        }
    }
    return MESSI_OK;
}

messi_status messi_set_batch_mode(messi_index *ix, int mode)
{
    if (!ix || (mode != MESSI_BATCH_LB_REFINE && mode != MESSI_BATCH_TC_SCREEN))
        return fail(MESSI_EINVAL, "messi_set_batch_mode: unknown mode");
    ix->batch_mode = mode;
    return MESSI_OK;
}

messi_status messi_set_tuning(messi_index *ix, const messi_tuning *t)
{
    if (!ix || !t) return fail(MESSI_EINVAL, "messi_set_tuning: null argument");
    if (t->batch == 0 || t->batch > 65535 || t->chunk_tiles == 0 || t->chunk_tiles > 1024 ||
        (t->ctas_per_sm != 1 && t->ctas_per_sm != 2))
        return fail(MESSI_EINVAL, "messi_set_tuning: batch 1..65535, chunk_tiles 1..1024, ctas_per_sm 1 or 2");
    ix->tune_batch = t->batch;
    ix->tune_chunk_tiles = t->chunk_tiles;
    ix->tune_ctas_per_sm = t->ctas_per_sm;
    return MESSI_OK;
}

messi_status messi_autotune(messi_index *ix, const float *queries, uint32_t nq, uint32_t k, messi_stream stream,
                            messi_tuning *out)
{
    if (!ix || !queries) return fail(MESSI_EINVAL, "messi_autotune: null argument");
    if (nq < 32) return fail(MESSI_EINVAL, "messi_autotune: needs at least 32 queries");
    if (!is_device_ptr(queries)) return fail(MESSI_EINVAL, "messi_autotune: queries must be a device pointer");
    if (k == 0 || k > (uint32_t)kMaxK || k > ix->N) return fail(MESSI_EINVAL, "messi_autotune: bad k");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    struct Shape { unsigned B, ct, cps; };
    std::vector<Shape> cand;
    if (ix->batch_mode == MESSI_BATCH_TC_SCREEN) {
        for (unsigned B : {128u, 256u, 512u, 1024u})
            if (B <= nq) cand.push_back({B, ix->tune_chunk_tiles, ix->tune_ctas_per_sm});
    } else {
        for (unsigned B : {32u, 64u, 128u, 256u})
            for (unsigned ct : {16u, 32u, 64u})
                for (unsigned cps : {1u, 2u})
                    if (B <= nq) cand.push_back({B, ct, cps});
    }
    if (cand.empty()) cand.push_back({std::min(nq, 32u), ix->tune_chunk_tiles, ix->tune_ctas_per_sm});
    const unsigned Bmax = std::max_element(cand.begin(), cand.end(), [](const Shape &a, const Shape &b) {
                              return a.B < b.B;
                          })->B;
    char *buf = nullptr;
    if (cudaMalloc(&buf, (size_t)Bmax * k * 12) != cudaSuccess) {
        cudaGetLastError();
        return fail(MESSI_ENOMEM, "messi_autotune: cannot allocate result buffers");
    }
    int64_t *ids = reinterpret_cast<int64_t *>(buf);
    float *dists = reinterpret_cast<float *>(buf + (size_t)Bmax * k * 8);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int prof = ix->profiling;
    ix->profiling = 0;
    double best = 1e300;
    Shape pick = cand.front();
    messi_status st = MESSI_OK;
    for (const Shape &c : cand) {
        ix->tune_chunk_tiles = c.ct;
        ix->tune_ctas_per_sm = c.cps;
        // warm-up, then one timed batch of c.B queries (the last rows, so warm-up and
        // timing see different queries when nq allows)
        st = run_batched(ix, &ix->ws, queries, c.B, k, MESSI_ED, 0, c.B, ids, dists, stream);
        if (st != MESSI_OK) break;
        const float *tq = queries + (size_t)(nq - c.B) * ix->len;
        cudaEventRecord(e0, s);
        st = run_batched(ix, &ix->ws, tq, c.B, k, MESSI_ED, 0, c.B, ids, dists, stream);
        if (st != MESSI_OK) break;
        cudaEventRecord(e1, s);
        if (!cuda_ok(cudaEventSynchronize(e1), "messi_autotune: timing")) {
            st = MESSI_ECUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double per = ms / c.B;
        if (per < best) {
            best = per;
            pick = c;
        }
    }
    ix->profiling = prof;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    if (st != MESSI_OK) return st;
    ix->tune_batch = pick.B;
    ix->tune_chunk_tiles = pick.ct;
    ix->tune_ctas_per_sm = pick.cps;
    if (out) {
        *out = messi_tuning{};
        out->batch = pick.B;
        out->chunk_tiles = pick.ct;
        out->ctas_per_sm = pick.cps;
        out->mode = (uint32_t)ix->batch_mode;
        out->ms_per_query = best;
    }
    return MESSI_OK;
}

messi_status messi_debug_set_lock_fault(messi_index *ix, uint32_t spin_limit, int hold_lock)
{
    if (!ix) return fail(MESSI_EINVAL, "messi_debug_set_lock_fault: null index");
    ix->lock_spin = spin_limit;
    ix->hold_lock = hold_lock != 0;
    return MESSI_OK;
}

messi_status messi_set_profiling(messi_index *ix, int enable)
{
    if (!ix) return fail(MESSI_EINVAL, "messi_set_profiling: null index");
    if (enable < 0 || enable > 2) return fail(MESSI_EINVAL, "messi_set_profiling: level 0, 1 or 2");
    ix->profiling = enable;
    return MESSI_OK;
}

messi_status messi_check(const messi_index *ix, messi_stream stream)
{
    if (!ix) return fail(MESSI_EINVAL, "messi_check: null index");
    MESSI_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    unsigned st = 0;
    MESSI_CUDA(cudaMemcpy(&st, ix->status, 4, cudaMemcpyDeviceToHost));
    MESSI_CUDA(cudaMemset(ix->status, 0, 4));
    if (st & kStTimeout) return fail(MESSI_ETIMEOUT, "a device-side bounded wait ran out");
    if (st & kStTieOverflow) return fail(MESSI_ETIES, "accepted near-tie candidates were dropped from a full log");
    if (st & kStInvalidQuery) return fail(MESSI_EINVAL, "a query held a non-finite value");
    return MESSI_OK;
}

messi_status messi_lower_bounds(const messi_index *cix, const float *query, messi_dist dist, uint32_t window,
                                float *lb2, messi_stream stream)
{
    if (!cix || !query || !lb2) return fail(MESSI_EINVAL, "messi_lower_bounds: null argument");
    if (dist != MESSI_ED && dist != MESSI_DTW) return fail(MESSI_EINVAL, "messi_lower_bounds: unknown distance");
    if (dist == MESSI_DTW && window >= (uint32_t)cix->len) return fail(MESSI_EINVAL, "messi_lower_bounds: window must be < len");
    messi_index *ix = const_cast<messi_index *>(cix);
    const void *ptrs[2] = {query, lb2};
    messi_status chk = check_device(ix, ptrs, 2, "messi_lower_bounds");
    if (chk != MESSI_OK) return chk;
    Workspace *ws = &ix->ws;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    ensure_attributes();
    chk = ensure_workspace(ix, ws);
    if (chk != MESSI_OK) return chk;
    const bool hq = !is_device_ptr(query), ho = !is_device_ptr(lb2);
    const size_t qbytes = (size_t)ix->len * 4, obytes = (size_t)ix->N * 4;
    if ((hq || ho) && !ensure_stage(ws, align256(qbytes) + align256(obytes)))
        return fail(MESSI_ENOMEM, "messi_lower_bounds: cannot allocate staging buffers");
    char *stage = static_cast<char *>(ws->stage_block);
    const float *dq = query;
    float *dout = lb2;
    if (hq) {
        MESSI_CUDA(cudaMemcpyAsync(stage, query, qbytes, cudaMemcpyHostToDevice, s));
        dq = reinterpret_cast<const float *>(stage);
    }
    if (ho) dout = reinterpret_cast<float *>(stage + align256(qbytes));
    const IndexView iv = view_of(ix);
    const QueryParams qp = make_params(ix, 1, (int)dist, window);
    launch_prep(iv, qp, ws->slot, dq, s);
    launch_lower_bounds(iv, ws->slot, dout, s);
    ix->launches += 2;
    MESSI_CUDA(cudaGetLastError());
    if (ho) MESSI_CUDA(cudaMemcpyAsync(lb2, dout, obytes, cudaMemcpyDeviceToHost, s));
    if (hq || ho) MESSI_CUDA(cudaStreamSynchronize(s));
    return MESSI_OK;
}

messi_status messi_summarize(const float *series, uint64_t n, uint32_t len, uint32_t segments,
                             uint32_t cardinality, uint8_t *words, messi_stream stream)
{
    if (!series || !words) return fail(MESSI_EINVAL, "messi_summarize: null argument");
    messi_status chk = check_sizes(n, len, segments, cardinality);
    if (chk != MESSI_OK) return chk;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double b64[kMaxCard];
    float b32[kMaxCard];
    compute_breakpoints((int)cardinality, b64);
    for (unsigned j = 0; j + 1 < cardinality; ++j) b32[j] = (float)b64[j];
    const bool hs = !is_device_ptr(series), hw = !is_device_ptr(words);
    const size_t sbytes = (size_t)n * len * 4, wbytes = (size_t)n * 16;
    char *tmp = nullptr;
    const size_t tbytes = align256(kMaxCard * 8) + align256(kMaxCard * 4) + (hs ? align256(sbytes) : 0) +
                          (hw ? align256(wbytes) : 0);
    if (cudaMalloc(&tmp, tbytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(MESSI_ENOMEM, "messi_summarize: out of device memory");
    }
    double *d64 = reinterpret_cast<double *>(tmp);
    float *d32 = reinterpret_cast<float *>(tmp + align256(kMaxCard * 8));
    size_t o = align256(kMaxCard * 8) + align256(kMaxCard * 4);
    const float *ds = series;
    uint4 *dw = reinterpret_cast<uint4 *>(words);
    cudaError_t e = cudaMemcpyAsync(d64, b64, (cardinality - 1) * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d32, b32, (cardinality - 1) * 4, cudaMemcpyHostToDevice, s);
    if (hs && e == cudaSuccess) {
        e = cudaMemcpyAsync(tmp + o, series, sbytes, cudaMemcpyHostToDevice, s);
        ds = reinterpret_cast<const float *>(tmp + o);
        o += align256(sbytes);
    }
    if (hw) dw = reinterpret_cast<uint4 *>(tmp + o);
    if (e == cudaSuccess) {
        launch_summarize(ds, n, len, segments, cardinality, d64, d32, dw, nullptr, nullptr, nullptr, s);
        e = cudaGetLastError();
    }
    if (hw && e == cudaSuccess) e = cudaMemcpyAsync(words, dw, wbytes, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(tmp);
    if (e != cudaSuccess) return fail(MESSI_ECUDA, std::string("messi_summarize: ") + cudaGetErrorString(e));
    return MESSI_OK;
}

messi_status messi_index_layout(const messi_index *ix, uint32_t *order, uint64_t *leaf_off, uint8_t *leaf_depth)
{
    if (!ix) return fail(MESSI_EINVAL, "messi_index_layout: null index");
    MESSI_CUDA(cudaDeviceSynchronize());
    if (order) MESSI_CUDA(cudaMemcpy(order, ix->ids, ix->N * 4, cudaMemcpyDeviceToHost));
    if (leaf_off) MESSI_CUDA(cudaMemcpy(leaf_off, ix->leaf_off, (ix->L + 1) * 8, cudaMemcpyDeviceToHost));
    if (leaf_depth) MESSI_CUDA(cudaMemcpy(leaf_depth, ix->leaf_depth, ix->L, cudaMemcpyDeviceToHost));
    return MESSI_OK;
}

}  // extern "C"
