// server.cu -- continuous-batching request loop over a resident index (no
// counterpart in the paper, whose queries run one after another).
//
// Requests (one query each, any k / distance / window) enter an arrival queue
// on submit.  Worker threads, one per CUDA stream, repeatedly form a batch:
// they admit queued requests in arrival order while the device memory charged
// to admitted-but-unfinished requests stays within the budget, group them by
// (distance, window), run the group through the batched forms (ED: the
// tensor-core screen or the lower-bound batch kernels; DTW: per-query kernel
// sequences overlapped on several streams) with k = the largest k in the group, and hand each
// request the first k of its row -- the k-NN answer is a prefix of the
// (k_max)-NN answer under the (distance, id) order, so a request gets the same
// result alone or in any mix.  A batch on one stream overlaps with the batch
// of another; a request that arrives while batches run is taken by the next
// free worker.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include <algorithm>

#include "messi_internal.cuh"

using namespace messi;
using Clock = std::chrono::steady_clock;

namespace {

struct Request {
    uint64_t ticket;
    std::vector<float> q;
    uint32_t k;
    messi_dist dist;
    uint32_t window;
    Clock::time_point t_submit;
    size_t cost;
};

struct Result {
    std::vector<int64_t> ids;
    std::vector<float> dists;
    double latency_ms;
    messi_status status;
};

struct Worker {
    std::thread th;
    cudaStream_t stream = nullptr;
    Workspace ws;
    float *h_q = nullptr;          // pinned staging: queries of a batch
    int64_t *h_ids = nullptr;      // pinned: results of a batch
    float *h_d = nullptr;
    float *d_q = nullptr;          // device copies
    int64_t *d_ids = nullptr;
    float *d_d = nullptr;
};

}  // namespace

struct messi_server {
    messi_index *ix = nullptr;
    messi_server_config cfg{};
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request> arrivals;
    std::unordered_map<uint64_t, Result> done;
    size_t admitted_cost = 0;
    uint64_t next_ticket = 1;
    bool stop = false;
    bool paused = false;
    std::vector<Worker *> workers;
    // statistics
    uint64_t submitted = 0, completed = 0, rejected = 0, batches = 0, inflight = 0, inflight_peak = 0,
             budget_waits = 0;
    std::vector<double> latencies;
};

namespace {

size_t request_cost(const messi_index *ix, uint32_t k)
{
    // query row, result row and the per-query slot of the batch workspace
    // (table, state, k-array, near-tie log, seed buffer)
    return (size_t)ix->len * 4 + (size_t)k * 12 + kMaxSegments * kMaxCard * 4 + kMaxK * 8 + kBatchLogCap * 8 +
           kSeedMax * 8 + 3 * (size_t)ix->len * 4 + 256;
}

// The queued request a worker would open its batch with: the oldest of the
// worker's preferred distance (worker 0 prefers ED, the others DTW, so ED
// batches never queue behind DTW batches), else the oldest.  Caller holds mu.
std::deque<Request>::iterator first_request(messi_server *srv, Worker *w)
{
    const messi_dist pref = (w == srv->workers[0] || srv->workers.size() == 1) ? MESSI_ED : MESSI_DTW;
    for (auto it = srv->arrivals.begin(); it != srv->arrivals.end(); ++it)
        if (it->dist == pref) return it;
    return srv->arrivals.begin();
}

// Whether a worker may open a batch now: requests are queued, admission is not
// held, and the first request fits the memory budget next to the requests in
// flight (a request larger than the budget is admitted when nothing else is
// in flight, so it cannot wait forever).  Caller holds mu.
bool can_admit(messi_server *srv, Worker *w)
{
    if (srv->arrivals.empty() || srv->paused) return false;
    const size_t c = first_request(srv, w)->cost;
    return srv->admitted_cost == 0 || srv->admitted_cost + c <= srv->cfg.mem_budget;
}

void worker_loop(messi_server *srv, Worker *w)
{
    messi_index *ix = srv->ix;
    cudaSetDevice(ix->device);
    const unsigned len = (unsigned)ix->len;
    const unsigned maxB = srv->cfg.max_batch;
    std::vector<Request> batch;
    for (;;) {
        batch.clear();
        {
            std::unique_lock<std::mutex> lk(srv->mu);
            bool counted = false;
            srv->cv_work.wait(lk, [&] {
                if (srv->stop && (srv->arrivals.empty() || srv->paused)) return true;
                if (can_admit(srv, w)) return true;
                // requests wait for memory held by batches in flight
                if (!counted && !srv->arrivals.empty() && !srv->paused) {
                    ++srv->budget_waits;
                    counted = true;
                }
                return false;
            });
            if (srv->stop && (srv->arrivals.empty() || srv->paused)) return;
            // admit in arrival order: same (distance, window) as the first
            // request, while the memory budget allows
            auto first = first_request(srv, w);
            const messi_dist d0 = first->dist;
            const uint32_t w0 = first->window;
            for (auto it = srv->arrivals.begin(); it != srv->arrivals.end() && batch.size() < maxB;) {
                if (it->dist == d0 && (d0 == MESSI_ED || it->window == w0)) {
                    if (srv->admitted_cost > 0 && srv->admitted_cost + it->cost > srv->cfg.mem_budget) break;
                    srv->admitted_cost += it->cost;
                    batch.push_back(std::move(*it));
                    it = srv->arrivals.erase(it);
                } else {
                    ++it;
                }
            }
            srv->inflight += batch.size();
            if (srv->inflight > srv->inflight_peak) srv->inflight_peak = srv->inflight;
            ++srv->batches;
        }
        if (batch.empty()) continue;
        const unsigned B = (unsigned)batch.size();
        uint32_t kmax = 1;
        for (auto &r : batch) kmax = std::max(kmax, r.k);
        for (unsigned b = 0; b < B; ++b) std::copy(batch[b].q.begin(), batch[b].q.end(), w->h_q + (size_t)b * len);
        messi_status st = MESSI_OK;
        cudaError_t e = cudaMemcpyAsync(w->d_q, w->h_q, (size_t)B * len * 4, cudaMemcpyHostToDevice, w->stream);
        if (e != cudaSuccess) st = MESSI_ECUDA;
        if (st == MESSI_OK) {
            const messi_dist d = batch[0].dist;
            st = run_batched(ix, &w->ws, w->d_q, B, kmax, d, d == MESSI_DTW ? batch[0].window : 0u, B, w->d_ids,
                             w->d_d, w->stream);
        }
        if (st == MESSI_OK) {
            e = cudaMemcpyAsync(w->h_ids, w->d_ids, (size_t)B * kmax * 8, cudaMemcpyDeviceToHost, w->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(w->h_d, w->d_d, (size_t)B * kmax * 4, cudaMemcpyDeviceToHost, w->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(w->stream);
            if (e != cudaSuccess) st = MESSI_ECUDA;
        }
        const Clock::time_point now = Clock::now();
        {
            std::lock_guard<std::mutex> lk(srv->mu);
            for (unsigned b = 0; b < B; ++b) {
                Request &r = batch[b];
                Result res;
                res.status = st;
                res.ids.assign(w->h_ids + (size_t)b * kmax, w->h_ids + (size_t)b * kmax + r.k);
                res.dists.assign(w->h_d + (size_t)b * kmax, w->h_d + (size_t)b * kmax + r.k);
                res.latency_ms = std::chrono::duration<double, std::milli>(now - r.t_submit).count();
                srv->latencies.push_back(res.latency_ms);
                srv->done.emplace(r.ticket, std::move(res));
                srv->admitted_cost -= r.cost;
            }
            srv->inflight -= B;
            srv->completed += B;
        }
        srv->cv_done.notify_all();
        srv->cv_work.notify_all();
    }
}

void free_worker(Worker *w)
{
    if (w->h_q) cudaFreeHost(w->h_q);
    if (w->h_ids) cudaFreeHost(w->h_ids);
    if (w->h_d) cudaFreeHost(w->h_d);
    if (w->d_q) cudaFree(w->d_q);
    if (w->d_ids) cudaFree(w->d_ids);
    if (w->d_d) cudaFree(w->d_d);
    free_workspace(w->ws);
    if (w->stream) cudaStreamDestroy(w->stream);
    delete w;
}

}  // namespace

extern "C" {

messi_status messi_server_create(messi_index *ix, const messi_server_config *cfg, messi_server **out)
{
    if (!ix || !out) return fail(MESSI_EINVAL, "messi_server_create: null argument");
    *out = nullptr;
    messi_server *srv = new messi_server();
    srv->ix = ix;
    if (cfg) srv->cfg = *cfg;
    if (!srv->cfg.max_batch) srv->cfg.max_batch = 1024;
    if (!srv->cfg.max_k) srv->cfg.max_k = 64;
    if (!srv->cfg.streams) srv->cfg.streams = 2;
    if (srv->cfg.max_k > (uint32_t)kMaxK || srv->cfg.max_batch > 65535 || srv->cfg.streams > 8) {
        delete srv;
        return fail(MESSI_EINVAL, "messi_server_create: max_k <= 1024, max_batch <= 65535, streams <= 8");
    }
    if (!srv->cfg.mem_budget)
        srv->cfg.mem_budget = (uint64_t)srv->cfg.streams * srv->cfg.max_batch * request_cost(ix, srv->cfg.max_k);
    cudaSetDevice(ix->device);
    // build the screening copy now, before several workers could race to do it
    if (ix->batch_mode == 1) {
        messi_status st = ensure_screen_copy(ix, nullptr);
        if (st == MESSI_OK && !cuda_ok(cudaStreamSynchronize(nullptr), "messi_server_create: screening copy"))
            st = MESSI_ECUDA;
        if (st != MESSI_OK) {
            delete srv;
            return st;
        }
    }
    const unsigned maxB = srv->cfg.max_batch, len = (unsigned)ix->len, kx = srv->cfg.max_k;
    // worker 0 takes the ED batches: its stream gets the highest priority, so
    // that the block scheduler starts its (short, whole-SM) screen launches
    // ahead of the long DTW work queued on the other workers' streams
    int prio_low = 0, prio_high = 0;
    if (cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high) != cudaSuccess) {
        cudaGetLastError();
        prio_low = prio_high = 0;
    }
    for (uint32_t i = 0; i < srv->cfg.streams; ++i) {
        Worker *w = new Worker();
        const int prio = (i == 0 && srv->cfg.streams > 1) ? prio_high : prio_low;
        bool ok = cudaStreamCreateWithPriority(&w->stream, cudaStreamNonBlocking, prio) == cudaSuccess &&
                  cudaMallocHost(&w->h_q, (size_t)maxB * len * 4) == cudaSuccess &&
                  cudaMallocHost(&w->h_ids, (size_t)maxB * kx * 8) == cudaSuccess &&
                  cudaMallocHost(&w->h_d, (size_t)maxB * kx * 4) == cudaSuccess &&
                  cudaMalloc(&w->d_q, (size_t)maxB * len * 4) == cudaSuccess &&
                  cudaMalloc(&w->d_ids, (size_t)maxB * kx * 8) == cudaSuccess &&
                  cudaMalloc(&w->d_d, (size_t)maxB * kx * 4) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            free_worker(w);
            messi_server_destroy(srv);
            return fail(MESSI_ENOMEM, "messi_server_create: cannot allocate worker buffers");
        }
        srv->workers.push_back(w);
    }
    for (Worker *w : srv->workers) w->th = std::thread(worker_loop, srv, w);
    *out = srv;
    return MESSI_OK;
}

messi_status messi_server_submit(messi_server *srv, const float *query, uint32_t k, messi_dist dist, uint32_t window,
                                 uint64_t *ticket)
{
    if (!srv || !query || !ticket) return fail(MESSI_EINVAL, "messi_server_submit: null argument");
    messi_index *ix = srv->ix;
    if (k == 0 || k > srv->cfg.max_k || k > ix->N) return fail(MESSI_EINVAL, "messi_server_submit: k out of range");
    if (dist != MESSI_ED && dist != MESSI_DTW) return fail(MESSI_EINVAL, "messi_server_submit: unknown distance");
    if (dist == MESSI_DTW && window >= (uint32_t)ix->len) return fail(MESSI_EINVAL, "messi_server_submit: window must be < len");
    Request r;
    r.q.assign(query, query + ix->len);
    r.k = k;
    r.dist = dist;
    r.window = dist == MESSI_DTW ? window : 0;
    r.t_submit = Clock::now();
    r.cost = request_cost(ix, k);
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        if (srv->cfg.max_queued && srv->arrivals.size() >= srv->cfg.max_queued) {
            ++srv->rejected;
            return fail(MESSI_EBUSY, "messi_server_submit: arrival queue full");
        }
        r.ticket = srv->next_ticket++;
        *ticket = r.ticket;
        srv->arrivals.push_back(std::move(r));
        ++srv->submitted;
    }
    // every worker re-checks: which one may admit depends on its preferred
    // distance and on the memory budget
    srv->cv_work.notify_all();
    return MESSI_OK;
}

messi_status messi_server_poll(messi_server *srv, uint64_t ticket, int64_t *ids, float *dists, double *latency_ms,
                               uint64_t wait_us)
{
    if (!srv || !ids || !dists) return fail(MESSI_EINVAL, "messi_server_poll: null argument");
    std::unique_lock<std::mutex> lk(srv->mu);
    auto ready = [&] { return srv->done.count(ticket) != 0; };
    if (!ready() && wait_us) srv->cv_done.wait_for(lk, std::chrono::microseconds(wait_us), ready);
    auto it = srv->done.find(ticket);
    if (it == srv->done.end()) {
        if (ticket == 0 || ticket >= srv->next_ticket) return fail(MESSI_EINVAL, "messi_server_poll: unknown ticket");
        return MESSI_EBUSY;
    }
    Result res = std::move(it->second);
    srv->done.erase(it);
    lk.unlock();
    std::copy(res.ids.begin(), res.ids.end(), ids);
    std::copy(res.dists.begin(), res.dists.end(), dists);
    if (latency_ms) *latency_ms = res.latency_ms;
    if (res.status != MESSI_OK) return fail(res.status, "messi_server_poll: the batch of this request failed");
    return MESSI_OK;
}

messi_status messi_server_get_stats(messi_server *srv, messi_server_stats *out)
{
    if (!srv || !out) return fail(MESSI_EINVAL, "messi_server_get_stats: null argument");
    std::lock_guard<std::mutex> lk(srv->mu);
    *out = messi_server_stats{};
    out->submitted = srv->submitted;
    out->completed = srv->completed;
    out->rejected = srv->rejected;
    out->batches = srv->batches;
    out->inflight_peak = srv->inflight_peak;
    out->budget_waits = srv->budget_waits;
    std::vector<double> lat = srv->latencies;
    if (!lat.empty()) {
        std::sort(lat.begin(), lat.end());
        auto pct = [&](double p) { return lat[std::min(lat.size() - 1, (size_t)(p * (lat.size() - 1) + 0.5))]; };
        out->p50_ms = pct(0.50);
        out->p99_ms = pct(0.99);
        double s = 0;
        for (double v : lat) s += v;
        out->mean_ms = s / lat.size();
    }
    return MESSI_OK;
}

messi_status messi_server_pause(messi_server *srv, int paused)
{
    if (!srv) return fail(MESSI_EINVAL, "messi_server_pause: null server");
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->paused = paused != 0;
    }
    srv->cv_work.notify_all();
    return MESSI_OK;
}

void messi_server_destroy(messi_server *srv)
{
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
        srv->paused = false;   // the queued requests are answered before the workers stop
    }
    srv->cv_work.notify_all();
    for (Worker *w : srv->workers)
        if (w->th.joinable()) w->th.join();
    for (Worker *w : srv->workers) free_worker(w);
    delete srv;
}

}  // extern "C"
