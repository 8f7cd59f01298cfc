// order.cu -- the survivors of a filter step, ordered by lower bound.
//
// MESSI (Sec. 3, query answering with ED and with DTW) keeps the leaves that
// survive pruning in minimum priority queues keyed by their lower bound and
// examines them in increasing bound order; a worker gives a queue up as soon
// as the bound at its head exceeds the best-so-far, since nothing behind it
// can qualify.  The GPU counterpart: the survivors are counting-sorted into
// kOrderBuckets buckets keyed by the top bits of their FP32 bound (8 exponent
// and 4 mantissa bits, so one bucket spans at most a factor 1 + 1/16), and
// refinement walks the sorted list from the front.  Every thread's sequence
// of candidates then has non-decreasing buckets, and a thread stops at the
// first candidate whose bucket floor exceeds the best-so-far threshold.
//
// Three launches per query: per-bucket counts, an exclusive scan into write
// cursors (which also clears the counts for the next query), and a scatter in
// which each block reserves its ranges once per bucket and fills them through
// shared-memory cursors.  Candidates inside one bucket keep no particular
// order; exactness does not depend on the order at all, only the amount of
// refinement work does.
#include "device_common.cuh"

namespace messi {
namespace {

constexpr int kOrderThreads = 256;

// Visit the survivors of SRC: 0 = scan regions (surv_pos / surv_lb, region g
// at g * region_words holding region_count[g] entries), 1 = compact list
// (surv2 / surv2_lb, surv2_count entries).  A warp takes 32 entries at a time
// (for regions: 32-entry chunks numbered across all regions, so every block
// has work however the survivors are spread), and all 32 lanes step
// together (warp collectives see the whole warp); a lane past the end gets
// valid = false.  A block visits the same entries in the same order every
// time it is called within one launch.  `prefix` / `counts` hold the chunk
// prefix of the regions (chunk_prefix) for SRC 0.
template <int SRC, typename F>
__device__ __forceinline__ void for_each_survivor(const QuerySlot &slot, unsigned nchunks, const unsigned *prefix,
                                                  const unsigned *counts, F f)
{
    const QueryState *st = slot.st;
    const unsigned lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    if (SRC == 0) {
        const unsigned G = st->scan_grid;
        const unsigned long long RW = st->region_words;
        for (unsigned ch = blockIdx.x * wpb + wib; ch < nchunks; ch += gridDim.x * wpb) {
            const unsigned rg = region_of(ch, prefix, G);
            const unsigned within = (ch - prefix[rg]) * 32 + lane;
            const bool valid = within < counts[rg];
            const unsigned long long i = rg * RW + within;
            f(valid, valid ? slot.surv_pos[i] : 0u, valid ? slot.surv_lb[i] : 0.f);
        }
    } else {
        const unsigned n = st->surv2_count;
        for (unsigned i0 = blockIdx.x * blockDim.x + wib * 32; i0 < n; i0 += gridDim.x * blockDim.x) {
            const unsigned i = i0 + lane;
            const bool valid = i < n;
            f(valid, valid ? slot.surv2[i] : 0u, valid ? slot.surv2_lb[i] : 0.f);
        }
    }
}

// chunk prefix of the scan regions (SRC 0); also the block barrier that
// publishes the zeroed histogram
template <int SRC>
__device__ __forceinline__ unsigned survivor_chunks(const QuerySlot &slot, unsigned *prefix, unsigned *counts)
{
    if (SRC == 0) return chunk_prefix(slot, slot.st->scan_grid, prefix, counts);
    __syncthreads();
    return 0u;
}

// Shared-memory counter bump aggregated over the lanes of a warp that hit the
// same bucket: one atomic per distinct bucket, each lane gets its own slot.
// Returns the lane's slot (the counter's old value plus its rank), or 0 for
// a lane that takes part with take = false.
__device__ __forceinline__ unsigned bump_bucket(unsigned *h, bool take, unsigned b)
{
    const unsigned lane = threadIdx.x & 31;
    const unsigned want = __ballot_sync(0xffffffffu, take);
    const unsigned key = take ? b : 0xffffffffu;
    const unsigned same = __match_any_sync(0xffffffffu, key) & want;
    unsigned base = 0;
    const int leader = same ? __ffs(same) - 1 : -1;
    if (take && (int)lane == leader) base = atomicAdd(&h[b], (unsigned)__popc(same));
    base = __shfl_sync(0xffffffffu, base, leader < 0 ? (int)lane : leader);
    return take ? base + __popc(same & ((1u << lane) - 1u)) : 0u;
}

template <int SRC>
__global__ void __launch_bounds__(kOrderThreads)
k_order_count(QueryParams qp, QuerySlot slot)
{
    __shared__ unsigned h[kOrderBuckets];
    __shared__ unsigned prefix[kMaxScanGrid + 1], counts[kMaxScanGrid];
    const QueryState *st = slot.st;
    if (ld_volatile_u32(&st->invalid)) return;
    for (int b = threadIdx.x; b < kOrderBuckets; b += blockDim.x) h[b] = 0u;
    const unsigned nch = survivor_chunks<SRC>(slot, prefix, counts);
    const float thr = prune_threshold(st->thr, qp.F);
    for_each_survivor<SRC>(slot, nch, prefix, counts, [&](bool valid, unsigned, float lb) {
        const bool take = valid && lb <= thr;
        bump_bucket(h, take, take ? order_bucket(lb) : 0u);
    });
    __syncthreads();
    for (int b = threadIdx.x; b < kOrderBuckets; b += blockDim.x)
        if (h[b]) atomicAdd(&slot.bucket[b], h[b]);
}

// one block of 1024 threads, 4 buckets each
__global__ void __launch_bounds__(1024)
k_order_scan(QuerySlot slot)
{
    static_assert(kOrderBuckets == 4 * 1024, "scan layout");
    __shared__ unsigned part[32];
    unsigned *count = slot.bucket, *cursor = slot.bucket + kOrderBuckets;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    unsigned c[4], sum = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        c[j] = count[4 * t + j];
        sum += c[j];
    }
    unsigned inc = sum;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc += y;
    }
    if (lane == 31) part[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        unsigned v = part[lane];
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, v, off);
            if (lane >= off) v += y;
        }
        part[lane] = v;
    }
    __syncthreads();
    unsigned run = (warp ? part[warp - 1] : 0u) + inc - sum;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        cursor[4 * t + j] = run;
        count[4 * t + j] = 0u;
        run += c[j];
    }
    if (t == 1023) slot.st->ord_count = run;
}

template <int SRC>
__global__ void __launch_bounds__(kOrderThreads)
k_order_scatter(QueryParams qp, QuerySlot slot, unsigned *__restrict__ dst_pos, float *__restrict__ dst_lb)
{
    __shared__ unsigned h[kOrderBuckets];
    __shared__ unsigned prefix[kMaxScanGrid + 1], counts[kMaxScanGrid];
    const QueryState *st = slot.st;
    if (ld_volatile_u32(&st->invalid)) return;
    unsigned *cursor = slot.bucket + kOrderBuckets;
    for (int b = threadIdx.x; b < kOrderBuckets; b += blockDim.x) h[b] = 0u;
    const unsigned nch = survivor_chunks<SRC>(slot, prefix, counts);
    const float thr = prune_threshold(st->thr, qp.F);
    for_each_survivor<SRC>(slot, nch, prefix, counts, [&](bool valid, unsigned, float lb) {
        const bool take = valid && lb <= thr;
        bump_bucket(h, take, take ? order_bucket(lb) : 0u);
    });
    __syncthreads();
    for (int b = threadIdx.x; b < kOrderBuckets; b += blockDim.x)
        if (h[b]) h[b] = atomicAdd(&cursor[b], h[b]);
    __syncthreads();
    for_each_survivor<SRC>(slot, nch, prefix, counts, [&](bool valid, unsigned pos, float lb) {
        const bool take = valid && lb <= thr;
        const unsigned o = bump_bucket(h, take, take ? order_bucket(lb) : 0u);
        if (take) {
            dst_pos[o] = pos;
            dst_lb[o] = lb;
        }
    });
}

}  // namespace

void launch_order(const QueryParams &qp, const QuerySlot &slot, int src, unsigned *dst_pos, float *dst_lb,
                  cudaStream_t s)
{
    const unsigned grid = num_sms() * 4;
    if (src == 0) k_order_count<0><<<grid, kOrderThreads, 0, s>>>(qp, slot);
    else k_order_count<1><<<grid, kOrderThreads, 0, s>>>(qp, slot);
    k_order_scan<<<1, 1024, 0, s>>>(slot);
    if (src == 0) k_order_scatter<0><<<grid, kOrderThreads, 0, s>>>(qp, slot, dst_pos, dst_lb);
    else k_order_scatter<1><<<grid, kOrderThreads, 0, s>>>(qp, slot, dst_pos, dst_lb);
}

}  // namespace messi
