// query.cu -- exact k-NN query kernels (Sec. 3.3 for ED, Sec. 3.4 for DTW).
//
// Per query, in stream order:
//   k_prep      FP64 PAA of the query (ED) or of its LB_Keogh envelope (DTW),
//               the table T[s][v] = m * d_s(v)^2 rounded down, the query key
//               and the seed range (the query's own leaf; approxSearch,
//               Sec. 3.1).
//   k_seed_dist distances to every series of the seed range.
//   k_seed_sel  the k best of them become the initial best-so-far.
//   k_leaf_prune bounds every leaf from its symbol box and marks the scan
//               tiles of the leaves it cannot prune (k_live_tiles lists them).
//   k_lb_scan   streams the iSAX words of the live tiles through TMA bulk
//               copies into shared memory, sums their table entries and
//               compacts the survivors (LB^2 <= widened k-th best) warp by warp.
//   k_order_*   counting-sorts the survivors by lower-bound bucket (order.cu).
//   k_refine_ed warp per survivor, in bound order: re-checks its bound against
//               the live best-so-far, then ED with early abandoning
//               (Algorithm 9).
//   k_lbk/k_dtw_thread  DTW: LB_Keogh, then LB_Improved, on the raw survivor, bound
//               order, then banded DTW one candidate per thread (Algorithm 10).
//   k_finalize  resolves near-ties in FP64 and writes ids / distances.
//
// Exactness.  Lower bounds are summed with rounding toward -inf from table
// entries rounded toward -inf, so they never exceed the exact bound.  Real
// distances are FP32 with relative error at most gamma; a candidate is
// discarded only when it is certainly worse than the current k-th best: its
// bound or distance exceeds the k-th best's FP32 distance times
// F >= (1 + gamma)^2.  Every candidate within that band is logged, and at the
// end any ambiguity (more than k candidates in the band, or two of the k
// within the band of each other) is settled by recomputing those candidates
// in FP64 with the same operation order as the FP64 reference; ties of equal
// distance go to the lowest original id because the packed 64-bit
// (distance bits << 32 | id) compares that way.
#include <algorithm>

#include "device_common.cuh"

namespace messi {
namespace {

constexpr int kPrepThreads = 256;
constexpr int kScanThreads = 256;
constexpr int kScanWpt = 4;
constexpr int kScanTileWords = kScanThreads * kScanWpt;   // 1024 words, 16 KB
static_assert(kScanTileWords == kScanTileWordsHost, "scan tile size shared with the workspace layout");
constexpr int kScanStages = 4;
constexpr int kScanCtasPerSm = 3;
constexpr int kScanSmem = kScanStages * kScanTileWords * 16;   // 64 KB ring (+ 8 KB static code table)
constexpr int kFinThreads = 1024;

// ------------------------------------------------------------------ prep
__device__ __forceinline__ double region_lo(int v, const double *beta)
{
    return v == 0 ? -__longlong_as_double(0x7ff0000000000000ll) : beta[v - 1];
}
__device__ __forceinline__ double region_hi(int v, int card, const double *beta)
{
    return v == card - 1 ? __longlong_as_double(0x7ff0000000000000ll) : beta[v];
}

// Distance from a value to a region, rounded down and shrunk by a slack that
// covers the FP64 rounding of the PAA values the regions were chosen with.
__device__ __forceinline__ double gap_rd(double edge, double p)   // edge - p, edge > p
{
    double d = __dsub_rd(edge, p);
    d = __dsub_rd(d, 9.094947017729282e-13 * (fabs(edge) + fabs(p) + 1.0));   // 2^-40 (...)
    return d > 0.0 ? d : 0.0;
}

// Table entry (s, v): m * d^2, d the distance from the query's segment-s
// value (ED: PAA; DTW: PAA of U below the region, of L above it) to region v,
// every step rounded toward -inf; 0 beyond the index's segments and symbols.
__device__ __forceinline__ float table_entry(int s, int v, int w, int card, int m, int dist, double p, double pu,
                                             double pl, const double *sbeta)
{
    if (s >= w || v >= card) return 0.f;
    const double lo = region_lo(v, sbeta), hi = region_hi(v, card, sbeta);
    double d = 0.0;
    if (dist == 0) {
        if (p < lo) d = gap_rd(lo, p);
        else if (p > hi) d = gap_rd(p, hi);
    } else {
        if (pu < lo) d = gap_rd(lo, pu);            // ABOVE
        else if (pl > hi) d = gap_rd(pl, hi);       // BELOW
    }
    return __double2float_rd(__dmul_rd(__dmul_rd(d, d), (double)m));
}

// 1/m for m a power of two, built from its exponent bits.  A sum of at most
// 4096 floats divided by such an m neither overflows nor leaves the normal
// range of a double, so multiplying by 1/m gives the quotient exactly: the
// same bits as the correctly rounded division.
__device__ __forceinline__ double pow2_recip(int m)
{
    const int e = __ffs(m) - 1;   // m = 2^e
    return __longlong_as_double((long long)(1023 - e) << 52);
}

// k <= q in the order of the 128-bit interleaved keys (x most significant)
__device__ __forceinline__ bool key_le(const uint4 k, const uint4 q)
{
    return (k.x != q.x) ? k.x < q.x : (k.y != q.y) ? k.y < q.y : (k.z != q.z) ? k.z < q.z : k.w <= q.w;
}

// with_table = false leaves the table to k_prep's other blocks (one row each)
__device__ __forceinline__ void prep_body(const IndexView &iv, const QueryParams &qp, const QuerySlot &slot,
                                          const float *__restrict__ query, bool with_table = true)
{
    __shared__ double paa[kMaxSegments], paaU[kMaxSegments], paaL[kMaxSegments];
    __shared__ int sym[kMaxSegments];
    __shared__ int bad;
    __shared__ double sbeta[kMaxCard];
    QueryState *st = slot.st;
    const int tid = threadIdx.x;
    const int len = iv.len, w = iv.w, m = iv.m, card = iv.card;
    if (tid == 0) {
        bad = 0;
        st->thr = kEmpty;
        st->lock = 0u;
        st->kcount = 0u;
        st->surv_count = 0u;
        st->surv2_count = 0u;
        st->log_count = 0u;
        st->seed_count = 0u;
        st->invalid = 0u;
        st->live_tiles = 0u;
        st->c = QueryCounters{};
    }
    for (int i = tid; i < kMaxCard; i += blockDim.x) sbeta[i] = i < card - 1 ? iv.beta64[i] : 0.0;
    __syncthreads();
    for (int i = tid; i < len; i += blockDim.x) {
        const float v = query[i];
        if (!isfinite(v)) bad = 1;
        slot.q[i] = v;
    }
    __syncthreads();
    if (bad) {
        if (tid == 0) {
            st->invalid = 1u;
            atomicOr(iv.status, kStInvalidQuery);
        }
        return;
    }
    if (qp.dist == 1) {   // LB_Keogh envelope, window clipped at the ends
        for (int i = tid; i < len; i += blockDim.x) {
            const int a = max(0, i - qp.r), b = min(len - 1, i + qp.r);
            float hi = slot.q[a], lo = slot.q[a];
            for (int j = a + 1; j <= b; ++j) {
                const float v = slot.q[j];
                hi = fmaxf(hi, v);
                lo = fminf(lo, v);
            }
            slot.U[i] = hi;
            slot.L[i] = lo;
        }
    }
    __syncthreads();
    // FP64 segment means, each a sequential sum in index order: one warp per
    // segment reads 32 points at a time and adds them in turn from shuffles
    // (every lane carries the same sum)
    const int lane = tid & 31, wib = tid >> 5;
    for (int sg = wib; sg < w; sg += (int)(blockDim.x >> 5)) {
        double sm = 0.0, su = 0.0, sl = 0.0;
        for (int base = sg * m; base < (sg + 1) * m; base += 32) {
            const int t = base + lane, cnt = min(32, (sg + 1) * m - base);
            const float v = lane < cnt ? slot.q[t] : 0.f;
            const float vu = (qp.dist == 1 && lane < cnt) ? slot.U[t] : 0.f;
            const float vl = (qp.dist == 1 && lane < cnt) ? slot.L[t] : 0.f;
            for (int j = 0; j < cnt; ++j) {
                sm = __dadd_rn(sm, (double)__shfl_sync(0xffffffffu, v, j));
                if (qp.dist == 1) {
                    su = __dadd_rn(su, (double)__shfl_sync(0xffffffffu, vu, j));
                    sl = __dadd_rn(sl, (double)__shfl_sync(0xffffffffu, vl, j));
                }
            }
        }
        if (lane == 0) {
            const double inv_m = pow2_recip(m);
            paa[sg] = __dmul_rn(sm, inv_m);
            paaU[sg] = __dmul_rn(su, inv_m);
            paaL[sg] = __dmul_rn(sl, inv_m);
            int lo = 0, hi = card - 1;
            while (lo < hi) {
                int mid = (lo + hi) >> 1;
                if (sbeta[mid] <= paa[sg]) lo = mid + 1; else hi = mid;
            }
            sym[sg] = lo;
        }
    }
    __syncthreads();
    // table: T[s][v] = m * d^2, every step rounded toward -inf
    if (with_table)
        for (int e = tid; e < kMaxSegments * kMaxCard; e += blockDim.x) {
            const int s = e / kMaxCard, v = e % kMaxCard;
            slot.lut[e] = s < w ? table_entry(s, v, w, card, m, qp.dist, paa[s], paaU[s], paaL[s], sbeta) : 0.f;
        }
    __shared__ uint4 qkey;
    if (wib == 0) {
        // interleaved key of the query word: for each bit plane j, the j-th
        // most significant bit of every segment's symbol, segment 0 first
        const int sy = lane < w ? sym[lane] : 0;
        unsigned long long khi = 0ull, klo = 0ull;
        for (int j = 0; j < iv.bits; ++j) {
            const unsigned mask = __ballot_sync(0xffffffffu, lane < w && ((sy >> (iv.bits - 1 - j)) & 1));
            const unsigned field = __brev(mask) >> (32 - w);
            khi = (khi << w) | (klo >> (64 - w));
            klo = (klo << w) | field;
        }
        const int used = w * iv.bits;
        if (used < 128) {
            const int sh = 128 - used;
            if (sh >= 64) { khi = klo << (sh - 64); klo = 0ull; }
            else { khi = (khi << sh) | (klo >> (64 - sh)); klo <<= sh; }
        }
        if (lane == 0) {
            const uint4 qk = make_uint4((unsigned)(khi >> 32), (unsigned)khi, (unsigned)(klo >> 32), (unsigned)klo);
            qkey = qk;
            st->qkey = qk;
            // per segment a symbol where the table is 0: the query's own symbol
            // (for DTW it lies between the envelope's symbols, where the table is 0)
            unsigned qs[4] = {0u, 0u, 0u, 0u};
#pragma unroll
            for (int sg = 0; sg < kMaxSegments; ++sg)
                if (sg < w) qs[sg >> 2] |= (unsigned)sym[sg] << (8 * (sg & 3));
            st->qsym = make_uint4(qs[0], qs[1], qs[2], qs[3]);
        }
    }
    __syncthreads();
    // seed leaf: the last leaf whose first key is <= the query key.  The count
    // of such leaves (the keys ascend) lies in [lo, hi]; each round every
    // thread tests one of blockDim.x evenly spaced pivots and the count of
    // true answers narrows the range about blockDim.x + 1 times.
    const uint4 qk = qkey;
    unsigned long long lo = 0, hi = iv.L;
    const unsigned nb = blockDim.x;
    while (hi - lo > nb) {
        const unsigned long long step = (hi - lo + nb) / (nb + 1);
        const unsigned long long piv = lo + (tid + 1) * step - 1;
        const int c = __syncthreads_count(piv < hi && key_le(iv.leaf_key[piv], qk));
        const unsigned long long nlo = lo + (unsigned long long)c * step;
        if ((unsigned)c < nb) hi = min(hi, lo + (unsigned long long)(c + 1) * step - 1);
        lo = nlo;
    }
    lo += (unsigned long long)__syncthreads_count(lo + tid < hi && key_le(iv.leaf_key[lo + tid], qk));
    if (tid == 0) {
        const unsigned long long leaf = lo > 0 ? lo - 1 : 0;
        unsigned long long a = iv.leaf_off[leaf], b = iv.leaf_off[leaf + 1];
        if (b - a > (unsigned long long)kSeedMax) b = a + kSeedMax;
        // fewer than k series in the leaf: widen to neighbouring positions
        const unsigned long long want = (unsigned long long)qp.k;
        while (b - a < want) {
            if (a > 0) --a;
            if (b - a < want && b < iv.N) ++b;
        }
        st->seed_lo = (unsigned)a;
        st->seed_hi = (unsigned)b;
    }
}

// One row of the table (segment s, 256 symbols, one per thread): the row's
// FP64 work spread over its own block, since FP64 throughput per SM is low.
// The segment's PAA (ED) or PAAs of the envelope (DTW) are recomputed here in
// the same order as prep_body's.
__device__ __forceinline__ void prep_table_row(const IndexView &iv, const QueryParams &qp, const QuerySlot &slot,
                                               const float *__restrict__ query, int s)
{
    __shared__ double sbeta[kMaxCard];
    __shared__ double ps, psu, psl;
    const int tid = threadIdx.x;
    const int len = iv.len, w = iv.w, m = iv.m, card = iv.card;
    if (s >= w) {
        for (int v = tid; v < kMaxCard; v += blockDim.x) slot.lut[s * kMaxCard + v] = 0.f;
        return;
    }
    __shared__ float up_pts[kMaxLen], dn_pts[kMaxLen];
    for (int i = tid; i < kMaxCard; i += blockDim.x) sbeta[i] = i < card - 1 ? iv.beta64[i] : 0.0;
    if (qp.dist == 1)   // the LB_Keogh envelope on the segment, window clipped at the ends
        for (int i = tid; i < m; i += blockDim.x) {
            const int t = s * m + i, lo = max(0, t - qp.r), hi = min(len - 1, t + qp.r);
            float up = query[lo], dn = query[lo];
            for (int j = lo + 1; j <= hi; ++j) {
                up = fmaxf(up, query[j]);
                dn = fminf(dn, query[j]);
            }
            up_pts[i] = up;
            dn_pts[i] = dn;
        }
    __syncthreads();
    if (tid < 32) {   // sequential FP64 sums in prep_body's order, 32 points per load
        double a = 0.0, au = 0.0, al = 0.0;
        for (int base = 0; base < m; base += 32) {
            const int cnt = min(32, m - base);
            const float v = tid < cnt ? query[s * m + base + tid] : 0.f;
            const float vu = (qp.dist == 1 && tid < cnt) ? up_pts[base + tid] : 0.f;
            const float vl = (qp.dist == 1 && tid < cnt) ? dn_pts[base + tid] : 0.f;
            for (int j = 0; j < cnt; ++j) {
                a = __dadd_rn(a, (double)__shfl_sync(0xffffffffu, v, j));
                if (qp.dist == 1) {
                    au = __dadd_rn(au, (double)__shfl_sync(0xffffffffu, vu, j));
                    al = __dadd_rn(al, (double)__shfl_sync(0xffffffffu, vl, j));
                }
            }
        }
        if (tid == 0) {
            const double inv_m = pow2_recip(m);
            ps = __dmul_rn(a, inv_m);
            psu = __dmul_rn(au, inv_m);
            psl = __dmul_rn(al, inv_m);
        }
    }
    __syncthreads();
    for (int v = tid; v < kMaxCard; v += blockDim.x)
        slot.lut[s * kMaxCard + v] = table_entry(s, v, w, card, m, qp.dist, ps, psu, psl, sbeta);
}

// Block 0: query state, PAA, symbols, key and seed range; blocks 1..16: one
// row of the table each.
__global__ void __launch_bounds__(kPrepThreads)
k_prep(IndexView iv, QueryParams qp, QuerySlot slot, const float *__restrict__ query)
{
    if (blockIdx.x == 0) prep_body(iv, qp, slot, query, false);
    else prep_table_row(iv, qp, slot, query, (int)blockIdx.x - 1);
}

// one block per query of a batch
__global__ void __launch_bounds__(kPrepThreads)
k_prep_batch(IndexView iv, QueryParams qp, const QuerySlot *__restrict__ slots, const float *__restrict__ queries)
{
    prep_body(iv, qp, slots[blockIdx.x], queries + (size_t)blockIdx.x * iv.len);
}

// Graph-replayed form: the batch's query rows come from the argument table
// entry the cursor points at.
__global__ void __launch_bounds__(kPrepThreads)
k_prep_batch_args(IndexView iv, QueryParams qp, const QuerySlot *__restrict__ slots,
                  const BatchArgs *__restrict__ args, const unsigned *__restrict__ cursor)
{
    const BatchArgs a = args[*cursor];
    prep_body(iv, qp, slots[blockIdx.x], a.queries + (size_t)blockIdx.x * iv.len);
}

// ------------------------------------------------------------------ seed
template <int DIST>
__device__ __forceinline__ void seed_dist_body(const IndexView &iv, const QueryParams &qp, const QuerySlot &slot,
                                               unsigned part, unsigned nparts)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    QueryState *st = slot.st;
    if (ld_volatile_u32(&st->invalid)) return;
    const unsigned lo = st->seed_lo, hi = st->seed_hi;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    float *qs = reinterpret_cast<float *>(dsm);
    for (int i = threadIdx.x; i < iv.len; i += blockDim.x) qs[i] = slot.q[i];
    __syncthreads();
    float *diag = qs + iv.len + wib * 3 * iv.len;
    const unsigned nw = nparts * (blockDim.x >> 5);
    for (unsigned p = lo + part * (blockDim.x >> 5) + wib; p < hi; p += nw) {
        const float *x = iv.raw + (unsigned long long)p * iv.len;
        float d2 = DIST == 0 ? warp_ed2(qs, x, iv.len, f_inf())
                             : warp_dtw<float>(qs, x, iv.len, qp.r, diag, f_inf());
        if (lane == 0) slot.seedbuf[p - lo] = pack_cand(d2, iv.ids[p]);
        __syncwarp();
    }
}

template <int DIST>
__global__ void __launch_bounds__(256)
k_seed_dist(IndexView iv, QueryParams qp, QuerySlot slot)
{
    seed_dist_body<DIST>(iv, qp, slot, blockIdx.x, gridDim.x);
}

// blockIdx.y selects the query of the batch
template <int DIST>
__global__ void __launch_bounds__(256)
k_seed_dist_batch(IndexView iv, QueryParams qp, const QuerySlot *__restrict__ slots)
{
    seed_dist_body<DIST>(iv, qp, slots[blockIdx.y], blockIdx.x, gridDim.x);
}

// one block: sort the seed distances, keep the k best as the best-so-far
__device__ __forceinline__ void seed_select_body(const IndexView &iv, const QueryParams &qp, const QuerySlot &slot)
{
    __shared__ unsigned long long buf[kSeedMax];
    QueryState *st = slot.st;
    if (ld_volatile_u32(&st->invalid)) return;
    const unsigned cnt = st->seed_hi - st->seed_lo;
    if (qp.k == 1) {
        // the best seed alone: a block minimum instead of the sort (the
        // packed keys order by distance, then id, like the sorted list)
        __shared__ unsigned long long wmin[kFinThreads / 32];
        unsigned long long mn = kEmpty;
        for (unsigned i = threadIdx.x; i < cnt; i += blockDim.x) mn = min(mn, slot.seedbuf[i]);
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, off));
        if ((threadIdx.x & 31) == 0) wmin[threadIdx.x >> 5] = mn;
        __syncthreads();
        if (threadIdx.x < 32) {
            mn = threadIdx.x < (blockDim.x >> 5) ? wmin[threadIdx.x] : kEmpty;
#pragma unroll
            for (int off = 16; off >= 1; off >>= 1) mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, off));
            if (threadIdx.x == 0) wmin[0] = mn;
        }
        __syncthreads();
        const unsigned long long T = cnt >= 1 ? wmin[0] : kEmpty;
        if (threadIdx.x == 0 && cnt >= 1) slot.karr[0] = T;
        const float band = prune_threshold(T, qp.F);
        __shared__ unsigned nlog1;
        if (threadIdx.x == 0) nlog1 = 0;
        __syncthreads();
        for (unsigned i = threadIdx.x; i < cnt; i += blockDim.x) {
            const unsigned long long v = slot.seedbuf[i];
            if (cand_d2(v) <= band) {
                const unsigned li = atomicAdd(&nlog1, 1u);
                if (li < slot.log_cap) slot.log[li] = v;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            st->kcount = cnt >= 1 ? 1u : 0u;
            st->thr = T;
            st->log_count = nlog1;
            st->seed_count = cnt;
            st->c.seeded = cnt;
            st->c.bsf_updates = T != kEmpty ? 1ull : 0ull;
        }
        return;
    }
    unsigned npow = 1;
    while (npow < cnt) npow <<= 1;
    for (unsigned i = threadIdx.x; i < npow; i += blockDim.x) buf[i] = i < cnt ? slot.seedbuf[i] : kEmpty;
    __syncthreads();
    for (unsigned size = 2; size <= npow; size <<= 1)
        for (unsigned stride = size >> 1; stride > 0; stride >>= 1) {
            for (unsigned i = threadIdx.x; i < npow; i += blockDim.x) {
                const unsigned j = i ^ stride;
                if (j > i) {
                    const bool up = (i & size) == 0;
                    const unsigned long long a = buf[i], b = buf[j];
                    if ((a > b) == up) { buf[i] = b; buf[j] = a; }
                }
            }
            __syncthreads();
        }
    const unsigned k = (unsigned)qp.k;
    const unsigned kept = cnt < k ? cnt : k;
    for (unsigned i = threadIdx.x; i < kept; i += blockDim.x) slot.karr[i] = buf[i];
    const unsigned long long T = cnt >= k ? buf[k - 1] : kEmpty;
    const float band = prune_threshold(T, qp.F);
    __shared__ unsigned nlog;
    if (threadIdx.x == 0) nlog = 0;
    __syncthreads();
    for (unsigned i = threadIdx.x; i < cnt; i += blockDim.x)
        if (cand_d2(buf[i]) <= band) {
            const unsigned li = atomicAdd(&nlog, 1u);
            if (li < slot.log_cap) slot.log[li] = buf[i];
        }
    __syncthreads();
    if (threadIdx.x == 0) {
        st->kcount = kept;
        st->thr = T;
        st->log_count = nlog;
        st->seed_count = cnt;
        st->c.seeded = cnt;
        st->c.bsf_updates = T != kEmpty ? 1ull : 0ull;
    }
}

__global__ void __launch_bounds__(kFinThreads)
k_seed_select(IndexView iv, QueryParams qp, QuerySlot slot)
{
    seed_select_body(iv, qp, slot);
}

__global__ void __launch_bounds__(kFinThreads)
k_seed_select_batch(IndexView iv, QueryParams qp, const QuerySlot *__restrict__ slots)
{
    seed_select_body(iv, qp, slots[blockIdx.x]);
}

// ------------------------------------------------------------------ scan
// Persistent CTAs; CTA c owns the contiguous tiles [c*tpc, (c+1)*tpc) and
// writes its survivors into its own region of the survivor arrays (the same
// index range as its words), so compaction needs only a shared-memory counter.
// ------------------------------------------------------- leaf pruning
// Every word of a leaf lies in the leaf's symbol box, and each segment's table
// row is non-increasing up to the query's symbol and non-decreasing after it
// (the distance to a region grows with the region's distance from the
// query's value, and rounding down keeps that order), so the smallest entry
// over the box's range [lo, hi] sits at clamp(qsym, lo, hi).  Their sum,
// added rounding down, bounds every word of the leaf from below: a leaf above
// the threshold is skipped without reading its words -- the subtree pruning
// of the paper's traversal (Sec. 3, ED query answering), on leaf boxes.  One
// thread per leaf; the scan tiles a surviving leaf touches are stamped with
// the query's epoch.
__global__ void __launch_bounds__(256)
k_leaf_prune(IndexView iv, QueryParams qp, QuerySlot slot, unsigned epoch)
{
    __shared__ unsigned live;
    QueryState *st = slot.st;
    if (ld_volatile_u32(&st->invalid)) return;
    if (threadIdx.x == 0) live = 0;
    __syncthreads();
    const float thrp = prune_threshold(ld_volatile_u64(&st->thr), qp.F);
    const uint4 q = st->qsym;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    unsigned mine = 0;
    for (unsigned long long l = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; l < iv.L; l += stride) {
        const uint4 lo = iv.leaf_box[2 * l], hi = iv.leaf_box[2 * l + 1];
        const unsigned c[4] = {__vminu4(__vmaxu4(q.x, lo.x), hi.x), __vminu4(__vmaxu4(q.y, lo.y), hi.y),
                               __vminu4(__vmaxu4(q.z, lo.z), hi.z), __vminu4(__vmaxu4(q.w, lo.w), hi.w)};
        float lb = 0.f;
#pragma unroll
        for (int s = 0; s < kMaxSegments; ++s)
            lb = __fadd_rd(lb, __ldg(slot.lut + s * kMaxCard + ((c[s >> 2] >> (8 * (s & 3))) & 0xffu)));
        if (lb <= thrp) {
            ++mine;
            const unsigned long long a = iv.leaf_off[l], b = iv.leaf_off[l + 1];
            for (unsigned long long t = a / kScanTileWords; t <= (b - 1) / kScanTileWords; ++t)
                slot.tile_epoch[t] = epoch;
        }
    }
    if (mine) atomicAdd(&live, mine);
    __syncthreads();
    if (threadIdx.x == 0 && live) atomicAdd(&st->c.leaves_live, (unsigned long long)live);
}

// Compact the tiles stamped with this query's epoch into live_list.
__global__ void __launch_bounds__(256)
k_live_tiles(QuerySlot slot, unsigned long long ntiles, unsigned epoch)
{
    __shared__ unsigned wcount[8], wbase[8], bbase;
    QueryState *st = slot.st;
    if (ld_volatile_u32(&st->invalid)) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (unsigned long long t0 = (unsigned long long)blockIdx.x * blockDim.x; t0 < ntiles;
         t0 += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long t = t0 + threadIdx.x;
        const bool live = t < ntiles && slot.tile_epoch[t] == epoch;
        const unsigned ballot = __ballot_sync(0xffffffffu, live);
        if (lane == 0) wcount[warp] = __popc(ballot);
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned run = 0;
            for (int w = 0; w < 8; ++w) {
                wbase[w] = run;
                run += wcount[w];
            }
            bbase = run ? atomicAdd(&st->live_tiles, run) : 0u;
        }
        __syncthreads();
        if (live) slot.live_list[bbase + wbase[warp] + __popc(ballot & ((1u << lane) - 1u))] = (unsigned)t;
        __syncthreads();
    }
}

// The scan's table: every entry of the query's FP32 table (already rounded
// down) as a 16-bit multiple of a power of two D, rounded down and capped at
// 65535 -- code * D <= entry exactly, since dividing by a power of two is
// exact.  A word's bound is then (sum of its 16 codes) * D: an integer sum,
// at most 16 D below the sum of its FP32 entries, still never above the
// exact bound.  D is the smallest power of two >= R / 4096, R the pruning
// threshold (or, while no threshold exists, 16 x the largest entry, which
// bounds every word), so the looser bound costs at most R / 128 and a capped
// code alone already exceeds R.  Half the bytes of the FP32 table: a row of
// 256 entries spans 4 bank rows instead of 8, and the table lookups of a warp
// (the scan's bottleneck) meet fewer bank conflicts.
struct ScanCodes {
    float D;          // the power of two
    unsigned limit;   // largest code sum that survives: floor(threshold / D)
};

__device__ __forceinline__ ScanCodes scan_codes(const float *__restrict__ lut, float thrp, unsigned short *codes,
                                                 float *red)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float R = thrp;
    if (!(thrp < f_inf())) {   // no finite threshold: bound by the largest entry
        float mx = 0.f;
        for (int i = tid; i < kMaxSegments * kMaxCard; i += blockDim.x) mx = fmaxf(mx, lut[i]);
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
        if (lane == 0) red[warp] = mx;
        __syncthreads();
        mx = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mx = fmaxf(mx, red[w]);
        R = 16.f * mx;
    }
    int e = 0;
    const float f = frexpf(R * (1.f / 4096.f), &e);       // R / 4096 = f 2^e, f in [0.5, 1)
    ScanCodes sc;
    sc.D = (R > 0.f && f > 0.f) ? fmaxf(ldexpf(1.f, e), 1.17549435e-38f) : 1.17549435e-38f;   // >= R / 4096
    for (int i = tid; i < kMaxSegments * kMaxCard; i += blockDim.x) {
        const float c = lut[i] / sc.D;                    // exact (or overflow to inf)
        codes[i] = c >= 65535.f ? (unsigned short)65535 : (unsigned short)c;   // truncation = floor
    }
    if (thrp < f_inf()) {
        const float q = thrp / sc.D;                      // exact
        sc.limit = q >= 4294967040.f ? 0xffffffffu : (unsigned)q;
    } else {
        sc.limit = 0xffffffffu;
    }
    return sc;
}

// code sum of the 8 segments held in two 32-bit words starting at segment s0
// (symbol b of a word taken by one byte permute; the table sits in static
// shared memory, so its base folds into the loads' address offsets)
__device__ __forceinline__ unsigned code_half(unsigned w0, unsigned w1, const unsigned short *codes, int s0)
{
    unsigned v[8];
#pragma unroll
    for (int b = 0; b < 4; ++b) v[b] = codes[(s0 + b) * kMaxCard + __byte_perm(w0, 0u, 0x4440u + b)];
#pragma unroll
    for (int b = 0; b < 4; ++b) v[4 + b] = codes[(s0 + 4 + b) * kMaxCard + __byte_perm(w1, 0u, 0x4440u + b)];
    return ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]));
}

// Persistent CTAs; CTA c owns the contiguous run [c*tpc, (c+1)*tpc) of the
// live-tile list and writes its survivors into its own region of the
// survivor arrays, so compaction needs only a shared-memory counter.  Tiles
// arrive by 1-D bulk copies into a ring of kScanStages stages; no block-wide
// barrier per tile: each warp counts itself done with a stage, and the last
// warp to finish it refills it with the tile kScanStages further on, so warps
// drift apart by up to a few tiles instead of waiting for the slowest.
__global__ void __launch_bounds__(kScanThreads, kScanCtasPerSm)
k_lb_scan(IndexView iv, QueryParams qp, QuerySlot slot)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) unsigned long long bars[kScanStages];
    __shared__ unsigned done[kScanStages];
    __shared__ int issued_it[kScanStages];     // iteration of the last copy issued into each stage
    __shared__ int timed_out;
    __shared__ unsigned s_count;
    __shared__ float red[32];
    __shared__ __align__(16) unsigned short codes[kMaxSegments * kMaxCard];
    uint4 *stage = reinterpret_cast<uint4 *>(smem);
    QueryState *st = slot.st;
    if (ld_volatile_u32(&st->invalid)) return;
    const int tid = threadIdx.x, lane = tid & 31;
    constexpr unsigned kWarps = kScanThreads / 32;
    const float thrp = prune_threshold(ld_volatile_u64(&st->thr), qp.F);
    const unsigned long long seed_lo = st->seed_lo, seed_hi = st->seed_hi;
    const unsigned long long N = iv.N;
    // this CTA's share of the live tiles; its survivors go to its own region
    const unsigned nlive = st->live_tiles;
    const unsigned tpc = (nlive + gridDim.x - 1) / gridDim.x;
    const unsigned i0 = min(nlive, blockIdx.x * tpc), i1 = min(nlive, i0 + tpc);
    const unsigned long long region = (unsigned long long)blockIdx.x * tpc * kScanTileWords;
    auto issue = [&](unsigned idx, int s) {
        const unsigned long long first = (unsigned long long)slot.live_list[idx] * kScanTileWords;
        const unsigned long long cnt = min((unsigned long long)kScanTileWords, N - first);
        const unsigned bytes = (unsigned)(cnt * 16);
        issued_it[s] = (int)(idx - i0);
        mbar_arrive_expect_tx(&bars[s], bytes);
        bulk_g2s(stage + s * kScanTileWords, iv.sax + first, bytes, &bars[s]);
    };
    if (tid == 0) {
        timed_out = 0;
        s_count = 0;
        for (int s = 0; s < kScanStages; ++s) {
            mbar_init(&bars[s], 1);
            done[s] = 0;
            issued_it[s] = -1;
        }
        fence_barrier_init();
        fence_proxy_async();
        if (blockIdx.x == 0) {
            st->scan_grid = gridDim.x;
            st->region_words = tpc * kScanTileWords;
        }
        for (int s = 0; s < kScanStages && i0 + s < i1; ++s) issue(i0 + s, s);
    }
    const ScanCodes sc = scan_codes(slot.lut, thrp, codes, red);
    __syncthreads();
    unsigned iter = 0;
    unsigned tile_next = i0 < i1 ? slot.live_list[i0] : 0u;   // the next tile's number, loaded a tile ahead
    for (unsigned idx = i0; idx < i1; ++idx, ++iter) {
        if (__shfl_sync(0xffffffffu, *reinterpret_cast<volatile int *>(&timed_out), 0)) break;
        const unsigned tile = tile_next;
        if (idx + 1 < i1) tile_next = slot.live_list[idx + 1];
        const int s = iter % kScanStages;
        const unsigned parity = (iter / kScanStages) & 1u;
        if (!__all_sync(0xffffffffu, mbar_wait_bounded(&bars[s], parity))) {
            if (lane == 0) {
                atomicOr(iv.status, kStTimeout);
                timed_out = 1;
            }
            break;
        }
        const unsigned long long first = (unsigned long long)tile * kScanTileWords;
        const unsigned cnt = (unsigned)min((unsigned long long)kScanTileWords, N - first);
#pragma unroll
        for (int r = 0; r < kScanWpt; ++r) {
            const unsigned j = tid + r * kScanThreads;
            const bool valid = j < cnt;
            const uint4 wv = valid ? stage[s * kScanTileWords + j] : make_uint4(0, 0, 0, 0);
            // first half of the segments; the rest only if some lane can still survive
            unsigned sum = code_half(wv.x, wv.y, codes, 0);
            if (__any_sync(0xffffffffu, valid && sum <= sc.limit)) sum += code_half(wv.z, wv.w, codes, 8);
            const unsigned long long pos = first + j;
            const bool surv = valid && sum <= sc.limit && (pos < seed_lo || pos >= seed_hi);
            const unsigned ballot = __ballot_sync(0xffffffffu, surv);
            if (ballot) {   // warp-uniform
                unsigned base = 0;
                if (lane == 0) base = atomicAdd(&s_count, (unsigned)__popc(ballot));
                base = __shfl_sync(0xffffffffu, base, 0);
                if (surv) {
                    const unsigned long long o = region + base + __popc(ballot & ((1u << lane) - 1u));
                    slot.surv_pos[o] = (unsigned)pos;
                    slot.surv_lb[o] = (float)sum * sc.D;   // exact: sum < 2^24, D a power of two
                }
            }
        }
        // this warp is done with stage s; the last warp to finish it refills it
        __syncwarp();
        if (lane == 0) {
            __threadfence_block();
            if (atomicAdd(&done[s], 1u) == kWarps - 1) {
                done[s] = 0;
                if (idx + kScanStages < i1 && !*reinterpret_cast<volatile int *>(&timed_out)) {
                    fence_proxy_async();
                    issue(idx + kScanStages, s);
                }
            }
        }
    }
    __syncthreads();
    if (timed_out) {
        // each stage holds at most one copy in flight, the last one issued into
        // it (a stage is refilled only after every warp waited for and used
        // its previous copy); let those land before shared memory is released
        if (tid == 0)
            for (int s = 0; s < kScanStages; ++s)
                if (issued_it[s] >= 0) mbar_wait_bounded(&bars[s], ((unsigned)issued_it[s] / kScanStages) & 1u);
        if (tid == 0) slot.region_count[blockIdx.x] = 0;
        return;
    }
    if (tid == 0) {
        slot.region_count[blockIdx.x] = s_count;
        if (s_count) atomicAdd(&st->c.lb_survivors, (unsigned long long)s_count);
        if (i1 > i0) {
            unsigned long long wsum = 0;
            for (unsigned idx = i0; idx < i1; ++idx) {
                const unsigned long long first = (unsigned long long)slot.live_list[idx] * kScanTileWords;
                wsum += min((unsigned long long)kScanTileWords, N - first);
            }
            atomicAdd(&st->c.lb_evaluated, wsum);
        }
    }
}


// ------------------------------------------------------------ ED refine
// Refinement in bound order (the priority-queue order of Sec. 3, Algorithm
// 8), without sorting: the survivors stay in the scan's regions and the
// kernel sweeps them in kRefineBands passes over bands of the lower bound,
// band b holding bounds in [t (b / B)^2, t ((b + 1) / B)^2) of the scan's
// threshold t (uniform in distance).  Every warp finishes its share of band b
// before it starts band b + 1, and stops at the first band whose floor lies
// above the live best-so-far.  A warp owns a contiguous run of 128-entry
// survivor chunks and reads it chunk by chunk (each lane four consecutive
// positions and bounds by two 16-byte loads, the next chunk loaded while the
// current one is used); it gathers the entries inside the band and within
// the live threshold into a shared-memory buffer and, every 32 gathered,
// computes their real distances four rows at a time, re-checking each bound
// against the live threshold first.  Exactness does not depend on the order,
// only the number of rows read does.
constexpr int kRefineBands = 4;
constexpr int kRefineThreads = 256;
constexpr int kRefineRows = 4;
constexpr int kRefineChunkShift = 7;   // 128-entry chunks

__global__ void __launch_bounds__(kRefineThreads, 3)
k_refine_ed(IndexView iv, QueryParams qp, QuerySlot slot)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    __shared__ unsigned prefix[kMaxScanGrid + 1], counts[kMaxScanGrid];
    __shared__ unsigned gpos[kRefineThreads / 32][160];
    __shared__ float glb[kRefineThreads / 32][160];
    QueryState *st = slot.st;
    if (ld_volatile_u32(&st->invalid)) return;
    float *qs = reinterpret_cast<float *>(dsm);
    for (int i = threadIdx.x; i < iv.len; i += blockDim.x) qs[i] = slot.q[i];
    const unsigned G = st->scan_grid;
    const unsigned long long RW = st->region_words;
    const unsigned nchunks = chunk_prefix(slot, G, prefix, counts, kRefineChunkShift);   // ends with a block barrier
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    unsigned *bpos = gpos[wib];
    float *blb = glb[wib];
    const unsigned nw = gridDim.x * (blockDim.x >> 5);
    const unsigned wglob = blockIdx.x * (blockDim.x >> 5) + wib;
    const float t0 = prune_threshold(ld_volatile_u64(&st->thr), qp.F);
    const int bands = t0 < f_inf() ? kRefineBands : 1;
    unsigned long long done = 0, aband = 0, bytes = 0;
    // the live threshold, re-read after every group of rows (a stale value is
    // only looser: it skips fewer rows, and offer() re-checks what it accepts)
    float thr = t0;
    // refine the first `cnt` gathered entries (cnt <= 32), four rows at a time
    auto refine_buffered = [&](unsigned cnt) {
        for (unsigned e0 = 0; e0 < cnt; e0 += kRefineRows) {
            const float *x[kRefineRows];
            bool live[kRefineRows], take[kRefineRows];
            unsigned pos[kRefineRows];
#pragma unroll
            for (int r = 0; r < kRefineRows; ++r) {
                const unsigned e = e0 + r;
                take[r] = e < cnt && blb[e < cnt ? e : 0] <= thr;
                pos[r] = take[r] ? bpos[e] : bpos[0];
                x[r] = iv.raw + (unsigned long long)pos[r] * iv.len;
                live[r] = take[r];
            }
            // issued behind the row loads, so its latency overlaps theirs
            const unsigned long long T = ld_volatile_u64(&st->thr);
            float d[kRefineRows];
            int n[kRefineRows];
            warp_ed2_rows<kRefineRows>(qs, x, live, iv.len, thr, d, n);
#pragma unroll
            for (int r = 0; r < kRefineRows; ++r) {
                if (!take[r]) continue;
                bytes += 4ull * n[r];
                if (d[r] <= thr) {
                    ++done;
                    if (lane == 0) offer(qp, slot, iv.status, d[r], iv.ids[pos[r]]);
                } else {
                    ++aband;
                }
            }
            __syncwarp();
            thr = fminf(thr, prune_threshold(T, qp.F));
        }
    };
    // the warp's chunks: one contiguous run [c_lo, c_hi)
    const unsigned per = (nchunks + nw - 1) / nw;
    const unsigned c_lo = min(nchunks, wglob * per), c_hi = min(nchunks, c_lo + per);
    for (int band = 0; band < bands; ++band) {
        const float flo = bands == 1 ? 0.f : t0 * ((float)(band * band) / (float)(kRefineBands * kRefineBands));
        const float fhi = band == bands - 1 ? f_inf()
                                            : t0 * ((float)((band + 1) * (band + 1)) / (float)(kRefineBands * kRefineBands));
        thr = fminf(thr, prune_threshold(ld_volatile_u64(&st->thr), qp.F));
        if (flo > thr) break;   // every later band too
        unsigned nbuf = 0;      // warp-uniform
        // a chunk's region advances by at most a step or two from the
        // previous chunk's; lane l holds entries 4l .. 4l+3 of the chunk
        unsigned rg = c_lo < c_hi ? region_of(c_lo, prefix, G) : 0u;
        auto load = [&](unsigned ch, uint4 &pos, float4 &lb, unsigned &nvalid) {
            while (rg + 1 < G && prefix[rg + 1] <= ch) ++rg;
            const unsigned first = (ch - prefix[rg]) << kRefineChunkShift;
            nvalid = min(counts[rg] - first, 128u);
            const unsigned long long i = rg * RW + first + 4 * lane;   // 16-byte aligned
            if (4u * lane < nvalid) {
                pos = *reinterpret_cast<const uint4 *>(slot.surv_pos + i);
                lb = *reinterpret_cast<const float4 *>(slot.surv_lb + i);
            } else {
                pos = make_uint4(0, 0, 0, 0);
                lb = make_float4(f_inf(), f_inf(), f_inf(), f_inf());
            }
        };
        uint4 npos = make_uint4(0, 0, 0, 0);
        float4 nlb = make_float4(f_inf(), f_inf(), f_inf(), f_inf());
        unsigned nv = 0;
        if (c_lo < c_hi) load(c_lo, npos, nlb, nv);
        for (unsigned ch = c_lo; ch < c_hi; ++ch) {
            const uint4 cpos = npos;
            const float4 clb = nlb;
            const unsigned cnv = nv;
            if (ch + 1 < c_hi) load(ch + 1, npos, nlb, nv);
            const unsigned pp[4] = {cpos.x, cpos.y, cpos.z, cpos.w};
            const float ll[4] = {clb.x, clb.y, clb.z, clb.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float lb = ll[k];
                const bool keep = 4u * lane + k < cnv && lb >= flo && lb < fhi && lb <= thr;
                const unsigned ballot = __ballot_sync(0xffffffffu, keep);
                if (keep) {
                    const unsigned o = nbuf + __popc(ballot & ((1u << lane) - 1u));
                    bpos[o] = pp[k];
                    blb[o] = lb;
                }
                nbuf += __popc(ballot);
            }
            __syncwarp();
            while (nbuf >= 32) {
                refine_buffered(32);
                // move the rest (at most 127) to the front
                const unsigned rest = nbuf - 32;
                for (unsigned j = 0; j < rest; j += 32) {
                    unsigned p2 = 0;
                    float l2 = 0.f;
                    if (j + lane < rest) {
                        p2 = bpos[32 + j + lane];
                        l2 = blb[32 + j + lane];
                    }
                    __syncwarp();
                    if (j + lane < rest) {
                        bpos[j + lane] = p2;
                        blb[j + lane] = l2;
                    }
                    __syncwarp();
                }
                nbuf = rest;
            }
        }
        if (nbuf) refine_buffered(nbuf);
        __syncwarp();
    }
    if (lane == 0) {
        if (done) atomicAdd(&st->c.refined, done);
        if (aband) atomicAdd(&st->c.abandoned, aband);
        if (bytes) atomicAdd(&st->c.row_bytes, bytes);
    }
}

// ------------------------------------------------------ DTW: LB_Keogh
// Warp per survivor.  First LB_Keogh of the candidate C against the query's
// envelope [L, U] (Sec. 3.4); if that does not prune, Lemire's LB_Improved
// adds a second term: H = C clamped into [L, U], and the query against the
// envelope [L^H, U^H] of H (same window).  Why the sum still bounds the
// banded DTW from below: every cell (i, j) of a warping path has |i - j| <= r,
// so q_i lies in [L_j, U_j] and h_j lies between q_i and c_j; then
// (q_i - c_j)^2 >= (q_i - h_j)^2 + (h_j - c_j)^2.  Summed over the path, the
// second parts cover every j at least once (>= LB_Keogh(C; L, U)) and the
// first parts every i at least once, each with h_j inside [L^H_i, U^H_i]
// (>= the distance of q_i to that interval, squared).  The envelope of H
// comes from van Herk / Gil-Werman block prefix and suffix maxima (minima) in
// the warp's shared-memory buffer.  Every operation of both terms rounds
// toward -inf.
__device__ __forceinline__ float lbk_tail(float acc)
{
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) acc = __fadd_rd(acc, __shfl_xor_sync(0xffffffffu, acc, off));
    return acc;
}

__global__ void __launch_bounds__(256)
k_lbk(IndexView iv, QueryParams qp, QuerySlot slot, int wpb)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    __shared__ unsigned prefix[kMaxScanGrid + 1];
    __shared__ unsigned counts[kMaxScanGrid];
    QueryState *st = slot.st;
    if (ld_volatile_u32(&st->invalid)) return;
    const int len = iv.len;
    float *Us = reinterpret_cast<float *>(dsm);
    float *Ls = Us + len;
    float *qs = Ls + len;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    float *P = qs + len + (size_t)wib * 4 * len;      // per warp: prefix max, suffix max, prefix min, suffix min
    float *S = P + len, *Pm = S + len, *Sm = Pm + len;
    for (int i = threadIdx.x; i < len; i += blockDim.x) {
        Us[i] = slot.U[i];
        Ls[i] = slot.L[i];
        qs[i] = slot.q[i];
    }
    const unsigned G = st->scan_grid;
    const unsigned long long RW = st->region_words;
    const unsigned nchunks = chunk_prefix(slot, G, prefix, counts);
    const int r = qp.r < len - 1 ? qp.r : len - 1;
    const int w = 2 * r + 1;
    const int nblk = (len + w - 1) / w;
    const unsigned nw = gridDim.x * wpb;
    unsigned long long pass = 0;
    unsigned pend = 0, npend = 0;          // passing positions, one per lane, flushed by 32
    float pend_lb = 0.f;                   // and their LB_Keogh bounds
    for (unsigned ch = blockIdx.x * wpb + wib; ch < nchunks; ch += nw) {
        const unsigned rg = region_of(ch, prefix, G);
        const unsigned within = (ch - prefix[rg]) * 32 + lane;
        const bool valid = within < counts[rg];
        const unsigned long long i = rg * RW + within;
        const unsigned pos = valid ? slot.surv_pos[i] : 0u;
        const float lb = valid ? slot.surv_lb[i] : f_inf();
        const float thr = prune_threshold(ld_volatile_u64(&st->thr), qp.F);
        unsigned mask = __ballot_sync(0xffffffffu, valid && lb <= thr);
        while (mask) {
            const int a = __ffs(mask) - 1;
            mask &= mask - 1;
            const unsigned pa = __shfl_sync(0xffffffffu, pos, a);
            const float *x = iv.raw + (unsigned long long)pa * len;
            // candidate against the query's envelope
            float acc = 0.f, lbv = 0.f;
            bool pruned = false;
            for (int base = 0; base < len && !pruned; base += 256) {
                for (int t = lane; t < 256 && base + t < len; t += 32) {
                    const int idx = base + t;
                    const float c = __ldg(x + idx);
                    P[idx] = fminf(fmaxf(c, Ls[idx]), Us[idx]);   // H: C clamped into [L, U]
                    const float d = fmaxf(fmaxf(__fsub_rd(c, Us[idx]), __fsub_rd(Ls[idx], c)), 0.f);   // from [L, U]
                    acc = __fadd_rd(acc, __fmul_rd(d, d));
                }
                lbv = lbk_tail(acc);
                if (lbv > thr) pruned = true;
            }
            if (!pruned && r > 0) {
                __syncwarp();
                // block prefix / suffix extrema of H (blocks of w points)
                for (int blk = lane; blk < nblk; blk += 32) {
                    const int b0 = blk * w, b1 = min(len, b0 + w);
                    float mx = -f_inf(), mn = f_inf();
                    for (int t = b0; t < b1; ++t) {
                        const float v = P[t];
                        mx = fmaxf(mx, v);
                        mn = fminf(mn, v);
                        S[t] = mx;        // running prefix max, moved to P below
                        Sm[t] = mn;
                    }
                    mx = -f_inf();
                    mn = f_inf();
                    for (int t = b1 - 1; t >= b0; --t) {
                        const float v = P[t];
                        mx = fmaxf(mx, v);
                        mn = fminf(mn, v);
                        P[t] = S[t];      // prefix max
                        Pm[t] = Sm[t];    // prefix min
                        S[t] = mx;        // suffix max
                        Sm[t] = mn;       // suffix min
                    }
                }
                __syncwarp();
                const float fwd = lbv;            // LB_Keogh(C; L, U)
                float acc2 = 0.f;
                for (int base = 0; base < len && !pruned; base += 256) {
                    for (int t = lane; t < 256 && base + t < len; t += 32) {
                        const int idx = base + t;
                        const int lo = idx - r < 0 ? 0 : idx - r, hi = idx + r > len - 1 ? len - 1 : idx + r;
                        // [lo, hi] spans at most two adjacent blocks.  Within one
                        // block it starts at the block start (prefix extremum at
                        // hi) or ends at the block end (suffix extremum at lo);
                        // across two, the suffix of the first joins the prefix of
                        // the second.
                        float U, L;
                        if (lo / w == hi / w) {
                            if (lo % w == 0) { U = P[hi]; L = Pm[hi]; }
                            else { U = S[lo]; L = Sm[lo]; }
                        } else {
                            U = fmaxf(S[lo], P[hi]);
                            L = fminf(Sm[lo], Pm[hi]);
                        }
                        const float c = qs[idx];
                        const float d = fmaxf(fmaxf(__fsub_rd(c, U), __fsub_rd(L, c)), 0.f);   // from [L, U]
                        acc2 = __fadd_rd(acc2, __fmul_rd(d, d));
                    }
                    // LB_Improved so far: the first term plus the query's part
                    lbv = __fadd_rd(fwd, lbk_tail(acc2));
                    if (lbv > thr) pruned = true;
                }
            }
            __syncwarp();
            if (!pruned) {
                ++pass;
                if (lane == (int)npend) {
                    pend = pa;
                    pend_lb = lbv;
                }
                if (++npend == 32) {
                    unsigned o = 0;
                    if (lane == 0) o = atomicAdd(&st->surv2_count, 32u);
                    o = __shfl_sync(0xffffffffu, o, 0);
                    slot.surv2[o + lane] = pend;
                    slot.surv2_lb[o + lane] = pend_lb;
                    npend = 0;
                }
            }
        }
    }
    if (npend) {
        unsigned o = 0;
        if (lane == 0) o = atomicAdd(&st->surv2_count, npend);
        o = __shfl_sync(0xffffffffu, o, 0);
        if ((unsigned)lane < npend) {
            slot.surv2[o + lane] = pend;
            slot.surv2_lb[o + lane] = pend_lb;
        }
    }
    if (lane == 0 && pass) atomicAdd(&st->c.lbk_survivors, pass);
}

// ---------------------------------------------------------------- DTW
__global__ void __launch_bounds__(256)
k_dtw(IndexView iv, QueryParams qp, QuerySlot slot)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    QueryState *st = slot.st;
    if (ld_volatile_u32(&st->invalid)) return;
    float *qs = reinterpret_cast<float *>(dsm);
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *diag = qs + iv.len + wib * 3 * iv.len;
    for (int i = threadIdx.x; i < iv.len; i += blockDim.x) qs[i] = slot.q[i];
    __syncthreads();
    const unsigned count = ld_volatile_u32(&st->ord_count);
    const unsigned nw = gridDim.x * (blockDim.x >> 5);
    unsigned long long done = 0, aband = 0;
    for (unsigned i = blockIdx.x * (blockDim.x >> 5) + wib; i < count; i += nw) {
        // bound-ordered list: once a bucket floor exceeds the threshold, so
        // does everything later in this warp's sequence
        const unsigned pos = slot.surv_pos[i];
        const float lb = slot.surv_lb[i];
        const float thr = prune_threshold(ld_volatile_u64(&st->thr), qp.F);
        if (order_floor(order_bucket(lb)) > thr) break;
        if (lb > thr) continue;
        const float d2 = warp_dtw<float>(qs, iv.raw + (unsigned long long)pos * iv.len, iv.len, qp.r, diag, thr);
        if (d2 > thr) { ++aband; continue; }
        ++done;
        if (lane == 0) offer(qp, slot, iv.status, d2, iv.ids[pos]);
        __syncwarp();
    }
    if (lane == 0) {
        if (done) atomicAdd(&st->c.refined, done);
        if (aband) atomicAdd(&st->c.abandoned, aband);
    }
}

// ------------------------------------------------- batched fused (ED)
// One launch answers the lower-bound + refine part of a batch of queries.
// Work items are (chunk of consecutive scan tiles, query) pairs handed out by
// an atomic counter in chunk-major order, so all queries of a batch visit a
// chunk close in time and its iSAX words come from HBM once and from L2 after.
// Per item: the query's table and vector go to shared memory, the chunk's
// words stream through TMA bulk copies, each tile's survivors (bound <= the
// query's live best-so-far) are compacted in shared memory and refined right
// away by the block's warps, so later tiles prune against the improved bound.
constexpr int kFuThreads = 256;
constexpr int kFuWpt = kScanTileWords / kFuThreads;    // 4 words per thread per tile
constexpr int kFuStages = 4;
constexpr int kFuSmemFixed = kMaxSegments * kMaxCard * 4 + kFuStages * kScanTileWords * 16 +
                             kScanTileWords * 8;        // table + stages + survivor list

__global__ void __launch_bounds__(kFuThreads, 2)
k_fused_ed(IndexView iv, QueryParams qp, const QuerySlot *__restrict__ slots, unsigned B, unsigned chunk_tiles,
           unsigned *__restrict__ counter)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) unsigned long long bars[kFuStages];
    __shared__ unsigned s_item, s_n;
    __shared__ float s_thr;
    __shared__ int s_fail;
    float *lut = reinterpret_cast<float *>(smem);
    uint4 *stage = reinterpret_cast<uint4 *>(smem + kMaxSegments * kMaxCard * 4);
    unsigned *list_pos = reinterpret_cast<unsigned *>(smem + kMaxSegments * kMaxCard * 4 +
                                                      kFuStages * kScanTileWords * 16);
    float *list_lb = reinterpret_cast<float *>(list_pos + kScanTileWords);
    float *qs = list_lb + kScanTileWords;
    const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
    const unsigned long long N = iv.N;
    const unsigned long long ntiles = (N + kScanTileWords - 1) / kScanTileWords;
    const unsigned long long nchunks = (ntiles + chunk_tiles - 1) / chunk_tiles;
    const unsigned long long nitems = nchunks * B;
    if (tid == 0) {
        s_fail = 0;
        for (int s = 0; s < kFuStages; ++s) mbar_init(&bars[s], 1);
        fence_barrier_init();
        fence_proxy_async();
    }
    __syncthreads();
    unsigned uses[kFuStages] = {0, 0, 0, 0};   // completed phases per stage (thread-uniform)
    while (true) {
        if (tid == 0) s_item = atomicAdd(counter, 1u);
        __syncthreads();
        const unsigned long long item = s_item;
        if (item >= nitems || s_fail) break;
        const unsigned b = (unsigned)(item % B);
        const unsigned long long c = item / B;
        const QuerySlot slot = slots[b];
        QueryState *st = slot.st;
        if (ld_volatile_u32(&st->invalid)) {   // uniform: every thread takes this branch
            __syncthreads();
            continue;
        }
        for (int i = tid; i < kMaxSegments * kMaxCard; i += blockDim.x) lut[i] = slot.lut[i];
        for (int i = tid; i < iv.len; i += blockDim.x) qs[i] = slot.q[i];
        const unsigned long long seed_lo = st->seed_lo, seed_hi = st->seed_hi;
        const unsigned long long t0 = c * chunk_tiles, t1 = min(t0 + chunk_tiles, ntiles);
        const unsigned nt = (unsigned)(t1 - t0);
        auto issue = [&](unsigned long long tile, int sidx) {
            const unsigned long long first = tile * kScanTileWords;
            const unsigned long long cnt = min((unsigned long long)kScanTileWords, N - first);
            const unsigned bytes = (unsigned)(cnt * 16);
            mbar_arrive_expect_tx(&bars[sidx], bytes);
            bulk_g2s(stage + sidx * kScanTileWords, iv.sax + first, bytes, &bars[sidx]);
        };
        if (tid == 0)
            for (unsigned t = 0; t < nt && t < (unsigned)kFuStages; ++t) issue(t0 + t, (int)t);
        __syncthreads();
        unsigned long long evals = 0, nsurv = 0, done = 0, aband = 0, bytes = 0;
        for (unsigned t = 0; t < nt; ++t) {
            const int sidx = t % kFuStages;
            const bool ok = mbar_wait_bounded(&bars[sidx], uses[sidx] & 1u);
            if (tid == 0) {
                s_n = 0;
                s_thr = prune_threshold(ld_volatile_u64(&st->thr), qp.F);
            }
            if (__syncthreads_or(!ok)) {
                if (tid == 0) {
                    atomicOr(iv.status, kStTimeout);
                    s_fail = 1;
                }
                // let copies still in flight land before leaving
                if (tid == 0)
                    for (unsigned u = t; u < nt && u < t + kFuStages; ++u)
                        mbar_wait_bounded(&bars[u % kFuStages], (uses[u % kFuStages] + (u - t) / kFuStages) & 1u);
                return;
            }
            ++uses[sidx];
            const float thr = s_thr;
            const unsigned long long first = (t0 + t) * kScanTileWords;
            const unsigned cnt = (unsigned)min((unsigned long long)kScanTileWords, N - first);
            evals += cnt;
#pragma unroll
            for (int r = 0; r < kFuWpt; ++r) {
                const unsigned j = tid + r * kFuThreads;
                const bool valid = j < cnt;
                const uint4 wv = valid ? stage[sidx * kScanTileWords + j] : make_uint4(0, 0, 0, 0);
                float lb = lb2_half(wv.x, wv.y, lut, 0, 0.f);
                if (__any_sync(0xffffffffu, valid && lb <= thr)) lb = lb2_half(wv.z, wv.w, lut, 8, lb);
                const unsigned long long pos = first + j;
                const bool surv = valid && lb <= thr && (pos < seed_lo || pos >= seed_hi);
                const unsigned ballot = __ballot_sync(0xffffffffu, surv);
                if (ballot) {
                    unsigned base = 0;
                    if (lane == 0) base = atomicAdd(&s_n, (unsigned)__popc(ballot));
                    base = __shfl_sync(0xffffffffu, base, 0);
                    if (surv) {
                        const unsigned o = base + __popc(ballot & ((1u << lane) - 1u));
                        list_pos[o] = (unsigned)pos;
                        list_lb[o] = lb;
                    }
                }
            }
            __syncthreads();
            // words of this stage are consumed: prefetch the tile kFuStages ahead
            if (tid == 0 && t + kFuStages < nt) issue(t0 + t + kFuStages, sidx);
            const unsigned n = s_n;
            nsurv += n;
            // refine this tile's survivors: warps take two at a time
            for (unsigned e = 2 * wib; e < n; e += 2 * (kFuThreads / 32)) {
                const float live = prune_threshold(ld_volatile_u64(&st->thr), qp.F);
                const bool ua = list_lb[e] <= live;
                const bool ub = e + 1 < n && list_lb[e + 1] <= live;
                if (!ua && !ub) continue;
                const unsigned pa = list_pos[e], pb = (e + 1 < n) ? list_pos[e + 1] : pa;
                float da, db;
                int na, nb;
                warp_ed2_pair(qs, iv.raw + (unsigned long long)(ua ? pa : pb) * iv.len,
                              iv.raw + (unsigned long long)pb * iv.len, iv.len, live, da, db, na, nb);
                if (ua) {
                    bytes += 4ull * na;
                    if (da <= live) { ++done; if (lane == 0) offer(qp, slot, iv.status, da, iv.ids[pa]); }
                    else ++aband;
                }
                if (ub) {
                    bytes += 4ull * nb;
                    if (db <= live) { ++done; if (lane == 0) offer(qp, slot, iv.status, db, iv.ids[pb]); }
                    else ++aband;
                }
                __syncwarp();
            }
            __syncthreads();
        }
        if (tid == 0) {
            atomicAdd(&st->c.lb_evaluated, evals);
            if (nsurv) atomicAdd(&st->c.lb_survivors, nsurv);
        }
        if (lane == 0) {
            if (done) atomicAdd(&st->c.refined, done);
            if (aband) atomicAdd(&st->c.abandoned, aband);
            if (bytes) atomicAdd(&st->c.row_bytes, bytes);
        }
        __syncthreads();
    }
}

// ------------------------------------------------- DTW, one thread per candidate
// The recurrence is symmetric in its two series (the band |i - j| <= r and
// the three predecessors map onto themselves under a transpose, and
// (q_i - x_j)^2 = (x_j - q_i)^2 exactly), so the walk goes column by column
// of the candidate: D[b] is the cell (i, j) = (j - R + b, j) of column j in
// a band of width W = 2R+1 (R >= r; band cells farther than r from the
// diagonal are +inf), held in registers.  Column by column each thread
// updates its band in place (diagonal = old D[b], from the previous column
// = old D[b+1], from the same column = new D[b-1]) and abandons when a
// column minimum exceeds the live threshold (every warping path crosses
// every column; the minimum is taken every fourth column).  The candidate
// contributes one value per column; the query values of the band come from
// shared memory, where the query is stored four times, shifted by 0..3
// points and padded with +inf, so that any four consecutive values are one
// aligned 16-byte load (a broadcast: every thread of a warp walks the same
// query).  A band cell off the ends of the query meets a +inf value, so its
// cost (x_j - inf)^2 is +inf and it stays +inf without a test; when the
// window equals the reach (r == R) no cell needs a test at all.  Threads
// advance independently through their own candidates (a strided share of
// the list).
constexpr int kDtwPad = 36;   // padding of each shifted copy: >= 32 + 3, a multiple of 4

// floats per shifted copy of an n-point query (a multiple of 4, so that
// every copy starts 16-byte aligned)
__host__ __device__ __forceinline__ int dtw_qstride(int n) { return (n + 2 * kDtwPad + 3) & ~3; }

// minimum of three floats in one instruction
__device__ __forceinline__ float min3f(float a, float b, float c)
{
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// fill the four shifted copies: Qs[s * S + t] = q[t + s - kDtwPad] (+inf outside)
__device__ __forceinline__ void dtw_fill_query(float *Qs, const float *__restrict__ q, int n)
{
    const int S = dtw_qstride(n);
    for (int e = threadIdx.x; e < 4 * S; e += blockDim.x) {
        const int sh = e / S, t = e - sh * S;
        const int m = t + sh - kDtwPad;
        Qs[e] = (m >= 0 && m < n) ? q[m] : f_inf();
    }
}

// one column; BAND: cells farther than r from the diagonal are forced to
// +inf (only when r < R)
template <int R, bool BAND>
__device__ __forceinline__ void dtw_col(float (&D)[2 * R + 1], const float *__restrict__ Qs, int S, float xj, int j,
                                        int r)
{
    constexpr int W = 2 * R + 1;
    constexpr int NV = (W + 3) / 4;
    const float INF = f_inf();
    // q[j - R + b] for b = 0 .. W-1, from the copy whose shift aligns them
    const int t0 = j - R + kDtwPad;
    const int sh = t0 & 3;
    const float4 *qv = reinterpret_cast<const float4 *>(Qs + sh * S + (t0 - sh));
    float left = INF;
#pragma unroll
    for (int c = 0; c < NV; ++c) {
        const float4 q4 = qv[c];
        const float qq[4] = {q4.x, q4.y, q4.z, q4.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int b = 4 * c + u;
            if (b < W) {
                const float up = (b + 1 < W) ? D[b + 1] : INF;
                const float best = min3f(D[b], up, left);
                const float d = xj - qq[u];
                float v = d * d + best;
                if (BAND) v = (b - R <= r && R - b <= r) ? v : INF;
                D[b] = v;
                left = v;
            }
        }
    }
}

// minimum of the band
template <int R>
__device__ __forceinline__ float dtw_band_min(const float (&D)[2 * R + 1])
{
    constexpr int W = 2 * R + 1;
    float m = D[0];
#pragma unroll
    for (int b = 1; b + 1 < W; b += 2) m = min3f(m, D[b], D[b + 1]);
    return m;
}

template <int R>
__device__ __forceinline__ float thread_dtw(const float *__restrict__ Qs, const float *__restrict__ x, int n, int r,
                                            float thr, int &cols)
{
    constexpr int W = 2 * R + 1;
    const float INF = f_inf();
    const int S = dtw_qstride(n);
    float D[W];
#pragma unroll
    for (int b = 0; b < W; ++b) D[b] = (b == R) ? 0.f : INF;   // column -1: only the diagonal of (0, 0) is open
    const bool band = r != R;
    float xn = __ldg(x);
    for (int j = 0; j < n; ++j) {
        const float xj = xn;
        if (j + 1 < n) xn = __ldg(x + j + 1);
        if (band) dtw_col<R, true>(D, Qs, S, xj, j, r);
        else dtw_col<R, false>(D, Qs, S, xj, j, r);
        cols = j + 1;
        if ((j & 3) == 3) {
            const float cmin = dtw_band_min<R>(D);
            if (cmin > thr) return cmin;
        }
    }
    return D[R];
}

template <int R, int MODE>   // MODE 0: refine the LB_Keogh survivors, 1: seed range
__global__ void __launch_bounds__(128)
k_dtw_thread(IndexView iv, QueryParams qp, QuerySlot slot)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    QueryState *st = slot.st;
    if (ld_volatile_u32(&st->invalid)) return;
    float *Qs = reinterpret_cast<float *>(dsm);
    dtw_fill_query(Qs, slot.q, iv.len);
    __syncthreads();
    const unsigned lo = MODE ? st->seed_lo : 0u;
    const unsigned count = MODE ? st->seed_hi - st->seed_lo : ld_volatile_u32(&st->ord_count);
    const unsigned T = gridDim.x * blockDim.x;
    unsigned long long done = 0, aband = 0, cells = 0;
    for (unsigned e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += T) {
        const unsigned pos = MODE ? lo + e : slot.surv_pos[e];
        const float thr = MODE ? f_inf() : prune_threshold(ld_volatile_u64(&st->thr), qp.F);
        if (!MODE) {
            // bound-ordered list: this thread's later candidates lie in the
            // same or higher buckets
            const float lb = slot.surv_lb[e];
            if (order_floor(order_bucket(lb)) > thr) break;
            if (lb > thr) continue;
        }
        int cols = 0;
        const float d2 = thread_dtw<R>(Qs, iv.raw + (unsigned long long)pos * iv.len, iv.len, qp.r, thr, cols);
        cells += (unsigned long long)cols * (unsigned)(2 * qp.r + 1);   // band cells of the columns computed
        if (MODE) {
            slot.seedbuf[e] = pack_cand(d2, iv.ids[pos]);
        } else if (d2 <= thr) {
            ++done;
            offer(qp, slot, iv.status, d2, iv.ids[pos]);
        } else {
            ++aband;
        }
    }
    if (!MODE) {
        if (done) atomicAdd(&st->c.refined, done);
        if (aband) atomicAdd(&st->c.abandoned, aband);
    }
    if (cells) atomicAdd(&st->c.dtw_cells, cells);
}

// LB_Keogh + LB_Improved of one candidate, one thread, one pass over the row
// (the bounds of k_lbk, in the same FP32 operations, all rounded toward
// -inf).  Step i reads c_i, adds its LB_Keogh term and pushes h_i = c_i
// clamped into [L_i, U_i] into a register window of the last 2R + 1 h values;
// from step r on it adds the query term of position p = i - r, which needs
// the extremes of h over [p - r, p + r] = the newest 2r + 1 window slots.
// The window starts filled with h_0 and the steps past the end push h_{n-1}
// again: both are in every clipped window they stand in for, so the extremes
// are those of the clipped window.  Returns the bound, or a value above thr
// once the partial sum (a lower bound of the full one) exceeds it.
template <int R>
__device__ __forceinline__ float lbk_improved_thread(const float *__restrict__ qs, const float *__restrict__ Us,
                                                     const float *__restrict__ Ls, const float *__restrict__ x,
                                                     int n, int r, float thr)
{
    constexpr int W = 2 * R + 1;
    float hw[W];
    {
        const float c0 = __ldg(x);
        const float h0 = fminf(fmaxf(c0, Ls[0]), Us[0]);
#pragma unroll
        for (int b = 0; b < W; ++b) hw[b] = h0;
    }
    const int lo_b = 2 * (R - r);       // first window slot inside [p - r, p + r]
    float acc1 = 0.f, acc2 = 0.f;
    for (int i = 0; i < n + r; ++i) {
        if ((i & 31) == 0 && i + 64 < n) prefetch_l1(x + i + 64);   // two lines ahead
        float h = hw[W - 1];
        if (i < n) {
            const float c = __ldg(x + i), u = Us[i], l = Ls[i];
            const float d = fmaxf(fmaxf(__fsub_rd(c, u), __fsub_rd(l, c)), 0.f);   // distance from [l, u]
            acc1 = __fadd_rd(acc1, __fmul_rd(d, d));
            h = fminf(fmaxf(c, l), u);
        }
#pragma unroll
        for (int b = 0; b + 1 < W; ++b) hw[b] = hw[b + 1];
        hw[W - 1] = h;
        const int p = i - r;
        if (p >= 0) {
            float mx = h, mn = h;
#pragma unroll
            for (int b = 0; b + 1 < W; ++b) {
                const float v = (b >= lo_b) ? hw[b] : h;
                mx = fmaxf(mx, v);
                mn = fminf(mn, v);
            }
            const float qv = qs[p];
            const float d = fmaxf(fmaxf(__fsub_rd(qv, mx), __fsub_rd(mn, qv)), 0.f);   // distance from [mn, mx]
            acc2 = __fadd_rd(acc2, __fmul_rd(d, d));
        }
        if (__fadd_rd(acc1, acc2) > thr) return __fadd_rd(acc1, acc2);
    }
    return __fadd_rd(acc1, acc2);
}

// The same bound when the window is exactly R (r == R), with the extremes of
// each window from van Herk / Gil-Werman blocks instead of a scan of the
// window.  The blocks hold B = W + 1 = 2R + 2 steps, one more than the window
// W = 2R + 1, so that B is even (a multiple of 4 when R is odd) and every
// block starts on a vector boundary: the row and the envelope are read two or
// four points per load (the row's loads are the filter's bottleneck: each
// lane reads its own row, so a warp's load touches 32 lines).  A window
// ending at block slot k covers:
//   k <= B - 3: the previous block's slots k + 2 .. B - 1 (its suffix
//               extreme) and the current slots 0 .. k (a running prefix);
//   k =  B - 2: the current slots 0 .. B - 2 (the prefix);
//   k =  B - 1: the current slots 1 .. B - 1 (the block's own suffix from 1,
//               formed first at the block's end).
// The previous block's slot k is last read at step k - 2, so step k
// overwrites it with the new value, and the block's end turns the new values
// into suffix extremes in place.  About six min / max per step instead of 3W.
template <int R>
__device__ __forceinline__ float lbk_improved_blocks(const float *__restrict__ qs, const float *__restrict__ Us,
                                                     const float *__restrict__ Ls, const float *__restrict__ x,
                                                     int n, float thr)
{
    constexpr int W = 2 * R + 1;
    constexpr int B = W + 1;
    constexpr int VW = (B % 4 == 0) ? 4 : 2;   // points per vector load (n is a multiple of 4)
    float smx[B], smn[B];
    float hlast;
    {
        const float c0 = __ldg(x);
        hlast = fminf(fmaxf(c0, Ls[0]), Us[0]);
#pragma unroll
        for (int b = 0; b < B; ++b) {
            smx[b] = hlast;
            smn[b] = hlast;
        }
    }
    float acc1 = 0.f, acc2 = 0.f;
    for (int j0 = 0; j0 < n + R; j0 += B) {
        // this lane's row: ask L1 for the lines of the next block early so
        // several rows' misses overlap
        if (j0 + B < n) prefetch_l1(x + j0 + B);
        if (j0 + B + 32 < n) prefetch_l1(x + j0 + B + 32);
        float pmx = 0.f, pmn = 0.f;
        float cv[VW], uv[VW], lv[VW];
#pragma unroll
        for (int k = 0; k < B; ++k) {
            const int j = j0 + k;
            if (k % VW == 0 && j < n) {   // j0 and k are multiples of VW: aligned, and j + VW <= n
                if (VW == 4) {
                    const float4 c4 = __ldg(reinterpret_cast<const float4 *>(x + j));
                    const float4 u4 = *reinterpret_cast<const float4 *>(Us + j);
                    const float4 l4 = *reinterpret_cast<const float4 *>(Ls + j);
                    cv[0] = c4.x; cv[1] = c4.y; cv[VW > 2 ? 2 : 0] = c4.z; cv[VW > 3 ? 3 : 0] = c4.w;
                    uv[0] = u4.x; uv[1] = u4.y; uv[VW > 2 ? 2 : 0] = u4.z; uv[VW > 3 ? 3 : 0] = u4.w;
                    lv[0] = l4.x; lv[1] = l4.y; lv[VW > 2 ? 2 : 0] = l4.z; lv[VW > 3 ? 3 : 0] = l4.w;
                } else {
                    const float2 c2 = __ldg(reinterpret_cast<const float2 *>(x + j));
                    const float2 u2 = *reinterpret_cast<const float2 *>(Us + j);
                    const float2 l2 = *reinterpret_cast<const float2 *>(Ls + j);
                    cv[0] = c2.x; cv[1] = c2.y;
                    uv[0] = u2.x; uv[1] = u2.y;
                    lv[0] = l2.x; lv[1] = l2.y;
                }
            }
            float h = hlast;
            if (j < n) {
                const float c = cv[k % VW], u = uv[k % VW], l = lv[k % VW];
                // distance of c from [l, u] (at most one difference is
                // positive): no branch, so the lanes of a warp stay together
                const float d = fmaxf(fmaxf(__fsub_rd(c, u), __fsub_rd(l, c)), 0.f);
                acc1 = __fadd_rd(acc1, __fmul_rd(d, d));
                h = fminf(fmaxf(c, l), u);
                hlast = h;
            }
            pmx = (k == 0) ? h : fmaxf(pmx, h);
            pmn = (k == 0) ? h : fminf(pmn, h);
            float mx = pmx, mn = pmn;
            if (k + 2 < B) {
                mx = fmaxf(smx[k + 2 < B ? k + 2 : 0], pmx);
                mn = fminf(smn[k + 2 < B ? k + 2 : 0], pmn);
            }
            smx[k] = h;
            smn[k] = h;
            if (k + 1 == B) {
#pragma unroll
                for (int kk = B - 2; kk >= 0; --kk) {
                    smx[kk] = fmaxf(smx[kk], smx[kk + 1]);
                    smn[kk] = fminf(smn[kk], smn[kk + 1]);
                }
                mx = smx[1];
                mn = smn[1];
            }
            const int p = j - R;
            if (p >= 0 && p < n) {
                // distance of q_p from [mn, mx], without a branch as above
                const float qv = qs[p];
                const float d = fmaxf(fmaxf(__fsub_rd(qv, mx), __fsub_rd(mn, qv)), 0.f);
                acc2 = __fadd_rd(acc2, __fmul_rd(d, d));
            }
        }
        if (__fadd_rd(acc1, acc2) > thr) break;
    }
    return __fadd_rd(acc1, acc2);
}

template <int R>
__global__ void __launch_bounds__(256, (R <= 25) ? 2 : 1)
k_lbk_thread(IndexView iv, QueryParams qp, QuerySlot slot)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    __shared__ unsigned prefix[kMaxScanGrid + 1];
    __shared__ unsigned counts[kMaxScanGrid];
    QueryState *st = slot.st;
    if (ld_volatile_u32(&st->invalid)) return;
    const int len = iv.len;
    float *Us = reinterpret_cast<float *>(dsm);
    float *Ls = Us + len;
    float *qs = Ls + len;
    for (int i = threadIdx.x; i < len; i += blockDim.x) {
        Us[i] = slot.U[i];
        Ls[i] = slot.L[i];
        qs[i] = slot.q[i];
    }
    const unsigned G = st->scan_grid;
    const unsigned long long RW = st->region_words;
    const unsigned nchunks = chunk_prefix(slot, G, prefix, counts);   // also publishes the arrays above
    const int lane = threadIdx.x & 31;
    const unsigned nw = gridDim.x * (blockDim.x >> 5);
    unsigned long long pass = 0;
    for (unsigned ch = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); ch < nchunks; ch += nw) {
        const unsigned rg = region_of(ch, prefix, G);
        const unsigned within = (ch - prefix[rg]) * 32 + lane;
        const bool valid = within < counts[rg];
        const unsigned long long i = rg * RW + within;
        const unsigned pos = valid ? slot.surv_pos[i] : 0u;
        const float lb = valid ? slot.surv_lb[i] : f_inf();
        const float thr = prune_threshold(ld_volatile_u64(&st->thr), qp.F);
        bool keep = valid && lb <= thr;
        float lbv = 0.f;
        if (keep) {
            const float *x = iv.raw + (unsigned long long)pos * len;
            lbv = (qp.r == R) ? lbk_improved_blocks<R>(qs, Us, Ls, x, len, thr)
                              : lbk_improved_thread<R>(qs, Us, Ls, x, len, qp.r, thr);
            keep = lbv <= thr;
        }
        const unsigned ballot = __ballot_sync(0xffffffffu, keep);
        if (ballot) {
            unsigned o = 0;
            if (lane == 0) o = atomicAdd(&st->surv2_count, (unsigned)__popc(ballot));
            o = __shfl_sync(0xffffffffu, o, 0) + __popc(ballot & ((1u << lane) - 1u));
            if (keep) {
                slot.surv2[o] = pos;
                slot.surv2_lb[o] = lbv;
            }
            pass += (lane == 0) ? (unsigned long long)__popc(ballot) : 0ull;
        }
    }
    if (lane == 0 && pass) atomicAdd(&st->c.lbk_survivors, pass);
}

bool launch_lbk_thread(const IndexView &iv, const QueryParams &qp, const QuerySlot &slot, cudaStream_t s);

// smallest instantiated band reach >= r (or -1: use the warp wavefront)
int dtw_thread_reach(int r)
{
    static const int reaches[] = {0, 1, 2, 4, 6, 8, 12, 16, 20, 25, 32};
    for (int R : reaches)
        if (R >= r) return R;
    return -1;
}

template <int MODE>
bool launch_dtw_thread(const IndexView &iv, const QueryParams &qp, const QuerySlot &slot, cudaStream_t s)
{
    const int R = dtw_thread_reach(qp.r);
    const unsigned grid = num_sms() * 8;
    const size_t sm = (size_t)4 * dtw_qstride(iv.len) * sizeof(float);   // the four shifted query copies
    switch (R) {
#define MESSI_DTW_CASE(RR)                                                                                \
    case RR:                                                                                              \
        if (sm > 48 * 1024)                                                                               \
            cudaFuncSetAttribute(k_dtw_thread<RR, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); \
        k_dtw_thread<RR, MODE><<<grid, 128, sm, s>>>(iv, qp, slot);                                       \
        return true;
        MESSI_DTW_CASE(0)
        MESSI_DTW_CASE(1)
        MESSI_DTW_CASE(2)
        MESSI_DTW_CASE(4)
        MESSI_DTW_CASE(6)
        MESSI_DTW_CASE(8)
        MESSI_DTW_CASE(12)
        MESSI_DTW_CASE(16)
        MESSI_DTW_CASE(20)
        MESSI_DTW_CASE(25)
        MESSI_DTW_CASE(32)
#undef MESSI_DTW_CASE
        default: return false;
    }
}

bool launch_lbk_thread(const IndexView &iv, const QueryParams &qp, const QuerySlot &slot, cudaStream_t s)
{
    const int R = dtw_thread_reach(qp.r);
    const unsigned grid = num_sms() * 8;
    const size_t sm = (size_t)iv.len * 12;
    switch (R) {
#define MESSI_LBK_CASE(RR) \
    case RR: k_lbk_thread<RR><<<grid, 256, sm, s>>>(iv, qp, slot); return true;
        MESSI_LBK_CASE(0)
        MESSI_LBK_CASE(1)
        MESSI_LBK_CASE(2)
        MESSI_LBK_CASE(4)
        MESSI_LBK_CASE(6)
        MESSI_LBK_CASE(8)
        MESSI_LBK_CASE(12)
        MESSI_LBK_CASE(16)
        MESSI_LBK_CASE(20)
        MESSI_LBK_CASE(25)
        MESSI_LBK_CASE(32)
#undef MESSI_LBK_CASE
        default: return false;
    }
}

// ------------------------------------------------------------- finalize
// Bitonic sort of n (power of two) entries in shared memory with a caller
// ordering `less(i, j)` and swap `swap(i, j)`.
template <typename Less, typename Swap>
__device__ void block_bitonic(unsigned npow, Less less, Swap swap)
{
    for (unsigned size = 2; size <= npow; size <<= 1)
        for (unsigned stride = size >> 1; stride > 0; stride >>= 1) {
            for (unsigned i = threadIdx.x; i < npow; i += blockDim.x) {
                const unsigned j = i ^ stride;
                if (j > i) {
                    const bool up = (i & size) == 0;
                    if (less(j, i) == up) swap(i, j);
                }
            }
            __syncthreads();
        }
}

// candidates and their FP64 distances (kLogCap each), then a running top-k
// (kMaxK each) for band populations larger than one pass
constexpr int kFinSmem = kLogCap * (8 + 8) + kMaxK * (8 + 8);

// FP64 squared distance of each of the c candidates, in the operation order of
// the FP64 reference evaluation (ED: a thread per candidate; DTW: a warp).
__device__ __forceinline__ void fin_fp64(const IndexView &iv, const QueryParams &qp, const QuerySlot &slot,
                                         const unsigned long long *cand, double *d64, unsigned c)
{
    const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
    if (qp.dist == 0) {
        for (unsigned e = tid; e < c; e += blockDim.x) {
            const unsigned pos = iv.pos_of_id[cand_id(cand[e])];
            const float *x = iv.raw + (unsigned long long)pos * iv.len;
            double s = 0.0;
            for (int t = 0; t < iv.len; ++t) {
                const double d = __dsub_rn((double)slot.q[t], (double)x[t]);
                s = __dadd_rn(s, __dmul_rn(d, d));
            }
            d64[e] = s;
        }
    } else {
        double *diag = slot.dtw64 + (size_t)wib * 3 * iv.len;
        for (unsigned e = wib; e < c; e += blockDim.x >> 5) {
            const unsigned pos = iv.pos_of_id[cand_id(cand[e])];
            const double v = warp_dtw<double>(slot.q, iv.raw + (unsigned long long)pos * iv.len, iv.len, qp.r, diag,
                                              (double)f_inf());
            if (lane == 0) d64[e] = v;
            __syncwarp();
        }
    }
}

// Sort n (power of two) entries by (FP64 distance, id).
__device__ __forceinline__ void fin_sort64(unsigned long long *cand, double *d64, unsigned n)
{
    block_bitonic(
        n,
        [&](unsigned i, unsigned j) {
            return d64[i] < d64[j] || (d64[i] == d64[j] && cand_id(cand[i]) < cand_id(cand[j]));
        },
        [&](unsigned i, unsigned j) {
            const double td = d64[i];
            d64[i] = d64[j];
            d64[j] = td;
            const unsigned long long t = cand[i];
            cand[i] = cand[j];
            cand[j] = t;
        });
}

// More candidates in the band than one pass holds (a mass tie, e.g. many
// identical rows): the log is taken in windows of kLogCap entries; each
// window's in-band candidates are ranked in FP64 and merged with a running
// top-k, the same row never counted twice.  Exact for any band population.
__device__ void fin_streamed(const IndexView &iv, const QueryParams &qp, const QuerySlot &slot, float band,
                             unsigned nlog, unsigned long long *cand, double *d64, unsigned long long *rp, double *rd,
                             long long *ids, float *dists)
{
    __shared__ unsigned ncw, rc, wk;
    __shared__ unsigned long long seen;
    const int tid = threadIdx.x;
    const unsigned k = (unsigned)qp.k;
    if (tid == 0) {
        rc = 0;
        seen = 0;
    }
    __syncthreads();
    for (unsigned w0 = 0; w0 < nlog; w0 += kLogCap) {
        if (tid == 0) ncw = 0;
        __syncthreads();
        const unsigned w1 = min(nlog, w0 + (unsigned)kLogCap);
        for (unsigned i = w0 + tid; i < w1; i += blockDim.x) {
            const unsigned long long P = slot.log[i];
            if (cand_d2(P) <= band) cand[atomicAdd(&ncw, 1u)] = P;
        }
        __syncthreads();
        const unsigned c = ncw;
        if (tid == 0) seen += c;
        fin_fp64(iv, qp, slot, cand, d64, c);
        unsigned npow = 1;
        while (npow < c) npow <<= 1;
        for (unsigned i = c + tid; i < npow; i += blockDim.x) {
            cand[i] = kEmpty;
            d64[i] = (double)f_inf();
        }
        __syncthreads();
        fin_sort64(cand, d64, npow);
        // the window's best k distinct rows (a row logged twice has one FP64
        // distance, so it sorts next to itself whatever its FP32 keys: compare
        // ids with the last one kept), moved to the front in place
        if (tid == 0) {
            unsigned out = 0;
            for (unsigned i = 0; i < c && out < k; ++i) {
                if (out > 0 && cand_id(cand[i]) == cand_id(cand[out - 1])) continue;
                cand[out] = cand[i];
                d64[out] = d64[i];
                ++out;
            }
            wk = out;
        }
        __syncthreads();
        // then the running top-k, ranked together with them
        const unsigned m = wk, r0 = rc, tot = m + r0;
        for (unsigned i = tid; i < r0; i += blockDim.x) {
            cand[m + i] = rp[i];
            d64[m + i] = rd[i];
        }
        unsigned np2 = 1;
        while (np2 < tot) np2 <<= 1;
        for (unsigned i = tot + tid; i < np2; i += blockDim.x) {
            cand[i] = kEmpty;
            d64[i] = (double)f_inf();
        }
        __syncthreads();
        fin_sort64(cand, d64, np2);
        if (tid == 0) {
            unsigned out = 0;
            for (unsigned i = 0; i < tot && out < k; ++i) {
                if (i > 0 && cand_id(cand[i]) == cand_id(cand[i - 1])) continue;   // the same row logged twice
                rp[out] = cand[i];
                rd[out] = d64[i];
                ++out;
            }
            rc = out;
        }
        __syncthreads();
    }
    for (unsigned i = tid; i < k; i += blockDim.x) {
        ids[i] = i < rc ? (long long)cand_id(rp[i]) : -1;
        dists[i] = i < rc ? (float)sqrt(rd[i]) : f_inf();
    }
    if (tid == 0) slot.st->c.tie_rechecks += seen;
}

// redo (batched slots, may be null): instead of reporting a log overflow in the
// status word, mark the query so the caller answers it again on the per-query
// path, whose log cannot overflow.
__device__ __forceinline__ void finalize_body(const IndexView &iv, const QueryParams &qp, const QuerySlot &slot,
                                              long long *ids, float *dists, unsigned *redo = nullptr)
{
    extern __shared__ __align__(16) unsigned char fsm[];
    unsigned long long *cand = reinterpret_cast<unsigned long long *>(fsm);
    double *d64 = reinterpret_cast<double *>(fsm + kLogCap * 8);
    __shared__ unsigned ncand;
    __shared__ int ambiguous;
    QueryState *st = slot.st;
    const int tid = threadIdx.x;
    const unsigned k = (unsigned)qp.k;
    if (ld_volatile_u32(&st->invalid)) {
        for (unsigned i = tid; i < k; i += blockDim.x) {
            ids[i] = -1;
            dists[i] = __int_as_float(0x7fc00000);
        }
        return;
    }
    const unsigned long long T = st->thr;
    const float band = prune_threshold(T, qp.F);
    const unsigned logged = st->log_count;
    __shared__ int lost, many;
    if (tid == 0) {
        ncand = 0;
        ambiguous = 0;
        lost = logged > slot.log_cap;    // accepted candidates were dropped: cannot be exact
        many = 0;
    }
    __syncthreads();
    const unsigned nlog = min(logged, slot.log_cap);
    for (unsigned i = tid; i < nlog; i += blockDim.x) {
        const unsigned long long P = slot.log[i];
        if (cand_d2(P) <= band) {
            const unsigned o = atomicAdd(&ncand, 1u);
            if (o < (unsigned)kLogCap) cand[o] = P;
            else many = 1;
        }
    }
    __syncthreads();
    if (tid == 0) {
        if (redo) *redo = lost ? 1u : 0u;
        else if (lost) atomicOr(iv.status, kStTieOverflow);
    }
    if (many) {
        unsigned long long *rp = reinterpret_cast<unsigned long long *>(fsm + kLogCap * 16);
        double *rd = reinterpret_cast<double *>(fsm + kLogCap * 16 + kMaxK * 8);
        fin_streamed(iv, qp, slot, band, nlog, cand, d64, rp, rd, ids, dists);
        __syncthreads();
        QueryCounters *acc = slot.acc;
        if (tid == 0 && acc) {
            atomicAdd(&acc->lb_evaluated, st->c.lb_evaluated);
            atomicAdd(&acc->lb_survivors, st->c.lb_survivors);
            atomicAdd(&acc->lbk_survivors, st->c.lbk_survivors);
            atomicAdd(&acc->seeded, st->c.seeded);
            atomicAdd(&acc->refined, st->c.refined);
            atomicAdd(&acc->abandoned, st->c.abandoned);
            atomicAdd(&acc->bsf_updates, st->c.bsf_updates);
            atomicAdd(&acc->tie_rechecks, st->c.tie_rechecks);
            atomicAdd(&acc->leaves_live, st->c.leaves_live);
            atomicAdd(&acc->row_bytes, st->c.row_bytes);
            atomicAdd(&acc->dtw_cells, st->c.dtw_cells);
        }
        return;
    }
    const unsigned c = min(ncand, (unsigned)kLogCap);
    unsigned npow = 1;
    while (npow < c) npow <<= 1;
    for (unsigned i = c + tid; i < npow; i += blockDim.x) cand[i] = kEmpty;
    // the same row may have been offered more than once (screened batches
    // re-offer rows), possibly under two FP32 keys: ordered by (id, distance)
    // the entries of one row sit together, the smallest first; keep that one,
    // then order the rest by (distance, id)
    __shared__ unsigned nuniq;
    if (tid == 0) nuniq = 0;
    __syncthreads();
    auto by_id = [](unsigned long long P) { return (P << 32) | (P >> 32); };
    auto swap_cand = [&](unsigned i, unsigned j) {
        const unsigned long long t = cand[i];
        cand[i] = cand[j];
        cand[j] = t;
    };
    block_bitonic(npow, [&](unsigned i, unsigned j) { return by_id(cand[i]) < by_id(cand[j]); }, swap_cand);
    unsigned long long *mark = reinterpret_cast<unsigned long long *>(d64);
    for (unsigned i = tid; i < npow; i += blockDim.x)
        mark[i] = (i > 0 && i < c && cand_id(cand[i]) == cand_id(cand[i - 1])) ? 1ull : 0ull;
    __syncthreads();
    for (unsigned i = tid; i < npow; i += blockDim.x) {
        if (mark[i]) cand[i] = kEmpty;
        else if (i < c) atomicAdd(&nuniq, 1u);
    }
    __syncthreads();
    block_bitonic(npow, [&](unsigned i, unsigned j) { return cand[i] < cand[j]; }, swap_cand);
    const unsigned c_eff = nuniq;
    const unsigned cu = c_eff;
    // ambiguity: a candidate beyond the k-th inside the band, or two of the
    // first k within the band of each other (their order is not certain)
    if (tid == 0 && cu > k) ambiguous = 1;
    for (unsigned i = tid; i + 1 < min(cu, k); i += blockDim.x)
        if (cand_d2(cand[i + 1]) <= __fmul_ru(cand_d2(cand[i]), qp.F)) ambiguous = 1;
    __syncthreads();
    if (!ambiguous) {
        for (unsigned i = tid; i < k; i += blockDim.x) {
            ids[i] = i < cu ? (long long)cand_id(cand[i]) : -1;
            dists[i] = i < cu ? __fsqrt_rn(cand_d2(cand[i])) : f_inf();
        }
    } else {
        // FP64 recomputation of every candidate in the band, in the operation
        // order of the FP64 reference evaluation
        fin_fp64(iv, qp, slot, cand, d64, cu);
        for (unsigned i = cu + tid; i < npow; i += blockDim.x) d64[i] = (double)f_inf();
        __syncthreads();
        fin_sort64(cand, d64, npow);
        for (unsigned i = tid; i < k; i += blockDim.x) {
            ids[i] = i < cu ? (long long)cand_id(cand[i]) : -1;
            dists[i] = i < cu ? (float)sqrt(d64[i]) : f_inf();
        }
        if (tid == 0) st->c.tie_rechecks += cu;
    }
    __syncthreads();
    QueryCounters *acc = slot.acc;
    if (tid == 0 && acc) {
        atomicAdd(&acc->lb_evaluated, st->c.lb_evaluated);
        atomicAdd(&acc->lb_survivors, st->c.lb_survivors);
        atomicAdd(&acc->lbk_survivors, st->c.lbk_survivors);
        atomicAdd(&acc->seeded, st->c.seeded);
        atomicAdd(&acc->refined, st->c.refined);
        atomicAdd(&acc->abandoned, st->c.abandoned);
        atomicAdd(&acc->bsf_updates, st->c.bsf_updates);
        atomicAdd(&acc->tie_rechecks, st->c.tie_rechecks);
        atomicAdd(&acc->leaves_live, st->c.leaves_live);
        atomicAdd(&acc->row_bytes, st->c.row_bytes);
        atomicAdd(&acc->dtw_cells, st->c.dtw_cells);
    }
}

__global__ void __launch_bounds__(kFinThreads)
k_finalize(IndexView iv, QueryParams qp, QuerySlot slot, long long *ids, float *dists)
{
    finalize_body(iv, qp, slot, ids, dists);
}

__global__ void __launch_bounds__(kFinThreads)
k_finalize_batch(IndexView iv, QueryParams qp, const QuerySlot *__restrict__ slots, long long *ids, float *dists,
                 unsigned *redo)
{
    finalize_body(iv, qp, slots[blockIdx.x], ids + (size_t)blockIdx.x * qp.k, dists + (size_t)blockIdx.x * qp.k,
                  redo + blockIdx.x);
}

__global__ void __launch_bounds__(kFinThreads)
k_finalize_batch_args(IndexView iv, QueryParams qp, const QuerySlot *__restrict__ slots,
                      const BatchArgs *__restrict__ args, const unsigned *__restrict__ cursor)
{
    const BatchArgs a = args[*cursor];
    finalize_body(iv, qp, slots[blockIdx.x], a.ids + (size_t)blockIdx.x * qp.k, a.dists + (size_t)blockIdx.x * qp.k,
                  a.redo + blockIdx.x);
}

// Last node of a replayed batch: the next replay reads the next table entry.
__global__ void k_advance_cursor(unsigned *cursor) { *cursor += 1u; }

// lower bound of every series, written in original id order
__global__ void __launch_bounds__(256)
k_lb_all(IndexView iv, QuerySlot slot, float *__restrict__ out)
{
    __shared__ float lut[kMaxSegments * kMaxCard];
    for (int i = threadIdx.x; i < kMaxSegments * kMaxCard; i += blockDim.x) lut[i] = slot.lut[i];
    __syncthreads();
    if (ld_volatile_u32(&slot.st->invalid)) return;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long p = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; p < iv.N; p += stride)
        out[iv.ids[p]] = lb2_word(iv.sax[p], lut);
}

int dtw_warps_per_block(int len)
{
    const int per_warp = 3 * len * 4;
    int w = (96 * 1024 - len * 4) / per_warp;
    return std::max(1, std::min(8, w));
}

}  // namespace

float band_factor(int dist, int len)
{
    const double u = 5.9604644775390625e-08;   // 2^-24
    const double gamma = dist == 0 ? (len / 16.0 + 32.0) * u : (2.0 * len + 32.0) * u;
    const double F = (1.0 + gamma) * (1.0 + gamma) * (1.0 + 9.1e-13);
    return (float)F * (1.0f + 1.2e-7f);   // round up
}

void init_kernel_attributes()
{
    cudaFuncSetAttribute(k_lb_scan, cudaFuncAttributeMaxDynamicSharedMemorySize, kScanSmem);
    // three CTAs of 72 KB each per SM: ask for the largest shared-memory carveout
    cudaFuncSetAttribute(k_lb_scan, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    cudaFuncSetAttribute(k_finalize, cudaFuncAttributeMaxDynamicSharedMemorySize, kFinSmem);
    cudaFuncSetAttribute(k_finalize_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, kFinSmem);
    cudaFuncSetAttribute(k_finalize_batch_args, cudaFuncAttributeMaxDynamicSharedMemorySize, kFinSmem);
    cudaFuncSetAttribute(k_fused_ed, cudaFuncAttributeMaxDynamicSharedMemorySize, kFuSmemFixed + kMaxLen * 4);
    init_screen_attributes();
    cudaFuncSetAttribute(k_dtw, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
    cudaFuncSetAttribute(k_lbk, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_seed_dist<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
}

void launch_prep(const IndexView &iv, const QueryParams &qp, QuerySlot slot, const float *query,
                 cudaStream_t s)
{
    k_prep<<<1 + kMaxSegments, kPrepThreads, 0, s>>>(iv, qp, slot, query);
}

void launch_seed(const IndexView &iv, const QueryParams &qp, QuerySlot slot, cudaStream_t s,
                 unsigned long long *launches)
{
    if (qp.dist == 0) {
        const size_t sm = iv.len * 4;
        k_seed_dist<0><<<num_sms() * 2, 256, sm, s>>>(iv, qp, slot);
    } else if (!launch_dtw_thread<1>(iv, qp, slot, s)) {
        const int wpb = dtw_warps_per_block(iv.len);
        const size_t sm = (size_t)iv.len * 4 + (size_t)wpb * 3 * iv.len * 4;
        k_seed_dist<1><<<num_sms() * 4, wpb * 32, sm, s>>>(iv, qp, slot);
    }
    k_seed_select<<<1, kFinThreads, 0, s>>>(iv, qp, slot);
    if (launches) *launches += 2;
}

void launch_scan(const IndexView &iv, const QueryParams &qp, QuerySlot slot, unsigned epoch, cudaStream_t s)
{
    const unsigned long long ntiles = (iv.N + kScanTileWords - 1) / kScanTileWords;
    const unsigned long long lg = std::min<unsigned long long>((iv.L + 255) / 256, (unsigned long long)num_sms() * 8);
    k_leaf_prune<<<(unsigned)std::max(1ull, lg), 256, 0, s>>>(iv, qp, slot, epoch);
    const unsigned long long tg = std::min<unsigned long long>((ntiles + 255) / 256, (unsigned long long)num_sms() * 4);
    k_live_tiles<<<(unsigned)std::max(1ull, tg), 256, 0, s>>>(slot, ntiles, epoch);
    // the live tiles are shared out on the device; survivors of CTA c go to
    // region c of ceil(live / grid) tiles, which the survivor arrays hold
    // for any live count (they have room for ntiles + kMaxScanGrid tiles)
    unsigned long long g = std::min<unsigned long long>(ntiles, (unsigned long long)num_sms() * kScanCtasPerSm);
    g = std::min<unsigned long long>(g, kMaxScanGrid);
    k_lb_scan<<<(unsigned)std::max(1ull, g), kScanThreads, kScanSmem, s>>>(iv, qp, slot);
}

void launch_refine(const IndexView &iv, const QueryParams &qp, QuerySlot slot, cudaStream_t s,
                   unsigned long long *launches, cudaEvent_t ev0, cudaEvent_t ev1)
{
    if (qp.dist == 0) {
        if (ev0) cudaEventRecord(ev0, s);
        k_refine_ed<<<num_sms() * 3, kRefineThreads, iv.len * 4, s>>>(iv, qp, slot);   // one wave: 3 blocks per SM
        if (ev1) cudaEventRecord(ev1, s);
        if (launches) *launches += 1;
    } else {
        if (!launch_lbk_thread(iv, qp, slot, s)) {
            // windows wider than the register forms: warp per candidate, per
            // warp 4 rows of len floats (row / extrema), plus the query and its envelope
            const int wpb = std::max(1, std::min(8, (int)((96 * 1024 - 12 * iv.len) / (16 * iv.len))));
            k_lbk<<<num_sms() * 4, wpb * 32, (size_t)iv.len * 12 + (size_t)wpb * 16 * iv.len, s>>>(iv, qp, slot, wpb);
        }
        launch_order(qp, slot, 1, slot.surv_pos, slot.surv_lb, s);
        if (ev0) cudaEventRecord(ev0, s);
        if (!launch_dtw_thread<0>(iv, qp, slot, s)) {
            const int wpb = dtw_warps_per_block(iv.len);
            const size_t sm = (size_t)iv.len * 4 + (size_t)wpb * 3 * iv.len * 4;
            k_dtw<<<num_sms() * 4, wpb * 32, sm, s>>>(iv, qp, slot);
        }
        if (ev1) cudaEventRecord(ev1, s);
        if (launches) *launches += 5;
    }
}

void launch_finalize(const IndexView &iv, const QueryParams &qp, QuerySlot slot, long long *ids,
                     float *dists, cudaStream_t s)
{
    k_finalize<<<1, kFinThreads, kFinSmem, s>>>(iv, qp, slot, ids, dists);
}

void launch_batch(const IndexView &iv, const QueryParams &qp, const QuerySlot *slots_dev, unsigned B,
                  const float *queries, long long *ids, float *dists, unsigned *redo, unsigned chunk_tiles,
                  unsigned ctas_per_sm, unsigned *counter, cudaStream_t s, unsigned long long *launches,
                  cudaEvent_t ev0, cudaEvent_t ev1)
{
    k_prep_batch<<<B, kPrepThreads, 0, s>>>(iv, qp, slots_dev, queries);
    k_seed_dist_batch<0><<<dim3(8, B), 256, iv.len * 4, s>>>(iv, qp, slots_dev);
    k_seed_select_batch<<<B, kFinThreads, 0, s>>>(iv, qp, slots_dev);
    cudaMemsetAsync(counter, 0, 4, s);
    const size_t sm = kFuSmemFixed + (size_t)iv.len * 4;
    if (ev0) cudaEventRecord(ev0, s);
    k_fused_ed<<<num_sms() * ctas_per_sm, kFuThreads, sm, s>>>(iv, qp, slots_dev, B, chunk_tiles, counter);
    if (ev1) cudaEventRecord(ev1, s);
    k_finalize_batch<<<B, kFinThreads, kFinSmem, s>>>(iv, qp, slots_dev, ids, dists, redo);
    if (launches) *launches += 5;
}

void launch_batch_args(const IndexView &iv, const QueryParams &qp, const QuerySlot *slots_dev, unsigned B,
                       const BatchArgs *args, unsigned *cursor, unsigned chunk_tiles, unsigned ctas_per_sm,
                       unsigned *counter, cudaStream_t s)
{
    k_prep_batch_args<<<B, kPrepThreads, 0, s>>>(iv, qp, slots_dev, args, cursor);
    k_seed_dist_batch<0><<<dim3(8, B), 256, iv.len * 4, s>>>(iv, qp, slots_dev);
    k_seed_select_batch<<<B, kFinThreads, 0, s>>>(iv, qp, slots_dev);
    cudaMemsetAsync(counter, 0, 4, s);
    const size_t sm = kFuSmemFixed + (size_t)iv.len * 4;
    k_fused_ed<<<num_sms() * ctas_per_sm, kFuThreads, sm, s>>>(iv, qp, slots_dev, B, chunk_tiles, counter);
    k_finalize_batch_args<<<B, kFinThreads, kFinSmem, s>>>(iv, qp, slots_dev, args, cursor);
    k_advance_cursor<<<1, 1, 0, s>>>(cursor);
}

void launch_batch_seed(const IndexView &iv, const QueryParams &qp, const QuerySlot *slots_dev, unsigned B,
                       const float *queries, cudaStream_t s, unsigned long long *launches)
{
    k_prep_batch<<<B, kPrepThreads, 0, s>>>(iv, qp, slots_dev, queries);
    k_seed_dist_batch<0><<<dim3(8, B), 256, iv.len * 4, s>>>(iv, qp, slots_dev);
    k_seed_select_batch<<<B, kFinThreads, 0, s>>>(iv, qp, slots_dev);
    if (launches) *launches += 3;
}

void launch_batch_finalize(const IndexView &iv, const QueryParams &qp, const QuerySlot *slots_dev, unsigned B,
                           long long *ids, float *dists, unsigned *redo, cudaStream_t s, unsigned long long *launches)
{
    k_finalize_batch<<<B, kFinThreads, kFinSmem, s>>>(iv, qp, slots_dev, ids, dists, redo);
    if (launches) *launches += 1;
}

struct CounterSrcs {
    const QueryCounters *p[kDtwStreams];
};

__global__ void k_add_counters(QueryCounters *dst, CounterSrcs src, int n)
{
    if (threadIdx.x != 0) return;
    QueryCounters t{};
    for (int i = 0; i < n; ++i) {
        const QueryCounters &c = *src.p[i];
        t.lb_evaluated += c.lb_evaluated;
        t.lb_survivors += c.lb_survivors;
        t.lbk_survivors += c.lbk_survivors;
        t.seeded += c.seeded;
        t.refined += c.refined;
        t.abandoned += c.abandoned;
        t.bsf_updates += c.bsf_updates;
        t.tie_rechecks += c.tie_rechecks;
        t.leaves_live += c.leaves_live;
        t.row_bytes += c.row_bytes;
        t.dtw_cells += c.dtw_cells;
    }
    *dst = t;
}

void launch_add_counters(QueryCounters *dst, const QueryCounters *const *src, int n, cudaStream_t s)
{
    CounterSrcs cs{};
    for (int i = 0; i < n && i < kDtwStreams; ++i) cs.p[i] = src[i];
    k_add_counters<<<1, 32, 0, s>>>(dst, cs, std::min(n, kDtwStreams));
}

void launch_lower_bounds(const IndexView &iv, QuerySlot slot, float *lb2_by_id, cudaStream_t s)
{
    k_lb_all<<<num_sms() * 4, 256, 0, s>>>(iv, slot, lb2_by_id);
}

}  // namespace messi
