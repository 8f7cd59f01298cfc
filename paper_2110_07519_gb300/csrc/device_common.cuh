// device_common.cuh -- device helpers shared by the query kernels: packed
// best-so-far handling, PTX wrappers for mbarrier / bulk copies with bounded
// waits, warp reductions, the iSAX lower bound of one word, and the ED / DTW
// distance routines.
#pragma once

#include "messi_internal.cuh"

namespace messi {

__device__ __forceinline__ float f_inf() { return __int_as_float(0x7f800000); }

__device__ __forceinline__ unsigned long long pack_cand(float d2, unsigned id)
{
    return ((unsigned long long)__float_as_uint(d2) << 32) | id;
}
__device__ __forceinline__ float cand_d2(unsigned long long p) { return __uint_as_float((unsigned)(p >> 32)); }
__device__ __forceinline__ unsigned cand_id(unsigned long long p) { return (unsigned)p; }

__device__ __forceinline__ unsigned long long ld_volatile_u64(const unsigned long long *p)
{
    return *reinterpret_cast<const volatile unsigned long long *>(p);
}
__device__ __forceinline__ unsigned ld_volatile_u32(const unsigned *p)
{
    return *reinterpret_cast<const volatile unsigned *>(p);
}

// Pruning threshold from a packed k-th best: its squared distance widened by
// the near-tie factor, rounded up (+inf while fewer than k candidates exist).
__device__ __forceinline__ float prune_threshold(unsigned long long T, float F)
{
    return T == kEmpty ? f_inf() : __fmul_ru(cand_d2(T), F);
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}
__device__ __forceinline__ float warp_min(float v)
{
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, off));
    return v;
}

// Hint: bring the 128-byte line holding p into L1 (no effect on results; an
// address inside an allocation is required, as for a load).
__device__ __forceinline__ void prefetch_l1(const void *p)
{
    asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// ---------------------------------------------------------------- PTX: TMA
__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_barrier_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// 1-D bulk copy global -> shared through the TMA unit; completes `bytes`
// transaction bytes on `bar`.  Addresses 16-byte aligned, size a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: false when the phase did not complete within the limit.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, unsigned parity)
{
    for (unsigned it = 0; it < kSpinLimit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
// Non-blocking probe of a phase.
__device__ __forceinline__ bool mbar_test_wait(unsigned long long *bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for a thread that also issues tensor-core work: try_wait can
// hold the issuing thread for hundreds of cycles even on a completed phase,
// so the phase is probed with test_wait first and try_wait only takes over
// for long waits.
__device__ __forceinline__ bool mbar_wait_issuer(unsigned long long *bar, unsigned parity)
{
    for (unsigned it = 0; it < 4096; ++it)
        if (mbar_test_wait(bar, parity)) return true;
    return mbar_wait_bounded(bar, parity);
}

// ------------------------------------------------------ iSAX lower bound
// Squared lower bound of one iSAX word: sum over segments of the table entry
// of its symbol, added with rounding toward -inf so the result never exceeds
// the exact sum of the (already rounded-down) entries.  lb2_half adds the 8
// segments held in two 32-bit words starting at segment s0 to acc; a partial
// sum never exceeds the full one, so a partial sum above a threshold already
// rejects the word.
__device__ __forceinline__ float lb2_half(unsigned w0, unsigned w1, const float *lut, int s0, float acc)
{
    float v[8];
#pragma unroll
    for (int b = 0; b < 4; ++b) v[b] = lut[(s0 + b) * kMaxCard + ((w0 >> (8 * b)) & 0xffu)];
#pragma unroll
    for (int b = 0; b < 4; ++b) v[4 + b] = lut[(s0 + 4 + b) * kMaxCard + ((w1 >> (8 * b)) & 0xffu)];
#pragma unroll
    for (int b = 0; b < 8; ++b) acc = __fadd_rd(acc, v[b]);
    return acc;
}

__device__ __forceinline__ float lb2_word(const uint4 &wv, const float *lut)
{
    return lb2_half(wv.z, wv.w, lut, 8, lb2_half(wv.x, wv.y, lut, 0, 0.f));
}

// ------------------------------------------------------------------- ED
// Squared ED of query q (len floats, 16-byte aligned) and row x, one warp.
// Lanes take float4 i = lane, lane + 32, ...; chunks of 256 points are summed
// in order and, when `thr` is finite, the warp stops after a chunk whose
// running sum exceeds thr (returns that partial sum, > thr).  All lanes
// return the same value.
__device__ __forceinline__ float warp_ed2(const float *__restrict__ q, const float *__restrict__ x, int len,
                                          float thr)
{
    const int lane = threadIdx.x & 31;
    const int n4 = len >> 2;
    const float4 *q4 = reinterpret_cast<const float4 *>(q);
    const float4 *x4 = reinterpret_cast<const float4 *>(x);
    float acc = 0.f;
    for (int base = 0; base < n4; base += 64) {
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const int i = base + lane + 32 * t;
            if (i < n4) {
                const float4 xv = __ldg(x4 + i);
                const float4 qv = q4[i];
                float d;
                d = qv.x - xv.x; acc = fmaf(d, d, acc);
                d = qv.y - xv.y; acc = fmaf(d, d, acc);
                d = qv.z - xv.z; acc = fmaf(d, d, acc);
                d = qv.w - xv.w; acc = fmaf(d, d, acc);
            }
        }
        if (base + 64 < n4 && thr < f_inf()) {
            const float part = warp_sum(acc);
            if (part > thr) return part;
        }
    }
    return warp_sum(acc);
}

// Two rows at once (more loads in flight); same arithmetic as warp_ed2 for
// each row.  A row whose running sum exceeds thr after a 256-point chunk
// stops accumulating; its returned value is then that partial sum (> thr).
// na / nb receive the points of each row read (whole 256-point chunks
// loaded while the row was still live; len when it ran to the end).
__device__ __forceinline__ void warp_ed2_pair(const float *__restrict__ q, const float *__restrict__ xa,
                                              const float *__restrict__ xb, int len, float thr, float &da,
                                              float &db, int &na, int &nb)
{
    na = 0;
    nb = 0;
    const int lane = threadIdx.x & 31;
    const int n4 = len >> 2;
    const float4 *q4 = reinterpret_cast<const float4 *>(q);
    const float4 *a4 = reinterpret_cast<const float4 *>(xa);
    const float4 *b4 = reinterpret_cast<const float4 *>(xb);
    float aa = 0.f, ab = 0.f;
    bool live_a = true, live_b = true;
    for (int base = 0; base < n4; base += 64) {
        const int pts = min(256, 4 * (n4 - base));
        if (live_a) na += pts;
        if (live_b) nb += pts;
        float4 xv[4];
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const int i = base + lane + 32 * t;
            const bool in = i < n4;
            xv[t] = (in && live_a) ? __ldg(a4 + i) : make_float4(0.f, 0.f, 0.f, 0.f);
            xv[2 + t] = (in && live_b) ? __ldg(b4 + i) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const int i = base + lane + 32 * t;
            if (i < n4) {
                const float4 qv = q4[i];
                float d;
                if (live_a) {
                    d = qv.x - xv[t].x; aa = fmaf(d, d, aa);
                    d = qv.y - xv[t].y; aa = fmaf(d, d, aa);
                    d = qv.z - xv[t].z; aa = fmaf(d, d, aa);
                    d = qv.w - xv[t].w; aa = fmaf(d, d, aa);
                }
                if (live_b) {
                    d = qv.x - xv[2 + t].x; ab = fmaf(d, d, ab);
                    d = qv.y - xv[2 + t].y; ab = fmaf(d, d, ab);
                    d = qv.z - xv[2 + t].z; ab = fmaf(d, d, ab);
                    d = qv.w - xv[2 + t].w; ab = fmaf(d, d, ab);
                }
            }
        }
        if (base + 64 < n4 && thr < f_inf()) {
            if (live_a && warp_sum(aa) > thr) live_a = false;
            if (live_b && warp_sum(ab) > thr) live_b = false;
            if (!live_a && !live_b) break;
        }
    }
    da = warp_sum(aa);
    db = warp_sum(ab);
}

// R rows at once (R row loads in flight per lane); same arithmetic as
// warp_ed2 for each row.  A row with live[r] false on entry is not read (its
// d[r] and n[r] are 0 and mean nothing).  A row whose running sum exceeds
// thr after a 256-point chunk stops; d[r] is then that partial sum (> thr).
// n[r] receives the points of row r read (whole 256-point chunks loaded
// while it was live).
template <int R>
__device__ __forceinline__ void warp_ed2_rows(const float *__restrict__ q, const float *const (&x)[R], bool (&live)[R],
                                              int len, float thr, float (&d)[R], int (&n)[R])
{
    const int lane = threadIdx.x & 31;
    const int n4 = len >> 2;
    const float4 *q4 = reinterpret_cast<const float4 *>(q);
    float acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        acc[r] = 0.f;
        n[r] = 0;
    }
    for (int base = 0; base < n4; base += 64) {
        const int pts = min(256, 4 * (n4 - base));
        float4 xv[R][2];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (live[r]) n[r] += pts;
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                const int i = base + lane + 32 * t;
                xv[r][t] = (live[r] && i < n4) ? __ldg(reinterpret_cast<const float4 *>(x[r]) + i)
                                               : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const int i = base + lane + 32 * t;
            if (i < n4) {
                const float4 qv = q4[i];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    float e;
                    e = qv.x - xv[r][t].x; acc[r] = fmaf(e, e, acc[r]);
                    e = qv.y - xv[r][t].y; acc[r] = fmaf(e, e, acc[r]);
                    e = qv.z - xv[r][t].z; acc[r] = fmaf(e, e, acc[r]);
                    e = qv.w - xv[r][t].w; acc[r] = fmaf(e, e, acc[r]);
                }
            }
        }
        if (base + 64 < n4 && thr < f_inf()) {
            bool any = false;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (live[r] && warp_sum(acc[r]) > thr) live[r] = false;
                any = any || live[r];
            }
            if (!any) break;
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) d[r] = warp_sum(acc[r]);
}

// ------------------------------------------------------------------ DTW
// Banded DTW of q and x (length n, reach r) by one warp, anti-diagonal
// wavefront: cells (i, j) with i + j = a are independent; lane handles
// i = i_lo + lane, +32, ...  `diag` holds three diagonals (3*n values,
// indexed by i).  A cell's neighbours are read only when they lie inside the
// window and the matrix, so no diagonal needs clearing.  Every warping path
// meets diagonal a or a+1, so when the minimum over two consecutive
// diagonals exceeds `thr` the result would too and the warp stops early
// (returning a value > thr).  FP32 uses fminf / plain adds; the FP64
// instantiation uses explicitly rounded operations in the same order as the
// FP64 reference evaluation of the recurrence.
template <typename T>
__device__ __forceinline__ T dtw_cost(float qi, float xj);
template <>
__device__ __forceinline__ float dtw_cost<float>(float qi, float xj)
{
    const float d = qi - xj;
    return d * d;
}
template <>
__device__ __forceinline__ double dtw_cost<double>(float qi, float xj)
{
    const double d = __dsub_rn((double)qi, (double)xj);
    return __dmul_rn(d, d);
}
__device__ __forceinline__ float dtw_add(float a, float b) { return a + b; }
__device__ __forceinline__ double dtw_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float dtw_min(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double dtw_min(double a, double b) { return fmin(a, b); }

template <typename T>
__device__ T warp_dtw(const float *__restrict__ q, const float *__restrict__ x, int n, int r, T *diag, T thr)
{
    const int lane = threadIdx.x & 31;
    const T INF = (T)f_inf();
    if (r > n - 1) r = n - 1;
    T run_min = INF;      // min over the current diagonal (this lane)
    T prev_min = INF;     // min over the previous diagonal (this lane)
    const int last = 2 * n - 2;
    for (int a = 0; a <= last; ++a) {
        int i_lo = a - (n - 1);
        const int wlo = (a - r + 1) >> 1;                     // ceil((a - r) / 2)
        if (wlo > i_lo) i_lo = wlo;
        if (i_lo < 0) i_lo = 0;
        int i_hi = (a + r) >> 1;                              // floor((a + r) / 2)
        if (i_hi > a) i_hi = a;
        if (i_hi > n - 1) i_hi = n - 1;
        T *cur = diag + (a % 3) * n;
        const T *p1 = diag + ((a + 2) % 3) * n;
        const T *p2 = diag + ((a + 1) % 3) * n;
        T lmin = INF;
        for (int i = i_lo + lane; i <= i_hi; i += 32) {
            const int j = a - i;
            const T cost = dtw_cost<T>(q[i], x[j]);
            T D;
            if (a == 0) {
                D = cost;
            } else {
                T best = INF;
                if (i >= 1 && abs(i - 1 - j) <= r) best = dtw_min(best, p1[i - 1]);
                if (j >= 1 && abs(i - j + 1) <= r) best = dtw_min(best, p1[i]);
                if (i >= 1 && j >= 1) best = dtw_min(best, p2[i - 1]);
                D = dtw_add(cost, best);
            }
            cur[i] = D;
            lmin = dtw_min(lmin, D);
        }
        __syncwarp();
        prev_min = run_min;
        run_min = lmin;
        if ((a & 7) == 7 && a < last && thr < INF) {
            T both = dtw_min(prev_min, run_min);
#pragma unroll
            for (int off = 16; off >= 1; off >>= 1) both = dtw_min(both, __shfl_xor_sync(0xffffffffu, both, off));
            if (both > thr) return both;
        }
    }
    return diag[(last % 3) * n + (n - 1)];
}

// Survivors are stored in per-scan-CTA regions; a refine block turns the
// region counts into a prefix over chunks of 2^shift entries (default 32) so
// warps can take chunks by index.  Returns the number of chunks.
__device__ __forceinline__ unsigned chunk_prefix(const QuerySlot &slot, unsigned G, unsigned *prefix, unsigned *counts,
                                                 int shift = 5)
{
    __shared__ unsigned part[32];
    const unsigned per = (G + blockDim.x - 1) / blockDim.x;
    const unsigned lo = threadIdx.x * per, hi = min(lo + per, G);
    unsigned sum = 0;
    for (unsigned c = lo; c < hi; ++c) {
        const unsigned n = slot.region_count[c];
        counts[c] = n;
        sum += (n + (1u << shift) - 1u) >> shift;
    }
    // block-wide exclusive scan of the per-thread sums
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned inc = sum;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc += y;
    }
    if (lane == 31) part[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        unsigned v = lane < nw ? part[lane] : 0u;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, v, off);
            if (lane >= off) v += y;
        }
        if (lane < nw) part[lane] = v;
    }
    __syncthreads();
    unsigned run = (warp ? part[warp - 1] : 0u) + inc - sum;
    for (unsigned c = lo; c < hi; ++c) {
        prefix[c] = run;
        run += (counts[c] + (1u << shift) - 1u) >> shift;
    }
    if (threadIdx.x == blockDim.x - 1) prefix[G] = run;
    __syncthreads();
    return prefix[G];
}

// region holding chunk `ch`: the last c with prefix[c] <= ch
__device__ __forceinline__ unsigned region_of(unsigned ch, const unsigned *prefix, unsigned G)
{
    unsigned lo = 0, hi = G;
    while (hi - lo > 1) {
        const unsigned mid = (lo + hi) >> 1;
        if (prefix[mid] <= ch) lo = mid; else hi = mid;
    }
    return lo;
}

// ------------------------------------------------------- bound ordering
// Bucket of a non-negative FP32 lower bound: its exponent and top 4 mantissa
// bits, monotone in the bound.  order_floor(b) is the smallest bound in b.
__device__ __forceinline__ unsigned order_bucket(float lb) { return (__float_as_uint(lb) & 0x7fffffffu) >> 19; }
__device__ __forceinline__ float order_floor(unsigned b) { return __uint_as_float(b << 19); }

// ------------------------------------------------------------------ offer
// Present a computed candidate (squared FP32 distance, original id) to a
// query's best-so-far.  Candidates within the near-tie band of the current
// k-th best are logged for the final FP64 resolution.  k = 1 keeps the best
// as a packed 64-bit atomicMin; k > 1 inserts into a sorted k-array under a
// lock with a bounded spin (qp.lock_spin tries; a waiter that runs out sets
// the timeout bit of the status word and drops the candidate, so the query
// reports MESSI_ETIMEOUT).  Offering the same row twice changes nothing
// (its packed value is already in the array or no longer qualifies); the
// log may then hold it twice, which the final step removes.
static __device__ __noinline__ void offer(const QueryParams &qp, const QuerySlot &slot, unsigned *status, float d2,
                                   unsigned id)
{
    QueryState *st = slot.st;
    const unsigned long long P = pack_cand(d2, id);
    const unsigned long long T = ld_volatile_u64(&st->thr);
    if (!(d2 <= prune_threshold(T, qp.F))) return;
    const unsigned li = atomicAdd(&st->log_count, 1u);
    if (li < slot.log_cap) slot.log[li] = P;
    if (P >= T) return;
    if (qp.k == 1) {
        const unsigned long long old = atomicMin(&st->thr, P);
        if (P < old) atomicAdd(&st->c.bsf_updates, 1ull);
        return;
    }
    // many threads can finish candidates at once (one candidate per thread):
    // a waiter leaves as soon as the k-th best it would displace has dropped
    // below it, and backs off exponentially so the holder's release is not
    // queued behind a storm of failed exchanges
    unsigned spins = 0, nap = 32;
    while (atomicCAS(&st->lock, 0u, 1u) != 0u) {
        if (P >= ld_volatile_u64(&st->thr)) return;
        if (++spins > qp.lock_spin) {
            atomicOr(status, kStTimeout);
            return;
        }
        __nanosleep(nap);
        if (nap < 2048) nap <<= 1;
    }
    __threadfence();
    volatile unsigned long long *ka = slot.karr;
    volatile unsigned *kc = &st->kcount;
    const unsigned cnt = *kc;
    const unsigned k = (unsigned)qp.k;
    bool present = false;
    for (unsigned i = 0; i < cnt && !present; ++i) present = ka[i] == P;
    if (!present && (cnt < k || P < ka[k - 1])) {
        int pos = cnt < k ? (int)cnt : (int)k - 1;
        if (cnt < k) *kc = cnt + 1;
        while (pos > 0 && ka[pos - 1] > P) {
            ka[pos] = ka[pos - 1];
            --pos;
        }
        ka[pos] = P;
        if (cnt + 1 >= k) {
            atomicExch(&st->thr, ka[k - 1]);
            atomicAdd(&st->c.bsf_updates, 1ull);
        }
    }
    __threadfence();
    atomicExch(&st->lock, 0u);
}

}  // namespace messi
