// screen.cu -- tensor-core screening of a query batch (no counterpart in the
// paper, which answers one query at a time).
//
// For a batch of queries, squared ED is estimated for every (series, query)
// pair as  s = |x|^2 + |q|^2 - 2 q.x  with the dot products from tcgen05 MMAs
// on f16 copies of both (FP32 accumulation in TMEM).  Each estimate is
// widened by a rigorous bound eps(x, q) on its error:
//   |q.x - c| <= (2^-10 + (len + 16) 2^-23) 1.002 |q||x|
//               + 2^-24 sqrt(len) 1.002 (|q| + |x|)          (f16 rounding of
//                 both operands incl. subnormals, FP32 accumulation)
//   plus 4u (|x|^2 + |q|^2 + 2|q||x|) for the FP32 evaluation of s and the
//   FP32 rounding of the norms (computed in FP64).
// so s - eps <= true d^2 <= s + eps.  A pair is a candidate when
// s - eps <= U_q, U_q an upper bound of the query's true k-th squared
// distance; for k = 1 every s + eps also tightens U_q.  Candidates are then
// recomputed exactly in FP32 and offered to the query's best-so-far, and the
// usual FP64 near-tie resolution finishes the query.  A query whose candidate
// list overflows is screened again with its tightened bound.
//
// Operand tiles (see tc.cuh): rows of the collection are copied once to f16 in
// 128-row tiles already in the tensor-core layout, so one bulk copy loads a
// tile; queries are laid out the same way, 128 per tile.
#include <cuda_fp16.h>

#include <algorithm>

#include "tc.cuh"

namespace messi {
namespace {

constexpr int kTcRows = 128;        // M: series per tile
constexpr int kTcQ = 128;           // N: queries per tile
constexpr float kKappa = 2.4e-7f;   // 4u: FP32 evaluation of s and rounding of the norms
constexpr float kKappaP = 7.2e-7f;  // 12u: kappa plus the rounding of the rearranged test
constexpr int kTcMaxLen = 256;      // query tiles of 128 x len halves stay resident in shared memory
constexpr int kTcMaxStages = 16;
constexpr size_t kTcSmemBudget = 216 * 1024;   // dynamic shared memory of one screen CTA

// K width of one streamed chunk of a series tile: the largest of 64, 32, 16
// dividing len.  A tile is stored chunk-major: chunk c (k in [c*ck, c*ck+ck))
// is a 128 x ck operand in the tensor-core layout.
__host__ __device__ __forceinline__ unsigned chunk_k(unsigned len)
{
    return (len % 64 == 0) ? 64u : (len % 32 == 0) ? 32u : 16u;
}

__device__ __forceinline__ float tc_coef(int len)
{
    return 1.002f * (9.765625e-4f + (float)(len + 16) * 1.1920929e-7f);
}

// ------------------------------------------------------- screen copy
// One warp per series: f16 copy in tile layout, FP64 squared norm -> xn (FP32,
// nearest) and |x| rounded up.
__global__ void __launch_bounds__(256)
k_make_screen_copy(const float *__restrict__ raw, unsigned long long N, int len, __half *__restrict__ tiles,
                   float *__restrict__ xn, float *__restrict__ xnorm, unsigned *__restrict__ bad)
{
    const int lane = threadIdx.x & 31;
    const unsigned long long nw = (unsigned long long)gridDim.x * (blockDim.x >> 5);
    const unsigned long long ntile_rows = ((N + kTcRows - 1) / kTcRows) * kTcRows;
    for (unsigned long long row = (unsigned long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
         row < ntile_rows; row += nw) {
        const unsigned long long tile = row / kTcRows;
        const unsigned r = (unsigned)(row % kTcRows);
        unsigned char *tbase = reinterpret_cast<unsigned char *>(tiles) + tile * (unsigned long long)kTcRows * len * 2;
        double ss = 0.0;
        for (int k0 = lane * 8; k0 < len; k0 += 256) {
            float v[8];
            if (row < N) {
                const float4 *src = reinterpret_cast<const float4 *>(raw + row * (unsigned long long)len + k0);
                const float4 a = __ldg(src), b = __ldg(src + 1);
                v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
            } else {
#pragma unroll
                for (int i = 0; i < 8; ++i) v[i] = 0.f;
            }
            __align__(16) __half h[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                if (fabsf(v[i]) > 65000.f) atomicOr(bad, 1u);
                h[i] = __float2half_rn(v[i]);
                ss = __dadd_rn(ss, __dmul_rn((double)v[i], (double)v[i]));
            }
            const unsigned ck = chunk_k(len);
            *reinterpret_cast<uint4 *>(tbase + (unsigned)(k0 / ck) * (kTcRows * ck * 2) +
                                       tc_offset(r, (unsigned)(k0 % ck), ck)) = *reinterpret_cast<uint4 *>(h);
        }
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, off);
        if (lane == 0) {
            xn[row] = (float)ss;
            xnorm[row] = __double2float_ru(sqrt(ss * (1.0 + 1e-12)));
        }
    }
}

// ------------------------------------------------------- query prep
// One block per query: f16 copy into its query tile, |q|^2 and |q|, the
// per-query epilogue constants and the initial bound U_q from the seed.
__global__ void __launch_bounds__(256)
k_tc_qprep(const QuerySlot *__restrict__ slots, unsigned B, int len, QueryParams qp, __half *__restrict__ qtiles,
           float *__restrict__ qconst, unsigned *__restrict__ Ubits, unsigned *__restrict__ cand_count,
           unsigned *__restrict__ flags, unsigned *__restrict__ active)
{
    __shared__ double part[8];
    const unsigned b = blockIdx.x;        // padded up to a multiple of kTcQ
    const unsigned tile = b / kTcQ, r = b % kTcQ;
    unsigned char *tbase = reinterpret_cast<unsigned char *>(qtiles) + (unsigned long long)tile * kTcQ * len * 2;
    const bool real = b < B;
    const float *q = real ? slots[b].q : nullptr;
    double ss = 0.0;
    bool big = false;
    for (int k0 = threadIdx.x * 8; k0 < len; k0 += blockDim.x * 8) {
        __align__(16) __half h[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const float v = real ? q[k0 + i] : 0.f;
            big |= !(fabsf(v) <= 65000.f);
            h[i] = __float2half_rn(v);
            ss = __dadd_rn(ss, __dmul_rn((double)v, (double)v));
        }
        *reinterpret_cast<uint4 *>(tbase + tc_offset(r, (unsigned)k0, (unsigned)len)) = *reinterpret_cast<uint4 *>(h);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, off);
    big = __any_sync(0xffffffffu, big);
    if (lane == 0) part[warp] = ss;
    __shared__ int sbig;
    if (threadIdx.x == 0) sbig = 0;
    __syncthreads();
    if (big) sbig = 1;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
        const float qn = (float)t;
        const float qnorm = __double2float_ru(sqrt(t * (1.0 + 1e-12)));
        const float beta = 5.9604645e-8f * sqrtf((float)len) * 1.002f;
        const float alpha = (qnorm * (2.f * tc_coef(len) + 2.f * kKappaP) + beta) * (1.f + 1e-6f);
        const float gamma = (beta * qnorm + kKappaP * qn) * (1.f + 1e-6f);
        qconst[4 * b + 0] = qn;
        qconst[4 * b + 1] = alpha;
        qconst[4 * b + 2] = gamma;
        qconst[4 * b + 3] = 0.f;
        unsigned f = 0;
        float U = -1.f;                  // padded or unusable query: no candidates
        if (real) {
            QueryState *st = slots[b].st;
            if (ld_volatile_u32(&st->invalid)) f |= 2u;
            else if (sbig) f |= 4u;      // outside f16 range: answered by the per-query path
            else U = prune_threshold(ld_volatile_u64(&st->thr), qp.F);
        }
        Ubits[b] = __float_as_uint(U);
        cand_count[b] = 0;
        flags[b] = f;
        active[b] = (real && f == 0) ? 1u : 0u;
    }
}

// Between passes: a query whose candidate list overflowed is screened again
// with its bound tightened by the rechecked candidates; the others stop.
__global__ void k_tc_next_pass(const QuerySlot *__restrict__ slots, unsigned B, QueryParams qp, unsigned cap,
                               unsigned *__restrict__ Ubits, unsigned *__restrict__ cand_count,
                               unsigned *__restrict__ active, unsigned *__restrict__ n_active)
{
    const unsigned b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    if (active[b] && cand_count[b] > cap) {
        const float U = prune_threshold(ld_volatile_u64(&slots[b].st->thr), qp.F);
        if (U < __uint_as_float(Ubits[b])) Ubits[b] = __float_as_uint(U);
        cand_count[b] = 0;
        atomicAdd(n_active, 1u);
    } else {
        active[b] = 0;
    }
}

// ------------------------------------------------------------ screen
struct ScreenArgs {
    const __half *rtiles;     // [RT][128 x len] f16 rows
    const float *xn, *xnorm;  // [RT * 128]
    const unsigned *ids_unused;
    const __half *qtiles;     // [QT][128 x len] f16 queries
    const float *qconst;      // [QT*128][4]
    unsigned *Ubits;          // [QT*128] float bits, atomically lowered (k = 1)
    unsigned *cand_count;     // [QT*128]
    unsigned *cand_pos;       // [QT*128][cap]
    const unsigned *active;   // [QT*128]: nonzero when the query collects candidates this pass
    unsigned cap;
    unsigned qpc;             // query tiles per CTA (1 or 2)
    unsigned stages;          // chunk stages of the ring
    unsigned long long N;
    unsigned len;
    unsigned QT;
    int k;
    unsigned *status;
};

// Operand roles: A = a query tile (M = 128 queries, TMEM lane = query), B = a
// tile of 128 series (N = 128, TMEM column = series).  Warp-specialised:
//   warp 8 (producer)  streams the series tiles as K-chunks through an NS-deep
//                      ring of shared-memory stages with TMA bulk copies;
//   warp 9 (MMA)       issues tcgen05 MMAs chunk by chunk (one MMA per query
//                      tile and 16-wide k step), commits each chunk to free its
//                      stage and each finished tile to its accumulator buffer;
//   warps 0-7          read accumulators from TMEM (double-buffered) and test
//                      every (query, series) pair.
// A CTA owns QPC (1 or 2) query tiles, so each series tile read from L2 serves
// QPC * 128 queries.  An epilogue thread owns one query, whose constants stay
// in registers; the candidate test, rearranged so that only one per-series
// pair of constants is needed,
//     lower <= U  <=>  xnorm * alpha + (2 c - xn (1 - kappa'))  >=  qn - gamma' - U
// costs two FMAs and a compare; a warp vote skips the rare candidate path.
// The extra 8u in kappa' and gamma' covers the rounding of this form.
constexpr int kTcEpiWarps = 8;
constexpr int kTcCtrlThreads = kTcEpiWarps * 32 + 64;     // + producer warp + MMA warp

// Named barrier of the 256 epilogue threads that also ORs a predicate over
// them, so a bounded wait that ran out in one warp stops all of them at once.
__device__ __forceinline__ bool epi_bar_any(bool v)
{
    unsigned r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, 1, 256, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((unsigned)v)
        : "memory");
    return r != 0;
}

__global__ void __launch_bounds__(kTcCtrlThreads, 1)
k_tc_screen(ScreenArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) unsigned long long bar_full[kTcMaxStages], bar_empty[kTcMaxStages];
    __shared__ __align__(8) unsigned long long bar_accf[2], bar_acce[2], bar_q;
    __shared__ unsigned tmem_base;
    __shared__ float2 rowc[2][kTcRows];     // (-xn (1 - kappa'), xnorm) per accumulator buffer
    __shared__ int s_fail;
    const unsigned len = a.len;
    const unsigned ck = chunk_k(len), nch = len / ck;
    const unsigned chunk_bytes = kTcRows * ck * 2;
    const unsigned qtile_bytes = kTcQ * len * 2;
    const unsigned QPC = a.qpc, NS = a.stages;
    unsigned char *qbuf = smem;                               // QPC query tiles
    unsigned char *ring = smem + QPC * qtile_bytes;           // NS chunk stages
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned QG = (a.QT + QPC - 1) / QPC;               // query-tile groups
    const unsigned groups = gridDim.x / QG;                   // CTAs per query-tile group
    const unsigned qg = blockIdx.x % QG, g = blockIdx.x / QG;
    const unsigned qt0 = qg * QPC;
    const unsigned nq = min(QPC, a.QT - qt0);                 // query tiles of this CTA
    const unsigned long long RT = (a.N + kTcRows - 1) / kTcRows;
    const unsigned long long nt = g < RT ? (RT - g + groups - 1) / groups : 0;

    if (warp == 0) tmem_alloc(&tmem_base, 512);
    if (tid == 0) {
        s_fail = 0;
        for (unsigned i = 0; i < NS; ++i) {
            mbar_init(&bar_full[i], 1);
            mbar_init(&bar_empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&bar_accf[i], 1);
            mbar_init(&bar_acce[i], kTcEpiWarps);
        }
        mbar_init(&bar_q, 1);
        fence_barrier_init();
        fence_proxy_async();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = tmem_base;
    const unsigned acc_cols = QPC * 128;                      // columns of one accumulator buffer

    if (warp == kTcEpiWarps) {
        // ------------------------------------------------ producer
        if (lane == 0 && nt > 0) {
            mbar_arrive_expect_tx(&bar_q, nq * qtile_bytes);
            for (unsigned qi = 0; qi < nq; ++qi)
                bulk_g2s(qbuf + qi * qtile_bytes,
                         reinterpret_cast<const unsigned char *>(a.qtiles) + (unsigned long long)(qt0 + qi) * qtile_bytes,
                         qtile_bytes, &bar_q);
            const unsigned long long total = nt * nch;
            for (unsigned long long n = 0; n < total && !s_fail; ++n) {
                const unsigned st = (unsigned)(n % NS);
                const unsigned long long use = n / NS;
                if (use > 0 && !mbar_wait_bounded(&bar_empty[st], (unsigned)((use - 1) & 1))) {
                    s_fail = 1;
                    break;
                }
                const unsigned long long j = n / nch, c = n % nch;
                const unsigned long long rt = g + j * groups;
                mbar_arrive_expect_tx(&bar_full[st], chunk_bytes);
                bulk_g2s(ring + st * chunk_bytes,
                         reinterpret_cast<const unsigned char *>(a.rtiles) + (rt * nch + c) * chunk_bytes, chunk_bytes,
                         &bar_full[st]);
            }
        }
    } else if (warp == kTcEpiWarps + 1) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0 && nt > 0) {
            const unsigned idesc = tc_idesc_f16(kTcQ, kTcRows);
            const unsigned sq = smem_u32(qbuf), sr = smem_u32(ring);
            const unsigned sbo_q = (len / 8) * 128, sbo_r = (ck / 8) * 128;
            bool ok = mbar_wait_bounded(&bar_q, 0);
            for (unsigned long long j = 0; j < nt && ok && !s_fail; ++j) {
                const unsigned ab = (unsigned)(j & 1);
                if (j >= 2 && !mbar_wait_bounded(&bar_acce[ab], (unsigned)(((j >> 1) - 1) & 1))) { ok = false; break; }
                tc_fence_after();
                for (unsigned c = 0; c < nch; ++c) {
                    const unsigned long long n = j * nch + c;
                    const unsigned st = (unsigned)(n % NS);
                    if (!mbar_wait_bounded(&bar_full[st], (unsigned)((n / NS) & 1))) { ok = false; break; }
                    tc_fence_after();
                    for (unsigned kk = 0; kk < ck / 16; ++kk) {
                        const unsigned long long bdesc = tc_desc(sr + st * chunk_bytes + kk * 256, 128, sbo_r);
                        for (unsigned qi = 0; qi < nq; ++qi)
                            tc_mma_f16(tmem + ab * acc_cols + qi * 128,
                                       tc_desc(sq + qi * qtile_bytes + (c * (ck / 16) + kk) * 256, 128, sbo_q), bdesc,
                                       idesc, (c | kk) != 0);
                    }
                    tc_commit(&bar_empty[st]);
                }
                if (!ok) break;
                tc_commit(&bar_accf[ab]);
            }
            if (!ok) s_fail = 1;
        }
    } else {
        // ------------------------------------------------ epilogue
        const unsigned qi = (QPC == 2) ? (unsigned)(warp >> 2) : 0u;
        const unsigned qloc = (unsigned)((warp & 3) * 32 + lane);
        const unsigned qj = (qt0 + qi) * kTcQ + qloc;
        const bool have = qt0 + qi < a.QT;
        const float qn = have ? a.qconst[4 * qj + 0] : 0.f;
        const float alpha = have ? a.qconst[4 * qj + 1] : 0.f;
        const float gamma = have ? a.qconst[4 * qj + 2] : 0.f;
        const bool act = have && a.active[qj] != 0;
        float U = have ? __uint_as_float(a.Ubits[qj]) : -1.f;
        float E = act ? qn - gamma - U : __int_as_float(0x7f800000);
        const float one_m_kappa = 1.f - kKappaP;
        // columns of this warp in an accumulator buffer: QPC = 2: all 128 series of
        // its query tile; QPC = 1: half of them
        const unsigned cbeg = (QPC == 2) ? qi * 128 : (unsigned)(warp >> 2) * 64;
        const unsigned ncol = (QPC == 2) ? 128u : 64u;
        const unsigned rbeg = (QPC == 2) ? 0u : (unsigned)(warp >> 2) * 64;   // first series of the tile
        // series norms of the next tile are fetched one tile ahead
        float nxt_xn = 0.f, nxt_nrm = 0.f;
        auto fetch_norms = [&](unsigned long long j) {
            const unsigned long long row = (g + j * groups) * kTcRows + tid;
            const bool rv = tid < kTcRows && j < nt && row < a.N;
            nxt_xn = rv ? a.xn[row] : 0.f;
            nxt_nrm = rv ? a.xnorm[row] : 0.f;
        };
        fetch_norms(0);
        for (unsigned long long j = 0; j < nt; ++j) {
            const unsigned ab = (unsigned)(j & 1);
            const unsigned long long rt = g + j * groups;
            if (tid < kTcRows) rowc[ab][tid] = make_float2(-nxt_xn * one_m_kappa, nxt_nrm);
            fetch_norms(j + 1);
            const bool okw = mbar_wait_bounded(&bar_accf[ab], (unsigned)((j >> 1) & 1));
            // also the barrier that publishes rowc to all epilogue warps
            if (epi_bar_any(!okw)) {
                s_fail = 1;
                break;
            }
            tc_fence_after();
            for (unsigned h = 0; h < ncol; h += 32) {
                float acc[32];
                tmem_ld32(tmem + ((unsigned)((warp & 3) * 32) << 16) + ab * acc_cols + cbeg + h, acc);
                bool hit = false;
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const float2 rc = rowc[ab][rbeg + h + i];
                    const float lhs = fmaf(rc.y, alpha, fmaf(2.f, acc[i], rc.x));
                    hit |= lhs >= E;
                }
                if (__any_sync(0xffffffffu, hit)) {
                    for (int i = 0; i < 32; ++i) {
                        const float2 rc = rowc[ab][rbeg + h + i];
                        const float lhs = fmaf(rc.y, alpha, fmaf(2.f, acc[i], rc.x));
                        if (!(lhs >= E)) continue;
                        const unsigned long long row = rt * kTcRows + rbeg + h + i;
                        if (row >= a.N) continue;
                        const unsigned o = atomicAdd(&a.cand_count[qj], 1u);
                        if (o < a.cap) a.cand_pos[(unsigned long long)qj * a.cap + o] = (unsigned)row;
                        if (a.k == 1) {
                            // upper end of the estimate: s + eps, rounded up
                            const float xn = a.xn[row];
                            const float shat = fmaf(-2.f, acc[i], xn + qn);
                            const float eps = fmaf(rc.y, alpha, gamma + kKappaP * xn);
                            const float up = fmaxf(__fmul_ru(__fadd_ru(shat, eps), 1.0000003f), 0.f);
                            if (up < U) {
                                U = up;
                                E = qn - gamma - U;
                                atomicMin(&a.Ubits[qj], __float_as_uint(up));
                            }
                        }
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&bar_acce[ab]);
            // pick up bounds lowered by the other CTAs of these query tiles
            if (act && (j & 63) == 63) {
                const float G = __uint_as_float(ld_volatile_u32(&a.Ubits[qj]));
                if (G < U) {
                    U = G;
                    E = qn - gamma - U;
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (s_fail && tid == 0) atomicOr(a.status, kStTimeout);
    if (warp == 0) tmem_dealloc(tmem, 512);
}

// ----------------------------------------------------------- recheck
// blockIdx.y: query; warps take its candidates, recompute the exact FP32
// distance and offer it (offer is idempotent for a row offered before).
__global__ void __launch_bounds__(256)
k_tc_recheck(IndexView iv, QueryParams qp, const QuerySlot *__restrict__ slots, unsigned B,
             const unsigned *__restrict__ cand_count, const unsigned *__restrict__ cand_pos, unsigned cap,
             const unsigned *__restrict__ active)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    const unsigned b = blockIdx.y;
    if (b >= B || !active[b]) return;
    const QuerySlot slot = slots[b];
    QueryState *st = slot.st;
    float *qs = reinterpret_cast<float *>(dsm);
    for (int i = threadIdx.x; i < iv.len; i += blockDim.x) qs[i] = slot.q[i];
    __syncthreads();
    const unsigned n = min(cand_count[b], cap);
    const int lane = threadIdx.x & 31;
    const unsigned nw = gridDim.x * (blockDim.x >> 5);
    unsigned long long done = 0, aband = 0;
    for (unsigned e = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); e < n; e += nw) {
        const unsigned pos = cand_pos[(unsigned long long)b * cap + e];
        if (pos >= st->seed_lo && pos < st->seed_hi) continue;      // offered by the seed already
        const float thr = prune_threshold(ld_volatile_u64(&st->thr), qp.F);
        const float d2 = warp_ed2(qs, iv.raw + (unsigned long long)pos * iv.len, iv.len, thr);
        if (d2 <= thr) {
            ++done;
            if (lane == 0) offer(qp, slot, iv.status, d2, iv.ids[pos]);
        } else {
            ++aband;
        }
        __syncwarp();
    }
    if (lane == 0) {
        if (done) atomicAdd(&st->c.refined, done);
        if (aband) atomicAdd(&st->c.abandoned, aband);
    }
}

// --------------------------------------------------- diagnostic GEMM
__global__ void __launch_bounds__(128)
k_tc_gemm_test(const __half *A, const __half *Bm, float *D, unsigned K, unsigned N, unsigned lbo, unsigned sbo,
               unsigned *status)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) unsigned long long bar_ld, bar_mma;
    __shared__ unsigned tmem_base;
    const unsigned abytes = 128 * K * 2, bbytes = N * K * 2;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) tmem_alloc(&tmem_base, 256);
    if (tid == 0) {
        mbar_init(&bar_ld, 1);
        mbar_init(&bar_mma, 1);
        fence_barrier_init();
        fence_proxy_async();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = tmem_base;
    bool ok = true;
    if (tid == 0) {
        mbar_arrive_expect_tx(&bar_ld, abytes + bbytes);
        bulk_g2s(smem, A, abytes, &bar_ld);
        bulk_g2s(smem + abytes, Bm, bbytes, &bar_ld);
        ok = mbar_wait_bounded(&bar_ld, 0);
        if (ok) {
            tc_fence_after();
            const unsigned sa = smem_u32(smem), sb = smem_u32(smem + abytes);
            for (unsigned kk = 0; kk < K / 16; ++kk)
                tc_mma_f16(tmem, tc_desc(sa + kk * 256, lbo, sbo), tc_desc(sb + kk * 256, lbo, sbo),
                           tc_idesc_f16(128, N), kk > 0);
            tc_commit(&bar_mma);
            ok = mbar_wait_bounded(&bar_mma, 0);
        }
        if (!ok) atomicOr(status, kStTimeout);
    }
    __syncthreads();
    tc_fence_after();
    for (unsigned c0 = 0; c0 < N; c0 += 32) {
        float v[32];
        tmem_ld32(tmem + ((unsigned)(warp * 32) << 16) + c0, v);
        for (int i = 0; i < 32; ++i) D[(warp * 32 + lane) * N + c0 + i] = v[i];
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, 256);
}

}  // namespace

// At least 120 KB so that a single screen CTA fits on an SM: each CTA holds
// 256 TMEM columns for its whole (persistent) life, and a second or third
// resident CTA would wait in tcgen05.alloc for columns that never free up.
// Shared memory is always the full budget (kTcSmemBudget): one screen CTA per
// SM, because each CTA holds all 512 TMEM columns for its whole (persistent)
// life and a second resident CTA would wait in tcgen05.alloc forever.
size_t screen_smem_bytes(int len)
{
    (void)len;
    return kTcSmemBudget;
}

// ring stages that fit next to `qpc` resident query tiles
unsigned screen_stages(int len, unsigned qpc)
{
    const size_t chunk = (size_t)kTcRows * chunk_k((unsigned)len) * 2;
    const size_t q = (size_t)qpc * kTcQ * len * 2;
    const size_t left = kTcSmemBudget > q ? kTcSmemBudget - q : 0;
    return (unsigned)std::min<size_t>(kTcMaxStages, left / chunk);
}

void init_screen_attributes()
{
    cudaFuncSetAttribute(k_tc_screen, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmemBudget);
}

void launch_make_screen_copy(const float *raw, unsigned long long N, int len, __half *tiles, float *xn, float *xnorm,
                             unsigned *bad, cudaStream_t s)
{
    const unsigned long long rows = ((N + kTcRows - 1) / kTcRows) * kTcRows;
    const unsigned long long want = (rows + 7) / 8;
    const unsigned long long cap = (unsigned long long)num_sms() * 16;
    k_make_screen_copy<<<(unsigned)std::min(want, cap), 256, 0, s>>>(raw, N, len, tiles, xn, xnorm, bad);
}

void launch_tc_qprep(const QuerySlot *slots, unsigned B, int len, const QueryParams &qp, __half *qtiles,
                     float *qconst, unsigned *Ubits, unsigned *cand_count, unsigned *flags, unsigned *active,
                     cudaStream_t s)
{
    const unsigned padded = (B + kTcQ - 1) / kTcQ * kTcQ;
    k_tc_qprep<<<padded, 256, 0, s>>>(slots, B, len, qp, qtiles, qconst, Ubits, cand_count, flags, active);
}

void launch_tc_next_pass(const QuerySlot *slots, unsigned B, const QueryParams &qp, unsigned cap, unsigned *Ubits,
                         unsigned *cand_count, unsigned *active, unsigned *n_active, cudaStream_t s)
{
    k_tc_next_pass<<<(B + 255) / 256, 256, 0, s>>>(slots, B, qp, cap, Ubits, cand_count, active, n_active);
}

void launch_tc_screen(const __half *rtiles, const float *xn, const float *xnorm, const __half *qtiles,
                      const float *qconst, unsigned *Ubits, unsigned *cand_count, unsigned *cand_pos,
                      const unsigned *active, unsigned cap, unsigned long long N, int len, unsigned B, int k,
                      unsigned *status, cudaStream_t s)
{
    ScreenArgs a;
    a.rtiles = rtiles;
    a.xn = xn;
    a.xnorm = xnorm;
    a.ids_unused = nullptr;
    a.qtiles = qtiles;
    a.qconst = qconst;
    a.Ubits = Ubits;
    a.cand_count = cand_count;
    a.cand_pos = cand_pos;
    a.active = active;
    a.cap = cap;
    a.N = N;
    a.len = (unsigned)len;
    a.QT = (B + kTcQ - 1) / kTcQ;
    a.k = k;
    a.status = status;
    a.qpc = (a.QT >= 2 && screen_stages(len, 2) >= 4) ? 2u : 1u;
    a.stages = screen_stages(len, a.qpc);
    const unsigned QG = (a.QT + a.qpc - 1) / a.qpc;
    const unsigned groups = std::max(1u, (unsigned)num_sms() / QG);
    k_tc_screen<<<groups * QG, kTcCtrlThreads, screen_smem_bytes(len), s>>>(a);
}

void launch_tc_recheck(const IndexView &iv, const QueryParams &qp, const QuerySlot *slots, unsigned B,
                       const unsigned *cand_count, const unsigned *cand_pos, unsigned cap, const unsigned *active,
                       cudaStream_t s)
{
    k_tc_recheck<<<dim3(4, B), 256, iv.len * 4, s>>>(iv, qp, slots, B, cand_count, cand_pos, cap, active);
}

messi_status debug_tc_gemm(const uint16_t *A_host, const uint16_t *B_host, unsigned K, unsigned N, unsigned lbo,
                           unsigned sbo, float *D_host)
{
    const size_t ab = 128ull * K * 2, bb = (size_t)N * K * 2, db = 128ull * N * 4;
    char *d = nullptr;
    if (cudaMalloc(&d, ab + bb + db + 256) != cudaSuccess) {
        cudaGetLastError();
        return fail(MESSI_ENOMEM, "messi_debug_tc_gemm: out of device memory");
    }
    unsigned *status = reinterpret_cast<unsigned *>(d + ab + bb + db);
    cudaError_t e = cudaMemcpy(d, A_host, ab, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d + ab, B_host, bb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(status, 0, 4);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_tc_gemm_test, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(ab + bb));
    if (e == cudaSuccess) {
        k_tc_gemm_test<<<1, 128, ab + bb>>>(reinterpret_cast<const __half *>(d), reinterpret_cast<const __half *>(d + ab),
                                            reinterpret_cast<float *>(d + ab + bb), K, N, lbo, sbo, status);
        e = cudaDeviceSynchronize();
    }
    unsigned st = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&st, status, 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(D_host, d + ab + bb, db, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return fail(MESSI_ECUDA, std::string("messi_debug_tc_gemm: ") + cudaGetErrorString(e));
    if (st) return fail(MESSI_ETIMEOUT, "messi_debug_tc_gemm: a bounded wait ran out");
    return MESSI_OK;
}

}  // namespace messi

extern "C" messi_status messi_debug_tc_gemm(const uint16_t *a_tile, const uint16_t *b_tile, uint32_t k, uint32_t n,
                                            uint32_t lbo, uint32_t sbo, float *d)
{
    if (!a_tile || !b_tile || !d) return messi::fail(MESSI_EINVAL, "messi_debug_tc_gemm: null argument");
    if (k == 0 || k % 16 || k > 256 || n == 0 || n % 32 || n > 256)
        return messi::fail(MESSI_EINVAL, "messi_debug_tc_gemm: k must be a multiple of 16 <= 256, n a multiple of 32 <= 256");
    return messi::debug_tc_gemm(a_tile, b_tile, k, n, lbo, sbo, d);
}
