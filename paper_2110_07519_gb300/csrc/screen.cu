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
//   FP32 rounding of the norms (the query norms computed in FP64, the row
//   norms as compensated FP32 sums within 1e-9 of exact before rounding;
//   the bound's constant carries 0.03u of slack for that).
// so s - eps <= true d^2 <= s + eps.  A pair is a candidate when
// s - eps <= U_q, U_q an upper bound of the query's true k-th squared
// distance; for k <= 16 the k-th smallest s + eps met so far also tightens
// U_q.  Candidates are then recomputed exactly in FP32 and offered to the
// query's best-so-far, and the usual FP64 near-tie resolution finishes the
// query.  A query whose candidate list overflows is screened again with its
// tightened bound, together with the other such queries only.
//
// Operand tiles (see tc.cuh): rows of the collection are copied once to f16 in
// 128-row tiles already in the tensor-core layout, chunk-major along K, so
// one bulk copy loads a K chunk of a tile; queries are laid out the same way,
// 128 per tile (whole-K while they stay resident in shared memory, chunk-major
// when they are streamed with the series chunks).
#include <cuda_fp16.h>

#include <algorithm>

#include "tc.cuh"

namespace messi {
namespace {

constexpr int kTcRows = 128;        // M: series per tile
constexpr int kTcQ = 128;           // N: queries per tile
constexpr float kKappa = 2.4e-7f;   // 4u: FP32 evaluation of s and rounding of the norms
constexpr float kKappaP = 7.2e-7f;  // 12u: kappa plus the rounding of the rearranged test
static_assert(kKappaP >= 3.f * kKappa, "the rearranged test's slack covers kappa and 8u more");
constexpr int kTcMaxStages = 16;
// dynamic shared memory of one screen CTA: the 227 KB a block may hold, less
// the kernel's 8 KB of static shared memory (barriers, per-query bounds,
// the candidate queue) and some margin, so that at 256 points two resident
// query tiles (128 KB) and five 16 KB ring stages fit together
constexpr size_t kTcSmemBudget = 217 * 1024;

// K width of one streamed chunk of a series tile: the largest of 64, 32, 16
// dividing len.  A tile is stored chunk-major: chunk c (k in [c*ck, c*ck+ck))
// is a 128 x ck operand in the tensor-core layout.
__host__ __device__ __forceinline__ unsigned chunk_k(unsigned len)
{
    return (len % 64 == 0) ? 64u : (len % 32 == 0) ? 32u : 16u;
}

// Query tiles stay resident in shared memory up to kTcResidentLen points (two
// per CTA, so each MMA has N = 256); longer queries are stored chunk-major
// like the series tiles and streamed through the ring with each series chunk,
// still two tiles per CTA.  Measured at 512 points: one resident 128 KB tile
// per CTA (N = 128) ran 0.65 of the tensor peak, streaming two reaches 0.9 at
// 1024 points.
constexpr unsigned kTcResidentLen = 256;

__host__ __device__ __forceinline__ unsigned query_chunk(unsigned len)
{
    return len > kTcResidentLen ? chunk_k(len) : 0u;
}

// byte offset of element (r, k) in a query tile: full-K core-matrix layout
// when resident, chunk-major when streamed
__host__ __device__ __forceinline__ unsigned qtile_offset(unsigned r, unsigned k, unsigned len)
{
    const unsigned qc = query_chunk(len);
    return qc ? (k / qc) * (kTcQ * qc * 2) + tc_offset(r, k % qc, qc) : tc_offset(r, k, len);
}

// minimum of three floats in one instruction
__device__ __forceinline__ float min3f(float a, float b, float c)
{
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

__device__ __forceinline__ float tc_coef(int len)
{
    return 1.002f * (9.765625e-4f + (float)(len + 16) * 1.1920929e-7f);
}

// ------------------------------------------------------- screen copy
// Squared norms in FP32 arithmetic, carried as an unevaluated sum hi + lo of
// two floats (GB300's FP64 rate is low): each product x*x is split exactly
// into p + e (e = fma(x, x, -p)), both are added into (hi, lo) with an exact
// two-sum on hi; lanes then combine their pairs across the warp the same way.
// For all-positive terms the pair differs from the exact sum by at most
// about (n u)^2 of it (n terms per lane or per warp step, u = 2^-24), far
// below the FP32 rounding of the final norm; hi + lo is rounded once, to
// nearest for |x|^2 and upward (then widened) for |x|.  No FP64: this GPU's
// FP64 rate made the square root the copy's bottleneck.
struct F2 {
    float hi, lo;
};
__device__ __forceinline__ F2 f2_add(F2 a, float b)
{
    const float s = a.hi + b;
    const float bb = s - a.hi;
    const float err = (a.hi - (s - bb)) + (b - bb);   // a.hi + b = s + err exactly
    return {s, a.lo + err};
}
__device__ __forceinline__ F2 f2_add2(F2 a, F2 b)
{
    F2 t = f2_add(a, b.hi);
    t.lo += b.lo;
    return t;
}

// One CTA per 128-row tile: each K chunk of the tile is converted into its
// tensor-core layout in shared memory and written out as one contiguous
// 4-16 KB block, so every global store is a full coalesced line; each warp
// reads 16 rows, ck / 4 lanes per row with 16-byte loads, and every lane
// keeps a compensated pair of its rows' squares across the chunks.  The
// lanes of a row then combine their pairs by an xor butterfly: squared norm
// -> xn (FP32, nearest) and |x| rounded up.
__global__ void __launch_bounds__(256)
k_make_screen_copy(const float *__restrict__ raw, unsigned long long N, int len, __half *__restrict__ tiles,
                   float *__restrict__ xn, float *__restrict__ xnorm, unsigned *__restrict__ bad)
{
    __shared__ __align__(16) unsigned char cbuf[kTcRows * 64 * 2];   // one chunk of the tile (at most 16 KB)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned ck = chunk_k((unsigned)len);
    const unsigned nch = (unsigned)len / ck;
    const unsigned lpr = ck / 4;                 // lanes per row: one float4 each
    const unsigned rpi = 32 / lpr;               // rows per warp load
    const unsigned iters = 16 / rpi;             // loads per chunk for the warp's 16 rows (2, 4 or 8)
    const unsigned sub = (unsigned)lane / lpr, part = (unsigned)lane % lpr;
    const unsigned cbytes = kTcRows * ck * 2;
    const unsigned long long RT = (N + kTcRows - 1) / kTcRows;
    for (unsigned long long tile = blockIdx.x; tile < RT; tile += gridDim.x) {
        unsigned char *tb = reinterpret_cast<unsigned char *>(tiles) + tile * (unsigned long long)kTcRows * len * 2;
        F2 ss[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) ss[i] = {0.f, 0.f};
        bool big = false;
        for (unsigned c = 0; c < nch; ++c) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                if ((unsigned)i < iters) {
                    const unsigned r = (unsigned)warp * 16 + (unsigned)i * rpi + sub;   // row within the tile
                    const unsigned long long row = tile * kTcRows + r;
                    const unsigned k = part * 4;                                     // column within the chunk
                    float v[4] = {0.f, 0.f, 0.f, 0.f};
                    if (row < N) {
                        const float4 a4 = __ldg(reinterpret_cast<const float4 *>(
                            raw + row * (unsigned long long)len + (unsigned long long)c * ck + k));
                        v[0] = a4.x; v[1] = a4.y; v[2] = a4.z; v[3] = a4.w;
                    }
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        big = big || fabsf(v[e]) > 65000.f;
                        const float pr = __fmul_rn(v[e], v[e]);
                        const float pe = __fmaf_rn(v[e], v[e], -pr);     // v^2 = pr + pe exactly
                        ss[i] = f2_add(ss[i], pr);
                        ss[i].lo = __fadd_rn(ss[i].lo, pe);
                    }
                    __align__(8) __half2 h[2] = {__floats2half2_rn(v[0], v[1]), __floats2half2_rn(v[2], v[3])};
                    *reinterpret_cast<uint2 *>(cbuf + tc_offset(r, k, ck)) = *reinterpret_cast<const uint2 *>(h);
                }
            }
            __syncthreads();
            for (unsigned o = threadIdx.x * 16u; o < cbytes; o += blockDim.x * 16u)
                *reinterpret_cast<uint4 *>(tb + (unsigned long long)c * cbytes + o) =
                    *reinterpret_cast<const uint4 *>(cbuf + o);
            __syncthreads();
        }
        if (big) atomicOr(bad, 1u);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if ((unsigned)i < iters) {
                F2 t = ss[i];
                for (unsigned off = lpr / 2; off >= 1; off >>= 1) {
                    const F2 o = {__shfl_xor_sync(0xffffffffu, t.hi, off), __shfl_xor_sync(0xffffffffu, t.lo, off)};
                    t = f2_add2(t, o);
                }
                if (part == 0) {
                    const unsigned long long row = tile * kTcRows + (unsigned)warp * 16 + (unsigned)i * rpi + sub;
                    // |x|^2 to nearest (one correctly rounded addition of the
                    // pair); |x| rounded up from the pair's sum rounded up and
                    // widened by 2^-20 (far above the pair's 1e-9 relative
                    // error), all in FP32
                    xn[row] = __fadd_rn(t.hi, t.lo);
                    xnorm[row] = __fsqrt_ru(__fmul_ru(__fadd_ru(t.hi, t.lo), 1.00000095367431640625f));
                }
            }
        }
    }
}

// ------------------------------------------------------- query prep
// One block per query: f16 copy into its query tile, |q|^2 and |q|, the
// per-query epilogue constants and the initial bound U_q from the seed.
__global__ void __launch_bounds__(256)
k_tc_qprep(const QuerySlot *__restrict__ slots, unsigned B, int len, QueryParams qp, __half *__restrict__ qtiles,
           float *__restrict__ qconst, unsigned *__restrict__ Ubits, unsigned *__restrict__ cand_count,
           unsigned *__restrict__ flags, unsigned *__restrict__ active, float *__restrict__ tkinit,
           unsigned *__restrict__ glock, uint2 *__restrict__ srange)
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
        *reinterpret_cast<uint4 *>(tbase + qtile_offset(r, (unsigned)k0, (unsigned)len)) = *reinterpret_cast<uint4 *>(h);
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
        // the seed leaf's k best, widened like U (their k-th is U itself)
        uint2 sr = make_uint2(0u, 0u);
        if (real && f == 0) {
            const QueryState *st = slots[b].st;
            sr = make_uint2(st->seed_lo, st->seed_hi);
            const unsigned kc = st->kcount;
            for (int j = 0; j < (int)kTcTopKHost; ++j)
                tkinit[b * (int)kTcTopKHost + j] = (j < qp.k && (unsigned)j < kc) ? prune_threshold(slots[b].karr[j], qp.F)
                                                                         : __int_as_float(0x7f800000);
        } else {
            for (int j = 0; j < (int)kTcTopKHost; ++j) tkinit[b * (int)kTcTopKHost + j] = __int_as_float(0x7f800000);
        }
        srange[b] = sr;
        glock[b] = 0u;
    }
}

// Between passes: a query whose candidate list overflowed is screened again
// with its bound tightened by the rechecked candidates; the others stop.  The
// queries screened again are gathered into the first rows of `qtiles2`
// (their f16 rows copied over, `qmap` giving each one's batch index), so the
// next pass runs over as many query tiles as they fill, not the batch's.
__global__ void k_tc_next_pass(const QuerySlot *__restrict__ slots, unsigned B, QueryParams qp, unsigned cap,
                               unsigned *__restrict__ Ubits, unsigned *__restrict__ cand_count,
                               unsigned *__restrict__ active, unsigned *__restrict__ n_active,
                               const __half *__restrict__ qtiles, __half *__restrict__ qtiles2,
                               unsigned *__restrict__ qmap, int len)
{
    const unsigned b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    if (active[b] && cand_count[b] > cap) {
        const float U = prune_threshold(ld_volatile_u64(&slots[b].st->thr), qp.F);
        if (U < __uint_as_float(Ubits[b])) Ubits[b] = __float_as_uint(U);
        cand_count[b] = 0;
        const unsigned o = atomicAdd(n_active, 1u);
        qmap[o] = b;
        const size_t tile_bytes = (size_t)kTcQ * len * 2;
        const unsigned char *src = reinterpret_cast<const unsigned char *>(qtiles) + (b / kTcQ) * tile_bytes;
        unsigned char *dst = reinterpret_cast<unsigned char *>(qtiles2) + (o / kTcQ) * tile_bytes;
        for (unsigned k0 = 0; k0 < (unsigned)len; k0 += 8)
            *reinterpret_cast<uint4 *>(dst + qtile_offset(o % kTcQ, k0, (unsigned)len)) =
                *reinterpret_cast<const uint4 *>(src + qtile_offset(b % kTcQ, k0, (unsigned)len));
    } else {
        active[b] = 0;
    }
}

// ------------------------------------------------------------ screen
struct ScreenArgs {
    const __half *rtiles;     // [RT][128 x len] f16 rows
    const float *xn, *xnorm;  // [RT * 128]
    const __half *qtiles;     // [QT][128 x len] f16 queries
    const float *qconst;      // [QT*128][4]
    unsigned *Ubits;          // [QT*128] float bits, atomically lowered (k = 1)
    unsigned *cand_count;     // [QT*128]
    unsigned *cand_pos;       // [QT*128][cap]
    const unsigned *active;   // [QT*128]: nonzero when the query collects candidates this pass
    const unsigned *qmap;     // [B]: batch index of each screened query (nullptr: the identity)
    float *topk;              // [batch][kTcTopK]: the query's k smallest upper ends met so far (1 < k <= kTcTopK),
                              // starting from the seed leaf's k best; updated under glock
    unsigned *glock;          // [batch]: lock of each query's list
    int lists;                // 1: this pass adds to the lists (the first; later passes meet the rows again)
    const uint2 *srange;      // [batch]: the seed leaf's positions [x, y)
    unsigned B;               // queries screened (rows of qtiles in use)
    unsigned cap;
    unsigned qpc;             // query tiles per CTA (1 or 2)
    unsigned stages;          // chunk stages of the ring
    unsigned long long N;
    unsigned len;
    unsigned QT;
    int k;
    unsigned *status;
};

// Operand roles: A = a tile of 128 series (M = 128, TMEM lane = series), B =
// the CTA's QPC query tiles side by side (N = QPC * 128, TMEM column =
// query).  The query tiles are resident next to each other in the same
// core-matrix layout, so together they are one operand of QPC * 128 rows and
// one MMA per 16-wide k step covers every query of the CTA: for QPC = 2 it
// reads 12 KB of operands from shared memory where two MMAs of N = 128 read
// 16 KB, and the issuing thread issues half as many instructions.
// Warp-specialised:
//   warps 8, 10        (producers) stream the series tiles as K-chunks through
//                      an NS-deep ring of shared-memory stages with TMA bulk
//                      copies, taking alternate chunks: one thread's bulk
//                      copies complete one after another, two threads keep
//                      twice as many in flight;
//   warp 9 (MMA)       issues tcgen05 MMAs chunk by chunk (one MMA per
//                      16-wide k step), commits each chunk to free its stage
//                      and each finished tile to its accumulator buffer;
//   warp 11 (relay)    waits on the mbarriers the MMA warp depends on (chunk
//                      loaded, accumulator buffer drained) and meets the MMA
//                      warp at a named barrier once per two chunks (once per
//                      chunk when a tile has an odd number): an mbarrier
//                      wait in the thread that issues the MMAs costs it
//                      hundreds of cycles even when the phase is complete,
//                      a named barrier does not;
//   warps 0-7          read accumulators from TMEM (double-buffered) and test
//                      every (query, series) pair.
// An epilogue thread owns one series of the tile (its TMEM lane; warp w reads
// lanes 32 (w mod 4) ...) and half of the CTA's queries (warps 0-3 the first
// half of the columns, warps 4-7 the second).  The candidate test, rearranged
// so that one per-series and one per-query constant meet the accumulator,
//     lower <= U_q  <=>  xnorm * alpha_q + (2 c - xn (1 - kappa'))  >=  qn - gamma' - U_q  =: E_q,
// is first applied with alpha_q replaced by the largest alpha of the CTA's
// queries (xnorm >= 0, so the left side only grows): the per-series
//     r = xnorm * alpha_max - xn (1 - kappa')   (rounded up)
// stays in a register, E_q is read four queries at a time from shared memory
// (every lane of a warp tests the same queries: a broadcast), and each pair
// costs one FMA (rounded up) and a compare.  A warp vote skips the rare path,
// which re-tests the pair with its query's own alpha before taking it as a
// candidate.  The extra 8u in kappa' and gamma' covers the rounding of the
// exact form.
// The bounds are per query and shared by the CTA: U_q (float bits, only
// lowered, by atomicMin) and E_q derived from it.  Two racing stores of E_q
// may leave the looser one in place; every stored E_q still derives from a
// valid U_q, so the test stays conservative.
constexpr int kTcEpiWarps = 8;
// + 2 producer warps + MMA warp + relay warp + candidate warp
constexpr int kTcCtrlThreads = kTcEpiWarps * 32 + 160;
constexpr int kTcProdWarp0 = kTcEpiWarps, kTcMmaWarp = kTcEpiWarps + 1, kTcProdWarp1 = kTcEpiWarps + 2,
              kTcRelayWarp = kTcEpiWarps + 3, kTcCandWarp = kTcEpiWarps + 4;
// Candidate queue of a CTA: the epilogue warps append the pairs that pass
// their test and the candidate warp records them (global slot, top-k list,
// bounds), so the epilogue never waits on that work.  Entry t lives in slot
// t mod kTcCq and is ready once its sequence word holds t + 1.
constexpr unsigned kTcCq = 256;

// Named barrier 3: the MMA warp and the relay warp, once per chunk.
__device__ __forceinline__ void relay_bar_sync() { asm volatile("bar.sync 3, 64;" ::: "memory"); }

// 64 consecutive FP32 columns of this thread's TMEM lane, one load and one wait.
__device__ __forceinline__ void tmem_ld64(unsigned taddr, float (&v)[64])
{
    unsigned r[64];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x64.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, "
        "%32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47, "
        "%48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63}, [%64];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]),
          "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]),
          "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]),
          "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]),
          "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 64; ++i) v[i] = __uint_as_float(r[i]);
}

// Named barrier over the 256 epilogue threads.
__device__ __forceinline__ void epi_bar_sync() { asm volatile("bar.sync 2, 256;" ::: "memory"); }

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

// k <= kTcTopK: each query keeps, in global memory, the k smallest upper
// ends met by any CTA (ascending; each from a different row, since the
// screen meets every (query, row) pair once and the list starts from the
// seed leaf's k best, whose rows it skips), and the k-th of them bounds the
// query's k-th squared distance from above just as the single best does for
// k = 1.  The candidate warps update it under a per-query lock taken with a
// bounded spin; a lane that does not get the lock skips its update, which
// only leaves the bound looser.  One list for all CTAs, not one per CTA: a
// CTA meets 1/G of the rows, so its own k-th would sit far above the
// query's.
constexpr int kTcTopK = 16;
static_assert(kTcTopK == (int)kTcTopKHost, "top-k list length shared with the workspace layout");
static_assert((kTcSmemBudget - (size_t)2 * kTcQ * kTcResidentLen * 2) / (kTcRows * 64 * 2) >= 4,
              "two query tiles of the longest resident length and 4 ring stages fit");
static_assert(kTcSmemBudget / (3 * kTcRows * 64 * 2) >= 4,
              "streamed queries: 4 stages of a series chunk and two query chunks fit");

__device__ __forceinline__ bool list_lock(unsigned *l)
{
    for (int it = 0; it < 4096; ++it) {
        if (atomicCAS(l, 0u, 1u) == 0u) {
            __threadfence();
            return true;
        }
        __nanosleep(64);
    }
    return false;
}

__device__ __forceinline__ void list_unlock(unsigned *l)
{
    __threadfence();
    atomicExch(l, 0u);
}

// A queued pair (query, series row) passed the epilogue's test with the CTA's
// largest alpha: the candidate warp re-tests it with the query's own alpha,
// records it as a candidate, and for k <= kTcTopK lowers the query's bound U
// with the upper end of its estimate.
struct CandidateSink {
    const float *qconst;
    unsigned *cand_count, *cand_pos, *Ubits;
    float *sE;           // shared: E_q per query of the CTA
    unsigned *sU;        // shared: U_q bits
    float *topk;         // global: [batch][kTcTopK] lists (1 < k <= kTcTopK)
    unsigned *glock;     // global: [batch] list locks
    const unsigned *qmap;
    const uint2 *srange; // the seed leaf's positions, whose rows the lists already hold
    unsigned long long N;
    unsigned cap, B;
    int k, lists;
};

__device__ __forceinline__ void screen_candidate(const CandidateSink &a, unsigned ql, unsigned qc, unsigned long long row,
                                                 float acc, float xn, float xnrm)
{
    if (row >= a.N || qc >= a.B) return;
    const unsigned qj = a.qmap ? a.qmap[qc] : qc;      // the query's batch index
    const float qn = a.qconst[4 * qj + 0], alpha = a.qconst[4 * qj + 1], gamma = a.qconst[4 * qj + 2];
    const float one_m_kappa = 1.f - kKappaP;
    const float lhs = fmaf(xnrm, alpha, fmaf(2.f, acc, -xn * one_m_kappa));
    if (!(lhs >= *(volatile float *)&a.sE[ql])) return;
    const unsigned o = atomicAdd(&a.cand_count[qj], 1u);
    if (o < a.cap) a.cand_pos[(unsigned long long)qj * a.cap + o] = (unsigned)row;
    if (a.k > kTcTopK) return;
    // a row of the seed leaf is already in the lists (they start from the
    // seed's k best): a second entry for it would make the k-th too small
    if (a.k > 1) {
        const uint2 sr = a.srange[qj];
        if (row >= sr.x && row < sr.y) return;
    }
    // upper end of the estimate: s + eps, rounded up
    const float shat = fmaf(-2.f, acc, xn + qn);
    const float eps = fmaf(xnrm, alpha, gamma + kKappaP * xn);
    const float up = fmaxf(__fmul_ru(__fadd_ru(shat, eps), 1.0000003f), 0.f);
    float bound = up;
    if (a.k > 1) {
        if (!a.lists) return;   // a later pass: the pair may already be in the list
        volatile float *t = a.topk + (size_t)qj * kTcTopK;
        if (!(up < t[a.k - 1])) return;   // (read without the lock: a shortcut only)
        if (!list_lock(&a.glock[qj])) return;
        int j = a.k - 1;
        if (up < t[j]) {
            while (j > 0 && t[j - 1] > up) {
                t[j] = t[j - 1];
                --j;
            }
            t[j] = up;
        }
        bound = t[a.k - 1];
        list_unlock(&a.glock[qj]);
    }
    // bounds are >= 0 (or +inf): their bits order like the values
    const unsigned bb = __float_as_uint(bound);
    const unsigned old = atomicMin(&a.sU[ql], bb);
    if (bb < old) {
        atomicMin(&a.Ubits[qj], bb);
        a.sE[ql] = __fsub_rd(__fsub_rd(qn, gamma), bound);
    }
}

// Epilogue side of the candidate queue (the warp converged): the lanes whose
// pair passed reserve consecutive entries with one shared atomic, each waits
// (bounded) until its slot is free, writes the entry and publishes it.  A
// slot t stays free once the candidate warp has taken entries up to t - kTcCq.
__device__ __forceinline__ void cq_push(bool pass, unsigned row, unsigned ql, float acc, uint4 *q, unsigned *seq,
                                        unsigned *tail, volatile unsigned *head, volatile int *fail)
{
    const unsigned bal = __ballot_sync(0xffffffffu, pass);
    if (!bal) return;
    const unsigned lane = threadIdx.x & 31;
    unsigned base = 0;
    if (lane == 0) base = atomicAdd(tail, (unsigned)__popc(bal));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (!pass) return;
    const unsigned t = base + __popc(bal & ((1u << lane) - 1u));
    for (unsigned it = 0; t - *head >= kTcCq; ++it) {
        if (it >= kSpinLimit || *fail) {   // (after a failure the candidate warp may be gone)
            *fail = 1;
            return;
        }
        __nanosleep(32);
    }
    __threadfence_block();
    q[t % kTcCq] = make_uint4(row, ql, __float_as_uint(acc), 0u);
    __threadfence_block();
    *reinterpret_cast<volatile unsigned *>(&seq[t % kTcCq]) = t + 1u;
}

// One chunk of KS 16-wide k-steps: series operand `rd` (ring stage) against
// the query operand `qd`; k-step kk starts kk * 256 bytes further in both.
template <int KS>
__device__ __forceinline__ void mma_chunk(unsigned d, unsigned long long rd, unsigned long long qd, unsigned idesc,
                                          bool accumulate)
{
#pragma unroll
    for (int kk = 0; kk < KS; ++kk)
        tc_mma_f16(d, rd + kk * 16u, qd + kk * 16u, idesc, (kk > 0 || accumulate) ? 1u : 0u);
}

// KS = chunk width / 16 (1, 2 or 4)
template <int KS>
__global__ void __launch_bounds__(kTcCtrlThreads, 1)
k_tc_screen(ScreenArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) unsigned long long bar_full[kTcMaxStages], bar_empty[kTcMaxStages];
    __shared__ __align__(8) unsigned long long bar_accf[2], bar_acce[2], bar_q;
    __shared__ unsigned tmem_base;
    __shared__ __align__(16) float sE[2 * kTcQ];     // E_q per query of the CTA (+inf: not tested)
    __shared__ unsigned sU[2 * kTcQ];                // U_q bits
    __shared__ unsigned s_amax;                      // bits of the CTA's largest alpha
    __shared__ volatile int s_fail;
    __shared__ unsigned s_fills[kTcMaxStages];                 // bulk-copy fills issued per ring stage
    __shared__ __align__(8) unsigned long long bar_drain;      // the MMA warp's last commit
    __shared__ uint4 s_cq[kTcCq];                              // candidate queue: row, query slot, acc bits
    __shared__ unsigned s_cq_seq[kTcCq];                       // slot ready for entry t: t + 1
    __shared__ unsigned s_cq_tail;                             // entries reserved
    __shared__ volatile unsigned s_cq_head;                    // entries taken by the candidate warp
    __shared__ unsigned s_epi_done;                            // epilogue warps finished
    __shared__ volatile unsigned s_epi_tiles;                  // tiles finished by epilogue warp 0
    const unsigned len = a.len;
    constexpr unsigned ck = KS * 16;
    const unsigned nch = len / ck;
    const unsigned chunk_bytes = kTcRows * ck * 2;
    const unsigned qtile_bytes = kTcQ * len * 2;
    const unsigned QPC = a.qpc, NS = a.stages;
    // resident queries: QPC query tiles, then NS stages of one series chunk;
    // streamed queries (len > kTcResidentLen): NS stages of a series chunk
    // followed by the same K chunk of each of the QPC query tiles
    const bool qstream = query_chunk(len) != 0;
    const unsigned stage_bytes = chunk_bytes * (qstream ? 1 + QPC : 1);
    unsigned char *qbuf = smem;
    unsigned char *ring = smem + (qstream ? 0 : QPC * qtile_bytes);
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
        s_amax = 0u;
        for (unsigned i = 0; i < NS; ++i) {
            mbar_init(&bar_full[i], 1);
            mbar_init(&bar_empty[i], 1);
            s_fills[i] = 0u;
        }
        mbar_init(&bar_drain, 1);
        for (unsigned i = 0; i < kTcCq; ++i) s_cq_seq[i] = 0u;
        s_cq_tail = 0u;
        s_cq_head = 0u;
        s_epi_done = 0u;
        s_epi_tiles = 0u;
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

    if (warp == kTcProdWarp0 || warp == kTcProdWarp1) {
        // ------------------------------------------------ producers
        const unsigned p = (warp == kTcProdWarp0) ? 0u : 1u;
        if (lane == 0 && nt > 0) {
            if (p == 0 && !qstream) {
                mbar_arrive_expect_tx(&bar_q, nq * qtile_bytes);
                for (unsigned qi = 0; qi < nq; ++qi)
                    bulk_g2s(qbuf + qi * qtile_bytes,
                             reinterpret_cast<const unsigned char *>(a.qtiles) +
                                 (unsigned long long)(qt0 + qi) * qtile_bytes,
                             qtile_bytes, &bar_q);
            }
            // chunk n = p, p + 2, ...: ring stage st = n mod NS in use u = n / NS
            // (a stage in use u > 0 waits for its release in use u - 1), and
            // series tile j, chunk c of the chunk sequence, all advanced by 2
            const unsigned long long total = nt * nch;
            unsigned st = p, u = 0, c = p % nch;
            unsigned long long j = p / nch;
            for (unsigned long long n = p; n < total && !s_fail; n += 2) {
                if (u > 0 && !mbar_wait_issuer(&bar_empty[st], (u - 1u) & 1u)) {
                    s_fail = 1;
                    break;
                }
                const unsigned long long rt = g + j * groups;
                unsigned char *stage = ring + st * stage_bytes;
                mbar_arrive_expect_tx(&bar_full[st], chunk_bytes * (qstream ? 1 + nq : 1));
                bulk_g2s(stage, reinterpret_cast<const unsigned char *>(a.rtiles) + (rt * nch + c) * chunk_bytes,
                         chunk_bytes, &bar_full[st]);
                if (qstream)
                    for (unsigned qi = 0; qi < nq; ++qi)
                        bulk_g2s(stage + (1 + qi) * chunk_bytes,
                                 reinterpret_cast<const unsigned char *>(a.qtiles) +
                                     ((unsigned long long)(qt0 + qi) * nch + c) * chunk_bytes,
                                 chunk_bytes, &bar_full[st]);
                atomicAdd(&s_fills[st], 1u);
                st += 2;
                while (st >= NS) {
                    st -= NS;
                    ++u;
                }
                c += 2;
                while (c >= nch) {
                    c -= nch;
                    ++j;
                }
            }
        }
    } else if (warp == kTcMmaWarp) {
        // ------------------------------------------------ MMA issuer
        // The whole warp meets the relay once per chunk (so neither warp can
        // wait at the named barrier for one that has left: both run every
        // iteration, and after a failure lane 0 only stops issuing).
        if (nt > 0) {
            const unsigned idesc = tc_idesc_f16(kTcRows, nq * kTcQ);
            const unsigned sq = smem_u32(qbuf), sr = smem_u32(ring);
            const unsigned sbo_r = (ck / 8) * 128, sbo_q = qstream ? sbo_r : (len / 8) * 128;
            // descriptors of k-step 0 of ring stage 0 and of the query
            // operand; the others differ only in the start-address field
            // (address >> 4, bits 0-13), reached by plain adds since every
            // shared-memory address here is below 256 KB.  Query tile 1
            // starts 16 row groups (16 * sbo_q bytes) after tile 0, so one
            // descriptor spans both.
            // (streamed queries: the query operand sits chunk_bytes into each
            // stage and advances with the stage)
            const unsigned long long rd0 = tc_desc(sr, 128, sbo_r);
            const unsigned long long qd0 = qstream ? tc_desc(sr + chunk_bytes, 128, sbo_q) : tc_desc(sq, 128, sbo_q);
            const unsigned sstride16 = stage_bytes >> 4;
            unsigned st = 0;
            const unsigned G = (nch % 2 == 0) ? 2u : 1u;    // chunks per meeting with the relay
            for (unsigned long long j = 0; j < nt; ++j) {
                const unsigned ab = (unsigned)(j & 1);
                for (unsigned c = 0; c < nch; ++c) {
                    if (c % G == 0) relay_bar_sync();
                    tc_fence_after();
                    if (lane == 0 && !s_fail) {
                        const unsigned long long qd = qstream ? qd0 + st * sstride16 : qd0 + c * (KS * 16u);
                        mma_chunk<KS>(tmem + ab * acc_cols, rd0 + st * sstride16, qd, idesc, c != 0);
                        tc_commit(&bar_empty[st]);
                    }
                    __syncwarp();
                    if (++st == NS) st = 0;
                }
                if (lane == 0 && !s_fail) tc_commit(&bar_accf[ab]);
                __syncwarp();
            }
            // completes once every MMA this thread issued has finished
            if (lane == 0) tc_commit(&bar_drain);
        }
    } else if (warp == kTcRelayWarp) {
        // ------------------------------------------------ relay
        if (nt > 0) {
            if (lane == 0 && !qstream && !mbar_wait_bounded(&bar_q, 0)) s_fail = 1;
            unsigned st = 0, fpar = 0;          // ring stage and the parity of its current fill
            for (unsigned long long j = 0; j < nt; ++j) {
                const unsigned ab = (unsigned)(j & 1);
                // accumulator buffer ab drained by the epilogue (tile j - 2)
                if (lane == 0 && j >= 2 && !s_fail &&
                    !mbar_wait_bounded(&bar_acce[ab], (unsigned)(((j >> 1) - 1) & 1)))
                    s_fail = 1;
                const unsigned G = (nch % 2 == 0) ? 2u : 1u;
                for (unsigned c = 0; c < nch; ++c) {
                    if (lane == 0 && !s_fail && !mbar_wait_bounded(&bar_full[st], fpar)) s_fail = 1;
                    __syncwarp();
                    if (c % G == G - 1) relay_bar_sync();
                    if (++st == NS) {
                        st = 0;
                        fpar ^= 1u;
                    }
                }
            }
        }
    } else if (warp == kTcCandWarp) {
        // ------------------------------------------------ candidates
        // Takes the queued pairs in order, up to 32 at a time (one per lane),
        // until every epilogue warp has finished and the queue is empty.  The
        // idle wait is bounded and counts only while the epilogue makes no
        // progress.
        const CandidateSink sink{a.qconst, a.cand_count, a.cand_pos, a.Ubits, sE, sU, a.topk, a.glock, a.qmap,
                                 a.srange, a.N, a.cap, a.B, a.k, a.lists};
        unsigned head = 0, idle = 0, seen = 0;
        bool ok = true;
        for (;;) {
            const unsigned tail = ld_volatile_u32(&s_cq_tail);
            if (head == tail) {
                if (ld_volatile_u32(&s_epi_done) == kTcEpiWarps) {
                    __threadfence_block();
                    if (ld_volatile_u32(&s_cq_tail) == head) break;
                    continue;
                }
                const unsigned prog = s_epi_tiles + ld_volatile_u32(&s_epi_done);
                if (prog != seen) {
                    seen = prog;
                    idle = 0;
                } else if (++idle >= kSpinLimit) {
                    ok = false;
                    break;
                }
                __nanosleep(64);
                continue;
            }
            const unsigned n = min(32u, tail - head);
            uint4 e = make_uint4(0u, 0u, 0u, 0u);
            bool got = true;
            if ((unsigned)lane < n) {
                const unsigned t = head + lane;
                for (unsigned it = 0; ld_volatile_u32(&s_cq_seq[t % kTcCq]) != t + 1u; ++it) {
                    if (it >= kSpinLimit) {
                        got = false;
                        break;
                    }
                    __nanosleep(32);
                }
                __threadfence_block();
                if (got) e = s_cq[t % kTcCq];
            }
            if (!__all_sync(0xffffffffu, got)) {
                ok = false;
                break;
            }
            head += n;
            __syncwarp();
            if (lane == 0) {
                __threadfence_block();
                s_cq_head = head;   // the slots read above may be written again
            }
            if ((unsigned)lane < n) {
                const unsigned long long row = e.x;
                const bool rv = row < a.N;
                screen_candidate(sink, e.y, qt0 * kTcQ + e.y, row, __uint_as_float(e.z), rv ? a.xn[row] : 0.f,
                                 rv ? a.xnorm[row] : 0.f);
            }
            __syncwarp();
        }
        if (!ok) s_fail = 1;
    } else {
        // ------------------------------------------------ epilogue
        const unsigned lg = (unsigned)(warp & 3);             // TMEM lane group of this warp
        const unsigned srow = lg * 32 + lane;                 // this thread's series within a tile
        const unsigned ncol = acc_cols / 2;                   // queries (columns) of this warp: 128 or 64
        const unsigned cbeg = (unsigned)(warp >> 2) * ncol;
        const bool cols_live = cbeg < nq * kTcQ;              // one query tile in a QPC = 2 CTA: half idle
        // thread t sets up (and later refreshes) the bounds of query t of the CTA
        const unsigned own_qc = qt0 * kTcQ + tid;
        const bool own_have = (unsigned)tid < nq * kTcQ && own_qc < a.B;
        const unsigned own_qj = own_have ? (a.qmap ? a.qmap[own_qc] : own_qc) : 0u;
        const float own_qn = own_have ? a.qconst[4 * own_qj + 0] : 0.f;
        const float own_gamma = own_have ? a.qconst[4 * own_qj + 2] : 0.f;
        const bool own_act = own_have && a.active[own_qj] != 0;
        if ((unsigned)tid < acc_cols) {
            const float U = own_have ? __uint_as_float(a.Ubits[own_qj]) : -1.f;
            sU[tid] = __float_as_uint(U);
            sE[tid] = own_act ? __fsub_rd(__fsub_rd(own_qn, own_gamma), U) : __int_as_float(0x7f800000);
            // alpha >= 0: its bits order like the values
            if (own_act) atomicMax(&s_amax, __float_as_uint(a.qconst[4 * own_qj + 1]));
        }
        epi_bar_sync();
        const float amax = __uint_as_float(s_amax);
        const float one_m_kappa = 1.f - kKappaP;
        // series norms of the next tile are fetched one tile ahead
        float nxt_xn = 0.f, nxt_nrm = 0.f;
        auto fetch_norms = [&](unsigned long long j) {
            const unsigned long long row = (g + j * groups) * kTcRows + srow;
            const bool rv = j < nt && row < a.N;
            nxt_xn = rv ? a.xn[row] : 0.f;
            nxt_nrm = rv ? a.xnorm[row] : 0.f;
        };
        fetch_norms(0);
        for (unsigned long long j = 0; j < nt; ++j) {
            const unsigned ab = (unsigned)(j & 1);
            const unsigned long long row = (g + j * groups) * kTcRows + srow;
            const float xn = nxt_xn, xnrm = nxt_nrm;
            // a padding row never passes: r = -inf
            const float r = row < a.N ? __fmaf_ru(xnrm, amax, __fmul_ru(-xn, one_m_kappa)) : __int_as_float(0xff800000);
            fetch_norms(j + 1);
            const bool okw = mbar_wait_bounded(&bar_accf[ab], (unsigned)((j >> 1) & 1));
            if (epi_bar_any(!okw || s_fail)) {
                s_fail = 1;
                break;
            }
            tc_fence_after();
            if (cols_live) {
                for (unsigned h = 0; h < ncol; h += 64) {
                    float acc[64];
                    tmem_ld64(tmem + ((lg * 32) << 16) + ab * acc_cols + cbeg + h, acc);
                    const float4 *e4 = reinterpret_cast<const float4 *>(&sE[cbeg + h]);
                    // v = E_q - 2 acc rounded down is at most its exact value, so
                    // min over q of v <= r whenever a pair passes 2 acc + r >= E_q
                    // exactly; one minimum per group of 16 queries
                    float mn[4];
#pragma unroll
                    for (int gq = 0; gq < 4; ++gq) {
                        float m0 = __int_as_float(0x7f800000), m1 = m0;
#pragma unroll
                        for (int i = 4 * gq; i < 4 * gq + 4; ++i) {
                            const float4 e = e4[i];
                            m0 = min3f(m0, __fmaf_rd(-2.f, acc[4 * i + 0], e.x), __fmaf_rd(-2.f, acc[4 * i + 1], e.y));
                            m1 = min3f(m1, __fmaf_rd(-2.f, acc[4 * i + 2], e.z), __fmaf_rd(-2.f, acc[4 * i + 3], e.w));
                        }
                        mn[gq] = fminf(m0, m1);
                    }
                    const bool hit = min3f(mn[0], mn[1], fminf(mn[2], mn[3])) <= r;
                    if (__any_sync(0xffffffffu, hit)) {
                        // the groups some lane flagged, each pair re-tested in the
                        // kernel's rearranged form and queued for the candidate
                        // warp; unrolled so the accumulators stay in registers
#pragma unroll
                        for (int gq = 0; gq < 4; ++gq) {
                            if (!__any_sync(0xffffffffu, mn[gq] <= r)) continue;
#pragma unroll
                            for (int i = 16 * gq; i < 16 * gq + 16; ++i) {
                                const unsigned ql = cbeg + h + i;
                                cq_push(__fmaf_ru(2.f, acc[i], r) >= sE[ql], (unsigned)row, ql, acc[i], s_cq, s_cq_seq,
                                        &s_cq_tail, &s_cq_head, &s_fail);
                            }
                        }
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&bar_acce[ab]);
            if (warp == 0 && lane == 0) s_epi_tiles = (unsigned)(j + 1);   // progress, for the candidate warp
            // pick up bounds lowered by the other CTAs of these query tiles
            // (and repair an E_q that a race left looser than its U_q)
            if (own_act && (j & 63) == 63) {
                const unsigned G = ld_volatile_u32(&a.Ubits[own_qj]);
                const unsigned old = atomicMin(&sU[tid], G);
                sE[tid] = __fsub_rd(__fsub_rd(own_qn, own_gamma), __uint_as_float(min(old, G)));
            }
        }
        // this warp's entries are all published: tell the candidate warp
        __syncwarp();
        if (lane == 0) {
            __threadfence_block();
            atomicAdd(&s_epi_done, 1u);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0 && nt > 0) {
        // the MMA warp's final commit arrives once every MMA it issued has
        // finished (and after its earlier commits): wait for it before TMEM
        // and the barriers in shared memory are released
        const bool drained = mbar_wait_bounded(&bar_drain, 0);
        if (s_fail || !drained) {
            atomicOr(a.status, kStTimeout);
            // after a wait ran out, copies may also be in flight: the last
            // bulk-copy fill of every ring stage (fill f completes phase f of
            // its barrier) and the query tiles land first; each wait bounded
            for (unsigned i = 0; i < NS; ++i)
                if (s_fills[i]) mbar_wait_bounded(&bar_full[i], (s_fills[i] - 1u) & 1u);
            if (!qstream) mbar_wait_bounded(&bar_q, 0);
        }
    } else if (s_fail && tid == 0) {
        atomicOr(a.status, kStTimeout);
    }
    __syncthreads();
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

// Shared memory is always the full budget (kTcSmemBudget): one screen CTA per
// SM, because each CTA holds all 512 TMEM columns for its whole (persistent)
// life and a second resident CTA would wait in tcgen05.alloc forever.
size_t screen_smem_bytes(int len)
{
    (void)len;
    return kTcSmemBudget;
}

// ring stages that fit next to `qpc` resident query tiles (or, streamed, with
// their chunks inside each stage)
unsigned screen_stages(int len, unsigned qpc)
{
    const bool qstream = query_chunk((unsigned)len) != 0;
    const size_t chunk = (size_t)kTcRows * chunk_k((unsigned)len) * 2;
    const size_t stage = chunk * (qstream ? 1 + qpc : 1);
    const size_t q = qstream ? 0 : (size_t)qpc * kTcQ * len * 2;
    const size_t left = kTcSmemBudget > q ? kTcSmemBudget - q : 0;
    return (unsigned)std::min<size_t>(kTcMaxStages, left / stage);
}

void init_screen_attributes()
{
    cudaFuncSetAttribute(k_tc_screen<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmemBudget);
    cudaFuncSetAttribute(k_tc_screen<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmemBudget);
    cudaFuncSetAttribute(k_tc_screen<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmemBudget);
}

void launch_make_screen_copy(const float *raw, unsigned long long N, int len, __half *tiles, float *xn, float *xnorm,
                             unsigned *bad, cudaStream_t s)
{
    const unsigned long long RT = (N + kTcRows - 1) / kTcRows;
    const unsigned long long cap = (unsigned long long)num_sms() * 4;   // the resident CTAs
    k_make_screen_copy<<<(unsigned)std::max(1ull, std::min(RT, cap)), 256, 0, s>>>(raw, N, len, tiles, xn, xnorm, bad);
}

void launch_tc_qprep(const QuerySlot *slots, unsigned B, int len, const QueryParams &qp, __half *qtiles,
                     float *qconst, unsigned *Ubits, unsigned *cand_count, unsigned *flags, unsigned *active,
                     float *tkinit, unsigned *glock, uint2 *srange, cudaStream_t s)
{
    const unsigned padded = (B + kTcQ - 1) / kTcQ * kTcQ;
    k_tc_qprep<<<padded, 256, 0, s>>>(slots, B, len, qp, qtiles, qconst, Ubits, cand_count, flags, active, tkinit,
                                      glock, srange);
}

void launch_tc_next_pass(const QuerySlot *slots, unsigned B, const QueryParams &qp, unsigned cap, unsigned *Ubits,
                         unsigned *cand_count, unsigned *active, unsigned *n_active, const __half *qtiles,
                         __half *qtiles2, unsigned *qmap, int len, cudaStream_t s)
{
    k_tc_next_pass<<<(B + 255) / 256, 256, 0, s>>>(slots, B, qp, cap, Ubits, cand_count, active, n_active, qtiles,
                                                   qtiles2, qmap, len);
}

void launch_tc_screen(const __half *rtiles, const float *xn, const float *xnorm, const __half *qtiles,
                      const float *qconst, unsigned *Ubits, unsigned *cand_count, unsigned *cand_pos,
                      const unsigned *active, const unsigned *qmap, float *topk, unsigned *glock, int lists,
                      const uint2 *srange, unsigned cap, unsigned long long N, int len, unsigned B, int k,
                      unsigned *status, cudaStream_t s)
{
    ScreenArgs a;
    a.topk = topk;
    a.glock = glock;
    a.lists = lists;
    a.srange = srange;
    a.rtiles = rtiles;
    a.xn = xn;
    a.xnorm = xnorm;
    a.qtiles = qtiles;
    a.qconst = qconst;
    a.Ubits = Ubits;
    a.cand_count = cand_count;
    a.cand_pos = cand_pos;
    a.active = active;
    a.qmap = qmap;
    a.B = B;
    a.cap = cap;
    a.N = N;
    a.len = (unsigned)len;
    a.QT = (B + kTcQ - 1) / kTcQ;
    a.k = k;
    a.status = status;
    // two query tiles per CTA when they leave room for 4 ring stages: always
    // for len <= 256 (resident, 128 KB of tiles) and for every streamed length
    // (4 stages of 48 KB); one when the batch has a single query tile
    a.qpc = (a.QT >= 2 && screen_stages(len, 2) >= 4) ? 2u : 1u;
    a.stages = screen_stages(len, a.qpc);
    const unsigned QG = (a.QT + a.qpc - 1) / a.qpc;
    const unsigned groups = std::max(1u, (unsigned)num_sms() / QG);
    const unsigned ks = chunk_k((unsigned)len) / 16;
    if (ks == 4) k_tc_screen<4><<<groups * QG, kTcCtrlThreads, screen_smem_bytes(len), s>>>(a);
    else if (ks == 2) k_tc_screen<2><<<groups * QG, kTcCtrlThreads, screen_smem_bytes(len), s>>>(a);
    else k_tc_screen<1><<<groups * QG, kTcCtrlThreads, screen_smem_bytes(len), s>>>(a);
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
