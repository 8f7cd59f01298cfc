// summarize.cu -- PAA + SAX of every series (Sec. 2.2; ConvertToiSAX in
// Algorithm 3).
//
// One warp per pair of series.  Lanes read each row as float4 (coalesced), sum each
// segment in FP32 with shuffles and pick the symbol by binary search over
// FP32 copies of the breakpoints.  The symbol must equal the one an exact
// FP64 evaluation gives (PAA as the FP64 sequential sum divided by m, then
// symbol = #{beta_j <= PAA}), so the FP32 choice is kept only when the PAA
// lies farther from both edges of its region than a bound on the FP32
// summation error plus the FP32 rounding of the breakpoints; otherwise the
// lane recomputes that segment in FP64 in index order and decides again.
//
// Outputs per series: the iSAX word (uint4, byte s = symbol s), the 128-bit
// interleaved key (bit planes MSB first: bit p = j*w + s from the top holds
// bit (b-1-j) of symbol s) and the row id, which seed the radix sort.
#include "messi_internal.cuh"

namespace messi {
namespace {

constexpr int kSumThreads = 256;

// ((hi, lo) << sh) | v for 0 < sh < 64
__device__ __forceinline__ void shl128_or(unsigned long long &hi, unsigned long long &lo, int sh,
                                          unsigned long long v)
{
    hi = (hi << sh) | (lo >> (64 - sh));
    lo = (lo << sh) | v;
}

// Symbol of an FP64 PAA value: number of breakpoints <= p (upper region on
// equality).  sb64 holds card-1 values padded with +inf to 256.
__device__ __forceinline__ int symbol_fp64(double p, const double *sb64, int card)
{
    int lo = 0, hi = card - 1;   // answer in [0, card-1]
    while (lo < hi) {
        int mid = (lo + hi) >> 1;          // test breakpoint index mid (beta_{mid+1})
        if (sb64[mid] <= p) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ int symbol_fp32(float p, const float *sb32, int card)
{
    int lo = 0, hi = card - 1;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (sb32[mid] <= p) lo = mid + 1; else hi = mid;
    }
    return lo;
}

template <int M4>   // float4s per segment (m / 4); a power of two
__global__ void __launch_bounds__(kSumThreads)
k_summarize(const float *__restrict__ series, unsigned long long n, int len, int w, int card,
            int bits, const double *__restrict__ beta64, const float *__restrict__ beta32,
            uint4 *__restrict__ sax_out, uint4 *__restrict__ key_out,
            unsigned int *__restrict__ id_out, unsigned int *__restrict__ status)
{
    __shared__ float sb32[kMaxCard];
    __shared__ double sb64[kMaxCard];
    __shared__ float seg_sum[kSumThreads / 32][2 * kMaxSegments];
    __shared__ float seg_abs[kSumThreads / 32][2 * kMaxSegments];
    for (int i = threadIdx.x; i < kMaxCard; i += blockDim.x) {
        sb32[i] = i < card - 1 ? beta32[i] : __int_as_float(0x7f800000);
        sb64[i] = i < card - 1 ? beta64[i] : __longlong_as_double(0x7ff0000000000000ll);
    }
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const unsigned long long nwarps = (unsigned long long)gridDim.x * (blockDim.x >> 5);
    const int n4 = len >> 2;
    const int m = len / w;
    const int rounds = (n4 + 31) >> 5;
    // rows are taken two at a time: both are read and reduced as before, then
    // lanes 0-15 finish the first row and lanes 16-31 the second (symbols,
    // key, word), so the per-row work after the sums is shared by a pair
    const int half = lane >> 4, seg = lane & 15;

    for (unsigned long long pair = (unsigned long long)blockIdx.x * (blockDim.x >> 5) + wib; 2 * pair < n;
         pair += nwarps) {
        // the next pair of this warp: into L2 while this one is reduced
        {
            const unsigned long long nxt = 2 * (pair + nwarps);
            for (int i = lane * 32; i < 2 * len; i += 32 * 32)
                if (nxt * (unsigned long long)len + i < n * (unsigned long long)len)
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(series + nxt * (unsigned long long)len + i));
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const unsigned long long row = 2 * pair + h;
            if (row >= n) break;
            const float4 *x4 = reinterpret_cast<const float4 *>(series + row * (unsigned long long)len);
            float acc = 0.f, aac = 0.f;
            for (int t = 0; t < rounds; ++t) {
                int i = lane + 32 * t;
                float v = 0.f, a = 0.f;
                if (i < n4) {
                    float4 f = __ldg(x4 + i);
                    v = (f.x + f.y) + (f.z + f.w);
                    a = (fabsf(f.x) + fabsf(f.y)) + (fabsf(f.z) + fabsf(f.w));
                }
                if (M4 <= 32) {
#pragma unroll
                    for (int off = M4 / 2; off >= 1; off >>= 1) {
                        v += __shfl_xor_sync(0xffffffffu, v, off);
                        a += __shfl_xor_sync(0xffffffffu, a, off);
                    }
                    if ((lane & (M4 - 1)) == 0 && i < n4) {
                        seg_sum[wib][16 * h + i / M4] = v;
                        seg_abs[wib][16 * h + i / M4] = a;
                    }
                } else {
                    acc += v;
                    aac += a;
                    if (((t + 1) & (M4 / 32 - 1)) == 0) {
#pragma unroll
                        for (int off = 16; off >= 1; off >>= 1) {
                            acc += __shfl_xor_sync(0xffffffffu, acc, off);
                            aac += __shfl_xor_sync(0xffffffffu, aac, off);
                        }
                        if (lane == 0) {
                            seg_sum[wib][16 * h + (32 * t) / M4] = acc;
                            seg_abs[wib][16 * h + (32 * t) / M4] = aac;
                        }
                        acc = 0.f;
                        aac = 0.f;
                    }
                }
            }
        }
        __syncwarp();

        const unsigned long long row = 2 * pair + half;
        const bool has = seg < w && row < n;
        int sym = 0;
        if (has) {
            const float S = seg_sum[wib][lane];
            const float A = seg_abs[wib][lane];
            if (status && !(isfinite(S) && isfinite(A))) atomicOr(status, kStInvalidQuery);
            const float p = S / (float)m;                 // exact: m is a power of two
            sym = symbol_fp32(p, sb32, card);
            // |p - PAA_exact| <= (m-1) u A / m; the breakpoints carry <= u|beta|
            // rounding; the comparison below adds <= u of its own.
            const float marg = 1.01f * 5.9604645e-8f * (A + 2.f * fabsf(p) + 2.f) + 1e-30f;
            bool ok = true;
            if (sym > 0) ok = ok && (p - sb32[sym - 1] > marg);
            if (sym < card - 1) ok = ok && (sb32[sym] - p > marg);
            if (!ok) {
                const float *xs = series + row * (unsigned long long)len + seg * m;
                double sum = 0.0;
                for (int t = 0; t < m; ++t) sum = __dadd_rn(sum, (double)xs[t]);
                sym = symbol_fp64(__ddiv_rn(sum, (double)m), sb64, card);
            }
        }

        // interleaved key: for each bit plane j, the j-th most significant
        // bit of every segment's symbol, segment 0 first (each half of the
        // warp builds its own row's key from its 16 ballot bits)
        unsigned long long khi = 0ull, klo = 0ull;
        for (int j = 0; j < bits; ++j) {
            const unsigned mask = __ballot_sync(0xffffffffu, has && ((sym >> (bits - 1 - j)) & 1));
            const unsigned mh = half ? (mask >> 16) : (mask & 0xffffu);
            const unsigned field = __brev(mh) >> (32 - w);
            shl128_or(khi, klo, w, field);
        }
        const int used = w * bits;
        if (used < 128) {
            int sh = 128 - used;
            if (sh >= 64) { khi = klo << (sh - 64); klo = 0ull; }
            else { khi = (khi << sh) | (klo >> (64 - sh)); klo <<= sh; }
        }

        unsigned v = has ? ((unsigned)sym << (8 * (seg & 3))) : 0u;
        v |= __shfl_xor_sync(0xffffffffu, v, 1);
        v |= __shfl_xor_sync(0xffffffffu, v, 2);
        const int hb = lane & 16;
        unsigned w1 = __shfl_sync(0xffffffffu, v, hb + 4);
        unsigned w2 = __shfl_sync(0xffffffffu, v, hb + 8);
        unsigned w3 = __shfl_sync(0xffffffffu, v, hb + 12);
        if (seg == 0 && row < n) {
            sax_out[row] = make_uint4(v, w1, w2, w3);
            if (key_out)
                key_out[row] = make_uint4((unsigned)(khi >> 32), (unsigned)khi, (unsigned)(klo >> 32),
                                          (unsigned)klo);
            if (id_out) id_out[row] = (unsigned)row;
        }
        __syncwarp();
    }
}

}  // namespace

void launch_summarize(const float *series, unsigned long long n, int len, int w, int card,
                      const double *beta64, const float *beta32, uint4 *sax_out, uint4 *key_out,
                      unsigned int *id_out, unsigned int *status, cudaStream_t s)
{
    if (n == 0) return;
    int bits = 0;
    while ((1 << bits) < card) ++bits;
    const int m4 = (len / w) / 4;
    unsigned long long rows_per_block = 2 * (kSumThreads / 32);   // a pair of rows per warp
    unsigned long long want = (n + rows_per_block - 1) / rows_per_block;
    unsigned long long cap = (unsigned long long)num_sms() * 8;
    unsigned grid = (unsigned)(want < cap ? want : cap);
#define MESSI_SUM_CASE(M4)                                                                    \
    case M4:                                                                                  \
        k_summarize<M4><<<grid, kSumThreads, 0, s>>>(series, n, len, w, card, bits, beta64,   \
                                                     beta32, sax_out, key_out, id_out, status);       \
        break;
    switch (m4) {
        MESSI_SUM_CASE(1)
        MESSI_SUM_CASE(2)
        MESSI_SUM_CASE(4)
        MESSI_SUM_CASE(8)
        MESSI_SUM_CASE(16)
        MESSI_SUM_CASE(32)
        MESSI_SUM_CASE(64)
        MESSI_SUM_CASE(128)
        MESSI_SUM_CASE(256)
        MESSI_SUM_CASE(512)
        MESSI_SUM_CASE(1024)
        default: break;
    }
#undef MESSI_SUM_CASE
}

}  // namespace messi
