// radix_sort.cu -- device LSD radix sort of 128-bit interleaved iSAX keys with
// a 32-bit payload, and an exclusive prefix sum.
//
// The paper groups series into root subtrees through per-worker iSAX buffers
// and splits leaves one series at a time (Sec. 3.2, Algorithms 3 and 4).  On
// the GPU the same grouping falls out of one sort: once the keys are sorted,
// every node of the iSAX trie (a key prefix) is a contiguous run.
//
// Each pass sorts by one 8-bit digit and is stable, so passes from the least
// significant used byte up give (key, original id) order.  A pass is
//   1. per-tile digit histograms (tile = 4096 items),
//   2. an exclusive scan over the digit-major histogram table,
//   3. a stable scatter: inside a tile, items are ranked by (warp, round,
//      lane) with __match_any_sync, so equal digits keep their input order,
//      sorted within the tile in shared memory and written out digit run by
//      digit run.
#include "messi_internal.cuh"

namespace messi {
namespace {

constexpr int kRsThreads = 256;
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kRsRounds = 16;
constexpr int kRsTile = kRsThreads * kRsRounds;   // 4096 items
constexpr int kScanThreads = 256;
constexpr int kScanIpt = 16;
constexpr int kScanChunk = kScanThreads * kScanIpt;

__device__ __forceinline__ unsigned digit_of(const uint4 &k, int byte)
{
    // byte 0 is the least significant byte of the 128-bit key; .x holds the
    // most significant word
    unsigned word = (byte < 4) ? k.w : (byte < 8) ? k.z : (byte < 12) ? k.y : k.x;
    return (word >> (8 * (byte & 3))) & 0xffu;
}

__global__ void __launch_bounds__(kRsThreads)
k_hist(const uint4 *__restrict__ keys, unsigned long long n, int byte, unsigned int *__restrict__ hist,
       unsigned long long ntiles)
{
    __shared__ unsigned h[256];
    h[threadIdx.x] = 0u;
    __syncthreads();
    const unsigned long long base = (unsigned long long)blockIdx.x * kRsTile;
#pragma unroll 4
    for (int r = 0; r < kRsRounds; ++r) {
        unsigned long long idx = base + (unsigned long long)r * kRsThreads + threadIdx.x;
        if (idx < n) atomicAdd(&h[digit_of(keys[idx], byte)], 1u);
    }
    __syncthreads();
    hist[(unsigned long long)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter of one tile through shared memory: the tile's keys and
// payloads are staged in input order (coalesced), each item gets its place
// in the tile sorted by digit -- the digit's start in the tile, plus the
// items of that digit in earlier warps, plus its rank among the warp's equal
// digits (ranked by round, then lane, so input order is kept) -- and the
// sorted tile is written out so that consecutive threads write consecutive
// addresses of a digit's run.
constexpr int kRsSmem = kRsTile * 16 + kRsTile * 4 + kRsTile * 2;   // keys, payloads, local permutation

__global__ void __launch_bounds__(kRsThreads, 2)
k_scatter(const uint4 *__restrict__ keys, const unsigned int *__restrict__ vals, uint4 *__restrict__ keys_out,
          unsigned int *__restrict__ vals_out, unsigned long long n, int byte,
          const unsigned int *__restrict__ offs, unsigned long long ntiles)
{
    extern __shared__ __align__(16) unsigned char rsm[];
    uint4 *sk = reinterpret_cast<uint4 *>(rsm);
    unsigned *sv = reinterpret_cast<unsigned *>(rsm + kRsTile * 16);
    unsigned short *perm = reinterpret_cast<unsigned short *>(rsm + kRsTile * 20);
    __shared__ unsigned whist[kRsWarps][256];
    __shared__ unsigned lstart[256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned long long tbase = (unsigned long long)blockIdx.x * kRsTile;
    const unsigned tn = (unsigned)min((unsigned long long)kRsTile, n - tbase);
    for (unsigned i = threadIdx.x; i < tn; i += kRsThreads) {
        sk[i] = keys[tbase + i];
        sv[i] = vals[tbase + i];
    }
    for (int d = lane; d < 256; d += 32) whist[warp][d] = 0u;
    __syncthreads();
    // ranks within the warp: items warp*512 + r*32 + lane of the tile
    const unsigned lt = (1u << lane) - 1u;
    unsigned dr[kRsRounds];   // digit << 16 | rank
#pragma unroll
    for (int r = 0; r < kRsRounds; ++r) {
        const unsigned i = warp * 32 * kRsRounds + r * 32 + lane;
        const bool valid = i < tn;
        const unsigned d = valid ? digit_of(sk[i], byte) : 256u;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        unsigned before = 0u;
        if (valid) before = whist[warp][d];
        __syncwarp();
        dr[r] = (d << 16) | (before + __popc(peers & lt));
        if (valid && (__ffs(peers) - 1) == lane) whist[warp][d] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    {
        // per digit (one per thread): earlier warps' counts, and the tile total
        const int d = threadIdx.x;
        unsigned run = 0u;
#pragma unroll
        for (int w = 0; w < kRsWarps; ++w) {
            const unsigned t = whist[w][d];
            whist[w][d] = run;
            run += t;
        }
        lstart[d] = run;   // the digit's count for now
    }
    __syncthreads();
    if (warp == 0) {
        // exclusive scan of the 256 digit counts, 8 per lane
        unsigned c[8], sum = 0u;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            c[j] = lstart[lane * 8 + j];
            sum += c[j];
        }
        unsigned inc = sum;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, inc, off);
            if (lane >= off) inc += y;
        }
        unsigned run = inc - sum;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            lstart[lane * 8 + j] = run;
            run += c[j];
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kRsRounds; ++r) {
        const unsigned i = warp * 32 * kRsRounds + r * 32 + lane;
        if (i < tn) {
            const unsigned d = dr[r] >> 16;
            perm[lstart[d] + whist[warp][d] + (dr[r] & 0xffffu)] = (unsigned short)i;
        }
    }
    __syncthreads();
    for (unsigned i = threadIdx.x; i < tn; i += kRsThreads) {
        const unsigned src = perm[i];
        const uint4 k = sk[src];
        const unsigned d = digit_of(k, byte);
        const unsigned long long dst = (unsigned long long)offs[(unsigned long long)d * ntiles + blockIdx.x] + (i - lstart[d]);
        keys_out[dst] = k;
        vals_out[dst] = sv[src];
    }
}

// ------------------------------------------------------------------ scan
__device__ __forceinline__ unsigned block_exclusive_scan(unsigned x, unsigned *total)
{
    __shared__ unsigned wsum[kScanThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned inc = x;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        unsigned y = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc += y;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        unsigned s = lane < kScanThreads / 32 ? wsum[lane] : 0u;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            unsigned y = __shfl_up_sync(0xffffffffu, s, off);
            if (lane >= off) s += y;
        }
        if (lane < kScanThreads / 32) wsum[lane] = s;      // inclusive warp totals
    }
    __syncthreads();
    unsigned warp_off = warp ? wsum[warp - 1] : 0u;
    *total = wsum[kScanThreads / 32 - 1];
    __syncthreads();
    return warp_off + inc - x;
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_reduce(const unsigned *__restrict__ in, unsigned long long n, unsigned *__restrict__ sums)
{
    unsigned long long base = (unsigned long long)blockIdx.x * kScanChunk + (unsigned long long)threadIdx.x * kScanIpt;
    unsigned s = 0u;
#pragma unroll
    for (int i = 0; i < kScanIpt; ++i)
        if (base + i < n) s += in[base + i];
    unsigned total;
    block_exclusive_scan(s, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// single block: exclusive scan of the per-chunk sums, in place
__global__ void __launch_bounds__(kScanThreads) k_scan_top(unsigned *sums, unsigned long long nb)
{
    unsigned carry = 0u;
    for (unsigned long long lo = 0; lo < nb; lo += kScanThreads) {
        unsigned long long i = lo + threadIdx.x;
        unsigned x = i < nb ? sums[i] : 0u;
        unsigned total;
        unsigned ex = block_exclusive_scan(x, &total);
        if (i < nb) sums[i] = carry + ex;
        carry += total;
    }
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_down(const unsigned *__restrict__ in, unsigned *__restrict__ out, unsigned long long n,
            const unsigned *__restrict__ sums)
{
    unsigned long long base = (unsigned long long)blockIdx.x * kScanChunk + (unsigned long long)threadIdx.x * kScanIpt;
    unsigned vals[kScanIpt];
    unsigned s = 0u;
#pragma unroll
    for (int i = 0; i < kScanIpt; ++i) {
        vals[i] = (base + i < n) ? in[base + i] : 0u;
        s += vals[i];
    }
    unsigned total;
    unsigned ex = block_exclusive_scan(s, &total) + sums[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kScanIpt; ++i) {
        if (base + i < n) out[base + i] = ex;
        ex += vals[i];
    }
}

}  // namespace

size_t scan_temp_bytes(unsigned long long n)
{
    unsigned long long nb = (n + kScanChunk - 1) / kScanChunk;
    return (size_t)(nb + 1) * sizeof(unsigned);
}

void exclusive_scan_u32(const unsigned int *in, unsigned int *out, unsigned long long n, void *temp,
                        cudaStream_t s, unsigned long long *launches)
{
    if (n == 0) return;
    unsigned long long nb = (n + kScanChunk - 1) / kScanChunk;
    unsigned *sums = static_cast<unsigned *>(temp);
    k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, sums);
    k_scan_top<<<1, kScanThreads, 0, s>>>(sums, nb);
    k_scan_down<<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, sums);
    if (launches) *launches += 3;
}

size_t radix_sort_temp_bytes(unsigned long long n)
{
    unsigned long long ntiles = (n + kRsTile - 1) / kRsTile;
    unsigned long long entries = 256ull * ntiles;
    size_t b = (size_t)entries * sizeof(unsigned) * 2;
    b = (b + 255) & ~(size_t)255;
    return b + scan_temp_bytes(entries);
}

void radix_sort_keys(uint4 *keys, unsigned int *vals, uint4 *keys_alt, unsigned int *vals_alt,
                     unsigned long long n, int key_bits, void *temp, cudaStream_t s,
                     unsigned long long *launches)
{
    if (n <= 1) return;
    unsigned long long ntiles = (n + kRsTile - 1) / kRsTile;
    unsigned long long entries = 256ull * ntiles;
    unsigned *hist = static_cast<unsigned *>(temp);
    unsigned *offs = hist + entries;
    size_t b = (size_t)entries * sizeof(unsigned) * 2;
    b = (b + 255) & ~(size_t)255;
    void *scan_tmp = static_cast<char *>(temp) + b;

    static bool attr_set[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !attr_set[dev]) {
        cudaFuncSetAttribute(k_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, kRsSmem);
        attr_set[dev] = true;
    }
    int first = (128 - key_bits) / 8;          // least significant byte holding used bits
    uint4 *ki = keys, *ko = keys_alt;
    unsigned *vi = vals, *vo = vals_alt;
    int passes = 0;
    for (int byte = first; byte < 16; ++byte, ++passes) {
        k_hist<<<(unsigned)ntiles, kRsThreads, 0, s>>>(ki, n, byte, hist, ntiles);
        exclusive_scan_u32(hist, offs, entries, scan_tmp, s, launches);
        k_scatter<<<(unsigned)ntiles, kRsThreads, kRsSmem, s>>>(ki, vi, ko, vo, n, byte, offs, ntiles);
        if (launches) *launches += 2;
        uint4 *tk = ki; ki = ko; ko = tk;
        unsigned *tv = vi; vi = vo; vo = tv;
    }
    if (passes & 1) {
        cudaMemcpyAsync(keys, keys_alt, n * sizeof(uint4), cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(vals, vals_alt, n * sizeof(unsigned), cudaMemcpyDeviceToDevice, s);
    }
}

}  // namespace messi
