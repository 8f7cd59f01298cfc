// leaves.cu -- leaf grouping over the sorted interleaved keys, and the copy
// of the raw series into leaf order (Sec. 3.2, TreeConstruction in
// Algorithm 4; node splits as in Sec. 2.2).
//
// After the sort, every iSAX trie node is a contiguous run of keys that share
// a prefix.  The root's children are the runs of equal first-w-bit prefix
// (one bit per segment).  A node with more than `cap` series is replaced by
// its two children on the next interleaved bit -- the policy that refines
// the segments round-robin -- and empty children are dropped.  Nodes are
// split level by level: one thread per active node finds the split point by
// binary search (the bit is monotone inside a run that shares the prefix)
// and appends the children to the next level's list.  A node whose prefix is
// the whole key (identical words) stays a leaf whatever its size.
#include "messi_internal.cuh"

#include <algorithm>

namespace messi {
namespace {

struct Node {
    unsigned start, end, depth;
};

__global__ void k_root_flags(const uint4 *__restrict__ keys, unsigned long long n, int w,
                             unsigned *__restrict__ flags)
{
    unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsigned f = 1u;
    if (i > 0) f = (keys[i].x >> (32 - w)) != (keys[i - 1].x >> (32 - w));
    flags[i] = f;
}

__global__ void k_root_nodes(const unsigned *__restrict__ flags, const unsigned *__restrict__ idx,
                             unsigned long long n, int w, Node *__restrict__ nodes, unsigned nroots)
{
    unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !flags[i]) return;
    unsigned j = idx[i];
    nodes[j].start = (unsigned)i;
    nodes[j].depth = (unsigned)w;
    if (j > 0) nodes[j - 1].end = (unsigned)i;
    if (j == nroots - 1) nodes[j].end = (unsigned)n;
}

__device__ __forceinline__ unsigned key_bit(const uint4 &k, unsigned p)
{
    unsigned word = (p < 32) ? k.x : (p < 64) ? k.y : (p < 96) ? k.z : k.w;
    return (word >> (31 - (p & 31))) & 1u;
}

__global__ void k_split_level(const Node *__restrict__ in, const unsigned *__restrict__ count_in,
                              Node *__restrict__ out, unsigned *__restrict__ count_out,
                              const uint4 *__restrict__ keys, unsigned cap, unsigned total_bits,
                              unsigned *__restrict__ leaf_flag, unsigned char *__restrict__ depth_at)
{
    unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= *count_in) return;
    Node nd = in[i];
    unsigned size = nd.end - nd.start;
    if (size <= cap || nd.depth >= total_bits) {
        leaf_flag[nd.start] = 1u;
        depth_at[nd.start] = (unsigned char)nd.depth;
        return;
    }
    unsigned lo = nd.start, hi = nd.end;       // first index with bit `depth` set
    while (lo < hi) {
        unsigned mid = lo + ((hi - lo) >> 1);
        if (key_bit(keys[mid], nd.depth)) hi = mid; else lo = mid + 1;
    }
    if (lo > nd.start) {
        unsigned j = atomicAdd(count_out, 1u);
        out[j] = Node{nd.start, lo, nd.depth + 1};
    }
    if (nd.end > lo) {
        unsigned j = atomicAdd(count_out, 1u);
        out[j] = Node{lo, nd.end, nd.depth + 1};
    }
}

__global__ void k_make_leaves(const unsigned *__restrict__ flags, const unsigned *__restrict__ idx,
                              const unsigned char *__restrict__ depth_at, const uint4 *__restrict__ keys,
                              unsigned long long n, unsigned long long *__restrict__ leaf_off,
                              uint4 *__restrict__ leaf_key, unsigned char *__restrict__ leaf_depth,
                              unsigned long long L)
{
    unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) leaf_off[L] = n;
    if (i >= n || !flags[i]) return;
    unsigned l = idx[i];
    leaf_off[l] = i;
    leaf_key[l] = keys[i];
    leaf_depth[l] = depth_at[i];
}

// Per-leaf symbol box: for every segment the smallest and largest symbol of
// the leaf's words (one warp per leaf, bytewise min / max over its rows).
// Every word of the leaf lies in the box, so the table minimum over the box
// bounds all of them from below.
__global__ void __launch_bounds__(256)
k_leaf_boxes(const uint4 *__restrict__ sax, const unsigned long long *__restrict__ leaf_off, unsigned long long L,
             uint4 *__restrict__ box)
{
    const int lane = threadIdx.x & 31;
    const unsigned long long nw = (unsigned long long)gridDim.x * (blockDim.x >> 5);
    for (unsigned long long l = (unsigned long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); l < L;
         l += nw) {
        const unsigned long long a = leaf_off[l], b = leaf_off[l + 1];
        uint4 mn = make_uint4(0xffffffffu, 0xffffffffu, 0xffffffffu, 0xffffffffu), mx = make_uint4(0, 0, 0, 0);
        for (unsigned long long i = a + lane; i < b; i += 32) {
            const uint4 w = sax[i];
            mn = make_uint4(__vminu4(mn.x, w.x), __vminu4(mn.y, w.y), __vminu4(mn.z, w.z), __vminu4(mn.w, w.w));
            mx = make_uint4(__vmaxu4(mx.x, w.x), __vmaxu4(mx.y, w.y), __vmaxu4(mx.z, w.z), __vmaxu4(mx.w, w.w));
        }
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) {
            mn.x = __vminu4(mn.x, __shfl_xor_sync(0xffffffffu, mn.x, off));
            mn.y = __vminu4(mn.y, __shfl_xor_sync(0xffffffffu, mn.y, off));
            mn.z = __vminu4(mn.z, __shfl_xor_sync(0xffffffffu, mn.z, off));
            mn.w = __vminu4(mn.w, __shfl_xor_sync(0xffffffffu, mn.w, off));
            mx.x = __vmaxu4(mx.x, __shfl_xor_sync(0xffffffffu, mx.x, off));
            mx.y = __vmaxu4(mx.y, __shfl_xor_sync(0xffffffffu, mx.y, off));
            mx.z = __vmaxu4(mx.z, __shfl_xor_sync(0xffffffffu, mx.z, off));
            mx.w = __vmaxu4(mx.w, __shfl_xor_sync(0xffffffffu, mx.w, off));
        }
        if (lane == 0) {
            box[2 * l] = mn;
            box[2 * l + 1] = mx;
        }
    }
}

__global__ void k_max_leaf(const unsigned long long *__restrict__ leaf_off, unsigned long long L,
                           unsigned long long *__restrict__ out)
{
    unsigned long long l = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= L) return;
    atomicMax(out, leaf_off[l + 1] - leaf_off[l]);
}

// one warp per position: copy row ids[pos] of the input into raw[pos]
__global__ void __launch_bounds__(256)
k_permute(const float *__restrict__ series, const unsigned *__restrict__ ids, const uint4 *__restrict__ sax_in,
          unsigned long long n, int len, float *__restrict__ raw, uint4 *__restrict__ sax,
          unsigned *__restrict__ pos_of_id)
{
    const int lane = threadIdx.x & 31;
    const unsigned long long nwarps = (unsigned long long)gridDim.x * (blockDim.x >> 5);
    const int n4 = len >> 2;
    for (unsigned long long pos = (unsigned long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
         pos < n; pos += nwarps) {
        unsigned id = ids[pos];
        const float4 *src = reinterpret_cast<const float4 *>(series + (unsigned long long)id * len);
        float4 *dst = reinterpret_cast<float4 *>(raw + pos * len);
        for (int i = lane; i < n4; i += 32) dst[i] = __ldg(src + i);
        if (lane == 0) {
            sax[pos] = sax_in[id];
            pos_of_id[id] = (unsigned)pos;
        }
    }
}

template <typename T>
bool dalloc(T **p, size_t count, std::vector<void *> &owned)
{
    void *q = nullptr;
    if (cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    owned.push_back(q);
    *p = static_cast<T *>(q);
    return true;
}

}  // namespace

messi_status build_leaves(messi_index *ix, const uint4 *keys, const uint4 *sax_unsorted,
                          const float *series, cudaStream_t s)
{
    const unsigned long long n = ix->N;
    const unsigned total_bits = (unsigned)(ix->w * ix->bits);
    std::vector<void *> tmp;
    auto cleanup = [&]() {
        for (void *p : tmp) cudaFree(p);
        tmp.clear();
    };

    unsigned *flags = nullptr, *idx = nullptr, *counts = nullptr;
    unsigned char *depth_at = nullptr;
    void *scan_tmp = nullptr;
    const unsigned long long roots_max = std::min<unsigned long long>(n, 1ull << ix->w);
    const unsigned long long nodes_max =
        std::max<unsigned long long>(roots_max, 2ull * ((n + ix->cap) / (ix->cap + 1ull))) + 16;
    Node *na = nullptr, *nb = nullptr;
    if (!dalloc(&flags, n, tmp) || !dalloc(&idx, n, tmp) || !dalloc(&counts, 4, tmp) ||
        !dalloc(&depth_at, n, tmp) || !dalloc((char **)&scan_tmp, scan_temp_bytes(n), tmp) ||
        !dalloc(&na, nodes_max, tmp) || !dalloc(&nb, nodes_max, tmp)) {
        cleanup();
        return fail(MESSI_ENOMEM, "messi_build: cannot allocate leaf-building temporaries");
    }
    const unsigned tpb = 256;
    const unsigned nblk = (unsigned)((n + tpb - 1) / tpb);

    // root children
    k_root_flags<<<nblk, tpb, 0, s>>>(keys, n, ix->w, flags);
    exclusive_scan_u32(flags, idx, n, scan_tmp, s, &ix->launches);
    unsigned last_idx = 0, last_flag = 0;
    MESSI_CUDA(cudaMemcpyAsync(&last_idx, idx + n - 1, 4, cudaMemcpyDeviceToHost, s));
    MESSI_CUDA(cudaMemcpyAsync(&last_flag, flags + n - 1, 4, cudaMemcpyDeviceToHost, s));
    MESSI_CUDA(cudaStreamSynchronize(s));
    unsigned nroots = last_idx + last_flag;
    k_root_nodes<<<nblk, tpb, 0, s>>>(flags, idx, n, ix->w, na, nroots);
    ix->launches += 2;

    // split level by level
    MESSI_CUDA(cudaMemsetAsync(flags, 0, n * sizeof(unsigned), s));
    MESSI_CUDA(cudaMemcpyAsync(counts, &nroots, 4, cudaMemcpyHostToDevice, s));
    unsigned active = nroots;
    int cur = 0;
    for (int level = 0; active > 0 && level <= 130; ++level) {
        MESSI_CUDA(cudaMemsetAsync(counts + 1 - cur, 0, 4, s));
        Node *in = cur ? nb : na, *out = cur ? na : nb;
        k_split_level<<<(active + tpb - 1) / tpb, tpb, 0, s>>>(in, counts + cur, out, counts + 1 - cur,
                                                               keys, ix->cap, total_bits, flags, depth_at);
        ++ix->launches;
        MESSI_CUDA(cudaMemcpyAsync(&active, counts + 1 - cur, 4, cudaMemcpyDeviceToHost, s));
        MESSI_CUDA(cudaStreamSynchronize(s));
        cur = 1 - cur;
    }
    if (active != 0) {
        cleanup();
        return fail(MESSI_ECUDA, "messi_build: leaf splitting did not terminate");
    }

    // leaf table
    exclusive_scan_u32(flags, idx, n, scan_tmp, s, &ix->launches);
    MESSI_CUDA(cudaMemcpyAsync(&last_idx, idx + n - 1, 4, cudaMemcpyDeviceToHost, s));
    MESSI_CUDA(cudaMemcpyAsync(&last_flag, flags + n - 1, 4, cudaMemcpyDeviceToHost, s));
    MESSI_CUDA(cudaStreamSynchronize(s));
    const unsigned long long L = (unsigned long long)last_idx + last_flag;
    ix->L = L;
    if (cudaMalloc(&ix->leaf_off, (L + 1) * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc(&ix->leaf_key, L * sizeof(uint4)) != cudaSuccess ||
        cudaMalloc(&ix->leaf_depth, L) != cudaSuccess || cudaMalloc(&ix->leaf_box, L * 2 * sizeof(uint4)) != cudaSuccess) {
        cudaGetLastError();
        cleanup();
        return fail(MESSI_ENOMEM, "messi_build: cannot allocate the leaf table");
    }
    ix->device_bytes += (L + 1) * 8 + L * 17 + L * 32;
    k_make_leaves<<<nblk, tpb, 0, s>>>(flags, idx, depth_at, keys, n, ix->leaf_off, ix->leaf_key,
                                       ix->leaf_depth, L);
    unsigned long long *dmax = reinterpret_cast<unsigned long long *>(counts);
    MESSI_CUDA(cudaMemsetAsync(dmax, 0, 8, s));
    k_max_leaf<<<(unsigned)((L + tpb - 1) / tpb), tpb, 0, s>>>(ix->leaf_off, L, dmax);
    MESSI_CUDA(cudaMemcpyAsync(&ix->max_leaf, dmax, 8, cudaMemcpyDeviceToHost, s));

    // raw series and iSAX words in leaf order
    unsigned long long want = (n + 7) / 8;
    unsigned long long capb = (unsigned long long)num_sms() * 16;
    k_permute<<<(unsigned)std::min(want, capb), 256, 0, s>>>(series, ix->ids, sax_unsorted, n, ix->len,
                                                             ix->raw, ix->sax, ix->pos_of_id);
    const unsigned long long bw = (L + 7) / 8;
    k_leaf_boxes<<<(unsigned)std::min(bw, capb), 256, 0, s>>>(ix->sax, ix->leaf_off, L, ix->leaf_box);
    ix->launches += 4;
    MESSI_CUDA(cudaStreamSynchronize(s));
    cleanup();
    return MESSI_OK;
}

}  // namespace messi
