// windows.cu -- sliding-window subsequences of one long series.
//
// MESSI answers whole-matching queries over a collection of equal-length
// series; a streaming or long series is first cut into subsequences of the
// query's length by a sliding window, and those are indexed (Sec. 2, and the
// subsequence-matching adaptation of Sec. 6).  This file produces that
// collection on the device: window i is series[i * stride, i * stride + n),
// optionally z-normalised (mean 0, standard deviation 1, the normalisation
// of Sec. 2).  The normalisation is specified operation by operation in FP64
// with round-to-nearest (no contraction), so any other implementation of the
// same steps produces the same float32 rows bit for bit:
//   mean = (x_0 + x_1 + ... + x_{n-1}, summed left to right) / n
//   var  = ((x_0 - mean)^2 + ... + (x_{n-1} - mean)^2, left to right) / n
//   inv  = 1 / sqrt(var), or 0 when var = 0 (a constant window)
//   out_j = float32(round((x_j - mean) * inv))
#include <algorithm>

#include "messi_internal.cuh"

namespace messi {
namespace {

constexpr int kWinBlock = 128;          // windows per block iteration
constexpr uint32_t kWinMaxLen = 65536;  // block-local element counts stay in 32 bits

// One thread per window computes its mean and 1/std (two sequential FP64
// passes; neighbouring threads read neighbouring windows, so the loads of a
// warp are coalesced for stride 1 and cached for larger strides); then the
// block writes its windows row by row with consecutive threads on consecutive
// elements.
__global__ void __launch_bounds__(kWinBlock)
k_windows(const float *__restrict__ series, unsigned long long count, unsigned n, unsigned stride, int znorm,
          float *__restrict__ out)
{
    __shared__ double s_mean[kWinBlock], s_inv[kWinBlock];
    for (unsigned long long base = (unsigned long long)blockIdx.x * kWinBlock; base < count;
         base += (unsigned long long)gridDim.x * kWinBlock) {
        const unsigned long long i = base + threadIdx.x;
        double mean = 0.0, inv = 0.0;
        if (znorm && i < count) {
            const float *x = series + i * stride;
            double s = 0.0;
            for (unsigned j = 0; j < n; ++j) s = __dadd_rn(s, (double)__ldg(x + j));
            mean = __ddiv_rn(s, (double)n);
            double v = 0.0;
            for (unsigned j = 0; j < n; ++j) {
                const double d = __dsub_rn((double)__ldg(x + j), mean);
                v = __dadd_rn(v, __dmul_rn(d, d));
            }
            v = __ddiv_rn(v, (double)n);
            inv = v > 0.0 ? __ddiv_rn(1.0, __dsqrt_rn(v)) : 0.0;
        }
        s_mean[threadIdx.x] = mean;
        s_inv[threadIdx.x] = inv;
        __syncthreads();
        const unsigned nw = (unsigned)min((unsigned long long)kWinBlock, count - base);
        for (unsigned w = 0; w < nw; ++w) {
            const float *x = series + (base + w) * stride;
            float *o = out + (base + w) * n;
            const double m = s_mean[w], r = s_inv[w];
            for (unsigned j = threadIdx.x; j < n; j += kWinBlock) {
                const float v = __ldg(x + j);
                o[j] = znorm ? __double2float_rn(__dmul_rn(__dsub_rn((double)v, m), r)) : v;
            }
        }
        __syncthreads();
    }
}

bool device_pointer(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace messi

using namespace messi;

extern "C" messi_status messi_windows(const float *series, uint64_t length, uint32_t n, uint32_t stride,
                                      int32_t znorm, float *out, uint64_t *count, messi_stream stream)
{
    if (!series || !out) return fail(MESSI_EINVAL, "messi_windows: null argument");
    if (n == 0 || n > kWinMaxLen || stride == 0)
        return fail(MESSI_EINVAL, "messi_windows: n must be in 1..65536 and stride at least 1");
    if (length < n) return fail(MESSI_EINVAL, "messi_windows: the series is shorter than one window");
    if (!device_pointer(series) || !device_pointer(out))
        return fail(MESSI_EINVAL, "messi_windows: series and out must be device pointers");
    const unsigned long long W = (length - n) / stride + 1;
    const unsigned long long blocks = std::min<unsigned long long>((W + kWinBlock - 1) / kWinBlock,
                                                                   (unsigned long long)num_sms() * 16);
    k_windows<<<(unsigned)blocks, kWinBlock, 0, static_cast<cudaStream_t>(stream)>>>(series, W, n, stride,
                                                                                    znorm ? 1 : 0, out);
    if (!cuda_ok(cudaGetLastError(), "messi_windows: launch")) return MESSI_ECUDA;
    if (count) *count = W;
    return MESSI_OK;
}
