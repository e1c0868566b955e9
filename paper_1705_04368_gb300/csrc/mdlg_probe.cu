// mdlg_probe.cu -- measurement probes for the roofline denominators: a
// binary32 fused multiply-add loop (the CUDA-core peak the force kernel is
// compared with) and a streaming copy (the HBM bandwidth the binning kernels
// are compared with).  The paper has no counterpart; nothing of the method
// runs here.
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/mdlg.h"

namespace {

constexpr int kFmaChains = 8;   // independent accumulators per thread

// Every thread runs kFmaChains independent chains a <- a * b + c, `iters`
// times each, then stores their sum so that no chain can be removed.
__global__ void __launch_bounds__(256) k_probe_fma(int64_t iters, float b, float c, float *out) {
    float a[kFmaChains];
#pragma unroll
    for (int k = 0; k < kFmaChains; ++k) a[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (int64_t t = 0; t < iters; ++t) {
#pragma unroll
        for (int k = 0; k < kFmaChains; ++k) a[k] = fmaf(a[k], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kFmaChains; ++k) s += a[k];
    out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Grid-stride copy of 16-byte words, four independent words per thread and trip.
__global__ void __launch_bounds__(256) k_probe_copy(const uint4 *__restrict__ src, uint4 *__restrict__ dst,
                                                    int64_t words) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + 3 * stride < words; i += 4 * stride) {
        const uint4 w0 = src[i], w1 = src[i + stride], w2 = src[i + 2 * stride], w3 = src[i + 3 * stride];
        dst[i] = w0;
        dst[i + stride] = w1;
        dst[i + 2 * stride] = w2;
        dst[i + 3 * stride] = w3;
    }
    for (; i < words; i += stride) dst[i] = src[i];
}

}  // namespace

extern "C" {

int mdlg_probe_fma(int32_t blocks, int32_t threads, int64_t iters, float *out, double *flops,
                   void *stream) {
    if (blocks < 1 || threads < 32 || threads > 256 || threads % 32 || iters < 1 || !out)
        return MDLG_EINVAL;
    k_probe_fma<<<blocks, threads, 0, static_cast<cudaStream_t>(stream)>>>(iters, 0.999999f, 1e-7f, out);
    if (flops) *flops = 2.0 * kFmaChains * (double)iters * (double)blocks * (double)threads;
    return cudaGetLastError() == cudaSuccess ? MDLG_OK : MDLG_ECUDA;
}

int mdlg_probe_copy(const void *src, void *dst, int64_t bytes, void *stream) {
    if (!src || !dst || bytes < 0 || bytes % 16 ||
        ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15))
        return MDLG_EINVAL;
    if (bytes == 0) return MDLG_OK;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t words = bytes / 16;
    int64_t blocks = (words + 255) / 256;
    if (blocks > (int64_t)sms * 8) blocks = (int64_t)sms * 8;
    k_probe_copy<<<(unsigned)blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const uint4 *>(src), static_cast<uint4 *>(dst), words);
    return cudaGetLastError() == cudaSuccess ? MDLG_OK : MDLG_ECUDA;
}

}  // extern "C"
