// Device copy kernel used to measure the copy bandwidth of HBM and of L2 in
// the same process as the search (the roofline denominators).
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/mbe.h"

namespace mbe {
namespace {

__global__ void copy_kernel(const int4 *__restrict__ src, int4 *__restrict__ dst, int64_t n)
{
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) dst[i] = src[i];
}

} // namespace
} // namespace mbe

extern "C" int mbe_copy_bandwidth(int64_t bytes, int32_t iters, void *stream, double *gbps)
{
    if (!gbps || bytes < (1 << 20) || (bytes & 15) || iters < 1) return MBE_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int4 *a = nullptr, *b = nullptr;
    if (cudaMalloc(&a, (size_t)bytes) != cudaSuccess || cudaMalloc(&b, (size_t)bytes) != cudaSuccess) {
        cudaFree(a);
        cudaGetLastError();
        return MBE_ERR_OOM;
    }
    cudaMemsetAsync(a, 1, (size_t)bytes, s);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int64_t n = bytes / 16;
    float best = 1e30f;
    for (int it = 0; it < iters + 1; ++it) { // first iteration warms up
        cudaEventRecord(e0, s);
        mbe::copy_kernel<<<sms * 4, 512, 0, s>>>(a, b, n);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (it > 0) best = std::min(best, ms);
    }
    cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(a);
    cudaFree(b);
    if (err != cudaSuccess) return MBE_ERR_CUDA;
    *gbps = 2.0 * (double)bytes / (best * 1e-3) / 1e9;
    return MBE_OK;
}
