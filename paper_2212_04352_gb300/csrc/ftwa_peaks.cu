// Micro-benchmarks of the on-chip peaks the stepper is measured against:
// FP32 and FP64 fused multiply-add throughput and shared-memory load
// bandwidth.  These are not part of the method; they supply the roofline
// denominators that a driver-side STREAM copy and cuBLAS GEMM do not cover.
#include <cuda_runtime.h>

#include <algorithm>

#include "ftwa_internal.h"

namespace ftwa {
namespace peaks {

constexpr int kChains = 16;   // independent FMA chains per thread

template <typename T>
__global__ void __launch_bounds__(256) fma_kernel(T *out, int iters, T a, T b)
{
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == (T)-1.2345) out[blockIdx.x] = s;   // keeps the chains live
}

// FP32 with packed pairs (two FMAs per instruction, the form the stepper uses)
__global__ void __launch_bounds__(256) ffma2_kernel(float *out, int iters, float a, float b)
{
    float2 x[kChains / 2];
#pragma unroll
    for (int c = 0; c < kChains / 2; ++c) x[c] = make_float2((float)threadIdx.x + c, (float)c);
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains / 2; ++c) x[c] = __ffma2_rn(x[c], a2, b2);
    }
    float s = 0;
#pragma unroll
    for (int c = 0; c < kChains / 2; ++c) s += x[c].x + x[c].y;
    if (s == -1.2345f) out[blockIdx.x] = s;
}

// shared-memory loads: each warp streams 16-byte vectors, conflict-free
__global__ void __launch_bounds__(1024) smem_kernel(float *out, int iters)
{
    extern __shared__ float4 buf[];
    const int n = 4096;   // 64 KB: two CTAs per SM
    for (int i = threadIdx.x; i < n; i += blockDim.x) buf[i] = make_float4((float)i, 1.f, 2.f, 3.f);
    __syncthreads();
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    int idx = threadIdx.x;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const float4 v = buf[(idx + u * 512) & (n - 1)];   // eight distinct vectors
            acc.x += v.x;
            acc.y += v.y;
            acc.z += v.z;
            acc.w += v.w;
        }
        idx = (idx + 32) & (n - 1);
    }
    if (acc.x + acc.y + acc.z + acc.w == -1.2345f) out[blockIdx.x] = acc.x;
}

}  // namespace peaks
}  // namespace ftwa

extern "C" int ftwa_measure_peak(int32_t kind, double *value, void *stream)
{
    using namespace ftwa;
    using namespace ftwa::peaks;
    if (!value || kind < 0 || kind > 3) return FTWA_ERR_INVALID_ARGUMENT;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FTWA_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return FTWA_ERR_CUDA;
    cudaError_t e = cudaSuccess;
    if (kind == 2) {
        e = cudaFuncSetAttribute(smem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 4096 * 16);
        if (e != cudaSuccess) return set_cuda_error(e);
    }
    float *sink = nullptr;
    e = cudaMalloc(&sink, sizeof(double) * 65536);
    if (e != cudaSuccess) return set_cuda_error(e);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int blocks_fma = sms * 8, threads_fma = 256;
    const int iters_fma = kind == 1 ? 2048 : 65536;
    const int blocks_smem = sms * 4, iters_smem = 4096;
    auto launch = [&]() {
        if (kind == 0)
            fma_kernel<float><<<blocks_fma, threads_fma, 0, s>>>(sink, iters_fma, 0.999f, 0.001f);
        else if (kind == 1)
            fma_kernel<double><<<blocks_fma, threads_fma, 0, s>>>(reinterpret_cast<double *>(sink), iters_fma, 0.999,
                                                                  0.001);
        else if (kind == 2)
            smem_kernel<<<blocks_smem, 1024, 4096 * 16, s>>>(sink, iters_smem);
        else
            ffma2_kernel<<<blocks_fma, threads_fma, 0, s>>>(sink, iters_fma, 0.999f, 0.001f);
    };
    launch();   // warm-up
    float best = 0.f;
    for (int r = 0; r < 5; ++r) {
        cudaEventRecord(e0, s);
        launch();
        cudaEventRecord(e1, s);
        e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r == 0 || ms < best) best = ms;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (e != cudaSuccess) return set_cuda_error(e);
    const double sec = best / 1000.0;
    if (kind == 2)
        *value = (double)blocks_smem * 1024 * iters_smem * 8 * 16 / sec;    // bytes/s
    else
        *value = 2.0 * blocks_fma * threads_fma * (double)iters_fma * kChains / sec;   // flop/s
    return FTWA_OK;
}
