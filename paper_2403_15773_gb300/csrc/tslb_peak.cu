// FP32 arithmetic rate of the GPU (tslb_fp32_lane_rate): the second roofline
// of the step kernel, whose collision and streaming sweeps are FP32 work.
//
// Every thread runs kChains independent fused multiply-add chains on values
// held in registers, either scalar (FFMA: one lane operation per thread and
// instruction) or packed (fma.rn.f32x2 through __ffma2_rn: two lane
// operations per thread and instruction).  With enough warps per SM and
// independent chains per warp, the dependent-issue latency is hidden and the
// kernel runs at the rate of the FMA pipes.  The chains' final values are
// written to a small device sink so that the compiler keeps the arithmetic.
#include <cuda_runtime.h>

#include "tslb.h"
#include "tslb_internal.h"

namespace {

constexpr int kThreads = 512;
constexpr int kChains = 8;
constexpr int kIters = 4096;
constexpr int kSink = 4096;

static __device__ float g_sink[kSink];

template <bool PACKED>
__global__ void __launch_bounds__(kThreads) fma_chain_kernel(float a0, float b0, int iters) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    if constexpr (PACKED) {
        float2 acc[kChains];
#pragma unroll
        for (int k = 0; k < kChains; ++k) acc[k] = make_float2(a0 + tid + k, a0 - tid - k);
        const float2 b = make_float2(b0, b0 * 0.5f), c = make_float2(1e-7f, -1e-7f);
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int k = 0; k < kChains; ++k) acc[k] = __ffma2_rn(acc[k], b, c);
        }
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < kChains; ++k) s += acc[k].x + acc[k].y;
        g_sink[tid % kSink] = s;
    } else {
        float acc[kChains];
#pragma unroll
        for (int k = 0; k < kChains; ++k) acc[k] = a0 + tid + k;
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int k = 0; k < kChains; ++k) acc[k] = fmaf(acc[k], b0, 1e-7f);
        }
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < kChains; ++k) s += acc[k];
        g_sink[tid % kSink] = s;
    }
}

}  // namespace

extern "C" TSLB_API tslb_status tslb_fp32_lane_rate(int32_t packed, void* cuda_stream, double* lane_ops_per_s) {
    if (!lane_ops_per_s || (packed != 0 && packed != 1)) {
        tslb::set_global_error("tslb_fp32_lane_rate: packed must be 0 or 1 and lane_ops_per_s non-NULL");
        return TSLB_ERR_INVALID_ARG;
    }
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    const int blocks = 4 * sms;  // 4 x 16 warps per SM
    float ms = 0.f;
    if (e == cudaSuccess) {
        for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // the first launch warms up
            e = cudaEventRecord(t0, s);
            if (packed)
                fma_chain_kernel<true><<<blocks, kThreads, 0, s>>>(1.0f, 0.999999f, kIters);
            else
                fma_chain_kernel<false><<<blocks, kThreads, 0, s>>>(1.0f, 0.999999f, kIters);
            if (e == cudaSuccess) e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaEventRecord(t1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(t1);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
        }
    }
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    if (e != cudaSuccess) {
        tslb::set_global_error(cudaGetErrorString(e));
        return TSLB_ERR_CUDA;
    }
    const double lanes = (double)blocks * kThreads * kChains * 8.0 * kIters * (packed ? 2.0 : 1.0);
    *lane_ops_per_s = lanes / (ms * 1e-3);
    return TSLB_OK;
}
