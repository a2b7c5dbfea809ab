// Allocation-free FP64 totals of caller-owned fields (tslb_field_sums_noalloc).
//
// Who needs this: code that must not allocate device memory at the moment it
// asks for the mass / phase-field totals.  cudaMalloc and cudaFree
// synchronise the whole device, so callers running an asynchronous pipeline
// (a solver loop that keeps several streams busy, a monitor called from a
// latency-critical path) cannot afford them; callers whose device memory is
// entirely held by another allocator (a framework's caching pool) may find no
// memory left to allocate at all.  The context API (tslb_init / tslb_sums)
// keeps its partial sums in a workspace that someone has to allocate first;
// this entry point needs only the caller's input and output pointers.
//
// The scratch is one file-scope __device__ array of kMaxBlocks FP64 partial
// pairs (256 KiB).  Every GPU that loads this library holds it until the
// process exits.  All calls share it, so calls whose work overlaps on the GPU
// (different streams, or different host threads, without ordering) race on it.
// Each call writes every partial it later reads, so nothing in the array has
// to start at zero and no clearing is needed between calls.
#include <cuda_runtime.h>

#include <mutex>

#include "tslb.h"
#include "tslb_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = 16384;           // partial pairs held by the scratch array
constexpr long long kChunk = 16384;         // values summed by one block
constexpr long long kMaxValues = (long long)kMaxBlocks * kChunk;  // 268,435,456 = 512 x 512 x 1024
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_partials[2 * kMaxBlocks];

std::mutex g_mutex;
double* g_scratch[kMaxDevices] = {};

// Per block: FP64 sums of rho and phi over one chunk of kChunk values.
__global__ void __launch_bounds__(kThreads) chunk_sums_kernel(const float* __restrict__ rho,
                                                              const float* __restrict__ phi, long long n,
                                                              double* __restrict__ partials) {
    __shared__ double sa[kThreads], sb[kThreads];
    const long long start = (long long)blockIdx.x * kChunk;
    const long long end = start + kChunk < n ? start + kChunk : n;
    double a = 0.0, b = 0.0;
    for (long long i = start + threadIdx.x; i < end; i += kThreads) {
        a += (double)rho[i];
        b += (double)phi[i];
    }
    sa[threadIdx.x] = a;
    sb[threadIdx.x] = b;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sa[threadIdx.x] += sa[threadIdx.x + w];
            sb[threadIdx.x] += sb[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = sa[0];
        partials[2 * blockIdx.x + 1] = sb[0];
    }
}

// Fixed-order reduction of the block partials into out[0..1].
__global__ void __launch_bounds__(kThreads) chunk_finish_kernel(const double* __restrict__ partials, int nblocks,
                                                                double* __restrict__ out) {
    __shared__ double sa[kThreads], sb[kThreads];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nblocks; i += kThreads) {
        a += partials[2 * i];
        b += partials[2 * i + 1];
    }
    sa[threadIdx.x] = a;
    sb[threadIdx.x] = b;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sa[threadIdx.x] += sa[threadIdx.x + w];
            sb[threadIdx.x] += sb[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = sa[0];
        out[1] = sb[0];
    }
}

// Device address of the scratch array on the current device, looked up once
// per device (the set-up of the first call on that device) and kept until the
// process exits.  In host code the name g_partials is only a host-side
// stand-in, not an address the GPU can use.  The cached address belongs to the
// device's primary context: a caller that resets the device (cudaDeviceReset)
// and goes on using this library in the same process would hand the kernels
// an address that is no longer mapped, so the device must not be reset.
cudaError_t scratch_on(int device, double** ptr) {
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_partials);
        if (e != cudaSuccess) return e;
        g_scratch[device] = static_cast<double*>(p);
    }
    *ptr = g_scratch[device];
    return cudaSuccess;
}

}  // namespace

extern "C" TSLB_API tslb_status tslb_field_sums_noalloc(const float* rho, const float* phi, int64_t n,
                                                        double* out, void* cuda_stream) {
    if (!rho || !phi || !out) {
        tslb::set_global_error("tslb_field_sums_noalloc: rho, phi and out are required");
        return TSLB_ERR_INVALID_ARG;
    }
    if (n < 1 || n > kMaxValues) {
        tslb::set_global_error(
            "tslb_field_sums_noalloc: n must lie in [1, 268435456]: its fixed scratch holds 16384 "
            "block partials of 16384 values each");
        return TSLB_ERR_INVALID_ARG;
    }
    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    double* scratch = nullptr;
    if (e == cudaSuccess) e = scratch_on(device, &scratch);
    if (e != cudaSuccess) {
        tslb::set_global_error(cudaGetErrorString(e));
        return TSLB_ERR_CUDA;
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const int nblocks = (int)((n + kChunk - 1) / kChunk);
    chunk_sums_kernel<<<nblocks, kThreads, 0, s>>>(rho, phi, (long long)n, scratch);
    chunk_finish_kernel<<<1, kThreads, 0, s>>>(scratch, nblocks, out);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        tslb::set_global_error(cudaGetErrorString(e));
        return TSLB_ERR_CUDA;
    }
    return TSLB_OK;
}
