// Throughput probe of the MUFU (XU-pipe) operations the decode kernels issue per edge-update of
// Eq. (1): ex2.approx, rcp.approx and lg2.approx (FP32, flush-to-zero).  Every thread runs
// `iters` rounds of 8 independent chains x <- f(x) that stay in range (2^-x on [0, 1], 1/(1 + x)
// on [1/2, 1], lg2(2 + x) on [1, 1.6]); with many warps per SM the pipe, not the chains'
// latency, limits the rate.  Each round also issues one FP32 add or negation per chain (FMA pipe,
// four times the XU rate).  The caller times the launch; ops = blocks x threads x iters x 8.
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "ndgsbp_internal.h"

namespace ndgsbp {

template <int OP>
__global__ void __launch_bounds__(1024) mufu_probe_kernel(long long iters, float* __restrict__ sink) {
    float x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = 0.5f + 0.01f * k + 1e-6f * (threadIdx.x & 31);
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if (OP == 0) x[k] = ex2_approx(-x[k]);
            if (OP == 1) x[k] = rcp_approx(x[k] + 1.f);
            if (OP == 2) x[k] = lg2_approx(x[k] + 2.f);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    if (s == -1.f) sink[blockIdx.x] = s;   // never true: keeps the chains live
}

}  // namespace ndgsbp

using namespace ndgsbp;

extern "C" ndgsbp_status ndgsbp_mufu_probe(int32_t op, int64_t iters, int32_t blocks, int32_t threads, float* d_sink,
                                           void* stream) {
    clear_error();
    if (op < 0 || op > 2 || iters < 1 || blocks < 1 || threads < 32 || threads > 1024 || threads % 32 || !d_sink)
        return fail(NDGSBP_ERR_INVALID, "mufu_probe: bad arguments");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    switch (op) {
        case 0: mufu_probe_kernel<0><<<blocks, threads, 0, s>>>(iters, d_sink); break;
        case 1: mufu_probe_kernel<1><<<blocks, threads, 0, s>>>(iters, d_sink); break;
        default: mufu_probe_kernel<2><<<blocks, threads, 0, s>>>(iters, d_sink); break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(NDGSBP_ERR_CUDA, "mufu_probe launch: %s", cudaGetErrorString(e));
    return NDGSBP_OK;
}
