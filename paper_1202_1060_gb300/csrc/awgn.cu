// BPSK/AWGN channel LLR generator (Sec. II-C: L_n = 2 y_n / sigma^2) for sm_103a.
//
// One thread per block of four VNs of one frame: a Philox4x32-10 block (Salmon, Moraes, Dror,
// Shaw, SC'11) keyed by the seed with counter (b, frame low, frame high, 0) gives four 32-bit
// words; u = ((x >> 9) + 1/2) 2^-23 is exact in FP32; Box-Muller turns (u0, u1) and (u2, u3) into
// two normal pairs (cos, then sin); y = (1 - 2 c) + sigma z and L = (2 / sigma^2) y.  The
// kernel writes HBM once per LLR (16-byte stores for FP32 when N is a multiple of 4 and the
// output is 16-byte aligned, element stores otherwise), but its time goes
// to the arithmetic: the ten Philox rounds and the accurate logarithm, sine and cosine of
// Box-Muller (about a fifth of the HBM store bandwidth on the n=2304 sweep; 2 % of its step).
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>

#include "ndgsbp_internal.h"

namespace ndgsbp {

__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(M0, c[0]), lo0 = M0 * c[0];
        const uint32_t hi1 = __umulhi(M1, c[2]), lo1 = M1 * c[2];
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
        k0 += W0;
        k1 += W1;
    }
}

template <typename T> __device__ __forceinline__ T cvt(float v);
template <> __device__ __forceinline__ float cvt<float>(float v) { return v; }
template <> __device__ __forceinline__ __half cvt<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 cvt<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

// VEC4: every row starts on a 16-byte boundary (FP32, N % 4 == 0, 16-byte aligned output), so
// each thread's four LLRs go out as one 16-byte store.
template <typename T, bool VEC4>
__global__ void awgn_kernel(int N, long long n_frames, float scale, float scale_sigma, uint32_t k0,
                            uint32_t k1, const uint32_t* __restrict__ cw, int cw_per_frame, T* __restrict__ out) {
    const int nb = (N + 3) >> 2;
    const int W = (N + 31) >> 5;
    // flat index idx = f nb + b, stepped by the grid stride: one division per thread, then the
    // (frame, block) pair advances by (stride / nb, stride % nb) with a carry
    const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
    const long long idx0 = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    const long long step_f = stride / nb;
    const int step_b = static_cast<int>(stride - step_f * nb);
    long long f = idx0 / nb;
    int b = static_cast<int>(idx0 - f * nb);
    for (; f < n_frames; f += step_f, b += step_b) {
        if (b >= nb) {
            b -= nb;
            ++f;
            if (f >= n_frames) break;
        }
        uint32_t c[4] = {static_cast<uint32_t>(b), static_cast<uint32_t>(f), static_cast<uint32_t>(f >> 32), 0u};
        philox4x32_10(c, k0, k1);
        float u[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) u[i] = (static_cast<float>(c[i] >> 9) + 0.5f) * 1.1920928955078125e-07f;
        float s0, c0, s1, c1;
        sincospif(2.f * u[1], &s0, &c0);
        sincospif(2.f * u[3], &s1, &c1);
        const float r0 = sqrtf(-2.f * logf(u[0])), r1 = sqrtf(-2.f * logf(u[2]));
        const float z[4] = {r0 * c0, r0 * s0, r1 * c1, r1 * s1};
        float L[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int n = 4 * b + i;
            float x = 1.f;
            if (cw && n < N) {
                const uint32_t word = cw[(cw_per_frame ? f * W : 0) + (n >> 5)];
                x = ((word >> (n & 31)) & 1u) ? -1.f : 1.f;
            }
            L[i] = fmaf(scale_sigma, z[i], scale * x);
        }
        T* row = out + f * N;
        if constexpr (VEC4) {
            reinterpret_cast<float4*>(row)[b] = make_float4(L[0], L[1], L[2], L[3]);
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (4 * b + i < N) row[4 * b + i] = cvt<T>(L[i]);
        }
    }
}

__global__ void philox_kernel(const uint32_t* __restrict__ ctr, uint32_t k0, uint32_t k1, long long n,
                              uint32_t* __restrict__ out) {
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        uint32_t c[4] = {ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]};
        philox4x32_10(c, k0, k1);
        for (int j = 0; j < 4; ++j) out[4 * i + j] = c[j];
    }
}

static int grid_for(long long work, int threads) {
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long blocks = (work + threads - 1) / threads;
    long long cap = static_cast<long long>(sms) * 8;
    return static_cast<int>(std::max<long long>(1, std::min(blocks, cap)));
}

}  // namespace ndgsbp

using namespace ndgsbp;

extern "C" {

ndgsbp_status ndgsbp_awgn_llr(const ndgsbp_code* code, int64_t n_frames, double ebn0_db, double rate,
                              uint64_t seed, const uint32_t* d_codeword_bits, int32_t codeword_per_frame,
                              void* d_llr, int32_t dtype, void* stream) {
    clear_error();
    if (!code) return fail(NDGSBP_ERR_INVALID, "awgn_llr: null code");
    if (n_frames < 0 || !(rate > 0.0)) return fail(NDGSBP_ERR_INVALID, "awgn_llr: bad n_frames or rate");
    if (n_frames == 0) return NDGSBP_OK;
    if (!d_llr) return fail(NDGSBP_ERR_INVALID, "awgn_llr: d_llr is null");
    const int N = code->c->N;
    const double sigma2 = 1.0 / (2.0 * rate * std::pow(10.0, ebn0_db / 10.0));
    const float scale = static_cast<float>(2.0 / sigma2);
    const float scale_sigma = static_cast<float>(2.0 / std::sqrt(sigma2));
    const uint32_t k0 = static_cast<uint32_t>(seed), k1 = static_cast<uint32_t>(seed >> 32);
    const long long work = n_frames * ((N + 3) / 4);
    const int threads = 256;
    const int grid = grid_for(work, threads);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (dtype != NDGSBP_F32 && dtype != NDGSBP_F16 && dtype != NDGSBP_BF16)
        return fail(NDGSBP_ERR_INVALID, "awgn_llr: dtype must be F32, F16 or BF16");
    const uintptr_t addr = reinterpret_cast<uintptr_t>(d_llr);
    const size_t esize = dtype == NDGSBP_F32 ? 4 : 2;
    if (addr % esize) return fail(NDGSBP_ERR_INVALID, "awgn_llr: d_llr is not aligned to its element size");
    // 16-byte stores only when every row starts on a 16-byte boundary
    const bool vec4 = dtype == NDGSBP_F32 && (N & 3) == 0 && addr % 16 == 0;
    switch (dtype) {
        case NDGSBP_F32:
            if (vec4)
                awgn_kernel<float, true><<<grid, threads, 0, s>>>(N, n_frames, scale, scale_sigma, k0, k1,
                                                                  d_codeword_bits, codeword_per_frame,
                                                                  static_cast<float*>(d_llr));
            else
                awgn_kernel<float, false><<<grid, threads, 0, s>>>(N, n_frames, scale, scale_sigma, k0, k1,
                                                                   d_codeword_bits, codeword_per_frame,
                                                                   static_cast<float*>(d_llr));
            break;
        case NDGSBP_F16:
            awgn_kernel<__half, false><<<grid, threads, 0, s>>>(N, n_frames, scale, scale_sigma, k0, k1, d_codeword_bits,
                                                         codeword_per_frame, static_cast<__half*>(d_llr));
            break;
        case NDGSBP_BF16:
            awgn_kernel<__nv_bfloat16, false><<<grid, threads, 0, s>>>(N, n_frames, scale, scale_sigma, k0, k1,
                                                                d_codeword_bits, codeword_per_frame,
                                                                static_cast<__nv_bfloat16*>(d_llr));
            break;
        default: return fail(NDGSBP_ERR_INVALID, "awgn_llr: dtype must be F32, F16 or BF16");
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(NDGSBP_ERR_CUDA, "awgn_llr launch: %s", cudaGetErrorString(e));
    return NDGSBP_OK;
}

ndgsbp_status ndgsbp_philox4x32_10(const uint32_t* d_ctr, uint32_t key0, uint32_t key1, int64_t n,
                                   uint32_t* d_out, void* stream) {
    clear_error();
    if (n < 0 || (n > 0 && (!d_ctr || !d_out))) return fail(NDGSBP_ERR_INVALID, "philox: bad arguments");
    if (n == 0) return NDGSBP_OK;
    philox_kernel<<<grid_for(n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(d_ctr, key0, key1, n, d_out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(NDGSBP_ERR_CUDA, "philox launch: %s", cudaGetErrorString(e));
    return NDGSBP_OK;
}

}  // extern "C"
