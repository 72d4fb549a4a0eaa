// Device-side pieces shared by the decode kernels: run arguments, MUFU approximations, message
// storage types, LLR loads and the per-frame epilogue (hard decisions, outputs, statistics).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "ndgsbp.h"

namespace ndgsbp {

// Arguments every decode kernel takes: the batch, the decoder parameters and the outputs.
struct RunArgs {
    int N, E, W;                   // VNs, edges, packed words per frame
    const void* llr;
    int llr_dtype;
    long long n_frames;
    int max_iter;
    float llr_max;                 // clip limit of Eq. (1) inputs and outputs, in log2 units
    int early_stop;
    unsigned long long* counter;   // next-frame counter (workspace, zeroed per launch)
    uint32_t* hard_bits;
    int32_t* iters;
    uint8_t* synd_ok;
    float* posterior;
    const uint32_t* ref_bits;
    int ref_per_frame;
    unsigned long long* stats;
    unsigned long long* iter_hist;
    unsigned long long* start_ns;
    unsigned long long* retire_ns;
    float* msgs_out;
};

// Largest CTA of a kernel instance: the per-edge register arrays grow with the degree bound.
__host__ __device__ constexpr int max_threads_for(int maxdc) { return maxdc <= 8 ? 1024 : maxdc <= 16 ? 512 : 256; }

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2_approx(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ unsigned long long global_timer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <typename T> __device__ __forceinline__ float to_f(T v);
template <> __device__ __forceinline__ float to_f<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f<__half>(__half v) { return __half2float(v); }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <typename T> __device__ __forceinline__ T from_f(float v);
template <> __device__ __forceinline__ float from_f<float>(float v) { return v; }
template <> __device__ __forceinline__ __half from_f<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

// The kernels keep posteriors and messages in log2 units (an LLR times log2 e): Eq. (1) then
// takes exp(-x) as ex2(-x) and ln(w) as lg2(w) with no scaling, and Eqs. (2)-(3) are linear, so
// scaling them changes nothing but the unit.  Channel LLRs are converted when a frame is loaded,
// posteriors and messages are converted back when they are written out, and the clip limit is
// given in log2 units (kernel_llr_limit on the host).
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.69314718055994531f;

// Channel LLR i of the input, in log2 units.  A NaN or an infinity sets `bad` (the frame is then
// not decoded: see load_frame_llrs).
__device__ __forceinline__ float load_llr(const void* p, int dtype, long long i, bool& bad) {
    float v;
    switch (dtype) {
        case NDGSBP_F64: {
            const double d = static_cast<const double*>(p)[i];
            bad |= !isfinite(d);
            v = static_cast<float>(d);   // FP32 first
            break;
        }
        case NDGSBP_F16: v = __half2float(static_cast<const __half*>(p)[i]); break;
        case NDGSBP_BF16: v = __bfloat162float(static_cast<const __nv_bfloat16*>(p)[i]); break;
        default: v = static_cast<const float*>(p)[i]; break;
    }
    bad |= !isfinite(v);
    return v * kLog2e;
}

// P[n] = L_n (log2 units) for the N channel LLRs of frame f (all threads; ends with a barrier).
// Returns, in every thread, whether any of them is a NaN or an infinity; such a frame gets P = 0
// (all messages stay 0 and it retires after one iteration) and its outputs mark it invalid
// (write_frame_outputs with invalid = true).
__device__ __forceinline__ bool load_frame_llrs(const RunArgs& r, float* __restrict__ P, long long f) {
    const int tid = threadIdx.x, nt = blockDim.x;
    bool bad = false;
    for (int n = tid; n < r.N; n += nt) P[n] = load_llr(r.llr, r.llr_dtype, f * r.N + n, bad);
    if (!__syncthreads_or(bad)) return false;
    for (int n = tid; n < r.N; n += nt) P[n] = 0.f;
    __syncthreads();
    return true;
}

// Eq. (1) on the d <= MAXDC edges of one CN, in the positive-pair tanh-product form.
// Input: t[k] (VN->CN messages, log2 units).  For every edge, emit(k, L_{m->n_k}) receives the
// signed CN->VN message in log2 units, clipped to lim (log2 units; called in descending k).
// With x = |t| ln 2 the natural magnitude: u = exp(-x) = 2^-|t| and the output ln(w) / ln 2 =
// lg2(w), so neither transcendental needs a scaling multiply.
// tanh(x/2) = N / (N + E) with, for u = exp(-x), (N, E) = ((1 - u) / 2, u); pairs combine as
// (Na Nb, Ea (Eb + Nb) + Na Eb); 2 atanh(N / (N + E)) = ln(1 + 2 N / E).  Every term is
// positive, so neither saturated nor tiny inputs lose relative accuracy.  The product over
// "all edges but k" is prefix(k) (x) suffix(k + 1); no division.
template <int MAXDC, typename Emit>
__device__ __forceinline__ void check_node_update(const float (&t)[MAXDC], int d, float lim, Emit emit) {
    // xs[k]: u_k = exp(-|L_k|) >= 0 carrying the sign of t[k] in its sign bit (every use of u
    // takes |xs|, a free operand modifier); par: bit 31 = parity of the input signs
    float xs[MAXDC], pn[MAXDC], pe[MAXDC];
    unsigned par = 0u;
    float cn = 1.f, ce = 0.f;
#pragma unroll
    for (int k = 0; k < MAXDC; ++k) {
        if (k < d) {
            const unsigned tb = __float_as_uint(t[k]);
            par ^= tb;
            const float x = fminf(fabsf(t[k]), lim);
            const float u = ex2_approx(-x);            // exp(-|L|)
            const float n = fmaf(-0.5f, u, 0.5f);      // (1 - u) / 2
            xs[k] = __uint_as_float(__float_as_uint(u) | (tb & 0x80000000u));
            pn[k] = cn;
            pe[k] = ce;
            ce = fmaf(ce, fmaf(0.5f, u, 0.5f), cn * u);   // n + u = (1 + u) / 2
            cn = cn * n;
        }
    }
    // sign of output k: the parity of all input signs xor sign k
    const unsigned pm = par & 0x80000000u;
    float sn = 1.f, se = 0.f;
#pragma unroll
    for (int k = MAXDC - 1; k >= 0; --k) {
        if (k < d) {
            const float u = fabsf(xs[k]);
            const float n = fmaf(-0.5f, u, 0.5f);
            const float en = pn[k] * sn;
            const float ss = sn + se;
            const float ee = fmaf(pe[k], ss, pn[k] * se);
            const float w = fmaf(en * rcp_approx(ee), 2.f, 1.f);
            const float mag = fminf(lg2_approx(w), lim);
            const unsigned sgn = (__float_as_uint(xs[k]) ^ pm) & 0x80000000u;
            emit(k, __uint_as_float(__float_as_uint(mag) | sgn));
            se = fmaf(u, ss, se * n);   // se (n + u) + sn u, reusing sn + se
            sn = sn * n;
        }
    }
}

// Claim the next frame for this CTA (tid 0 writes *slot); returns after a barrier.  The leading
// barrier keeps tid 0 from overwriting *slot before every thread has read the previous value
// (a serving launch skips a listed slot that is no longer running without any other barrier).
__device__ __forceinline__ long long next_frame(const RunArgs& r, long long* slot) {
    __syncthreads();
    if (threadIdx.x == 0) *slot = static_cast<long long>(atomicAdd(r.counter, 1ull));
    __syncthreads();
    return *slot;
}

// Frame epilogue: hard decisions (packed), optional posterior, per-frame outputs and the fused
// statistics (errors against the transmitted word, iteration histogram, timestamps).  The
// frame's posterior of VN n is P[n * pstride].  invalid: the frame's channel LLRs held a NaN or
// an infinity (P = 0): iteration count 0, syndrome flag 0, counted in NDGSBP_STAT_INVALID only.
__device__ __forceinline__ void write_frame_outputs(const RunArgs& a, const float* __restrict__ P, long long f,
                                                    int iters, int unsat, unsigned* s_err, int pstride = 1,
                                                    bool invalid = false) {
    if (invalid) {
        iters = 0;
        unsat = 1;
    }
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const int W = a.W;
    unsigned err = 0u;
    for (int w = warp; w < W; w += nw) {
        const int n = 32 * w + lane;
        const bool bit = (n < a.N) && (P[n * pstride] < 0.f);
        const unsigned word = __ballot_sync(0xffffffffu, bit);
        if (lane == 0) {
            a.hard_bits[f * W + w] = word;
            if (a.stats) {
                const unsigned ref = a.ref_bits ? a.ref_bits[(a.ref_per_frame ? f * W : 0) + w] : 0u;
                err += __popc(word ^ ref);
            }
        }
    }
    if (a.posterior)
        for (int n = tid; n < a.N; n += nt) a.posterior[f * a.N + n] = P[n * pstride] * kLn2;
    if (a.stats && lane == 0 && err) atomicAdd(s_err, err);
    __syncthreads();
    if (tid == 0) {
        if (a.iters) a.iters[f] = iters;
        if (a.synd_ok) a.synd_ok[f] = unsat ? 0 : 1;
        if (a.stats && invalid) {
            atomicAdd(a.stats + NDGSBP_STAT_INVALID, 1ull);
            *s_err = 0u;
        } else if (a.stats) {
            const unsigned e = *s_err;
            atomicAdd(a.stats + NDGSBP_STAT_FRAMES, 1ull);
            atomicAdd(a.stats + NDGSBP_STAT_ITERATIONS, static_cast<unsigned long long>(iters));
            if (e) {
                atomicAdd(a.stats + NDGSBP_STAT_FRAME_ERRORS, 1ull);
                atomicAdd(a.stats + NDGSBP_STAT_BIT_ERRORS, static_cast<unsigned long long>(e));
                if (!unsat) atomicAdd(a.stats + NDGSBP_STAT_UNDETECTED, 1ull);
            }
            if (unsat) atomicAdd(a.stats + NDGSBP_STAT_UNSATISFIED, 1ull);
            *s_err = 0u;
        }
        if (a.iter_hist && !invalid) atomicAdd(a.iter_hist + iters, 1ull);
        if (a.retire_ns) a.retire_ns[f] = global_timer_ns();
    }
}

}  // namespace ndgsbp
