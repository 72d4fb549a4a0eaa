// Layered QC decode kernel with two frames per thread (sm_103a).
//
// qc_frames2_kernel is qc_decode_kernel (thread t owns window position j = t / Z and CN
// c = t mod Z of every group) run on two frames at once: a CTA holds two frame slots whose
// posteriors and messages are interleaved (P2[n] = (P_n of slot 0, P_n of slot 1), the same for
// each stored message), so one shared-memory access and one piece of index arithmetic serve
// both frames, and Eq. (1) runs as float2 packed FP32 instructions.  Each lane is rounded
// exactly as the scalar kernel's operation, so every frame gets the same result as from
// qc_decode_kernel, bit for bit.
//
// The slots step through the same group schedule but keep their own iteration counts: at the
// end of an iteration each slot whose frame stops (Step 4 b, or max_iter) writes its outputs
// and takes the next frame from the launch's counter, which starts at group 1 of iteration 1
// while the other slot carries on.  A slot with no frame left idles (its lane computes on
// zeros and is never written out) until the other slot finishes.
#include "decode_qc.h"
#include "qc_device.cuh"

namespace ndgsbp {

template <typename MsgT> struct Pair2;
template <> struct Pair2<float> {
    using T = float2;
    static __device__ __forceinline__ float2 to(float2 v) { return v; }
    static __device__ __forceinline__ float2 from(float2 v) { return v; }
};
template <> struct Pair2<__half> {
    using T = __half2;
    static __device__ __forceinline__ float2 to(__half2 v) { return __half22float2(v); }
    static __device__ __forceinline__ __half2 from(float2 v) { return __floats2half2_rn(v.x, v.y); }
};
template <> struct Pair2<__nv_bfloat16> {
    using T = __nv_bfloat162;
    static __device__ __forceinline__ float2 to(__nv_bfloat162 v) { return __bfloat1622float2(v); }
    static __device__ __forceinline__ __nv_bfloat162 from(float2 v) { return __floats2bfloat162_rn(v.x, v.y); }
};

// Byte offset of the VN pair of table entry e for CN c; the table holds (8 (b Z + s), Z - s).
__device__ __forceinline__ int qc2_vb(int2 e, int c, int c8, int Z8) { return e.x + c8 - (c >= e.y ? Z8 : 0); }

__device__ __forceinline__ float2& at_byte2(float2* P, int vb) {
    return *reinterpret_cast<float2*>(reinterpret_cast<char*>(P) + vb);
}

template <int D, int MAXDC, typename MsgT>
__device__ __forceinline__ void f2_phase_a(const int2* __restrict__ et, int c, int c8, int Z8, float2* __restrict__ P,
                                           typename Pair2<MsgT>::T* __restrict__ m, float lim, int (&vb)[MAXDC],
                                           float2 (&dl)[MAXDC]) {
    static_assert(D <= MAXDC, "degree above the bound");
    float2 t[D], old[D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
        vb[k] = qc2_vb(et[k], c, c8, Z8);
        old[k] = Pair2<MsgT>::to(m[k]);
        t[k] = __ffma2_rn(old[k], f2(-1.f), at_byte2(P, vb[k]));   // P - old, one rounding
    }
    check_node_update2<D>(t, lim, [&](int k, float2 val) {
        const typename Pair2<MsgT>::T q = Pair2<MsgT>::from(val);
        m[k] = q;
        dl[k] = __ffma2_rn(old[k], f2(-1.f), Pair2<MsgT>::to(q));
    });
}

template <int D, int MAXDC>
__device__ __forceinline__ void f2_phase_b(float2* __restrict__ P, const int (&vb)[MAXDC], const float2 (&dl)[MAXDC]) {
#pragma unroll
    for (int k = 0; k < D; ++k) {
        float2& p = at_byte2(P, vb[k]);
        p = __fadd2_rn(p, dl[k]);
    }
}

// Parities of CN c in both frames: bit 0 = slot 0, bit 1 = slot 1.
template <int D>
__device__ __forceinline__ unsigned f2_parity(const int2* __restrict__ et, int c, int c8, int Z8, float2* __restrict__ P) {
    unsigned p0 = 0u, p1 = 0u;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        const float2 v = at_byte2(P, qc2_vb(et[k], c, c8, Z8));
        p0 ^= v.x < 0.f ? 1u : 0u;
        p1 ^= v.y < 0.f ? 1u : 0u;
    }
    return p0 | (p1 << 1);
}

__host__ __device__ constexpr int frames2_max_threads(int maxdc) { return maxdc <= 8 ? 512 : 256; }

// Load frame f (or zeros for f < 0) into lane s of the interleaved posterior, zero its messages.
template <typename MsgT>
__device__ __forceinline__ void f2_load_lane(const RunArgs& r, float2* P, typename Pair2<MsgT>::T* msg, int msg_slots,
                                             int s, long long f) {
    const int tid = threadIdx.x, nt = blockDim.x;
    float* Pl = reinterpret_cast<float*>(P) + s;
    MsgT* ml = reinterpret_cast<MsgT*>(msg) + s;
    if (f >= 0 && r.start_ns && tid == 0) r.start_ns[f] = global_timer_ns();
    for (int n = tid; n < r.N; n += nt) Pl[2 * n] = f >= 0 ? load_llr(r.llr, r.llr_dtype, f * r.N + n) : 0.f;
    for (int e = tid; e < msg_slots; e += nt) ml[2 * e] = from_f<MsgT>(0.f);
}

template <typename MsgT, bool MSG_SMEM, int MAXDC>
__global__ void __launch_bounds__(frames2_max_threads(MAXDC)) qc_frames2_kernel(const QcArgs a) {
    using M2 = typename Pair2<MsgT>::T;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long s_frame[2];
    __shared__ int s_iter[2];
    __shared__ unsigned s_bad;
    __shared__ unsigned s_err;
    const RunArgs& r = a.r;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int Z = a.Z, W = a.window, nl = a.nl, md = a.maxdeg, Z8 = 8 * a.Z;
    // shared memory: P2 [N], messages [msg_slots] (when in shared memory), tables
    float2* P = reinterpret_cast<float2*>(smem);
    size_t off = (static_cast<size_t>(r.N) * 8 + 15) & ~static_cast<size_t>(15);
    M2* msg = MSG_SMEM ? reinterpret_cast<M2*>(smem + off)
                       : static_cast<M2*>(a.ws_msgs) + static_cast<size_t>(blockIdx.x) * a.msg_slots;
    if (MSG_SMEM) off += (static_cast<size_t>(a.msg_slots) * sizeof(M2) + 15) & ~static_cast<size_t>(15);
    int2* tab = reinterpret_cast<int2*>(smem + off);
    int* ldeg = reinterpret_cast<int*>(tab + nl * md);
    int* lstride = ldeg + nl;
    int* loff = lstride + nl;
    int* glay = loff + nl;
    for (int i = tid; i < nl * md; i += nt) {
        const int2 e = a.edge_tab[i];
        tab[i] = make_int2(2 * e.x, e.y);   // byte offsets into the float2 posterior
    }
    for (int i = tid; i < nl; i += nt) {
        ldeg[i] = a.layer_deg[i];
        lstride[i] = a.layer_stride[i];
        loff[i] = a.layer_off[i];
    }
    for (int i = tid; i < a.G * W; i += nt) glay[i] = a.group_layers[i];
    const int j = tid / Z;
    const int c = tid - j * Z, c8 = 8 * c;
    const bool active = j < W;
    const float lim = r.llr_max;
    if (tid == 0) {
        s_err = 0u;
        for (int s = 0; s < 2; ++s) {
            const long long f = static_cast<long long>(atomicAdd(r.counter, 1ull));
            s_frame[s] = f < r.n_frames ? f : -1;
            s_iter[s] = 0;
        }
    }
    __syncthreads();
    for (int s = 0; s < 2; ++s) f2_load_lane<MsgT>(r, P, msg, a.msg_slots, s, s_frame[s]);
    __syncthreads();
    while (s_frame[0] >= 0 || s_frame[1] >= 0) {
        for (int g = 0; g < a.G; ++g) {
            float2 dl[MAXDC];
            int vb[MAXDC];
            int d = 0;
            if (active) {
                const int l = glay[g * W + j];
                d = ldeg[l];
                const int2* et = tab + l * md;
                M2* m = msg + loff[l] + c * lstride[l];
#define NDGSBP_CASE_F2A(D) \
    if (d == D) f2_phase_a<NDGSBP_DD(D), MAXDC, MsgT>(et, c, c8, Z8, P, m, lim, vb, dl);
                NDGSBP_DEGREE_CASES(MAXDC, NDGSBP_CASE_F2A)
#undef NDGSBP_CASE_F2A
            }
            __syncthreads();
            for (int jj = 0; jj < W; ++jj) {
                if (active && j == jj) {
#define NDGSBP_CASE_F2B(D) \
    if (d == D) f2_phase_b<NDGSBP_DD(D), MAXDC>(P, vb, dl);
                    NDGSBP_DEGREE_CASES(MAXDC, NDGSBP_CASE_F2B)
#undef NDGSBP_CASE_F2B
                }
                __syncthreads();
            }
        }
        // ---- end of an iteration: Step 4 for each slot ----------------------------------------
        const int it0 = s_iter[0] + (s_frame[0] >= 0 ? 1 : 0);
        const int it1 = s_iter[1] + (s_frame[1] >= 0 ? 1 : 0);
        const bool need = r.early_stop || it0 >= r.max_iter || it1 >= r.max_iter;
        unsigned bad = 0u;
        if (need && active) {
            for (int l = j; l < nl; l += W) {
                const int d = ldeg[l];
                const int2* et = tab + l * md;
#define NDGSBP_CASE_F2S(D) \
    if (d == D) bad |= f2_parity<NDGSBP_DD(D)>(et, c, c8, Z8, P);
                NDGSBP_DEGREE_CASES(MAXDC, NDGSBP_CASE_F2S)
#undef NDGSBP_CASE_F2S
            }
        }
        if (tid == 0) s_bad = 0u;
        __syncthreads();
        if (bad) atomicOr(&s_bad, bad);
        __syncthreads();
        const unsigned unsat_bits = need ? s_bad : 3u;
        for (int s = 0; s < 2; ++s) {
            const long long f = s_frame[s];
            if (f < 0) continue;
            const int it = s ? it1 : it0;
            const int unsat = (unsat_bits >> s) & 1u;
            const bool done = (r.early_stop && !unsat) || it >= r.max_iter;
            if (!done) continue;
            if (r.msgs_out) {
                const MsgT* ml = reinterpret_cast<const MsgT*>(msg) + s;
                for (int e = tid; e < a.msg_slots; e += nt) {
                    const int csr = __ldg(a.csr_of + e);
                    if (csr >= 0) r.msgs_out[f * r.E + csr] = to_f(ml[2 * e]) * kLn2;
                }
            }
            write_frame_outputs(r, reinterpret_cast<const float*>(P) + s, f, it, unsat, &s_err, 2);
            if (tid == 0) {
                const long long nf = static_cast<long long>(atomicAdd(r.counter, 1ull));
                s_frame[s] = nf < r.n_frames ? nf : -1;
                s_iter[s] = -1;   // becomes 0 below
            }
            __syncthreads();
            f2_load_lane<MsgT>(r, P, msg, a.msg_slots, s, s_frame[s]);
        }
        __syncthreads();
        if (tid == 0) {
            s_iter[0] = s_iter[0] < 0 ? 0 : it0;
            s_iter[1] = s_iter[1] < 0 ? 0 : it1;
        }
        __syncthreads();
    }
}

template <typename MsgT, int MAXDC>
static QcKernelFn pick_f2_storage(bool msg_smem) {
    return msg_smem ? qc_frames2_kernel<MsgT, true, MAXDC> : qc_frames2_kernel<MsgT, false, MAXDC>;
}

template <typename MsgT>
static QcKernelFn pick_f2_degree(int maxdc, bool msg_smem) {
    switch (maxdc) {
        case 8: return pick_f2_storage<MsgT, 8>(msg_smem);
        case 16: return pick_f2_storage<MsgT, 16>(msg_smem);
        default: return nullptr;
    }
}

QcKernelFn pick_qc_frames2_kernel(int msg_dtype, int maxdc, bool msg_smem) {
    switch (msg_dtype) {
        case NDGSBP_F32: return pick_f2_degree<float>(maxdc, msg_smem);
        case NDGSBP_F16: return pick_f2_degree<__half>(maxdc, msg_smem);
        case NDGSBP_BF16: return pick_f2_degree<__nv_bfloat16>(maxdc, msg_smem);
        default: return nullptr;
    }
}

int qc_frames2_max_threads(int maxdc) { return frames2_max_threads(maxdc); }

}  // namespace ndgsbp
