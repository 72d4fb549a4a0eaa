// Layered QC decode kernels for sm_103a.
//
// For QC codes grouped in whole layers (windows of `window` layers of Z CNs each), the VN of
// edge k of CN c in layer l is b_k Z + (c + s_k) mod Z, with (b_k, s_k) the block column and
// circulant shift of the layer's k-th base entry.  The kernels compute those indices instead of
// reading per-edge tables: each layer contributes one (4 (b Z + s), Z - s) pair per edge, held
// in shared memory and read as a broadcast, and the index is kept as a byte offset into the
// posterior.  The messages of CN c of layer l sit at layer_off[l] + c S_l + k with an odd
// stride S_l >= d_l, so 32 consecutive CNs touch 32 distinct banks and k is a compile-time
// offset.
//
// qc_decode_kernel: thread t owns window position j = t / Z and CN c = t mod Z in every group.
// qc_pair_kernel:   thread t owns position j = t / (Z/2) and the two CNs c and c + Z/2; all the
//                   arithmetic of Eq. (1) runs on float2 pairs (packed FP32 instructions, each
//                   lane rounded exactly as the scalar operation), so the two kernels give
//                   identical results while the pair kernel issues about half the FP work.
// Both run phase A (Eq. (1) on every CN of the group; VN offsets and message changes kept in
// registers) and phase B (changes added layer position by layer position, the same fixed order
// as the colour order of the table-driven kernel, whose results they therefore reproduce).
// Layers get fully unrolled code for their exact degree when every layer degree lies in
// (MAXDC/2, MAXDC] (the usual QC case); other codes use the degree-generic instances.
#include <cstring>

#include "qc_kernel.cuh"

namespace ndgsbp {

// ---- pair kernel --------------------------------------------------------------------------

template <int D, int MAXDC, typename MsgT>
__device__ __forceinline__ void qc2_phase_a(const int2* __restrict__ et, int c0, int c1, int Z4, float* __restrict__ P,
                                            MsgT* __restrict__ m0, MsgT* __restrict__ m1, float lim, int (&vb0)[MAXDC],
                                            int (&vb1)[MAXDC], float2 (&dl)[MAXDC]) {
    static_assert(D <= MAXDC, "degree above the bound");
    float2 t[D], old[D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
        const int2 e = et[k];
        vb0[k] = qc_vb(e, c0, 4 * c0, Z4);
        vb1[k] = qc_vb(e, c1, 4 * c1, Z4);
        old[k] = make_float2(to_f(m0[k]), to_f(m1[k]));
        // P - old with one rounding, as the scalar kernel's subtraction
        t[k] = __ffma2_rn(old[k], f2(-1.f), make_float2(at_byte(P, vb0[k]), at_byte(P, vb1[k])));
    }
    check_node_update2<D>(t, lim, [&](int k, float2 val) {
        const MsgT q0 = from_f<MsgT>(val.x), q1 = from_f<MsgT>(val.y);
        m0[k] = q0;
        m1[k] = q1;
        dl[k] = __ffma2_rn(old[k], f2(-1.f), make_float2(to_f(q0), to_f(q1)));
    });
}

template <int D, int MAXDC>
__device__ __forceinline__ void qc2_phase_b(float* __restrict__ P, const int (&vb0)[MAXDC], const int (&vb1)[MAXDC],
                                            const float2 (&dl)[MAXDC]) {
#pragma unroll
    for (int k = 0; k < D; ++k) {
        at_byte(P, vb0[k]) += dl[k].x;
        at_byte(P, vb1[k]) += dl[k].y;
    }
}

template <int D>
__device__ __forceinline__ unsigned qc2_parity(const int2* __restrict__ et, int c0, int c1, int Z4, float* __restrict__ P) {
    unsigned p0 = 0u, p1 = 0u;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        const int2 e = et[k];
        p0 ^= (at_byte(P, qc_vb(e, c0, 4 * c0, Z4)) < 0.f) ? 1u : 0u;
        p1 ^= (at_byte(P, qc_vb(e, c1, 4 * c1, Z4)) < 0.f) ? 1u : 0u;
    }
    return p0 | p1;
}

__host__ __device__ constexpr int pair_max_threads(int maxdc) { return maxdc <= 8 ? 512 : 256; }

template <typename MsgT, bool MSG_SMEM, int MAXDC>
__global__ void __launch_bounds__(pair_max_threads(MAXDC)) qc_pair_kernel(const QcArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long s_frame;
    __shared__ unsigned s_err;
    const RunArgs& r = a.r;
    const int tid = threadIdx.x;
    const int Z = a.Z, Zh = a.Z >> 1, W = a.window, nl = a.nl, md = a.maxdeg, Z4 = 4 * a.Z;
    const QcSmem s = qc_smem_layout<MsgT, MSG_SMEM>(smem, a);
    float* P = s.P;
    MsgT* msg = MSG_SMEM ? reinterpret_cast<MsgT*>(s.msg)
                         : static_cast<MsgT*>(a.ws_msgs) + static_cast<size_t>(blockIdx.x) * a.msg_slots;
    const int j = tid / Zh;
    const int c0 = tid - j * Zh, c1 = c0 + Zh;
    const bool active = j < W;
    const float lim = r.llr_max;
    (void)Z;
    if (tid == 0) s_err = 0u;
    for (;;) {
        const long long f = next_frame(r, &s_frame);
        if (f >= r.n_frames) break;
        qc_frame_begin(a, s, msg, f);
        __syncthreads();
        int it = 1, unsat = 1;
        for (;; ++it) {
            const int* gl = s.glay + ((it - 1) % a.n_groupings) * a.G * W;   // this iteration's grouping
            for (int g = 0; g < a.G; ++g) {
                float2 dl[MAXDC];
                int vb0[MAXDC], vb1[MAXDC];
                int d = 0;
                if (active) {
                    const int l = gl[g * W + j];
                    d = s.ldeg[l];
                    const int S = s.lstride[l];
                    const int2* et = s.tab + l * md;
                    MsgT* m0 = msg + s.loff[l] + c0 * S;
                    MsgT* m1 = m0 + Zh * S;
#define NDGSBP_CASE_A2(D) \
    if (d == D) qc2_phase_a<NDGSBP_DD(D), MAXDC, MsgT>(et, c0, c1, Z4, P, m0, m1, lim, vb0, vb1, dl);
                    NDGSBP_DEGREE_CASES(MAXDC, NDGSBP_CASE_A2)
#undef NDGSBP_CASE_A2
                }
                __syncthreads();
                for (int jj = 0; jj < W; ++jj) {
                    if (active && j == jj) {
#define NDGSBP_CASE_B2(D) \
    if (d == D) qc2_phase_b<NDGSBP_DD(D), MAXDC>(P, vb0, vb1, dl);
                        NDGSBP_DEGREE_CASES(MAXDC, NDGSBP_CASE_B2)
#undef NDGSBP_CASE_B2
                    }
                    __syncthreads();
                }
            }
            const bool last = it >= r.max_iter;
            if (r.early_stop || last) {
                unsigned bad = 0u;
                if (active) {
                    for (int l = j; l < nl; l += W) {
                        const int d = s.ldeg[l];
                        const int2* et = s.tab + l * md;
                        unsigned p = 0u;
#define NDGSBP_CASE_S2(D) \
    if (d == D) p = qc2_parity<NDGSBP_DD(D)>(et, c0, c1, Z4, P);
                        NDGSBP_DEGREE_CASES(MAXDC, NDGSBP_CASE_S2)
#undef NDGSBP_CASE_S2
                        bad |= p;
                    }
                }
                unsat = __syncthreads_or(bad);
                if (!unsat && r.early_stop) break;
            }
            if (last) break;
        }
        qc_frame_messages_out(a, msg, f);
        write_frame_outputs(r, P, f, it, unsat, &s_err);
        __syncthreads();
    }
}

// ---- kernel selection ---------------------------------------------------------------------
template <typename MsgT, int MAXDC>
static QcKernelFn pick_qc_storage(bool msg_smem, bool spec, bool pair, bool w2) {
    if (pair) return msg_smem ? qc_pair_kernel<MsgT, true, MAXDC> : qc_pair_kernel<MsgT, false, MAXDC>;
    if (spec && w2)
        return msg_smem ? qc_decode_kernel<MsgT, true, MAXDC, true, true> : qc_decode_kernel<MsgT, false, MAXDC, true, true>;
    if (spec)
        return msg_smem ? qc_decode_kernel<MsgT, true, MAXDC, true, false>
                        : qc_decode_kernel<MsgT, false, MAXDC, true, false>;
    return msg_smem ? qc_decode_kernel<MsgT, true, MAXDC, false, false> : qc_decode_kernel<MsgT, false, MAXDC, false, false>;
}

template <typename MsgT>
static QcKernelFn pick_qc_degree(int maxdc, bool msg_smem, bool spec, bool pair, bool w2, bool occ6) {
    if (occ6) {
        // 6 CTAs of <= 192 threads per SM: degree <= 8, messages in shared memory, 16-bit storage
        if (maxdc != 8 || !msg_smem || !spec || pair || w2 || sizeof(MsgT) != 2) return nullptr;
        return qc_decode_kernel<MsgT, true, 8, true, false, 6>;
    }
    switch (maxdc) {
        case 8: return pick_qc_storage<MsgT, 8>(msg_smem, spec, pair, w2);
        case 16: return pick_qc_storage<MsgT, 16>(msg_smem, spec, pair, w2);
        case 32:
            if (spec || pair) return nullptr;
            return msg_smem ? qc_decode_kernel<MsgT, true, 32, false, false> : qc_decode_kernel<MsgT, false, 32, false, false>;
        default: return nullptr;
    }
}

bool qc_degrees_specialised(const QcLayout& Q, int maxdc) {
    if (maxdc > 16) return false;
    for (int d : Q.layer_deg)
        if (d <= maxdc / 2 || d > maxdc) return false;
    return true;
}

int qc_pair_max_threads(int maxdc) { return pair_max_threads(maxdc); }

int qc_occ_threads() { return kOccThreads; }

QcKernelFn pick_qc_kernel(int msg_dtype, int maxdc, bool msg_smem, bool spec, bool pair, bool w2, bool occ6) {
    switch (msg_dtype) {
        case NDGSBP_F32: return pick_qc_degree<float>(maxdc, msg_smem, spec, pair, w2, occ6);
        case NDGSBP_F16: return pick_qc_degree<__half>(maxdc, msg_smem, spec, pair, w2, occ6);
        case NDGSBP_BF16: return pick_qc_degree<__nv_bfloat16>(maxdc, msg_smem, spec, pair, w2, occ6);
        default: return nullptr;
    }
}

static size_t a16(size_t x) { return (x + 15) & ~static_cast<size_t>(15); }

size_t qc_table_bytes(const QcLayout& Q, bool w2) {
    const size_t G = Q.window ? Q.group_layers.size() / Q.window : 0;
    size_t b = a16(static_cast<size_t>(Q.n_layers) * Q.max_deg * 8) + 3 * a16(static_cast<size_t>(Q.n_layers) * 4) +
               a16(G * Q.window * 4) + G * Q.window * 16;
    if (w2) b += a16(G * 2 * 4) + a16(static_cast<size_t>(Q.Z) * (Q.max_deg | 1) * 4);
    return b;
}

void fill_qc_args(QcArgs& a, const QcLayout& Q, const DeviceQc& D, void* ws_msgs, bool w2) {
    a.Z = Q.Z;
    a.nl = Q.n_layers;
    a.window = Q.window;
    a.n_groupings = Q.n_groupings;
    a.G = static_cast<int>(Q.group_layers.size() / (static_cast<size_t>(Q.window) * Q.n_groupings));
    a.maxdeg = Q.max_deg;
    a.msg_slots = Q.msg_slots;
    a.edge_tab = reinterpret_cast<const int2*>(D.edge_tab);
    a.layer_deg = D.layer_deg;
    a.layer_stride = D.layer_stride;
    a.layer_off = D.layer_off;
    a.group_layers = D.group_layers;
    a.csr_of = D.csr_of;
    a.ws_msgs = ws_msgs;
    a.win2 = w2 ? reinterpret_cast<const int2*>(D.win2) : nullptr;
}

}  // namespace ndgsbp
