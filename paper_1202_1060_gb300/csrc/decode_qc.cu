// Layered QC decode kernel for sm_103a.
//
// For QC codes grouped in whole layers (windows of `window` consecutive-in-schedule layers of
// Z CNs each), the VN of edge k of CN c in layer l is b_k Z + (c + s_k) mod Z, with (b_k, s_k)
// the block column and circulant shift of the layer's k-th base entry.  The kernel computes
// those indices instead of reading per-edge tables: each layer contributes one (b Z + s, Z - s)
// pair per edge, held in shared memory and read as a broadcast.
//
// Thread t of the CTA owns window position j = t / Z and CN c = t mod Z for every group, so a
// warp covers consecutive CNs of one layer: posterior reads P[b Z + (c + s) mod Z] and message
// accesses msg[layer_off + k Z + c] are consecutive words (conflict-free).  Phase A (Eq. (1) on
// every CN of the group) keeps each edge's message change in registers; phase B
// applies the changes layer position by layer position (a layer holds each VN at most once),
// which is the same fixed order as the colour order of the general kernel, so the two kernels
// produce identical results.
#include <cstring>

#include "decode_qc.h"

namespace ndgsbp {

__device__ __forceinline__ int qc_vn(int2 e, int c, int Z) { return e.x + c - (c >= e.y ? Z : 0); }

// Phase A for the CN of this thread in a layer of exactly D edges: VN->CN messages from the
// posterior, Eq. (1), new messages stored; the VN indices and message changes stay in registers
// for phase B.
template <int D, int MAXDC, typename MsgT>
__device__ __forceinline__ void qc_phase_a(const int2* __restrict__ et, int c, int Z, const float* __restrict__ P,
                                           MsgT* __restrict__ m, float lim, int (&vv)[MAXDC], float (&dl)[MAXDC]) {
    static_assert(D <= MAXDC, "degree above the bound");
    float t[D], old[D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
        vv[k] = qc_vn(et[k], c, Z);
        old[k] = to_f(m[k * Z]);
        t[k] = P[vv[k]] - old[k];
    }
    check_node_update<D>(t, D, lim, [&](int k, float val) {
        const MsgT q = from_f<MsgT>(val);
        m[k * Z] = q;
        dl[k] = to_f(q) - old[k];
    });
}

template <int D, int MAXDC>
__device__ __forceinline__ void qc_phase_b(float* __restrict__ P, const int (&vv)[MAXDC], const float (&dl)[MAXDC]) {
#pragma unroll
    for (int k = 0; k < D; ++k) P[vv[k]] += dl[k];
}

template <int D>
__device__ __forceinline__ unsigned qc_parity(const int2* __restrict__ et, int c, int Z, const float* __restrict__ P) {
    unsigned p = 0u;
#pragma unroll
    for (int k = 0; k < D; ++k) p ^= (P[qc_vn(et[k], c, Z)] < 0.f) ? 1u : 0u;
    return p;
}

// Degree-generic versions (any d <= MAXDC), used for degrees outside the specialised set.
template <int MAXDC, typename MsgT>
__device__ __forceinline__ void qc_phase_a_any(const int2* __restrict__ et, int c, int Z, int d, const float* __restrict__ P,
                                               MsgT* __restrict__ m, float lim, int (&vv)[MAXDC], float (&dl)[MAXDC]) {
    float t[MAXDC], old[MAXDC];
#pragma unroll
    for (int k = 0; k < MAXDC; ++k) {
        if (k < d) {
            vv[k] = qc_vn(et[k], c, Z);
            old[k] = to_f(m[k * Z]);
            t[k] = P[vv[k]] - old[k];
        }
    }
    check_node_update<MAXDC>(t, d, lim, [&](int k, float val) {
        const MsgT q = from_f<MsgT>(val);
        m[k * Z] = q;
        dl[k] = to_f(q) - old[k];
    });
}

// Warp-uniform dispatch on the layer degree (a warp covers one layer when 32 divides Z).
#define NDGSBP_DEGREE_CASES(MAXDC, X) \
    if (MAXDC == 8) { X(5) X(6) X(7) X(8) } else if (MAXDC == 16) { X(9) X(10) X(11) X(12) X(13) X(14) X(15) X(16) }

// SPEC instances run fully unrolled code for the layer's exact degree, chosen per layer by a
// warp-uniform dispatch; they serve codes whose layer degrees all lie in (MAXDC/2, MAXDC] (one
// or two row degrees just below the bound, the usual QC case).  Other instances run the
// degree-generic predicated code.  Keeping the two apart keeps the register footprint of the
// specialised code small (a shared fallback path raises it for every case).
template <typename MsgT, bool MSG_SMEM, int MAXDC, bool SPEC>
__global__ void __launch_bounds__(max_threads_for(MAXDC)) qc_decode_kernel(const QcArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long s_frame;
    __shared__ unsigned s_err;
    const RunArgs& r = a.r;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int Z = a.Z, W = a.window, nl = a.nl, md = a.maxdeg;
    float* P = reinterpret_cast<float*>(smem);
    size_t off = (static_cast<size_t>(r.N) * 4 + 15) & ~static_cast<size_t>(15);
    MsgT* msg;
    if (MSG_SMEM) {
        msg = reinterpret_cast<MsgT*>(smem + off);
        off += (static_cast<size_t>(r.E) * sizeof(MsgT) + 15) & ~static_cast<size_t>(15);
    } else {
        msg = static_cast<MsgT*>(a.ws_msgs) + static_cast<size_t>(blockIdx.x) * r.E;
    }
    int2* tab = reinterpret_cast<int2*>(smem + off);
    off += (static_cast<size_t>(nl) * md * 8 + 15) & ~static_cast<size_t>(15);
    int* ldeg = reinterpret_cast<int*>(smem + off);
    off += (static_cast<size_t>(nl) * 4 + 15) & ~static_cast<size_t>(15);
    int* loff = reinterpret_cast<int*>(smem + off);
    off += (static_cast<size_t>(nl) * 4 + 15) & ~static_cast<size_t>(15);
    int* glay = reinterpret_cast<int*>(smem + off);
    for (int i = tid; i < nl * md; i += nt) tab[i] = a.edge_tab[i];
    for (int i = tid; i < nl; i += nt) {
        ldeg[i] = a.layer_deg[i];
        loff[i] = a.layer_off[i];
    }
    for (int i = tid; i < a.G * W; i += nt) glay[i] = a.group_layers[i];
    const int j = tid / Z;
    const int c = tid - j * Z;
    const bool active = j < W;
    const float lim = r.llr_max;
    if (tid == 0) s_err = 0u;
    for (;;) {
        const long long f = next_frame(r, &s_frame);   // barrier: also orders the table loads
        if (f >= r.n_frames) break;
        if (r.start_ns && tid == 0) r.start_ns[f] = global_timer_ns();
        for (int n = tid; n < r.N; n += nt) P[n] = load_llr(r.llr, r.llr_dtype, f * r.N + n);
        for (int e = tid; e < r.E; e += nt) msg[e] = from_f<MsgT>(0.f);
        __syncthreads();
        int it = 1, unsat = 1;
        for (;; ++it) {
            for (int g = 0; g < a.G; ++g) {
                float dl[MAXDC];
                int vv[MAXDC];
                int d = 0;
                if (active) {
                    const int l = glay[g * W + j];
                    d = ldeg[l];
                    const int2* et = tab + l * md;
                    MsgT* m = msg + loff[l] + c;
                    if constexpr (SPEC) {
#define NDGSBP_CASE_A(D) \
    if (d == D) qc_phase_a<(D <= MAXDC ? D : MAXDC), MAXDC, MsgT>(et, c, Z, P, m, lim, vv, dl);
                        NDGSBP_DEGREE_CASES(MAXDC, NDGSBP_CASE_A)
#undef NDGSBP_CASE_A
                    } else {
                        qc_phase_a_any<MAXDC, MsgT>(et, c, Z, d, P, m, lim, vv, dl);
                    }
                }
                __syncthreads();
                for (int jj = 0; jj < W; ++jj) {
                    if (active && j == jj) {
                        if constexpr (SPEC) {
#define NDGSBP_CASE_B(D) \
    if (d == D) qc_phase_b<(D <= MAXDC ? D : MAXDC), MAXDC>(P, vv, dl);
                            NDGSBP_DEGREE_CASES(MAXDC, NDGSBP_CASE_B)
#undef NDGSBP_CASE_B
                        } else {
#pragma unroll
                            for (int k = 0; k < MAXDC; ++k)
                                if (k < d) P[vv[k]] += dl[k];
                        }
                    }
                    __syncthreads();
                }
            }
            const bool last = it >= r.max_iter;
            if (r.early_stop || last) {
                unsigned bad = 0u;
                if (active) {
                    for (int l = j; l < nl; l += W) {
                        const int d = ldeg[l];
                        const int2* et = tab + l * md;
                        unsigned p = 0u;
                        if constexpr (SPEC) {
#define NDGSBP_CASE_S(D) \
    if (d == D) p = qc_parity<(D <= MAXDC ? D : MAXDC)>(et, c, Z, P);
                            NDGSBP_DEGREE_CASES(MAXDC, NDGSBP_CASE_S)
#undef NDGSBP_CASE_S
                        } else {
#pragma unroll
                            for (int k = 0; k < MAXDC; ++k)
                                if (k < d) p ^= (P[qc_vn(et[k], c, Z)] < 0.f) ? 1u : 0u;
                        }
                        bad |= p;
                    }
                }
                unsat = __syncthreads_or(bad);
                if (!unsat && r.early_stop) break;
            }
            if (last) break;
        }
        if (r.msgs_out)
            for (int e = tid; e < r.E; e += nt) r.msgs_out[f * r.E + __ldg(a.csr_of + e)] = to_f(msg[e]);
        write_frame_outputs(r, P, f, it, unsat, &s_err);
        __syncthreads();
    }
}

template <typename MsgT, int MAXDC>
static QcKernelFn pick_qc_storage(bool msg_smem, bool spec) {
    if (spec) return msg_smem ? qc_decode_kernel<MsgT, true, MAXDC, true> : qc_decode_kernel<MsgT, false, MAXDC, true>;
    return msg_smem ? qc_decode_kernel<MsgT, true, MAXDC, false> : qc_decode_kernel<MsgT, false, MAXDC, false>;
}

template <typename MsgT>
static QcKernelFn pick_qc_degree(int maxdc, bool msg_smem, bool spec) {
    switch (maxdc) {
        case 8: return pick_qc_storage<MsgT, 8>(msg_smem, spec);
        case 16: return pick_qc_storage<MsgT, 16>(msg_smem, spec);
        case 32: return msg_smem ? qc_decode_kernel<MsgT, true, 32, false> : qc_decode_kernel<MsgT, false, 32, false>;
        default: return nullptr;
    }
}

bool qc_degrees_specialised(const QcLayout& Q, int maxdc) {
    if (maxdc > 16) return false;
    for (int d : Q.layer_deg)
        if (d <= maxdc / 2 || d > maxdc) return false;
    return true;
}

QcKernelFn pick_qc_kernel(int msg_dtype, int maxdc, bool msg_smem, bool spec) {
    switch (msg_dtype) {
        case NDGSBP_F32: return pick_qc_degree<float>(maxdc, msg_smem, spec);
        case NDGSBP_F16: return pick_qc_degree<__half>(maxdc, msg_smem, spec);
        case NDGSBP_BF16: return pick_qc_degree<__nv_bfloat16>(maxdc, msg_smem, spec);
        default: return nullptr;
    }
}

static size_t a16(size_t x) { return (x + 15) & ~static_cast<size_t>(15); }

size_t qc_table_bytes(const QcLayout& Q) {
    const size_t G = Q.window ? Q.group_layers.size() / Q.window : 0;
    return a16(static_cast<size_t>(Q.n_layers) * Q.max_deg * 8) + 2 * a16(static_cast<size_t>(Q.n_layers) * 4) +
           a16(G * Q.window * 4);
}

void fill_qc_args(QcArgs& a, const QcLayout& Q, const DeviceQc& D, void* ws_msgs) {
    a.Z = Q.Z;
    a.nl = Q.n_layers;
    a.window = Q.window;
    a.G = static_cast<int>(Q.group_layers.size() / Q.window);
    a.maxdeg = Q.max_deg;
    a.edge_tab = reinterpret_cast<const int2*>(D.edge_tab);
    a.layer_deg = D.layer_deg;
    a.layer_off = D.layer_off;
    a.group_layers = D.group_layers;
    a.csr_of = D.csr_of;
    a.ws_msgs = ws_msgs;
}

}  // namespace ndgsbp
