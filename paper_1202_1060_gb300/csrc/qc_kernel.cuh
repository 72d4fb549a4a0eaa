// The single-CN layered QC decode kernel (qc_decode_kernel) and its device helpers, included by
// decode_qc.cu (decode instances) and decode_qc_serve.cu (serving instances).  The index
// scheme, phases and write-back order are described at the top of decode_qc.cu.  Per group a
// CN reads one 16-byte record (table offset, degree, message offset, stride) for its layer;
// the syndrome check of Step 4 stops per warp once a lane has found an unsatisfied check.
#pragma once

#include "decode_qc.h"
#include "decode_tile.h"
#include "qc_device.cuh"

namespace ndgsbp {


// ---- single-CN kernel ---------------------------------------------------------------------
template <int D, int MAXDC, typename MsgT>
__device__ __forceinline__ void qc_phase_a(const int2* __restrict__ et, int c, int c4, int Z4, float* __restrict__ P,
                                           MsgT* __restrict__ m, float lim, int (&vb)[MAXDC], float (&dl)[MAXDC]) {
    static_assert(D <= MAXDC, "degree above the bound");
    float t[D], old[D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
        vb[k] = qc_vb(et[k], c, c4, Z4);
        old[k] = to_f(m[k]);
        t[k] = at_byte(P, vb[k]) - old[k];
    }
    check_node_update<D>(t, D, lim, [&](int k, float val) {
        const MsgT q = from_f<MsgT>(val);
        m[k] = q;
        dl[k] = to_f(q) - old[k];
    });
}

template <int MAXDC, typename MsgT>
__device__ __forceinline__ void qc_phase_a_any(const int2* __restrict__ et, int c, int c4, int Z4, int d,
                                               float* __restrict__ P, MsgT* __restrict__ m, float lim,
                                               int (&vb)[MAXDC], float (&dl)[MAXDC]) {
    float t[MAXDC], old[MAXDC];
#pragma unroll
    for (int k = 0; k < MAXDC; ++k) {
        if (k < d) {
            vb[k] = qc_vb(et[k], c, c4, Z4);
            old[k] = to_f(m[k]);
            t[k] = at_byte(P, vb[k]) - old[k];
        }
    }
    check_node_update<MAXDC>(t, d, lim, [&](int k, float val) {
        const MsgT q = from_f<MsgT>(val);
        m[k] = q;
        dl[k] = to_f(q) - old[k];
    });
}

template <int D, int MAXDC>
__device__ __forceinline__ void qc_phase_b(float* __restrict__ P, const int (&vb)[MAXDC], const float (&dl)[MAXDC]) {
#pragma unroll
    for (int k = 0; k < D; ++k) at_byte(P, vb[k]) += dl[k];
}

template <int D>
__device__ __forceinline__ unsigned qc_parity(const int2* __restrict__ et, int c, int c4, int Z4, float* __restrict__ P) {
    unsigned p = 0u;
#pragma unroll
    for (int k = 0; k < D; ++k) p ^= (at_byte(P, qc_vb(et[k], c, c4, Z4)) < 0.f) ? 1u : 0u;
    return p;
}


// Shared-memory tables of a QC launch (loaded once per CTA).
struct QcSmem {
    float* P;
    unsigned char* msg;   // used when messages are in shared memory
    int2* tab;
    int* ldeg;
    int* lstride;
    int* loff;
    int* glay;
    int4* gtab;         // per (grouping, group, position): (l maxdeg, d_l, layer_off[l], layer_stride[l])
};

template <typename MsgT, bool MSG_SMEM>
__device__ __forceinline__ QcSmem qc_smem_layout(unsigned char* smem, const QcArgs& a) {
    QcSmem s;
    const RunArgs& r = a.r;
    s.P = reinterpret_cast<float*>(smem);
    size_t off = (static_cast<size_t>(r.N) * 4 + 15) & ~static_cast<size_t>(15);
    s.msg = smem + off;
    if (MSG_SMEM) off += (static_cast<size_t>(a.msg_slots) * sizeof(MsgT) + 15) & ~static_cast<size_t>(15);
    s.tab = reinterpret_cast<int2*>(smem + off);
    off += (static_cast<size_t>(a.nl) * a.maxdeg * 8 + 15) & ~static_cast<size_t>(15);
    s.ldeg = reinterpret_cast<int*>(smem + off);
    off += (static_cast<size_t>(a.nl) * 4 + 15) & ~static_cast<size_t>(15);
    s.lstride = reinterpret_cast<int*>(smem + off);
    off += (static_cast<size_t>(a.nl) * 4 + 15) & ~static_cast<size_t>(15);
    s.loff = reinterpret_cast<int*>(smem + off);
    off += (static_cast<size_t>(a.nl) * 4 + 15) & ~static_cast<size_t>(15);
    const int gw = a.G * a.window * a.n_groupings;
    s.glay = reinterpret_cast<int*>(smem + off);
    off += (static_cast<size_t>(gw) * 4 + 15) & ~static_cast<size_t>(15);
    s.gtab = reinterpret_cast<int4*>(smem + off);
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int i = tid; i < a.nl * a.maxdeg; i += nt) s.tab[i] = a.edge_tab[i];
    for (int i = tid; i < a.nl; i += nt) {
        s.ldeg[i] = a.layer_deg[i];
        s.lstride[i] = a.layer_stride[i];
        s.loff[i] = a.layer_off[i];
    }
    for (int i = tid; i < gw; i += nt) {
        const int l = a.group_layers[i];
        s.glay[i] = l;
        s.gtab[i] = make_int4(l * a.maxdeg, a.layer_deg[l], a.layer_off[l], a.layer_stride[l]);
    }
    return s;
}

// Start frame f: P = L, messages 0 (all threads; ends with a barrier).  Returns whether the
// frame's LLRs hold a NaN or an infinity (see load_frame_llrs).
template <typename MsgT>
__device__ __forceinline__ bool qc_frame_begin(const QcArgs& a, const QcSmem& s, MsgT* msg, long long f) {
    const RunArgs& r = a.r;
    const int tid = threadIdx.x, nt = blockDim.x;
    if (r.start_ns && tid == 0) r.start_ns[f] = global_timer_ns();
    for (int e = tid; e < a.msg_slots; e += nt) msg[e] = from_f<MsgT>(0.f);
    return load_frame_llrs(r, s.P, f);
}

template <typename MsgT>
__device__ __forceinline__ void qc_frame_messages_out(const QcArgs& a, const MsgT* msg, long long f) {
    const RunArgs& r = a.r;
    if (!r.msgs_out) return;
    for (int e = threadIdx.x; e < a.msg_slots; e += blockDim.x) {
        const int csr = __ldg(a.csr_of + e);
        if (csr >= 0) r.msgs_out[f * r.E + csr] = to_f(msg[e]) * kLn2;
    }
}

// OCC > 0: an instance for blocks of at most kOccThreads threads compiled for OCC resident CTAs
// per SM (fewer registers), for launches whose shared memory allows that many.
constexpr int kOccThreads = 192;

// SERVE: a serving launch advances the pool slots of serve_list.  A new slot starts from its
// staged LLRs, a running one resumes from its saved posterior and messages; a frame runs until
// it retires (zero syndrome or I_max: outputs written, slot marked done and listed) or has run
// epoch_iters iterations in this launch (state saved, slot stays running).
template <typename MsgT, bool MSG_SMEM, int MAXDC, bool SPEC, int OCC = 0, bool SERVE = false>
__global__ void __launch_bounds__(OCC ? kOccThreads : max_threads_for(MAXDC), OCC ? OCC : 1)
    qc_decode_kernel(const QcArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long s_frame;
    __shared__ unsigned s_err;
    const RunArgs& r = a.r;
    const int tid = threadIdx.x;
    const int Z = a.Z, W = a.window, nl = a.nl, md = a.maxdeg, Z4 = 4 * a.Z;
    const QcSmem s = qc_smem_layout<MsgT, MSG_SMEM>(smem, a);
    float* P = s.P;
    MsgT* msg = MSG_SMEM ? reinterpret_cast<MsgT*>(s.msg)
                         : (SERVE ? nullptr : static_cast<MsgT*>(a.ws_msgs) + static_cast<size_t>(blockIdx.x) * a.msg_slots);
    const int j = tid / Z;
    const int c = tid - j * Z, c4 = 4 * c;
    const bool active = j < W;
    const float lim = r.llr_max;
    // every warp full and every lane through the same layers: the syndrome loop may vote per warp
    const bool warp_vote = (W * Z) % 32 == 0 && blockDim.x == W * Z && nl % W == 0;
    if (tid == 0) s_err = 0u;
    for (;;) {
        const long long fi = next_frame(r, &s_frame);   // barrier: also orders the table loads
        if (fi >= r.n_frames) break;
        long long f = fi;
        int it0 = 0;   // iterations done before this launch
        bool invalid = false;   // NaN or infinity among the frame's LLRs: not decoded
        if constexpr (SERVE) {
            f = a.serve_list[fi];
            const int fl = a.state_flag[f];
            if (fl != kSlotNew && fl != kSlotRunning) continue;   // uniform: every thread read the same flag
            if (!MSG_SMEM) msg = static_cast<MsgT*>(a.state_msgs) + static_cast<size_t>(f) * a.msg_slots;
            if (fl == kSlotNew) {
                invalid = qc_frame_begin(a, s, msg, f);
            } else {
                it0 = a.state_iter[f];
                const float* sp = a.state_P + static_cast<size_t>(f) * r.N;
                for (int n = tid; n < r.N; n += blockDim.x) P[n] = sp[n];
                if (MSG_SMEM) {
                    const MsgT* sm = static_cast<const MsgT*>(a.state_msgs) + static_cast<size_t>(f) * a.msg_slots;
                    for (int e = tid; e < a.msg_slots; e += blockDim.x) msg[e] = sm[e];
                }
            }
            __syncthreads();   // every thread has read the flag before it changes
            if (tid == 0) a.state_flag[f] = kSlotRunning;
        } else {
            invalid = qc_frame_begin(a, s, msg, f);
        }
        __syncthreads();
        int it = it0 + 1, unsat = 1;
        const int gw1 = a.G * W, gwk = gw1 * a.n_groupings;
        int gsel = (it0 % a.n_groupings) * gw1;   // iteration it uses grouping (it - 1) mod n_groupings
        bool park = false;
        for (; !invalid; ++it) {
            const int* gl = s.glay + gsel;   // this iteration's grouping
            const int4* gt = s.gtab + gsel;
            for (int g = 0; g < a.G; ++g) {
                float dl[MAXDC];
                int vb[MAXDC];
                int d = 0;
                if (active) {
                    const int4 ge = gt[g * W + j];   // one 16-byte load: table offset, degree, message offset, stride
                    d = ge.y;
                    const int2* et = s.tab + ge.x;
                    MsgT* m = msg + ge.z + c * ge.w;
                    if constexpr (SPEC) {
#define NDGSBP_CASE_A(D) \
    if (d == D) qc_phase_a<NDGSBP_DD(D), MAXDC, MsgT>(et, c, c4, Z4, P, m, lim, vb, dl);
                        NDGSBP_DEGREE_CASES(MAXDC, NDGSBP_CASE_A)
#undef NDGSBP_CASE_A
                    } else {
                        qc_phase_a_any<MAXDC, MsgT>(et, c, c4, Z4, d, P, m, lim, vb, dl);
                    }
                }
                __syncthreads();
                for (int jj = 0; jj < W; ++jj) {
                    if (active && j == jj) {
                        if constexpr (SPEC) {
#define NDGSBP_CASE_B(D) \
    if (d == D) qc_phase_b<NDGSBP_DD(D), MAXDC>(P, vb, dl);
                            NDGSBP_DEGREE_CASES(MAXDC, NDGSBP_CASE_B)
#undef NDGSBP_CASE_B
                        } else {
#pragma unroll
                            for (int k = 0; k < MAXDC; ++k)
                                if (k < d) at_byte(P, vb[k]) += dl[k];
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
                        const int d = s.ldeg[l];
                        const int2* et = s.tab + l * md;
                        unsigned p = 0u;
                        if constexpr (SPEC) {
#define NDGSBP_CASE_S(D) \
    if (d == D) p = qc_parity<NDGSBP_DD(D)>(et, c, c4, Z4, P);
                            NDGSBP_DEGREE_CASES(MAXDC, NDGSBP_CASE_S)
#undef NDGSBP_CASE_S
                        } else {
#pragma unroll
                            for (int k = 0; k < MAXDC; ++k)
                                if (k < d) p ^= (at_byte(P, qc_vb(et[k], c, c4, Z4)) < 0.f) ? 1u : 0u;
                        }
                        bad |= p;
                        // once a lane of the warp has found an unsatisfied check the frame's
                        // syndrome is decided (the OR below), so the warp stops checking
                        if (warp_vote && __any_sync(0xffffffffu, bad)) break;
                    }
                }
                unsat = __syncthreads_or(bad);
                if (!unsat && r.early_stop) break;
            }
            if (last) break;
            if (SERVE && it - it0 >= a.epoch_iters) {
                park = true;
                break;
            }
            gsel += gw1;
            if (gsel == gwk) gsel = 0;
        }
        if constexpr (SERVE) {
            if (park) {
                float* sp = a.state_P + static_cast<size_t>(f) * r.N;
                for (int n = tid; n < r.N; n += blockDim.x) sp[n] = P[n];
                if (MSG_SMEM) {
                    MsgT* sm = static_cast<MsgT*>(a.state_msgs) + static_cast<size_t>(f) * a.msg_slots;
                    for (int e = tid; e < a.msg_slots; e += blockDim.x) sm[e] = msg[e];
                }
                if (tid == 0) a.state_iter[f] = it;
                __syncthreads();
                continue;
            }
        }
        qc_frame_messages_out(a, msg, f);
        write_frame_outputs(r, P, f, it, unsat, &s_err, 1, invalid);
        if (SERVE && tid == 0) {
            a.state_flag[f] = kSlotDone;
            a.done_list[atomicAdd(a.done_count, 1)] = static_cast<int>(f);
        }
        __syncthreads();
    }
}

}  // namespace ndgsbp
