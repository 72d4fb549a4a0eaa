// Tile decode kernel for sm_103a: layered QC codes of any window size and row degree up to 32,
// several frames per CTA, and any mix of codes in one launch.
//
// Work comes in tiles (code, first frame, frame count) handed out by an atomic counter; a CTA
// decodes a tile's frames in `slots` frame slots at once and refills a slot from the tile as
// soon as its frame retires (Step 4 b), so early-stopping frames free their slot immediately.
// All slots of a CTA step through the same group schedule.
//
// A CN of degree d is spread over tpc lanes (consecutive threads of one warp), lane p holding
// edges [p le, min(d, (p+1) le)) with le <= 8.  Each lane forms the tanh product of its own edges
// in the positive-pair form (N, E) of Eq. (1) (see check_node_update), the lanes exchange their
// totals with two shuffles, and every lane seeds its suffix pass with the product of the other
// lanes' totals, so the exclusion "all edges but k" costs nothing extra per edge.  With tpc = 1
// the operations are those of the other kernels, in the same order.
//
// A group's CNs are processed in rounds over the block.  When one round covers the group (the
// REGB instances) every lane keeps its message changes in registers; otherwise they go to a
// per-slot delta buffer in shared memory.  Phase B adds them to the posterior layer position by
// layer position (the fixed order of the other kernels).  Posteriors, messages (when they fit)
// and deltas of every slot live in shared memory, after the code's tables.  Kernel instances
// differ in the unrolled lane width LE (4, 6, 8), REGB, and SINGLE (a launch over one code,
// whose parameters are then read at fixed offsets).  Posteriors and messages are in log2 units
// (see load_llr).
#include <cstring>

#include "decode_tile.h"
#include "lane_cnu.cuh"

namespace ndgsbp {

constexpr int kMaxSlots = 16;   // largest number of frame slots per CTA

// A code's tables at the start of shared memory: edge table [nl][md] (int2), layer degrees
// [nl], then, 16-byte aligned, one record per (grouping, group, position):
// (l md, d_l, l Z tpc msg_stride, 0).
__device__ __forceinline__ int4* tile_group_records(int2* tab, int nl, int md) {
    const size_t off = static_cast<size_t>(nl) * md * 8 + static_cast<size_t>(nl) * 4;
    return reinterpret_cast<int4*>(reinterpret_cast<unsigned char*>(tab) + ((off + 15) & ~static_cast<size_t>(15)));
}

// Shared state of a CTA (static part).
struct TileShared {
    long long frame[kMaxSlots];
    int iter[kMaxSlots];
    int epoch[kMaxSlots];
    int gofs[kMaxSlots];        // offset of the slot's grouping for its next iteration in the group tables
    unsigned unsat[kMaxSlots];
    int bad[kMaxSlots];         // the slot's frame had a NaN or an infinity among its LLRs (see load_frame)
    unsigned err;
    int tile, code, cur_code, next, end, active;
};

// Iterations done by slot s, and the grouping its next iteration uses (iteration l uses
// grouping (l - 1) mod n_groupings).
__device__ __forceinline__ void set_iter(TileShared& sh, const TileCode& C, int s, int it) {
    sh.iter[s] = it;
    sh.gofs[s] = (it % C.n_groupings) * C.G * C.window;
}

template <typename MsgT, bool SERVE>
__device__ __forceinline__ MsgT* slot_msgs(const TileCode& C, unsigned char* slot_base, int s, long long f) {
    if (C.m_bytes) return reinterpret_cast<MsgT*>(slot_base + C.p_bytes);
    if (SERVE) return static_cast<MsgT*>(C.state_msgs) + static_cast<size_t>(f) * C.msg_slots;
    return static_cast<MsgT*>(C.ws_msgs) + (static_cast<size_t>(blockIdx.x) * C.slots + s) * C.msg_slots;
}

// Next frame of the tile for a slot (tid 0 only); in serving mode only pool slots that hold a
// new or running frame are taken.
template <bool SERVE>
__device__ __forceinline__ long long claim_frame(TileShared& sh, const TileCode& C) {
    if (SERVE) {
        while (sh.next < sh.end) {
            const int fl = C.state_flag[sh.next];
            if (fl == kSlotNew || fl == kSlotRunning) return sh.next++;
            ++sh.next;
        }
        return -1;
    }
    return sh.next < sh.end ? sh.next++ : -1;
}

// Fill slot s with the tile's next frame (tid 0 only).
template <bool SERVE>
__device__ __forceinline__ void fill_slot(TileShared& sh, const TileCode& C, int s) {
    const long long f = claim_frame<SERVE>(sh, C);
    sh.frame[s] = f;
    set_iter(sh, C, s, (SERVE && f >= 0) ? (C.state_flag[f] == kSlotNew ? 0 : C.state_iter[f]) : 0);
    sh.epoch[s] = 0;
    if (SERVE && f >= 0) C.state_flag[f] = kSlotRunning;
}

// Load frame f into slot s (all threads): a fresh frame starts from P = L, messages 0; in
// serving mode a running frame resumes from its saved state.  A fresh frame whose LLRs hold a
// NaN or an infinity starts from P = 0 instead and is marked bad: its messages stay 0, it
// retires after its first iteration and its outputs mark it invalid (write_frame_outputs).
template <typename MsgT, bool SERVE>
__device__ __forceinline__ void load_frame(const TileCode& C, TileShared& sh, unsigned char* base, int s, long long f,
                                           int saved_iter) {
    const RunArgs& r = C.r;
    const int tid = threadIdx.x, nt = blockDim.x;
    float* P = reinterpret_cast<float*>(base);
    MsgT* msg = slot_msgs<MsgT, SERVE>(C, base, s, f);
    if (tid == 0) sh.bad[s] = 0;
    if (SERVE && saved_iter > 0) {
        const float* sp = C.state_P + static_cast<size_t>(f) * r.N;
        for (int n = tid; n < r.N; n += nt) P[n] = sp[n];
        if (C.m_bytes) {
            const MsgT* sm = static_cast<const MsgT*>(C.state_msgs) + static_cast<size_t>(f) * C.msg_slots;
            for (int e = tid; e < C.msg_slots; e += nt) msg[e] = sm[e];
        }
        return;
    }
    if (r.start_ns && tid == 0) r.start_ns[f] = global_timer_ns();
    for (int e = tid; e < C.msg_slots; e += nt) msg[e] = from_f<MsgT>(0.f);
    if (load_frame_llrs(r, P, f) && tid == 0) sh.bad[s] = 1;
}

// Serving mode: save a running frame's state at the end of its share of the launch.
template <typename MsgT>
__device__ __forceinline__ void save_frame(const TileCode& C, unsigned char* base, long long f) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const float* P = reinterpret_cast<const float*>(base);
    float* sp = C.state_P + static_cast<size_t>(f) * C.N;
    for (int n = tid; n < C.N; n += nt) sp[n] = P[n];
    if (C.m_bytes) {
        const MsgT* msg = reinterpret_cast<const MsgT*>(base + C.p_bytes);
        MsgT* sm = static_cast<MsgT*>(C.state_msgs) + static_cast<size_t>(f) * C.msg_slots;
        for (int e = tid; e < C.msg_slots; e += nt) sm[e] = msg[e];
    }
}

// Decode the frames of one tile until none is left (all threads).  LE >= the code's edges per
// lane le: the lane positions past a CN's degree (and in [le, LE)) are neutral.  REGB: one
// round of the block covers a group (slots x window x Z x tpc <= threads, for every code of the
// launch), so every lane keeps its message changes in registers for phase B; otherwise they go
// through the slot's delta buffer.
template <typename MsgT, bool SERVE, int LE, bool REGB>
__device__ __forceinline__ void run_tile(const TileCode& C, const int2* tab, unsigned char* slots_base,
                                         TileShared& sh) {
    const RunArgs& r = C.r;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int Z = C.Z, Z4 = 4 * C.Z, W = C.window, nl = C.nl, md = C.maxdeg, tpc = C.tpc, le = C.le;
    const int tsh = tpc == 1 ? 0 : (tpc == 2 ? 1 : 2);
    const int* ldeg = reinterpret_cast<const int*>(tab + nl * md);
    const int4* gtab = tile_group_records(const_cast<int2*>(tab), nl, md);
    const int per_slot = W * Z * tpc;           // CN-lanes of one group in one slot
    const int work = C.slots * per_slot;
    const int rounds = REGB ? 1 : (work + nt - 1) / nt;
    const float lim = r.llr_max;
    const unsigned gmask = tpc == 1 ? 0u : ((1u << tpc) - 1u) << ((tid & 31) & ~(tpc - 1));
    for (;;) {
        for (int g = 0; g < C.G; ++g) {
            // ---- phase A: Eq. (1) on every CN of the group in every filled slot ----------
            bool live = false;
            int j = 0, c = 0, L = 0;
            float* P = nullptr;
            const int2* et = tab;
            float dreg[LE];
            for (int rr = 0; rr < rounds; ++rr) {
                const int i = rr * nt + tid;
                const int s = fast_div(i, C.div_slot);
                live = i < work && sh.frame[s] >= 0;
                const int w = i - s * per_slot;
                const int cnl = w >> tsh, p = w & (tpc - 1);
                j = fast_div(cnl, C.div_z);
                c = cnl - j * Z;
                L = 0;
                float t[LE], old[LE], xu[LE], pn[LE], pe[LE];
                float cn = 1.f, ce = 0.f;
                unsigned lpar = 0u;   // bit 31: parity of this lane's input signs
                MsgT* m = nullptr;
                float* dl = nullptr;
                if (live) {
                    unsigned char* base = slots_base + static_cast<size_t>(s) * C.slot_bytes;
                    P = reinterpret_cast<float*>(base);
                    // (l maxdeg, d_l, first message of layer l) of this slot's grouping, position j
                    const int4 ge = gtab[sh.gofs[s] + g * W + j];
                    const int k0 = p * le;
                    L = min(max(ge.y - k0, 0), le);
                    m = slot_msgs<MsgT, SERVE>(C, base, s, sh.frame[s]) + ge.z + (c * tpc + p) * C.msg_stride;
                    dl = reinterpret_cast<float*>(base + C.p_bytes + C.m_bytes) + (cnl * tpc + p) * C.delta_stride;
                    et = tab + ge.x + k0;
#pragma unroll
                    for (int k = 0; k < LE; ++k) {
                        if (k < L) {
                            old[k] = to_f(m[k]);
                            t[k] = at_b(P, tile_vb(et[k], c, Z4)) - old[k];
                        }
                    }
                    lane_forward<LE>(t, L, lim, xu, pn, pe, cn, ce, lpar);
                }
                // product over the other lanes of the CN, and the total sign parity
                float on, oe;
                unsigned par;
                lane_exchange(tpc, gmask, cn, ce, lpar, on, oe, par);
                if (live) {
                    lane_backward<LE>(xu, pn, pe, L, on, oe, par & 0x80000000u, lim, [&](int k, float val) {
                        const MsgT q = from_f<MsgT>(val);
                        m[k] = q;
                        const float d = to_f(q) - old[k];
                        if (REGB)
                            dreg[k] = d;
                        else
                            dl[k] = d;
                    });
                }
            }
            __syncthreads();
            // ---- phase B: posterior += changes, layer position by layer position -----------
            if (REGB) {
                for (int jj = 0; jj < W; ++jj) {
                    if (live && j == jj) {
#pragma unroll
                        for (int k = 0; k < LE; ++k)
                            if (k < L) at_b(P, tile_vb(et[k], c, Z4)) += dreg[k];
                    }
                    __syncthreads();
                }
            } else {
                const int per_pos = Z * tpc;
                const int pwork = C.slots * per_pos;
                for (int jj = 0; jj < W; ++jj) {
                    for (int i = tid; i < pwork; i += nt) {
                        const int s = fast_div(i, C.div_pos);
                        if (sh.frame[s] < 0) continue;
                        const int w = i - s * per_pos;
                        const int cb = w >> tsh, p = w & (tpc - 1);
                        const int cnl = jj * Z + cb;
                        const int4 ge = gtab[sh.gofs[s] + g * W + jj];
                        const int k0 = p * le;
                        const int Lb = min(max(ge.y - k0, 0), le);
                        unsigned char* base = slots_base + static_cast<size_t>(s) * C.slot_bytes;
                        float* Pb = reinterpret_cast<float*>(base);
                        const float* dl = reinterpret_cast<const float*>(base + C.p_bytes + C.m_bytes) +
                                          (cnl * tpc + p) * C.delta_stride;
                        const int2* eb = tab + ge.x + k0;
#pragma unroll
                        for (int k = 0; k < LE; ++k)
                            if (k < Lb) at_b(Pb, tile_vb(eb[k], cb, Z4)) += dl[k];
                    }
                    __syncthreads();
                }
            }
        }
        // ---- Step 4: syndrome of every slot that needs it -----------------------------------
        if (tid < C.slots) {
            const int act = sh.frame[tid] >= 0 ? 1 : 0;
            set_iter(sh, C, tid, sh.iter[tid] + act);
            sh.epoch[tid] += act;
            sh.unsat[tid] = 0u;
        }
        __syncthreads();
        {
            const int per_s = nl * Z * tpc;
            const int swork = C.slots * per_s;
            const int srounds = (swork + nt - 1) / nt;
            for (int rr = 0; rr < srounds; ++rr) {
                const int i = rr * nt + tid;
                const int s = fast_div(i, C.div_syn);
                unsigned pbit = 0u;
                // a slot already found unsatisfied is decided: its remaining checks are skipped (the
                // flag only goes from 0 to 1 in this pass; the lanes of a CN read it together)
                const bool live = i < swork && sh.frame[s] >= 0 && (r.early_stop || sh.iter[s] >= r.max_iter) &&
                                  !(r.early_stop && *reinterpret_cast<volatile unsigned*>(&sh.unsat[s]));
                const int w = i - s * per_s;
                const int cn_i = w >> tsh, p = w & (tpc - 1);
                if (live) {
                    const int l = fast_div(cn_i, C.div_z), cs = cn_i - l * Z;
                    const int k0 = p * le;
                    const int Ls = min(max(ldeg[l] - k0, 0), le);
                    float* Ps = reinterpret_cast<float*>(slots_base + static_cast<size_t>(s) * C.slot_bytes);
                    const int2* es = tab + l * md + k0;
#pragma unroll
                    for (int k = 0; k < LE; ++k)
                        if (k < Ls) pbit ^= (at_b(Ps, tile_vb(es[k], cs, Z4)) < 0.f) ? 1u : 0u;
                }
                if (tpc > 1) {
                    pbit ^= __shfl_xor_sync(gmask, pbit, 1);
                    if (tpc == 4) pbit ^= __shfl_xor_sync(gmask, pbit, 2);
                }
                if (live && p == 0 && pbit) sh.unsat[s] = 1u;
            }
        }
        __syncthreads();
        // ---- retire finished frames (or, serving, park them) and refill their slots ---------
        for (int s = 0; s < C.slots; ++s) {
            const long long f = sh.frame[s];
            if (f < 0) continue;
            const int it = sh.iter[s];
            const bool done = (r.early_stop && !sh.unsat[s]) || it >= r.max_iter || sh.bad[s];
            const bool park = SERVE && !done && sh.epoch[s] >= C.epoch_iters;
            if (!done && !park) continue;
            unsigned char* base = slots_base + static_cast<size_t>(s) * C.slot_bytes;
            float* P = reinterpret_cast<float*>(base);
            if (done) {
                MsgT* msg = slot_msgs<MsgT, SERVE>(C, base, s, f);
                if (r.msgs_out) {
                    // edge k of CN c of layer l is CSR entry ebase(l) + c d_l + k (the rows of a
                    // layer share its degree and list their VNs by block column)
                    int ebase = 0;
                    for (int l = 0; l < nl; ++l) {
                        const int d = ldeg[l];
                        for (int i = tid; i < Z * d; i += nt) {
                            const int cc = i / d, k = i - cc * d, pl = k / le, kl = k - pl * le;
                            r.msgs_out[f * r.E + ebase + i] =
                                to_f(msg[((l * Z + cc) * tpc + pl) * C.msg_stride + kl]) * kLn2;
                        }
                        ebase += Z * d;
                    }
                }
                write_frame_outputs(r, P, f, it, sh.unsat[s] ? 1 : 0, &sh.err, 1, sh.bad[s] != 0);
                if (SERVE && tid == 0) {
                    C.state_flag[f] = kSlotDone;
                    if (C.done_list) C.done_list[atomicAdd(C.done_count, 1)] = static_cast<int>(f);
                }
            } else {
                save_frame<MsgT>(C, base, f);
                if (tid == 0) C.state_iter[f] = it;
            }
            __syncthreads();
            if (tid == 0) fill_slot<SERVE>(sh, C, s);
            __syncthreads();
            const long long nf = sh.frame[s];
            if (nf >= 0) load_frame<MsgT, SERVE>(C, sh, base, s, nf, sh.iter[s]);
            __syncthreads();
        }
        if (tid == 0) {
            int any = 0;
            for (int s = 0; s < C.slots; ++s) any |= sh.frame[s] >= 0;
            sh.active = any;
        }
        __syncthreads();
        if (!sh.active) break;
    }
}

// SINGLE: a launch over one code (codes[0]), whose parameters are read at fixed offsets of the
// kernel's parameter block (free operands); a multi-code launch indexes the parameter block by
// the tile's code at run time, a constant load at every use.  (Copying the current code's
// parameters to shared memory instead measured 2-3 % slower on the ragged and serving mixes.)
template <typename MsgT, bool SERVE, int LE, bool REGB, bool SINGLE>
__global__ void __launch_bounds__(1024) tile_decode_kernel(const TileArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ TileShared sh;
    const int tid = threadIdx.x, nt = blockDim.x;
    // tables of the current code at the start of shared memory, frame slots after them
    int2* tab = reinterpret_cast<int2*>(smem);
    unsigned char* slots_base = smem + a.table_bytes;
    if (tid == 0) {
        sh.cur_code = -1;
        sh.err = 0u;
    }
    for (;;) {
        if (tid == 0) sh.tile = static_cast<int>(atomicAdd(a.tile_counter, 1ull));
        __syncthreads();
        const int ti = sh.tile;
        if (ti >= a.n_tiles) break;
        int4 tile;
        if (a.tiles) {
            tile = a.tiles[ti];
        } else {
            const long long first = static_cast<long long>(ti) * a.tile_frames;
            tile = make_int4(0, static_cast<int>(first),
                             static_cast<int>(min(static_cast<long long>(a.tile_frames), a.codes[0].r.n_frames - first)), 0);
        }
        const TileCode& C = SINGLE ? a.codes[0] : a.codes[tile.x];
        const int nl = C.nl, md = C.maxdeg;
        // code tables: (4 (b Z + s), Z - s) per edge, layer degrees, per-group records
        int* ldeg = reinterpret_cast<int*>(tab + nl * md);
        const int gwk = C.G * C.window * C.n_groupings;
        int4* gtab = tile_group_records(tab, nl, md);
        if (sh.cur_code != tile.x) {
            for (int i = tid; i < nl * md; i += nt) tab[i] = C.edge_tab[i];
            for (int i = tid; i < nl; i += nt) ldeg[i] = C.layer_deg[i];
            for (int i = tid; i < gwk; i += nt) {
                const int l = C.group_layers[i];
                gtab[i] = make_int4(l * md, C.layer_deg[l], l * C.Z * C.tpc * C.msg_stride, 0);
            }
        }
        __syncthreads();
        if (tid == 0) {
            sh.cur_code = tile.x;
            sh.next = tile.y;
            sh.end = tile.y + tile.z;
            for (int s = 0; s < C.slots; ++s) fill_slot<SERVE>(sh, C, s);
        }
        __syncthreads();
        // initialisation of every filled slot: P_n = L_n, L_{m->n} = 0 (or the saved state)
        for (int s = 0; s < C.slots; ++s) {
            const long long f = sh.frame[s];
            if (f < 0) continue;
            load_frame<MsgT, SERVE>(C, sh, slots_base + static_cast<size_t>(s) * C.slot_bytes, s, f, sh.iter[s]);
        }
        __syncthreads();
        run_tile<MsgT, SERVE, LE, REGB>(C, tab, slots_base, sh);
    }
}

template <typename MsgT, bool SERVE, bool SINGLE>
static TileKernelFn pick_width(int lane_width, bool regb) {
    switch (lane_width) {
        case 4: return regb ? tile_decode_kernel<MsgT, SERVE, 4, true, SINGLE> : tile_decode_kernel<MsgT, SERVE, 4, false, SINGLE>;
        case 6: return regb ? tile_decode_kernel<MsgT, SERVE, 6, true, SINGLE> : tile_decode_kernel<MsgT, SERVE, 6, false, SINGLE>;
        case 8: return regb ? tile_decode_kernel<MsgT, SERVE, 8, true, SINGLE> : tile_decode_kernel<MsgT, SERVE, 8, false, SINGLE>;
        default: return nullptr;
    }
}

template <typename MsgT>
static TileKernelFn pick_mode(bool serve, int lane_width, bool regb, bool single) {
    // serving launches always take the multi-code form
    if (serve) return pick_width<MsgT, true, false>(lane_width, regb);
    return single ? pick_width<MsgT, false, true>(lane_width, regb) : pick_width<MsgT, false, false>(lane_width, regb);
}

TileKernelFn pick_tile_kernel(int msg_dtype, bool serve, int lane_width, bool regb, bool single) {
    switch (msg_dtype) {
        case NDGSBP_F32: return pick_mode<float>(serve, lane_width, regb, single);
        case NDGSBP_F16: return pick_mode<__half>(serve, lane_width, regb, single);
        case NDGSBP_BF16: return pick_mode<__nv_bfloat16>(serve, lane_width, regb, single);
        default: return nullptr;
    }
}

int tile_lane_width(int le) { return le < 1 ? 0 : le <= 4 ? 4 : le <= 6 ? 6 : le <= 8 ? 8 : 0; }

size_t tile_table_bytes(const QcLayout& Q) {
    const size_t G = Q.window ? Q.group_layers.size() / Q.window : 0;   // groups of every grouping
    size_t b = static_cast<size_t>(Q.n_layers) * Q.max_deg * 8 + static_cast<size_t>(Q.n_layers) * 4;
    b = (b + 15) & ~static_cast<size_t>(15);   // the per-group records (tile_group_records)
    return b + G * Q.window * 16;
}

TileShape tile_shape(const QcLayout& Q, int tpc, int msg_dtype) {
    TileShape t;
    t.tpc = tpc;
    t.le = (Q.max_deg + tpc - 1) / tpc;
    t.delta_stride = t.le | 1;
    // 16-bit messages: an even stride whose half (in 4-byte words) is odd
    t.msg_stride = msg_dtype == NDGSBP_F32 ? (t.le | 1) : 2 * (((t.le + 1) / 2) | 1);
    t.msg_slots = Q.n_layers * Q.Z * tpc * t.msg_stride;
    t.delta_floats = Q.window * Q.Z * tpc * t.delta_stride;
    return t;
}

void tile_code_finish(TileCode& C) {
    C.div_slot = make_fastdiv(static_cast<unsigned>(C.window * C.Z * C.tpc));
    C.div_pos = make_fastdiv(static_cast<unsigned>(C.Z * C.tpc));
    C.div_syn = make_fastdiv(static_cast<unsigned>(C.nl * C.Z * C.tpc));
    C.div_z = make_fastdiv(static_cast<unsigned>(C.Z));
    if (C.n_groupings < 1) C.n_groupings = 1;
}

int tile_lanes_per_cn(int maxdeg) { return maxdeg <= 8 ? 1 : maxdeg <= 16 ? 2 : maxdeg <= 32 ? 4 : 0; }

}  // namespace ndgsbp
