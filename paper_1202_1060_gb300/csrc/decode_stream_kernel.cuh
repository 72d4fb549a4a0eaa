// Stream decode kernel for sm_103a: layered QC codes whose window is too large for one thread
// per CN of the window (n=16200: 2 layers of Z = 360 CNs; n=8192: degree 22).
//
// A CTA decodes one frame at a time (persistent CTAs, frames from an atomic counter, so a frame
// that stops early frees its CTA at once).  Thread t = p Z + c owns lane p of CN c of a layer
// (tpc = 1, or 2 for degrees above 11: lane p holds edges [p le, (p+1) le), le =
// ceil(maxdeg / tpc), as in the tile kernel; the two lanes of a CN are in different warps and
// exchange their pair totals through shared memory, see pair_exchange) and steps
// through the W layers of each group in window order:
//   phase A, position j = 0..W-1: Eq. (1) for CN c of layer L_g[j] from t = P - L_old (P as it
//     stood at the start of the sub-iteration: phase A writes no posterior), new messages stored,
//     their changes kept in a shared delta buffer (positions < W-1) or in registers (W-1);
//   phase B: P += changes, position by position (a barrier after each), the fixed order of the
//     other kernels -- with tpc = 1 the results equal the QC and tile kernels bit for bit, with
//     tpc = 2 those of the tile kernel at 2 lanes per CN (the same lane split and pair products).
// Messages are stored per layer, CN-major with an odd word stride in shared memory (each thread's
// messages at compile-time offsets, consecutive CNs in distinct banks) and edge-major in global
// memory (edge k of CN c at k Zr + c, Zr = Z rounded up to 16 elements: the lanes of a warp
// write whole sectors); see stream_layer_elems.  MODE picks where they live:
//   kStreamSmem:   the frame's messages in shared memory;
//   kStreamGlobal: in the CTA's workspace slot (mostly L2-resident), read and written in place;
//   kStreamBulk:   in the CTA's workspace slot, each layer's slab (d_l Z messages, one contiguous
//                  block) staged in shared memory: for cyclic windows advancing one layer per
//                  group, layer k of the layer sequence (k counts windows' newest layers across
//                  iterations) lives in slab buffer k mod (W + 2); at the start of group g one
//                  thread writes back the slab that left the window (cp.async.bulk store) and
//                  loads the layer group g + 1 adds (cp.async.bulk load completing on that
//                  buffer's mbarrier), so loads and stores overlap a whole group of work.  A
//                  layer's first use in a frame reads no messages (they start at 0).  Every
//                  mbarrier wait is bounded: a wait that gives up sets bit 0 of the status word,
//                  the CTA drains its copies and returns.
// Posteriors and messages are in log2 units (see load_llr).
#pragma once

#include <type_traits>

#include "decode_stream.h"
#include "lane_cnu.cuh"

namespace ndgsbp {

// ---- bulk copies and mbarriers (inline PTX) ------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Arrive (count 1) and add `bytes` to the transaction count of the barrier's current phase.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Wait until the phase of `bar` with the given parity has completed, at most `limit` polls
// (after the first 32, each poll sleeps ~64 ns).  Returns false when the wait gave up.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, unsigned limit) {
    for (unsigned i = 0; i < limit; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if (i >= 32) __nanosleep(64);
    }
    return false;
}

// Global -> shared bulk copy (16-byte aligned addresses, size a multiple of 16) completing on bar.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// Shared -> global bulk copy in the issuing thread's current bulk async-group.
__device__ __forceinline__ void bulk_store(void* dst, const void* src, unsigned bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_addr(src)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

// Wait until at most N of this thread's committed bulk groups are still pending (complete: the
// writes are performed).
template <int N>
__device__ __forceinline__ void bulk_wait() {
    asm volatile("cp.async.bulk.wait_group %0;" ::"n"(N) : "memory");
}

// Order this thread's generic-proxy shared-memory writes before later async-proxy accesses.
__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// OLD16: 16-bit messages whose new values phase B reads back from shared memory (shared-memory
// and bulk-staged modes) keep the old message (2 bytes) instead of the change (4 bytes): half the
// buffer, which lets n=8192 keep 2 CTAs per SM beside the pair-exchange slots.  In global mode
// the read-back would be a global load, so the change is kept.
template <typename MsgT, int MODE>
struct Old16 {
    static constexpr bool value = sizeof(MsgT) == 2 && MODE != kStreamGlobal;
};
template <typename MsgT, int MODE>
using DeltaT = typename std::conditional<Old16<MsgT, MODE>::value, MsgT, float>::type;

// ---- shared-memory layout (stream_smem_bytes on the host computes the same sizes) ------------
__host__ __device__ constexpr size_t sa16(size_t x) { return (x + 15) & ~static_cast<size_t>(15); }

struct StreamSmem {
    float* P;          // [N] posterior (log2 units)
    void* dbuf;        // [W - 1][Z][maxdeg | 1] per position 0 .. W-2 (entry p le + k for lane p): the
                       // message changes, or the old messages where Old16 holds (phase B forms the
                       // change from the new message, the same FP32 value)
    unsigned char* msg;  // SMEM: [msg_elems] messages; BULK: [n_slabs][slab_elems] slab buffers
    int2* tab;         // [nl][maxdeg] edge table
    int* ldeg;         // [nl] layer degrees
    int4* gtab;        // [n_groupings][G][W] (l maxdeg, d_l, lbase[l], first use in iteration 1)
    uint64_t* bar;     // BULK: [n_slabs] one mbarrier per slab buffer
    float2* xbuf;      // tpc = 2: [2 slots][2 lanes][Z] pair totals exchanged between the lanes of a CN
    size_t slab_bytes;
};

template <typename MsgT, int MODE>
__device__ __forceinline__ StreamSmem stream_smem(unsigned char* smem, const StreamArgs& a) {
    StreamSmem s;
    size_t off = 0;
    s.P = reinterpret_cast<float*>(smem);
    off += sa16(static_cast<size_t>(a.r.N) * 4);
    s.dbuf = smem + off;
    off += sa16(static_cast<size_t>(a.window - 1) * (a.maxdeg | 1) * a.Z * (Old16<MsgT, MODE>::value ? 2 : 4));
    s.msg = smem + off;
    s.slab_bytes = sa16(static_cast<size_t>(a.slab_elems) * sizeof(MsgT));
    if (MODE == kStreamSmem) off += sa16(static_cast<size_t>(a.msg_elems) * sizeof(MsgT));
    if (MODE == kStreamBulk) off += static_cast<size_t>(a.n_slabs) * s.slab_bytes;
    s.tab = reinterpret_cast<int2*>(smem + off);
    off += sa16(static_cast<size_t>(a.nl) * a.maxdeg * 8);
    s.ldeg = reinterpret_cast<int*>(smem + off);
    off += sa16(static_cast<size_t>(a.nl) * 4);
    s.gtab = reinterpret_cast<int4*>(smem + off);
    off += static_cast<size_t>(a.n_groupings) * a.G * a.window * 16;
    s.xbuf = reinterpret_cast<float2*>(smem + off);
    if (a.tpc == 2) off += static_cast<size_t>(4) * a.Z * sizeof(float2);
    s.bar = reinterpret_cast<uint64_t*>(smem + off);
    return s;
}

// Bytes of a layer's CN-major block (a bulk copy's size).
template <typename MsgT>
__device__ __forceinline__ unsigned stream_slab_bytes(int d, int Z) {
    return static_cast<unsigned>(stream_layer_elems(d, Z, 0, sizeof(MsgT), kStreamBulk) * sizeof(MsgT));
}

// The two lanes of a CN (tpc = 2) sit in different warps: lane p of CN c is thread p Z + c, so
// the 32 threads of a warp read one block column of P at 32 consecutive VNs -- distinct banks
// (with both lanes of a CN in one warp, two block columns at unrelated circulant shifts shared
// the banks: 41.6 % of the shared-memory wavefronts were conflicts for n=8192).  The lanes swap
// their pair totals through shared memory (xw: this lane's entry, xr: the other lane's) and
// meet at a named barrier of their two warps (id xid); two slots alternate, so an entry is
// rewritten only after the other lane has passed the next barrier, i.e. after it has read it.
// cn >= 0, so its sign bit carries the lane's sign parity.  The values are those lane_exchange
// gives for two lanes: the other lane's (cn, ce), and the parity of all the CN's input signs.
// Raw bits of a 16-bit message and back (HOLD in stream_lane).
template <typename MsgT>
__device__ __forceinline__ unsigned short msg_bits(MsgT v);
template <>
__device__ __forceinline__ unsigned short msg_bits<__half>(__half v) { return __half_as_ushort(v); }
template <>
__device__ __forceinline__ unsigned short msg_bits<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat16_as_ushort(v); }
template <>
__device__ __forceinline__ unsigned short msg_bits<float>(float) { return 0; }
template <typename MsgT>
__device__ __forceinline__ MsgT msg_from_bits(unsigned short b);
template <>
__device__ __forceinline__ __half msg_from_bits<__half>(unsigned short b) { return __ushort_as_half(b); }
template <>
__device__ __forceinline__ __nv_bfloat16 msg_from_bits<__nv_bfloat16>(unsigned short b) { return __ushort_as_bfloat16(b); }
template <>
__device__ __forceinline__ float msg_from_bits<float>(unsigned short) { return 0.f; }

struct PairX {
    uint32_t xw, xr;   // shared-memory addresses of this lane's and the other lane's entry
    int xid;
};

__device__ __forceinline__ void pair_exchange(const PairX& x, float cn, float ce, unsigned lpar, float& on, float& oe,
                                              unsigned& par) {
    const float sc = __uint_as_float(__float_as_uint(cn) | (lpar & 0x80000000u));
    asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"(x.xw), "f"(sc), "f"(ce) : "memory");
    asm volatile("bar.sync %0, 64;" ::"r"(x.xid) : "memory");
    float o0, o1;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(o0), "=f"(o1) : "r"(x.xr) : "memory");
    on = __uint_as_float(__float_as_uint(o0) & 0x7fffffffu);
    oe = o1;
    par = lpar ^ (__float_as_uint(o0) & 0x80000000u);
}

// Eq. (1) for one lane of CN c (its L <= NP edges at edge-table entries et[0..L-1]) with the
// messages of that lane at m[k Z], k < L: t = P - L_old (L_old = 0 on a layer's first use in
// the frame), new messages written back to m, changes to drow[k Z] (shared delta buffer; for
// 16-bit messages the old message instead) or dreg[k] (TO_REG).  NP positions are computed: NP = L exactly (no predicates), or NP = LE with
// the positions past L neutral (see lane_forward).  The old message is read again from m when
// its change is formed rather than held in a register through the pass (fewer live registers;
// measured faster).  Lanes of a CN (tpc = 2) run it together and exchange through x.
template <typename MsgT, int MODE, int TPC, int LE, int NP, bool TO_REG>
__device__ __forceinline__ void stream_lane(const int2* __restrict__ et, int L, int c, int Zm, int Zd, int Z4,
                                            const float* __restrict__ P, MsgT* m, bool first, float lim,
                                            const PairX& x, DeltaT<MsgT, MODE>* __restrict__ drow, float (&dreg)[LE]) {
    static_assert(NP <= LE, "positions above the lane width");
    if (NP < LE) L = NP;   // exact instance: L is the constant NP
    float t[NP], xu[NP], pn[NP], pe[NP];
    float cn = 1.f, ce = 0.f;
    unsigned lpar = 0u;
    // 16-bit messages in global memory at one lane per CN: the old messages stay in registers, two
    // per word, for the backward pass (a re-read would be a global load); otherwise (and at two
    // lanes per CN, whose 64-register budget they would push into spills) they are read again
    constexpr bool HOLD = sizeof(MsgT) == 2 && MODE == kStreamGlobal && TPC == 1;
    uint32_t ob[HOLD ? (NP + 1) / 2 : 1];
#pragma unroll
    for (int i = 0; i < (HOLD ? (NP + 1) / 2 : 1); ++i) ob[i] = 0u;
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        if (k < L) {
            const MsgT om = first ? from_f<MsgT>(0.f) : m[k * Zm];
            if constexpr (HOLD) ob[k / 2] |= static_cast<uint32_t>(msg_bits(om)) << (16 * (k & 1));
            t[k] = at_b(const_cast<float*>(P), tile_vb(et[k], c, Z4)) - to_f(om);
        }
    }
    lane_forward<NP>(t, L, lim, xu, pn, pe, cn, ce, lpar);
    float on = 1.f, oe = 0.f;
    unsigned par = lpar;
    if (TPC == 2) pair_exchange(x, cn, ce, lpar, on, oe, par);
    lane_backward<NP>(xu, pn, pe, L, on, oe, par & 0x80000000u, lim, [&](int k, float val) {
        const MsgT q = from_f<MsgT>(val);
        MsgT om;
        if constexpr (HOLD)
            om = msg_from_bits<MsgT>(static_cast<unsigned short>(ob[k / 2] >> (16 * (k & 1))));
        else
            om = first ? from_f<MsgT>(0.f) : m[k * Zm];
        m[k * Zm] = q;
        const float d = to_f(q) - to_f(om);
        if constexpr (TO_REG)
            dreg[k] = d;
        else if constexpr (Old16<MsgT, MODE>::value)
            drow[k * Zd] = om;   // phase B forms to_f(new) - to_f(old): the same value d
        else
            drow[k * Zd] = d;
    });
}

// Exact-degree dispatch for a CN of degree d split into L-edge lanes: a layer's CNs share their
// degree, so the branch is uniform across a warp (for tpc = 2 only when both lanes hold LE
// edges); other degrees take the padded width-LE path.
template <typename MsgT, int MODE, int LE, int TPC, bool TO_REG>
__device__ __forceinline__ void stream_lane_d(int d, const int2* __restrict__ et, int L, int c, int Zm, int Zd, int Z4,
                                              const float* __restrict__ P, MsgT* m, bool first, float lim,
                                              const PairX& x, DeltaT<MsgT, MODE>* __restrict__ drow, float (&dreg)[LE]) {
    if (d == TPC * LE)
        stream_lane<MsgT, MODE, TPC, LE, LE, TO_REG>(et, LE, c, Zm, Zd, Z4, P, m, first, lim, x, drow, dreg);
    else if (TPC == 1 && d == LE - 1)
        stream_lane<MsgT, MODE, TPC, LE, LE - 1, TO_REG>(et, L, c, Zm, Zd, Z4, P, m, first, lim, x, drow, dreg);
    else if (TPC == 1 && d == LE - 2)
        stream_lane<MsgT, MODE, TPC, LE, LE - 2, TO_REG>(et, L, c, Zm, Zd, Z4, P, m, first, lim, x, drow, dreg);
    else
        stream_lane<MsgT, MODE, TPC, LE, LE, TO_REG>(et, L, c, Zm, Zd, Z4, P, m, first, lim, x, drow, dreg);
}

// P += changes of one lane, change k = src(k) for k < L: EXACT instances take L = NP (no
// predicates).  src is a functor so that register arrays stay in registers.
template <int NP, bool EXACT, typename Src>
__device__ __forceinline__ void stream_add(float* __restrict__ P, const int2* __restrict__ et, int L, int c, int Z4,
                                           Src src) {
    if (EXACT) L = NP;
#pragma unroll
    for (int k = 0; k < NP; ++k)
        if (k < L) at_b(P, tile_vb(et[k], c, Z4)) += src(k);
}

template <int LE, int TPC, typename Src>
__device__ __forceinline__ void stream_add_d(int d, float* __restrict__ P, const int2* __restrict__ et, int L, int c,
                                             int Z4, Src src) {
    if (d == TPC * LE)
        stream_add<LE, true>(P, et, L, c, Z4, src);
    else if (TPC == 1 && d == LE - 1)
        stream_add<LE - 1, true>(P, et, L, c, Z4, src);
    else if (TPC == 1 && d == LE - 2)
        stream_add<LE - 2, true>(P, et, L, c, Z4, src);
    else
        stream_add<LE, false>(P, et, L, c, Z4, src);
}

// Parity of the hard decisions on one lane's L edges, with the same dispatch.
template <int NP, bool EXACT>
__device__ __forceinline__ unsigned stream_parity(const float* __restrict__ P, const int2* __restrict__ et, int L,
                                                  int c, int Z4) {
    if (EXACT) L = NP;
    unsigned pb = 0u;
#pragma unroll
    for (int k = 0; k < NP; ++k)
        if (k < L) pb ^= (at_b(const_cast<float*>(P), tile_vb(et[k], c, Z4)) < 0.f) ? 1u : 0u;
    return pb;
}

template <int LE, int TPC>
__device__ __forceinline__ unsigned stream_parity_d(int d, const float* __restrict__ P, const int2* __restrict__ et,
                                                    int L, int c, int Z4) {
    if (d == TPC * LE) return stream_parity<LE, true>(P, et, L, c, Z4);
    if (TPC == 1 && d == LE - 1) return stream_parity<LE - 1, true>(P, et, L, c, Z4);
    if (TPC == 1 && d == LE - 2) return stream_parity<LE - 2, true>(P, et, L, c, Z4);
    return stream_parity<LE, false>(P, et, L, c, Z4);
}

// Launch bounds: 2 resident CTAs of up to 384 threads (tpc = 1; 85 registers) or 512 (tpc = 2;
// 64 registers).
__host__ __device__ constexpr int stream_block_bound(int tpc) { return tpc == 1 ? 384 : 512; }

// SERVE (shared-memory and global modes): a serving launch advances the pool slots of
// serve_list.  A new slot starts from its staged LLRs, a running one resumes from its saved
// posterior (and, with shared-memory messages, its saved messages; global-mode messages live in
// the slot's state); a frame runs until it retires (zero syndrome or I_max: outputs written, slot
// marked done and listed) or has run epoch_iters iterations in this launch (state saved, slot
// stays running).
template <typename MsgT, int LE, int TPC, int MODE, bool SERVE = false>
__global__ void __launch_bounds__(stream_block_bound(TPC), 2) stream_decode_kernel(const StreamArgs a) {
    static_assert(!SERVE || MODE != kStreamBulk, "serving launches keep messages in shared or global memory");
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long s_frame;
    __shared__ unsigned s_err;
    const RunArgs& r = a.r;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int Z = a.Z, Z4 = 4 * a.Z, W = a.window, nl = a.nl, md = a.maxdeg;
    const int Zr = a.zr;   // global edge-major row stride (Z rounded up to 16 elements)
    const int Sd = md | 1; // delta buffer: CN-major, odd stride
    const int le = a.le;   // edges per lane (<= LE): lane p holds edges [p le, (p + 1) le) of its CN
    const StreamSmem s = stream_smem<MsgT, MODE>(smem, a);
    float* P = s.P;
    for (int i = tid; i < nl * md; i += nt) s.tab[i] = a.edge_tab[i];
    for (int i = tid; i < nl; i += nt) s.ldeg[i] = a.layer_deg[i];
    const int gw1 = a.G * W, gwk = gw1 * a.n_groupings;
    for (int i = tid; i < gwk; i += nt) {
        const int l = a.group_layers[i];
        s.gtab[i] = make_int4(l * md, a.layer_deg[l], a.lbase[l], i < gw1 ? a.first_use[i] : 0);
    }
    if (MODE == kStreamBulk && tid == 0) {
        for (int b = 0; b < a.n_slabs; ++b) mbar_init(s.bar + b, 1);
        fence_mbar_init();
    }
    if (tid == 0) s_err = 0u;
    // (the leading barrier of next_frame orders the tables and barrier set-up before any use)
    // lane p of CN c: thread p Z + c (for tpc = 2 the plan makes Z a multiple of 32 and the block
    // 2 Z threads, so a warp holds one lane of 32 consecutive CNs)
    const int p = TPC == 1 ? 0 : tid / Z;
    const int c = tid - p * Z;
    const bool active = c < Z && p < TPC;
    int xs = 0;   // exchange slot (tpc = 2)
    const uint32_t xb0 = smem_addr(s.xbuf);
    const float lim = r.llr_max;
    MsgT* gmsg = MODE != kStreamSmem ? static_cast<MsgT*>(a.ws_msgs) + static_cast<size_t>(blockIdx.x) * a.ws_stride
                                     : nullptr;
    MsgT* smsg = reinterpret_cast<MsgT*>(s.msg);
    const int S = a.n_slabs;
    // BULK bookkeeping, the same in every thread: bit b of ph = parity of the next wait on buffer
    // b, bit b of pend = a load into buffer b has been issued and not yet waited for
    unsigned ph = 0u, pend = 0u;
    bool abort = false;
    for (;;) {
        const long long fi = next_frame(r, &s_frame);
        if (fi >= r.n_frames) break;
        long long f = fi;
        int it0 = 0;            // iterations done before this launch
        bool invalid = false;   // NaN or infinity among the frame's LLRs: not decoded
        if constexpr (SERVE) {
            f = a.serve_list[fi];
            const int fl = a.state_flag[f];
            if (fl != kSlotNew && fl != kSlotRunning) continue;   // uniform: every thread read the same flag
            if (MODE == kStreamGlobal) gmsg = static_cast<MsgT*>(a.state_msgs) + static_cast<size_t>(f) * a.ws_stride;
            if (fl == kSlotNew) {
                if (r.start_ns && tid == 0) r.start_ns[f] = global_timer_ns();
                invalid = load_frame_llrs(r, P, f);
            } else {
                it0 = a.state_iter[f];
                const float* sp = a.state_P + static_cast<size_t>(f) * r.N;
                for (int n = tid; n < r.N; n += nt) P[n] = sp[n];
                if (MODE == kStreamSmem) {
                    const MsgT* sm = static_cast<const MsgT*>(a.state_msgs) + static_cast<size_t>(f) * a.ws_stride;
                    for (int e = tid; e < a.msg_elems; e += nt) smsg[e] = sm[e];
                }
            }
            __syncthreads();   // every thread has read the flag before it changes
            if (tid == 0) a.state_flag[f] = kSlotRunning;
        } else {
            if (r.start_ns && tid == 0) r.start_ns[f] = global_timer_ns();
            invalid = load_frame_llrs(r, P, f);
        }
        int it = it0 + 1, unsat = 1;
        int gsel = (it0 % a.n_groupings) * gw1;   // iteration it uses grouping (it - 1) mod n_groupings
        bool park = false;
        // BULK: kg = layer-sequence index of the current group's position 0 (it never reaches
        // 2^31: max_iter G < 2^31), kb = kg mod S (its slab buffer), kr = kg mod nl (its ring position)
        int kg = 0, kb = 0, kr = 0;
        bool failed = false;    // BULK: a bounded wait of this thread gave up
        for (; !invalid; ++it) {
            const int4* gt = s.gtab + gsel;
            for (int g = 0; g < a.G; ++g) {
                if (MODE == kStreamBulk && !failed) {   // after a failed wait: no more copies
                    // the window's newest layer (sequence kg + W - 1) was loaded at the start of
                    // group g - 1, unless it is that layer's first use in the frame
                    int bn = kb + W - 1;
                    bn -= bn >= S ? S : 0;
                    if ((pend >> bn) & 1u) {
                        failed |= !mbar_wait_bounded(s.bar + bn, (ph >> bn) & 1u, a.wait_limit);
                        ph ^= 1u << bn;
                        pend &= ~(1u << bn);
                    }
                    const int kl = kg + W;   // the layer group g + 1 adds
                    int bl = kb + W;           // its buffer, (kb + W) mod S
                    bl -= bl >= S ? S : 0;
                    if (tid == 0 && !failed) {
                        if (kg >= 1) {   // write back the layer that left the window (sequence kg - 1)
                            const int bo = kb == 0 ? S - 1 : kb - 1;
                            const int lo = a.ring[kr == 0 ? nl - 1 : kr - 1];
                            bulk_store(gmsg + a.lbase[lo], s.msg + static_cast<size_t>(bo) * s.slab_bytes,
                                       stream_slab_bytes<MsgT>(s.ldeg[lo], Z));
                        }
                        bulk_commit();
                        // the store committed one group ago (buffer bl) has completed
                        bulk_wait<1>();
                        if (kl >= nl) {
                            int rl = kr + W;   // ring position of the new layer, (kr + W) mod nl
                            rl -= rl >= nl ? nl : 0;
                            const int ll = a.ring[rl];
                            const unsigned bytes = stream_slab_bytes<MsgT>(s.ldeg[ll], Z);
                            mbar_arrive_expect_tx(s.bar + bl, bytes);
                            if (!(a.test_skip_load && kl == nl))
                                bulk_load(s.msg + static_cast<size_t>(bl) * s.slab_bytes, gmsg + a.lbase[ll], bytes,
                                          s.bar + bl);
                        }
                    }
                    if (kl >= nl) pend |= 1u << bl;
                }
                // ---- phase A: Eq. (1) on CN c of every layer of the window, in window order ----
                float dreg[LE];
                // this lane's messages of window position j (layer record ge)
                auto msg_at = [&](int j, const int4& ge) -> MsgT* {
                    if constexpr (MODE == kStreamSmem) {
                        return smsg + ge.z + c * stream_cn_stride(ge.y, sizeof(MsgT)) + p * le;
                    } else if constexpr (MODE == kStreamGlobal) {
                        return gmsg + ge.z + p * le * Zr + c;
                    } else {
                        const int bj = kb + j < S ? kb + j : kb + j - S;
                        return reinterpret_cast<MsgT*>(s.msg + static_cast<size_t>(bj) * s.slab_bytes) +
                               c * stream_cn_stride(ge.y, sizeof(MsgT)) + p * le;
                    }
                };
                DeltaT<MsgT, MODE>* dbuf = static_cast<DeltaT<MsgT, MODE>*>(s.dbuf);
                if (active) {
                    for (int j = 0; j < W; ++j) {
                        const int4 ge = gt[g * W + j];
                        const int L = min(max(ge.y - p * le, 0), le);
                        const int2* et = s.tab + ge.x + p * le;
                        const bool first = it == 1 && ge.w;
                        MsgT* m = msg_at(j, ge);
                        // row stride of a thread's messages: 1 (CN-major) or Zr (edge-major)
                        const int Zm = MODE == kStreamGlobal ? Zr : 1;
                        const PairX x{xb0 + static_cast<uint32_t>((2 * xs + p) * Z + c) * 8u,
                                      xb0 + static_cast<uint32_t>((2 * xs + 1 - p) * Z + c) * 8u, 1 + (c >> 5)};
                        xs ^= 1;
                        if (j == W - 1) {
                            stream_lane_d<MsgT, MODE, LE, TPC, true>(ge.y, et, L, c, Zm, 1, Z4, P, m, first, lim, x,
                                                               nullptr, dreg);
                        } else {
                            DeltaT<MsgT, MODE>* drow = dbuf + static_cast<size_t>(j * Z + c) * Sd + p * le;
                            stream_lane_d<MsgT, MODE, LE, TPC, false>(ge.y, et, L, c, Zm, 1, Z4, P, m, first, lim, x,
                                                                drow, dreg);
                        }
                    }
                    if constexpr (MODE == kStreamBulk) fence_async_shared();   // slabs written before their store
                }
                __syncthreads();
                // ---- phase B: P += changes, layer position by layer position --------------------
                for (int jj = 0; jj < W; ++jj) {
                    if (active) {
                        const int4 ge = gt[g * W + jj];
                        const int L = min(max(ge.y - p * le, 0), le);
                        const int2* et = s.tab + ge.x + p * le;
                        if (jj == W - 1) {
                            stream_add_d<LE, TPC>(ge.y, P, et, L, c, Z4, [&](int k) { return dreg[k]; });
                        } else {
                            const DeltaT<MsgT, MODE>* drow = dbuf + static_cast<size_t>(jj * Z + c) * Sd + p * le;
                            if constexpr (Old16<MsgT, MODE>::value) {
                                const MsgT* mj = msg_at(jj, ge);
                                const int Zm = MODE == kStreamGlobal ? Zr : 1;
                                stream_add_d<LE, TPC>(ge.y, P, et, L, c, Z4,
                                                      [&](int k) { return to_f(mj[k * Zm]) - to_f(drow[k]); });
                            } else {
                                stream_add_d<LE, TPC>(ge.y, P, et, L, c, Z4, [&](int k) { return drow[k]; });
                            }
                        }
                    }
                    __syncthreads();
                }
                if constexpr (MODE == kStreamBulk) {
                    ++kg;
                    kb = kb + 1 == S ? 0 : kb + 1;
                    kr = kr + 1 == nl ? 0 : kr + 1;
                }
            }
            if constexpr (MODE == kStreamBulk) {
                if (__syncthreads_or(failed)) {
                    abort = true;
                    break;
                }
            }
            const bool last = it >= r.max_iter;
            if (r.early_stop || last) {
                unsigned bad = 0u;
                // one thread per CN and layer: with tpc = 2 lane p checks whole CNs of the layers
                // l = p, p + 2, ... (both halves of the edge list), uniform across its warp
                for (int l = p; l < nl; l += TPC) {
                    unsigned pb = 0u;
                    if (active) {
                        const int d = s.ldeg[l];
                        const int2* et = s.tab + l * md;
                        pb = stream_parity_d<LE, TPC>(d, P, et, min(d, le), c, Z4);
                        if (TPC == 2) pb ^= stream_parity_d<LE, TPC>(d, P, et + le, max(d - le, 0), c, Z4);
                    }
                    bad |= pb;
                    // once a lane has found an unsatisfied check the frame's syndrome is decided
                    if (__any_sync(0xffffffffu, bad)) break;
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
                for (int n = tid; n < r.N; n += nt) sp[n] = P[n];
                if (MODE == kStreamSmem) {
                    MsgT* sm = static_cast<MsgT*>(a.state_msgs) + static_cast<size_t>(f) * a.ws_stride;
                    for (int e = tid; e < a.msg_elems; e += nt) sm[e] = smsg[e];
                }
                if (tid == 0) a.state_iter[f] = it;
                continue;   // (next_frame's leading barrier orders these reads before P is reused)
            }
        }
        if constexpr (MODE == kStreamBulk) {
            // drain: the load issued at the start of the last group, then every store
            for (int b = 0; b < S; ++b) {
                if (!failed && ((pend >> b) & 1u)) {
                    failed |= !mbar_wait_bounded(s.bar + b, (ph >> b) & 1u, a.wait_limit);
                    ph ^= 1u << b;
                }
            }
            pend = 0u;
            if (tid == 0) {
                if (!failed && !invalid && !abort && r.msgs_out) {
                    // the last window's layers (sequences kg - 1 .. kg + W - 2) are only in shared memory
                    for (int j = 0; j < W; ++j) {
                        const int kk = kg - 1 + j;
                        const int lj = a.ring[kk % nl];
                        bulk_store(gmsg + a.lbase[lj], s.msg + static_cast<size_t>(kk % S) * s.slab_bytes,
                                   stream_slab_bytes<MsgT>(s.ldeg[lj], Z));
                    }
                }
                bulk_commit();
                bulk_wait<0>();
                fence_async_global();
            }
            if (__syncthreads_or(failed)) abort = true;
        }
        if (abort) break;   // uniform: this CTA's frame is incomplete and its outputs are not written
        if (r.msgs_out) {
            // edge k of CN c of layer l is CSR entry layer_csr[l] + c d_l + k (the rows of a layer
            // share its degree and list their VNs by block column)
            for (int l = 0; l < nl; ++l) {
                const int d = s.ldeg[l];
                const int csr = a.layer_csr[l];
                const int cb = csr < 0 ? -csr - 1 : csr;
                const bool zero = csr < 0 || invalid;
                const MsgT* src = (MODE == kStreamSmem ? smsg : gmsg) + a.lbase[l];
                const int S_l = stream_cn_stride(d, sizeof(MsgT));
                for (int i = tid; i < d * Z; i += nt) {
                    const int rr = i / Z, cc = i - rr * Z;
                    const int at = MODE == kStreamGlobal ? rr * Zr + cc : cc * S_l + rr;
                    r.msgs_out[f * r.E + cb + cc * d + rr] = zero ? 0.f : to_f(src[at]) * kLn2;
                }
            }
        }
        write_frame_outputs(r, P, f, it, unsat, &s_err, 1, invalid);
        if (SERVE && tid == 0) {
            a.state_flag[f] = kSlotDone;
            a.done_list[atomicAdd(a.done_count, 1)] = static_cast<int>(f);
        }
    }
    if (MODE == kStreamBulk && abort && tid == 0) atomicOr(a.status, 1u);
}

}  // namespace ndgsbp
