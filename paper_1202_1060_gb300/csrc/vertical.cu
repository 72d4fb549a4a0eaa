// Vertical (VN-group) shuffled BP, the shuffled schedule over variable nodes that Sec. I cites
// beside the CN-group schedules: the VNs are split into G disjoint groups; for each group in
// turn, every edge of the group's VNs receives its CN->VN message by Eq. (1) from the VN->CN
// messages as they stand when the group starts, and then every such edge gets its VN->CN
// message by Eq. (2).  Groups later in the iteration see the earlier groups' new messages.
// G = 1 is flooding; G = N updates one VN at a time.
//
// Kernel design: one CTA per frame, frames claimed from an atomic counter (persistent grid).
// A frame keeps its channel LLRs L_n and the running totals P_n = L_n + sum of the CN->VN
// messages into n in shared memory; the VN->CN message of edge (m, n) is P_n - L_{m->n} at any
// time, because the messages into a VN change only while its own group runs, when P_n is
// recomputed from them.  Per group: (1) Eq. (1) in the positive-pair tanh-product form of the
// other kernels into a staging array, either one thread per group edge (the product over the
// CN's other edges) or, for groups whose edges reach few CNs, one thread per CN (one
// prefix/suffix pass, outputs for the CN's group edges); (2) one thread per VN of the group
// stores its new messages and recomputes P_n.  Two barriers per group.  The CN->VN messages (CSR order) live in shared memory when
// the frame fits, else in the CTA's workspace slot.
#include <algorithm>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <vector>

#include "device_common.cuh"
#include "ndgsbp_internal.h"

namespace ndgsbp {

#define VCUDA_TRY(expr)                                                                        \
    do {                                                                                       \
        cudaError_t _e = (expr);                                                               \
        if (_e != cudaSuccess) return fail(NDGSBP_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(_e)); \
    } while (0)

constexpr size_t kVHeaderBytes = 256;   // workspace header: frame counter (bytes 0-7)

struct DeviceVTables {
    void* blob = nullptr;
    const int32_t* col_idx = nullptr;   // [E] VN of each CSR edge
    const int4* gtab = nullptr;         // [E] group edge a: (CSR edge e, row start b, row degree d, e - b)
    const int32_t* grp_ptr = nullptr;   // [G+1] into grp_vn
    const int32_t* grp_vn = nullptr;    // [N]
    const int32_t* vn_epos = nullptr;   // [N+1] group-edge position of grp_vn[i]'s first edge
    const int32_t* row_ptr = nullptr;   // [M+1]
    const int4* vtask = nullptr;        // per-CN groups: the CNs the group's edges reach, (row start b,
                                        // degree d, mask of their group edges' row positions, output base)
    const int32_t* gtask_ptr = nullptr; // [G+1] into vtask (an empty range: a per-edge group)
    const int32_t* vtout = nullptr;     // staging positions of each task's group edges, by row position
};

}  // namespace ndgsbp

struct ndgsbp_vgroups {
    std::shared_ptr<const ndgsbp::Code> code;
    int G = 0;
    std::vector<int32_t> grp_ptr, grp_vn;    // a partition of the N VNs
    std::vector<int4> gtab;                  // [E] group edges, VN-major within each group
    std::vector<int32_t> vn_epos;            // [N+1]
    std::vector<int4> vtask;                 // CN tasks of every group (see DeviceVTables)
    std::vector<int32_t> gtask_ptr, vtout;
    int max_group_edges = 0, max_group_vns = 0, max_group_work = 0;
    bool per_cn = false;                     // every group takes the per-CN form
    mutable std::mutex mu;
    mutable std::map<int, ndgsbp::DeviceVTables> dev;
    ~ndgsbp_vgroups();
};

namespace ndgsbp {

static ndgsbp_status finish_vgroups(const std::shared_ptr<const Code>& code, std::vector<int32_t> gp,
                                    std::vector<int32_t> gv, ndgsbp_vgroups** out) {
    const Code& c = *code;
    const int G = static_cast<int>(gp.size()) - 1;
    if (G < 1 || gp[0] != 0 || gp[G] != c.N || static_cast<int>(gv.size()) != c.N)
        return fail(NDGSBP_ERR_INVALID, "vgroups: the groups must list each of the %d VNs once", c.N);
    std::vector<uint8_t> seen(c.N, 0);
    for (int g = 0; g < G; ++g)
        if (gp[g + 1] <= gp[g]) return fail(NDGSBP_ERR_INVALID, "vgroups: group %d is empty", g);
    for (int32_t n : gv) {
        if (n < 0 || n >= c.N || seen[n]) return fail(NDGSBP_ERR_INVALID, "vgroups: VN %d missing or repeated", n);
        seen[n] = 1;
    }
    // columns: the CSR edges of each VN, in row order
    std::vector<int32_t> col_ptr(c.N + 1, 0), col_edge(c.E), edge_row(c.E);
    for (int64_t e = 0; e < c.E; ++e) col_ptr[c.col_idx[e] + 1]++;
    for (int n = 0; n < c.N; ++n) col_ptr[n + 1] += col_ptr[n];
    std::vector<int32_t> fill(col_ptr.begin(), col_ptr.end() - 1);
    for (int m = 0; m < c.M; ++m)
        for (int e = c.row_ptr[m]; e < c.row_ptr[m + 1]; ++e) {
            col_edge[fill[c.col_idx[e]]++] = e;
            edge_row[e] = m;
        }
    auto* h = new (std::nothrow) ndgsbp_vgroups();
    if (!h) return fail(NDGSBP_ERR_NOMEM, "vgroups: out of memory");
    h->code = code;
    h->G = G;
    h->gtab.reserve(c.E);
    h->vn_epos.assign(c.N + 1, 0);
    for (int g = 0; g < G; ++g) {
        const size_t first = h->gtab.size();
        for (int i = gp[g]; i < gp[g + 1]; ++i) {
            const int n = gv[i];
            h->vn_epos[i] = static_cast<int32_t>(h->gtab.size());
            for (int a = col_ptr[n]; a < col_ptr[n + 1]; ++a) {
                const int e = col_edge[a], m = edge_row[e], b = c.row_ptr[m];
                h->gtab.push_back(make_int4(e, b, c.row_ptr[m + 1] - b, e - b));
            }
        }
        h->max_group_edges = std::max(h->max_group_edges, static_cast<int>(h->gtab.size() - first));
        h->max_group_vns = std::max(h->max_group_vns, gp[g + 1] - gp[g]);
    }
    h->vn_epos[c.N] = static_cast<int32_t>(h->gtab.size());
    // Phase 1 runs either one thread per group edge (the product over the CN's other edges
    // directly) or one thread per CN the group reaches (one prefix/suffix pass over the CN, outputs
    // at the group's row positions).  A barrier ends the phase, so its time is that of the slowest
    // thread: the per-CN form is taken when in every group the edges average >= 4 per CN they
    // reach (e.g. one group of all VNs), the per-edge form otherwise, for the whole decode
    // (measured on n=2304, 10 iterations of 65,536 frames: one group, 6.6 edges per CN, per-CN
    // 34.5 against 59.2 ms; 4 groups, 1.9 edges per CN, 73.7 against 62.1 ms; mixing the two
    // forms in one phase, or keeping the per-CN code in the per-edge kernel, ran 12-70 % slower
    // than the plain per-edge kernel).
    h->gtask_ptr.assign(1, 0);
    h->vtout.assign(c.E, 0);
    std::vector<int32_t> task_of(c.M, -1);
    size_t obase = 0;
    for (int g = 0; g < G; ++g) {
        const size_t q0 = static_cast<size_t>(h->vn_epos[gp[g]]), q1 = static_cast<size_t>(h->vn_epos[gp[g + 1]]);
        std::vector<std::vector<std::pair<int, int>>> outs;   // per CN: (row position k, staging position)
        std::vector<int32_t> touched;
        for (size_t q = q0; q < q1; ++q) {
            const int4 ge = h->gtab[q];
            const int m = edge_row[ge.x];
            if (task_of[m] < 0) {
                task_of[m] = static_cast<int32_t>(outs.size());
                touched.push_back(m);
                outs.emplace_back();
            }
            outs[task_of[m]].push_back({ge.w, static_cast<int>(q - q0)});
        }
        for (int32_t m : touched) task_of[m] = -1;
        const size_t edges = q1 - q0;
        const bool dense = c.max_row <= 32 && edges >= 4 * touched.size();
        if (g == 0) h->per_cn = dense;
        h->per_cn = h->per_cn && dense;
        if (c.max_row <= 32) {   // the per-CN tasks (row-position masks need degrees <= 32)
            for (size_t i = 0; i < touched.size(); ++i) {
                const int m = touched[i], b = c.row_ptr[m], d = c.row_ptr[m + 1] - b;
                auto& o = outs[i];
                std::sort(o.begin(), o.end());
                uint32_t mask = 0u;
                for (const auto& kv : o) {
                    mask |= 1u << kv.first;
                    h->vtout[obase++] = kv.second;
                }
                h->vtask.push_back(make_int4(b, d, static_cast<int>(mask), static_cast<int>(obase - o.size())));
            }
        }
        h->gtask_ptr.push_back(static_cast<int32_t>(h->vtask.size()));
    }
    // threads: the most work items of a group phase in the chosen form
    for (int g = 0; g < G; ++g) {
        const int items = h->per_cn ? h->gtask_ptr[g + 1] - h->gtask_ptr[g] : h->vn_epos[gp[g + 1]] - h->vn_epos[gp[g]];
        h->max_group_work = std::max({h->max_group_work, items, gp[g + 1] - gp[g]});
    }
    h->grp_ptr = std::move(gp);
    h->grp_vn = std::move(gv);
    *out = h;
    return NDGSBP_OK;
}

// Device copy of a handle's tables for the current device (uploaded on first use).
static ndgsbp_status vgroups_device(const ndgsbp_vgroups* h, const DeviceVTables*& out) {
    int dev = 0;
    VCUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(h->mu);
    auto it = h->dev.find(dev);
    if (it != h->dev.end()) {
        out = &it->second;
        return NDGSBP_OK;
    }
    const Code& c = *h->code;
    auto al = [](size_t x) { return (x + 255) & ~static_cast<size_t>(255); };
    const size_t o_col = 0, o_gtab = al(o_col + 4 * c.E), o_gp = al(o_gtab + 16 * c.E),
                 o_gv = al(o_gp + 4 * (h->G + 1)), o_ep = al(o_gv + 4 * c.N), o_rp = al(o_ep + 4 * (c.N + 1)),
                 o_vt = al(o_rp + 4 * (c.M + 1)), o_tp = al(o_vt + 16 * h->vtask.size()),
                 o_vo = al(o_tp + 4 * h->gtask_ptr.size()), total = al(o_vo + 4 * h->vtout.size());
    std::vector<unsigned char> host(total, 0);
    std::memcpy(host.data() + o_col, c.col_idx.data(), 4 * c.E);
    std::memcpy(host.data() + o_gtab, h->gtab.data(), 16 * c.E);
    std::memcpy(host.data() + o_gp, h->grp_ptr.data(), 4 * (h->G + 1));
    std::memcpy(host.data() + o_gv, h->grp_vn.data(), 4 * c.N);
    std::memcpy(host.data() + o_ep, h->vn_epos.data(), 4 * (c.N + 1));
    std::memcpy(host.data() + o_rp, c.row_ptr.data(), 4 * (c.M + 1));
    std::memcpy(host.data() + o_vt, h->vtask.data(), 16 * h->vtask.size());
    std::memcpy(host.data() + o_tp, h->gtask_ptr.data(), 4 * h->gtask_ptr.size());
    std::memcpy(host.data() + o_vo, h->vtout.data(), 4 * h->vtout.size());
    void* d = nullptr;
    VCUDA_TRY(cudaMalloc(&d, total));
    cudaError_t e = cudaMemcpy(d, host.data(), total, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(d);
        return fail(NDGSBP_ERR_CUDA, "vgroups upload: %s", cudaGetErrorString(e));
    }
    DeviceVTables t;
    auto* b = static_cast<unsigned char*>(d);
    t.blob = d;
    t.col_idx = reinterpret_cast<const int32_t*>(b + o_col);
    t.gtab = reinterpret_cast<const int4*>(b + o_gtab);
    t.grp_ptr = reinterpret_cast<const int32_t*>(b + o_gp);
    t.grp_vn = reinterpret_cast<const int32_t*>(b + o_gv);
    t.vn_epos = reinterpret_cast<const int32_t*>(b + o_ep);
    t.row_ptr = reinterpret_cast<const int32_t*>(b + o_rp);
    t.vtask = reinterpret_cast<const int4*>(b + o_vt);
    t.gtask_ptr = reinterpret_cast<const int32_t*>(b + o_tp);
    t.vtout = reinterpret_cast<const int32_t*>(b + o_vo);
    out = &(h->dev[dev] = t);
    return NDGSBP_OK;
}

// ---- kernel --------------------------------------------------------------------------------
struct VArgs {
    RunArgs r;
    int M, G;
    DeviceVTables t;
    int msg_smem;        // 1: the frame's CN->VN messages in shared memory, 0: in the CTA's slot
    int stage_smem;      // 1: the staging array in shared memory, 0: in the CTA's slot
    void* ws_slots;      // [grid][slot_bytes]
    long long slot_bytes;
    int msg_bytes;       // E messages rounded up to 16 bytes
    int cidx_off;        // kernels with CSMEM: byte offset in shared memory of a copy of col_idx (E entries)
};

// Column index i: from the shared-memory copy (CSMEM) or through the read-only cache.
template <bool CSMEM>
__device__ __forceinline__ int32_t col_at(const int32_t* __restrict__ col_idx, int i) {
    if constexpr (CSMEM)
        return col_idx[i];
    else
        return __ldg(col_idx + i);
}

// Eq. (1) for one group edge (row position k) of a CN of degree d: the product over the CN's
// other edges directly, in the same (N, E) pair form.  A CN of degree 1 gives +lim.
template <bool CSMEM, typename MsgT>
__device__ __forceinline__ float vertical_edge_message(const float* __restrict__ P, const MsgT* msg,
                                                       const int32_t* __restrict__ col_idx, int b, int d, int k,
                                                       float lim) {
    unsigned par = 0u;
    float cn = 1.f, ce = 0.f;
    for (int j = 0; j < d; ++j) {
        if (j == k) continue;
        const float v = P[col_at<CSMEM>(col_idx, b + j)] - to_f(msg[b + j]);   // L_{n'->m} = P_n' - L_{m->n'}
        par ^= __float_as_uint(v);
        const float u = ex2_approx(-fminf(fabsf(v), lim));
        ce = fmaf(ce, fmaf(0.5f, u, 0.5f), cn * u);
        cn = cn * fmaf(-0.5f, u, 0.5f);
    }
    const float w = fmaf(cn * rcp_approx(ce), 2.f, 1.f);
    const float mag = fminf(lg2_approx(w), lim);
    return __uint_as_float(__float_as_uint(mag) | (par & 0x80000000u));
}

// Eq. (1) for one CN of degree d <= MAXDC (row start b): the VN->CN messages of its edges
// (P_n - L_{m->n}, log2 units) as a product of (N, E) pairs (tanh(x/2) = N / (N + E), u = e^-x,
// (N, E) = ((1 - u) / 2, u); pairs combine as (Na Nb, Ea (Eb + Nb) + Na Eb)), "all edges but k" =
// prefix(k) x suffix(k + 1), and 2 atanh(N / (N + E)) = ln(1 + 2 N / E); inputs and outputs
// clipped to lim.  Only the row positions in mask (the group's edges) get an output: written to
// stage[out[i]], the i-th set bit of mask counted from position 0.  A CN of degree 1 gives +lim
// (the empty product is 1).
template <int MAXDC, bool CSMEM, typename MsgT>
__device__ __forceinline__ void vertical_cn_task(const float* __restrict__ P, const MsgT* msg,
                                                 const int32_t* __restrict__ col_idx, int b, int d, unsigned mask,
                                                 const int32_t* __restrict__ out, float* stage, float lim) {
    float xs[MAXDC], pn[MAXDC], pe[MAXDC];
    unsigned par = 0u;
    float cn = 1.f, ce = 0.f;
#pragma unroll
    for (int k = 0; k < MAXDC; ++k) {
        if (k < d) {
            const float v = P[col_at<CSMEM>(col_idx, b + k)] - to_f(msg[b + k]);   // L_{n->m} = P_n - L_{m->n}
            const unsigned tb = __float_as_uint(v);
            par ^= tb;
            const float u = ex2_approx(-fminf(fabsf(v), lim));
            xs[k] = __uint_as_float(__float_as_uint(u) | (tb & 0x80000000u));
            pn[k] = cn;
            pe[k] = ce;
            ce = fmaf(ce, fmaf(0.5f, u, 0.5f), cn * u);
            cn = cn * fmaf(-0.5f, u, 0.5f);
        }
    }
    const unsigned pm = par & 0x80000000u;
    int o = __popc(mask) - 1;   // outputs in decreasing row position
    float sn = 1.f, se = 0.f;
#pragma unroll
    for (int k = MAXDC - 1; k >= 0; --k) {
        if (k < d) {
            const float u = fabsf(xs[k]);
            const float ss = sn + se;
            if ((mask >> k) & 1u) {
                const float en = pn[k] * sn;
                const float ee = fmaf(pe[k], ss, pn[k] * se);
                const float w = fmaf(en * rcp_approx(ee), 2.f, 1.f);
                const float mag = fminf(lg2_approx(w), lim);
                stage[__ldg(out + o)] = __uint_as_float(__float_as_uint(mag) | ((__float_as_uint(xs[k]) ^ pm) & 0x80000000u));
                --o;
            }
            se = fmaf(u, ss, se * fmaf(-0.5f, u, 0.5f));
            sn = sn * fmaf(-0.5f, u, 0.5f);
        }
    }
}

// CSMEM: col_idx read from a shared-memory copy (the plan found room for it without losing a CTA
// per SM), else through the read-only cache.
template <typename MsgT, int MAXDC, bool PCN, bool CSMEM>
__global__ void __launch_bounds__(512) vertical_decode_kernel(const VArgs a) {
    extern __shared__ __align__(16) unsigned char vsm[];
    __shared__ long long s_frame;
    __shared__ unsigned s_err;
    const RunArgs& r = a.r;
    const DeviceVTables& t = a.t;
    const int N = r.N, E = r.E, tid = threadIdx.x, nt = blockDim.x;
    const float lim = r.llr_max;
    float* Lch = reinterpret_cast<float*>(vsm);   // [N] channel LLRs
    float* P = Lch + N;                           // [N] running totals
    unsigned char* rest = vsm + 8 * static_cast<size_t>(N);
    unsigned char* slot = static_cast<unsigned char*>(a.ws_slots) + static_cast<size_t>(blockIdx.x) * a.slot_bytes;
    MsgT* msg = reinterpret_cast<MsgT*>(a.msg_smem ? rest : slot);
    float* stage = reinterpret_cast<float*>(a.stage_smem ? (a.msg_smem ? rest + a.msg_bytes : rest)
                                                         : (a.msg_smem ? slot : slot + a.msg_bytes));
    // the column indices, read d times per edge output (the copy is made once; next_frame's
    // barrier orders it)
    const int32_t* col_idx = t.col_idx;
    if constexpr (CSMEM) {
        int32_t* cs = reinterpret_cast<int32_t*>(vsm + a.cidx_off);
        for (int e = tid; e < E; e += nt) cs[e] = __ldg(t.col_idx + e);
        col_idx = cs;
    }
    if (tid == 0) s_err = 0u;
    for (long long f = next_frame(r, &s_frame); f < r.n_frames; f = next_frame(r, &s_frame)) {
        if (r.start_ns && tid == 0) r.start_ns[f] = global_timer_ns();
        const bool invalid = load_frame_llrs(r, Lch, f);
        for (int n = tid; n < N; n += nt) P[n] = Lch[n];
        for (int e = tid; e < E; e += nt) msg[e] = from_f<MsgT>(0.f);
        __syncthreads();
        int it = 1, unsat = 1;
        for (; !invalid; ++it) {
            for (int g = 0; g < a.G; ++g) {
                const int v0 = __ldg(t.grp_ptr + g), v1 = __ldg(t.grp_ptr + g + 1);
                const int a0 = __ldg(t.vn_epos + v0);
                // Eq. (1) into every edge of the group's VNs, from the messages at the group's
                // start: one pass per CN the group reaches, or one thread per group edge
                if constexpr (PCN) {
                    const int t1 = __ldg(t.gtask_ptr + g + 1);
                    for (int i = __ldg(t.gtask_ptr + g) + tid; i < t1; i += nt) {
                        const int4 tk = __ldg(t.vtask + i);
                        vertical_cn_task<MAXDC, CSMEM>(P, msg, col_idx, tk.x, tk.y, static_cast<unsigned>(tk.z),
                                                t.vtout + tk.w, stage, lim);
                    }
                } else {
                    const int a1 = __ldg(t.vn_epos + v1);
                    for (int q = a0 + tid; q < a1; q += nt) {
                        const int4 ge = __ldg(t.gtab + q);
                        stage[q - a0] = vertical_edge_message<CSMEM>(P, msg, col_idx, ge.y, ge.z, ge.w, lim);
                    }
                }
                __syncthreads();
                // Eq. (2): store the group's messages; P_n = L_n + their sum
                for (int i = v0 + tid; i < v1; i += nt) {
                    const int n = __ldg(t.grp_vn + i);
                    const int q1 = __ldg(t.vn_epos + i + 1);
                    float s = Lch[n];
                    for (int q = __ldg(t.vn_epos + i); q < q1; ++q) {
                        const MsgT mq = from_f<MsgT>(stage[q - a0]);
                        msg[__ldg(&t.gtab[q].x)] = mq;
                        s += to_f(mq);
                    }
                    P[n] = s;
                }
                __syncthreads();
            }
            // Step 4: d_n = 1 iff P_n < 0; stop when every check is satisfied (early_stop)
            bool bad = false;
            for (int m = tid; m < a.M && !bad; m += nt) {
                bool p = false;
                const int e1 = __ldg(t.row_ptr + m + 1);
                for (int e = __ldg(t.row_ptr + m); e < e1; ++e) p ^= P[col_at<CSMEM>(col_idx, e)] < 0.f;
                bad = p;
            }
            unsat = __syncthreads_or(bad);
            if ((!unsat && r.early_stop) || it >= r.max_iter) break;
        }
        if (r.msgs_out)
            for (int e = tid; e < E; e += nt) r.msgs_out[f * E + e] = to_f(msg[e]) * kLn2;
        write_frame_outputs(r, P, f, it, unsat, &s_err, 1, invalid);
    }
}

typedef void (*VKernelFn)(const VArgs);

template <typename MsgT, bool CSMEM>
static VKernelFn pick_vertical_degree(int maxdc, bool per_cn) {
    if (!per_cn) return vertical_decode_kernel<MsgT, 8, false, CSMEM>;   // the degree bound is not used
    if (maxdc <= 8) return vertical_decode_kernel<MsgT, 8, true, CSMEM>;
    if (maxdc <= 16) return vertical_decode_kernel<MsgT, 16, true, CSMEM>;
    if (maxdc <= 32) return vertical_decode_kernel<MsgT, 32, true, CSMEM>;
    return nullptr;
}

template <bool CSMEM>
static VKernelFn pick_vertical_csmem(int msg_dtype, int maxdc, bool per_cn) {
    switch (msg_dtype) {
        case NDGSBP_F16: return pick_vertical_degree<__half, CSMEM>(maxdc, per_cn);
        case NDGSBP_BF16: return pick_vertical_degree<__nv_bfloat16, CSMEM>(maxdc, per_cn);
        default: return pick_vertical_degree<float, CSMEM>(maxdc, per_cn);
    }
}

static VKernelFn pick_vertical_kernel(int msg_dtype, int maxdc, bool per_cn, bool csmem) {
    return csmem ? pick_vertical_csmem<true>(msg_dtype, maxdc, per_cn)
                 : pick_vertical_csmem<false>(msg_dtype, maxdc, per_cn);
}

// ---- planning --------------------------------------------------------------------------------
struct VPlan {
    VKernelFn fn = nullptr;
    int threads = 0, per_sm = 0, msg_smem = 0, stage_smem = 0, msg_bytes = 0, cidx_off = -1;
    size_t smem = 0, slot_bytes = 0;
    int64_t grid = 0, ws_bytes = 0;
};

static ndgsbp_status validate_vparams(const ndgsbp_params* p) {
    if (!p) return fail(NDGSBP_ERR_INVALID, "params is null");
    if (p->max_iter < 1) return fail(NDGSBP_ERR_INVALID, "max_iter must be >= 1");
    if (p->msg_dtype != NDGSBP_F32 && p->msg_dtype != NDGSBP_F16 && p->msg_dtype != NDGSBP_BF16)
        return fail(NDGSBP_ERR_INVALID, "msg_dtype must be F32, F16 or BF16");
    if (!(p->llr_max > 0.f && p->llr_max <= 30.f)) return fail(NDGSBP_ERR_INVALID, "llr_max must be in (0, 30]");
    if (p->block_threads < 0 || p->block_threads > 512 || p->block_threads % 32)
        return fail(NDGSBP_ERR_INVALID, "vertical: block_threads must be 0 or a multiple of 32 up to 512");
    if (p->ctas_per_sm < 0) return fail(NDGSBP_ERR_INVALID, "ctas_per_sm must be >= 0");
    if (p->variant != NDGSBP_VARIANT_AUTO && p->variant != NDGSBP_VARIANT_SMEM && p->variant != NDGSBP_VARIANT_GLOBAL)
        return fail(NDGSBP_ERR_INVALID, "vertical: variant must be AUTO, SMEM or GLOBAL");
    return NDGSBP_OK;
}

static ndgsbp_status make_vplan(const ndgsbp_vgroups* h, const ndgsbp_params* p, int64_t n_frames, VPlan& vp) {
    ndgsbp_status st = validate_vparams(p);
    if (st) return st;
    const Code& c = *h->code;
    int dev = 0, sms = 0, optin = 0;
    VCUDA_TRY(cudaGetDevice(&dev));
    VCUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    VCUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const int msz = p->msg_dtype == NDGSBP_F32 ? 4 : 2;
    auto a16 = [](size_t x) { return (x + 15) & ~static_cast<size_t>(15); };
    const size_t base = 8 * static_cast<size_t>(c.N);
    const size_t mb = a16(static_cast<size_t>(c.E) * msz), sb = a16(4 * static_cast<size_t>(h->max_group_edges));
    // messages and staging in shared memory when they fit, then the staging alone, then neither
    // (SMEM: the first only; GLOBAL: the messages in the workspace)
    const int opts[3][2] = {{1, 1}, {0, 1}, {0, 0}};
    const int k0 = p->variant == NDGSBP_VARIANT_GLOBAL ? 1 : 0, k1 = p->variant == NDGSBP_VARIANT_SMEM ? 1 : 3;
    int k = k0;
    for (; k < k1; ++k) {
        const size_t need = base + (opts[k][0] ? mb : 0) + (opts[k][1] ? sb : 0);
        if (need <= static_cast<size_t>(optin)) break;
    }
    if (k == k1)
        return fail(NDGSBP_ERR_UNSUPPORTED, "vertical: %d VNs and %lld edges do not fit in %d bytes of shared memory%s",
                    c.N, static_cast<long long>(c.E), optin, p->variant == NDGSBP_VARIANT_SMEM ? " (variant SMEM)" : "");
    vp.fn = pick_vertical_kernel(p->msg_dtype, c.max_row, h->per_cn, false);
    vp.msg_smem = opts[k][0];
    vp.stage_smem = opts[k][1];
    vp.msg_bytes = static_cast<int>(mb);
    vp.smem = base + (vp.msg_smem ? mb : 0) + (vp.stage_smem ? sb : 0);
    vp.slot_bytes = ((vp.msg_smem ? 0 : mb) + (vp.stage_smem ? 0 : sb) + 255) & ~static_cast<size_t>(255);
    const int work = h->max_group_work;
    vp.threads = p->block_threads ? p->block_threads : std::min(512, std::max(64, (work + 31) / 32 * 32));
    const void* fn = reinterpret_cast<const void*>(vp.fn);
    VCUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(vp.smem)));
    VCUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&vp.per_sm, fn, vp.threads, vp.smem));
    if (vp.per_sm < 1) return fail(NDGSBP_ERR_UNSUPPORTED, "vertical kernel does not fit on an SM with %d threads", vp.threads);
    // the kernel reading a copy of col_idx placed after the rest, when it costs no CTA per SM
    const size_t cb = a16(4 * static_cast<size_t>(c.E));
    if (vp.smem + cb <= static_cast<size_t>(optin)) {
        const VKernelFn fn2 = pick_vertical_kernel(p->msg_dtype, c.max_row, h->per_cn, true);
        const void* f2 = reinterpret_cast<const void*>(fn2);
        int per_sm2 = 0;
        VCUDA_TRY(cudaFuncSetAttribute(f2, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(vp.smem + cb)));
        VCUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm2, f2, vp.threads, vp.smem + cb));
        if (per_sm2 >= vp.per_sm) {
            vp.fn = fn2;
            vp.cidx_off = static_cast<int>(vp.smem);
            vp.smem += cb;
        }
    }
    if (p->ctas_per_sm > 0) vp.per_sm = std::min(vp.per_sm, p->ctas_per_sm);
    vp.grid = std::max<int64_t>(1, std::min<int64_t>(static_cast<int64_t>(vp.per_sm) * sms, std::max<int64_t>(n_frames, 1)));
    vp.ws_bytes = static_cast<int64_t>(kVHeaderBytes) + vp.grid * static_cast<int64_t>(vp.slot_bytes);
    return NDGSBP_OK;
}

}  // namespace ndgsbp

using namespace ndgsbp;

ndgsbp_vgroups::~ndgsbp_vgroups() {
    int cur = 0;
    if (cudaGetDevice(&cur) != cudaSuccess) return;
    for (auto& kv : dev)
        if (cudaSetDevice(kv.first) == cudaSuccess) cudaFree(kv.second.blob);
    dev.clear();
    cudaSetDevice(cur);
    cudaGetLastError();
}

extern "C" {

ndgsbp_status ndgsbp_vgroups_build(const ndgsbp_code* code, int32_t G, uint64_t seed, int32_t flags,
                                   ndgsbp_vgroups** out) {
    clear_error();
    if (!code || !out) return fail(NDGSBP_ERR_INVALID, "vgroups_build: null pointer");
    if (flags & ~NDGSBP_GROUPS_NATURAL) return fail(NDGSBP_ERR_INVALID, "vgroups_build: flags may hold NATURAL only");
    const Code& c = *code->c;
    std::vector<std::vector<int>> ug;
    ndgsbp_status st = draw_groups(c.N, G, 0.0, seed, flags, ug);
    if (st) return st;
    std::vector<int32_t> gp(1, 0), gv;
    gv.reserve(c.N);
    for (auto& grp : ug) {
        gv.insert(gv.end(), grp.begin(), grp.end());
        gp.push_back(static_cast<int32_t>(gv.size()));
    }
    return finish_vgroups(code->c, std::move(gp), std::move(gv), out);
}

ndgsbp_status ndgsbp_vgroups_from_lists(const ndgsbp_code* code, const int32_t* grp_ptr, const int32_t* grp_vn,
                                        int32_t G, ndgsbp_vgroups** out) {
    clear_error();
    if (!code || !grp_ptr || !grp_vn || !out || G < 1) return fail(NDGSBP_ERR_INVALID, "vgroups_from_lists: bad argument");
    const Code& c = *code->c;
    if (grp_ptr[0] != 0 || grp_ptr[G] != c.N)
        return fail(NDGSBP_ERR_INVALID, "vgroups_from_lists: grp_ptr must run from 0 to N = %d", c.N);
    std::vector<int32_t> gp(grp_ptr, grp_ptr + G + 1), gv(grp_vn, grp_vn + c.N);
    return finish_vgroups(code->c, std::move(gp), std::move(gv), out);
}

ndgsbp_status ndgsbp_vgroups_query(const ndgsbp_vgroups* vg, int32_t* G, int32_t* grp_ptr, int32_t* grp_vn,
                                   int32_t* max_group_edges) {
    clear_error();
    if (!vg) return fail(NDGSBP_ERR_INVALID, "vgroups_query: null handle");
    if (G) *G = vg->G;
    if (grp_ptr) std::copy(vg->grp_ptr.begin(), vg->grp_ptr.end(), grp_ptr);
    if (grp_vn) std::copy(vg->grp_vn.begin(), vg->grp_vn.end(), grp_vn);
    if (max_group_edges) *max_group_edges = vg->max_group_edges;
    return NDGSBP_OK;
}

ndgsbp_status ndgsbp_vgroups_destroy(ndgsbp_vgroups* vg) {
    delete vg;
    return NDGSBP_OK;
}

ndgsbp_status ndgsbp_vertical_workspace_size(const ndgsbp_vgroups* vg, const ndgsbp_params* params,
                                             int64_t n_frames, size_t* bytes) {
    clear_error();
    if (!vg || !bytes) return fail(NDGSBP_ERR_INVALID, "vertical_workspace_size: null pointer");
    VPlan vp;
    ndgsbp_status st = make_vplan(vg, params, n_frames, vp);
    if (st) return st;
    *bytes = static_cast<size_t>(vp.ws_bytes);
    return NDGSBP_OK;
}

ndgsbp_status ndgsbp_decode_vertical(const ndgsbp_vgroups* vg, const ndgsbp_params* params, const void* d_llr,
                                     int32_t llr_dtype, int64_t n_frames, void* d_workspace, size_t workspace_bytes,
                                     uint32_t* d_hard_bits, int32_t* d_iters, uint8_t* d_syndrome_ok,
                                     float* d_posterior, const ndgsbp_extras* extras, void* stream) {
    clear_error();
    if (!vg) return fail(NDGSBP_ERR_INVALID, "decode_vertical: null handle");
    if (n_frames < 0) return fail(NDGSBP_ERR_INVALID, "decode_vertical: n_frames < 0");
    if (llr_dtype != NDGSBP_F32 && llr_dtype != NDGSBP_F64 && llr_dtype != NDGSBP_F16 && llr_dtype != NDGSBP_BF16)
        return fail(NDGSBP_ERR_INVALID, "decode_vertical: unknown llr_dtype %d", llr_dtype);
    if (n_frames > 0 && (!d_llr || !d_hard_bits))
        return fail(NDGSBP_ERR_INVALID, "decode_vertical: d_llr and d_hard_bits are required");
    const size_t le = llr_dtype == NDGSBP_F64 ? 8 : llr_dtype == NDGSBP_F32 ? 4 : 2;
    if (reinterpret_cast<uintptr_t>(d_llr) % le || reinterpret_cast<uintptr_t>(d_hard_bits) % 4 ||
        reinterpret_cast<uintptr_t>(d_iters) % 4 || reinterpret_cast<uintptr_t>(d_posterior) % 4)
        return fail(NDGSBP_ERR_INVALID, "decode_vertical: a buffer is not aligned to its element");
    VPlan vp;
    ndgsbp_status st = make_vplan(vg, params, n_frames, vp);
    if (st) return st;
    if (n_frames == 0) return NDGSBP_OK;
    if (!d_workspace || workspace_bytes < static_cast<size_t>(vp.ws_bytes))
        return fail(NDGSBP_ERR_WORKSPACE, "decode_vertical: workspace of %zu bytes, need %lld", workspace_bytes,
                    static_cast<long long>(vp.ws_bytes));
    if (reinterpret_cast<uintptr_t>(d_workspace) % 256)
        return fail(NDGSBP_ERR_WORKSPACE, "decode_vertical: workspace must be 256-byte aligned");
    const DeviceVTables* t = nullptr;
    st = vgroups_device(vg, t);
    if (st) return st;
    const Code& c = *vg->code;
    VArgs a;
    std::memset(&a, 0, sizeof(a));
    RunArgs& r = a.r;
    r.N = c.N;
    r.E = static_cast<int>(c.E);
    r.W = (c.N + 31) / 32;
    r.llr = d_llr;
    r.llr_dtype = llr_dtype;
    r.n_frames = n_frames;
    r.max_iter = params->max_iter;
    r.llr_max = kernel_llr_limit(params->llr_max);
    r.early_stop = params->early_stop ? 1 : 0;
    auto* ws = static_cast<unsigned char*>(d_workspace);
    r.counter = reinterpret_cast<unsigned long long*>(ws);
    r.hard_bits = d_hard_bits;
    r.iters = d_iters;
    r.synd_ok = d_syndrome_ok;
    r.posterior = d_posterior;
    if (extras) {
        r.ref_bits = extras->d_ref_bits;
        r.ref_per_frame = extras->ref_per_frame;
        r.stats = reinterpret_cast<unsigned long long*>(extras->d_stats);
        r.iter_hist = reinterpret_cast<unsigned long long*>(extras->d_iter_hist);
        r.start_ns = reinterpret_cast<unsigned long long*>(extras->d_start_ns);
        r.retire_ns = reinterpret_cast<unsigned long long*>(extras->d_retire_ns);
        r.msgs_out = extras->d_messages;
    }
    a.M = c.M;
    a.G = vg->G;
    a.t = *t;
    a.msg_smem = vp.msg_smem;
    a.stage_smem = vp.stage_smem;
    a.ws_slots = ws + kVHeaderBytes;
    a.slot_bytes = static_cast<long long>(vp.slot_bytes);
    a.msg_bytes = vp.msg_bytes;
    a.cidx_off = vp.cidx_off;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    VCUDA_TRY(cudaMemsetAsync(ws, 0, 16, s));   // frame counter
    vp.fn<<<static_cast<unsigned>(vp.grid), vp.threads, vp.smem, s>>>(a);
    VCUDA_TRY(cudaGetLastError());
    return NDGSBP_OK;
}

}  // extern "C"
