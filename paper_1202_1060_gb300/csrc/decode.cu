// Batched NDGSBP decoding for sm_103a: the general (table-driven) kernel and the host-side
// planner and launcher for every decode kernel.
//
// One persistent CTA decodes one frame at a time and takes the next frame from an atomic
// counter when it finishes, so frames that stop early (Step 4 b) free their CTA at once.
// The frame's running total LLR P_n (Eq. (3)) lives in shared memory.  CN->VN messages live
// in shared memory when they fit (SMEM variant) or in a per-CTA slot of the workspace
// (GLOBAL variant), stored in tiles of 32 CNs so that a warp touches 32 consecutive words per
// edge index.
//
// Sub-iteration g (Step 2 of Sec. II-C) runs in two phases separated by a barrier:
//   A) every CN of G_g, one thread per CN: t_k = P_{n_k} - L_{m->n_k} (the VN->CN message of
//      Eq. (2), taken at the start of the sub-iteration), then Eq. (1) for all its edges, the
//      new message stored and its change recorded;
//   B) P_n += change for every edge of the group, in "colour" order: colour c of an edge is
//      the number of earlier edges of the group on the same VN, so each colour touches a VN at
//      most once and the sum order is fixed (results do not depend on scheduling or batch).
// The layered QC kernel (decode_qc.cu) runs the same two phases with circulant index
// arithmetic instead of tables.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <new>

#include "decode_qc.h"
#include "decode_stream.h"
#include "decode_tile.h"
#include "device_common.cuh"
#include "ndgsbp_internal.h"

namespace ndgsbp {

struct DecodeArgs {
    RunArgs r;
    int M, Epad, G, max_gd;
    const int32_t* slot_deg;
    const int32_t* tile_base;
    const int32_t* edge_vn;
    const int32_t* edge_csr;
    const int32_t* grp_ptr;
    const int32_t* ge_slot;
    const int32_t* ge_dpos;
    const int32_t* grp_colbase;
    const int32_t* grp_ncol;
    const uint8_t* gcol;
    void* ws_msgs;
    float* ws_delta;
};

// Phase A for one group entry: Eq. (1) on every edge of the entry's CN.
template <int MAXDC, typename MsgT>
__device__ __forceinline__ void cn_update_entry(const DecodeArgs& a, const float* __restrict__ P,
                                                MsgT* __restrict__ msg, float* __restrict__ delta, int i) {
    const int s = __ldg(a.ge_slot + i);
    const int d = __ldg(a.slot_deg + s);
    const int eb = __ldg(a.tile_base + (s >> 5)) + (s & 31);
    const int db = __ldg(a.ge_dpos + i);
    float t[MAXDC], old[MAXDC];
#pragma unroll
    for (int k = 0; k < MAXDC; ++k) {
        if (k < d) {
            const int v = __ldg(a.edge_vn + eb + 32 * k);
            old[k] = to_f(msg[eb + 32 * k]);
            t[k] = P[v] - old[k];
        }
    }
    check_node_update<MAXDC>(t, d, a.r.llr_max, [&](int k, float val) {
        const MsgT q = from_f<MsgT>(val);
        msg[eb + 32 * k] = q;
        delta[db + 32 * k] = to_f(q) - old[k];
    });
}

// Phase B for one group entry and one colour.
template <int MAXDC>
__device__ __forceinline__ void push_entry(const DecodeArgs& a, float* __restrict__ P,
                                           const float* __restrict__ delta,
                                           const uint8_t* __restrict__ col, int i, int c) {
    const int s = __ldg(a.ge_slot + i);
    const int d = __ldg(a.slot_deg + s);
    const int eb = __ldg(a.tile_base + (s >> 5)) + (s & 31);
    const int db = __ldg(a.ge_dpos + i);
#pragma unroll
    for (int k = 0; k < MAXDC; ++k) {
        if (k < d && __ldg(col + db + 32 * k) == c) {
            const int v = __ldg(a.edge_vn + eb + 32 * k);
            P[v] += delta[db + 32 * k];
        }
    }
}

__device__ __forceinline__ unsigned slot_parity(const DecodeArgs& a, const float* __restrict__ P, int s) {
    const int d = __ldg(a.slot_deg + s);
    const int eb = __ldg(a.tile_base + (s >> 5)) + (s & 31);
    unsigned p = 0u;
    for (int k = 0; k < d; ++k) p ^= (P[__ldg(a.edge_vn + eb + 32 * k)] < 0.f) ? 1u : 0u;
    return p;
}

template <typename MsgT, bool MSG_SMEM, bool DELTA_SMEM, int MAXDC>
__global__ void __launch_bounds__(max_threads_for(MAXDC)) decode_kernel(const DecodeArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long s_frame;
    __shared__ unsigned s_err;
    const RunArgs& r = a.r;
    const int tid = threadIdx.x, nt = blockDim.x;
    float* P = reinterpret_cast<float*>(smem);
    size_t off = (static_cast<size_t>(r.N) * 4 + 15) & ~static_cast<size_t>(15);
    MsgT* msg;
    if (MSG_SMEM) {
        msg = reinterpret_cast<MsgT*>(smem + off);
        off += (static_cast<size_t>(a.Epad) * sizeof(MsgT) + 15) & ~static_cast<size_t>(15);
    } else {
        msg = static_cast<MsgT*>(a.ws_msgs) + static_cast<size_t>(blockIdx.x) * a.Epad;
    }
    float* delta = DELTA_SMEM ? reinterpret_cast<float*>(smem + off)
                              : a.ws_delta + static_cast<size_t>(blockIdx.x) * a.max_gd;
    if (tid == 0) s_err = 0u;
    for (;;) {
        const long long f = next_frame(r, &s_frame);
        if (f >= r.n_frames) break;
        if (r.start_ns && tid == 0) r.start_ns[f] = global_timer_ns();
        // initialisation: P_n = L_n, L_{m->n} = 0
        for (int e = tid; e < a.Epad; e += nt) msg[e] = from_f<MsgT>(0.f);
        const bool invalid = load_frame_llrs(r, P, f);
        int it = 1, unsat = 1;
        for (; !invalid; ++it) {
            for (int g = 0; g < a.G; ++g) {
                const int gb = __ldg(a.grp_ptr + g), ge = __ldg(a.grp_ptr + g + 1);
                for (int i = gb + tid; i < ge; i += nt) cn_update_entry<MAXDC, MsgT>(a, P, msg, delta, i);
                __syncthreads();
                const int ncol = __ldg(a.grp_ncol + g);
                const uint8_t* col = a.gcol + __ldg(a.grp_colbase + g);
                for (int c = 0; c < ncol; ++c) {
                    for (int i = gb + tid; i < ge; i += nt) push_entry<MAXDC>(a, P, delta, col, i, c);
                    __syncthreads();
                }
            }
            const bool last = it >= r.max_iter;
            if (r.early_stop || last) {
                unsigned bad = 0u;
                for (int s = tid; s < a.M && !bad; s += nt) bad |= slot_parity(a, P, s);
                unsat = __syncthreads_or(bad);
                if (!unsat && r.early_stop) break;
            }
            if (last) break;
        }
        if (r.msgs_out) {
            for (int e = tid; e < a.Epad; e += nt) {
                const int csr = __ldg(a.edge_csr + e);
                if (csr >= 0) r.msgs_out[f * r.E + csr] = to_f(msg[e]) * kLn2;
            }
        }
        write_frame_outputs(r, P, f, it, unsat, &s_err, 1, invalid);
        __syncthreads();
    }
}

// ---- kernel table -------------------------------------------------------------------------
typedef void (*KernelFn)(const DecodeArgs);

template <typename MsgT, int MAXDC>
static KernelFn pick_storage(bool msg_smem, bool delta_smem) {
    if (msg_smem) return decode_kernel<MsgT, true, true, MAXDC>;
    if (delta_smem) return decode_kernel<MsgT, false, true, MAXDC>;
    return decode_kernel<MsgT, false, false, MAXDC>;
}

template <typename MsgT>
static KernelFn pick_degree(int maxdc, bool msg_smem, bool delta_smem) {
    switch (maxdc) {
        case 8: return pick_storage<MsgT, 8>(msg_smem, delta_smem);
        case 16: return pick_storage<MsgT, 16>(msg_smem, delta_smem);
        case 32: return pick_storage<MsgT, 32>(msg_smem, delta_smem);
        default: return nullptr;
    }
}

static KernelFn pick_kernel(int msg_dtype, int maxdc, bool msg_smem, bool delta_smem) {
    switch (msg_dtype) {
        case NDGSBP_F32: return pick_degree<float>(maxdc, msg_smem, delta_smem);
        case NDGSBP_F16: return pick_degree<__half>(maxdc, msg_smem, delta_smem);
        case NDGSBP_BF16: return pick_degree<__nv_bfloat16>(maxdc, msg_smem, delta_smem);
        default: return nullptr;
    }
}

static int msg_size(int dt) { return dt == NDGSBP_F32 ? 4 : 2; }
static size_t align16(size_t x) { return (x + 15) & ~static_cast<size_t>(15); }
static size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }
static int degree_bound(int d) { return d <= 8 ? 8 : d <= 16 ? 16 : d <= 32 ? 32 : 0; }
static constexpr size_t kHeaderBytes = 256;   // workspace header: frame counter (bytes 0-7), status word (8-11)
static constexpr size_t kStatusEnd = 16;

#define CUDA_TRY(expr)                                                                         \
    do {                                                                                       \
        cudaError_t _e = (expr);                                                               \
        if (_e != cudaSuccess) return fail(NDGSBP_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(_e)); \
    } while (0)

// ---- device copies of layouts -------------------------------------------------------------
struct BlobBuilder {
    std::vector<std::pair<const void*, size_t>> parts;
    std::vector<size_t> at;
    size_t off = 0;
    template <typename T>
    size_t add(const std::vector<T>& v) {
        at.push_back(off);
        parts.push_back({v.data(), v.size() * sizeof(T)});
        off = align256(off + v.size() * sizeof(T) + 1);
        return at.back();
    }
    ndgsbp_status upload(void** blob) {
        std::vector<unsigned char> host(off, 0);
        for (size_t i = 0; i < parts.size(); ++i)
            if (parts[i].second) std::memcpy(host.data() + at[i], parts[i].first, parts[i].second);
        CUDA_TRY(cudaMalloc(blob, off));
        cudaError_t e = cudaMemcpy(*blob, host.data(), off, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(*blob);
            *blob = nullptr;
            return fail(NDGSBP_ERR_CUDA, "descriptor upload: %s", cudaGetErrorString(e));
        }
        return NDGSBP_OK;
    }
};

static ndgsbp_status upload_layout(const Layout& L, DeviceLayout& D) {
    BlobBuilder b;
    const size_t o_deg = b.add(L.slot_deg), o_tb = b.add(L.tile_base), o_vn = b.add(L.edge_vn);
    const size_t o_csr = b.add(L.edge_csr), o_gp = b.add(L.grp_ptr), o_gs = b.add(L.ge_slot);
    const size_t o_gd = b.add(L.ge_dpos), o_cb = b.add(L.grp_colbase), o_nc = b.add(L.grp_ncol);
    const size_t o_col = b.add(L.gcol);
    void* blob = nullptr;
    ndgsbp_status st = b.upload(&blob);
    if (st) return st;
    auto* p = static_cast<unsigned char*>(blob);
    D.blob = blob;
    D.bytes = b.off;
    D.slot_deg = reinterpret_cast<const int32_t*>(p + o_deg);
    D.tile_base = reinterpret_cast<const int32_t*>(p + o_tb);
    D.edge_vn = reinterpret_cast<const int32_t*>(p + o_vn);
    D.edge_csr = reinterpret_cast<const int32_t*>(p + o_csr);
    D.grp_ptr = reinterpret_cast<const int32_t*>(p + o_gp);
    D.ge_slot = reinterpret_cast<const int32_t*>(p + o_gs);
    D.ge_dpos = reinterpret_cast<const int32_t*>(p + o_gd);
    D.grp_colbase = reinterpret_cast<const int32_t*>(p + o_cb);
    D.grp_ncol = reinterpret_cast<const int32_t*>(p + o_nc);
    D.gcol = reinterpret_cast<const uint8_t*>(p + o_col);
    return NDGSBP_OK;
}

// Tables of the stream kernel for a layered QC grouping (decode_stream.cu): which group of
// grouping 0 first uses each layer, the CSR position of each layer's first edge (negative,
// -(pos + 1), for a layer no group holds), and -- when the groups are cyclic windows advancing one
// layer per group (G = n_layers, one grouping, group g = ring positions g .. g + W - 1) -- the
// layer ring.  The message layout (stream_layer_elems) depends on the storage mode and message
// type and is set per launch (stream_bases).
struct StreamLayout {
    std::vector<int32_t> first_use, layer_csr, ring;
    bool ring_ok = false;
};

// Layer block offsets of a stream launch (elements), the per-frame total and the largest block.
static void stream_bases(const QcLayout& Q, int msz, int mode, int32_t* lbase, int* msg_elems, int* slab_elems) {
    const int zr = (Q.Z + 15) / 16 * 16;
    int off = 0, mx = 0;
    for (int l = 0; l < Q.n_layers; ++l) {
        const int e = stream_layer_elems(Q.layer_deg[l], Q.Z, zr, msz, mode);
        lbase[l] = off;
        off += e;
        mx = std::max(mx, e);
    }
    *msg_elems = off;
    *slab_elems = mx;
}

static void stream_layout(const QcLayout& Q, StreamLayout& S) {
    const int nl = Q.n_layers, Z = Q.Z, W = Q.window;
    const int G = W ? static_cast<int>(Q.group_layers.size() / (static_cast<size_t>(W) * Q.n_groupings)) : 0;
    std::vector<char> seen(nl, 0), used(nl, 0);
    S.first_use.assign(static_cast<size_t>(G) * W, 0);
    for (int g = 0; g < G; ++g)
        for (int j = 0; j < W; ++j) {
            const int l = Q.group_layers[static_cast<size_t>(g) * W + j];
            if (!seen[l]) S.first_use[static_cast<size_t>(g) * W + j] = 1;
            seen[l] = 1;
        }
    for (int l : Q.group_layers) used[l] = 1;
    S.layer_csr.assign(nl, 0);
    for (int l = 0; l < nl; ++l) {
        const int csr = Q.csr_of[Q.layer_off[l]];
        S.layer_csr[l] = used[l] ? csr : -(csr + 1);
    }
    S.ring.assign(nl, 0);
    S.ring_ok = Q.n_groupings == 1 && G == nl && W >= 1;
    for (int g = 0; S.ring_ok && g < G; ++g)
        for (int j = 0; j < W; ++j)
            if (Q.group_layers[static_cast<size_t>(g) * W + j] != Q.group_layers[static_cast<size_t>((g + j) % G) * W])
                S.ring_ok = false;
    if (S.ring_ok)
        for (int i = 0; i < nl; ++i) S.ring[i] = Q.group_layers[static_cast<size_t>(i) * W];
}

static ndgsbp_status upload_qc(const QcLayout& Q, DeviceQc& D) {
    StreamLayout SL;
    stream_layout(Q, SL);
    BlobBuilder b;
    const size_t o_tab = b.add(Q.edge_tab), o_deg = b.add(Q.layer_deg), o_off = b.add(Q.layer_off);
    const size_t o_gl = b.add(Q.group_layers), o_csr = b.add(Q.csr_of), o_str = b.add(Q.layer_stride);
    const size_t o_fu = b.add(SL.first_use), o_lc = b.add(SL.layer_csr);
    const size_t o_ring = b.add(SL.ring);
    void* blob = nullptr;
    ndgsbp_status st = b.upload(&blob);
    if (st) return st;
    auto* p = static_cast<unsigned char*>(blob);
    D.blob = blob;
    D.edge_tab = reinterpret_cast<const int32_t*>(p + o_tab);
    D.layer_deg = reinterpret_cast<const int32_t*>(p + o_deg);
    D.layer_stride = reinterpret_cast<const int32_t*>(p + o_str);
    D.layer_off = reinterpret_cast<const int32_t*>(p + o_off);
    D.group_layers = reinterpret_cast<const int32_t*>(p + o_gl);
    D.csr_of = reinterpret_cast<const int32_t*>(p + o_csr);
    D.first_use = reinterpret_cast<const int32_t*>(p + o_fu);
    D.layer_csr = reinterpret_cast<const int32_t*>(p + o_lc);
    D.ring = reinterpret_cast<const int32_t*>(p + o_ring);
    return NDGSBP_OK;
}

static ndgsbp_status device_layout(const Groups& g, bool flood, const Layout*& L, const DeviceLayout*& D,
                                   bool allow_upload = true) {
    L = flood ? &flood_layout(g) : &g.grouped;
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(g.mu);
    auto& cache = flood ? g.dev_flood : g.dev_grouped;
    auto it = cache.find(dev);
    if (it == cache.end()) {
        if (!allow_upload)
            return fail(NDGSBP_ERR_INVALID, "grouping tables are not on device %d yet: call ndgsbp_decode_plan "
                                            "with the same parameters on this device first", dev);
        DeviceLayout dl;
        ndgsbp_status st = upload_layout(*L, dl);
        if (st) return st;
        it = cache.emplace(dev, dl).first;
    }
    D = &it->second;
    return NDGSBP_OK;
}

static ndgsbp_status device_qc(const Groups& g, bool flood, const QcLayout*& Q, const DeviceQc*& D,
                               bool allow_upload = true) {
    Q = flood ? &flood_qc_layout(g) : &g.qc;
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(g.mu);
    auto& cache = flood ? g.dev_flood_qc : g.dev_qc;
    auto it = cache.find(dev);
    if (it == cache.end()) {
        if (!allow_upload)
            return fail(NDGSBP_ERR_INVALID, "grouping tables are not on device %d yet: call ndgsbp_decode_plan "
                                            "with the same parameters on this device first", dev);
        DeviceQc dq;
        ndgsbp_status st = upload_qc(*Q, dq);
        if (st) return st;
        it = cache.emplace(dev, dq).first;
    }
    D = &it->second;
    return NDGSBP_OK;
}

ndgsbp_status device_qc_tables(const Groups& g, const QcLayout*& Q, const DeviceQc*& D) {
    return device_qc(g, false, Q, D);
}

void release_device_layouts(Groups& g) {
    int cur = 0;
    if (cudaGetDevice(&cur) != cudaSuccess) return;
    for (auto* cache : {&g.dev_grouped, &g.dev_flood}) {
        for (auto& kv : *cache)
            if (cudaSetDevice(kv.first) == cudaSuccess) cudaFree(kv.second.blob);
        cache->clear();
    }
    for (auto* cache : {&g.dev_qc, &g.dev_flood_qc}) {
        for (auto& kv : *cache)
            if (cudaSetDevice(kv.first) == cudaSuccess) cudaFree(kv.second.blob);
        cache->clear();
    }
    cudaSetDevice(cur);
    cudaGetLastError();
}

Groups::~Groups() { release_device_layouts(*this); }

// ---- planning -----------------------------------------------------------------------------
struct Plan {
    ndgsbp_plan pub;
    bool qc = false;
    bool tile = false;
    KernelFn fn = nullptr;
    QcKernelFn qfn = nullptr;
    TileKernelFn tfn = nullptr;
    bool stream = false;
    StreamKernelFn sfn = nullptr;
    int stream_mode = 0, stream_tpc = 1, stream_le = 1, stream_slabs = 0, stream_ws_stride = 0;
    int stream_msg_elems = 0, stream_slab_elems = 0;
    std::vector<int32_t> stream_lbase;
    int tile_tpc = 1, tile_le = 1, tile_slots = 1, tile_slot_bytes = 0, tile_p_bytes = 0, tile_m_bytes = 0;
    int tile_delta_stride = 1, tile_frames = 1, tile_table_bytes = 0, n_tiles = 0;
    bool msg_smem = false, delta_smem = false;
    const Layout* L = nullptr;
    const DeviceLayout* D = nullptr;
    const QcLayout* Q = nullptr;
    const DeviceQc* DQ = nullptr;
};

static ndgsbp_status validate_params(const ndgsbp_params* p) {
    if (!p) return fail(NDGSBP_ERR_INVALID, "params is null");
    if (p->schedule != NDGSBP_SCHEDULE_GROUPS && p->schedule != NDGSBP_SCHEDULE_FLOOD)
        return fail(NDGSBP_ERR_INVALID, "unknown schedule %d", p->schedule);
    if (p->max_iter < 1) return fail(NDGSBP_ERR_INVALID, "max_iter must be >= 1");
    if (p->msg_dtype != NDGSBP_F32 && p->msg_dtype != NDGSBP_F16 && p->msg_dtype != NDGSBP_BF16)
        return fail(NDGSBP_ERR_INVALID, "msg_dtype must be F32, F16 or BF16");
    if (!(p->llr_max > 0.f && p->llr_max <= 30.f)) return fail(NDGSBP_ERR_INVALID, "llr_max must be in (0, 30]");
    if (p->block_threads < 0 || p->block_threads > 1024 || p->block_threads % 32)
        return fail(NDGSBP_ERR_INVALID, "block_threads must be 0 or a multiple of 32 up to 1024");
    if (p->ctas_per_sm < 0) return fail(NDGSBP_ERR_INVALID, "ctas_per_sm must be >= 0");
    if (p->frames_per_cta < 0 || p->frames_per_cta > 16)
        return fail(NDGSBP_ERR_INVALID, "frames_per_cta must be in [0, 16]");
    if (p->lanes_per_cn != 0 && p->lanes_per_cn != 1 && p->lanes_per_cn != 2 && p->lanes_per_cn != 4)
        return fail(NDGSBP_ERR_INVALID, "lanes_per_cn must be 0, 1, 2 or 4");
    if (p->variant < NDGSBP_VARIANT_AUTO || p->variant > NDGSBP_VARIANT_STREAM_BULK ||
        (p->variant > NDGSBP_VARIANT_QC_GLOBAL && p->variant < NDGSBP_VARIANT_TILE) ||
        (p->variant > NDGSBP_VARIANT_TILE && p->variant < NDGSBP_VARIANT_RAGGED_PER_CODE))
        return fail(NDGSBP_ERR_INVALID, "unknown variant %d", p->variant);
    if (p->variant == NDGSBP_VARIANT_RAGGED_PER_CODE)
        return fail(NDGSBP_ERR_INVALID, "variant RAGGED_PER_CODE applies to ragged launches only");
    return NDGSBP_OK;
}

struct DeviceInfo {
    int dev = 0, sms = 0, smem_optin = 0, smem_sm = 0, smem_reserved = 0;
};

static ndgsbp_status device_info(DeviceInfo& di) {
    CUDA_TRY(cudaGetDevice(&di.dev));
    CUDA_TRY(cudaDeviceGetAttribute(&di.sms, cudaDevAttrMultiProcessorCount, di.dev));
    CUDA_TRY(cudaDeviceGetAttribute(&di.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, di.dev));
    CUDA_TRY(cudaDeviceGetAttribute(&di.smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, di.dev));
    CUDA_TRY(cudaDeviceGetAttribute(&di.smem_reserved, cudaDevAttrReservedSharedMemoryPerBlock, di.dev));
    return NDGSBP_OK;
}

static ndgsbp_status finish_grid(const void* fn, int threads, size_t smem, const ndgsbp_params* p,
                                 int64_t n_frames, const DeviceInfo& di, int& per_sm, int64_t& grid) {
    CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
    per_sm = 0;
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem));
    if (per_sm < 1) return fail(NDGSBP_ERR_UNSUPPORTED, "kernel does not fit on an SM with %d threads", threads);
    if (p->ctas_per_sm > 0) per_sm = std::min(per_sm, p->ctas_per_sm);
    grid = static_cast<int64_t>(per_sm) * di.sms;
    grid = std::max<int64_t>(1, std::min<int64_t>(grid, std::max<int64_t>(n_frames, 1)));
    return NDGSBP_OK;
}

// Layered QC kernel plan, when the grouping is made of whole layers and a window fits a CTA
// with one thread per CN (QC, QC_GLOBAL and AUTO).
static ndgsbp_status make_qc_plan(const Groups& g, const ndgsbp_params* p, int64_t n_frames, bool flood,
                                  const DeviceInfo& di, Plan& plan, bool* ok, bool allow_upload = true) {
    *ok = false;
    const QcLayout& Q = flood ? flood_qc_layout(g) : g.qc;
    if (!Q.ok) return NDGSBP_OK;
    const int maxdc = degree_bound(Q.max_deg);
    if (!maxdc) return NDGSBP_OK;
    const bool spec = qc_degrees_specialised(Q, maxdc);
    const bool force_global = p->variant == NDGSBP_VARIANT_QC_GLOBAL;
    const int active = Q.window * Q.Z;
    const int threads = p->block_threads ? p->block_threads : (active + 31) / 32 * 32;
    if (threads < active || threads > max_threads_for(maxdc)) return NDGSBP_OK;
    const size_t budget = static_cast<size_t>(di.smem_optin) - 64;
    const size_t p_bytes = align16(static_cast<size_t>(g.code->N) * 4);
    const size_t m_bytes = align16(static_cast<size_t>(Q.msg_slots) * msg_size(p->msg_dtype));
    const size_t t_bytes = qc_table_bytes(Q);
    if (p_bytes + t_bytes > budget) return NDGSBP_OK;
    const bool msg_smem = !force_global && p_bytes + m_bytes + t_bytes <= budget;
    const size_t smem = p_bytes + t_bytes + (msg_smem ? m_bytes : 0);
    // 16-bit messages halve the shared memory of a frame: when 6 CTAs fit, use the instance
    // compiled for 6 resident CTAs (56 registers) instead of the 64-register one (5 CTAs)
    QcKernelFn fn = nullptr;
    const bool occ_ok = spec && maxdc == 8 && msg_smem && p->msg_dtype != NDGSBP_F32 &&
                        threads <= qc_occ_threads() && (p->ctas_per_sm == 0 || p->ctas_per_sm >= 6) &&
                        6 * (smem + static_cast<size_t>(di.smem_reserved) + 1024) <= static_cast<size_t>(di.smem_sm);
    if (occ_ok) fn = pick_qc_kernel(p->msg_dtype, maxdc, msg_smem, spec, true);
    if (!fn) fn = pick_qc_kernel(p->msg_dtype, maxdc, msg_smem, spec);
    if (!fn) return NDGSBP_OK;
    int per_sm = 0;
    int64_t grid = 0;
    ndgsbp_status st = finish_grid(reinterpret_cast<const void*>(fn), threads, smem, p, n_frames, di, per_sm, grid);
    if (st) return st;
    st = device_qc(g, flood, plan.Q, plan.DQ, allow_upload);
    if (st) return st;
    plan.qc = true;
    plan.qfn = fn;
    plan.msg_smem = msg_smem;
    ndgsbp_plan& o = plan.pub;
    o.variant = msg_smem ? NDGSBP_VARIANT_QC : NDGSBP_VARIANT_QC_GLOBAL;
    o.block_threads = threads;
    o.grid = static_cast<int32_t>(grid);
    o.ctas_per_sm = per_sm;
    o.max_row_degree = maxdc;
    o.delta_in_smem = 0;
    o.smem_bytes = static_cast<int64_t>(smem);
    o.workspace_bytes = static_cast<int64_t>(
        kHeaderBytes + (msg_smem ? 0 : align256(static_cast<size_t>(grid) * Q.msg_slots * msg_size(p->msg_dtype))));
    o.stored_edges = Q.msg_slots;
    o.edge_updates_per_iter = flood ? g.code->E : g.edge_updates;
    *ok = true;
    return NDGSBP_OK;
}

// Stream kernel plan: a QC grouping in whole layers whose window does not fit one CTA with one
// thread per CN, CN degree <= 22 (one or two lanes per CN).  The message storage mode is the
// variant's (STREAM_SMEM / _GLOBAL / _BULK) or, for AUTO and STREAM, the one that keeps the most
// CTAs resident per SM (ties: shared memory, then global, then bulk-staged slabs -- the order
// measured on GB300 for n=16200 and n=8192).
static ndgsbp_status make_stream_plan(const Groups& g, const ndgsbp_params* p, int64_t n_frames, bool flood,
                                      const DeviceInfo& di, Plan& plan, bool* ok, bool allow_upload = true) {
    *ok = false;
    const QcLayout& Q = flood ? flood_qc_layout(g) : g.qc;
    if (!Q.ok) return NDGSBP_OK;
    const int tpc = p->lanes_per_cn ? p->lanes_per_cn : (Q.max_deg <= 11 ? 1 : 2);
    if (tpc != 1 && tpc != 2) return NDGSBP_OK;
    const int LE = stream_lane_width((Q.max_deg + tpc - 1) / tpc, tpc);
    if (!LE || LE * tpc < Q.max_deg) return NDGSBP_OK;
    const int active = Q.Z * tpc;
    const int threads = p->block_threads ? p->block_threads : (active + 31) / 32 * 32;
    if (threads < active || threads > stream_max_threads(tpc)) return NDGSBP_OK;
    // two lanes per CN: each lane in its own warps (Z a multiple of 32, a block of exactly 2 Z)
    if (tpc == 2 && (Q.Z % 32 != 0 || threads != active)) return NDGSBP_OK;
    if (Q.n_layers > kStreamMaxLayers) return NDGSBP_OK;
    StreamLayout SL;
    stream_layout(Q, SL);
    const int msz = msg_size(p->msg_dtype);
    StreamArgs a;
    std::memset(&a, 0, sizeof(a));
    a.r.N = g.code->N;
    a.Z = Q.Z;
    a.nl = Q.n_layers;
    a.window = Q.window;
    a.n_groupings = Q.n_groupings;
    a.G = static_cast<int>(Q.group_layers.size() / (static_cast<size_t>(Q.window) * Q.n_groupings));
    a.maxdeg = Q.max_deg;
    a.tpc = tpc;
    a.le = (Q.max_deg + tpc - 1) / tpc;
    a.zr = (Q.Z + 15) / 16 * 16;
    a.n_slabs = Q.window + 2;
    const bool bulk_ok = SL.ring_ok && Q.n_layers >= Q.window + 2 && a.n_slabs <= kStreamMaxSlabs;
    int want = -1;
    if (p->variant == NDGSBP_VARIANT_STREAM_SMEM) want = kStreamSmem;
    if (p->variant == NDGSBP_VARIANT_STREAM_GLOBAL) want = kStreamGlobal;
    if (p->variant == NDGSBP_VARIANT_STREAM_BULK) want = kStreamBulk;
    if (want == kStreamBulk && !bulk_ok) return NDGSBP_OK;
    const size_t budget = static_cast<size_t>(di.smem_optin) - 64;
    int best_mode = -1, best_per_sm = 0;
    size_t best_smem = 0;
    for (int mode : {kStreamSmem, kStreamGlobal, kStreamBulk}) {
        if (want >= 0 && mode != want) continue;
        if (mode == kStreamBulk && !bulk_ok) continue;
        stream_bases(Q, msz, mode, a.lbase, &a.msg_elems, &a.slab_elems);
        const size_t smem = stream_smem_bytes(a, msz, mode);
        if (smem > budget) continue;
        StreamKernelFn fn = pick_stream_kernel(p->msg_dtype, LE, tpc, mode);
        if (!fn) continue;
        CUDA_TRY(cudaFuncSetAttribute(reinterpret_cast<const void*>(fn), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      static_cast<int>(smem)));
        int per_sm = 0;
        CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, reinterpret_cast<const void*>(fn), threads, smem));
        if (p->ctas_per_sm > 0) per_sm = std::min(per_sm, p->ctas_per_sm);
        if (per_sm > best_per_sm) {
            best_per_sm = per_sm;
            best_mode = mode;
            best_smem = smem;
        }
    }
    if (best_mode < 0) return NDGSBP_OK;
    StreamKernelFn fn = pick_stream_kernel(p->msg_dtype, LE, tpc, best_mode);
    int per_sm = 0;
    int64_t grid = 0;
    ndgsbp_status st = finish_grid(reinterpret_cast<const void*>(fn), threads, best_smem, p, n_frames, di, per_sm, grid);
    if (st) return st;
    st = device_qc(g, flood, plan.Q, plan.DQ, allow_upload);
    if (st) return st;
    stream_bases(Q, msz, best_mode, a.lbase, &a.msg_elems, &a.slab_elems);
    const int ws_stride = static_cast<int>(align256(static_cast<size_t>(a.msg_elems) * msz) / msz);
    plan.stream_lbase.assign(a.lbase, a.lbase + Q.n_layers);
    plan.stream_msg_elems = a.msg_elems;
    plan.stream_slab_elems = a.slab_elems;
    plan.stream = true;
    plan.sfn = fn;
    plan.stream_mode = best_mode;
    plan.stream_tpc = tpc;
    plan.stream_le = LE;
    plan.stream_slabs = a.n_slabs;
    plan.stream_ws_stride = ws_stride;
    plan.msg_smem = best_mode == kStreamSmem;
    ndgsbp_plan& o = plan.pub;
    o.variant = best_mode == kStreamSmem ? NDGSBP_VARIANT_STREAM_SMEM
                                         : (best_mode == kStreamBulk ? NDGSBP_VARIANT_STREAM_BULK : NDGSBP_VARIANT_STREAM_GLOBAL);
    o.block_threads = threads;
    o.grid = static_cast<int32_t>(grid);
    o.ctas_per_sm = per_sm;
    o.max_row_degree = Q.max_deg;
    o.delta_in_smem = 1;
    o.smem_bytes = static_cast<int64_t>(best_smem);
    o.workspace_bytes = static_cast<int64_t>(
        kHeaderBytes + (best_mode == kStreamSmem ? 0 : align256(static_cast<size_t>(grid) * ws_stride * msz)));
    o.stored_edges = a.msg_elems;
    o.edge_updates_per_iter = flood ? g.code->E : g.edge_updates;
    *ok = true;
    return NDGSBP_OK;
}

// Tile kernel plan: any QC grouping in whole layers, row degree <= 32.
static ndgsbp_status make_tile_plan(const Groups& g, const ndgsbp_params* p, int64_t n_frames, bool flood,
                                    const DeviceInfo& di, Plan& plan, bool* ok, bool allow_upload = true) {
    *ok = false;
    const QcLayout& Q = flood ? flood_qc_layout(g) : g.qc;
    if (!Q.ok) return NDGSBP_OK;
    const int tpc = p->lanes_per_cn ? p->lanes_per_cn : tile_lanes_per_cn(Q.max_deg);
    if (!tpc) return NDGSBP_OK;
    const int le = (Q.max_deg + tpc - 1) / tpc;
    if (le > 8) return fail(NDGSBP_ERR_UNSUPPORTED, "lanes_per_cn %d leaves %d edges per lane (at most 8)", tpc, le);
    const TileShape shp = tile_shape(Q, tpc, p->msg_dtype);
    const int ds = shp.delta_stride;
    const int per_slot = Q.window * Q.Z * tpc;
    int threads = p->block_threads ? p->block_threads : std::min(512, std::max(128, (per_slot + 31) / 32 * 32));
    const size_t table = tile_table_bytes(Q);
    const size_t p_bytes = align16(static_cast<size_t>(g.code->N) * 4);
    const size_t m_bytes = align16(static_cast<size_t>(shp.msg_slots) * msg_size(p->msg_dtype));
    const size_t d_bytes = align16(static_cast<size_t>(shp.delta_floats) * 4);
    // Shared memory per CTA under a residency target of k CTAs per SM: ctas_per_sm when set,
    // else 2 when a frame's posterior and deltas fit under half an SM, else 1.  Messages that
    // do not fit under the cap live in workspace slots (a code whose messages would fill a whole
    // SM runs two CTAs with global messages rather than one with shared ones).
    auto cap_for = [&](int k) {
        const size_t per = static_cast<size_t>(di.smem_sm) / k - static_cast<size_t>(di.smem_reserved) - 1024;
        return std::min(static_cast<size_t>(di.smem_optin) - 256, per) & ~static_cast<size_t>(15);
    };
    const int target = p->ctas_per_sm > 0 ? p->ctas_per_sm : (table + p_bytes + d_bytes <= cap_for(2) ? 2 : 1);
    const size_t budget = cap_for(target);
    const bool msg_smem = p->variant != NDGSBP_VARIANT_GLOBAL && table + p_bytes + m_bytes + d_bytes <= budget;
    const size_t slot_bytes = p_bytes + (msg_smem ? m_bytes : 0) + d_bytes;
    if (table + slot_bytes > budget) return NDGSBP_OK;
    const int max_slots = static_cast<int>(std::min<size_t>(16, (budget - table) / slot_bytes));
    int slots = p->frames_per_cta ? p->frames_per_cta : std::max(1, std::min(16, threads / per_slot));
    slots = std::min(slots, max_slots);
    const size_t smem = table + static_cast<size_t>(slots) * slot_bytes;
    TileKernelFn fn = pick_tile_kernel(p->msg_dtype, false, tile_lane_width(le), slots * per_slot <= threads, true);
    if (!fn) return NDGSBP_OK;
    int per_sm = 0;
    int64_t grid = 0;
    ndgsbp_status st = finish_grid(reinterpret_cast<const void*>(fn), threads, smem, p, n_frames, di, per_sm, grid);
    if (st) return st;
    const int tile_frames = slots * 4;
    const int64_t n_tiles = std::max<int64_t>(1, (n_frames + tile_frames - 1) / tile_frames);
    grid = std::min<int64_t>(grid, n_tiles);
    st = device_qc(g, flood, plan.Q, plan.DQ, allow_upload);
    if (st) return st;
    plan.tile = true;
    plan.tfn = fn;
    plan.msg_smem = msg_smem;
    plan.tile_tpc = tpc;
    plan.tile_le = le;
    plan.tile_slots = slots;
    plan.tile_slot_bytes = static_cast<int>(slot_bytes);
    plan.tile_p_bytes = static_cast<int>(p_bytes);
    plan.tile_m_bytes = msg_smem ? static_cast<int>(m_bytes) : 0;
    plan.tile_delta_stride = ds;
    plan.tile_frames = tile_frames;
    plan.tile_table_bytes = static_cast<int>(table);
    plan.n_tiles = static_cast<int>(n_tiles);
    ndgsbp_plan& o = plan.pub;
    o.variant = NDGSBP_VARIANT_TILE;
    o.block_threads = threads;
    o.grid = static_cast<int32_t>(grid);
    o.ctas_per_sm = per_sm;
    o.max_row_degree = Q.max_deg;
    o.delta_in_smem = 1;
    o.smem_bytes = static_cast<int64_t>(smem);
    o.workspace_bytes = static_cast<int64_t>(
        kHeaderBytes +
        (msg_smem ? 0 : align256(static_cast<size_t>(grid) * slots * shp.msg_slots * msg_size(p->msg_dtype))));
    o.stored_edges = shp.msg_slots;
    o.edge_updates_per_iter = flood ? g.code->E : g.edge_updates;
    *ok = true;
    return NDGSBP_OK;
}

static ndgsbp_status make_plan(const Groups& g, const ndgsbp_params* p, int64_t n_frames, Plan& plan,
                               bool allow_upload = true) {
    ndgsbp_status st = validate_params(p);
    if (st) return st;
    const bool flood = p->schedule == NDGSBP_SCHEDULE_FLOOD;
    DeviceInfo di;
    st = device_info(di);
    if (st) return st;
    if (p->variant == NDGSBP_VARIANT_TILE) {
        bool ok = false;
        st = make_tile_plan(g, p, n_frames, flood, di, plan, &ok, allow_upload);
        if (st) return st;
        if (ok) return NDGSBP_OK;
        return fail(NDGSBP_ERR_UNSUPPORTED, "TILE variant needs a QC code grouped in whole layers, row degree <= 32");
    }
    if (p->variant >= NDGSBP_VARIANT_STREAM && p->variant <= NDGSBP_VARIANT_STREAM_BULK) {
        bool ok = false;
        st = make_stream_plan(g, p, n_frames, flood, di, plan, &ok, allow_upload);
        if (st) return st;
        if (ok) return NDGSBP_OK;
        return fail(NDGSBP_ERR_UNSUPPORTED, "STREAM variant needs a QC code grouped in whole layers, row degree "
                                            "<= 22 (bulk staging: cyclic windows advancing one layer per group)");
    }
    const bool want_qc = p->variant == NDGSBP_VARIANT_QC || p->variant == NDGSBP_VARIANT_QC_GLOBAL;
    if (p->variant == NDGSBP_VARIANT_AUTO || want_qc) {
        bool ok = false;
        st = make_qc_plan(g, p, n_frames, flood, di, plan, &ok, allow_upload);
        if (st) return st;
        if (ok) return NDGSBP_OK;
        if (want_qc)
            return fail(NDGSBP_ERR_UNSUPPORTED, "QC variant needs a QC code grouped in whole layers with a window "
                                                "that fits one CTA");
        // QC code whose window does not fit one CTA with one CN per thread: stream kernel, else
        // tile kernel
        st = make_stream_plan(g, p, n_frames, flood, di, plan, &ok, allow_upload);
        if (st) return st;
        if (ok) return NDGSBP_OK;
        st = make_tile_plan(g, p, n_frames, flood, di, plan, &ok, allow_upload);
        if (st) return st;
        if (ok) return NDGSBP_OK;
    }
    if (g.n_groupings > 1 && !flood)
        return fail(NDGSBP_ERR_UNSUPPORTED, "groupings cycled by iteration need a QC kernel (groups of whole layers)");
    st = device_layout(g, flood, plan.L, plan.D, allow_upload);
    if (st) return st;
    const Layout& L = *plan.L;
    const int maxdc = degree_bound(L.max_deg);
    if (!maxdc) return fail(NDGSBP_ERR_UNSUPPORTED, "CN degree %d above 32", L.max_deg);
    const size_t budget = static_cast<size_t>(di.smem_optin) - 64;
    const size_t p_bytes = align16(static_cast<size_t>(L.N) * 4);
    const size_t m_bytes = align16(static_cast<size_t>(L.Epad) * msg_size(p->msg_dtype));
    const size_t d_bytes = align16(static_cast<size_t>(L.max_gd) * 4);
    if (p_bytes > budget) return fail(NDGSBP_ERR_UNSUPPORTED, "posterior of %d VNs does not fit in shared memory", L.N);
    bool msg_smem, delta_smem;
    if (p->variant == NDGSBP_VARIANT_SMEM) {
        if (p_bytes + m_bytes + d_bytes > budget)
            return fail(NDGSBP_ERR_UNSUPPORTED, "SMEM variant needs %zu bytes of shared memory, device has %zu",
                        p_bytes + m_bytes + d_bytes, budget);
        msg_smem = delta_smem = true;
    } else if (p->variant == NDGSBP_VARIANT_GLOBAL) {
        msg_smem = false;
        delta_smem = p_bytes + d_bytes <= budget;
    } else {
        msg_smem = p_bytes + m_bytes + d_bytes <= budget;
        delta_smem = msg_smem || p_bytes + d_bytes <= budget;
    }
    const size_t smem = p_bytes + (msg_smem ? m_bytes : 0) + (delta_smem ? d_bytes : 0);
    const int tmax = max_threads_for(maxdc);
    int threads = p->block_threads;
    if (!threads) threads = std::min(tmax, std::max(64, (L.max_group_entries + 31) / 32 * 32));
    if (threads > tmax)
        return fail(NDGSBP_ERR_UNSUPPORTED, "block_threads %d above %d for CN degree %d", threads, tmax, L.max_deg);
    KernelFn fn = pick_kernel(p->msg_dtype, maxdc, msg_smem, delta_smem);
    if (!fn) return fail(NDGSBP_ERR_UNSUPPORTED, "no kernel instance for this configuration");
    int per_sm = 0;
    int64_t grid = 0;
    st = finish_grid(reinterpret_cast<const void*>(fn), threads, smem, p, n_frames, di, per_sm, grid);
    if (st) return st;
    size_t ws = kHeaderBytes;
    if (!msg_smem) ws += align256(static_cast<size_t>(grid) * L.Epad * msg_size(p->msg_dtype));
    if (!delta_smem) ws += align256(static_cast<size_t>(grid) * L.max_gd * 4);
    plan.fn = fn;
    plan.msg_smem = msg_smem;
    plan.delta_smem = delta_smem;
    ndgsbp_plan& o = plan.pub;
    o.variant = msg_smem ? NDGSBP_VARIANT_SMEM : NDGSBP_VARIANT_GLOBAL;
    o.block_threads = threads;
    o.grid = static_cast<int32_t>(grid);
    o.ctas_per_sm = per_sm;
    o.max_row_degree = maxdc;
    o.delta_in_smem = delta_smem ? 1 : 0;
    o.smem_bytes = static_cast<int64_t>(smem);
    o.workspace_bytes = static_cast<int64_t>(ws);
    o.stored_edges = L.Epad;
    o.edge_updates_per_iter = L.edge_updates;
    return NDGSBP_OK;
}

static void fill_run(RunArgs& r, const Groups& g, const ndgsbp_params* params, const void* d_llr, int32_t llr_dtype,
                     int64_t n_frames, void* ws, uint32_t* d_hard_bits, int32_t* d_iters, uint8_t* d_syndrome_ok,
                     float* d_posterior, const ndgsbp_extras* extras) {
    std::memset(&r, 0, sizeof(r));
    r.N = g.code->N;
    r.E = static_cast<int>(g.code->E);
    r.W = (r.N + 31) / 32;
    r.llr = d_llr;
    r.llr_dtype = llr_dtype;
    r.n_frames = n_frames;
    r.max_iter = params->max_iter;
    r.llr_max = kernel_llr_limit(params->llr_max);
    r.early_stop = params->early_stop ? 1 : 0;
    r.counter = static_cast<unsigned long long*>(ws);
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
}


// ---- decoding with the library's own scratch --------------------------------------------
// Scratch of ndgsbp_decode_static: one array per device, held by every GPU that loads the
// library until the process exits.  Host code may not use its name as a device address (it is
// only a host-side stand-in); static_scratch_address() asks the runtime for the real one.
static __device__ __align__(256) unsigned char g_static_scratch[NDGSBP_STATIC_SCRATCH_BYTES];

static std::mutex g_static_mu;
static std::map<int, void*> g_static_addr;   // device -> device address of g_static_scratch

// Set-up, once per device, with that device current.
static ndgsbp_status static_scratch_address(void** out) {
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(g_static_mu);
    auto it = g_static_addr.find(dev);
    if (it == g_static_addr.end()) {
        void* p = nullptr;
        CUDA_TRY(cudaGetSymbolAddress(&p, g_static_scratch));
        it = g_static_addr.emplace(dev, p).first;
    }
    *out = it->second;
    return NDGSBP_OK;
}

// Launch a plan with `ws` as its scratch (its counter already cleared on the stream).
// Test hooks of the bulk-staged stream kernel (ndgsbp_test_hooks): leave the first bulk load of
// each CTA unissued, and the polls a bounded wait makes before it gives up (0 = the default).
static std::atomic<int> g_hook_skip_load{0};
static std::atomic<unsigned> g_hook_wait_polls{0};
constexpr unsigned kDefaultWaitPolls = 1u << 22;   // about 0.3 s of polling

// The table and shape arguments of a stream-kernel launch (everything but the run arguments,
// the message slots and the status word).
static void fill_stream_args(StreamArgs& a, const Plan& plan) {
    const QcLayout& Q = *plan.Q;
    const DeviceQc& D = *plan.DQ;
    a.Z = Q.Z;
    a.nl = Q.n_layers;
    a.window = Q.window;
    a.n_groupings = Q.n_groupings;
    a.G = static_cast<int>(Q.group_layers.size() / (static_cast<size_t>(Q.window) * Q.n_groupings));
    a.maxdeg = Q.max_deg;
    a.tpc = plan.stream_tpc;
    a.le = (Q.max_deg + plan.stream_tpc - 1) / plan.stream_tpc;
    a.zr = (Q.Z + 15) / 16 * 16;
    a.msg_elems = plan.stream_msg_elems;
    a.slab_elems = plan.stream_slab_elems;
    for (size_t l = 0; l < plan.stream_lbase.size(); ++l) a.lbase[l] = plan.stream_lbase[l];
    a.edge_tab = reinterpret_cast<const int2*>(D.edge_tab);
    a.layer_deg = D.layer_deg;
    a.group_layers = D.group_layers;
    a.first_use = D.first_use;
    a.layer_csr = D.layer_csr;
    a.ring = D.ring;
    a.n_slabs = plan.stream_slabs;
    a.ws_stride = plan.stream_ws_stride;
    const unsigned polls = g_hook_wait_polls.load();
    a.wait_limit = polls ? polls : kDefaultWaitPolls;
    a.test_skip_load = g_hook_skip_load.load();
}

static ndgsbp_status launch_plan(const Groups& g, const Plan& plan, const ndgsbp_params* params, const void* d_llr,
                                 int32_t llr_dtype, int64_t n_frames, unsigned char* ws, uint32_t* d_hard_bits,
                                 int32_t* d_iters, uint8_t* d_syndrome_ok, float* d_posterior,
                                 const ndgsbp_extras* extras, cudaStream_t s) {
    if (plan.stream) {
        StreamArgs a;
        std::memset(&a, 0, sizeof(a));
        fill_run(a.r, g, params, d_llr, llr_dtype, n_frames, ws, d_hard_bits, d_iters, d_syndrome_ok, d_posterior,
                 extras);
        fill_stream_args(a, plan);
        // per-CTA message slots are ws_stride elements apart (256-byte multiples)
        a.ws_msgs = plan.stream_mode == kStreamSmem ? nullptr : ws + kHeaderBytes;
        a.status = reinterpret_cast<unsigned*>(ws + 8);
        plan.sfn<<<plan.pub.grid, plan.pub.block_threads, plan.pub.smem_bytes, s>>>(a);
    } else if (plan.tile) {
        TileArgs a;
        std::memset(&a, 0, sizeof(a));
        TileCode& C = a.codes[0];
        fill_run(C.r, g, params, d_llr, llr_dtype, n_frames, ws, d_hard_bits, d_iters, d_syndrome_ok, d_posterior,
                 extras);
        const QcLayout& Q = *plan.Q;
        const DeviceQc& D = *plan.DQ;
        C.N = g.code->N;
        C.E = static_cast<int>(g.code->E);
        C.Z = Q.Z;
        C.nl = Q.n_layers;
        C.n_groupings = Q.n_groupings;
        C.G = static_cast<int>(Q.group_layers.size() / (static_cast<size_t>(Q.window) * Q.n_groupings));
        C.window = Q.window;
        C.maxdeg = Q.max_deg;
        const TileShape shp = tile_shape(Q, plan.tile_tpc, params->msg_dtype);
        C.msg_slots = shp.msg_slots;
        C.msg_stride = shp.msg_stride;
        C.tpc = plan.tile_tpc;
        C.le = plan.tile_le;
        C.slots = plan.tile_slots;
        C.slot_bytes = plan.tile_slot_bytes;
        C.p_bytes = plan.tile_p_bytes;
        C.m_bytes = plan.tile_m_bytes;
        C.delta_stride = plan.tile_delta_stride;
        C.edge_tab = reinterpret_cast<const int2*>(D.edge_tab);
        C.layer_deg = D.layer_deg;
        C.group_layers = D.group_layers;
        C.csr_of = D.csr_of;
        tile_code_finish(C);
        C.ws_msgs = plan.msg_smem ? nullptr : ws + kHeaderBytes;
        a.n_codes = 1;
        a.tiles = nullptr;
        a.n_tiles = plan.n_tiles;
        a.tile_frames = plan.tile_frames;
        a.tile_counter = reinterpret_cast<unsigned long long*>(ws);
        a.table_bytes = plan.tile_table_bytes;
        plan.tfn<<<plan.pub.grid, plan.pub.block_threads, plan.pub.smem_bytes, s>>>(a);
    } else if (plan.qc) {
        QcArgs a;
        std::memset(&a, 0, sizeof(a));
        fill_run(a.r, g, params, d_llr, llr_dtype, n_frames, ws, d_hard_bits, d_iters, d_syndrome_ok, d_posterior,
                 extras);
        fill_qc_args(a, *plan.Q, *plan.DQ, plan.msg_smem ? nullptr : ws + kHeaderBytes);
        plan.qfn<<<plan.pub.grid, plan.pub.block_threads, plan.pub.smem_bytes, s>>>(a);
    } else {
        const Layout& L = *plan.L;
        const DeviceLayout& D = *plan.D;
        DecodeArgs a;
        std::memset(&a, 0, sizeof(a));
        fill_run(a.r, g, params, d_llr, llr_dtype, n_frames, ws, d_hard_bits, d_iters, d_syndrome_ok, d_posterior,
                 extras);
        a.M = L.M;
        a.Epad = L.Epad;
        a.G = L.G;
        a.max_gd = L.max_gd;
        a.slot_deg = D.slot_deg;
        a.tile_base = D.tile_base;
        a.edge_vn = D.edge_vn;
        a.edge_csr = D.edge_csr;
        a.grp_ptr = D.grp_ptr;
        a.ge_slot = D.ge_slot;
        a.ge_dpos = D.ge_dpos;
        a.grp_colbase = D.grp_colbase;
        a.grp_ncol = D.grp_ncol;
        a.gcol = D.gcol;
        size_t off = kHeaderBytes;
        if (!plan.msg_smem) {
            a.ws_msgs = ws + off;
            off += align256(static_cast<size_t>(plan.pub.grid) * L.Epad * msg_size(params->msg_dtype));
        }
        if (!plan.delta_smem) a.ws_delta = reinterpret_cast<float*>(ws + off);
        plan.fn<<<plan.pub.grid, plan.pub.block_threads, plan.pub.smem_bytes, s>>>(a);
    }
    CUDA_TRY(cudaGetLastError());
    return NDGSBP_OK;
}

ndgsbp_status qc_serve_plan(const Groups& g, const ndgsbp_params* p, QcServePlan* out, bool* ok) {
    *ok = false;
    ndgsbp_status st = validate_params(p);
    if (st) return st;
    ndgsbp_params q = *p;
    q.variant = NDGSBP_VARIANT_QC;
    q.block_threads = 0;
    q.ctas_per_sm = 0;
    q.frames_per_cta = 0;
    q.lanes_per_cn = 0;
    DeviceInfo di;
    st = device_info(di);
    if (st) return st;
    Plan plan;
    bool qok = false;
    st = make_qc_plan(g, &q, int64_t{1} << 30, /*flood=*/false, di, plan, &qok);
    if (st || !qok) return st;
    const int maxdc = plan.pub.max_row_degree;
    if (!qc_degrees_specialised(*plan.Q, maxdc)) return NDGSBP_OK;
    QcKernelFn fn = pick_qc_serve_kernel(q.msg_dtype, maxdc, plan.msg_smem);
    if (!fn) return NDGSBP_OK;
    out->fn = fn;
    out->threads = plan.pub.block_threads;
    out->smem = static_cast<size_t>(plan.pub.smem_bytes);
    out->msg_smem = plan.msg_smem;
    out->msg_slots = plan.Q->msg_slots;
    std::memset(&out->args, 0, sizeof(out->args));
    fill_qc_args(out->args, *plan.Q, *plan.DQ, nullptr);
    *ok = true;
    return NDGSBP_OK;
}

ndgsbp_status stream_serve_plan(const Groups& g, const ndgsbp_params* p, StreamServePlan* out, bool* ok) {
    *ok = false;
    ndgsbp_status st = validate_params(p);
    if (st) return st;
    ndgsbp_params q = *p;
    q.variant = NDGSBP_VARIANT_AUTO;
    q.block_threads = 0;
    q.ctas_per_sm = 0;
    q.frames_per_cta = 0;
    q.lanes_per_cn = 0;
    DeviceInfo di;
    st = device_info(di);
    if (st) return st;
    // the plain decode's choice: the QC kernel first (then the pool is a QC pool), else the stream kernel
    {
        Plan qp;
        bool qok = false;
        st = make_qc_plan(g, &q, int64_t{1} << 30, /*flood=*/false, di, qp, &qok);
        if (st || qok) return st;
    }
    Plan plan;
    bool sok = false;
    st = make_stream_plan(g, &q, int64_t{1} << 30, /*flood=*/false, di, plan, &sok);
    if (st || !sok) return st;
    if (plan.stream_mode == kStreamBulk) {   // served in global mode: the same arithmetic
        q.variant = NDGSBP_VARIANT_STREAM_GLOBAL;
        plan = Plan();
        st = make_stream_plan(g, &q, int64_t{1} << 30, /*flood=*/false, di, plan, &sok);
        if (st || !sok) return st;
    }
    StreamKernelFn fn = pick_stream_serve_kernel(q.msg_dtype, plan.stream_le, plan.stream_tpc, plan.stream_mode);
    if (!fn) return NDGSBP_OK;
    out->fn = fn;
    out->threads = plan.pub.block_threads;
    out->per_sm = plan.pub.ctas_per_sm;
    out->mode = plan.stream_mode;
    out->smem = static_cast<size_t>(plan.pub.smem_bytes);
    out->msg_elems_per_slot = plan.stream_ws_stride;
    std::memset(&out->args, 0, sizeof(out->args));
    fill_stream_args(out->args, plan);
    *ok = true;
    return NDGSBP_OK;
}

Plan* plan_create(const Groups& g, const ndgsbp_params* p, int64_t n_frames, ndgsbp_status* st) {
    Plan* plan = new (std::nothrow) Plan;
    if (!plan) {
        *st = fail(NDGSBP_ERR_NOMEM, "out of host memory");
        return nullptr;
    }
    *st = make_plan(g, p, n_frames, *plan);
    if (*st) {
        delete plan;
        return nullptr;
    }
    return plan;
}

void plan_destroy(Plan* plan) { delete plan; }

const ndgsbp_plan& plan_info(const Plan& plan) { return plan.pub; }

ndgsbp_status plan_enqueue(const Groups& g, const Plan& plan, const ndgsbp_params* p, const void* d_llr,
                           int32_t llr_dtype, int64_t n_frames, void* ws, uint32_t* d_hard_bits, int32_t* d_iters,
                           uint8_t* d_syndrome_ok, float* d_posterior, const ndgsbp_extras* extras, cudaStream_t s) {
    if (n_frames == 0) return NDGSBP_OK;
    CUDA_TRY(cudaMemsetAsync(ws, 0, kStatusEnd, s));   // frame counter and status word
    return launch_plan(g, plan, p, d_llr, llr_dtype, n_frames, static_cast<unsigned char*>(ws), d_hard_bits, d_iters,
                       d_syndrome_ok, d_posterior, extras, s);
}

}  // namespace ndgsbp

using namespace ndgsbp;

// Element alignment of the caller's buffers (the kernels read and write them element by element).
static ndgsbp_status check_alignment(const char* who, const void* d_llr, int32_t llr_dtype, const uint32_t* d_hard_bits,
                                     const int32_t* d_iters, const float* d_posterior) {
    const size_t le = llr_dtype == NDGSBP_F64 ? 8 : llr_dtype == NDGSBP_F32 ? 4 : 2;
    if (reinterpret_cast<uintptr_t>(d_llr) % le) return fail(NDGSBP_ERR_INVALID, "%s: d_llr not aligned to its element", who);
    if (reinterpret_cast<uintptr_t>(d_hard_bits) % 4 || reinterpret_cast<uintptr_t>(d_iters) % 4 ||
        reinterpret_cast<uintptr_t>(d_posterior) % 4)
        return fail(NDGSBP_ERR_INVALID, "%s: output buffers must be 4-byte aligned", who);
    return NDGSBP_OK;
}

extern "C" {

ndgsbp_status ndgsbp_decode_plan(const ndgsbp_groups* groups, const ndgsbp_params* params,
                                 int64_t n_frames, ndgsbp_plan* plan) {
    clear_error();
    if (!groups || !plan) return fail(NDGSBP_ERR_INVALID, "decode_plan: null pointer");
    Plan p;
    ndgsbp_status st = make_plan(groups->g, params, n_frames, p);
    if (st) return st;
    *plan = p.pub;
    return NDGSBP_OK;
}

ndgsbp_status ndgsbp_workspace_size(const ndgsbp_groups* groups, const ndgsbp_params* params,
                                    int64_t n_frames, size_t* bytes) {
    clear_error();
    if (!groups || !bytes) return fail(NDGSBP_ERR_INVALID, "workspace_size: null pointer");
    Plan p;
    ndgsbp_status st = make_plan(groups->g, params, n_frames, p);
    if (st) return st;
    *bytes = static_cast<size_t>(p.pub.workspace_bytes);
    return NDGSBP_OK;
}

ndgsbp_status ndgsbp_decode_ex(const ndgsbp_groups* groups, const ndgsbp_params* params,
                               const void* d_llr, int32_t llr_dtype, int64_t n_frames,
                               void* d_workspace, size_t workspace_bytes, uint32_t* d_hard_bits,
                               int32_t* d_iters, uint8_t* d_syndrome_ok, float* d_posterior,
                               const ndgsbp_extras* extras, void* stream) {
    clear_error();
    if (!groups) return fail(NDGSBP_ERR_INVALID, "decode: null groups handle");
    if (n_frames < 0) return fail(NDGSBP_ERR_INVALID, "decode: n_frames < 0");
    if (llr_dtype != NDGSBP_F32 && llr_dtype != NDGSBP_F64 && llr_dtype != NDGSBP_F16 && llr_dtype != NDGSBP_BF16)
        return fail(NDGSBP_ERR_INVALID, "decode: unknown llr_dtype %d", llr_dtype);
    if (n_frames > 0 && (!d_llr || !d_hard_bits)) return fail(NDGSBP_ERR_INVALID, "decode: d_llr and d_hard_bits are required");
    ndgsbp_status sa = check_alignment("decode", d_llr, llr_dtype, d_hard_bits, d_iters, d_posterior);
    if (sa) return sa;
    const Groups& g = groups->g;
    Plan plan;
    ndgsbp_status st = make_plan(g, params, n_frames, plan);
    if (st) return st;
    if (n_frames == 0) return NDGSBP_OK;
    if (!d_workspace || workspace_bytes < static_cast<size_t>(plan.pub.workspace_bytes))
        return fail(NDGSBP_ERR_WORKSPACE, "decode: workspace of %zu bytes, need %lld", workspace_bytes,
                    static_cast<long long>(plan.pub.workspace_bytes));
    if (reinterpret_cast<uintptr_t>(d_workspace) % 256)
        return fail(NDGSBP_ERR_WORKSPACE, "decode: workspace must be 256-byte aligned");
    auto* ws = static_cast<unsigned char*>(d_workspace);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CUDA_TRY(cudaMemsetAsync(ws, 0, kStatusEnd, s));   // frame counter and status word
    return launch_plan(g, plan, params, d_llr, llr_dtype, n_frames, ws, d_hard_bits, d_iters, d_syndrome_ok,
                       d_posterior, extras, s);
}

ndgsbp_status ndgsbp_decode(const ndgsbp_groups* groups, const ndgsbp_params* params,
                            const void* d_llr, int32_t llr_dtype, int64_t n_frames,
                            void* d_workspace, size_t workspace_bytes, uint32_t* d_hard_bits,
                            int32_t* d_iters, uint8_t* d_syndrome_ok, float* d_posterior,
                            void* stream) {
    return ndgsbp_decode_ex(groups, params, d_llr, llr_dtype, n_frames, d_workspace, workspace_bytes,
                            d_hard_bits, d_iters, d_syndrome_ok, d_posterior, nullptr, stream);
}

ndgsbp_status ndgsbp_test_hooks(int32_t skip_first_bulk_load, uint32_t wait_polls) {
    clear_error();
    if (skip_first_bulk_load != 0 && skip_first_bulk_load != 1)
        return fail(NDGSBP_ERR_INVALID, "test_hooks: skip_first_bulk_load must be 0 or 1");
    g_hook_skip_load.store(skip_first_bulk_load);
    g_hook_wait_polls.store(wait_polls);
    return NDGSBP_OK;
}

ndgsbp_status ndgsbp_workspace_status(const void* d_workspace, uint32_t* status, void* stream) {
    clear_error();
    if (!d_workspace || !status) return fail(NDGSBP_ERR_INVALID, "workspace_status: null pointer");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CUDA_TRY(cudaMemcpyAsync(status, static_cast<const unsigned char*>(d_workspace) + 8, 4, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return NDGSBP_OK;
}

ndgsbp_status ndgsbp_decode_static(const ndgsbp_groups* groups, const ndgsbp_params* params,
                                   const void* d_llr, int32_t llr_dtype, int64_t n_frames,
                                   uint32_t* d_hard_bits, int32_t* d_iters, uint8_t* d_syndrome_ok,
                                   float* d_posterior, void* stream) {
    clear_error();
    if (!groups) return fail(NDGSBP_ERR_INVALID, "decode_static: null groups handle");
    if (n_frames < 0) return fail(NDGSBP_ERR_INVALID, "decode_static: n_frames < 0");
    if (llr_dtype != NDGSBP_F32 && llr_dtype != NDGSBP_F64 && llr_dtype != NDGSBP_F16 && llr_dtype != NDGSBP_BF16)
        return fail(NDGSBP_ERR_INVALID, "decode_static: unknown llr_dtype %d", llr_dtype);
    if (n_frames > 0 && (!d_llr || !d_hard_bits))
        return fail(NDGSBP_ERR_INVALID, "decode_static: d_llr and d_hard_bits are required");
    ndgsbp_status sa = check_alignment("decode_static", d_llr, llr_dtype, d_hard_bits, d_iters, d_posterior);
    if (sa) return sa;
    const Groups& g = groups->g;
    Plan plan;
    ndgsbp_status st = make_plan(g, params, n_frames, plan, /*allow_upload=*/false);
    if (st) return st;
    if (n_frames == 0) return NDGSBP_OK;
    if (plan.pub.workspace_bytes > static_cast<int64_t>(NDGSBP_STATIC_SCRATCH_BYTES))
        return fail(NDGSBP_ERR_WORKSPACE,
                    "decode_static: this launch needs %lld bytes of scratch but the static array holds %u; "
                    "lower ctas_per_sm, let the messages stay in shared memory, or use ndgsbp_decode",
                    static_cast<long long>(plan.pub.workspace_bytes), NDGSBP_STATIC_SCRATCH_BYTES);
    void* ws = nullptr;
    st = static_scratch_address(&ws);
    if (st) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the frame counter must start at zero; message and delta slots are written before read
    CUDA_TRY(cudaMemsetAsync(ws, 0, kStatusEnd, s));   // frame counter and status word
    return launch_plan(g, plan, params, d_llr, llr_dtype, n_frames, static_cast<unsigned char*>(ws), d_hard_bits,
                       d_iters, d_syndrome_ok, d_posterior, nullptr, s);
}

}  // extern "C"
