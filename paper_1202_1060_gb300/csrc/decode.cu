// Batched NDGSBP decode kernels for sm_103a and their launcher.
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
//
// Eq. (1) is evaluated as a product of tanh(x/2) factors held as pairs (N, E) with
// tanh(x/2) = N / (N + E): one edge with u = exp(-|x|) is (1 - u, 2 u) up to a common scale,
// two pairs combine as (Na Nb, Ea (Eb + Nb) + Na Eb), and 2 atanh(N / (N + E)) = ln(1 + 2 N / E).
// All terms are positive, so nothing cancels: both saturated inputs (tanh near 1) and tiny
// ones keep full FP32 relative accuracy, and each edge costs one exp2, one reciprocal and one
// log2.  The exclusion "all edges but k" uses prefix and suffix combinations (no division).
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "ndgsbp_internal.h"

namespace ndgsbp {

struct DecodeArgs {
    int M, N, E, Epad, G, max_gd, W;
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
    const void* llr;
    int llr_dtype;
    long long n_frames;
    int max_iter;
    float llr_max;
    int early_stop;
    void* ws_msgs;
    float* ws_delta;
    unsigned long long* counter;
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

// ---- small device helpers ---------------------------------------------------------------
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

__device__ __forceinline__ float load_llr(const void* p, int dtype, long long i) {
    switch (dtype) {
        case NDGSBP_F64: return static_cast<float>(static_cast<const double*>(p)[i]);
        case NDGSBP_F16: return __half2float(static_cast<const __half*>(p)[i]);
        case NDGSBP_BF16: return __bfloat162float(static_cast<const __nv_bfloat16*>(p)[i]);
        default: return static_cast<const float*>(p)[i];
    }
}

// Phase A for one group entry: Eq. (1) on every edge of the entry's CN.
template <int MAXDC, typename MsgT>
__device__ __forceinline__ void cn_update_entry(const DecodeArgs& a, const float* __restrict__ P,
                                                MsgT* __restrict__ msg, float* __restrict__ delta, int i) {
    const int s = __ldg(a.ge_slot + i);
    const int d = __ldg(a.slot_deg + s);
    const int eb = __ldg(a.tile_base + (s >> 5)) + (s & 31);
    const int db = __ldg(a.ge_dpos + i);
    const float lim = a.llr_max;
    float xn[MAXDC], xe[MAXDC], old[MAXDC], pn[MAXDC], pe[MAXDC];
    unsigned neg = 0u;
    float cn = 1.f, ce = 0.f;
#pragma unroll
    for (int k = 0; k < MAXDC; ++k) {
        if (k < d) {
            const int v = __ldg(a.edge_vn + eb + 32 * k);
            const float o = to_f(msg[eb + 32 * k]);
            const float t = P[v] - o;
            old[k] = o;
            neg |= (t < 0.f ? 1u : 0u) << k;
            const float x = fminf(fabsf(t), lim);
            const float u = ex2_approx(x * -1.4426950408889634f);   // exp(-x)
            xn[k] = fmaf(-0.5f, u, 0.5f);                           // (1 - u) / 2
            xe[k] = u;                                              // (2 u) / 2
            pn[k] = cn;
            pe[k] = ce;
            ce = fmaf(ce, xn[k] + xe[k], cn * xe[k]);
            cn = cn * xn[k];
        }
    }
    const unsigned par = __popc(neg) & 1u;
    float sn = 1.f, se = 0.f;
#pragma unroll
    for (int k = MAXDC - 1; k >= 0; --k) {
        if (k < d) {
            const float en = pn[k] * sn;
            const float ee = fmaf(pe[k], sn + se, pn[k] * se);
            const float w = 2.f * en * rcp_approx(ee);
            const float mag = fminf(0.69314718055994531f * lg2_approx(1.f + w), lim);
            const float val = ((par ^ (neg >> k)) & 1u) ? -mag : mag;
            const MsgT q = from_f<MsgT>(val);
            msg[eb + 32 * k] = q;
            delta[db + 32 * k] = to_f(q) - old[k];
            se = fmaf(se, xn[k] + xe[k], sn * xe[k]);
            sn = sn * xn[k];
        }
    }
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

// Frame epilogue shared by the kernels: hard decisions, outputs, fused statistics.
__device__ void write_frame_outputs(const DecodeArgs& a, const float* __restrict__ P, long long f,
                                    int iters, int unsat, unsigned* s_err) {
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const int W = a.W;
    unsigned err = 0u;
    for (int w = warp; w < W; w += nw) {
        const int n = 32 * w + lane;
        const bool bit = (n < a.N) && (P[n] < 0.f);
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
        for (int n = tid; n < a.N; n += nt) a.posterior[f * a.N + n] = P[n];
    if (a.stats && lane == 0 && err) atomicAdd(s_err, err);
    __syncthreads();
    if (tid == 0) {
        if (a.iters) a.iters[f] = iters;
        if (a.synd_ok) a.synd_ok[f] = unsat ? 0 : 1;
        if (a.stats) {
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
        if (a.iter_hist) atomicAdd(a.iter_hist + iters, 1ull);
        if (a.retire_ns) a.retire_ns[f] = global_timer_ns();
    }
}

// Largest CTA of a kernel instance: the per-edge register arrays grow with the degree bound.
__host__ __device__ constexpr int max_threads_for(int maxdc) { return maxdc <= 8 ? 1024 : maxdc <= 16 ? 512 : 256; }

template <typename MsgT, bool MSG_SMEM, bool DELTA_SMEM, int MAXDC>
__global__ void __launch_bounds__(max_threads_for(MAXDC)) decode_kernel(const DecodeArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long s_frame;
    __shared__ unsigned s_err;
    const int tid = threadIdx.x, nt = blockDim.x;
    float* P = reinterpret_cast<float*>(smem);
    size_t off = (static_cast<size_t>(a.N) * 4 + 15) & ~static_cast<size_t>(15);
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
        if (tid == 0) s_frame = static_cast<long long>(atomicAdd(a.counter, 1ull));
        __syncthreads();
        const long long f = s_frame;
        if (f >= a.n_frames) break;
        if (a.start_ns && tid == 0) a.start_ns[f] = global_timer_ns();
        // initialisation: P_n = L_n, L_{m->n} = 0
        for (int n = tid; n < a.N; n += nt) P[n] = load_llr(a.llr, a.llr_dtype, f * a.N + n);
        for (int e = tid; e < a.Epad; e += nt) msg[e] = from_f<MsgT>(0.f);
        __syncthreads();
        int it = 1, unsat = 1;
        for (;; ++it) {
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
            const bool last = it >= a.max_iter;
            if (a.early_stop || last) {
                unsigned bad = 0u;
                for (int s = tid; s < a.M && !bad; s += nt) bad |= slot_parity(a, P, s);
                unsat = __syncthreads_or(bad);
                if (!unsat && a.early_stop) break;
            }
            if (last) break;
        }
        if (a.msgs_out) {
            for (int e = tid; e < a.Epad; e += nt) {
                const int csr = __ldg(a.edge_csr + e);
                if (csr >= 0) a.msgs_out[f * a.E + csr] = to_f(msg[e]);
            }
        }
        write_frame_outputs(a, P, f, it, unsat, &s_err);
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
static constexpr size_t kHeaderBytes = 256;

#define CUDA_TRY(expr)                                                                         \
    do {                                                                                       \
        cudaError_t _e = (expr);                                                               \
        if (_e != cudaSuccess) return fail(NDGSBP_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(_e)); \
    } while (0)

// ---- device copies of layouts -------------------------------------------------------------
template <typename T>
static size_t push_array(std::vector<std::pair<const void*, size_t>>& parts, const std::vector<T>& v,
                         size_t& off) {
    const size_t at = off;
    parts.push_back({v.data(), v.size() * sizeof(T)});
    off = align256(off + v.size() * sizeof(T) + 1);
    return at;
}

static ndgsbp_status upload_layout(const Layout& L, DeviceLayout& D) {
    std::vector<std::pair<const void*, size_t>> parts;
    size_t off = 0;
    const size_t o_deg = push_array(parts, L.slot_deg, off);
    const size_t o_tb = push_array(parts, L.tile_base, off);
    const size_t o_vn = push_array(parts, L.edge_vn, off);
    const size_t o_csr = push_array(parts, L.edge_csr, off);
    const size_t o_gp = push_array(parts, L.grp_ptr, off);
    const size_t o_gs = push_array(parts, L.ge_slot, off);
    const size_t o_gd = push_array(parts, L.ge_dpos, off);
    const size_t o_cb = push_array(parts, L.grp_colbase, off);
    const size_t o_nc = push_array(parts, L.grp_ncol, off);
    const size_t o_col = push_array(parts, L.gcol, off);
    std::vector<unsigned char> host(off, 0);
    size_t at[] = {o_deg, o_tb, o_vn, o_csr, o_gp, o_gs, o_gd, o_cb, o_nc, o_col};
    for (size_t i = 0; i < parts.size(); ++i)
        if (parts[i].second) std::memcpy(host.data() + at[i], parts[i].first, parts[i].second);
    void* blob = nullptr;
    CUDA_TRY(cudaMalloc(&blob, off));
    cudaError_t e = cudaMemcpy(blob, host.data(), off, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(blob);
        return fail(NDGSBP_ERR_CUDA, "descriptor upload: %s", cudaGetErrorString(e));
    }
    auto* b = static_cast<unsigned char*>(blob);
    D.blob = blob;
    D.bytes = off;
    D.slot_deg = reinterpret_cast<const int32_t*>(b + o_deg);
    D.tile_base = reinterpret_cast<const int32_t*>(b + o_tb);
    D.edge_vn = reinterpret_cast<const int32_t*>(b + o_vn);
    D.edge_csr = reinterpret_cast<const int32_t*>(b + o_csr);
    D.grp_ptr = reinterpret_cast<const int32_t*>(b + o_gp);
    D.ge_slot = reinterpret_cast<const int32_t*>(b + o_gs);
    D.ge_dpos = reinterpret_cast<const int32_t*>(b + o_gd);
    D.grp_colbase = reinterpret_cast<const int32_t*>(b + o_cb);
    D.grp_ncol = reinterpret_cast<const int32_t*>(b + o_nc);
    D.gcol = reinterpret_cast<const uint8_t*>(b + o_col);
    return NDGSBP_OK;
}

static ndgsbp_status device_layout(const Groups& g, bool flood, const Layout*& L, const DeviceLayout*& D) {
    L = flood ? &flood_layout(g) : &g.grouped;
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(g.mu);
    auto& cache = flood ? g.dev_flood : g.dev_grouped;
    auto it = cache.find(dev);
    if (it == cache.end()) {
        DeviceLayout dl;
        ndgsbp_status st = upload_layout(*L, dl);
        if (st) return st;
        it = cache.emplace(dev, dl).first;
    }
    D = &it->second;
    return NDGSBP_OK;
}

void release_device_layouts(Groups& g) {
    int cur = 0;
    if (cudaGetDevice(&cur) != cudaSuccess) return;
    for (auto* cache : {&g.dev_grouped, &g.dev_flood}) {
        for (auto& kv : *cache) {
            if (cudaSetDevice(kv.first) == cudaSuccess) cudaFree(kv.second.blob);
        }
        cache->clear();
    }
    for (auto* cache : {&g.dev_qc, &g.dev_flood_qc}) {
        for (auto& kv : *cache) {
            if (cudaSetDevice(kv.first) == cudaSuccess) cudaFree(kv.second);
        }
        cache->clear();
    }
    cudaSetDevice(cur);
    cudaGetLastError();
}

Groups::~Groups() { release_device_layouts(*this); }

// ---- planning -----------------------------------------------------------------------------
struct Plan {
    ndgsbp_plan pub;
    KernelFn fn = nullptr;
    bool msg_smem = false, delta_smem = false;
    const Layout* L = nullptr;
    const DeviceLayout* D = nullptr;
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
    if (p->variant < NDGSBP_VARIANT_AUTO || p->variant > NDGSBP_VARIANT_QC)
        return fail(NDGSBP_ERR_INVALID, "unknown variant %d", p->variant);
    return NDGSBP_OK;
}

static ndgsbp_status make_plan(const Groups& g, const ndgsbp_params* p, int64_t n_frames, Plan& plan) {
    ndgsbp_status st = validate_params(p);
    if (st) return st;
    const bool flood = p->schedule == NDGSBP_SCHEDULE_FLOOD;
    st = device_layout(g, flood, plan.L, plan.D);
    if (st) return st;
    const Layout& L = *plan.L;
    const int maxdc = degree_bound(L.max_deg);
    if (!maxdc) return fail(NDGSBP_ERR_UNSUPPORTED, "CN degree %d above 32", L.max_deg);
    int dev = 0, sms = 0, smem_optin = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CUDA_TRY(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const size_t static_smem = 64;
    const size_t budget = static_cast<size_t>(smem_optin) - static_smem;
    const size_t p_bytes = align16(static_cast<size_t>(L.N) * 4);
    const size_t m_bytes = align16(static_cast<size_t>(L.Epad) * msg_size(p->msg_dtype));
    const size_t d_bytes = align16(static_cast<size_t>(L.max_gd) * 4);
    bool msg_smem, delta_smem;
    int variant = p->variant == NDGSBP_VARIANT_QC ? NDGSBP_VARIANT_AUTO : p->variant;
    if (variant == NDGSBP_VARIANT_SMEM) {
        if (p_bytes + m_bytes + d_bytes > budget)
            return fail(NDGSBP_ERR_UNSUPPORTED, "SMEM variant needs %zu bytes of shared memory, device has %zu",
                        p_bytes + m_bytes + d_bytes, budget);
        msg_smem = delta_smem = true;
    } else if (variant == NDGSBP_VARIANT_GLOBAL) {
        msg_smem = false;
        delta_smem = p_bytes + d_bytes <= budget;
    } else {
        msg_smem = p_bytes + m_bytes + d_bytes <= budget;
        delta_smem = msg_smem || p_bytes + d_bytes <= budget;
    }
    if (p_bytes > budget) return fail(NDGSBP_ERR_UNSUPPORTED, "posterior of %d VNs does not fit in shared memory", L.N);
    const size_t smem = p_bytes + (msg_smem ? m_bytes : 0) + (delta_smem ? d_bytes : 0);
    const int tmax = max_threads_for(maxdc);
    int threads = p->block_threads;
    if (!threads) threads = std::min(tmax, std::max(64, (L.max_group_entries + 31) / 32 * 32));
    if (threads > tmax) return fail(NDGSBP_ERR_UNSUPPORTED, "block_threads %d above %d for CN degree %d", threads, tmax, L.max_deg);
    KernelFn fn = pick_kernel(p->msg_dtype, maxdc, msg_smem, delta_smem);
    if (!fn) return fail(NDGSBP_ERR_UNSUPPORTED, "no kernel instance for this configuration");
    CUDA_TRY(cudaFuncSetAttribute(reinterpret_cast<const void*>(fn), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  static_cast<int>(smem)));
    int per_sm = 0;
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, reinterpret_cast<const void*>(fn), threads, smem));
    if (per_sm < 1) return fail(NDGSBP_ERR_UNSUPPORTED, "kernel does not fit on an SM with %d threads", threads);
    if (p->ctas_per_sm > 0) per_sm = std::min(per_sm, p->ctas_per_sm);
    int64_t grid = static_cast<int64_t>(per_sm) * sms;
    grid = std::max<int64_t>(1, std::min<int64_t>(grid, std::max<int64_t>(n_frames, 1)));
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

}  // namespace ndgsbp

using namespace ndgsbp;

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
    Plan plan;
    ndgsbp_status st = make_plan(groups->g, params, n_frames, plan);
    if (st) return st;
    if (n_frames == 0) return NDGSBP_OK;
    if (!d_workspace || workspace_bytes < static_cast<size_t>(plan.pub.workspace_bytes))
        return fail(NDGSBP_ERR_WORKSPACE, "decode: workspace of %zu bytes, need %lld", workspace_bytes,
                    static_cast<long long>(plan.pub.workspace_bytes));
    if (reinterpret_cast<uintptr_t>(d_workspace) % 256)
        return fail(NDGSBP_ERR_WORKSPACE, "decode: workspace must be 256-byte aligned");
    const Layout& L = *plan.L;
    const DeviceLayout& D = *plan.D;
    DecodeArgs a;
    std::memset(&a, 0, sizeof(a));
    a.M = L.M;
    a.N = L.N;
    a.E = static_cast<int>(groups->g.code->E);
    a.Epad = L.Epad;
    a.G = L.G;
    a.max_gd = L.max_gd;
    a.W = (L.N + 31) / 32;
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
    a.llr = d_llr;
    a.llr_dtype = llr_dtype;
    a.n_frames = n_frames;
    a.max_iter = params->max_iter;
    a.llr_max = params->llr_max;
    a.early_stop = params->early_stop ? 1 : 0;
    auto* ws = static_cast<unsigned char*>(d_workspace);
    a.counter = reinterpret_cast<unsigned long long*>(ws);
    size_t off = kHeaderBytes;
    if (!plan.msg_smem) {
        a.ws_msgs = ws + off;
        off += align256(static_cast<size_t>(plan.pub.grid) * L.Epad * msg_size(params->msg_dtype));
    }
    if (!plan.delta_smem) a.ws_delta = reinterpret_cast<float*>(ws + off);
    a.hard_bits = d_hard_bits;
    a.iters = d_iters;
    a.synd_ok = d_syndrome_ok;
    a.posterior = d_posterior;
    if (extras) {
        a.ref_bits = extras->d_ref_bits;
        a.ref_per_frame = extras->ref_per_frame;
        a.stats = reinterpret_cast<unsigned long long*>(extras->d_stats);
        a.iter_hist = reinterpret_cast<unsigned long long*>(extras->d_iter_hist);
        a.start_ns = reinterpret_cast<unsigned long long*>(extras->d_start_ns);
        a.retire_ns = reinterpret_cast<unsigned long long*>(extras->d_retire_ns);
        a.msgs_out = extras->d_messages;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CUDA_TRY(cudaMemsetAsync(a.counter, 0, sizeof(unsigned long long), s));
    plan.fn<<<plan.pub.grid, plan.pub.block_threads, plan.pub.smem_bytes, s>>>(a);
    CUDA_TRY(cudaGetLastError());
    return NDGSBP_OK;
}

ndgsbp_status ndgsbp_decode(const ndgsbp_groups* groups, const ndgsbp_params* params,
                            const void* d_llr, int32_t llr_dtype, int64_t n_frames,
                            void* d_workspace, size_t workspace_bytes, uint32_t* d_hard_bits,
                            int32_t* d_iters, uint8_t* d_syndrome_ok, float* d_posterior,
                            void* stream) {
    return ndgsbp_decode_ex(groups, params, d_llr, llr_dtype, n_frames, d_workspace, workspace_bytes,
                            d_hard_bits, d_iters, d_syndrome_ok, d_posterior, nullptr, stream);
}

}  // extern "C"
