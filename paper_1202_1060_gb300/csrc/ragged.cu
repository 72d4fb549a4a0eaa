// Ragged batches: several QC codes decoded by one persistent launch of the tile kernel, with
// an optional CUDA-graph replay of that launch.  In the per-code mode every code runs its own
// decode plan instead, the launches forked onto concurrent streams and joined.
#include <algorithm>
#include <cstring>
#include <memory>
#include <new>
#include <vector>

#include "decode_tile.h"
#include "ndgsbp_internal.h"

struct ndgsbp_ragged {
    ndgsbp::TileArgs args;
    ndgsbp::TileKernelFn fn = nullptr;
    int grid = 0, threads = 0;
    size_t smem = 0;
    int device = 0;
    void* workspace = nullptr;   // tile counter, then global message slots when needed
    int4* d_tiles = nullptr;
    int n_tiles = 0;
    ndgsbp_plan plan{};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    // per-code mode: one plan, batch and workspace offset per code; streams for codes 1..n-1,
    // events[0] forks, events[i] joins code i
    bool per_code = false;
    ndgsbp_params params{};
    std::vector<ndgsbp::Plan*> plans;
    std::vector<ndgsbp_batch> batches;
    std::vector<size_t> ws_off;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;
    ~ndgsbp_ragged() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        for (ndgsbp::Plan* p : plans) ndgsbp::plan_destroy(p);
        int cur = 0;
        if (cudaGetDevice(&cur) == cudaSuccess && cudaSetDevice(device) == cudaSuccess) {
            for (cudaStream_t st : streams) cudaStreamDestroy(st);
            for (cudaEvent_t ev : events) cudaEventDestroy(ev);
            cudaFree(workspace);
            cudaFree(d_tiles);
            cudaSetDevice(cur);
        }
        cudaGetLastError();
    }
};

namespace ndgsbp {

// Device tables of a grouping's QC layout (defined with the other layout uploads).
ndgsbp_status device_qc_tables(const Groups& g, const QcLayout*& Q, const DeviceQc*& D);

static size_t a16(size_t x) { return (x + 15) & ~static_cast<size_t>(15); }
static size_t a256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

}  // namespace ndgsbp

using namespace ndgsbp;

#define RAGGED_TRY(expr)                                                                           \
    do {                                                                                           \
        cudaError_t _e = (expr);                                                                   \
        if (_e != cudaSuccess) return fail(NDGSBP_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(_e)); \
    } while (0)

// Per-code mode: one ndgsbp_decode plan per batch (the library's default choice for its code),
// their workspaces in one allocation, streams and events for the fork and the join.
static ndgsbp_status create_per_code(const ndgsbp_batch* batches, int32_t n_batches, const ndgsbp_params* params,
                                     ndgsbp_ragged** out) {
    std::unique_ptr<ndgsbp_ragged> h(new (std::nothrow) ndgsbp_ragged);
    if (!h) return fail(NDGSBP_ERR_NOMEM, "out of host memory");
    RAGGED_TRY(cudaGetDevice(&h->device));
    std::memset(&h->args, 0, sizeof(h->args));
    h->per_code = true;
    h->params = *params;
    h->params.variant = NDGSBP_VARIANT_AUTO;
    h->params.block_threads = 0;
    h->params.ctas_per_sm = 0;
    h->params.frames_per_cta = 0;
    h->params.lanes_per_cn = 0;
    h->batches.assign(batches, batches + n_batches);
    ndgsbp_plan& o = h->plan;
    std::memset(&o, 0, sizeof(o));
    o.variant = NDGSBP_VARIANT_RAGGED_PER_CODE;
    size_t ws = 0;
    for (int i = 0; i < n_batches; ++i) {
        const ndgsbp_batch& b = batches[i];
        if (!b.groups || b.n_frames < 0 || (b.n_frames > 0 && (!b.d_llr || !b.d_hard_bits)))
            return fail(NDGSBP_ERR_INVALID, "ragged_create: batch %d is incomplete", i);
        ndgsbp_status st = NDGSBP_OK;
        Plan* plan = plan_create(b.groups->g, &h->params, std::max<int64_t>(1, b.n_frames), &st);
        if (!plan) return st;
        h->plans.push_back(plan);
        const ndgsbp_plan& pi = plan_info(*plan);
        h->ws_off.push_back(ws);
        ws += a256(static_cast<size_t>(std::max<int64_t>(pi.workspace_bytes, 256)));
        o.block_threads = std::max(o.block_threads, pi.block_threads);
        o.grid += pi.grid;
        o.ctas_per_sm = std::max(o.ctas_per_sm, pi.ctas_per_sm);
        o.max_row_degree = std::max(o.max_row_degree, pi.max_row_degree);
        o.smem_bytes = std::max(o.smem_bytes, pi.smem_bytes);
    }
    o.workspace_bytes = static_cast<int64_t>(ws);
    RAGGED_TRY(cudaMalloc(&h->workspace, ws));
    for (int i = 0; i < n_batches; ++i) {
        cudaEvent_t ev = nullptr;
        RAGGED_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        h->events.push_back(ev);
        if (i == 0) continue;
        cudaStream_t st = nullptr;
        RAGGED_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        h->streams.push_back(st);
    }
    h->n_tiles = n_batches;
    *out = h.release();
    return NDGSBP_OK;
}

extern "C" {

ndgsbp_status ndgsbp_ragged_create(const ndgsbp_batch* batches, int32_t n_batches, const ndgsbp_params* params,
                                   ndgsbp_ragged** out) {
    clear_error();
    if (!batches || !params || !out || n_batches < 1 || n_batches > kTileMaxCodes)
        return fail(NDGSBP_ERR_INVALID, "ragged_create: need 1..%d batches", kTileMaxCodes);
    if (params->max_iter < 1 || !(params->llr_max > 0.f && params->llr_max <= 30.f))
        return fail(NDGSBP_ERR_INVALID, "ragged_create: bad max_iter or llr_max");
    if (params->variant == NDGSBP_VARIANT_RAGGED_PER_CODE) return create_per_code(batches, n_batches, params, out);
    const int ms = params->msg_dtype == NDGSBP_F32 ? 4 : 2;
    if (!pick_tile_kernel(params->msg_dtype, false, 8, false, false))
        return fail(NDGSBP_ERR_INVALID, "ragged_create: msg_dtype must be F32, F16 or BF16");
    int dev = 0, sms = 0, optin = 0, smem_sm = 0, reserved = 0;
    RAGGED_TRY(cudaGetDevice(&dev));
    RAGGED_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    RAGGED_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    RAGGED_TRY(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    RAGGED_TRY(cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev));
    auto* h = new (std::nothrow) ndgsbp_ragged;
    if (!h) return fail(NDGSBP_ERR_NOMEM, "out of host memory");
    h->device = dev;
    std::memset(&h->args, 0, sizeof(h->args));
    // per code: layout, lanes per CN, slots
    struct CodePlan {
        const QcLayout* Q;
        const DeviceQc* D;
        int tpc, le, ds, msl, per_slot, slots, msg_slots;
        size_t table, p_bytes, m_bytes, d_bytes;
        double tile_cost;
    };
    std::vector<CodePlan> cp(n_batches);
    int threads = params->block_threads;
    size_t table_max = 0;
    for (int i = 0; i < n_batches; ++i) {
        const ndgsbp_batch& b = batches[i];
        if (!b.groups || b.n_frames < 0 || (b.n_frames > 0 && (!b.d_llr || !b.d_hard_bits))) {
            delete h;
            return fail(NDGSBP_ERR_INVALID, "ragged_create: batch %d is incomplete", i);
        }
        const Groups& g = b.groups->g;
        ndgsbp_status st = device_qc_tables(g, cp[i].Q, cp[i].D);
        if (st) {
            delete h;
            return st;
        }
        const QcLayout& Q = *cp[i].Q;
        if (!Q.ok) {
            delete h;
            return fail(NDGSBP_ERR_UNSUPPORTED, "ragged_create: batch %d is not a QC code grouped in whole layers", i);
        }
        const int tpc = b.lanes_per_cn ? b.lanes_per_cn : tile_lanes_per_cn(Q.max_deg);
        if (tpc != 1 && tpc != 2 && tpc != 4) {
            delete h;
            return fail(NDGSBP_ERR_UNSUPPORTED, "ragged_create: batch %d: row degree %d above 32 or bad lanes_per_cn",
                        i, Q.max_deg);
        }
        cp[i].tpc = tpc;
        cp[i].le = (Q.max_deg + tpc - 1) / tpc;
        if (cp[i].le > 8) {
            delete h;
            return fail(NDGSBP_ERR_UNSUPPORTED, "ragged_create: batch %d: %d edges per lane (at most 8)", i, cp[i].le);
        }
        const TileShape shp = tile_shape(Q, tpc, params->msg_dtype);
        cp[i].ds = shp.delta_stride;
        cp[i].msl = shp.msg_stride;
        cp[i].msg_slots = shp.msg_slots;
        cp[i].per_slot = Q.window * Q.Z * tpc;
        cp[i].table = tile_table_bytes(Q);
        cp[i].p_bytes = a16(static_cast<size_t>(g.code->N) * 4);
        cp[i].m_bytes = a16(static_cast<size_t>(shp.msg_slots) * ms);
        cp[i].d_bytes = a16(static_cast<size_t>(shp.delta_floats) * 4);
        cp[i].tile_cost = static_cast<double>(g.edge_updates);
        table_max = std::max(table_max, cp[i].table);
        if (!params->block_threads)
            threads = std::max(threads, std::min(512, std::max(128, (cp[i].per_slot + 31) / 32 * 32)));
    }
    if (threads <= 0 || threads > 1024 || threads % 32) {
        delete h;
        return fail(NDGSBP_ERR_INVALID, "ragged_create: block_threads must be a multiple of 32 up to 1024");
    }
    // Shared memory per CTA: one launch reserves the same amount for every code, so a code with
    // large frame slots would hold every CTA to its size.  A residency target of k CTAs per SM
    // caps each CTA at 1/k of the SM's shared memory; a code whose messages do not fit under the
    // cap keeps them in global memory.  Default: 2 CTAs per SM when every code fits, else 1.
    auto cap_for = [&](int k) {
        const size_t per = static_cast<size_t>(smem_sm) / k - static_cast<size_t>(reserved) - 1024;
        return std::min(static_cast<size_t>(optin) - 256, per) & ~static_cast<size_t>(15);
    };
    auto fits = [&](size_t cap) {
        for (int i = 0; i < n_batches; ++i)
            if (table_max + cp[i].p_bytes + cp[i].d_bytes > cap) return false;
        return true;
    };
    const int target = params->ctas_per_sm > 0 ? params->ctas_per_sm : (fits(cap_for(2)) ? 2 : 1);
    const size_t budget = cap_for(target);
    // slots and shared memory per code; the launch reserves the largest
    size_t smem = table_max;
    size_t ws = 256;
    std::vector<size_t> msg_off(n_batches, 0);
    for (int i = 0; i < n_batches; ++i) {
        CodePlan& c = cp[i];
        const bool msg_smem = table_max + c.p_bytes + c.m_bytes + c.d_bytes <= budget;
        const size_t slot = c.p_bytes + (msg_smem ? c.m_bytes : 0) + c.d_bytes;
        if (table_max + slot > budget) {
            delete h;
            return fail(NDGSBP_ERR_UNSUPPORTED, "ragged_create: batch %d does not fit in shared memory at %d CTAs per SM",
                        i, target);
        }
        const int max_slots = static_cast<int>(std::min<size_t>(16, (budget - table_max) / slot));
        const int want = batches[i].frames_per_cta ? batches[i].frames_per_cta
                                                   : std::max(1, std::min(16, threads / c.per_slot));
        c.slots = std::max(1, std::min(want, max_slots));
        smem = std::max(smem, table_max + c.slots * slot);
        TileCode& C = h->args.codes[i];
        const Groups& g = batches[i].groups->g;
        C.N = g.code->N;
        C.E = static_cast<int>(g.code->E);
        C.Z = c.Q->Z;
        C.nl = c.Q->n_layers;
        C.n_groupings = c.Q->n_groupings;
        C.G = static_cast<int>(c.Q->group_layers.size() / (static_cast<size_t>(c.Q->window) * c.Q->n_groupings));
        C.window = c.Q->window;
        C.maxdeg = c.Q->max_deg;
        C.msg_slots = c.msg_slots;
        C.msg_stride = c.msl;
        C.tpc = c.tpc;
        C.le = c.le;
        C.slots = c.slots;
        C.slot_bytes = static_cast<int>(slot);
        C.p_bytes = static_cast<int>(c.p_bytes);
        C.m_bytes = msg_smem ? static_cast<int>(c.m_bytes) : 0;
        C.delta_stride = c.ds;
        C.edge_tab = reinterpret_cast<const int2*>(c.D->edge_tab);
        C.layer_deg = c.D->layer_deg;
        C.group_layers = c.D->group_layers;
        C.csr_of = c.D->csr_of;
        tile_code_finish(C);
        RunArgs& r = C.r;
        const ndgsbp_batch& b = batches[i];
        r.N = C.N;
        r.E = C.E;
        r.W = (C.N + 31) / 32;
        r.llr = b.d_llr;
        r.llr_dtype = b.llr_dtype;
        r.n_frames = b.n_frames;
        r.max_iter = params->max_iter;
        r.llr_max = kernel_llr_limit(params->llr_max);
        r.early_stop = params->early_stop ? 1 : 0;
        r.hard_bits = b.d_hard_bits;
        r.iters = b.d_iters;
        r.synd_ok = b.d_syndrome_ok;
        r.posterior = b.d_posterior;
        r.stats = reinterpret_cast<unsigned long long*>(b.d_stats);
        r.start_ns = reinterpret_cast<unsigned long long*>(b.d_start_ns);
        r.retire_ns = reinterpret_cast<unsigned long long*>(b.d_retire_ns);
        if (!msg_smem) {
            msg_off[i] = ws;   // grid not known yet: sized below
        }
    }
    // kernel instance: the widest lane of the launch's codes; message changes in registers when
    // one round of the block covers a group of every code
    int lane_width = 0;
    bool regb = true;
    for (int i = 0; i < n_batches; ++i) {
        lane_width = std::max(lane_width, tile_lane_width(cp[i].le));
        regb = regb && cp[i].slots * cp[i].per_slot <= threads;
    }
    TileKernelFn fn = pick_tile_kernel(params->msg_dtype, false, lane_width, regb, n_batches == 1);
    if (!fn) {
        delete h;
        return fail(NDGSBP_ERR_UNSUPPORTED, "ragged_create: no kernel instance for lane width %d", lane_width);
    }
    RAGGED_TRY(cudaFuncSetAttribute(reinterpret_cast<const void*>(fn), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    static_cast<int>(smem)));
    int per_sm = 0;
    RAGGED_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, reinterpret_cast<const void*>(fn), threads, smem));
    if (per_sm < 1) {
        delete h;
        return fail(NDGSBP_ERR_UNSUPPORTED, "ragged_create: the launch does not fit on an SM");
    }
    per_sm = std::min(per_sm, target);
    // tiles: codes with the most work per tile first, so long tiles do not trail the launch
    std::vector<int> order(n_batches);
    for (int i = 0; i < n_batches; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        return cp[x].tile_cost * cp[x].slots > cp[y].tile_cost * cp[y].slots;
    });
    std::vector<int4> tiles;
    for (int i : order) {
        const int tf = cp[i].slots * 4;
        for (int64_t f = 0; f < batches[i].n_frames; f += tf)
            tiles.push_back(make_int4(i, static_cast<int>(f), static_cast<int>(std::min<int64_t>(tf, batches[i].n_frames - f)), 0));
    }
    h->n_tiles = static_cast<int>(tiles.size());
    int64_t grid = std::max<int64_t>(1, std::min<int64_t>(static_cast<int64_t>(per_sm) * sms, h->n_tiles));
    for (int i = 0; i < n_batches; ++i) {
        if (h->args.codes[i].m_bytes == 0) {
            msg_off[i] = ws;
            ws += a256(static_cast<size_t>(grid) * cp[i].slots * cp[i].msg_slots * ms);
        }
    }
    cudaError_t e = cudaMalloc(&h->workspace, ws);
    if (e == cudaSuccess && !tiles.empty()) e = cudaMalloc(reinterpret_cast<void**>(&h->d_tiles), tiles.size() * sizeof(int4));
    if (e == cudaSuccess && !tiles.empty())
        e = cudaMemcpy(h->d_tiles, tiles.data(), tiles.size() * sizeof(int4), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        delete h;
        return fail(NDGSBP_ERR_CUDA, "ragged_create: %s", cudaGetErrorString(e));
    }
    for (int i = 0; i < n_batches; ++i)
        h->args.codes[i].ws_msgs = h->args.codes[i].m_bytes ? nullptr : static_cast<unsigned char*>(h->workspace) + msg_off[i];
    h->args.n_codes = n_batches;
    h->args.tiles = h->d_tiles;
    h->args.n_tiles = h->n_tiles;
    h->args.tile_frames = 0;
    h->args.tile_counter = static_cast<unsigned long long*>(h->workspace);
    h->args.table_bytes = static_cast<int>(table_max);
    h->fn = fn;
    h->grid = static_cast<int>(grid);
    h->threads = threads;
    h->smem = smem;
    ndgsbp_plan& o = h->plan;
    o.variant = NDGSBP_VARIANT_TILE;
    o.block_threads = threads;
    o.grid = h->grid;
    o.ctas_per_sm = per_sm;
    o.max_row_degree = 0;
    for (int i = 0; i < n_batches; ++i) o.max_row_degree = std::max(o.max_row_degree, cp[i].Q->max_deg);
    o.delta_in_smem = 1;
    o.smem_bytes = static_cast<int64_t>(smem);
    o.workspace_bytes = static_cast<int64_t>(ws);
    o.stored_edges = 0;
    o.edge_updates_per_iter = 0;
    *out = h;
    return NDGSBP_OK;
}

ndgsbp_status ndgsbp_ragged_info(const ndgsbp_ragged* ragged, ndgsbp_plan* plan, int32_t* n_tiles) {
    if (!ragged) return fail(NDGSBP_ERR_INVALID, "ragged_info: null handle");
    if (plan) *plan = ragged->plan;
    if (n_tiles) *n_tiles = ragged->n_tiles;
    return NDGSBP_OK;
}

static ndgsbp_status enqueue(ndgsbp_ragged* h, cudaStream_t s) {
    if (h->per_code) {
        // fork: codes 1..n-1 on the handle's streams after everything before on s; join: s waits
        // for all of them
        const int n = static_cast<int>(h->plans.size());
        RAGGED_TRY(cudaEventRecord(h->events[0], s));
        for (int i = 0; i < n; ++i) {
            cudaStream_t si = i == 0 ? s : h->streams[i - 1];
            if (i > 0) RAGGED_TRY(cudaStreamWaitEvent(si, h->events[0], 0));
            const ndgsbp_batch& b = h->batches[i];
            ndgsbp_extras ex;
            std::memset(&ex, 0, sizeof(ex));
            ex.d_stats = b.d_stats;
            ex.d_start_ns = b.d_start_ns;
            ex.d_retire_ns = b.d_retire_ns;
            ndgsbp_status st = plan_enqueue(b.groups->g, *h->plans[i], &h->params, b.d_llr, b.llr_dtype, b.n_frames,
                                            static_cast<unsigned char*>(h->workspace) + h->ws_off[i], b.d_hard_bits,
                                            b.d_iters, b.d_syndrome_ok, b.d_posterior, &ex, si);
            if (st) return st;
            if (i > 0) RAGGED_TRY(cudaEventRecord(h->events[i], si));
        }
        for (int i = 1; i < n; ++i) RAGGED_TRY(cudaStreamWaitEvent(s, h->events[i], 0));
        return NDGSBP_OK;
    }
    RAGGED_TRY(cudaMemsetAsync(h->workspace, 0, sizeof(unsigned long long), s));
    if (h->n_tiles > 0) h->fn<<<h->grid, h->threads, h->smem, s>>>(h->args);
    RAGGED_TRY(cudaGetLastError());
    return NDGSBP_OK;
}

ndgsbp_status ndgsbp_ragged_launch(ndgsbp_ragged* ragged, void* stream) {
    clear_error();
    if (!ragged) return fail(NDGSBP_ERR_INVALID, "ragged_launch: null handle");
    return enqueue(ragged, static_cast<cudaStream_t>(stream));
}

ndgsbp_status ndgsbp_ragged_graph_launch(ndgsbp_ragged* ragged, void* stream) {
    clear_error();
    if (!ragged) return fail(NDGSBP_ERR_INVALID, "ragged_graph_launch: null handle");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!ragged->exec) {
        cudaStream_t cap = nullptr;
        RAGGED_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        ndgsbp_status st = NDGSBP_OK;
        if (e == cudaSuccess) {
            st = enqueue(ragged, cap);
            cudaGraph_t graph = nullptr;
            cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
            if (st == NDGSBP_OK && e2 != cudaSuccess) st = fail(NDGSBP_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e2));
            if (st == NDGSBP_OK) {
                ragged->graph = graph;
                e2 = cudaGraphInstantiate(&ragged->exec, graph, 0);
                if (e2 != cudaSuccess) st = fail(NDGSBP_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e2));
            } else if (graph) {
                cudaGraphDestroy(graph);
            }
        } else {
            st = fail(NDGSBP_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
        }
        cudaStreamDestroy(cap);
        if (st) return st;
    }
    RAGGED_TRY(cudaGraphLaunch(ragged->exec, s));
    return NDGSBP_OK;
}

ndgsbp_status ndgsbp_ragged_destroy(ndgsbp_ragged* ragged) {
    delete ragged;
    return NDGSBP_OK;
}

}  // extern "C"
