// Serving: continuous batching of decode requests over device-resident frame slots.
//
// Per code the server owns a pool of slots.  The decoding state of a running frame (posterior,
// messages, iteration count, status flag) lives in device memory; its channel LLRs are staged in
// pinned host memory that the kernel reads when the frame starts, and its outputs go straight
// to pinned host memory that the kernel writes when the frame retires.  A worker thread repeats
// one epoch:
//   1. admit: frames that the staging threads have already placed (queued requests' frames, in
//      arrival order, take free slots of their code's pool and have their LLRs copied to the
//      slots' staging, concurrently with the epochs) are listed for a small admit kernel that
//      marks their slots new;
//   2. run: per pool whose code the layered QC kernel or the stream kernel decodes (the plain
//      decode's choice), one serving launch of that kernel over the pool's running slots, on the
//      pool's own stream; for the other pools, one launch of the tile kernel in serving mode over
//      the tiles of their occupied slots; all launches of the epoch run concurrently and join before the
//      harvest.  Each running frame advances by at most epoch_iters iterations, then retires
//      (zero syndrome or max_iter: outputs written, slot listed as done) or is parked with its
//      state in device memory;
//   3. harvest (on the host while the next epoch runs on the GPU; epochs alternate between two
//      done lists): the done lists come back (a count per pool); retired frames free their slots
//      and their outputs are copied into their requests' buffers; a request completes when all
//      its frames have retired.
// Frames of different requests and codes share every launch, and new requests join as soon as
// slots free up.  Each frame is computed exactly as by its pool's kernel in a plain decode.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <functional>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "decode_qc.h"
#include "decode_stream.h"
#include "decode_tile.h"
#include "ndgsbp_internal.h"

namespace ndgsbp {
ndgsbp_status device_qc_tables(const Groups& g, const QcLayout*& Q, const DeviceQc*& D);
}

using namespace ndgsbp;
using Clock = std::chrono::steady_clock;

namespace {

constexpr int kMaxPoolSlots = 16384;

struct AdmitArgs {
    int* flags[kTileMaxCodes];
    const int* list;   // entries pool << 24 | slot
    int n;
};

// Marks the admitted slots new (their LLRs are already staged).
__global__ void admit_kernel(const AdmitArgs a) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += gridDim.x * blockDim.x) {
        const int e = a.list[i];
        a.flags[e >> 24][e & 0xffffff] = kSlotNew;
    }
}

struct Request {
    int64_t ticket = 0;
    int code = 0;
    int64_t n_frames = 0;
    const float* llr = nullptr;
    uint32_t* hard = nullptr;
    int32_t* iters = nullptr;
    uint8_t* ok = nullptr;
    int64_t admitted = 0, retired = 0;
    Clock::time_point t_submit, t_done;
    bool done = false;
};

struct Pool {
    const Groups* g = nullptr;
    const QcLayout* Q = nullptr;
    const DeviceQc* D = nullptr;
    int N = 0, W = 0, slots = 0, tpc = 1, le = 1, ds = 1, msl = 1, cta_slots = 1, tile_frames = 1, msg_slots = 0;
    size_t slot_bytes = 0, p_bytes = 0, m_bytes = 0, d_bytes = 0;
    // device: state of running frames
    int* flag = nullptr;
    int* st_iter = nullptr;
    float* st_P = nullptr;
    void* st_msgs = nullptr;
    // pinned host, mapped into the device: LLR staging (read by the kernel), outputs and the
    // done list (written by the kernel)
    float* h_stage = nullptr;
    uint32_t* h_hard = nullptr;
    int32_t* h_iters = nullptr;
    uint8_t* h_ok = nullptr;
    int* h_done[2] = {nullptr, nullptr};   // two done lists: epochs alternate between them
    int* d_done[2] = {nullptr, nullptr};   // their device views
    std::vector<int> free_slots;   // tile pools: kept in descending order (the lowest free slot is taken first)
    std::vector<std::pair<Request*, int64_t>> owner;   // frame held by each slot (staged or running)
    std::vector<uint8_t> running;   // the slot's frame has been launched
    std::vector<int> ready;         // staged slots waiting for the next epoch
    // QC pools: advanced by the serving instance of the layered QC kernel (one launch per epoch
    // over the listed running slots, on the pool's own stream); stream pools likewise by the
    // serving instance of the stream kernel; the others by the tile launch
    bool qc = false;
    QcServePlan qp;
    QcArgs qargs{};
    bool stream = false;
    StreamServePlan sp;
    StreamArgs sargs{};
    int qc_grid = 1, n_list = 0;
    bool listed() const { return qc || stream; }   // runs its own launch over a slot list
    int* h_list = nullptr;          // pinned, mapped: this epoch's running slots
    cudaStream_t qstream = nullptr;
    cudaEvent_t qdone = nullptr;    // the pool's launch of this epoch has completed (join)
};

constexpr int kStageBatch = 512;   // frames a staging thread places per lock hold
// Staging threads: each takes the next batch of queued frames (slots are assigned in arrival
// order under the lock) and copies their LLRs concurrently with the others; one thread's copy
// rate (about 10 GB/s) would otherwise bound the saturated serving rate.
constexpr int kStagers = 3;

template <typename T>
T* device_view(T* host) {
    void* d = nullptr;
    return cudaHostGetDevicePointer(&d, host, 0) == cudaSuccess ? static_cast<T*>(d) : nullptr;
}

}  // namespace

struct ndgsbp_server {
    std::vector<Pool> pools;
    ndgsbp_params params{};
    int epoch_iters = 1;
    int device = 0;
    TileArgs args{};
    TileKernelFn fn = nullptr;
    int max_grid = 0, threads = 0;
    size_t smem = 0;
    int4* d_tiles = nullptr;
    int4* h_tiles = nullptr;
    int* d_admit = nullptr;
    int* h_admit = nullptr;
    int* d_done_count = nullptr;
    int* h_done_count = nullptr;
    unsigned long long* d_counter = nullptr;   // [0] the tile launch, [1 + i] QC pool i
    cudaStream_t stream = nullptr;
    cudaEvent_t fork = nullptr;     // QC pool launches start after the epoch's admission
    std::mutex mu;
    std::condition_variable cv_work, cv_done, cv_stage;
    std::deque<Request*> queue;
    std::unordered_map<int64_t, std::unique_ptr<Request>> reqs;
    int64_t next_ticket = 1;
    int64_t in_flight = 0;   // frames holding a slot (staged or running)
    int64_t n_running = 0;   // launched frames not yet retired
    int64_t n_ready = 0;     // staged frames waiting for an epoch
    bool stop = false;
    ndgsbp_status failed = NDGSBP_OK;
    std::string failure;
    std::thread worker;
    std::vector<std::thread> stagers;
    ndgsbp_server_stats stats{};

    ~ndgsbp_server();
    void run();
    void stage();
    bool enqueue(int par, bool* launched);
    void harvest(int par);
    bool can_stage() const {
        for (const Request* r : queue)
            if (!pools[r->code].free_slots.empty()) return true;
        return false;
    }
};

ndgsbp_server::~ndgsbp_server() {
    {
        std::lock_guard<std::mutex> lock(mu);
        stop = true;
    }
    cv_work.notify_all();
    cv_stage.notify_all();
    for (std::thread& t : stagers)
        if (t.joinable()) t.join();
    if (worker.joinable()) worker.join();
    int cur = 0;
    if (cudaGetDevice(&cur) == cudaSuccess && cudaSetDevice(device) == cudaSuccess) {
        if (stream) cudaStreamSynchronize(stream);
        for (Pool& p : pools) {
            if (p.qstream) cudaStreamDestroy(p.qstream);
            if (p.qdone) cudaEventDestroy(p.qdone);
            cudaFreeHost(p.h_list);
            cudaFree(p.flag);
            cudaFree(p.st_iter);
            cudaFree(p.st_P);
            cudaFree(p.st_msgs);
            cudaFreeHost(p.h_stage);
            cudaFreeHost(p.h_hard);
            cudaFreeHost(p.h_iters);
            cudaFreeHost(p.h_ok);
            cudaFreeHost(p.h_done[0]);
            cudaFreeHost(p.h_done[1]);
        }
        cudaFree(d_tiles);
        cudaFreeHost(h_tiles);
        cudaFree(d_admit);
        cudaFreeHost(h_admit);
        cudaFree(d_done_count);
        cudaFreeHost(h_done_count);
        cudaFree(d_counter);
        if (fork) cudaEventDestroy(fork);
        if (stream) cudaStreamDestroy(stream);
        cudaSetDevice(cur);
    }
    cudaGetLastError();
}

#define SRV_CUDA(expr)                                                                        \
    do {                                                                                      \
        cudaError_t _e = (expr);                                                              \
        if (_e != cudaSuccess) {                                                              \
            std::lock_guard<std::mutex> lock(mu);                                             \
            failed = NDGSBP_ERR_CUDA;                                                         \
            failure = std::string(#expr) + ": " + cudaGetErrorString(_e);                     \
            return false;                                                                     \
        }                                                                                     \
    } while (0)

// Enqueue one epoch on `stream` with done-list buffer `par` (the previous epoch has been
// synchronised): admission, slot lists and tiles, launches.  *launched = false when no frame is
// running or staged.  False on a CUDA error (recorded, the worker stops).
bool ndgsbp_server::enqueue(int par, bool* launched) {
    *launched = false;
    int n_admit = 0, n_tiles = 0;
    {
        std::lock_guard<std::mutex> lock(mu);
        // 1. admission of the staged frames
        for (int i = 0; i < static_cast<int>(pools.size()); ++i) {
            Pool& p = pools[i];
            for (int slot : p.ready) {
                h_admit[n_admit++] = (i << 24) | slot;
                p.running[slot] = 1;
            }
            n_running += static_cast<int64_t>(p.ready.size());
            p.ready.clear();
        }
        n_ready = 0;
        // listed pools: their running slots (slots whose frame retired in the epoch not yet
        // harvested are still listed: the kernel skips them, their flag says done); tile pools:
        // tiles over the running slots, ranges holding up to tile_frames running slots (other
        // slots inside a range are skipped)
        for (int i = 0; i < static_cast<int>(pools.size()); ++i) {
            Pool& p = pools[i];
            if (p.listed()) {
                p.n_list = 0;
                for (int slot = 0; slot < p.slots; ++slot)
                    if (p.running[slot]) p.h_list[p.n_list++] = slot;
                continue;
            }
            int first = -1, count = 0, last = -1;
            for (int slot = 0; slot < p.slots; ++slot) {
                if (!p.running[slot]) continue;
                if (first < 0) first = slot;
                last = slot;
                if (++count == p.tile_frames) {
                    h_tiles[n_tiles++] = make_int4(i, first, last - first + 1, 0);
                    first = -1;
                    count = 0;
                }
            }
            if (first >= 0) h_tiles[n_tiles++] = make_int4(i, first, last - first + 1, 0);
        }
    }
    int n_listed = 0, n_launches = 0;
    for (const Pool& p : pools) n_listed += p.listed() ? p.n_list : 0;
    if (n_tiles == 0 && n_listed == 0) return true;
    int* d_count = d_done_count + par * kTileMaxCodes;
    // 2. admit, then the launches
    if (n_admit) {
        SRV_CUDA(cudaMemcpyAsync(d_admit, h_admit, sizeof(int) * n_admit, cudaMemcpyHostToDevice, stream));
        AdmitArgs aa{};
        for (size_t i = 0; i < pools.size(); ++i) aa.flags[i] = pools[i].flag;
        aa.list = d_admit;
        aa.n = n_admit;
        admit_kernel<<<std::min(1024, (n_admit + 255) / 256), 256, 0, stream>>>(aa);
        SRV_CUDA(cudaGetLastError());
        ++n_launches;
    }
    SRV_CUDA(cudaMemsetAsync(d_count, 0, sizeof(int) * pools.size(), stream));
    SRV_CUDA(cudaMemsetAsync(d_counter, 0, sizeof(unsigned long long) * (1 + pools.size()), stream));
    // fork: each listed pool's launch on its own stream, concurrent with the tile launch
    SRV_CUDA(cudaEventRecord(fork, stream));
    for (size_t i = 0; i < pools.size(); ++i) {
        Pool& p = pools[i];
        if (!p.listed() || p.n_list == 0) continue;
        SRV_CUDA(cudaStreamWaitEvent(p.qstream, fork, 0));
        if (p.qc) {
            QcArgs qa = p.qargs;
            qa.r.n_frames = p.n_list;
            qa.done_list = p.d_done[par];
            qa.done_count = d_count + i;
            p.qp.fn<<<std::min(p.qc_grid, p.n_list), p.qp.threads, p.qp.smem, p.qstream>>>(qa);
        } else {
            StreamArgs sa = p.sargs;
            sa.r.n_frames = p.n_list;
            sa.done_list = p.d_done[par];
            sa.done_count = d_count + i;
            p.sp.fn<<<std::min(p.qc_grid, p.n_list), p.sp.threads, p.sp.smem, p.qstream>>>(sa);
        }
        SRV_CUDA(cudaGetLastError());
        ++n_launches;
        SRV_CUDA(cudaEventRecord(p.qdone, p.qstream));
    }
    if (n_tiles > 0) {
        SRV_CUDA(cudaMemcpyAsync(d_tiles, h_tiles, sizeof(int4) * n_tiles, cudaMemcpyHostToDevice, stream));
        TileArgs a = args;
        a.n_tiles = n_tiles;
        for (size_t i = 0; i < pools.size(); ++i) {
            a.codes[i].done_list = pools[i].d_done[par];
            a.codes[i].done_count = d_count + i;
        }
        fn<<<std::min(max_grid, n_tiles), threads, smem, stream>>>(a);
        SRV_CUDA(cudaGetLastError());
        ++n_launches;
    }
    for (Pool& p : pools)
        if (p.listed() && p.n_list > 0) SRV_CUDA(cudaStreamWaitEvent(stream, p.qdone, 0));
    SRV_CUDA(cudaMemcpyAsync(h_done_count + par * kTileMaxCodes, d_count, sizeof(int) * pools.size(),
                             cudaMemcpyDeviceToHost, stream));
    *launched = true;
    std::lock_guard<std::mutex> lock(mu);
    stats.epochs += 1;
    stats.launches += n_launches;
    return true;
}

// 3. Harvest the frames that retired in the (synchronised) epoch with done-list buffer par:
// free their slots, copy their outputs into their requests, complete finished requests.
void ndgsbp_server::harvest(int par) {
    const auto t0 = Clock::now();
    std::vector<Request*> finished;
    {
        std::lock_guard<std::mutex> lock(mu);
        for (size_t i = 0; i < pools.size(); ++i) {
            Pool& p = pools[i];
            const int n_done = h_done_count[par * kTileMaxCodes + i];
            const int* done = p.h_done[par];
            for (int k = 0; k < n_done; ++k) {
                const int slot = done[k];
                Request* r = p.owner[slot].first;
                if (!r) continue;
                const int64_t f = p.owner[slot].second;
                std::memcpy(r->hard + static_cast<size_t>(f) * p.W, p.h_hard + static_cast<size_t>(slot) * p.W,
                            sizeof(uint32_t) * p.W);
                if (r->iters) r->iters[f] = p.h_iters[slot];
                if (r->ok) r->ok[f] = p.h_ok[slot];
                stats.frames_completed += 1;
                stats.iterations += p.h_iters[slot];
                if (!p.h_ok[slot]) stats.frame_errors_unsatisfied += 1;
                p.owner[slot] = {nullptr, 0};
                p.running[slot] = 0;
                p.free_slots.push_back(slot);
                --in_flight;
                --n_running;
                if (++r->retired == r->n_frames) finished.push_back(r);
            }
            // tile pools take the lowest free slots first (their tiles cover ranges of running
            // slots, so compact occupancy means fewer tiles); listed pools take any free slot
            if (n_done && !p.listed()) std::sort(p.free_slots.begin(), p.free_slots.end(), std::greater<int>());
        }
        const auto t1 = Clock::now();
        for (Request* r : finished) {
            r->done = true;
            r->t_done = t1;
            stats.requests_completed += 1;
        }
        stats.harvest_seconds += std::chrono::duration<double>(t1 - t0).count();
    }
    if (!finished.empty()) cv_done.notify_all();
    cv_stage.notify_all();
}

// The worker: enqueue epoch k, harvest epoch k - 1 on the host while epoch k runs, synchronise,
// repeat.  A frame that retires in epoch k frees its slot when epoch k is harvested (during
// epoch k + 1), so the next frame can take it from epoch k + 2 on.
void ndgsbp_server::run() {
    cudaSetDevice(device);
    int par = 0;
    bool have_prev = false;   // an epoch has been synchronised and not yet harvested
    for (;;) {
        {
            std::unique_lock<std::mutex> lock(mu);
            cv_work.wait(lock, [&] { return stop || have_prev || n_ready > 0 || n_running > 0; });
            if (stop) return;
        }
        const auto t0 = Clock::now();
        bool launched = false;
        if (!enqueue(par, &launched)) break;
        if (have_prev) harvest(par ^ 1);
        have_prev = false;
        const auto t1 = Clock::now();
        if (launched) {
            const cudaError_t e = cudaStreamSynchronize(stream);
            if (e != cudaSuccess) {
                std::lock_guard<std::mutex> lock(mu);
                failed = NDGSBP_ERR_CUDA;
                failure = std::string("cudaStreamSynchronize: ") + cudaGetErrorString(e);
                break;
            }
            have_prev = true;
            par ^= 1;
        }
        const auto t2 = Clock::now();
        std::lock_guard<std::mutex> lock(mu);
        stats.device_seconds += std::chrono::duration<double>(t2 - t1).count();
        stats.busy_seconds += std::chrono::duration<double>(t2 - t0).count();
    }
    cv_done.notify_all();
}

// Staging threads: place queued frames, in arrival order, into free slots and copy their LLRs
// to the slots' staging while epochs run; the next epoch admits them.
void ndgsbp_server::stage() {
    struct Job {
        float* dst;
        const float* src;
        size_t n;
        int pool, slot;
    };
    std::vector<Job> jobs;
    jobs.reserve(kStageBatch);
    for (;;) {
        jobs.clear();
        {
            std::unique_lock<std::mutex> lock(mu);
            cv_stage.wait(lock, [&] { return stop || can_stage(); });
            if (stop) return;
            for (auto it = queue.begin(); it != queue.end() && static_cast<int>(jobs.size()) < kStageBatch;) {
                Request* r = *it;
                Pool& p = pools[r->code];
                while (r->admitted < r->n_frames && !p.free_slots.empty() && static_cast<int>(jobs.size()) < kStageBatch) {
                    const int slot = p.free_slots.back();
                    p.free_slots.pop_back();
                    p.owner[slot] = {r, r->admitted};
                    jobs.push_back({p.h_stage + static_cast<size_t>(slot) * p.N,
                                    r->llr + static_cast<size_t>(r->admitted) * p.N, static_cast<size_t>(p.N), r->code,
                                    slot});
                    ++r->admitted;
                    ++in_flight;
                }
                it = (r->admitted == r->n_frames) ? queue.erase(it) : std::next(it);
            }
        }
        const auto t0 = Clock::now();
        for (const Job& j : jobs) std::memcpy(j.dst, j.src, sizeof(float) * j.n);
        const auto t1 = Clock::now();
        {
            std::lock_guard<std::mutex> lock(mu);
            for (const Job& j : jobs) pools[j.pool].ready.push_back(j.slot);
            n_ready += static_cast<int64_t>(jobs.size());
            stats.admit_seconds += std::chrono::duration<double>(t1 - t0).count();
        }
        cv_work.notify_one();
    }
}

static size_t a16(size_t x) { return (x + 15) & ~static_cast<size_t>(15); }

extern "C" {

ndgsbp_status ndgsbp_server_create(const ndgsbp_groups* const* codes, int32_t n_codes, const double* weights,
                                   const ndgsbp_params* params, size_t hbm_budget_bytes, int32_t epoch_iters,
                                   ndgsbp_server** out) {
    clear_error();
    if (!codes || !params || !out || n_codes < 1 || n_codes > kTileMaxCodes || epoch_iters < 1)
        return fail(NDGSBP_ERR_INVALID, "server_create: need 1..%d codes, params and epoch_iters >= 1", kTileMaxCodes);
    if (params->max_iter < 1 || !(params->llr_max > 0.f && params->llr_max <= 30.f))
        return fail(NDGSBP_ERR_INVALID, "server_create: bad max_iter or llr_max");
    if (!pick_tile_kernel(params->msg_dtype, /*serve=*/true, 8, false, false))
        return fail(NDGSBP_ERR_INVALID, "server_create: msg_dtype must be F32, F16 or BF16");
    const int ms = params->msg_dtype == NDGSBP_F32 ? 4 : 2;
    std::unique_ptr<ndgsbp_server> h(new (std::nothrow) ndgsbp_server);
    if (!h) return fail(NDGSBP_ERR_NOMEM, "out of host memory");
    int dev = 0, sms = 0, optin = 0, smem_sm = 0, reserved = 0, mapped = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) ||
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) ||
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) ||
        cudaDeviceGetAttribute(&mapped, cudaDevAttrCanMapHostMemory, dev))
        return fail(NDGSBP_ERR_CUDA, "server_create: no CUDA device");
    if (!mapped) return fail(NDGSBP_ERR_UNSUPPORTED, "server_create: the device cannot map host memory");
    h->device = dev;
    h->params = *params;
    h->epoch_iters = epoch_iters;
    h->pools.resize(n_codes);
    double wsum = 0.0;
    for (int i = 0; i < n_codes; ++i) wsum += weights ? std::max(0.0, weights[i]) : 1.0;
    if (!(wsum > 0.0)) return fail(NDGSBP_ERR_INVALID, "server_create: weights sum to zero");
    size_t table_max = 0;
    int threads = params->block_threads;
    int n_tile_pools = 0;
    for (int i = 0; i < n_codes; ++i) {
        Pool& p = h->pools[i];
        if (!codes[i]) return fail(NDGSBP_ERR_INVALID, "server_create: code %d is null", i);
        p.g = &codes[i]->g;
        if (!p.g->qc.ok) return fail(NDGSBP_ERR_UNSUPPORTED, "server_create: code %d is not QC grouped in whole layers", i);
        ndgsbp_status st = device_qc_tables(*p.g, p.Q, p.D);
        if (st) return st;
        // the QC kernel where the grouping's plain decode would use it (unless TILE is asked for)
        if (params->variant != NDGSBP_VARIANT_TILE) {
            bool ok = false;
            st = qc_serve_plan(*p.g, params, &p.qp, &ok);
            if (st) return st;
            p.qc = ok;
            if (!ok) {   // the stream kernel where the plain decode uses it
                st = stream_serve_plan(*p.g, params, &p.sp, &ok);
                if (st) return st;
                p.stream = ok;
            }
        }
        p.tpc = tile_lanes_per_cn(p.Q->max_deg);
        if (!p.tpc) return fail(NDGSBP_ERR_UNSUPPORTED, "server_create: code %d has row degree above 32", i);
        p.le = (p.Q->max_deg + p.tpc - 1) / p.tpc;
        const TileShape shp = tile_shape(*p.Q, p.tpc, params->msg_dtype);
        p.ds = shp.delta_stride;
        p.msl = shp.msg_stride;
        p.msg_slots = shp.msg_slots;
        p.N = p.g->code->N;
        p.W = (p.N + 31) / 32;
        p.p_bytes = a16(static_cast<size_t>(p.N) * 4);
        p.m_bytes = a16(static_cast<size_t>(p.msg_slots) * ms);
        p.d_bytes = a16(static_cast<size_t>(shp.delta_floats) * 4);
        if (p.qc) {
            p.msg_slots = p.qp.msg_slots;
            continue;
        }
        if (p.stream) {
            p.msg_slots = p.sp.msg_elems_per_slot;
            continue;
        }
        ++n_tile_pools;
        table_max = std::max(table_max, tile_table_bytes(*p.Q));
        if (!params->block_threads)
            threads = std::max(threads, std::min(512, std::max(128, (p.Q->window * p.Q->Z * p.tpc + 31) / 32 * 32)));
    }
    if (n_tile_pools > 0 && (threads <= 0 || threads > 1024 || threads % 32))
        return fail(NDGSBP_ERR_INVALID, "server_create: block_threads must be a multiple of 32 up to 1024");
    // Shared memory per CTA under a residency target of k CTAs per SM (as for ragged launches):
    // a code whose messages do not fit under the cap works on them in device memory, where a
    // parked frame keeps them anyway.  Default k: 2 when every code fits, else 1.
    auto cap_for = [&](int k) {
        const size_t per = static_cast<size_t>(smem_sm) / k - static_cast<size_t>(reserved) - 1024;
        return std::min(static_cast<size_t>(optin) - 256, per) & ~static_cast<size_t>(15);
    };
    auto fits = [&](size_t cap) {
        for (const Pool& p : h->pools)
            if (!p.listed() && table_max + p.p_bytes + p.d_bytes > cap) return false;
        return true;
    };
    const int target = params->ctas_per_sm > 0 ? params->ctas_per_sm : (fits(cap_for(2)) ? 2 : 1);
    const size_t budget = cap_for(target);
    size_t smem = table_max;
    for (int i = 0; i < n_codes; ++i) {
        Pool& p = h->pools[i];
        if (!p.listed()) {
            if (table_max + p.p_bytes + p.m_bytes + p.d_bytes > budget) p.m_bytes = 0;
            p.slot_bytes = p.p_bytes + p.m_bytes + p.d_bytes;
            if (table_max + p.slot_bytes > budget)
                return fail(NDGSBP_ERR_UNSUPPORTED, "server_create: code %d does not fit at %d CTAs per SM", i, target);
            const int per_slot = p.Q->window * p.Q->Z * p.tpc;
            p.cta_slots = std::max(1, std::min<int>({16, std::max(1, threads / per_slot),
                                                     static_cast<int>((budget - table_max) / p.slot_bytes)}));
            p.tile_frames = 2 * p.cta_slots;
            smem = std::max(smem, table_max + p.cta_slots * p.slot_bytes);
        }
        // pool size from the budget share: posterior and messages of a running frame, LLR
        // staging, outputs and status per slot
        const double share = (weights ? std::max(0.0, weights[i]) : 1.0) / wsum;
        const size_t per = sizeof(float) * p.N * 2 + static_cast<size_t>(p.msg_slots) * ms + sizeof(uint32_t) * p.W + 16;
        p.slots = static_cast<int>(std::min<double>(kMaxPoolSlots, std::floor(share * hbm_budget_bytes / per)));
        if (p.slots < 1) return fail(NDGSBP_ERR_BUDGET, "server_create: the budget leaves no slot for code %d", i);
    }
    // kernel instance: the widest lane of the pools' codes; message changes in registers when one
    // round of the block covers a group of every code
    int lane_width = 0;
    bool regb = true;
    for (int i = 0; i < n_codes; ++i) {
        const Pool& p = h->pools[i];
        if (p.listed()) continue;
        lane_width = std::max(lane_width, tile_lane_width(p.le));
        regb = regb && p.cta_slots * p.Q->window * p.Q->Z * p.tpc <= threads;
    }
    TileKernelFn fn = nullptr;
    if (n_tile_pools > 0) {
        fn = pick_tile_kernel(params->msg_dtype, /*serve=*/true, lane_width, regb, false);
        if (!fn) return fail(NDGSBP_ERR_UNSUPPORTED, "server_create: no kernel instance for lane width %d", lane_width);
    }
    cudaError_t e = cudaSuccess;
    auto dmalloc = [&](void** ptr, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(ptr, bytes);
        if (e == cudaSuccess) e = cudaMemset(*ptr, 0, bytes);
    };
    auto hmalloc = [&](void** ptr, size_t bytes) {
        if (e == cudaSuccess) e = cudaHostAlloc(ptr, bytes, cudaHostAllocMapped);
        if (e == cudaSuccess) std::memset(*ptr, 0, bytes);
    };
    int max_tiles = 0;
    for (int i = 0; i < n_codes; ++i) {
        Pool& p = h->pools[i];
        dmalloc(reinterpret_cast<void**>(&p.flag), sizeof(int) * p.slots);
        dmalloc(reinterpret_cast<void**>(&p.st_iter), sizeof(int) * p.slots);
        dmalloc(reinterpret_cast<void**>(&p.st_P), sizeof(float) * p.N * static_cast<size_t>(p.slots));
        dmalloc(&p.st_msgs, static_cast<size_t>(p.msg_slots) * ms * p.slots);
        hmalloc(reinterpret_cast<void**>(&p.h_stage), sizeof(float) * p.N * static_cast<size_t>(p.slots));
        hmalloc(reinterpret_cast<void**>(&p.h_hard), sizeof(uint32_t) * p.W * static_cast<size_t>(p.slots));
        hmalloc(reinterpret_cast<void**>(&p.h_iters), sizeof(int32_t) * p.slots);
        hmalloc(reinterpret_cast<void**>(&p.h_ok), p.slots);
        hmalloc(reinterpret_cast<void**>(&p.h_done[0]), sizeof(int) * p.slots);
        hmalloc(reinterpret_cast<void**>(&p.h_done[1]), sizeof(int) * p.slots);
        if (p.listed()) {
            hmalloc(reinterpret_cast<void**>(&p.h_list), sizeof(int) * p.slots);
            if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p.qstream, cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p.qdone, cudaEventDisableTiming);
        }
        if (e != cudaSuccess) return fail(NDGSBP_ERR_NOMEM, "server_create: %s", cudaGetErrorString(e));
        p.owner.assign(p.slots, {nullptr, 0});
        p.running.assign(p.slots, 0);
        for (int s = p.slots - 1; s >= 0; --s) p.free_slots.push_back(s);
        if (!p.listed()) max_tiles += (p.slots + p.tile_frames - 1) / p.tile_frames;
        h->stats.slots_total += p.slots;
    }
    dmalloc(reinterpret_cast<void**>(&h->d_tiles), sizeof(int4) * max_tiles);
    hmalloc(reinterpret_cast<void**>(&h->h_tiles), sizeof(int4) * max_tiles);
    dmalloc(reinterpret_cast<void**>(&h->d_admit), sizeof(int) * h->stats.slots_total);
    hmalloc(reinterpret_cast<void**>(&h->h_admit), sizeof(int) * h->stats.slots_total);
    dmalloc(reinterpret_cast<void**>(&h->d_done_count), sizeof(int) * 2 * kTileMaxCodes);
    hmalloc(reinterpret_cast<void**>(&h->h_done_count), sizeof(int) * 2 * kTileMaxCodes);
    dmalloc(reinterpret_cast<void**>(&h->d_counter), 256);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming);
    int per_sm = 1;
    if (fn) {
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(reinterpret_cast<const void*>(fn), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     static_cast<int>(smem));
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, reinterpret_cast<const void*>(fn), threads, smem);
        if (e != cudaSuccess) return fail(NDGSBP_ERR_CUDA, "server_create: %s", cudaGetErrorString(e));
        if (per_sm < 1) return fail(NDGSBP_ERR_UNSUPPORTED, "server_create: the launch does not fit on an SM");
        per_sm = std::min(per_sm, target);
    }
    for (Pool& p : h->pools) {
        if (!p.listed()) continue;
        const void* lfn = p.qc ? reinterpret_cast<const void*>(p.qp.fn) : reinterpret_cast<const void*>(p.sp.fn);
        const int lthreads = p.qc ? p.qp.threads : p.sp.threads;
        const size_t lsmem = p.qc ? p.qp.smem : p.sp.smem;
        int q_sm = 0;
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(lfn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(lsmem));
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&q_sm, lfn, lthreads, lsmem);
        if (e != cudaSuccess) return fail(NDGSBP_ERR_CUDA, "server_create: %s", cudaGetErrorString(e));
        if (q_sm < 1) return fail(NDGSBP_ERR_UNSUPPORTED, "server_create: a pool's launch does not fit on an SM");
        if (p.stream) q_sm = std::min(q_sm, std::max(1, p.sp.per_sm));
        p.qc_grid = q_sm * sms;
    }
    for (int i = 0; i < n_codes; ++i) {
        Pool& p = h->pools[i];
        TileCode& C = h->args.codes[i];
        C.N = p.N;
        C.E = static_cast<int>(p.g->code->E);
        C.Z = p.Q->Z;
        C.nl = p.Q->n_layers;
        C.n_groupings = p.Q->n_groupings;
        C.G = static_cast<int>(p.Q->group_layers.size() / (static_cast<size_t>(p.Q->window) * p.Q->n_groupings));
        C.window = p.Q->window;
        C.maxdeg = p.Q->max_deg;
        C.msg_slots = p.msg_slots;
        C.msg_stride = p.msl;
        C.tpc = p.tpc;
        C.le = p.le;
        C.slots = p.cta_slots;
        C.slot_bytes = static_cast<int>(p.slot_bytes);
        C.p_bytes = static_cast<int>(p.p_bytes);
        C.m_bytes = static_cast<int>(p.m_bytes);
        C.delta_stride = p.ds;
        C.edge_tab = reinterpret_cast<const int2*>(p.D->edge_tab);
        C.layer_deg = p.D->layer_deg;
        C.group_layers = p.D->group_layers;
        C.csr_of = p.D->csr_of;
        tile_code_finish(C);
        C.state_flag = p.flag;
        C.state_iter = p.st_iter;
        C.state_P = p.st_P;
        C.state_msgs = p.st_msgs;
        C.epoch_iters = epoch_iters;
        p.d_done[0] = device_view(p.h_done[0]);
        p.d_done[1] = device_view(p.h_done[1]);
        C.done_list = p.d_done[0];
        C.done_count = h->d_done_count + i;
        RunArgs& r = C.r;
        r.N = p.N;
        r.E = C.E;
        r.W = p.W;
        r.llr = device_view(p.h_stage);
        r.llr_dtype = NDGSBP_F32;
        r.n_frames = p.slots;
        r.max_iter = params->max_iter;
        r.llr_max = kernel_llr_limit(params->llr_max);
        r.early_stop = params->early_stop ? 1 : 0;
        r.hard_bits = device_view(p.h_hard);
        r.iters = device_view(p.h_iters);
        r.synd_ok = device_view(p.h_ok);
        if (!p.d_done[0] || !p.d_done[1] || !r.llr || !r.hard_bits || !r.iters || !r.synd_ok)
            return fail(NDGSBP_ERR_CUDA, "server_create: cannot map host buffers into the device");
        if (p.qc) {
            QcArgs& q = p.qargs;
            q = p.qp.args;
            q.r = r;
            q.r.counter = h->d_counter + 1 + i;
            q.serve_list = device_view(p.h_list);
            q.state_flag = p.flag;
            q.state_iter = p.st_iter;
            q.state_P = p.st_P;
            q.state_msgs = p.st_msgs;
            q.epoch_iters = epoch_iters;
            q.done_list = C.done_list;
            q.done_count = C.done_count;
            if (!q.serve_list) return fail(NDGSBP_ERR_CUDA, "server_create: cannot map host buffers into the device");
        }
        if (p.stream) {
            StreamArgs& a = p.sargs;
            a = p.sp.args;
            a.r = r;
            a.r.counter = h->d_counter + 1 + i;
            a.ws_msgs = nullptr;
            a.status = nullptr;
            a.serve_list = device_view(p.h_list);
            a.state_flag = p.flag;
            a.state_iter = p.st_iter;
            a.state_P = p.st_P;
            a.state_msgs = p.st_msgs;
            a.epoch_iters = epoch_iters;
            a.done_list = C.done_list;
            a.done_count = C.done_count;
            if (!a.serve_list) return fail(NDGSBP_ERR_CUDA, "server_create: cannot map host buffers into the device");
        }
    }
    h->args.n_codes = n_codes;
    h->args.tiles = h->d_tiles;
    h->args.n_tiles = 0;
    h->args.tile_counter = h->d_counter;
    h->args.table_bytes = static_cast<int>(table_max);
    h->fn = fn;
    h->threads = threads;
    h->smem = smem;
    h->max_grid = std::max(1, per_sm * sms);
    ndgsbp_server* raw = h.release();
    raw->worker = std::thread([raw] { raw->run(); });
    for (int k = 0; k < kStagers; ++k) raw->stagers.emplace_back([raw] { raw->stage(); });
    *out = raw;
    return NDGSBP_OK;
}

ndgsbp_status ndgsbp_server_submit(ndgsbp_server* s, int32_t code, const float* host_llr, int64_t n_frames,
                                   uint32_t* host_hard_bits, int32_t* host_iters, uint8_t* host_syndrome_ok,
                                   int64_t* ticket) {
    clear_error();
    if (!s || !ticket || code < 0 || code >= static_cast<int32_t>(s->pools.size()) || n_frames < 1 || !host_llr ||
        !host_hard_bits)
        return fail(NDGSBP_ERR_INVALID, "server_submit: bad arguments");
    auto r = std::make_unique<Request>();
    r->code = code;
    r->n_frames = n_frames;
    r->llr = host_llr;
    r->hard = host_hard_bits;
    r->iters = host_iters;
    r->ok = host_syndrome_ok;
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (s->failed) return fail(s->failed, "server stopped: %s", s->failure.c_str());
        r->ticket = s->next_ticket++;
        *ticket = r->ticket;
        s->queue.push_back(r.get());
        s->reqs.emplace(r->ticket, std::move(r));
        s->stats.requests_submitted += 1;
    }
    s->cv_stage.notify_one();
    return NDGSBP_OK;
}

ndgsbp_status ndgsbp_server_poll(ndgsbp_server* s, int64_t ticket, int32_t* done, double* latency_ms) {
    if (!s) return fail(NDGSBP_ERR_INVALID, "server_poll: null server");
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return fail(NDGSBP_ERR_INVALID, "server_poll: unknown ticket %lld", static_cast<long long>(ticket));
    if (s->failed) return fail(s->failed, "server stopped: %s", s->failure.c_str());
    const bool fin = it->second->done;
    if (done) *done = fin ? 1 : 0;
    if (latency_ms && fin)
        *latency_ms = std::chrono::duration<double, std::milli>(it->second->t_done - it->second->t_submit).count();
    if (fin) s->reqs.erase(it);   // reported once: the ticket is released
    return NDGSBP_OK;
}

ndgsbp_status ndgsbp_server_wait(ndgsbp_server* s, int64_t ticket, int32_t timeout_ms, double* latency_ms) {
    if (!s) return fail(NDGSBP_ERR_INVALID, "server_wait: null server");
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return fail(NDGSBP_ERR_INVALID, "server_wait: unknown ticket %lld", static_cast<long long>(ticket));
    Request* r = it->second.get();
    const bool ok = s->cv_done.wait_for(lock, std::chrono::milliseconds(std::max(0, timeout_ms)),
                                        [&] { return r->done || s->failed; });
    if (s->failed) return fail(s->failed, "server stopped: %s", s->failure.c_str());
    if (!ok) return fail(NDGSBP_ERR_TIMEOUT, "server_wait: request %lld not done after %d ms",
                         static_cast<long long>(ticket), timeout_ms);
    if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
    s->reqs.erase(it);   // reported once: the ticket is released
    return NDGSBP_OK;
}

ndgsbp_status ndgsbp_server_stats_get(ndgsbp_server* s, ndgsbp_server_stats* out) {
    if (!s || !out) return fail(NDGSBP_ERR_INVALID, "server_stats: null pointer");
    std::lock_guard<std::mutex> lock(s->mu);
    *out = s->stats;
    out->slots_in_use = s->in_flight;
    return NDGSBP_OK;
}

ndgsbp_status ndgsbp_server_destroy(ndgsbp_server* s) {
    delete s;
    return NDGSBP_OK;
}

}  // extern "C"
