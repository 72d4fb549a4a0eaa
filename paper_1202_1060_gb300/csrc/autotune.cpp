// Autotuner: times candidate launch shapes of a decode on a sample of the caller's frames and
// keeps the fastest.  Every candidate is an ordinary ndgsbp_decode call (or, for ragged
// batches, an ordinary ragged launch), so a tuned shape computes exactly what the default does.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "ndgsbp_internal.h"

using namespace ndgsbp;

namespace {

std::mutex g_cache_mu;
std::map<std::string, std::pair<ndgsbp_params, double>> g_cache;   // key -> best params, ms
std::map<std::string, bool> g_loaded_files;

uint64_t fnv1a(uint64_t h, const void* p, size_t n) {
    const unsigned char* b = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) {
        h ^= b[i];
        h *= 1099511628211ull;
    }
    return h;
}

template <typename T>
uint64_t fnv_vec(uint64_t h, const std::vector<T>& v) {
    return fnv1a(h, v.data(), v.size() * sizeof(T));
}

// Content key: the code, its grouping, the parameters that change the work, the sample size
// class and the device.
std::string tune_key(const Groups& g, const ndgsbp_params& p, int llr_dtype, int64_t n_frames, int flags) {
    uint64_t h = 14695981039346656037ull;
    h = fnv_vec(h, g.code->row_ptr);
    h = fnv_vec(h, g.code->col_idx);
    h = fnv_vec(h, g.grp_ptr);
    h = fnv_vec(h, g.grp_cn);
    const int32_t f[] = {p.schedule, p.max_iter, p.msg_dtype, p.early_stop, p.block_threads, llr_dtype, flags};
    h = fnv1a(h, f, sizeof(f));
    h = fnv1a(h, &p.llr_max, sizeof(p.llr_max));
    int dev = 0, sms = 0;
    cudaDeviceProp prop{};
    if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&prop, dev) == cudaSuccess) {
        h = fnv1a(h, prop.name, std::strlen(prop.name));
        sms = prop.multiProcessorCount;
    }
    int bucket = 0;
    while ((int64_t{1} << (bucket + 1)) <= n_frames) ++bucket;
    char buf[96];
    std::snprintf(buf, sizeof(buf), "%016llx-sm%d-f%d", static_cast<unsigned long long>(h), sms, bucket);
    return buf;
}

// Cache file: one line per key, "key variant block_threads ctas_per_sm frames_per_cta lanes_per_cn ms".
void load_cache_file(const char* path) {
    if (!path || !*path || g_loaded_files.count(path)) return;
    g_loaded_files[path] = true;
    std::ifstream in(path);
    std::string line;
    while (std::getline(in, line)) {
        std::istringstream ss(line);
        std::string key;
        ndgsbp_params p{};
        double ms = 0.0;
        if (ss >> key >> p.variant >> p.block_threads >> p.ctas_per_sm >> p.frames_per_cta >> p.lanes_per_cn >> ms)
            g_cache[key] = {p, ms};
    }
}

void append_cache_file(const char* path, const std::string& key, const ndgsbp_params& p, double ms) {
    if (!path || !*path) return;
    std::ofstream out(path, std::ios::app);
    out << key << ' ' << p.variant << ' ' << p.block_threads << ' ' << p.ctas_per_sm << ' ' << p.frames_per_cta << ' '
        << p.lanes_per_cn << ' ' << ms << '\n';
}

struct Scratch {
    void* ws = nullptr;
    size_t ws_bytes = 0;
    uint32_t* hard = nullptr;
    int32_t* iters = nullptr;
    uint8_t* ok = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ~Scratch() {
        cudaFree(ws);
        cudaFree(hard);
        cudaFree(iters);
        cudaFree(ok);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (stream) cudaStreamDestroy(stream);
    }
};

// Median of `reps` timed decodes after one untimed one; negative on failure.
double time_decode(const ndgsbp_groups* groups, const ndgsbp_params& p, const void* d_llr, int llr_dtype,
                   int64_t n_frames, Scratch& s, int reps) {
    std::vector<float> t;
    for (int i = 0; i <= reps; ++i) {
        if (cudaEventRecord(s.e0, s.stream) != cudaSuccess) return -1.0;
        if (ndgsbp_decode(groups, &p, d_llr, llr_dtype, n_frames, s.ws, s.ws_bytes, s.hard, s.iters, s.ok, nullptr,
                          s.stream) != NDGSBP_OK)
            return -1.0;
        if (cudaEventRecord(s.e1, s.stream) != cudaSuccess || cudaEventSynchronize(s.e1) != cudaSuccess) return -1.0;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, s.e0, s.e1);
        if (i > 0) t.push_back(ms);
    }
    std::sort(t.begin(), t.end());
    return t[t.size() / 2];
}

}  // namespace

extern "C" {

ndgsbp_status ndgsbp_autotune(const ndgsbp_groups* groups, const ndgsbp_params* params, const void* d_llr,
                              int32_t llr_dtype, int64_t n_frames, int32_t flags, const char* cache_path,
                              ndgsbp_tune_result* out) {
    clear_error();
    if (!groups || !params || !d_llr || !out || n_frames < 1)
        return fail(NDGSBP_ERR_INVALID, "autotune: groups, params, d_llr, out and n_frames >= 1 are required");
    const Groups& g = groups->g;
    const bool tile_only = flags & NDGSBP_TUNE_TILE_ONLY;
    const std::string key = tune_key(g, *params, llr_dtype, n_frames, flags);
    std::memset(out, 0, sizeof(*out));
    {
        std::lock_guard<std::mutex> lock(g_cache_mu);
        load_cache_file(cache_path);
        auto it = g_cache.find(key);
        if (it != g_cache.end()) {
            out->best = *params;
            out->best.variant = it->second.first.variant;
            out->best.block_threads = it->second.first.block_threads;
            out->best.ctas_per_sm = it->second.first.ctas_per_sm;
            out->best.frames_per_cta = it->second.first.frames_per_cta;
            out->best.lanes_per_cn = it->second.first.lanes_per_cn;
            out->best_ms = it->second.second;
            out->from_cache = 1;
            return NDGSBP_OK;
        }
    }
    // candidates: the library's choice, the QC kernels, and tile shapes
    std::vector<ndgsbp_params> cand;
    auto add = [&](int variant, int threads, int cps, int fpc, int lanes) {
        ndgsbp_params p = *params;
        p.variant = variant;
        if (!(tile_only && params->block_threads)) p.block_threads = threads;
        p.ctas_per_sm = cps;
        p.frames_per_cta = fpc;
        p.lanes_per_cn = lanes;
        ndgsbp_plan plan;
        if (ndgsbp_decode_plan(groups, &p, n_frames, &plan) == NDGSBP_OK) cand.push_back(p);
        clear_error();
    };
    if (!tile_only) {
        add(NDGSBP_VARIANT_AUTO, params->block_threads, params->ctas_per_sm, 0, 0);
        for (int cps : {0, 1, 2}) add(NDGSBP_VARIANT_QC, 0, cps, 0, 0);
        for (int cps : {0, 2, 3, 4}) add(NDGSBP_VARIANT_QC_GLOBAL, 0, cps, 0, 0);
        for (int v : {NDGSBP_VARIANT_STREAM_SMEM, NDGSBP_VARIANT_STREAM_GLOBAL, NDGSBP_VARIANT_STREAM_BULK})
            for (int lanes : {0, 2}) add(v, 0, 0, 0, lanes);
    }
    const int maxdeg = g.qc.ok ? g.qc.max_deg : 0;
    const int threads_list[] = {128, 256, 384, 512};
    for (int lanes : {1, 2, 4}) {
        if (!maxdeg || (maxdeg + lanes - 1) / lanes > 8) continue;
        if (lanes > 1 && (maxdeg + lanes / 2 - 1) / (lanes / 2) <= 2) continue;   // idle lanes only
        for (int fpc : {1, 2, 4, 8, 16})
            for (int t : threads_list) {
                if (tile_only && params->block_threads && t != threads_list[0]) continue;
                add(NDGSBP_VARIANT_TILE, t, params->ctas_per_sm, fpc, lanes);
                // one CTA per SM with the whole SM's shared memory (messages on chip when they fit)
                if (!tile_only && !params->ctas_per_sm) add(NDGSBP_VARIANT_TILE, t, 1, fpc, lanes);
            }
    }
    if (cand.empty()) return fail(NDGSBP_ERR_UNSUPPORTED, "autotune: no launch shape fits this grouping");
    // scratch sized for the largest candidate
    Scratch s;
    size_t ws = 0;
    for (const auto& p : cand) {
        size_t b = 0;
        if (ndgsbp_workspace_size(groups, &p, n_frames, &b) == NDGSBP_OK) ws = std::max(ws, b);
    }
    clear_error();
    const int N = g.code->N, W = (N + 31) / 32;
    cudaError_t e = cudaSuccess;
    s.ws_bytes = std::max<size_t>(ws, 256);
    if (e == cudaSuccess) e = cudaMalloc(&s.ws, s.ws_bytes);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&s.hard), sizeof(uint32_t) * W * n_frames);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&s.iters), sizeof(int32_t) * n_frames);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&s.ok), n_frames);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&s.e0);
    if (e == cudaSuccess) e = cudaEventCreate(&s.e1);
    if (e != cudaSuccess) return fail(NDGSBP_ERR_NOMEM, "autotune: %s", cudaGetErrorString(e));
    double best = -1.0;
    ndgsbp_params best_p = cand[0];
    for (size_t i = 0; i < cand.size(); ++i) {
        const double ms = time_decode(groups, cand[i], d_llr, llr_dtype, n_frames, s, 3);
        if (ms < 0.0) {
            const ndgsbp_status st = cudaGetLastError() != cudaSuccess ? NDGSBP_ERR_CUDA : NDGSBP_OK;
            if (st) return fail(st, "autotune: a candidate launch failed");
            clear_error();
            continue;
        }
        if (i == 0) out->default_ms = ms;
        if (best < 0.0 || ms < best) {
            best = ms;
            best_p = cand[i];
        }
        ++out->candidates;
    }
    if (best < 0.0) return fail(NDGSBP_ERR_UNSUPPORTED, "autotune: no candidate ran");
    out->best = best_p;
    out->best_ms = best;
    {
        std::lock_guard<std::mutex> lock(g_cache_mu);
        g_cache[key] = {best_p, best};
        append_cache_file(cache_path, key, best_p, best);
    }
    return NDGSBP_OK;
}

ndgsbp_status ndgsbp_ragged_autotune(ndgsbp_batch* batches, int32_t n_batches, const ndgsbp_params* params,
                                     int64_t sample_frames, const char* cache_path, ndgsbp_params* params_out,
                                     double* best_ms) {
    clear_error();
    if (!batches || !params || !params_out || n_batches < 1)
        return fail(NDGSBP_ERR_INVALID, "ragged_autotune: batches, params and params_out are required");
    const std::vector<ndgsbp_batch> orig(batches, batches + n_batches);
    std::vector<ndgsbp_batch> best_b = orig;
    ndgsbp_params best_p = *params;
    double best = -1.0;
    cudaStream_t stream = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    ndgsbp_status st = NDGSBP_OK;
    if (e != cudaSuccess) st = fail(NDGSBP_ERR_CUDA, "ragged_autotune: %s", cudaGetErrorString(e));
    for (int threads : {128, 256, 384, 512}) {
        if (st) break;
        ndgsbp_params p = *params;
        p.variant = NDGSBP_VARIANT_TILE;
        p.block_threads = threads;
        std::vector<ndgsbp_batch> b = orig;
        // per code: the fastest tile shape at this block size, on a sample of its frames
        for (int i = 0; i < n_batches && !st; ++i) {
            if (b[i].n_frames < 1 || !b[i].d_llr) continue;
            ndgsbp_tune_result r;
            const int64_t n = sample_frames > 0 ? std::min(sample_frames, b[i].n_frames) : b[i].n_frames;
            st = ndgsbp_autotune(b[i].groups, &p, b[i].d_llr, b[i].llr_dtype, n, NDGSBP_TUNE_TILE_ONLY, cache_path, &r);
            if (st == NDGSBP_ERR_UNSUPPORTED) {   // this block size does not fit the code
                st = NDGSBP_OK;
                clear_error();
                b.clear();
                break;
            }
            b[i].frames_per_cta = r.best.frames_per_cta;
            b[i].lanes_per_cn = r.best.lanes_per_cn;
        }
        if (st || b.empty()) continue;
        // the whole launch at this block size and each residency target
        for (int k = 1; k <= 4 && !st; ++k) {
            p.ctas_per_sm = k;
            ndgsbp_ragged* rg = nullptr;
            if (ndgsbp_ragged_create(b.data(), n_batches, &p, &rg) != NDGSBP_OK) {
                clear_error();
                continue;
            }
            std::vector<float> t;
            for (int rep = 0; rep < 3 && !st; ++rep) {
                cudaEventRecord(e0, stream);
                st = ndgsbp_ragged_launch(rg, stream);
                cudaEventRecord(e1, stream);
                if (!st && cudaEventSynchronize(e1) != cudaSuccess)
                    st = fail(NDGSBP_ERR_CUDA, "ragged_autotune: launch failed");
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0) t.push_back(ms);
            }
            ndgsbp_ragged_destroy(rg);
            if (st) break;
            const double ms = std::min(t[0], t[1]);
            if (best < 0.0 || ms < best) {
                best = ms;
                best_b = b;
                best_p = p;
            }
        }
    }
    // every code on its own default plan, forked onto concurrent streams
    if (!st) {
        ndgsbp_params p = *params;
        p.variant = NDGSBP_VARIANT_RAGGED_PER_CODE;
        ndgsbp_ragged* rg = nullptr;
        if (ndgsbp_ragged_create(orig.data(), n_batches, &p, &rg) != NDGSBP_OK) {
            clear_error();
        } else {
            std::vector<float> t;
            for (int rep = 0; rep < 3 && !st; ++rep) {
                cudaEventRecord(e0, stream);
                st = ndgsbp_ragged_launch(rg, stream);
                cudaEventRecord(e1, stream);
                if (!st && cudaEventSynchronize(e1) != cudaSuccess)
                    st = fail(NDGSBP_ERR_CUDA, "ragged_autotune: launch failed");
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0) t.push_back(ms);
            }
            ndgsbp_ragged_destroy(rg);
            if (!st) {
                const double ms = std::min(t[0], t[1]);
                if (best < 0.0 || ms < best) {
                    best = ms;
                    best_b = orig;
                    best_p = p;
                }
            }
        }
    }
    if (e1) cudaEventDestroy(e1);
    if (e0) cudaEventDestroy(e0);
    if (stream) cudaStreamDestroy(stream);
    if (st) return st;
    if (best < 0.0) return fail(NDGSBP_ERR_UNSUPPORTED, "ragged_autotune: no block size fits every code");
    for (int i = 0; i < n_batches; ++i) {
        batches[i].frames_per_cta = best_b[i].frames_per_cta;
        batches[i].lanes_per_cn = best_b[i].lanes_per_cn;
    }
    *params_out = best_p;
    if (best_ms) *best_ms = best;
    return NDGSBP_OK;
}

}  // extern "C"
