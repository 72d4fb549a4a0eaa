// Host side of the NDGSBP library: error reporting, code handles, Step 1 grouping and the
// layout compiler that turns (H, groups) into the edge storage the decode kernels read.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <set>
#include <unordered_set>

#include "ndgsbp_internal.h"

namespace ndgsbp {

static thread_local std::string t_error;

ndgsbp_status fail(ndgsbp_status status, const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    t_error = buf;
    return status;
}

void clear_error() { t_error.clear(); }

// ------------------------------------------------------------------------------------------
// SplitMix64 (Steele, Lea, Flood 2014): the random source of the grouping step.
// ------------------------------------------------------------------------------------------
class SplitMix64 {
  public:
    explicit SplitMix64(uint64_t seed) : state_(seed) {}
    uint64_t next() {
        uint64_t z = (state_ += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }

  private:
    uint64_t state_;
};

// Group sizes from G N_G - (G-1) N_G r = M (Sec. II-A); the integer reading is documented on
// ndgsbp_group_sizes in the public header.
static ndgsbp_status group_sizes(int Mu, int G, double r, int flags, int* NG, int* o,
                                 std::vector<int>* fresh) {
    if (Mu < 1 || G < 1 || G > Mu)
        return fail(NDGSBP_ERR_INVALID, "group count G=%d must be in [1, %d]", G, Mu);
    if (!(r >= 0.0 && r < 1.0)) return fail(NDGSBP_ERR_INVALID, "overlap ratio r=%g not in [0, 1)", r);
    std::vector<int> f(G);
    if (flags & NDGSBP_GROUPS_CYCLIC) {
        if (Mu % G) return fail(NDGSBP_ERR_INFEASIBLE, "cyclic groups: G=%d does not divide %d units", G, Mu);
        const int s = Mu / G;
        *o = static_cast<int>(std::floor(r * s / (1.0 - r) + 0.5 + 1e-9));
        *NG = s + *o;
        if (*NG > Mu) return fail(NDGSBP_ERR_INFEASIBLE, "cyclic window %d exceeds %d units", *NG, Mu);
        std::fill(f.begin(), f.end(), s);
    } else {
        if (G == 1) {
            *NG = Mu;
            *o = 0;
        } else {
            const double x = static_cast<double>(Mu) / (static_cast<double>(G) - (G - 1) * r);
            *NG = std::min(Mu, static_cast<int>(std::ceil(x - 1e-9 * x)));
            *o = static_cast<int>(std::floor(r * (*NG) + 0.5 + 1e-9));
        }
        f[0] = *NG;
        if (G > 1) {
            const int rest = Mu - *NG, share = rest / (G - 1), extra = rest % (G - 1);
            for (int g = 1; g < G; ++g) {
                f[g] = share + (g - 1 < extra ? 1 : 0);
                if (f[g] < 1)
                    return fail(NDGSBP_ERR_INFEASIBLE,
                                "group %d would get no fresh unit (M=%d, G=%d, r=%g)", g + 1, Mu, G, r);
            }
        }
    }
    if (fresh) *fresh = std::move(f);
    return NDGSBP_OK;
}

// Step 1 of Sec. II-C on unit indices.  Draws are forward Fisher-Yates steps over the pool of
// unused units; a group's overlap is the tail of its predecessor.
// Structure-aware Step 1 (the paper's future-work direction of choosing groups for a larger
// CoCSG l, the number of VNs two consecutive groups share): group 1 and every overlap as in
// Step 1; the f_g fresh CNs of group g >= 2 are picked one at a time, each the unused CN that
// adds the most VNs of N(G_{g-1}) not yet in N(G_g) (a greedy for |N(G_g) & N(G_{g-1})|), ties
// going to the earlier CN of the random draw order (the rest of the Fisher-Yates draw).
static void structured_groups(const Code& c, int G, int NG, int o, const std::vector<int>& fresh,
                              const std::vector<int>& pool, std::vector<std::vector<int>>& groups) {
    std::vector<char> used(c.M, 0), in_prev(c.N, 0), covered(c.N, 0);
    groups.assign(G, {});
    groups[0].assign(pool.begin(), pool.begin() + NG);
    for (int m : groups[0]) used[m] = 1;
    for (int g = 1; g < G; ++g) {
        const std::vector<int>& prev = groups[g - 1];
        std::fill(in_prev.begin(), in_prev.end(), 0);
        std::fill(covered.begin(), covered.end(), 0);
        for (int m : prev)
            for (int e = c.row_ptr[m]; e < c.row_ptr[m + 1]; ++e) in_prev[c.col_idx[e]] = 1;
        groups[g].assign(prev.end() - o, prev.end());
        for (int m : groups[g])
            for (int e = c.row_ptr[m]; e < c.row_ptr[m + 1]; ++e) covered[c.col_idx[e]] = 1;
        for (int k = 0; k < fresh[g]; ++k) {
            int best = -1, best_gain = -1;
            for (size_t i = NG; i < pool.size(); ++i) {
                const int m = pool[i];
                if (used[m]) continue;
                int gain = 0;
                for (int e = c.row_ptr[m]; e < c.row_ptr[m + 1]; ++e) {
                    const int v = c.col_idx[e];
                    gain += in_prev[v] && !covered[v];
                }
                if (gain > best_gain) {
                    best_gain = gain;
                    best = static_cast<int>(i);
                }
            }
            const int m = pool[best];
            used[m] = 1;
            groups[g].push_back(m);
            for (int e = c.row_ptr[m]; e < c.row_ptr[m + 1]; ++e) covered[c.col_idx[e]] = 1;
        }
    }
}

static ndgsbp_status draw_unit_groups(int Mu, int G, double r, uint64_t seed, int flags,
                                      std::vector<std::vector<int>>& groups, const Code* structure = nullptr) {
    int NG = 0, o = 0;
    std::vector<int> fresh;
    ndgsbp_status st = group_sizes(Mu, G, r, flags, &NG, &o, &fresh);
    if (st) return st;
    std::vector<int> pool(Mu);
    std::iota(pool.begin(), pool.end(), 0);
    SplitMix64 rng(seed);
    size_t drawn = 0;
    const bool shuffle = !(flags & NDGSBP_GROUPS_NATURAL);
    auto draw = [&](int k) {
        for (int i = 0; i < k; ++i, ++drawn) {
            if (shuffle) {
                const size_t j = drawn + static_cast<size_t>(rng.next() % static_cast<uint64_t>(Mu - drawn));
                std::swap(pool[drawn], pool[j]);
            }
        }
    };
    groups.assign(G, {});
    if (flags & NDGSBP_GROUPS_STRUCTURED) {
        draw(Mu);   // the whole random order: group 1, then the tie-break order
        structured_groups(*structure, G, NG, o, fresh, pool, groups);
        return NDGSBP_OK;
    }
    if (flags & NDGSBP_GROUPS_CYCLIC) {
        draw(Mu);
        const int s = Mu / G;
        for (int g = 0; g < G; ++g)
            for (int j = 0; j < NG; ++j) groups[g].push_back(pool[(static_cast<size_t>(g) * s + j) % Mu]);
    } else {
        draw(NG);
        groups[0].assign(pool.begin(), pool.begin() + NG);
        for (int g = 1; g < G; ++g) {
            const std::vector<int>& prev = groups[g - 1];
            groups[g].assign(prev.end() - o, prev.end());
            const size_t first = drawn;
            draw(fresh[g]);
            groups[g].insert(groups[g].end(), pool.begin() + first, pool.begin() + drawn);
        }
    }
    return NDGSBP_OK;
}

ndgsbp_status draw_groups(int n_units, int G, double r, uint64_t seed, int flags,
                          std::vector<std::vector<int>>& groups) {
    return draw_unit_groups(n_units, G, r, seed, flags & ~NDGSBP_GROUPS_STRUCTURED, groups);
}

// ------------------------------------------------------------------------------------------
// Layout compiler
// ------------------------------------------------------------------------------------------
void compile_layout(const Code& c, const std::vector<int32_t>& gp, const std::vector<int32_t>& gc,
                    Layout& L) {
    const int M = c.M, G = static_cast<int>(gp.size()) - 1;
    L = Layout();
    L.M = M;
    L.N = c.N;
    L.G = G;
    // CN slots in order of first appearance
    std::vector<int32_t> slot_of(M, -1);
    L.slot_cn.reserve(M);
    for (int32_t cn : gc)
        if (slot_of[cn] < 0) { slot_of[cn] = static_cast<int32_t>(L.slot_cn.size()); L.slot_cn.push_back(cn); }
    for (int cn = 0; cn < M; ++cn)
        if (slot_of[cn] < 0) { slot_of[cn] = static_cast<int32_t>(L.slot_cn.size()); L.slot_cn.push_back(cn); }
    L.slot_deg.resize(M);
    for (int s = 0; s < M; ++s) {
        const int cn = L.slot_cn[s];
        L.slot_deg[s] = c.row_ptr[cn + 1] - c.row_ptr[cn];
        L.max_deg = std::max(L.max_deg, L.slot_deg[s]);
    }
    // tiles of 32 slots, padded to the tile's largest degree
    const int T = (M + 31) / 32;
    L.tile_base.assign(T + 1, 0);
    for (int t = 0; t < T; ++t) {
        int D = 0;
        for (int s = 32 * t; s < std::min(M, 32 * t + 32); ++s) D = std::max(D, L.slot_deg[s]);
        L.tile_base[t + 1] = L.tile_base[t] + 32 * D;
    }
    L.Epad = L.tile_base[T];
    L.edge_vn.assign(L.Epad, 0);
    L.edge_csr.assign(L.Epad, -1);
    for (int s = 0; s < M; ++s) {
        const int cn = L.slot_cn[s];
        const int base = L.tile_base[s >> 5] + (s & 31);
        for (int k = 0; k < L.slot_deg[s]; ++k) {
            L.edge_vn[base + 32 * k] = c.col_idx[c.row_ptr[cn] + k];
            L.edge_csr[base + 32 * k] = c.row_ptr[cn] + k;
        }
    }
    // groups: entries, delta positions and VN colours
    L.grp_ptr.assign(gp.begin(), gp.end());
    L.U = gp[G];
    L.ge_slot.resize(L.U);
    L.ge_dpos.resize(L.U);
    L.grp_colbase.resize(G);
    L.grp_ncol.resize(G);
    std::vector<int32_t> occ(c.N, 0);
    std::vector<int32_t> touched;
    for (int g = 0; g < G; ++g) {
        const int b = gp[g], n = gp[g + 1] - gp[g];
        L.max_group_entries = std::max(L.max_group_entries, n);
        const int gt = (n + 31) / 32;
        std::vector<int32_t> gtb(gt + 1, 0);
        for (int j = 0; j < gt; ++j) {
            int D = 0;
            for (int i = 32 * j; i < std::min(n, 32 * j + 32); ++i) D = std::max(D, L.slot_deg[slot_of[gc[b + i]]]);
            gtb[j + 1] = gtb[j] + 32 * D;
        }
        L.max_gd = std::max(L.max_gd, gtb[gt]);
        L.grp_colbase[g] = static_cast<int32_t>(L.gcol.size());
        L.gcol.resize(L.gcol.size() + gtb[gt], 0xFF);
        int ncol = 0;
        for (int i = 0; i < n; ++i) {
            const int s = slot_of[gc[b + i]];
            L.ge_slot[b + i] = s;
            const int dpos = gtb[i >> 5] + (i & 31);
            L.ge_dpos[b + i] = dpos;
            const int cn = L.slot_cn[s];
            for (int k = 0; k < L.slot_deg[s]; ++k) {
                const int v = c.col_idx[c.row_ptr[cn] + k];
                if (occ[v] == 0) touched.push_back(v);
                const int colour = occ[v]++;
                ncol = std::max(ncol, colour + 1);
                L.gcol[L.grp_colbase[g] + dpos + 32 * k] = static_cast<uint8_t>(colour);
            }
            L.edge_updates += L.slot_deg[s];
        }
        for (int v : touched) occ[v] = 0;
        touched.clear();
        L.grp_ncol[g] = ncol;
        L.max_colors = std::max(L.max_colors, ncol);
    }
}

// Layer view of a grouping for the QC kernel: every group must be a list of whole layers
// (each layer's Z CNs consecutive and ascending), all groups the same number of layers.
void compile_qc_layout(const Code& c, const std::vector<int32_t>& gp, const std::vector<int32_t>& gc,
                       QcLayout& Q) {
    Q = QcLayout();
    if (c.Z <= 0 || c.M % c.Z || c.N % c.Z) return;
    const int Z = c.Z, nl = c.M / Z, G = static_cast<int>(gp.size()) - 1;
    Q.Z = Z;
    Q.n_layers = nl;
    Q.nb = c.N / Z;
    // per-layer circulant description, checked against every row of the layer
    Q.layer_deg.resize(nl);
    for (int l = 0; l < nl; ++l) {
        const int r0 = l * Z;
        const int d = c.row_ptr[r0 + 1] - c.row_ptr[r0];
        Q.layer_deg[l] = d;
        Q.max_deg = std::max(Q.max_deg, d);
    }
    Q.edge_tab.assign(static_cast<size_t>(nl) * Q.max_deg * 2, 0);
    Q.layer_off.assign(nl, 0);
    Q.layer_stride.assign(nl, 0);
    std::vector<std::vector<std::pair<int, int>>> circ(nl);
    for (int l = 0; l < nl; ++l) {
        const int r0 = l * Z, d = Q.layer_deg[l];
        std::vector<std::pair<int, int>> bs;
        for (int k = 0; k < d; ++k) {
            const int v = c.col_idx[c.row_ptr[r0] + k];
            bs.push_back({v / Z, v % Z});
        }
        std::sort(bs.begin(), bs.end());
        for (int k = 1; k < d; ++k)
            if (bs[k].first == bs[k - 1].first) return;   // two circulants in one base entry
        for (int cc = 0; cc < Z; ++cc) {
            const int row = r0 + cc;
            if (c.row_ptr[row + 1] - c.row_ptr[row] != d) return;
            std::vector<int> want;
            for (auto& e : bs) want.push_back(e.first * Z + (cc + e.second) % Z);
            std::sort(want.begin(), want.end());
            for (int k = 0; k < d; ++k)
                if (c.col_idx[c.row_ptr[row] + k] != want[k]) return;
        }
        circ[l] = bs;
    }
    // messages of CN c of layer l at layer_off[l] + c S_l + k with an odd stride S_l >= d_l:
    // 32 consecutive CNs then touch 32 distinct banks, and k is a compile-time offset
    int off = 0;
    for (int l = 0; l < nl; ++l) {
        const int d = Q.layer_deg[l];
        Q.layer_stride[l] = d | 1;
        Q.layer_off[l] = off;
        off += Q.layer_stride[l] * Z;
    }
    Q.msg_slots = off;
    Q.csr_of.assign(off, -1);
    for (int l = 0; l < nl; ++l) {
        const int r0 = l * Z, d = Q.layer_deg[l];
        const auto& bs = circ[l];
        // edges ordered by block column = by VN index within every row, i.e. CSR order
        for (int k = 0; k < d; ++k) {
            Q.edge_tab[(static_cast<size_t>(l) * Q.max_deg + k) * 2] = 4 * (bs[k].first * Z + bs[k].second);
            Q.edge_tab[(static_cast<size_t>(l) * Q.max_deg + k) * 2 + 1] = Z - bs[k].second;
            for (int cc = 0; cc < Z; ++cc)
                Q.csr_of[Q.layer_off[l] + cc * Q.layer_stride[l] + k] = c.row_ptr[r0 + cc] + k;
        }
    }
    // groups as lists of whole layers
    int window = -1;
    for (int g = 0; g < G; ++g) {
        const int b = gp[g], n = gp[g + 1] - gp[g];
        if (n % Z) return;
        if (window < 0) window = n / Z;
        if (n / Z != window) return;
        for (int j = 0; j < window; ++j) {
            const int first = gc[b + j * Z];
            if (first % Z) return;
            for (int cc = 0; cc < Z; ++cc)
                if (gc[b + j * Z + cc] != first + cc) return;
            Q.group_layers.push_back(first / Z);
        }
    }
    if (window < 1 || window > 1024 / 32) return;   // at most 32 layers per group for the kernel
    Q.window = window;
    Q.ok = true;
}

const Layout& flood_layout(const Groups& g) {
    std::lock_guard<std::mutex> lock(g.mu);
    if (!g.flood) {
        std::vector<int32_t> gp = {0, g.code->M};
        std::vector<int32_t> gc(g.code->M);
        std::iota(gc.begin(), gc.end(), 0);
        auto L = std::make_unique<Layout>();
        compile_layout(*g.code, gp, gc, *L);
        compile_qc_layout(*g.code, gp, gc, g.flood_qc);
        g.flood = std::move(L);
    }
    return *g.flood;
}

const QcLayout& flood_qc_layout(const Groups& g) {
    flood_layout(g);
    return g.flood_qc;
}

static double compute_cocsg(const Code& c, const std::vector<int32_t>& gp, const std::vector<int32_t>& gc) {
    const int G = static_cast<int>(gp.size()) - 1;
    if (G < 2) return 0.0;
    std::vector<int32_t> mark(c.N, -1);
    double sum = 0.0;
    std::vector<std::vector<int32_t>> vsets(G);
    for (int g = 0; g < G; ++g) {
        std::unordered_set<int32_t> s;
        for (int i = gp[g]; i < gp[g + 1]; ++i) {
            const int m = gc[i];
            for (int e = c.row_ptr[m]; e < c.row_ptr[m + 1]; ++e) s.insert(c.col_idx[e]);
        }
        vsets[g].assign(s.begin(), s.end());
    }
    for (int g = 1; g < G; ++g) {
        for (int32_t v : vsets[g - 1]) mark[v] = g;
        int both = 0;
        for (int32_t v : vsets[g]) both += (mark[v] == g);
        sum += both;
    }
    return sum / (G - 1);
}

static ndgsbp_status finish_groups(std::shared_ptr<const Code> code, std::vector<int32_t> gp,
                                   std::vector<int32_t> gc, ndgsbp_groups** out) {
    auto* h = new (std::nothrow) ndgsbp_groups;
    if (!h) return fail(NDGSBP_ERR_NOMEM, "out of host memory");
    Groups& g = h->g;
    g.code = std::move(code);
    g.G = static_cast<int>(gp.size()) - 1;
    g.grp_ptr = std::move(gp);
    g.grp_cn = std::move(gc);
    try {
        compile_layout(*g.code, g.grp_ptr, g.grp_cn, g.grouped);
        compile_qc_layout(*g.code, g.grp_ptr, g.grp_cn, g.qc);
    } catch (const std::bad_alloc&) {
        delete h;
        return fail(NDGSBP_ERR_NOMEM, "out of host memory");
    }
    g.cn_updates = g.grouped.U;
    g.edge_updates = g.grouped.edge_updates;
    g.cocsg = compute_cocsg(*g.code, g.grp_ptr, g.grp_cn);
    *out = h;
    return NDGSBP_OK;
}

}  // namespace ndgsbp

using namespace ndgsbp;

extern "C" {

void ndgsbp_params_default(ndgsbp_params* p) {
    if (!p) return;
    p->schedule = NDGSBP_SCHEDULE_GROUPS;
    p->max_iter = 50;
    p->msg_dtype = NDGSBP_F32;
    p->llr_max = 20.0f;
    p->early_stop = 1;
    p->variant = NDGSBP_VARIANT_AUTO;
    p->block_threads = 0;
    p->ctas_per_sm = 0;
    p->frames_per_cta = 0;
    p->lanes_per_cn = 0;
}

const char* ndgsbp_last_error(void) { return t_error.c_str(); }

const char* ndgsbp_version(void) { return "ndgsbp 1.0 sm_103a"; }

ndgsbp_status ndgsbp_code_create(const int32_t* row_ptr, const int32_t* col_idx, int32_t M,
                                 int32_t N, int32_t lift_Z, ndgsbp_code** out) {
    clear_error();
    if (!row_ptr || !out || M < 1 || N < 1) return fail(NDGSBP_ERR_INVALID, "code_create: null pointer or empty H");
    if (row_ptr[0] != 0) return fail(NDGSBP_ERR_INVALID, "code_create: row_ptr[0] must be 0");
    for (int m = 0; m < M; ++m)
        if (row_ptr[m + 1] < row_ptr[m]) return fail(NDGSBP_ERR_INVALID, "code_create: row_ptr decreases at row %d", m);
    const int64_t E = row_ptr[M];
    if (E > 0 && !col_idx) return fail(NDGSBP_ERR_INVALID, "code_create: col_idx is null");
    auto c = std::make_shared<Code>();
    c->M = M;
    c->N = N;
    c->Z = lift_Z;
    c->E = E;
    c->row_ptr.assign(row_ptr, row_ptr + M + 1);
    c->col_idx.assign(col_idx, col_idx + E);
    std::vector<int32_t> coldeg(N, 0);
    for (int m = 0; m < M; ++m) {
        std::vector<int32_t> r(c->col_idx.begin() + row_ptr[m], c->col_idx.begin() + row_ptr[m + 1]);
        for (int32_t v : r)
            if (v < 0 || v >= N) return fail(NDGSBP_ERR_INVALID, "code_create: column %d out of range in row %d", v, m);
        std::sort(r.begin(), r.end());
        for (size_t k = 1; k < r.size(); ++k)
            if (r[k] == r[k - 1]) return fail(NDGSBP_ERR_INVALID, "code_create: column %d repeated in row %d", r[k], m);
        std::copy(r.begin(), r.end(), c->col_idx.begin() + row_ptr[m]);
        c->max_row = std::max<int>(c->max_row, static_cast<int>(r.size()));
        for (int32_t v : r) coldeg[v]++;
    }
    for (int n = 0; n < N; ++n) c->max_col = std::max(c->max_col, coldeg[n]);
    if (lift_Z < 0) return fail(NDGSBP_ERR_INVALID, "code_create: lift_Z must be >= 0");
    if (lift_Z > 0) {
        if (M % lift_Z) return fail(NDGSBP_ERR_INVALID, "code_create: M=%d is not a multiple of lift_Z=%d", M, lift_Z);
        std::vector<int32_t> seen(N, -1);
        for (int l = 0; l < M / lift_Z; ++l)
            for (int m = l * lift_Z; m < (l + 1) * lift_Z; ++m)
                for (int e = row_ptr[m]; e < row_ptr[m + 1]; ++e) {
                    const int v = c->col_idx[e];
                    if (seen[v] == l) return fail(NDGSBP_ERR_INVALID, "code_create: VN %d appears twice in layer %d", v, l);
                    seen[v] = l;
                }
    }
    auto* h = new (std::nothrow) ndgsbp_code;
    if (!h) return fail(NDGSBP_ERR_NOMEM, "out of host memory");
    h->c = std::move(c);
    *out = h;
    return NDGSBP_OK;
}

ndgsbp_status ndgsbp_code_destroy(ndgsbp_code* code) {
    delete code;
    return NDGSBP_OK;
}

ndgsbp_status ndgsbp_code_info(const ndgsbp_code* code, int32_t* M, int32_t* N, int64_t* E,
                               int32_t* max_row_degree, int32_t* max_col_degree, int32_t* lift_Z) {
    if (!code) return fail(NDGSBP_ERR_INVALID, "code_info: null handle");
    const Code& c = *code->c;
    if (M) *M = c.M;
    if (N) *N = c.N;
    if (E) *E = c.E;
    if (max_row_degree) *max_row_degree = c.max_row;
    if (max_col_degree) *max_col_degree = c.max_col;
    if (lift_Z) *lift_Z = c.Z;
    return NDGSBP_OK;
}

ndgsbp_status ndgsbp_group_sizes(int32_t M_units, int32_t G, double r, int32_t flags, int32_t* NG,
                                 int32_t* overlap) {
    clear_error();
    int ng = 0, o = 0;
    ndgsbp_status st = group_sizes(M_units, G, r, flags, &ng, &o, nullptr);
    if (st) return st;
    if (NG) *NG = ng;
    if (overlap) *overlap = o;
    return NDGSBP_OK;
}

ndgsbp_status ndgsbp_groups_build(const ndgsbp_code* code, int32_t G, double r, uint64_t seed,
                                  int32_t unit, int32_t flags, ndgsbp_groups** out) {
    clear_error();
    if (!code || !out) return fail(NDGSBP_ERR_INVALID, "groups_build: null pointer");
    const Code& c = *code->c;
    int usize = 1;
    if (unit == NDGSBP_UNIT_LAYER) {
        if (c.Z <= 0) return fail(NDGSBP_ERR_INVALID, "groups_build: layer units need a code with lift_Z > 0");
        usize = c.Z;
    } else if (unit != NDGSBP_UNIT_CN) {
        return fail(NDGSBP_ERR_INVALID, "groups_build: unknown unit %d", unit);
    }
    if ((flags & NDGSBP_GROUPS_STRUCTURED) &&
        (unit != NDGSBP_UNIT_CN || (flags & (NDGSBP_GROUPS_CYCLIC | NDGSBP_GROUPS_NATURAL))))
        return fail(NDGSBP_ERR_INVALID, "groups_build: STRUCTURED takes CN units, without CYCLIC or NATURAL");
    std::vector<std::vector<int>> ug;
    ndgsbp_status st = draw_unit_groups(c.M / usize, G, r, seed, flags, ug, &c);
    if (st) return st;
    std::vector<int32_t> gp(1, 0), gc;
    for (auto& grp : ug) {
        for (int u : grp)
            for (int k = 0; k < usize; ++k) gc.push_back(u * usize + k);
        gp.push_back(static_cast<int32_t>(gc.size()));
    }
    return finish_groups(code->c, std::move(gp), std::move(gc), out);
}

ndgsbp_status ndgsbp_groups_build_cycled(const ndgsbp_code* code, int32_t G, double r, uint64_t seed,
                                         int32_t unit, int32_t flags, int32_t n_groupings, ndgsbp_groups** out) {
    clear_error();
    if (!code || !out || n_groupings < 1 || n_groupings > 64)
        return fail(NDGSBP_ERR_INVALID, "groups_build_cycled: need 1..64 groupings");
    ndgsbp_groups* h = nullptr;
    ndgsbp_status st = ndgsbp_groups_build(code, G, r, seed, unit, flags, &h);
    if (st) return st;
    Groups& g = h->g;
    for (int k = 1; k < n_groupings; ++k) {
        ndgsbp_groups* hk = nullptr;
        st = ndgsbp_groups_build(code, G, r, seed + static_cast<uint64_t>(k), unit, flags, &hk);
        if (st) {
            ndgsbp_groups_destroy(h);
            return st;
        }
        const Groups& gk = hk->g;
        // the QC layout takes the further groupings as more group -> layer tables
        if (g.qc.ok && gk.qc.ok && gk.qc.window == g.qc.window &&
            gk.qc.group_layers.size() == static_cast<size_t>(g.G) * g.qc.window) {
            g.qc.group_layers.insert(g.qc.group_layers.end(), gk.qc.group_layers.begin(), gk.qc.group_layers.end());
        } else {
            g.qc.ok = false;
        }
        g.cyc_ptr.push_back(gk.grp_ptr);
        g.cyc_cn.push_back(gk.grp_cn);
        ndgsbp_groups_destroy(hk);
    }
    g.n_groupings = n_groupings;
    g.qc.n_groupings = n_groupings;
    *out = h;
    return NDGSBP_OK;
}

ndgsbp_status ndgsbp_groups_query_grouping(const ndgsbp_groups* groups, int32_t k, int32_t* n_groupings,
                                           int64_t* n_entries, int32_t* grp_ptr, int32_t* cn_idx) {
    if (!groups) return fail(NDGSBP_ERR_INVALID, "groups_query_grouping: null handle");
    const Groups& g = groups->g;
    if (n_groupings) *n_groupings = g.n_groupings;
    if (k < 0 || k >= g.n_groupings) return fail(NDGSBP_ERR_INVALID, "groups_query_grouping: no grouping %d", k);
    const std::vector<int32_t>& gp = k ? g.cyc_ptr[k - 1] : g.grp_ptr;
    const std::vector<int32_t>& gc = k ? g.cyc_cn[k - 1] : g.grp_cn;
    if (n_entries) *n_entries = static_cast<int64_t>(gc.size());
    if (grp_ptr) std::copy(gp.begin(), gp.end(), grp_ptr);
    if (cn_idx) std::copy(gc.begin(), gc.end(), cn_idx);
    return NDGSBP_OK;
}

ndgsbp_status ndgsbp_groups_from_lists(const ndgsbp_code* code, const int32_t* grp_ptr,
                                       const int32_t* cn_idx, int32_t G, ndgsbp_groups** out) {
    clear_error();
    if (!code || !grp_ptr || !out || G < 1) return fail(NDGSBP_ERR_INVALID, "groups_from_lists: bad arguments");
    const Code& c = *code->c;
    if (grp_ptr[0] != 0) return fail(NDGSBP_ERR_INVALID, "groups_from_lists: grp_ptr[0] must be 0");
    std::vector<int32_t> gp(grp_ptr, grp_ptr + G + 1);
    for (int g = 0; g < G; ++g)
        if (gp[g + 1] < gp[g]) return fail(NDGSBP_ERR_INVALID, "groups_from_lists: grp_ptr decreases at %d", g);
    if (gp[G] > 0 && !cn_idx) return fail(NDGSBP_ERR_INVALID, "groups_from_lists: cn_idx is null");
    std::vector<int32_t> gc(cn_idx, cn_idx + gp[G]);
    std::vector<int32_t> last(c.M, -1);
    for (int g = 0; g < G; ++g)
        for (int i = gp[g]; i < gp[g + 1]; ++i) {
            const int m = gc[i];
            if (m < 0 || m >= c.M) return fail(NDGSBP_ERR_INVALID, "groups_from_lists: CN %d out of range", m);
            if (last[m] == g) return fail(NDGSBP_ERR_INVALID, "groups_from_lists: CN %d twice in group %d", m, g);
            last[m] = g;
        }
    return finish_groups(code->c, std::move(gp), std::move(gc), out);
}

ndgsbp_status ndgsbp_groups_query(const ndgsbp_groups* groups, int32_t* G, int64_t* n_entries,
                                  int32_t* grp_ptr, int32_t* cn_idx, double* cocsg,
                                  int64_t* cn_updates_per_iter, int64_t* edge_updates_per_iter) {
    if (!groups) return fail(NDGSBP_ERR_INVALID, "groups_query: null handle");
    const Groups& g = groups->g;
    if (G) *G = g.G;
    if (n_entries) *n_entries = static_cast<int64_t>(g.grp_cn.size());
    if (grp_ptr) std::copy(g.grp_ptr.begin(), g.grp_ptr.end(), grp_ptr);
    if (cn_idx) std::copy(g.grp_cn.begin(), g.grp_cn.end(), cn_idx);
    if (cocsg) *cocsg = g.cocsg;
    if (cn_updates_per_iter) *cn_updates_per_iter = g.cn_updates;
    if (edge_updates_per_iter) *edge_updates_per_iter = g.edge_updates;
    return NDGSBP_OK;
}

ndgsbp_status ndgsbp_groups_destroy(ndgsbp_groups* groups) {
    if (groups) release_device_layouts(groups->g);
    delete groups;
    return NDGSBP_OK;
}

}  // extern "C"
