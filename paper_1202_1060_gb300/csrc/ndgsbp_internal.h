// Internal declarations shared by the host code and the CUDA launchers of the library.
#pragma once

#include <cstdint>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime_api.h>

#include "ndgsbp.h"

namespace ndgsbp {

// Record a message for ndgsbp_last_error() on this thread and return `status`.
ndgsbp_status fail(ndgsbp_status status, const char* fmt, ...);
void clear_error();

struct Code {
    int M = 0, N = 0, Z = 0;
    int64_t E = 0;
    int max_row = 0, max_col = 0;
    std::vector<int32_t> row_ptr, col_idx;
};

// Edge storage used by the decode kernels.  CN "slots" are the CNs in order of first
// appearance in the group sequence (then any CN no group holds).  Slots come in tiles of 32;
// tile t stores edge k of slot s at tile_base[t] + 32 k + (s mod 32), with the tile padded to
// its largest degree, so a warp that handles 32 consecutive slots reads 32 consecutive
// messages per edge index.
struct Layout {
    int M = 0, N = 0, G = 0;
    int Epad = 0;            // stored edge slots per frame (with tile padding)
    int max_deg = 0;         // largest CN degree
    int max_gd = 0;          // largest per-group delta buffer (entries in tiles of 32)
    int max_group_entries = 0;
    int max_colors = 0;      // largest VN multiplicity inside one group
    int64_t U = 0;           // group entries per iteration (CN updates)
    int64_t edge_updates = 0;
    std::vector<int32_t> slot_deg;    // [M]
    std::vector<int32_t> slot_cn;     // [M] CN index of each slot
    std::vector<int32_t> tile_base;   // [ceil(M/32) + 1]
    std::vector<int32_t> edge_vn;     // [Epad] VN of each stored edge (0 in padding)
    std::vector<int32_t> edge_csr;    // [Epad] CSR position of each stored edge (-1 in padding)
    std::vector<int32_t> grp_ptr;     // [G+1] into the entry arrays
    std::vector<int32_t> ge_slot;     // [U] slot of each group entry
    std::vector<int32_t> ge_dpos;     // [U] delta-buffer position of edge 0 of the entry (stride 32)
    std::vector<int32_t> grp_colbase; // [G] offset of the group's colour bytes in gcol
    std::vector<int32_t> grp_ncol;    // [G] number of colours of the group
    std::vector<uint8_t> gcol;        // colour of each group edge, laid out like the delta buffer
};

// Device copy of a Layout: one allocation, arrays at fixed offsets.
struct DeviceLayout {
    void* blob = nullptr;
    size_t bytes = 0;
    const int32_t* slot_deg = nullptr;
    const int32_t* tile_base = nullptr;
    const int32_t* edge_vn = nullptr;
    const int32_t* edge_csr = nullptr;
    const int32_t* grp_ptr = nullptr;
    const int32_t* ge_slot = nullptr;
    const int32_t* ge_dpos = nullptr;
    const int32_t* grp_colbase = nullptr;
    const int32_t* grp_ncol = nullptr;
    const uint8_t* gcol = nullptr;
};

// Layered QC description used by the QC kernel: groups are windows of whole layers.
struct QcLayout {
    bool ok = false;          // the grouping is made of whole layers and the code is QC
    int Z = 0, n_layers = 0, nb = 0;
    int window = 0;           // layers per group (all groups the same size)
    int max_deg = 0;
    int msg_slots = 0;                  // stored messages per frame (with stride padding)
    std::vector<int32_t> layer_deg;     // [n_layers]
    std::vector<int32_t> layer_stride;  // [n_layers] messages per CN: the degree rounded up to odd
    std::vector<int32_t> layer_off;     // [n_layers] first stored message of the layer
    std::vector<int32_t> edge_tab;      // [n_layers][max_deg][2]: (4 (b Z + s), Z - s), edges by block column
    int n_groupings = 1;                // groupings cycled by iteration (all with this window)
    std::vector<int32_t> group_layers;  // [n_groupings][G][window] layer ids in group order
    std::vector<int32_t> csr_of;        // [msg_slots] CSR position of message layer_off[l] + c S_l + k, -1 = pad
};

// Device copy of a QcLayout.
struct DeviceQc {
    void* blob = nullptr;
    const int32_t* edge_tab = nullptr;
    const int32_t* layer_deg = nullptr;
    const int32_t* layer_stride = nullptr;
    const int32_t* layer_off = nullptr;
    const int32_t* group_layers = nullptr;
    const int32_t* csr_of = nullptr;
    // stream kernel tables (see StreamLayout in decode.cu)
    const int32_t* first_use = nullptr;
    const int32_t* layer_csr = nullptr;
    const int32_t* ring = nullptr;
};

struct Groups {
    std::shared_ptr<const Code> code;
    int G = 0;
    std::vector<int32_t> grp_ptr, grp_cn;
    // further groupings cycled by iteration (iteration l uses grouping (l - 1) mod n_groupings;
    // grouping 0 is grp_ptr / grp_cn)
    int n_groupings = 1;
    std::vector<std::vector<int32_t>> cyc_ptr, cyc_cn;
    double cocsg = 0.0;
    int64_t cn_updates = 0, edge_updates = 0;
    Layout grouped;
    QcLayout qc;
    mutable std::mutex mu;
    mutable std::unique_ptr<Layout> flood;        // built on first FLOOD use
    mutable QcLayout flood_qc;
    mutable std::map<int, DeviceLayout> dev_grouped, dev_flood;   // per CUDA device
    mutable std::map<int, DeviceQc> dev_qc, dev_flood_qc;
    ~Groups();
};

void compile_layout(const Code& code, const std::vector<int32_t>& grp_ptr,
                    const std::vector<int32_t>& grp_cn, Layout& out);
void compile_qc_layout(const Code& code, const std::vector<int32_t>& grp_ptr,
                       const std::vector<int32_t>& grp_cn, QcLayout& out);
const Layout& flood_layout(const Groups& g);
const QcLayout& flood_qc_layout(const Groups& g);
void release_device_layouts(Groups& g);   // frees device copies (defined in the CUDA file)

// Step 1 over n_units units (the draw of ndgsbp_groups_build, without the structured option):
// groups[g] lists group g's units.  Used for CN groups and for the VN groups of the vertical
// schedule.
ndgsbp_status draw_groups(int n_units, int G, double r, uint64_t seed, int flags,
                          std::vector<std::vector<int>>& groups);

// The clip limit llr_max (natural LLR units) in the kernels' log2 units (LLR times log2 e).
inline float kernel_llr_limit(float llr_max) { return llr_max * 1.4426950408889634f; }

// A decode plan kept across launches (ragged launches in the per-code mode): what
// ndgsbp_decode plans for (groups, params, n_frames), with the grouping's tables on the device.
struct Plan;
Plan* plan_create(const Groups& g, const ndgsbp_params* p, int64_t n_frames, ndgsbp_status* st);
void plan_destroy(Plan* plan);
const ndgsbp_plan& plan_info(const Plan& plan);
// Enqueue the plan's decode on stream s with ws (plan_info(plan).workspace_bytes, 256-aligned)
// as its scratch: the counter reset and the kernel, as ndgsbp_decode_ex does.
ndgsbp_status plan_enqueue(const Groups& g, const Plan& plan, const ndgsbp_params* p, const void* d_llr,
                           int32_t llr_dtype, int64_t n_frames, void* ws, uint32_t* d_hard_bits, int32_t* d_iters,
                           uint8_t* d_syndrome_ok, float* d_posterior, const ndgsbp_extras* extras, cudaStream_t s);

}  // namespace ndgsbp

struct ndgsbp_code {
    std::shared_ptr<const ndgsbp::Code> c;
};

struct ndgsbp_groups {
    ndgsbp::Groups g;
};
