// Layered QC decode kernel interface (decode_qc.cu), used by the planner in decode.cu.
#pragma once

#include "device_common.cuh"
#include "ndgsbp_internal.h"

namespace ndgsbp {

struct QcArgs {
    RunArgs r;
    int Z, nl, G, window, maxdeg, msg_slots;
    const int2* edge_tab;         // [nl][maxdeg]: (4 (b Z + s), Z - s) of edge k of the layer
    const int32_t* layer_deg;     // [nl]
    const int32_t* layer_stride;  // [nl] messages per CN (odd)
    const int32_t* layer_off;     // [nl] first message of the layer
    const int32_t* group_layers;  // [G][window]
    const int32_t* csr_of;        // [msg_slots] CSR position of each stored message, -1 = padding
    void* ws_msgs;                // per-CTA message slots when messages are not in shared memory
    int n_groupings;              // group -> layer tables cycled by iteration (group_layers holds all)
    // serving instances: frame i of the launch (r.n_frames of them) is pool slot serve_list[i],
    // whose decoding state persists in the pool between launches (as for the tile kernel)
    const int* serve_list;
    int* state_flag;              // [pool] kSlotNew / kSlotRunning / kSlotDone ...
    int* state_iter;              // [pool] iterations done so far
    float* state_P;               // [pool][N] posteriors of running frames
    void* state_msgs;             // [pool][msg_slots] messages of running frames
    int epoch_iters;              // iterations a frame may run in one launch before it is parked
    int* done_list;               // [pool] slots whose frame retired in this launch
    int* done_count;              // entries in done_list (zeroed before the launch)
};

typedef void (*QcKernelFn)(const QcArgs);

// occ6: the instance compiled for 6 resident CTAs of at most qc_occ_threads() threads (16-bit
// messages in shared memory, degree <= 8); nullptr when it does not apply.
QcKernelFn pick_qc_kernel(int msg_dtype, int maxdc, bool msg_smem, bool spec, bool occ6 = false);
int qc_occ_threads();
bool qc_degrees_specialised(const QcLayout& Q, int maxdc);
// Serving instance of the single-CN kernel (decode_qc_serve.cu): degree-specialised codes with
// MAXDC 8 or 16; nullptr otherwise.
QcKernelFn pick_qc_serve_kernel(int msg_dtype, int maxdc, bool msg_smem);
// The serving form of a grouping's QC plan (server pools): the single-CN kernel's serving
// instance with the block, shared bytes and table arguments ndgsbp_decode would use for the
// grouping (variant QC, the library's shape).  *ok = false when that plan does not apply (window
// too large for one CTA, degrees not specialised, MAXDC above 16).
struct QcServePlan {
    QcKernelFn fn = nullptr;
    int threads = 0;
    size_t smem = 0;
    bool msg_smem = false;
    int msg_slots = 0;
    QcArgs args{};
};
ndgsbp_status qc_serve_plan(const Groups& g, const ndgsbp_params* p, QcServePlan* out, bool* ok);

// Shared bytes of a launch's tables.
size_t qc_table_bytes(const QcLayout& Q);
void fill_qc_args(QcArgs& a, const QcLayout& Q, const DeviceQc& D, void* ws_msgs);

}  // namespace ndgsbp
