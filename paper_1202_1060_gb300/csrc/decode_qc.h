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
    const int2* win2;             // [G][2][maxdeg] block columns shared by 2-layer windows, or null
    int n_groupings;              // group -> layer tables cycled by iteration (group_layers holds all)
};

typedef void (*QcKernelFn)(const QcArgs);

// w2: the 2-layer-window instance (direct write-back off shared block columns; needs win2).
// occ6: the instance compiled for 6 resident CTAs of at most qc_occ_threads() threads (16-bit
// messages in shared memory, degree <= 8); nullptr when it does not apply.
QcKernelFn pick_qc_kernel(int msg_dtype, int maxdc, bool msg_smem, bool spec, bool pair, bool w2 = false,
                          bool occ6 = false);
int qc_occ_threads();
// Two frames per thread (decode_qc2.cu); degree-specialised codes with MAXDC 8 or 16 only.
QcKernelFn pick_qc_frames2_kernel(int msg_dtype, int maxdc, bool msg_smem);
int qc_frames2_max_threads(int maxdc);
bool qc_degrees_specialised(const QcLayout& Q, int maxdc);
int qc_pair_max_threads(int maxdc);
// Shared bytes of a launch's tables (w2: with the 2-layer window masks and change buffer).
size_t qc_table_bytes(const QcLayout& Q, bool w2 = false);
void fill_qc_args(QcArgs& a, const QcLayout& Q, const DeviceQc& D, void* ws_msgs, bool w2 = false);

}  // namespace ndgsbp
