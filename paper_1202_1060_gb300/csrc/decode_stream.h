// Stream decode kernel interface (decode_stream.cu): layered QC codes whose window of W layers
// is too large for one thread per CN of the window (the QC kernel), e.g. n=16200 (Z = 360) and
// n=8192 (Z = 256, degree 22).
#pragma once

#include "decode_tile.h"
#include "device_common.cuh"
#include "ndgsbp_internal.h"

namespace ndgsbp {

// Where a frame's CN->VN messages live.
constexpr int kStreamSmem = 0;     // all of the frame's messages in shared memory
constexpr int kStreamGlobal = 1;   // in the CTA's workspace slot, read and written in place
constexpr int kStreamBulk = 2;     // in the CTA's workspace slot, layer slabs staged in shared memory
                                   // by cp.async.bulk (see decode_stream.cu)

// Largest number of layer slabs a bulk-staged launch keeps in shared memory, and of layers.
constexpr int kStreamMaxSlabs = 8;
constexpr int kStreamMaxLayers = 64;

// Message layout of one layer.  In shared memory (SMEM) and in the slabs of BULK launches the
// messages are CN-major: edge k of CN c at c S + k with S = stream_cn_stride(d) (an odd number of
// 4-byte words for FP32; d for 16-bit messages, an odd number of words whenever d/2 is odd), so
// each thread's messages sit at compile-time offsets and 32 consecutive CNs hit distinct banks.
// In global memory (GLOBAL) they are edge-major: edge k of CN c at k zr + c, coalesced across the
// CNs of a warp.  A layer's block is rounded up to 16 bytes (a bulk copy's granularity).
__host__ __device__ constexpr int stream_cn_stride(int d, int msg_size) { return msg_size == 4 ? (d | 1) : d; }
__host__ __device__ constexpr int stream_layer_elems(int d, int Z, int zr, int msg_size, int mode) {
    return mode == kStreamGlobal ? d * zr : (Z * stream_cn_stride(d, msg_size) * msg_size + 15) / 16 * 16 / msg_size;
}

struct StreamArgs {
    RunArgs r;
    int Z, nl, G, window, maxdeg, n_groupings;
    int tpc;                      // lanes per CN (1 or 2)
    int le;                       // edges per lane, ceil(maxdeg / tpc) (<= the instance's width)
    int zr;                       // global edge-major row stride: Z rounded up to a multiple of 16
    int msg_elems;                // message elements per frame: sum of the layers' blocks
    const int2* edge_tab;         // [nl][maxdeg]: (4 (b Z + s), Z - s) of edge k of the layer
    const int32_t* layer_deg;     // [nl]
    const int32_t* group_layers;  // [n_groupings][G][window]
    const int32_t* first_use;     // [G][window] 1: grouping 0's group g is the first to use that
                                  // layer (iteration 1 reads no messages there: they are 0)
    const int32_t* layer_csr;     // [nl] CSR position of the layer's first edge, -1 for a layer no
                                  // group holds (its messages stay 0)
    void* ws_msgs;                // [grid][ws_stride] message slots (GLOBAL and BULK)
    int ws_stride;                // elements between CTAs' slots (msg_elems rounded up to 256 bytes)
    unsigned* status;             // workspace word: bit 0 set when a bounded wait gave up (BULK)
    // BULK only: group g of an iteration holds ring positions g .. g + window - 1 (mod nl)
    const int32_t* ring;          // [nl] layer at each ring position
    int n_slabs;                  // window + 2 slab buffers in shared memory
    int slab_elems;               // elements per slab buffer (the largest layer block)
    unsigned wait_limit;          // polls before a bounded wait gives up
    int test_skip_load;           // test hook: 1 = arm the first load's barrier but issue no copy
    int lbase[kStreamMaxLayers];  // first message element of each layer's block (stream_layer_elems)
    // serving instances: frame i of the launch (r.n_frames of them) is pool slot serve_list[i],
    // whose decoding state persists in the pool between launches (as for the QC kernel)
    const int* serve_list;
    int* state_flag;              // [pool] kSlotNew / kSlotRunning / kSlotDone ...
    int* state_iter;              // [pool] iterations done so far
    float* state_P;               // [pool][N] posteriors of running frames
    void* state_msgs;             // [pool][ws_stride] messages of running frames (the launch's layout)
    int epoch_iters;              // iterations a frame may run in one launch before it is parked
    int* done_list;               // [pool] slots whose frame retired in this launch
    int* done_count;              // entries in done_list (zeroed before the launch)
};

typedef void (*StreamKernelFn)(const StreamArgs);

// Kernel instance for `le` edges per lane (a compiled width >= the code's: stream_lane_width),
// lanes per CN (1 or 2) and message storage mode; nullptr when no instance exists.
StreamKernelFn pick_stream_kernel(int msg_dtype, int le, int tpc, int mode);
// Compiled edges-per-lane width for le edges per lane at tpc lanes per CN (0 when none).
int stream_lane_width(int le, int tpc);
// Largest block of an instance at tpc lanes per CN (instances are compiled for 2 CTAs per SM).
int stream_max_threads(int tpc);
// Dynamic shared memory of a launch (a filled in; msg_size 2 or 4 bytes).
size_t stream_smem_bytes(const StreamArgs& a, int msg_size, int mode);
// Serving instance (decode_stream_serve.cu; shared-memory and global modes only).
StreamKernelFn pick_stream_serve_kernel(int msg_dtype, int le, int tpc, int mode);

// The serving form of a grouping's stream plan (server pools): the kernel, block, shared bytes,
// message elements per slot (ws_stride) and table arguments that ndgsbp_decode would use for the
// grouping with variant AUTO when that picks the stream kernel, restricted to the shared-memory
// and global modes (a bulk-staged plan is served in global mode: the same arithmetic).  *ok =
// false when the plain decode would not use the stream kernel.
struct StreamServePlan {
    StreamKernelFn fn = nullptr;
    int threads = 0, per_sm = 0, mode = 0;
    size_t smem = 0;
    int msg_elems_per_slot = 0;   // ws_stride
    StreamArgs args{};
};
ndgsbp_status stream_serve_plan(const Groups& g, const ndgsbp_params* p, StreamServePlan* out, bool* ok);

}  // namespace ndgsbp
