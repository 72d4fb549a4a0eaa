// Tile decode kernel interface (decode_tile.cu): QC codes of any window size and row degree
// up to 32, several frames per CTA, and several codes in one launch (ragged batches).
#pragma once

#include "device_common.cuh"
#include "ndgsbp_internal.h"

namespace ndgsbp {

// Division by a divisor fixed for a launch, as a multiply and a shift: q = (n m) >> k with
// k = 32 + ceil(log2 d) and m = ceil(2^k / d), exact for 0 <= n < 2^32 (2^k >= 2^32 d, so the
// rounding of m adds less than 1/d to n/d).
struct FastDiv {
    unsigned long long m;
    int k;
};

inline FastDiv make_fastdiv(unsigned d) {
    int l = 0;
    while ((1ull << l) < d) ++l;
    const int k = 32 + l;
    return FastDiv{((1ull << k) + d - 1) / d, k};
}

__device__ __forceinline__ int fast_div(int n, FastDiv f) {
    return static_cast<int>((static_cast<unsigned long long>(static_cast<unsigned>(n)) * f.m) >> f.k);
}

// One code of a launch: its layered QC description, its batch, and how a CTA lays it out.
struct TileCode {
    int N, E, Z, nl, G, window, maxdeg, msg_slots;
    int tpc;              // lanes per CN (1, 2 or 4)
    int le;               // edges per lane, ceil(maxdeg / tpc) <= 8
    int slots;            // frames a CTA holds at once
    int slot_bytes;       // shared bytes per frame slot: posterior, messages, deltas
    int p_bytes;          // posterior bytes at the start of a slot (16-aligned)
    int m_bytes;          // message bytes after it (0 when messages live in global memory)
    int delta_stride;     // lane segments: lane p of CN c of layer l keeps its messages at
    int msg_stride;       // ((l Z + c) tpc + p) msg_stride + k and its window's deltas at
                          // (cnl tpc + p) delta_stride + k; both strides are odd in 4-byte words,
                          // so the lanes of a warp hit distinct shared-memory banks
    const int2* edge_tab;
    const int32_t* layer_deg;
    const int32_t* group_layers;
    const int32_t* csr_of;
    RunArgs r;            // this code's batch, parameters and outputs (r.counter unused)
    void* ws_msgs;        // global message slots (blocks x slots x msg_slots) when m_bytes == 0
    // serving: frames are slots of a pool whose decoding state persists between launches
    int* state_flag;      // [pool] kSlotFree / kSlotNew / kSlotRunning / kSlotDone, or null
    int* state_iter;      // [pool] iterations done so far
    float* state_P;       // [pool][N] posteriors of running frames
    void* state_msgs;     // [pool][msg_slots] messages of running frames
    int epoch_iters;      // iterations a frame may run in one launch before its state is saved
    int n_groupings;      // group -> layer tables cycled by iteration (group_layers holds all)
    int* done_list;       // [pool] slots whose frame retired in this launch (serving), or null
    int* done_count;      // number of entries in done_list (zeroed before the launch)
    // divisions of the kernel's index arithmetic (set by tile_code_finish)
    FastDiv div_slot;     // by window * Z * tpc (CN-lanes of one group in one slot)
    FastDiv div_pos;      // by Z * tpc (CN-lanes of one layer)
    FastDiv div_syn;      // by nl * Z * tpc (CN-lanes of all layers)
    FastDiv div_z;        // by Z
};

// Fills the derived fields of a TileCode whose shape (window, Z, tpc, nl) is set.
void tile_code_finish(TileCode& C);

constexpr int kSlotFree = 0, kSlotNew = 1, kSlotRunning = 2, kSlotDone = 3;

constexpr int kTileMaxCodes = 8;

// A launch: a list of tiles (code, first frame, frame count) handed out by an atomic counter.
// With tiles == nullptr the tiles are implicit: code 0, tile t = frames [t tile_frames, ...).
struct TileArgs {
    TileCode codes[kTileMaxCodes];
    int n_codes;
    const int4* tiles;    // x = code, y = first frame, z = frames
    int n_tiles;
    int tile_frames;
    unsigned long long* tile_counter;
    int table_bytes;      // shared bytes reserved for the largest code's tables
};

typedef void (*TileKernelFn)(const TileArgs);

// Kernel instance for a launch: lane_width = tile_lane_width of the largest le among its codes
// (the unrolled edge positions per lane); regb when one round of the block covers a group of
// every code (slots x window x Z x tpc <= block threads), which keeps message changes in
// registers between phases A and B; single for a launch over one code (codes[0] only).  nullptr
// for an unknown dtype or width.
TileKernelFn pick_tile_kernel(int msg_dtype, bool serve, int lane_width, bool regb, bool single);

// Compiled lane width for le edges per lane: 4, 6 or 8 (0 when le is not in 1..8).
int tile_lane_width(int le);

// Storage shape of the tile kernel for a code at tpc lanes per CN: edges per lane, the odd lane
// segment stride, messages per frame (all layers) and deltas per frame (one window).
struct TileShape {
    int tpc, le, msg_stride, delta_stride, msg_slots, delta_floats;
};
TileShape tile_shape(const QcLayout& Q, int tpc, int msg_dtype);
size_t tile_table_bytes(const QcLayout& Q);
// Lanes per CN for a code of the given largest degree (edges per lane at most 8), 0 if above 32.
int tile_lanes_per_cn(int maxdeg);

}  // namespace ndgsbp
