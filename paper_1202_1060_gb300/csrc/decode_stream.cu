// Decode instances of the stream kernel (decode_stream_kernel.cuh) and its host-side helpers.
#include <cstring>

#include "decode_stream_kernel.cuh"

namespace ndgsbp {

size_t stream_smem_bytes(const StreamArgs& a, int msg_size, int mode) {
    size_t b = sa16(static_cast<size_t>(a.r.N) * 4) +
               sa16(static_cast<size_t>(a.window - 1) * (a.maxdeg | 1) * a.Z *
                    (msg_size == 2 && mode != kStreamGlobal ? 2 : 4));   // Old16 (decode_stream_kernel.cuh)
    const size_t slab = sa16(static_cast<size_t>(a.slab_elems) * msg_size);
    if (mode == kStreamSmem) b += sa16(static_cast<size_t>(a.msg_elems) * msg_size);
    if (mode == kStreamBulk) b += static_cast<size_t>(a.n_slabs) * slab;
    b += sa16(static_cast<size_t>(a.nl) * a.maxdeg * 8) + sa16(static_cast<size_t>(a.nl) * 4) +
         static_cast<size_t>(a.n_groupings) * a.G * a.window * 16;
    if (a.tpc == 2) b += static_cast<size_t>(4) * a.Z * 8;   // pair-exchange slots
    if (mode == kStreamBulk) b += static_cast<size_t>(a.n_slabs) * 8;
    return b;
}

// ---- instances ------------------------------------------------------------------------------
template <typename MsgT, int LE, int TPC>
static StreamKernelFn pick_mode(int mode) {
    switch (mode) {
        case kStreamSmem: return stream_decode_kernel<MsgT, LE, TPC, kStreamSmem>;
        case kStreamGlobal: return stream_decode_kernel<MsgT, LE, TPC, kStreamGlobal>;
        case kStreamBulk: return stream_decode_kernel<MsgT, LE, TPC, kStreamBulk>;
        default: return nullptr;
    }
}

template <typename MsgT>
static StreamKernelFn pick_shape(int le, int tpc, int mode) {
    if (tpc == 1 && le == 8) return pick_mode<MsgT, 8, 1>(mode);
    if (tpc == 1 && le == 11) return pick_mode<MsgT, 11, 1>(mode);
    if (tpc == 2 && le == 6) return pick_mode<MsgT, 6, 2>(mode);
    if (tpc == 2 && le == 11) return pick_mode<MsgT, 11, 2>(mode);
    return nullptr;
}

int stream_lane_width(int le, int tpc) {
    if (tpc == 1) return le <= 8 ? 8 : le <= 11 ? 11 : 0;
    if (tpc == 2) return le <= 6 ? 6 : le <= 11 ? 11 : 0;
    return 0;
}

int stream_max_threads(int tpc) { return stream_block_bound(tpc); }

StreamKernelFn pick_stream_kernel(int msg_dtype, int le, int tpc, int mode) {
    switch (msg_dtype) {
        case NDGSBP_F32: return pick_shape<float>(le, tpc, mode);
        case NDGSBP_F16: return pick_shape<__half>(le, tpc, mode);
        case NDGSBP_BF16: return pick_shape<__nv_bfloat16>(le, tpc, mode);
        default: return nullptr;
    }
}

}  // namespace ndgsbp
