// Serving instances of the stream kernel (decode_stream_kernel.cuh, SERVE = true): messages in
// shared memory or in global memory, the lane shapes of the decode instances.
#include "decode_stream_kernel.cuh"

namespace ndgsbp {

template <typename MsgT, int LE, int TPC>
static StreamKernelFn pick_serve_mode(int mode) {
    switch (mode) {
        case kStreamSmem: return stream_decode_kernel<MsgT, LE, TPC, kStreamSmem, true>;
        case kStreamGlobal: return stream_decode_kernel<MsgT, LE, TPC, kStreamGlobal, true>;
        default: return nullptr;
    }
}

template <typename MsgT>
static StreamKernelFn pick_serve_shape(int le, int tpc, int mode) {
    if (tpc == 1 && le == 8) return pick_serve_mode<MsgT, 8, 1>(mode);
    if (tpc == 1 && le == 11) return pick_serve_mode<MsgT, 11, 1>(mode);
    if (tpc == 2 && le == 6) return pick_serve_mode<MsgT, 6, 2>(mode);
    if (tpc == 2 && le == 11) return pick_serve_mode<MsgT, 11, 2>(mode);
    return nullptr;
}

StreamKernelFn pick_stream_serve_kernel(int msg_dtype, int le, int tpc, int mode) {
    switch (msg_dtype) {
        case NDGSBP_F32: return pick_serve_shape<float>(le, tpc, mode);
        case NDGSBP_F16: return pick_serve_shape<__half>(le, tpc, mode);
        case NDGSBP_BF16: return pick_serve_shape<__nv_bfloat16>(le, tpc, mode);
        default: return nullptr;
    }
}

}  // namespace ndgsbp
