// Serving instances of the layered QC kernel: pools of frame slots whose decoding state persists
// between launches (the server's epochs).  A launch advances the listed slots by at most
// epoch_iters iterations each; the arithmetic of a frame is that of qc_decode_kernel in a plain
// decode, so a frame decoded through the server equals the same frame decoded alone.
#include "qc_kernel.cuh"

namespace ndgsbp {

template <typename MsgT>
static QcKernelFn pick_serve(int maxdc, bool msg_smem) {
    switch (maxdc) {
        case 8:
            return msg_smem ? qc_decode_kernel<MsgT, true, 8, true, 0, true>
                            : qc_decode_kernel<MsgT, false, 8, true, 0, true>;
        case 16:
            return msg_smem ? qc_decode_kernel<MsgT, true, 16, true, 0, true>
                            : qc_decode_kernel<MsgT, false, 16, true, 0, true>;
        default: return nullptr;
    }
}

QcKernelFn pick_qc_serve_kernel(int msg_dtype, int maxdc, bool msg_smem) {
    switch (msg_dtype) {
        case NDGSBP_F32: return pick_serve<float>(maxdc, msg_smem);
        case NDGSBP_F16: return pick_serve<__half>(maxdc, msg_smem);
        case NDGSBP_BF16: return pick_serve<__nv_bfloat16>(maxdc, msg_smem);
        default: return nullptr;
    }
}

}  // namespace ndgsbp
