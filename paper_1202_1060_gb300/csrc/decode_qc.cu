// Layered QC decode kernels for sm_103a.
//
// For QC codes grouped in whole layers (windows of `window` layers of Z CNs each), the VN of
// edge k of CN c in layer l is b_k Z + (c + s_k) mod Z, with (b_k, s_k) the block column and
// circulant shift of the layer's k-th base entry.  The kernels compute those indices instead of
// reading per-edge tables: each layer contributes one (4 (b Z + s), Z - s) pair per edge, held
// in shared memory and read as a broadcast, and the index is kept as a byte offset into the
// posterior.  The messages of CN c of layer l sit at layer_off[l] + c S_l + k with an odd
// stride S_l >= d_l, so 32 consecutive CNs touch 32 distinct banks and k is a compile-time
// offset.
//
// qc_decode_kernel: thread t owns window position j = t / Z and CN c = t mod Z in every group.
// It runs phase A (Eq. (1) on every CN of the group; VN offsets and message changes kept in
// registers) and phase B (changes added layer position by layer position, the same fixed order
// as the colour order of the table-driven kernel, whose results it therefore reproduces).
// Layers get fully unrolled code for their exact degree when every layer degree lies in
// (MAXDC/2, MAXDC] (the usual QC case); other codes use the degree-generic instances.
#include <cstring>

#include "qc_kernel.cuh"

namespace ndgsbp {

// ---- kernel selection ---------------------------------------------------------------------
template <typename MsgT, int MAXDC>
static QcKernelFn pick_qc_storage(bool msg_smem, bool spec) {
    if (spec) return msg_smem ? qc_decode_kernel<MsgT, true, MAXDC, true> : qc_decode_kernel<MsgT, false, MAXDC, true>;
    return msg_smem ? qc_decode_kernel<MsgT, true, MAXDC, false> : qc_decode_kernel<MsgT, false, MAXDC, false>;
}

template <typename MsgT>
static QcKernelFn pick_qc_degree(int maxdc, bool msg_smem, bool spec, bool occ6) {
    if (occ6) {
        // 6 CTAs of <= 192 threads per SM: degree <= 8, messages in shared memory, 16-bit storage
        if (maxdc != 8 || !msg_smem || !spec || sizeof(MsgT) != 2) return nullptr;
        return qc_decode_kernel<MsgT, true, 8, true, 6>;
    }
    switch (maxdc) {
        case 8: return pick_qc_storage<MsgT, 8>(msg_smem, spec);
        case 16: return pick_qc_storage<MsgT, 16>(msg_smem, spec);
        case 32:
            if (spec) return nullptr;
            return msg_smem ? qc_decode_kernel<MsgT, true, 32, false> : qc_decode_kernel<MsgT, false, 32, false>;
        default: return nullptr;
    }
}

bool qc_degrees_specialised(const QcLayout& Q, int maxdc) {
    if (maxdc > 16) return false;
    for (int d : Q.layer_deg)
        if (d <= maxdc / 2 || d > maxdc) return false;
    return true;
}

int qc_occ_threads() { return kOccThreads; }

QcKernelFn pick_qc_kernel(int msg_dtype, int maxdc, bool msg_smem, bool spec, bool occ6) {
    switch (msg_dtype) {
        case NDGSBP_F32: return pick_qc_degree<float>(maxdc, msg_smem, spec, occ6);
        case NDGSBP_F16: return pick_qc_degree<__half>(maxdc, msg_smem, spec, occ6);
        case NDGSBP_BF16: return pick_qc_degree<__nv_bfloat16>(maxdc, msg_smem, spec, occ6);
        default: return nullptr;
    }
}

static size_t a16(size_t x) { return (x + 15) & ~static_cast<size_t>(15); }

size_t qc_table_bytes(const QcLayout& Q) {
    const size_t G = Q.window ? Q.group_layers.size() / Q.window : 0;
    return a16(static_cast<size_t>(Q.n_layers) * Q.max_deg * 8) + 3 * a16(static_cast<size_t>(Q.n_layers) * 4) +
           a16(G * Q.window * 4) + G * Q.window * 16;
}

void fill_qc_args(QcArgs& a, const QcLayout& Q, const DeviceQc& D, void* ws_msgs) {
    a.Z = Q.Z;
    a.nl = Q.n_layers;
    a.window = Q.window;
    a.n_groupings = Q.n_groupings;
    a.G = static_cast<int>(Q.group_layers.size() / (static_cast<size_t>(Q.window) * Q.n_groupings));
    a.maxdeg = Q.max_deg;
    a.msg_slots = Q.msg_slots;
    a.edge_tab = reinterpret_cast<const int2*>(D.edge_tab);
    a.layer_deg = D.layer_deg;
    a.layer_stride = D.layer_stride;
    a.layer_off = D.layer_off;
    a.group_layers = D.group_layers;
    a.csr_of = D.csr_of;
    a.ws_msgs = ws_msgs;
}

}  // namespace ndgsbp
