// Eq. (1) with a CN's edges split over consecutive lanes of a warp (1, 2 or 4 lanes per CN), in
// the positive-pair form of check_node_update (device_common.cuh), shared by the tile kernel
// (decode_tile.cu) and the stream kernel (decode_stream.cu): the same operations in the same
// order, so the two give bit-identical messages for the same lane split.
#pragma once

#include "device_common.cuh"

namespace ndgsbp {

__device__ __forceinline__ int tile_vb(int2 e, int c, int Z4) { return e.x + 4 * c - (c >= e.y ? Z4 : 0); }

__device__ __forceinline__ float& at_b(float* P, int vb) {
    return *reinterpret_cast<float*>(reinterpret_cast<char*>(P) + vb);
}

// Forward pass over the lane's LE edge positions, of which the first nreal are edges: prefix
// pairs, lane total (cn, ce), and the signs: xu[k] = exp(-|L_k|) >= 0 carries the sign of t[k]
// in its sign bit (every use takes |xu|, a free operand modifier), and bit 31 of par collects
// the parity of the lane's input signs.  Every lane runs the same LE, the kernel instance's
// compile-time width (no divergence between lanes holding different edge counts, no dispatch
// on the width at run time); a position past nreal is the neutral factor
// tanh = 1, i.e. u = 0 and (N, E) = (1/2, 0), which only scales the lane's pairs by exactly 1/2
// (t = +0 there, so no sign either): the outputs of the real edges do not change.
template <int LE>
__device__ __forceinline__ void lane_forward(const float (&t)[LE], int nreal, float lim, float (&xu)[LE],
                                             float (&pn)[LE], float (&pe)[LE], float& cn, float& ce,
                                             unsigned& par) {
#pragma unroll
    for (int k = 0; k < LE; ++k) {
        const bool real = k < nreal;
        const float tk = real ? t[k] : 0.f;
        const unsigned tb = __float_as_uint(tk);
        par ^= tb;
        const float x = fminf(fabsf(tk), lim);
        const float u = real ? ex2_approx(-x) : 0.f;   // exp(-|L|) (log2 units)
        const float n = fmaf(-0.5f, u, 0.5f);
        xu[k] = __uint_as_float(__float_as_uint(u) | (tb & 0x80000000u));
        pn[k] = cn;
        pe[k] = ce;
        ce = fmaf(ce, fmaf(0.5f, u, 0.5f), cn * u);   // n + u = (1 + u) / 2
        cn = cn * n;
    }
}

// Backward pass: the suffix starts from (sn, se), the product over the other lanes' edges;
// pm = bit 31 of the CN's sign parity (all lanes); outputs for the nreal real positions only.
template <int LE, typename Emit>
__device__ __forceinline__ void lane_backward(const float (&xu)[LE], const float (&pn)[LE], const float (&pe)[LE],
                                              int nreal, float sn, float se, unsigned pm, float lim, Emit emit) {
#pragma unroll
    for (int k = LE - 1; k >= 0; --k) {
        const float u = fabsf(xu[k]);
        const float n = fmaf(-0.5f, u, 0.5f);
        const float en = pn[k] * sn;
        const float ss = sn + se;
        const float ee = fmaf(pe[k], ss, pn[k] * se);
        const float w = fmaf(en * rcp_approx(ee), 2.f, 1.f);
        const float mag = fminf(lg2_approx(w), lim);
        const unsigned sgn = (__float_as_uint(xu[k]) ^ pm) & 0x80000000u;
        if (k < nreal) emit(k, __uint_as_float(__float_as_uint(mag) | sgn));
        se = fmaf(u, ss, se * n);   // se (n + u) + sn u, reusing sn + se
        sn = sn * n;
    }
}

// Product over the other lanes of a CN (tpc = 2 or 4 consecutive lanes, gmask their bits) and
// the total sign parity: (on, oe) seeds the lane's suffix pass.
__device__ __forceinline__ void lane_exchange(int tpc, unsigned gmask, float cn, float ce, unsigned lpar, float& on,
                                              float& oe, unsigned& par) {
    on = 1.f;
    oe = 0.f;
    par = lpar;
    if (tpc > 1) {
        const float xn = __shfl_xor_sync(gmask, cn, 1), xe = __shfl_xor_sync(gmask, ce, 1);
        par ^= __shfl_xor_sync(gmask, par, 1);
        if (tpc == 2) {
            on = xn;
            oe = xe;
        } else {
            const float pn2 = cn * xn, pe2 = fmaf(ce, xn + xe, cn * xe);   // this pair's total
            const float yn = __shfl_xor_sync(gmask, pn2, 2), ye = __shfl_xor_sync(gmask, pe2, 2);
            par ^= __shfl_xor_sync(gmask, par, 2);
            on = xn * yn;
            oe = fmaf(xe, yn + ye, xn * ye);
        }
    }
}

}  // namespace ndgsbp
