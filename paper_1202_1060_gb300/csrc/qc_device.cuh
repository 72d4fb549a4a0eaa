// Device helpers shared by the layered QC kernels (decode_qc.cu, decode_qc2.cu).
#pragma once

#include "device_common.cuh"

namespace ndgsbp {

// Byte offset of the VN of table entry e for CN c (c4 = 4 c, Z4 = 4 Z).
__device__ __forceinline__ int qc_vb(int2 e, int c, int c4, int Z4) { return e.x + c4 - (c >= e.y ? Z4 : 0); }

__device__ __forceinline__ float& at_byte(float* P, int vb) {
    return *reinterpret_cast<float*>(reinterpret_cast<char*>(P) + vb);
}

// Warp-uniform dispatch on the layer degree (a warp covers one layer when 32 divides the CNs a
// layer spreads over).
#define NDGSBP_DEGREE_CASES(MAXDC, X) \
    if (MAXDC == 8) { X(5) X(6) X(7) X(8) } else if (MAXDC == 16) { X(9) X(10) X(11) X(12) X(13) X(14) X(15) X(16) }
#define NDGSBP_DD(D) ((D) <= MAXDC ? (D) : MAXDC)

__device__ __forceinline__ float2 f2(float x) { return make_float2(x, x); }

// check_node_update on two independent CNs at once (two CNs of a frame, or one CN of two
// frames): the same operations, lane by lane, as float2 packed FP32 instructions, so each
// lane's result equals the scalar routine's bit for bit.
template <int D, typename Emit>
__device__ __forceinline__ void check_node_update2(const float2 (&t)[D], float lim, Emit emit) {
    float2 xu[D], pn[D], pe[D];
    unsigned sb0 = 0u, sb1 = 0u;
    float2 cn = f2(1.f), ce = f2(0.f);
#pragma unroll
    for (int k = 0; k < D; ++k) {
        sb0 |= (__float_as_uint(t[k].x) >> 31) << k;
        sb1 |= (__float_as_uint(t[k].y) >> 31) << k;
        const float2 x = make_float2(fminf(fabsf(t[k].x), lim), fminf(fabsf(t[k].y), lim));
        const float2 u = make_float2(ex2_approx(-x.x), ex2_approx(-x.y));   // exp(-|L|) (log2 units)
        const float2 n = __ffma2_rn(f2(-0.5f), u, f2(0.5f));             // (1 - u) / 2
        xu[k] = u;
        pn[k] = cn;
        pe[k] = ce;
        ce = __ffma2_rn(ce, __ffma2_rn(f2(0.5f), u, f2(0.5f)), __fmul2_rn(cn, u));   // n + u = (1 + u) / 2
        cn = __fmul2_rn(cn, n);
    }
    // bit k of sf0 / sf1 = sign of output k: the parity of all input signs xor sign k
    const unsigned sf0 = sb0 ^ (0u - (__popc(sb0) & 1u)), sf1 = sb1 ^ (0u - (__popc(sb1) & 1u));
    float2 sn = f2(1.f), se = f2(0.f);
#pragma unroll
    for (int k = D - 1; k >= 0; --k) {
        const float2 u = xu[k];
        const float2 n = __ffma2_rn(f2(-0.5f), u, f2(0.5f));
        const float2 en = __fmul2_rn(pn[k], sn);
        const float2 ss = __fadd2_rn(sn, se);
        const float2 ee = __ffma2_rn(pe[k], ss, __fmul2_rn(pn[k], se));
        const float2 w = __ffma2_rn(__fmul2_rn(en, make_float2(rcp_approx(ee.x), rcp_approx(ee.y))), f2(2.f), f2(1.f));
        const float2 lg = make_float2(lg2_approx(w.x), lg2_approx(w.y));
        const float m0 = fminf(lg.x, lim), m1 = fminf(lg.y, lim);
        const unsigned g0 = (sf0 << (31 - k)) & 0x80000000u, g1 = (sf1 << (31 - k)) & 0x80000000u;
        emit(k, make_float2(__uint_as_float(__float_as_uint(m0) | g0), __uint_as_float(__float_as_uint(m1) | g1)));
        se = __ffma2_rn(u, ss, __fmul2_rn(se, n));   // se (n + u) + sn u, reusing sn + se
        sn = __fmul2_rn(sn, n);
    }
}

}  // namespace ndgsbp
