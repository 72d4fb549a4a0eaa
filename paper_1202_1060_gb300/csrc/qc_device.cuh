// Device helpers of the layered QC kernels (qc_kernel.cuh).
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

}  // namespace ndgsbp
