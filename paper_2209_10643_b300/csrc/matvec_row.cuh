// One matrix row times a vector, spread over the 32 lanes of a warp (the
// inner loop of the matvec body, run SIMD-parallel).  Each lane streams
// 128-bit loads of the row with 16 FP32 accumulators, which are folded in a
// fixed pairwise order and then across the lanes with a butterfly: the
// result is deterministic and its rounding error is bounded by about
// (cols/512 + 9) unit roundoffs of sum_j |A_rj x_j|.
#pragma once

#include "device_common.cuh"

namespace upir {

__device__ __forceinline__ float row_dot(const float* __restrict__ a, const float* __restrict__ x,
                                         int64_t cols, int lane) {
    float acc[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = 0.0f;
    int64_t j0 = 0;
    const bool vec = ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(x)) & 15) == 0;
    if (vec) {
        const int64_t full = cols / 512 * 512;
        for (; j0 < full; j0 += 512) {
            float4 av[4], xv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                av[u] = __ldcs(reinterpret_cast<const float4*>(a + j0 + 128 * u + 4 * lane));
#pragma unroll
            for (int u = 0; u < 4; ++u)
                xv[u] = __ldg(reinterpret_cast<const float4*>(x + j0 + 128 * u + 4 * lane));
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                acc[4 * u + 0] = __fmaf_rn(av[u].x, xv[u].x, acc[4 * u + 0]);
                acc[4 * u + 1] = __fmaf_rn(av[u].y, xv[u].y, acc[4 * u + 1]);
                acc[4 * u + 2] = __fmaf_rn(av[u].z, xv[u].z, acc[4 * u + 2]);
                acc[4 * u + 3] = __fmaf_rn(av[u].w, xv[u].w, acc[4 * u + 3]);
            }
        }
        const int64_t full4 = cols / 128 * 128;
        for (; j0 < full4; j0 += 128) {
            const float4 av = __ldcs(reinterpret_cast<const float4*>(a + j0 + 4 * lane));
            const float4 xv = __ldg(reinterpret_cast<const float4*>(x + j0 + 4 * lane));
            acc[0] = __fmaf_rn(av.x, xv.x, acc[0]);
            acc[1] = __fmaf_rn(av.y, xv.y, acc[1]);
            acc[2] = __fmaf_rn(av.z, xv.z, acc[2]);
            acc[3] = __fmaf_rn(av.w, xv.w, acc[3]);
        }
    }
    float tail = 0.0f;
    for (int64_t j = j0 + lane; j < cols; j += 32) tail = __fmaf_rn(a[j], x[j], tail);
    acc[15] = __fadd_rn(acc[15], tail);
    // fixed pairwise tree over the 16 accumulators
#pragma unroll
    for (int w = 8; w >= 1; w >>= 1)
#pragma unroll
        for (int q = 0; q < w; ++q) acc[q] = __fadd_rn(acc[q], acc[q + w]);
    float v = acc[0];
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) v = __fadd_rn(v, __shfl_xor_sync(0xffffffffu, v, m));
    return v;
}

}  // namespace upir
