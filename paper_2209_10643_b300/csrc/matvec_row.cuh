// One matrix row times a vector, spread over the 32 lanes of a warp (the
// inner loop of the matvec body, run SIMD-parallel).  Each lane streams
// 128-bit loads of the row with 16 FP32 accumulators, which are folded in a
// fixed pairwise order and then across the lanes with a butterfly: the
// result is deterministic and its rounding error is bounded by about
// (cols/512 + 9) unit roundoffs of sum_j |A_rj x_j|.
//
// A row that does not start on a 16-byte boundary (a width that is not a
// multiple of 4) first takes the columns up to the boundary into the lane
// tail sums, then streams the rest of the row with 128-bit loads; x, then no
// longer in phase with the row, is read as four 32-bit loads per vector.
#pragma once

#include "device_common.cuh"

namespace upir {

template <bool XVEC>
__device__ __forceinline__ float4 row_dot_x4(const float* __restrict__ x, int64_t j) {
    if (XVEC) return __ldg(reinterpret_cast<const float4*>(x + j));
    return make_float4(__ldg(x + j), __ldg(x + j + 1), __ldg(x + j + 2), __ldg(x + j + 3));
}

// Columns [j0, ...) of the row in blocks of 512 and then the remaining whole
// groups of four, a + j0 16-byte aligned; returns the first column not done
// (fewer than four remain).
template <bool XVEC>
__device__ __forceinline__ int64_t row_dot_vec(const float* __restrict__ a, const float* __restrict__ x,
                                               int64_t cols, int lane, int64_t j0, float (&acc)[16]) {
    for (; j0 + 512 <= cols; j0 += 512) {
        float4 av[4], xv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) av[u] = __ldcs(reinterpret_cast<const float4*>(a + j0 + 128 * u + 4 * lane));
#pragma unroll
        for (int u = 0; u < 4; ++u) xv[u] = row_dot_x4<XVEC>(x, j0 + 128 * u + 4 * lane);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            acc[4 * u + 0] = __fmaf_rn(av[u].x, xv[u].x, acc[4 * u + 0]);
            acc[4 * u + 1] = __fmaf_rn(av[u].y, xv[u].y, acc[4 * u + 1]);
            acc[4 * u + 2] = __fmaf_rn(av[u].z, xv[u].z, acc[4 * u + 2]);
            acc[4 * u + 3] = __fmaf_rn(av[u].w, xv[u].w, acc[4 * u + 3]);
        }
    }
    // the rest of the whole 4-column groups, fewer than 512 columns: every
    // lane's (up to four) loads issued together, absent groups read as zero
    const int64_t ng = (cols - j0) >> 2;  // whole groups left, < 128
    if (ng > 0) {
        float4 av[4], xv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t g = 32 * u + lane;
            const bool in = g < ng;
            av[u] = in ? __ldcs(reinterpret_cast<const float4*>(a + j0 + 4 * g)) : make_float4(0.f, 0.f, 0.f, 0.f);
            xv[u] = in ? row_dot_x4<XVEC>(x, j0 + 4 * g) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            acc[4 * u + 0] = __fmaf_rn(av[u].x, xv[u].x, acc[4 * u + 0]);
            acc[4 * u + 1] = __fmaf_rn(av[u].y, xv[u].y, acc[4 * u + 1]);
            acc[4 * u + 2] = __fmaf_rn(av[u].z, xv[u].z, acc[4 * u + 2]);
            acc[4 * u + 3] = __fmaf_rn(av[u].w, xv[u].w, acc[4 * u + 3]);
        }
        j0 += 4 * ng;
    }
    return j0;
}

__device__ __forceinline__ float row_dot(const float* __restrict__ a, const float* __restrict__ x,
                                         int64_t cols, int lane) {
    float acc[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = 0.0f;
    float tail = 0.0f;
    int64_t j0 = 0;
    const uintptr_t am = reinterpret_cast<uintptr_t>(a) & 15;
    if ((reinterpret_cast<uintptr_t>(x) & 15) == 0 && (am & 3) == 0) {
        if (am == 0) {
            j0 = row_dot_vec<true>(a, x, cols, lane, 0, acc);
        } else {
            const int64_t p = min((int64_t)((16 - am) >> 2), cols);  // columns before the boundary
            if (lane < p) tail = __fmaf_rn(a[lane], x[lane], tail);
            j0 = row_dot_vec<false>(a, x, cols, lane, p, acc);
        }
    }
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
