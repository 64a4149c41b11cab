// Dense matrix-vector product y = A x (the matvec workload of §6).  The
// worksharing loop runs over rows; its worker is a warp, and the inner dot
// product over the row is spread over the warp's lanes (the inner loop is the
// SIMD-parallel one).  Each lane streams 128-bit loads of A with 16 FP32
// accumulators, which are folded in a fixed order and then across the lanes
// with a butterfly: the result is deterministic and its rounding error is
// bounded by about (cols/512 + 9) unit roundoffs of sum_j |A_rj x_j|.
#include "device_common.cuh"

namespace upir {

namespace {

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

__global__ void __launch_bounds__(1024) matvec_kernel(const MatvecParams p) {
    const int lane = threadIdx.x & 31;
    const int64_t wpb = blockDim.x >> 5;
    const int64_t W = (int64_t)gridDim.x * wpb;
    const int64_t w = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5);
    if (p.wait_prior) griddep_wait();
    griddep_launch_dependents();
    auto rows = [&](int64_t k0, int64_t k1) {
        for (int64_t k = k0; k < k1; ++k) {
            const int64_t r = p.lb + k * p.step;
            const float v = row_dot(p.A + r * p.cols, p.x, p.cols, lane);
            if (lane == 0) p.y[r] = v;
        }
    };
    if (p.sched == UPIR_SCHED_DYNAMIC) {
        const int64_t c = p.chunk > 0 ? p.chunk : 1;
        const int64_t nchunks = (p.trip + c - 1) / c;
        for (;;) {
            unsigned long long j = 0;
            if (lane == 0) j = atomicAdd(p.sc.chunk_counter, 1ull);
            j = __shfl_sync(0xffffffffu, j, 0);
            if ((int64_t)j >= nchunks) break;
            rows((int64_t)j * c, min((int64_t)j * c + c, p.trip));
        }
        __shared__ int last;
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            last = atomicAdd(p.sc.ticket, 1u) == gridDim.x - 1;
            if (last) {
                *p.sc.ticket = 0;
                *p.sc.chunk_counter = 0;
            }
        }
    } else {
        static_ranges(p.sk, p.trip, p.chunk, W, w, rows);
    }
}

}  // namespace

cudaError_t launch_matvec(int teams, int units, const MatvecParams& p, cudaStream_t s) {
    return launch_pdl(matvec_kernel, teams, units, 0, s, p);
}

}  // namespace upir
