// Many independent, uneven regions in one persistent launch.  The regions'
// loops are cut into tiles; the (region, tile) work items, largest regions
// first, are claimed one at a time from an atomic counter by persistent teams
// and dispatched on the region's body.  The tile loop of each region is thus
// workshared dynamically over all teams of the GPU (§3.2 schedule(dynamic)),
// and each region's reduction is finalized by its last tile: the tile
// partials are folded in tile order, so the result does not depend on which
// team ran which tile.
#include "matvec_row.cuh"

namespace upir {

namespace {

__device__ __forceinline__ void axpy_tile(const BatchParams& P, const BatchRegion& R, int64_t t) {
    __shared__ int last;
    const int64_t e0 = R.lb + t * P.axpy_tile;
    const int64_t e1 = min(e0 + (int64_t)P.axpy_tile, R.lb + R.trip);
    FAcc f = facc_identity(R.fop);
    const bool red = R.fop != 0;
    const bool xy = R.fterm == UPIR_TERM_XY;
    auto term = [&](float xv, float yn) {
        if (!red) return;
        if (!xy) {
            facc_add(f, yn, UPIR_RED_ADD);
        } else {
            const float pr = __fmul_rn(xv, yn);
            facc_add(f, pr, UPIR_RED_ADD, __fmaf_rn(xv, yn, -pr));
        }
    };
    const float* x = R.in0;
    float* y = R.out;
    const bool vec = ((reinterpret_cast<uintptr_t>(x + e0) | reinterpret_cast<uintptr_t>(y + e0)) & 15) == 0;
    if (vec) {
        const int64_t n4 = (e1 - e0) / 4;
#pragma unroll 4
        for (int64_t g = threadIdx.x; g < n4; g += blockDim.x) {
            const float4 xv = __ldcs(reinterpret_cast<const float4*>(x + e0) + g);
            const float4 yv = __ldcs(reinterpret_cast<const float4*>(y + e0) + g);
            float4 yn;
            yn.x = __fmaf_rn(R.a, xv.x, yv.x);
            yn.y = __fmaf_rn(R.a, xv.y, yv.y);
            yn.z = __fmaf_rn(R.a, xv.z, yv.z);
            yn.w = __fmaf_rn(R.a, xv.w, yv.w);
            __stcs(reinterpret_cast<float4*>(y + e0) + g, yn);
            term(xv.x, yn.x);
            term(xv.y, yn.y);
            term(xv.z, yn.z);
            term(xv.w, yn.w);
        }
        for (int64_t e = e0 + 4 * n4 + threadIdx.x; e < e1; e += blockDim.x) {
            const float yn = __fmaf_rn(R.a, x[e], y[e]);
            y[e] = yn;
            term(x[e], yn);
        }
    } else {
        for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
            const float yn = __fmaf_rn(R.a, x[e], y[e]);
            y[e] = yn;
            term(x[e], yn);
        }
    }
    if (!red) return;
    const Partial bp = block_reduce_partial(make_partial(f, 0), UPIR_RED_ADD, 0);
    if (threadIdx.x == 0) {
        P.partials[R.slot0 + t] = bp;
        __threadfence();
        last = atomicAdd(R.ticket, 1u) == (unsigned)R.tiles - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    const Partial fin = block_reduce_slots(P.partials + R.slot0, R.tiles, UPIR_RED_ADD, 0);
    if (threadIdx.x == 0) {
        RedVars rv{R.fvar, nullptr, UPIR_RED_ADD, 0, R.fterm, 0};
        write_reduction_vars(rv, fin);
        *R.ticket = 0;
    }
}

__device__ __forceinline__ void jacobi_tile(const BatchParams& P, const BatchRegion& R, int64_t t,
                                            float* halo) {
    constexpr int HW = kBatchJacCols + 2;
    const int64_t band = t / R.tiles_c, tc = t - band * R.tiles_c;
    const int64_t r0 = R.lb + band * P.jac_rows;
    const int nr = (int)min((int64_t)P.jac_rows, R.lb + R.trip - r0);
    const int64_t c0 = tc * kBatchJacCols;
    const int64_t cols = R.cols;
    const float* u = R.in0;
    for (int idx = threadIdx.x; idx < (nr + 2) * HW; idx += blockDim.x) {
        const int64_t rr = r0 - 1 + idx / HW, cc = c0 - 1 + idx % HW;
        halo[idx] = (cc >= 0 && cc < cols) ? u[rr * cols + cc] : 0.0f;
    }
    __syncthreads();
    float racc = R.fop == UPIR_RED_MIN ? __int_as_float(0x7f800000) : -__int_as_float(0x7f800000);
    for (int idx = threadIdx.x; idx < nr * kBatchJacCols; idx += blockDim.x) {
        const int i = idx / kBatchJacCols, j = idx % kBatchJacCols;
        const int64_t c = c0 + j;
        if (c < 1 || c > cols - 2) continue;
        const float* cen = halo + (i + 1) * HW + j + 1;
        const float v = __fmul_rn(0.25f, __fadd_rn(__fadd_rn(cen[-HW], cen[HW]), __fadd_rn(cen[-1], cen[1])));
        R.out[(r0 + i) * cols + c] = v;
        if (R.fop) racc = fold(racc, fabsf(__fsub_rn(v, cen[0])), R.fop);
    }
    if (R.fop) {
        const float b = block_fold(racc, R.fop);
        if (threadIdx.x == 0) atomic_fold_minmax(R.fvar, b, R.fop);
    }
    __syncthreads();  // the halo buffer is reused by the next item
}

__device__ __forceinline__ void matvec_tile(const BatchParams& P, const BatchRegion& R, int64_t t) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int64_t r0 = R.lb + t * P.mv_rows;
    const int64_t r1 = min(r0 + (int64_t)P.mv_rows, R.lb + R.trip);
    for (int64_t r = r0 + warp; r < r1; r += nw) {
        const float v = row_dot(R.in0 + r * R.cols, R.in1, R.cols, lane);
        if (lane == 0) R.out[r] = v;
    }
}

__global__ void __launch_bounds__(kBatchUnits) batch_persistent_kernel(const BatchParams P) {
    __shared__ float halo[(kBatchMaxJacRows + 2) * (kBatchJacCols + 2)];
    __shared__ int64_t item;
    __shared__ int last_team;
    griddep_wait();
    for (;;) {
        if (threadIdx.x == 0) item = (int64_t)atomicAdd(P.counter, 1ull);
        __syncthreads();
        const int64_t k = item;
        __syncthreads();
        if (k >= P.nitems) break;
        const int2 it = P.items[k];
        const BatchRegion& R = P.regions[it.x];
        switch (R.op) {
            case BOP_AXPY: axpy_tile(P, R, it.y); break;
            case BOP_JACOBI: jacobi_tile(P, R, it.y, halo); break;
            default: matvec_tile(P, R, it.y); break;
        }
    }
    // the last team returns the work counter to zero for the next launch
    if (threadIdx.x == 0) {
        __threadfence();
        last_team = atomicAdd(P.exit_ticket, 1u) == gridDim.x - 1;
        if (last_team) {
            *P.exit_ticket = 0;
            *P.counter = 0;
        }
    }
}

}  // namespace

int batch_persistent_teams_per_sm() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_persistent_kernel, kBatchUnits, 0) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return n > 0 ? n : 1;
}

cudaError_t launch_batch_persistent(int teams, const BatchParams& p, cudaStream_t s) {
    return launch_pdl(batch_persistent_kernel, teams, kBatchUnits, 0, s, p);
}

}  // namespace upir
