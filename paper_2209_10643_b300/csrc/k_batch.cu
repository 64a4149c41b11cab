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

// Halo rows of the tile are staged in shared memory; shared column j holds
// grid column c0 - 4 + j, so the tile's first column sits on a 16-byte
// boundary.  Rows whose width is a multiple of 4 use 128-bit loads, stores
// and shared-memory reads; other widths take the scalar path.
__device__ __forceinline__ void jacobi_tile(const BatchParams& P, const BatchRegion& R, int64_t t,
                                            float* halo) {
    constexpr int HW = kBatchJacCols + 8;
    const int64_t band = t / R.tiles_c, tc = t - band * R.tiles_c;
    const int64_t r0 = R.lb + band * P.jac_rows;
    const int nr = (int)min((int64_t)P.jac_rows, R.lb + R.trip - r0);
    const int64_t c0 = tc * kBatchJacCols;
    const int64_t cols = R.cols;
    const float* u = R.in0;
    const bool vec = (cols & 3) == 0 && ((reinterpret_cast<uintptr_t>(u) | reinterpret_cast<uintptr_t>(R.out)) & 15) == 0;
    if (vec) {
        // all of this thread's loads are issued before any shared-memory
        // store, so their DRAM latencies overlap instead of adding up
        constexpr int kMaxLd = ((kBatchMaxJacRows + 2) * (HW / 4) + kBatchUnits - 1) / kBatchUnits;
        const int n4 = (nr + 2) * (HW / 4);
        float4 v[kMaxLd];
#pragma unroll
        for (int k = 0; k < kMaxLd; ++k) {
            const int idx = threadIdx.x + k * kBatchUnits;
            v[k] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (idx < n4) {
                const int i = idx / (HW / 4), q = idx - i * (HW / 4);
                const int64_t rr = r0 - 1 + i, cc = c0 - 4 + 4 * q;
                if (cc >= 0 && cc + 3 < cols) v[k] = __ldcs(reinterpret_cast<const float4*>(u + rr * cols + cc));
            }
        }
#pragma unroll
        for (int k = 0; k < kMaxLd; ++k) {
            const int idx = threadIdx.x + k * kBatchUnits;
            if (idx < n4) *reinterpret_cast<float4*>(halo + 4 * idx) = v[k];
        }
    } else {
        for (int idx = threadIdx.x; idx < (nr + 2) * HW; idx += blockDim.x) {
            const int i = idx / HW, j = idx - i * HW;
            const int64_t rr = r0 - 1 + i, cc = c0 - 4 + j;
            halo[idx] = (cc >= 0 && cc < cols) ? u[rr * cols + cc] : 0.0f;
        }
    }
    __syncthreads();
    float racc = R.fop == UPIR_RED_MIN ? __int_as_float(0x7f800000) : -__int_as_float(0x7f800000);
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5, nty = blockDim.x >> 5;
    const int64_t c = c0 + 4 * tx;
    const bool full = vec && c >= 1 && c + 3 <= cols - 2;
    for (int i = ty; i < nr; i += nty) {
        const float* cen = halo + (i + 1) * HW + 4 + 4 * tx;
        const float4 C = *reinterpret_cast<const float4*>(cen);
        const float4 N = *reinterpret_cast<const float4*>(cen - HW);
        const float4 S = *reinterpret_cast<const float4*>(cen + HW);
        const float Wl = cen[-1], Er = cen[4];
        float vs[4], cs[4] = {C.x, C.y, C.z, C.w};
        vs[0] = __fmul_rn(0.25f, __fadd_rn(__fadd_rn(N.x, S.x), __fadd_rn(Wl, C.y)));
        vs[1] = __fmul_rn(0.25f, __fadd_rn(__fadd_rn(N.y, S.y), __fadd_rn(C.x, C.z)));
        vs[2] = __fmul_rn(0.25f, __fadd_rn(__fadd_rn(N.z, S.z), __fadd_rn(C.y, C.w)));
        vs[3] = __fmul_rn(0.25f, __fadd_rn(__fadd_rn(N.w, S.w), __fadd_rn(C.z, Er)));
        float* out = R.out + (r0 + i) * cols + c;
        if (full) {
            __stcs(reinterpret_cast<float4*>(out), make_float4(vs[0], vs[1], vs[2], vs[3]));
            if (R.fop)
#pragma unroll
                for (int j = 0; j < 4; ++j) racc = fold(racc, fabsf(__fsub_rn(vs[j], cs[j])), R.fop);
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (c + j >= 1 && c + j <= cols - 2) {
                    out[j] = vs[j];
                    if (R.fop) racc = fold(racc, fabsf(__fsub_rn(vs[j], cs[j])), R.fop);
                }
            }
        }
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

__global__ void __launch_bounds__(kBatchUnits, 4) batch_persistent_kernel(const BatchParams P) {
    __shared__ __align__(16) float halo[(kBatchMaxJacRows + 2) * (kBatchJacCols + 8)];
    __shared__ int64_t item, next_item;
    __shared__ int last_team;
    griddep_wait();
    if (threadIdx.x == 0) item = (int64_t)atomicAdd(P.counter, 1ull);
    __syncthreads();
    for (;;) {
        const int64_t k = item;
        if (k >= P.nitems) break;
        // claim the following item now, so the atomic's latency overlaps this one
        if (threadIdx.x == 0) next_item = (int64_t)atomicAdd(P.counter, 1ull);
        const int2 it = P.items[k];
        const BatchRegion& R = P.regions[it.x];
        switch (R.op) {
            case BOP_AXPY: axpy_tile(P, R, it.y); break;
            case BOP_JACOBI: jacobi_tile(P, R, it.y, halo); break;
            default: matvec_tile(P, R, it.y); break;
        }
        __syncthreads();  // every thread has read `item`
        if (threadIdx.x == 0) item = next_item;
        __syncthreads();
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
