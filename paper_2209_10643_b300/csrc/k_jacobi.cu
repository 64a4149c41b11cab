// Tiled 5-point Jacobi sweep (the 2D stencil workload of §6, 5-point form).
// The canonical loop collapse(2) over the interior is tiled by the runtime
// (tiling is one of the loop transformations the separation of loop and
// loop_parallel allows, §3.2) and the tile loop is workshared over teams.
// Each team stages a (TM + 2) x (TN + 8) halo box of u_in into shared memory
// with one TMA copy, computes TM x TN points from it and writes them with
// 128-bit stores.  The per-sweep max-norm residual is folded into the
// reduction variable with one atomic per team (max/min are exact in any
// order, so the result does not depend on the team order).
#include <cstring>

#include "device_common.cuh"

namespace upir {

namespace {

// maxNum / minNum folded into *addr; NaN operands are ignored.
__device__ __forceinline__ void atomic_fold_minmax(float* addr, float v, int op) {
    if (isnan(v)) return;
    int* ai = reinterpret_cast<int*>(addr);
    int old = *reinterpret_cast<volatile int*>(ai);
    for (;;) {
        const float of = __int_as_float(old);
        const bool better = op == UPIR_RED_MAX ? (v > of) : (v < of);
        if (!isnan(of) && !better) return;
        const int prev = atomicCAS(ai, old, __float_as_int(v));
        if (prev == old) return;
        old = prev;
    }
}

__device__ __forceinline__ float fold(float a, float b, int op) {
    return op == UPIR_RED_MIN ? fminf(a, b) : fmaxf(a, b);
}

__device__ __forceinline__ float block_fold(float v, int op) {
    __shared__ float part[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) v = fold(v, __shfl_xor_sync(0xffffffffu, v, m), op);
    if (lane == 0) part[warp] = v;
    __syncthreads();
    if (warp == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        float q = lane < nw ? part[lane] : v;
#pragma unroll
        for (int m = 16; m >= 1; m >>= 1) q = fold(q, __shfl_xor_sync(0xffffffffu, q, m), op);
        v = q;
    }
    return v;  // valid in thread 0
}

__global__ void __launch_bounds__(1024) jacobi_tma_kernel(const JacobiParams p,
                                                         const __grid_constant__ CUtensorMap tmap) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // the TMA destination starts on a 1024-byte boundary (the launch adds 1 KB of slack)
    float* tile = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ __align__(8) uint64_t bar;
    __shared__ int64_t next_tile;
    const int TM = p.tile_m, TN = p.tile_n, SW = TN + 8;
    const int tpr = TN / 4;                    // threads per tile row (4 columns each)
    const int tx = threadIdx.x % tpr, ty = threadIdx.x / tpr;
    const int nty = blockDim.x / tpr;          // thread rows
    const bool active = threadIdx.x < nty * tpr;
    const uint32_t box_bytes = (uint32_t)((TM + 2) * SW * sizeof(float));
    const bool has_red = p.rvar != nullptr;
    float racc = p.rop == UPIR_RED_MIN ? __int_as_float(0x7f800000) : -__int_as_float(0x7f800000);

    if (threadIdx.x == 0) {
        prefetch_tmap(&tmap);
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t phase = 0;
    bool failed = false;

    auto do_tile = [&](int64_t t) -> bool {
        const int64_t tr = t / p.tiles_c, tc = t % p.tiles_c;
        const int64_t r0 = p.r_lb + tr * TM;
        const int64_t c0 = tc * TN;
        if (threadIdx.x == 0) {
            mbar_arrive_expect_tx(&bar, box_bytes);
            tma_load_2d(tile, &tmap, &bar, (int32_t)(c0 - 4), (int32_t)(r0 - 1));
        }
        const bool ok = __syncthreads_and(mbar_wait_bounded(&bar, phase, p.spin_limit, p.err_word));
        phase ^= 1u;
        if (!ok) return false;
        if (active) {
            const int64_t rend = min(r0 + TM, p.r_ub);
            for (int i = ty; r0 + i < rend; i += nty) {
                const float* cen = tile + (i + 1) * SW + 4 + 4 * tx;
                const float4 C = *reinterpret_cast<const float4*>(cen);
                const float4 N = *reinterpret_cast<const float4*>(cen - SW);
                const float4 S = *reinterpret_cast<const float4*>(cen + SW);
                const float Wl = cen[-1], Er = cen[4];
                float4 v;
                v.x = __fmul_rn(0.25f, __fadd_rn(__fadd_rn(N.x, S.x), __fadd_rn(Wl, C.y)));
                v.y = __fmul_rn(0.25f, __fadd_rn(__fadd_rn(N.y, S.y), __fadd_rn(C.x, C.z)));
                v.z = __fmul_rn(0.25f, __fadd_rn(__fadd_rn(N.z, S.z), __fadd_rn(C.y, C.w)));
                v.w = __fmul_rn(0.25f, __fadd_rn(__fadd_rn(N.w, S.w), __fadd_rn(C.z, Er)));
                const int64_t c = c0 + 4 * tx;
                const int64_t r = r0 + i;
                float* out = p.uout + r * p.cols + c;
                if (c >= 1 && c + 3 <= p.cols - 2) {
                    __stcs(reinterpret_cast<float4*>(out), v);
                    if (has_red) {
                        racc = fold(racc, fabsf(__fsub_rn(v.x, C.x)), p.rop);
                        racc = fold(racc, fabsf(__fsub_rn(v.y, C.y)), p.rop);
                        racc = fold(racc, fabsf(__fsub_rn(v.z, C.z)), p.rop);
                        racc = fold(racc, fabsf(__fsub_rn(v.w, C.w)), p.rop);
                    }
                } else {
                    const float vs[4] = {v.x, v.y, v.z, v.w};
                    const float cs[4] = {C.x, C.y, C.z, C.w};
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        if (c + j >= 1 && c + j <= p.cols - 2) {
                            out[j] = vs[j];
                            if (has_red) racc = fold(racc, fabsf(__fsub_rn(vs[j], cs[j])), p.rop);
                        }
                    }
                }
            }
        }
        __syncthreads();  // the next copy overwrites the tile
        return true;
    };

    if (p.sched == UPIR_SCHED_DYNAMIC) {
        const int64_t c = p.chunk > 0 ? p.chunk : 1;
        const int64_t nchunks = (p.ntiles + c - 1) / c;
        for (;;) {
            if (threadIdx.x == 0) next_tile = (int64_t)atomicAdd(p.sc.chunk_counter, 1ull);
            __syncthreads();
            const int64_t j = next_tile;
            __syncthreads();
            if (j >= nchunks) break;
            for (int64_t t = j * c; t < min(j * c + c, p.ntiles) && !failed; ++t) failed = !do_tile(t);
            if (failed) break;
        }
    } else {
        static_ranges(p.ntiles, p.chunk, gridDim.x, blockIdx.x, [&](int64_t t0, int64_t t1) {
            for (int64_t t = t0; t < t1 && !failed; ++t) failed = !do_tile(t);
        });
    }

    if (has_red && !failed) {
        const float b = block_fold(racc, p.rop);
        if (threadIdx.x == 0) atomic_fold_minmax(p.rvar, b, p.rop);
    }
    if (p.sched == UPIR_SCHED_DYNAMIC) {
        // the last team returns the tile counter to zero for the next launch
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
    }
    if (failed && threadIdx.x == 0) {
        // give a copy still in flight a bounded chance to land before the
        // shared memory is released
        mbar_wait_bounded(&bar, phase ^ 1u, p.spin_limit, nullptr);
    }
}

}  // namespace

size_t jacobi_tma_smem_bytes(int tile_m, int tile_n) {
    return (size_t)(tile_m + 2) * (tile_n + 8) * sizeof(float);
}

cudaError_t launch_jacobi_tma(int teams, int units, const JacobiParams& p, const void* tmap,
                              cudaStream_t s) {
    const size_t smem = jacobi_tma_smem_bytes(p.tile_m, p.tile_n) + 1024;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(jacobi_tma_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, 201 * 1024);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    CUtensorMap m;
    memcpy(&m, tmap, sizeof(m));
    jacobi_tma_kernel<<<teams, units, smem, s>>>(p, m);
    return cudaGetLastError();
}

}  // namespace upir
