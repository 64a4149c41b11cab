// FP32 SIMT matrix multiplication C = A B (the matrix multiplication workload
// of §6) and the bfloat16 operand split used by the tensor-core bodies.
// GEMM: the loop over the rows of C (collapse 2 with its columns) is tiled in
// 128 x 128 output tiles; the tile loop is workshared over teams.  Each thread
// accumulates an 8 x 8 block with FMA in increasing k.
#include <cuda_bf16.h>

#include "device_common.cuh"

namespace upir {

namespace {

constexpr int BM = 128, BN = 128, BK = 16;
constexpr int AP = BM + 4;  // A tile pitch: the transposing stores of 16 k per row hit distinct banks

__global__ void __launch_bounds__(256, 2) gemm_f32_kernel(const GemmParams p) {
    __shared__ __align__(16) float As[2][BK][AP];
    __shared__ __align__(16) float Bs[2][BK][BN];
    const int t = threadIdx.x;
    const int tx = t % 16, ty = t / 16;
    const int64_t rows = p.row_ub - p.row_lb;
    const int64_t tiles_m = (rows + BM - 1) / BM, tiles_n = (p.N + BN - 1) / BN;
    const int64_t ntiles = tiles_m * tiles_n;
    // 128-bit loads of A rows (along k) and B rows (along n) when rows start
    // on 16-byte boundaries; element loads otherwise and at the edges
    const bool vec_a = (p.K & 3) == 0 && (reinterpret_cast<uintptr_t>(p.A) & 15) == 0;
    const bool vec_b = (p.N & 3) == 0 && (reinterpret_cast<uintptr_t>(p.B) & 15) == 0;

    auto do_tile = [&](int64_t tile) {
        const int64_t m0 = p.row_lb + (tile / tiles_n) * BM;
        const int64_t n0 = (tile % tiles_n) * BN;
        float acc[8][8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;

        // per k-tile each thread moves two groups of 4 of A (row f / 4, k
        // 4 (f % 4) ..) and two of B (k f / 32, columns 4 (f % 32) ..), f = t + 256 i
        float4 ra[2], rb[2];
        auto load_regs = [&](int64_t k0) {
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int f = t + i * 256;
                const int64_t gm = m0 + (f >> 2), gk = k0 + 4 * (f & 3);
                const float* pa = p.A + gm * p.K + gk;
                if (vec_a && gm < p.row_ub && gk + 3 < p.K) {
                    ra[i] = __ldg(reinterpret_cast<const float4*>(pa));
                } else {
                    const bool rin = gm < p.row_ub;
                    ra[i] = make_float4(rin && gk < p.K ? pa[0] : 0.f, rin && gk + 1 < p.K ? pa[1] : 0.f,
                                        rin && gk + 2 < p.K ? pa[2] : 0.f, rin && gk + 3 < p.K ? pa[3] : 0.f);
                }
                const int64_t gkb = k0 + (f >> 5), gn = n0 + 4 * (f & 31);
                const float* pb = p.B + gkb * p.N + gn;
                if (vec_b && gkb < p.K && gn + 3 < p.N) {
                    rb[i] = __ldg(reinterpret_cast<const float4*>(pb));
                } else {
                    const bool kin = gkb < p.K;
                    rb[i] = make_float4(kin && gn < p.N ? pb[0] : 0.f, kin && gn + 1 < p.N ? pb[1] : 0.f,
                                        kin && gn + 2 < p.N ? pb[2] : 0.f, kin && gn + 3 < p.N ? pb[3] : 0.f);
                }
            }
        };
        auto store_regs = [&](int buf) {
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int f = t + i * 256;
                const int r = f >> 2, kq = 4 * (f & 3);
                As[buf][kq + 0][r] = ra[i].x;
                As[buf][kq + 1][r] = ra[i].y;
                As[buf][kq + 2][r] = ra[i].z;
                As[buf][kq + 3][r] = ra[i].w;
                *reinterpret_cast<float4*>(&Bs[buf][f >> 5][4 * (f & 31)]) = rb[i];
            }
        };

        const int64_t nk = (p.K + BK - 1) / BK;
        load_regs(0);
        store_regs(0);
        __syncthreads();
        for (int64_t kt = 0; kt < nk; ++kt) {
            const int buf = kt & 1;
            if (kt + 1 < nk) load_regs((kt + 1) * BK);
#pragma unroll
            for (int k = 0; k < BK; ++k) {
                float a[8], b[8];
                const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][k][ty * 4]);
                const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][k][64 + ty * 4]);
                const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][k][tx * 4]);
                const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][k][64 + tx * 4]);
                a[0] = a0.x; a[1] = a0.y; a[2] = a0.z; a[3] = a0.w;
                a[4] = a1.x; a[5] = a1.y; a[6] = a1.z; a[7] = a1.w;
                b[0] = b0.x; b[1] = b0.y; b[2] = b0.z; b[3] = b0.w;
                b[4] = b1.x; b[5] = b1.y; b[6] = b1.z; b[7] = b1.w;
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) acc[i][j] = __fmaf_rn(a[i], b[j], acc[i][j]);
            }
            if (kt + 1 < nk) store_regs(buf ^ 1);
            __syncthreads();
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int64_t gm = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
            if (gm >= p.row_ub) continue;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int64_t gn = n0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4));
                if (gn < p.N) p.C[gm * p.N + gn] = acc[i][j];
            }
        }
    };

    if (p.sched == UPIR_SCHED_DYNAMIC) {
        __shared__ int64_t next;
        for (;;) {
            if (t == 0) next = (int64_t)atomicAdd(p.sc.chunk_counter, 1ull);
            __syncthreads();
            const int64_t j = next;
            __syncthreads();
            int64_t t0, t1;
            if (!dyn_chunk(p.sc, p.chunk, ntiles, j, t0, t1)) break;
            for (int64_t tile = t0; tile < t1; ++tile) do_tile(tile);
        }
        __shared__ int last;
        __syncthreads();
        if (t == 0) {
            __threadfence();
            last = atomicAdd(p.sc.ticket, 1u) == gridDim.x - 1;
            if (last) {
                *p.sc.ticket = 0;
                *p.sc.chunk_counter = 0;
            }
        }
    } else {
        static_ranges(p.sk, ntiles, p.chunk, gridDim.x, blockIdx.x, [&](int64_t t0, int64_t t1) {
            for (int64_t tile = t0; tile < t1; ++tile) do_tile(tile);
        });
    }
}

// hi = bf16(src), lo = bf16(src - hi), optionally transposed through a 32 x 32
// shared-memory tile so both the reads and the writes are coalesced.
__global__ void __launch_bounds__(256) split_bf16_kernel(const SplitParams p) {
    __shared__ uint16_t th[32][33], tl[32][33];
    const int64_t nrows = p.ub - p.lb;
    const int64_t tiles_c = (p.cols + 31) / 32;
    const int64_t ntiles = ((nrows + 31) / 32) * tiles_c;
    const int lx = threadIdx.x % 32, ly = threadIdx.x / 32;  // 32 x 8
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t r0 = p.lb + (tile / tiles_c) * 32, c0 = (tile % tiles_c) * 32;
        for (int i = ly; i < 32; i += 8) {
            const int64_t r = r0 + i, c = c0 + lx;
            uint16_t h = 0, l = 0;
            if (r < p.ub && c < p.cols) {
                const float v = p.src[r * p.cols + c];
                const __nv_bfloat16 hb = __float2bfloat16_rn(v);
                const __nv_bfloat16 lb = __float2bfloat16_rn(__fsub_rn(v, __bfloat162float(hb)));
                h = __bfloat16_as_ushort(hb);
                l = __bfloat16_as_ushort(lb);
                if (!p.transpose) {
                    p.hi[r * p.cols + c] = h;
                    if (p.lo) p.lo[r * p.cols + c] = l;
                }
            }
            th[i][lx] = h;
            tl[i][lx] = l;
        }
        if (p.transpose) {
            __syncthreads();
            for (int i = ly; i < 32; i += 8) {
                const int64_t c = c0 + i, r = r0 + lx;  // output row c, column r
                if (c < p.cols && r < p.ub) {
                    p.hi[c * p.rows + r] = th[lx][i];
                    if (p.lo) p.lo[c * p.rows + r] = tl[lx][i];
                }
            }
        }
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_gemm_f32(int teams, int units, const GemmParams& p, cudaStream_t s) {
    gemm_f32_kernel<<<teams, units, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_split_bf16(int teams, int units, const SplitParams& p, cudaStream_t s) {
    split_bf16_kernel<<<teams, units, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace upir
