// FP32 SIMT matrix multiplication C = A B (the matrix multiplication workload
// of §6) and the bfloat16 operand split used by the tensor-core bodies.
// GEMM: the loop over the rows of C (collapse 2 with its columns) is tiled in
// 128 x 128 output tiles; the tile loop is workshared over teams.  Each thread
// accumulates an 8 x 8 block with FMA in increasing k.  Under the planner's
// default the tiles of a last, partly filled wave are split in k: each share
// is summed in increasing k as above, and the last team to finish the tile
// adds the shares in share order (so the result does not depend on timing).
// Two kernels share this: one fed by TMA (16 x 128 and 128 x 16 boxes into a
// four-stage ring, edges zero-filled; rows and widths whose starts are
// 16-byte aligned), and one that stages 128-bit loads through registers into
// a transposed A tile (any shape).
#include <cuda_bf16.h>

#include "device_common.cuh"

namespace upir {

namespace {

constexpr int BM = 128, BN = 128, BK = 16;
constexpr int AP = BM + 4;  // A tile pitch: the transposing stores of 16 k per row hit distinct banks

// The team's work items: whole tiles (static ranges or dynamic chunks of the
// tile loop) or, for a split loop, the one item of the team (a whole tile or
// one share of k tiles of a split tile).  tile(t, kt0, kt1, part) runs k
// tiles [kt0, kt1) of output tile t (part < 0: the whole tile) and returns
// false when the team has to stop (a bounded wait ran out).
template <class F>
__device__ __forceinline__ void gemm_f32_work(const GemmParams& p, int64_t ntiles, int64_t nk, F&& tile) {
    if (p.sched == UPIR_SCHED_DYNAMIC) {
        __shared__ int64_t next;
        for (bool go = true; go;) {
            if (threadIdx.x == 0) next = (int64_t)atomicAdd(p.sc.chunk_counter, 1ull);
            __syncthreads();
            const int64_t j = next;
            __syncthreads();
            int64_t t0, t1;
            if (!dyn_chunk(p.sc, p.chunk, ntiles, j, t0, t1)) break;
            for (int64_t t = t0; t < t1 && go; ++t) go = tile(t, 0, nk, -1);
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
    } else if (p.kparts > 1) {
        const int64_t b = blockIdx.x;
        if (b < p.whole) {
            tile(b, 0, nk, -1);
        } else {
            const int64_t u = b - p.whole;
            const int part = (int)(u % p.kparts);
            tile(p.whole + u / p.kparts, nk * part / p.kparts, nk * (part + 1) / p.kparts, part);
        }
    } else {
        bool go = true;
        static_ranges(p.sk, ntiles, p.chunk, gridDim.x, blockIdx.x, [&](int64_t t0, int64_t t1) {
            for (int64_t t = t0; t < t1 && go; ++t) go = tile(t, 0, nk, -1);
        });
    }
}

// A share of a split tile goes to `work` (element e of thread t at slot
// e * 256 + t); the last share of the tile to arrive reads all shares back and
// leaves their sum, in share order, in acc.  False for the other shares.
__device__ __forceinline__ bool gemm_f32_meet_shares(const GemmParams& p, int64_t tile, int part,
                                                     float (&acc)[8][8]) {
    const int t = threadIdx.x;
    const int64_t st = tile - p.whole;
    float* w = p.work + (st * p.kparts + part) * (int64_t)(BM * BN);
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) __stcg(w + (i * 8 + j) * 256 + t, acc[i][j]);
    __shared__ int last_share;
    __threadfence();
    __syncthreads();
    if (t == 0) {
        const unsigned got = atomicAdd(p.tile_tickets + st, 1u);
        last_share = got == (unsigned)p.kparts - 1;
        if (last_share) p.tile_tickets[st] = 0;  // ready for the next submission
    }
    __syncthreads();
    if (!last_share) return false;
    __threadfence();
    const float* w0 = p.work + st * p.kparts * (int64_t)(BM * BN);
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int e = (i * 8 + j) * 256 + t;
            float v = __ldcg(w0 + e);
            for (int q = 1; q < p.kparts; ++q) v = __fadd_rn(v, __ldcg(w0 + (int64_t)q * BM * BN + e));
            acc[i][j] = v;
        }
    return true;
}

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

    const int64_t nk = (p.K + BK - 1) / BK;
    // k tiles [kt0, kt1) of the tile; part >= 0: a share of a split tile
    auto do_tile = [&](int64_t tile, int64_t kt0, int64_t kt1, int part) {
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

        if (kt0 < kt1) {
            load_regs(kt0 * BK);
            store_regs(0);
        }
        __syncthreads();
        for (int64_t kt = kt0; kt < kt1; ++kt) {
            const int buf = (kt - kt0) & 1;
            if (kt + 1 < kt1) load_regs((kt + 1) * BK);
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
            if (kt + 1 < kt1) store_regs(buf ^ 1);
            __syncthreads();
        }
        if (part >= 0 && !gemm_f32_meet_shares(p, tile, part, acc)) return;
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

    gemm_f32_work(p, ntiles, nk, [&](int64_t tile, int64_t kt0, int64_t kt1, int part) {
        do_tile(tile, kt0, kt1, part);
        return true;
    });
}

constexpr int kTS = 4;                             // TMA ring stages (a power of two)
constexpr int kStageFloats = BM * BK + BK * BN;    // A [128 rows][16 k], then B [16 k][128 columns]
constexpr uint32_t kStageBytes = kStageFloats * 4;

// The TMA-fed kernel.  Thread (tx, ty) = (t % 16, t / 16) owns rows ty + 16 i
// (i < 8) and columns 4 tx .. 4 tx + 3 and 64 + 4 tx .. of the tile: the two
// rows a warp reads at once are 64 bytes apart, in different banks, and A is
// read as 128-bit loads along k.  Thread 0 keeps up to four k tiles in flight;
// the team barrier that closes a k tile frees its stage for the next copy.
__global__ void __launch_bounds__(256, 2) gemm_f32_tma_kernel(const GemmParams p,
                                                              const __grid_constant__ CUtensorMap tm_a,
                                                              const __grid_constant__ CUtensorMap tm_b) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar[kTS];
    float* ring = smem_align1k<float>(smem_raw);
    const int t = threadIdx.x;
    const int tx = t % 16, ty = t / 16;
    const int64_t rows = p.row_ub - p.row_lb;
    const int64_t tiles_n = (p.N + BN - 1) / BN;
    const int64_t ntiles = ((rows + BM - 1) / BM) * tiles_n;
    const int64_t nk = (p.K + BK - 1) / BK;
    if (t == 0) {
        prefetch_tmap(&tm_a);
        prefetch_tmap(&tm_b);
#pragma unroll
        for (int s = 0; s < kTS; ++s) mbar_init(&bar[s], 1);
        fence_mbar_init();
    }
    __syncthreads();

    uint32_t used = 0;    // k tiles this team has consumed; k tile q sits in stage q % kTS
    uint32_t issued = 0;  // thread 0: k tiles whose copies it has issued
    auto issue = [&](int64_t m0, int64_t n0, int64_t kt) {
        const int s = (int)(issued % kTS);
        float* st = ring + s * kStageFloats;
        mbar_arrive_expect_tx(&bar[s], kStageBytes);
        tma_load_2d(st, &tm_a, &bar[s], (int32_t)(kt * BK), (int32_t)m0);
        tma_load_2d(st + BM * BK, &tm_b, &bar[s], (int32_t)n0, (int32_t)(kt * BK));
        ++issued;
    };

    gemm_f32_work(p, ntiles, nk, [&](int64_t tile, int64_t kt0, int64_t kt1, int part) -> bool {
        const int64_t m0 = p.row_lb + (tile / tiles_n) * BM;
        const int64_t n0 = (tile % tiles_n) * BN;
        // acc2[i][q]: columns 2q, 2q + 1 of the thread's eight in row i, one
        // paired FMA (each lane rounded once, like fmaf) per pair and k
        F2 acc2[8][4];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc2[i][q] = f2(0.0f, 0.0f);
        const int64_t n = kt1 - kt0;
        if (t == 0)
            for (int64_t j = 0; j < n && j < kTS; ++j) issue(m0, n0, kt0 + j);
        for (int64_t j = 0; j < n; ++j) {
            const int s = (int)(used % kTS);
            const bool ok = mbar_wait_bounded(&bar[s], (used / kTS) & 1u, p.spin_limit, p.err_word);
            if (ok) {
                const float* As = ring + s * kStageFloats;
                const float* Bs = As + BM * BK;
#pragma unroll 1
                for (int k2 = 0; k2 < BK; k2 += 2) {
                    float2 a2[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        a2[i] = *reinterpret_cast<const float2*>(As + (ty + 16 * i) * BK + k2);
#pragma unroll
                    for (int kk = 0; kk < 2; ++kk) {
                        const ulonglong2 b0 = *reinterpret_cast<const ulonglong2*>(Bs + (k2 + kk) * BN + 4 * tx);
                        const ulonglong2 b1 =
                            *reinterpret_cast<const ulonglong2*>(Bs + (k2 + kk) * BN + 64 + 4 * tx);
                        const F2 b[4] = {{b0.x}, {b0.y}, {b1.x}, {b1.y}};
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const float a = kk == 0 ? a2[i].x : a2[i].y;
                            const F2 aa = f2(a, a);
#pragma unroll
                            for (int q = 0; q < 4; ++q) acc2[i][q] = f2_fma(aa, b[q], acc2[i][q]);
                        }
                    }
                }
            }
            if (__syncthreads_or(!ok)) {
                // copies still in flight get a bounded chance to land before
                // the shared memory is released
                if (t == 0)
                    for (uint32_t q = used; q != issued; ++q)
                        mbar_wait_bounded(&bar[q % kTS], (q / kTS) & 1u, p.spin_limit, nullptr);
                return false;
            }
            ++used;
            if (t == 0 && j + kTS < n) issue(m0, n0, kt0 + j + kTS);
        }
        float acc[8][8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int q = 0; q < 4; ++q) f2_split(acc2[i][q], acc[i][2 * q], acc[i][2 * q + 1]);
        if (part >= 0 && !gemm_f32_meet_shares(p, tile, part, acc)) return true;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int64_t gm = m0 + ty + 16 * i;
            if (gm >= p.row_ub) continue;
            float* crow = p.C + gm * p.N;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int64_t gn = n0 + 64 * h + 4 * tx;
                if (gn + 3 < p.N) {
                    *reinterpret_cast<float4*>(crow + gn) =
                        make_float4(acc[i][4 * h], acc[i][4 * h + 1], acc[i][4 * h + 2], acc[i][4 * h + 3]);
                } else {
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if (gn + q < p.N) crow[gn + q] = acc[i][4 * h + q];
                }
            }
        }
        return true;
    });
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

cudaError_t launch_gemm_f32_tma(int teams, const GemmParams& p, const CUtensorMap* tm, cudaStream_t s) {
    const size_t smem = kTS * (size_t)kStageBytes + 1024;  // + slack to align the ring to 1 KB
    static bool attr = false;
    if (!attr) {
        const cudaError_t e = cudaFuncSetAttribute(gemm_f32_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    gemm_f32_tma_kernel<<<teams, 256, smem, s>>>(p, tm[0], tm[1]);
    return cudaGetLastError();
}

cudaError_t launch_split_bf16(int teams, int units, const SplitParams& p, cudaStream_t s) {
    split_bf16_kernel<<<teams, units, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace upir
