// Tensor-core GEMM bodies (the matrix multiplication workload of §6) on the
// 5th-generation tensor cores: C = A B with bfloat16 operands and FP32
// accumulation (GEMM_BF16), and the split form C = A_hi B_hi + A_hi B_lo +
// A_lo B_hi (GEMM_BF16X3) that recovers most of FP32's accuracy.
//
// The loop over the rows of C (collapse 2 with its columns) is tiled in
// 128 x 256 output tiles and the tile loop is workshared statically over
// persistent teams, one per SM.  Each team is warp-specialised:
//   warp 0      one thread issues TMA copies of the A and B^T k-blocks
//               (128 x BK and 256 x BK bfloat16, BK = 64 with the 128-byte
//               swizzle, or 32 with the 64-byte swizzle for the split form)
//               into a 4-stage shared-memory ring (full/empty mbarriers);
//   warp 1      allocates 512 TMEM columns (two 128 x 256 FP32 accumulators)
//               and one thread issues tcgen05.mma (M=128, N=256, K=16) from
//               shared-memory descriptors, committing each stage back to the
//               producer and each finished tile to the epilogue;
//   warps 2..17 read the accumulator with tcgen05.ld (32 rows x 64 columns
//               per warp) and release the buffer, so the MMAs of the next
//               K segment (or tile) overlap this epilogue work.
// K is accumulated in segments of seg_kb k-blocks: each segment starts a
// fresh TMEM accumulator and the epilogue adds the segments in FP32 registers
// (round to nearest, in segment order).  The split form uses segments of 1024
// by default; the plain bfloat16 form one segment, its error being dominated
// by the rounding of its operands to bfloat16.  The tensor core's own accumulation is not
// round-to-nearest, so its error grows with the number of accumulation steps;
// cutting the chain at every 1024 values of K keeps it near FP32 rounding.
// Every mbarrier wait is bounded: when one runs out the team records the
// timeout in the device error word, lets copies and MMAs in flight land
// (again bounded), frees its TMEM and returns.
#include <cstring>

#include "device_common.cuh"
#include "runtime_internal.h"

namespace upir {

namespace {

constexpr int TC_BM = 128, TC_BN = 256;
constexpr int TC_THREADS = 576;  // producer warp, MMA warp, 16 epilogue warps
constexpr int TC_EPI_THREADS = 512;
constexpr int TC_EPI_COLS = 64;  // accumulator columns per epilogue warp
constexpr int kSegK = 1024;      // default K per accumulation segment of the split form
constexpr uint32_t TC_TMEM_COLS = 512;

struct TcParams {
    float* C;
    int64_t M, N, K;
    int64_t row_lb, row_ub;
    int64_t tiles_m, tiles_n, ntiles;
    int64_t chunk;
    SchedConst sk;
    long long spin_limit;
    int* err_word;
    int seg_kb;  // k-blocks per accumulation segment
    // work units: full tiles first, then `split_tiles` tiles cut into `parts`
    // contiguous K ranges; parts > 0 land in `work`, added to C afterwards
    int64_t full_tiles, split_tiles, nunits;
    int parts;
    float* work;
};

struct TcUnit {
    int64_t tile;
    int kb0, kb1, part;
    int64_t split_idx;
};

__device__ __forceinline__ TcUnit tc_unit(int64_t u, const TcParams& p, int nkb) {
    if (u < p.full_tiles) return TcUnit{u, 0, nkb, 0, -1};
    const int64_t v = u - p.full_tiles;
    const int64_t si = v / p.parts;
    const int part = (int)(v - si * p.parts);
    return TcUnit{p.full_tiles + si, (int)((int64_t)part * nkb / p.parts),
                  (int)((int64_t)(part + 1) * nkb / p.parts), part, si};
}

// Per variant: bfloat16 uses 64-wide k-blocks (one 128-byte swizzled row,
// 4 stages); the split form, three MMAs per k-step, uses 32-wide k-blocks
// (64-byte swizzle, 4 stages of four operand tiles).
template <bool X3>
struct TcCfg {
    static constexpr int BK = X3 ? 32 : 64;
    static constexpr int ROW_BYTES = BK * 2;                 // swizzle width
    static constexpr uint32_t SBO = 8 * ROW_BYTES;           // 8-row swizzle atom
    static constexpr uint64_t LAYOUT = X3 ? 4 : 2;           // 64- or 128-byte swizzle
    static constexpr int A_BYTES = TC_BM * BK * 2;
    static constexpr int B_BYTES = TC_BN * BK * 2;
    static constexpr int STAGES = 4;
    static constexpr int STAGE_BYTES = X3 ? 2 * (A_BYTES + B_BYTES) : (A_BYTES + B_BYTES);
    static constexpr size_t SMEM = (size_t)STAGES * STAGE_BYTES + 1024;
};

// kind::f16 instruction descriptor: FP32 accumulator, bfloat16 A and B, both
// K-major, M = 128, N = 256.
constexpr uint32_t tc_idesc() {
    return (1u << 4)                        // D format: FP32
           | (1u << 7)                      // A format: BF16
           | (1u << 10)                     // B format: BF16
           | ((uint32_t)(TC_BN >> 3) << 17) // N / 8
           | ((uint32_t)(TC_BM >> 4) << 24);// M / 16
}

// Shared-memory matrix descriptor of a K-major operand tile written by TMA
// with a 64- or 128-byte swizzle: rows of ROW_BYTES, 8-row swizzle atoms
// stacked along M/N, so the stride between atoms is 8 * ROW_BYTES.
template <class Cfg>
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);   // start address
    d |= (uint64_t)(16u >> 4) << 16;            // leading byte offset (unused for these layouts)
    d |= (uint64_t)(Cfg::SBO >> 4) << 32;       // stride byte offset
    d |= (uint64_t)1 << 46;                     // descriptor version
    d |= Cfg::LAYOUT << 61;                     // swizzle mode
    return d;
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                       uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                   "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Bounded wait that also gives up as soon as another role has given up.
__device__ __forceinline__ bool tc_wait(uint64_t* bar, uint32_t parity, const TcParams& p,
                                        volatile int* abort_flag) {
    for (long long n = 0; n < p.spin_limit; ++n) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((n & 255) == 255 && *abort_flag) return false;
    }
    atomicCAS(p.err_word, 0, UPIR_ERR_WAIT_TIMEOUT);
    *abort_flag = 1;
    return false;
}

// Work units of this team under the loop's static schedule, in order.
struct TcTiles {
    int64_t next, end, chunk_j;
};

__device__ __forceinline__ int64_t tc_next_tile(TcTiles& it, const TcParams& p) {
    if (it.next < it.end) return it.next++;
    if (p.chunk > 0 && it.chunk_j < p.sk.nchunks) {
        it.next = it.chunk_j * p.chunk;
        it.end = min(it.next + p.chunk, p.nunits);
        it.chunk_j += gridDim.x;
        return it.next++;
    }
    return -1;
}

__device__ __forceinline__ TcTiles tc_first(const TcParams& p) {
    TcTiles it{0, 0, (int64_t)blockIdx.x};
    if (p.chunk == 0) {
        const int64_t w = blockIdx.x;
        it.next = w * p.sk.base + min(w, p.sk.extra);
        it.end = it.next + p.sk.base + (w < p.sk.extra ? 1 : 0);
    }
    return it;
}

template <bool X3>
__global__ void __launch_bounds__(TC_THREADS, 1)
gemm_tc_kernel(const TcParams p, const __grid_constant__ CUtensorMap tm_ah,
               const __grid_constant__ CUtensorMap tm_al, const __grid_constant__ CUtensorMap tm_bh,
               const __grid_constant__ CUtensorMap tm_bl) {
    using Cfg = TcCfg<X3>;
    constexpr int S = Cfg::STAGES;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[S], empty[S], tfull[2], tempty[2], mma_done;
    __shared__ uint32_t tmem_base_sh;
    __shared__ volatile int abort_flag;
    unsigned char* ring = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nkb = (int)((p.K + Cfg::BK - 1) / Cfg::BK);

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&tfull[a], 1);
            mbar_init(&tempty[a], TC_EPI_THREADS);
        }
        mbar_init(&mma_done, 1);
        abort_flag = 0;
        fence_mbar_init();
        prefetch_tmap(&tm_ah);
        prefetch_tmap(&tm_bh);
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(&tmem_base_sh)), "r"(TC_TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = tmem_base_sh;

    auto stage_a = [&](int s) { return ring + (size_t)s * Cfg::STAGE_BYTES; };
    auto stage_b = [&](int s) { return ring + (size_t)s * Cfg::STAGE_BYTES + Cfg::A_BYTES * (X3 ? 2 : 1); };

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- producer: TMA copies into the ring ----------------
            TcTiles it = tc_first(p);
            int s = 0;
            uint32_t ph = 0;
            uint32_t issued_parity[S];
            bool issued[S];
            for (int k = 0; k < S; ++k) issued[k] = false, issued_parity[k] = 0;
            for (int64_t u = tc_next_tile(it, p); u >= 0 && !abort_flag; u = tc_next_tile(it, p)) {
                const TcUnit w = tc_unit(u, p, nkb);
                const int64_t mt = w.tile % p.tiles_m, nt = w.tile / p.tiles_m;
                const int32_t m0 = (int32_t)(p.row_lb + mt * TC_BM), n0 = (int32_t)(nt * TC_BN);
                for (int kb = w.kb0; kb < w.kb1; ++kb) {
                    if (!tc_wait(&empty[s], ph ^ 1u, p, &abort_flag)) break;
                    mbar_arrive_expect_tx(&full[s], Cfg::STAGE_BYTES);
                    const int32_t k0 = kb * Cfg::BK;
                    unsigned char* a = stage_a(s);
                    unsigned char* b = stage_b(s);
                    tma_load_2d(a, &tm_ah, &full[s], k0, m0);
                    tma_load_2d(b, &tm_bh, &full[s], k0, n0);
                    if (X3) {
                        tma_load_2d(a + Cfg::A_BYTES, &tm_al, &full[s], k0, m0);
                        tma_load_2d(b + Cfg::B_BYTES, &tm_bl, &full[s], k0, n0);
                    }
                    issued[s] = true;
                    issued_parity[s] = ph;
                    if (++s == S) s = 0, ph ^= 1u;
                }
            }
            if (abort_flag) {
                // copies in flight get a bounded chance to land before the ring is released
                for (int k = 0; k < S; ++k)
                    if (issued[k]) mbar_wait_bounded(&full[k], issued_parity[k], p.spin_limit, nullptr);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            constexpr uint32_t idesc = tc_idesc();
            TcTiles it = tc_first(p);
            int s = 0, acc = 0;
            uint32_t ph = 0, aph = 0;
            bool issued_any = false, ok = true;
            for (int64_t u = tc_next_tile(it, p); u >= 0 && ok && !abort_flag; u = tc_next_tile(it, p)) {
                const TcUnit w = tc_unit(u, p, nkb);
                for (int kb0 = w.kb0; kb0 < w.kb1 && ok; kb0 += p.seg_kb) {
                    // one K segment into a fresh accumulator buffer
                    if (!tc_wait(&tempty[acc], aph ^ 1u, p, &abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d_tmem = tmem_base + (uint32_t)(acc * TC_BN);
                    const int kb1 = min(kb0 + p.seg_kb, w.kb1);
                    for (int kb = kb0; kb < kb1; ++kb) {
                        if (!tc_wait(&full[s], ph, p, &abort_flag)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t a = smem_u32(stage_a(s)), b = smem_u32(stage_b(s));
#pragma unroll
                        for (int k = 0; k < Cfg::BK / 16; ++k) {
                            const uint32_t koff = (uint32_t)k * 32u;  // 16 bfloat16 along K
                            const uint32_t accum = (kb > kb0 || k > 0) ? 1u : 0u;
                            tc_mma(d_tmem, smem_desc<Cfg>(a + koff), smem_desc<Cfg>(b + koff), idesc, accum);
                            if (X3) {
                                tc_mma(d_tmem, smem_desc<Cfg>(a + koff), smem_desc<Cfg>(b + Cfg::B_BYTES + koff), idesc, 1u);
                                tc_mma(d_tmem, smem_desc<Cfg>(a + Cfg::A_BYTES + koff), smem_desc<Cfg>(b + koff), idesc, 1u);
                            }
                        }
                        issued_any = true;
                        tc_commit(&empty[s]);  // the stage is free once these MMAs have read it
                        if (++s == S) s = 0, ph ^= 1u;
                    }
                    if (!ok) break;
                    tc_commit(&tfull[acc]);
                    if (++acc == 2) acc = 0, aph ^= 1u;
                }
            }
            if (abort_flag && issued_any) {
                // MMAs in flight must finish before the TMEM is freed
                tc_commit(&mma_done);
                mbar_wait_bounded(&mma_done, 0, p.spin_limit, nullptr);
            }
        }
    } else {
        // ---------------- epilogue: TMEM -> FP32 registers -> C ----------------
        const int q = warp & 3;               // TMEM lane quadrant this warp may access
        const int quarter = (warp - 2) >> 2;  // which 64 of the 256 columns
        TcTiles it = tc_first(p);
        int acc = 0;
        uint32_t aph = 0;
        const bool vec_ok = (p.N % 4) == 0;
        bool ok = true;
        for (int64_t u = tc_next_tile(it, p); u >= 0 && ok && !abort_flag; u = tc_next_tile(it, p)) {
            const TcUnit w = tc_unit(u, p, nkb);
            const int nseg = (w.kb1 - w.kb0 + p.seg_kb - 1) / p.seg_kb;
            float sum[TC_EPI_COLS];
            for (int seg = 0; seg < nseg; ++seg) {
                if (!tc_wait(&tfull[acc], aph, p, &abort_flag)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t taddr = tmem_base + ((uint32_t)(32 * q) << 16) +
                                       (uint32_t)(acc * TC_BN + quarter * TC_EPI_COLS);
#pragma unroll
                for (int c = 0; c < TC_EPI_COLS / 8; ++c) {
                    float v[8];
                    tmem_ld8(taddr + (uint32_t)(c * 8), v);
#pragma unroll
                    for (int j = 0; j < 8; ++j) sum[c * 8 + j] = seg ? __fadd_rn(sum[c * 8 + j], v[j]) : v[j];
                }
                tc_fence_before();
                mbar_arrive(&tempty[acc]);
                if (++acc == 2) acc = 0, aph ^= 1u;
            }
            if (!ok) break;
            if (w.part > 0) {
                // a later K part of a split tile: to its workspace tile, added to C afterwards
                float* dst = p.work + ((w.split_idx * (p.parts - 1) + (w.part - 1)) * TC_BM + 32 * q + lane) * TC_BN +
                             quarter * TC_EPI_COLS;
#pragma unroll
                for (int c = 0; c < TC_EPI_COLS; c += 4)
                    *reinterpret_cast<float4*>(dst + c) = make_float4(sum[c], sum[c + 1], sum[c + 2], sum[c + 3]);
                continue;
            }
            const int64_t mt = w.tile % p.tiles_m, nt = w.tile / p.tiles_m;
            const int64_t row = p.row_lb + mt * TC_BM + 32 * q + lane;
            const int64_t n0 = nt * TC_BN + quarter * TC_EPI_COLS;
            if (row < p.row_ub) {
                float* crow = p.C + row * p.N;
#pragma unroll
                for (int c = 0; c < TC_EPI_COLS; c += 4) {
                    const int64_t col = n0 + c;
                    if (vec_ok && col + 4 <= p.N) {
                        __stcs(reinterpret_cast<float4*>(crow + col),
                               make_float4(sum[c], sum[c + 1], sum[c + 2], sum[c + 3]));
                    } else {
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            if (col + j < p.N) crow[col + j] = sum[c + j];
                    }
                }
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                     ::"r"(tmem_base), "r"(TC_TMEM_COLS) : "memory");
    }
}

// C += the later K parts of each split tile, in part order.
__global__ void __launch_bounds__(256) tc_fixup_kernel(const TcParams p) {
    const int64_t per_tile = (int64_t)TC_BM * TC_BN;
    const int64_t total = p.split_tiles * per_tile;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t si = e / per_tile, r = (e % per_tile) / TC_BN, c = e % TC_BN;
        const int64_t tile = p.full_tiles + si;
        const int64_t mt = tile % p.tiles_m, nt = tile / p.tiles_m;
        const int64_t row = p.row_lb + mt * TC_BM + r, col = nt * TC_BN + c;
        if (row >= p.row_ub || col >= p.N) continue;
        float v = p.C[row * p.N + col];
        for (int part = 1; part < p.parts; ++part)
            v = __fadd_rn(v, p.work[((si * (p.parts - 1) + part - 1) * TC_BM + r) * TC_BN + c]);
        p.C[row * p.N + col] = v;
    }
}

template <bool X3>
bool tc_configure() {
    static bool done = false;
    if (!done) {
        if (cudaFuncSetAttribute(gemm_tc_kernel<X3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)TcCfg<X3>::SMEM) != cudaSuccess)
            return false;
        done = true;
    }
    return true;
}

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace

// The planned parameters live in the loop record's tc_params bytes; the four
// tensor maps in its tmap[] array (A_hi, A_lo, B_hi, B_lo).
static_assert(sizeof(TcParams) <= sizeof(LoopRec::tc_params), "TcParams must fit the loop record");

upir_status plan_gemm_tc(upir_region r, LoopRec& lp, int64_t M, int64_t N, int64_t K, upir_status st) {
    if (st != UPIR_OK) return st;
    upir_ctx ctx = r->ctx;
    const bool x3 = lp.body == UPIR_BODY_GEMM_BF16X3;
    const size_t na = x3 ? 2 : 1;
    // buffers: A (hi[, lo]) [M][K] bf16, Bt (hi[, lo]) [N][K] bf16, C [M][N] FP32
    for (size_t i = 0; i < na; ++i)
        if ((int64_t)(lp.bufs[i]->bytes / 2) < M * K)
            return fail(ctx, UPIR_EINVAL, "upir_loop: GEMM A operand smaller than M x K bfloat16");
    for (size_t i = na; i < 2 * na; ++i)
        if ((int64_t)(lp.bufs[i]->bytes / 2) < N * K)
            return fail(ctx, UPIR_EINVAL, "upir_loop: GEMM B^T operand smaller than N x K bfloat16");
    if ((int64_t)(lp.bufs[2 * na]->bytes / 4) < M * N)
        return fail(ctx, UPIR_EINVAL, "upir_loop: GEMM C smaller than M x N");
    if (K % 8 != 0)
        return fail(ctx, UPIR_EUNSUPPORTED, "upir_loop: tensor-core GEMM needs K %% 8 == 0 (16-byte rows)");
    for (size_t i = 0; i < 2 * na; ++i)
        if (reinterpret_cast<uintptr_t>(lp.bufs[i]->dev) & 15)
            return fail(ctx, UPIR_EUNSUPPORTED, "upir_loop: tensor-core GEMM operands must be 16-byte aligned");
    if (r->units && r->units != TC_THREADS)
        return fail(ctx, UPIR_EUNSUPPORTED, "upir_loop: tensor-core GEMM runs with num_units 576 (or 0)");
    if (lp.sched != UPIR_SCHED_STATIC)
        return fail(ctx, UPIR_EUNSUPPORTED, "upir_loop: tensor-core GEMM tiles are scheduled statically");
    lp.kind = LK_GEMM_TC;
    lp.units = TC_THREADS;
    TcParams tp;
    memset(&tp, 0, sizeof(tp));
    tp.C = static_cast<float*>(lp.bufs[2 * na]->dev);
    tp.M = M;
    tp.N = N;
    tp.K = K;
    tp.row_lb = lp.lb;
    tp.row_ub = lp.lb + lp.trip;
    tp.tiles_m = ceil_div(lp.trip, TC_BM);
    tp.tiles_n = ceil_div(N, TC_BN);
    tp.ntiles = tp.tiles_m * tp.tiles_n;
    tp.chunk = lp.chunk;
    tp.spin_limit = ctx->spin_limit;
    tp.err_word = ctx->err_word;
    // UPIR_HINT_TILE_M on a tensor-core GEMM: k-blocks per accumulation
    // segment (64 wide for GEMM_BF16, 32 for GEMM_BF16X3).  Default: one
    // segment for GEMM_BF16 (its error is dominated by the bfloat16 rounding of
    // the operands), K = 1024 per segment for GEMM_BF16X3.
    const int bk = x3 ? TcCfg<true>::BK : TcCfg<false>::BK;
    const int nkb = (int)ceil_div(K, bk);
    tp.seg_kb = lp.tile_m > 0 ? lp.tile_m : (x3 ? kSegK / bk : std::max(nkb, 1));
    lp.teams = r->teams ? r->teams : (int)std::max<int64_t>(1, std::min<int64_t>(tp.ntiles, kNumSMs));
    tp.full_tiles = tp.ntiles;
    tp.split_tiles = 0;
    tp.parts = 1;
    tp.nunits = tp.ntiles;
    int64_t chunk_eff = lp.chunk;
    const int bk0 = x3 ? TcCfg<true>::BK : TcCfg<false>::BK;
    const int nkb0 = (int)ceil_div(K, bk0);
    if (!r->teams && lp.chunk == 0 && tp.ntiles > 0) {
        // The planner sizes the grid.  The bfloat16 form (bound by
        // shared-memory traffic, sensitive to L2 contention) takes the fewest
        // teams that give every team the same number of tiles; the split form
        // (three MMAs per operand load) keeps one team per SM and cuts the
        // tiles of the last, partial wave into K parts for the idle teams.
        // With fewer tiles than SMs both cut every tile into K parts.  Units
        // are dealt round-robin (static, chunk 1).
        const int64_t waves = ceil_div(tp.ntiles, kNumSMs);
        if (!x3) lp.teams = (int)ceil_div(tp.ntiles, waves);
        const int64_t T = kNumSMs;
        const int64_t rem = (x3 || waves == 1) ? tp.ntiles % T : 0;
        if (rem > 0 && rem * 2 <= T) {
            const int64_t parts = std::min<int64_t>(std::min<int64_t>(T / rem, 4), std::max(nkb0 / 2, 1));
            if (parts > 1) {
                tp.split_tiles = rem;
                tp.full_tiles = tp.ntiles - rem;
                tp.parts = (int)parts;
                tp.nunits = tp.full_tiles + rem * parts;
                lp.teams = (int)std::min<int64_t>(T, tp.nunits);
            }
        }
        chunk_eff = 1;
    }
    tp.chunk = chunk_eff;
    tp.sk = make_sched_const(tp.nunits, chunk_eff, lp.teams);
    if (tp.parts > 1) {
        const size_t bytes = (size_t)tp.split_tiles * (tp.parts - 1) * TC_BM * TC_BN * sizeof(float);
        lp.scratch = dev_alloc(ctx, bytes);
        if (!lp.scratch) return fail(ctx, UPIR_ENOMEM, "upir_loop: GEMM split-K workspace of %zu bytes", bytes);
        lp.scratch_bytes = bytes;
        tp.work = static_cast<float*>(lp.scratch);
    }
    memcpy(lp.tc_params, &tp, sizeof(tp));
    lp.skip = lp.trip == 0 || N == 0;
    if (lp.skip || K == 0) {
        if (K == 0 && !lp.skip)
            return fail(ctx, UPIR_EUNSUPPORTED, "upir_loop: tensor-core GEMM needs K > 0");
        return UPIR_OK;
    }
    const void* bases[4] = {lp.bufs[0]->dev, lp.bufs[x3 ? 1 : 0]->dev, lp.bufs[na]->dev,
                            lp.bufs[x3 ? na + 1 : na]->dev};
    const uint64_t rows[4] = {(uint64_t)M, (uint64_t)M, (uint64_t)N, (uint64_t)N};
    const uint32_t box_rows[4] = {TC_BM, TC_BM, TC_BN, TC_BN};
    for (int i = 0; i < 4; ++i) {
        upir_status s2 = encode_tmap_2d(ctx, &lp.tmap[i], bases[i], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                                        (uint64_t)K, rows[i], (uint32_t)bk, box_rows[i], bk * 2);
        if (s2 != UPIR_OK) return s2;
    }
    return UPIR_OK;
}

cudaError_t launch_gemm_tc_loop(upir_ctx, LoopRec& lp, cudaStream_t s) {
    TcParams tp;
    memcpy(&tp, lp.tc_params, sizeof(tp));
    CUtensorMap m[4];
    memcpy(m, lp.tmap, sizeof(m));
    if (lp.body == UPIR_BODY_GEMM_BF16X3) {
        if (!tc_configure<true>()) return cudaGetLastError();
        gemm_tc_kernel<true><<<lp.teams, TC_THREADS, TcCfg<true>::SMEM, s>>>(tp, m[0], m[1], m[2], m[3]);
    } else {
        if (!tc_configure<false>()) return cudaGetLastError();
        gemm_tc_kernel<false><<<lp.teams, TC_THREADS, TcCfg<false>::SMEM, s>>>(tp, m[0], m[1], m[2], m[3]);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || tp.parts <= 1) return e;
    const int64_t elems = tp.split_tiles * TC_BM * TC_BN;
    tc_fixup_kernel<<<(unsigned)std::min<int64_t>((elems + 255) / 256, kNumSMs * 16), 256, 0, s>>>(tp);
    return cudaGetLastError();
}

}  // namespace upir
