// The bfloat16 GEMM bodies (the matrix multiplication workload of §6: plain
// bfloat16 and the split form with three products) on CTA pairs:
// tcgen05.mma with cta_group::2 computes a 256 x 256 output tile per pair of
// SMs, each SM holding 128 rows of the accumulator in its own TMEM.
//
// Why pairs: with one SM per 128 x 256 tile every k-block moves 48 KB of
// operands into shared memory (TMA) and 48 KB out of it (MMA), which caps the
// tensor pipe below its rate on one SM's shared-memory bandwidth.  A pair
// shares B: each SM loads its own 128 rows of A and half (128 rows) of the
// tile's 256 rows of B^T, and the pair's MMA reads A from each SM and B from
// both, so an SM moves 32 KB in and 32 KB out per k-block for the same flops.
//
// Roles per CTA (576 threads), as in the one-SM kernel:
//   warp 0      one thread copies this CTA's A and B^T halves of each
//               k-block (hi and lo parts for the split form) into a 6-stage
//               ring of 32 KB per CTA; the copies of both CTAs complete
//               on the leading CTA's (rank 0) full barrier, which the leading
//               producer arms with the bytes of both;
//   warp 1      allocates 512 TMEM columns in both CTAs (cta_group::2); in the
//               leading CTA one thread issues the pair's MMAs (M = 256,
//               N = 256, K = 16) and commits each stage back to the empty
//               barriers of both CTAs and each finished tile to the full-TMEM
//               barriers of both;
//   warps 2..17 read this CTA's 128 accumulator rows with tcgen05.ld, write
//               them to C with 32-byte stores and release the accumulator to
//               the leading CTA (one remote arrival per warp).
// Pair tiles are dealt to clusters round-robin; a last partial wave of tiles
// is cut into 128-column halves when that leaves fewer clusters idle.  K may
// run in accumulation segments (the split form's default: 1024 per segment),
// added in FP32 registers by the epilogue.  The planner uses this kernel when
// every resident cluster gets at least one tile.  Every wait is bounded; a CTA that gives up records
// the timeout, lets its copies and MMAs land, and both CTAs meet at a cluster
// barrier before the TMEM is freed.
#include <cstring>

#include "tc_common.cuh"

namespace upir {

namespace {

constexpr int P2_STAGES = 6;
constexpr int P2_STAGE_BYTES = 32 * 1024;  // per CTA: its 128 rows of A and of B^T, one or two operands each
constexpr size_t P2_SMEM = (size_t)P2_STAGES * P2_STAGE_BYTES + 1024;
constexpr int P2_TILE = 256;                             // pair tile: 256 x 256

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// The shared::cluster address of `p`'s counterpart in CTA `rank` of the pair.
__device__ __forceinline__ uint32_t pair_addr(const void* p, uint32_t rank) {
    uint32_t a;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(a) : "r"(smem_u32(p)), "r"(rank));
    return a;
}

__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_remote(uint32_t caddr) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(caddr) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait_cluster(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}

// A copy into this CTA's shared memory whose completion is counted on an
// mbarrier of either CTA of the pair (given by its shared::cluster address).
__device__ __forceinline__ void tma_load_2d_pair(void* dst, const void* tmap, uint32_t bar_caddr, int32_t x,
                                                 int32_t y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"(tmap), "r"(x), "r"(y), "r"(bar_caddr)
        : "memory");
}

__device__ __forceinline__ void mma_pair(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

// Arrive on the barrier at this offset in both CTAs once the pair's MMAs
// issued so far have completed.
__device__ __forceinline__ void commit_both(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;"
        ::"r"(smem_u32(bar)), "h"((uint16_t)3) : "memory");
}

__device__ __forceinline__ void commit_own(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(smem_u32(bar)) : "memory");
}

// kind::f16 instruction descriptor for the pair: FP32 accumulator, bfloat16
// A and B, both K-major, M = 256, N = 256 (128 for half tiles).
__host__ __device__ constexpr uint32_t pair_idesc(int n = P2_TILE) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(P2_TILE >> 4) << 24);
}

// Bounded wait; `cluster` waits acquire at cluster scope (the barrier is
// arrived on from the other CTA).
__device__ __forceinline__ bool p2_wait(uint64_t* bar, uint32_t parity, const TcParams& p, volatile int* abort_flag,
                                        bool cluster = false) {
    for (long long n = 0; n < p.spin_limit; ++n) {
        if (cluster ? mbar_try_wait_cluster(bar, parity) : mbar_try_wait(bar, parity)) return true;
        if ((n & 255) == 255 && *abort_flag) return false;
    }
    atomicCAS(p.err_word, 0, UPIR_ERR_WAIT_TIMEOUT);
    *abort_flag = 1;
    return false;
}

// Work units: the full pair tiles, then (a last partial wave) `half_tiles`
// tiles cut into two 128-column halves (N = 128 MMAs, 64 rows of B^T per CTA).
// Units are dealt to clusters round-robin.
struct P2Unit {
    int64_t tile;
    int half;  // 0: all 256 columns; 1, 2: the first or second 128
};

__device__ __forceinline__ P2Unit p2_unit(int64_t u, const TcParams& p) {
    if (u < p.full_tiles) return P2Unit{u, 0};
    const int64_t v = u - p.full_tiles;
    return P2Unit{p.full_tiles + (v >> 1), 1 + (int)(v & 1)};
}

// The plain bfloat16 form with one K segment (the planner's usual case), in
// a kernel of its own: the general template below runs it about 4 % slower.
// Its stages hold two 64-wide k-blocks (three stages of 64 KB per CTA), so
// the issuing thread waits on a barrier and commits once per eight MMAs
// instead of four: 4096^3 ran 104.5 us with one k-block per stage (six
// stages), 98.0 us with two, 111.6 us with three (two stages).
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(TC_THREADS, 1)
gemm_tc2_plain_kernel(const TcParams p, const __grid_constant__ CUtensorMap tm_a,
                      const __grid_constant__ CUtensorMap tm_b, const __grid_constant__ CUtensorMap tm_b64) {
    constexpr int NACC = 2;
    constexpr uint32_t kCols = 256u * NACC;
    using Cfg = TcCfg<false>;  // BK 64, 128-byte swizzle
    constexpr int P2_BK = 64, P2_A_BYTES = 128 * P2_BK * 2, P2_B_BYTES = 128 * P2_BK * 2;
    // a stage holds KS consecutive 64-wide k-blocks (slices) of each operand
    constexpr int KS = 2;
    constexpr int S = P2_STAGES / KS;
    constexpr int SLICE = 16 * 1024;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[S], empty[S], tfull[NACC], tempty[NACC], mma_done;
    __shared__ uint32_t tmem_base_sh;
    __shared__ volatile int abort_flag;
    unsigned char* ring = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_rank();
    const bool leader = rank == 0;
    const int nkb = (int)((p.K + P2_BK * KS - 1) / (P2_BK * KS));  // stages of KS slices

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < NACC; ++a) {
            mbar_init(&tfull[a], 1);
            mbar_init(&tempty[a], 2 * (TC_EPI_THREADS / 32));  // every epilogue warp of both CTAs
        }
        mbar_init(&mma_done, 1);
        abort_flag = 0;
        fence_mbar_init();
        prefetch_tmap(&tm_a);
        prefetch_tmap(&tm_b);
        prefetch_tmap(&tm_b64);
    }
    if (warp == 1) {
        // one warp of each CTA of the pair takes part in the allocation
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(&tmem_base_sh)), "r"(kCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    // both CTAs' barriers are initialised (and their TMEM allocated) before
    // either CTA's copies, commits or arrivals can reach them
    cluster_sync_all();
    tc_fence_after();
    const uint32_t tmem_base = tmem_base_sh;
    // the pair's MMAs write the same TMEM columns in both CTAs: a pair whose
    // allocations differ records an error and does no work
    uint32_t peer_base;
    asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(peer_base) : "r"(pair_addr(&tmem_base_sh, rank ^ 1u)) : "memory");
    const bool pair_bad = peer_base != tmem_base;
    if (pair_bad && threadIdx.x == 0) atomicCAS(p.err_word, 0, UPIR_ERR_WAIT_TIMEOUT);

    auto stage_a = [&](int s) { return ring + (size_t)s * KS * P2_STAGE_BYTES; };
    auto stage_b = [&](int s) { return ring + (size_t)s * KS * P2_STAGE_BYTES + KS * SLICE; };

    if (pair_bad) {
        // nothing to do: both CTAs go straight to the teardown
    } else if (warp == 0) {
        if (lane == 0) {
            // ---------------- producer: this CTA's halves of each k-block ----------------
            int s = 0;
            uint32_t ph = 0;
            uint32_t issued_parity[S];
            bool issued[S];
            for (int k = 0; k < S; ++k) issued[k] = false, issued_parity[k] = 0;
            for (int64_t u = blockIdx.x >> 1; u < p.nunits && !abort_flag; u += gridDim.x >> 1) {
                const P2Unit w = p2_unit(u, p);
                const int64_t mt = w.tile % p.tiles_m, nt = w.tile / p.tiles_m;
                const int bh = w.half ? 64 : 128;  // this CTA's rows of B^T
                const int32_t m0 = (int32_t)(p.row_lb + mt * P2_TILE + 128 * (int64_t)rank);
                const int32_t n0 = (int32_t)(nt * P2_TILE + (w.half == 2 ? 128 : 0) + bh * (int64_t)rank);
                const CUtensorMap* mb = w.half ? &tm_b64 : &tm_b;
                const uint32_t bytes = 2u * KS * (uint32_t)(P2_A_BYTES + (w.half ? P2_B_BYTES / 2 : P2_B_BYTES));
                for (int kb = 0; kb < nkb; ++kb) {
                    if (!p2_wait(&empty[s], ph ^ 1u, p, &abort_flag)) break;
                    const uint32_t fb = pair_addr(&full[s], 0);
                    if (leader) mbar_arrive_expect_tx(&full[s], bytes);
#pragma unroll
                    for (int j = 0; j < KS; ++j) {
                        tma_load_2d_pair(stage_a(s) + j * SLICE, &tm_a, fb, (kb * KS + j) * P2_BK, m0);
                        tma_load_2d_pair(stage_b(s) + j * SLICE, mb, fb, (kb * KS + j) * P2_BK, n0);
                    }
                    issued[s] = true;
                    issued_parity[s] = ph;
                    if (++s == S) s = 0, ph ^= 1u;
                }
            }
            if (abort_flag && leader) {
                // copies in flight get a bounded chance to land before the ring is released
                for (int k = 0; k < S; ++k)
                    if (issued[k]) mbar_wait_bounded(&full[k], issued_parity[k], p.spin_limit, nullptr);
            }
        }
    } else if (warp == 1) {
        if (lane == 0 && leader) {
            // ---------------- MMA issuer (leading CTA) ----------------
            constexpr uint32_t idesc_full = pair_idesc(), idesc_half = pair_idesc(P2_TILE / 2);
            int s = 0, acc = 0;
            uint32_t ph = 0, aph = 0;
            bool issued_any = false, ok = true;
            for (int64_t u = blockIdx.x >> 1; u < p.nunits && ok && !abort_flag; u += gridDim.x >> 1) {
                const uint32_t idesc = p2_unit(u, p).half ? idesc_half : idesc_full;
                if (!p2_wait(&tempty[acc], aph ^ 1u, p, &abort_flag, true)) break;
                tc_fence_after();
                const uint32_t d_tmem = tmem_base + (uint32_t)(acc * TC_BN);
                for (int kb = 0; kb < nkb; ++kb) {
                    if (!p2_wait(&full[s], ph, p, &abort_flag, true)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a = smem_u32(stage_a(s)), b = smem_u32(stage_b(s));
#pragma unroll
                    for (int j = 0; j < KS; ++j) {
#pragma unroll
                        for (int k = 0; k < P2_BK / 16; ++k) {
                            const uint32_t koff = (uint32_t)(j * SLICE + k * 32);  // 16 bfloat16 along K
                            mma_pair(d_tmem, smem_desc<Cfg>(a + koff), smem_desc<Cfg>(b + koff), idesc,
                                     (kb > 0 || j > 0 || k > 0) ? 1u : 0u);
                        }
                    }
                    issued_any = true;
                    commit_both(&empty[s]);  // both CTAs' stage s is free once these MMAs have read it
                    if (++s == S) s = 0, ph ^= 1u;
                }
                if (!ok) break;
                commit_both(&tfull[acc]);
                if (++acc == NACC) acc = 0, aph ^= 1u;
            }
            if (abort_flag && issued_any) {
                // MMAs in flight must finish before either CTA frees its TMEM
                commit_own(&mma_done);
                mbar_wait_bounded(&mma_done, 0, p.spin_limit, nullptr);
            }
        }
    } else {
        // ---------------- epilogue: this CTA's 128 accumulator rows -> C ----------------
        const int q = warp & 3;               // TMEM lane quadrant this warp may access
        const int quarter = (warp - 2) >> 2;  // which quarter of the tile's columns
        int acc = 0;
        uint32_t aph = 0;
        const bool v8_ok = (p.N % 8) == 0 && (reinterpret_cast<uintptr_t>(p.C) & 31) == 0;
        const uint32_t te0 = pair_addr(&tempty[0], 0), te1 = pair_addr(&tempty[NACC - 1], 0);
        for (int64_t u = blockIdx.x >> 1; u < p.nunits && !abort_flag; u += gridDim.x >> 1) {
            const P2Unit w = p2_unit(u, p);
            const int cw = w.half ? TC_EPI_COLS / 2 : TC_EPI_COLS;  // columns of this warp
            const int64_t mt = w.tile % p.tiles_m, nt = w.tile / p.tiles_m;
            const int64_t row = p.row_lb + mt * P2_TILE + 128 * (int64_t)rank + 32 * q + lane;
            const int64_t n0 = nt * P2_TILE + (w.half == 2 ? 128 : 0) + quarter * cw;
            float* crow = row < p.row_ub ? p.C + row * p.N : nullptr;
            const bool full_row = v8_ok && n0 + cw <= p.N;
            if (!p2_wait(&tfull[acc], aph, p, &abort_flag)) break;
            tc_fence_after();
            const uint32_t ta = tmem_base + ((uint32_t)(32 * q) << 16) + (uint32_t)(quarter * cw) +
                                (uint32_t)(acc * TC_BN);
#pragma unroll
            for (int h = 0; h < TC_EPI_COLS; h += 32) {
                if (h < cw) {
                    float v[32];
                    tmem_ld32(ta + (uint32_t)h, v);
                    if (crow) store_row(crow, n0 + h, p.N, full_row, v, 32);
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive_remote(acc ? te1 : te0);
            if (++acc == NACC) acc = 0, aph ^= 1u;
        }
    }

    tc_fence_before();
    __syncthreads();
    // neither CTA frees its TMEM or leaves while the pair's MMAs, copies or
    // arrivals may still reach it
    cluster_sync_all();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;"
                     ::"r"(tmem_base), "r"(kCols) : "memory");
    }
}

// Per-CTA ring geometry: the plain form streams 64-wide k-blocks of A and
// B^T (128-byte swizzle); the split form 32-wide k-blocks of A_hi, A_lo, B_hi
// and B_lo (64-byte swizzle).  A stage is 32 KB either way.
template <bool X3>
struct P2Cfg {
    using Tc = TcCfg<X3>;
    static constexpr int BK = Tc::BK;
    static constexpr int A_BYTES = 128 * BK * 2;  // one operand's 128 rows
    static constexpr int B_BYTES = 128 * BK * 2;  // one operand's 128 rows of B^T (half of N)
    static constexpr int STAGE_BYTES = (X3 ? 2 : 1) * (A_BYTES + B_BYTES);
    static_assert(STAGE_BYTES == P2_STAGE_BYTES, "one ring layout for both forms");
};

// Two accumulator buffers of 256 TMEM columns: the epilogue of one K segment
// (or tile) overlaps the MMAs of the next.  X3: the split form, three MMAs
// per 16-deep step (A_hi B_hi, A_hi B_lo, A_lo B_hi).  MSEG: K runs in
// segments of seg_kb k-blocks, each into a fresh accumulator, added in FP32
// registers by the epilogue in segment order.
template <bool X3, bool MSEG, int KS>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(TC_THREADS, 1)
gemm_tc2_kernel(const TcParams p, const __grid_constant__ CUtensorMap tm_ah, const __grid_constant__ CUtensorMap tm_al,
                const __grid_constant__ CUtensorMap tm_bh, const __grid_constant__ CUtensorMap tm_bl,
                const __grid_constant__ CUtensorMap tm_bh64, const __grid_constant__ CUtensorMap tm_bl64) {
    using Cfg = typename P2Cfg<X3>::Tc;
    using PC = P2Cfg<X3>;
    constexpr int NACC = 2;
    constexpr uint32_t kCols = 256u * NACC;
    constexpr int S = P2_STAGES / KS;  // a stage holds KS consecutive k-blocks
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[S], empty[S], tfull[NACC], tempty[NACC], mma_done;
    __shared__ uint32_t tmem_base_sh;
    __shared__ volatile int abort_flag;
    unsigned char* ring = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_rank();
    const bool leader = rank == 0;
    const int nst = (int)((p.K + PC::BK * KS - 1) / (PC::BK * KS));  // stages along K
    const int seg_st = MSEG ? p.seg_kb / KS : nst;                     // stages per K segment

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < NACC; ++a) {
            mbar_init(&tfull[a], 1);
            mbar_init(&tempty[a], 2 * (TC_EPI_THREADS / 32));  // every epilogue warp of both CTAs
        }
        mbar_init(&mma_done, 1);
        abort_flag = 0;
        fence_mbar_init();
        prefetch_tmap(&tm_ah);
        prefetch_tmap(&tm_bh);
    }
    if (warp == 1) {
        // one warp of each CTA of the pair takes part in the allocation
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(&tmem_base_sh)), "r"(kCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    // both CTAs' barriers are initialised (and their TMEM allocated) before
    // either CTA's copies, commits or arrivals can reach them
    cluster_sync_all();
    tc_fence_after();
    const uint32_t tmem_base = tmem_base_sh;
    // the pair's MMAs write the same TMEM columns in both CTAs: a pair whose
    // allocations differ records an error and does no work
    uint32_t peer_base;
    asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(peer_base) : "r"(pair_addr(&tmem_base_sh, rank ^ 1u)) : "memory");
    const bool pair_bad = peer_base != tmem_base;
    if (pair_bad && threadIdx.x == 0) atomicCAS(p.err_word, 0, UPIR_ERR_WAIT_TIMEOUT);

    // stage layout: KS slices of A_hi [, A_lo], B_hi [, B_lo], one k-block each
    auto stage_a = [&](int s, int j) { return ring + ((size_t)s * KS + j) * P2_STAGE_BYTES; };
    auto stage_b = [&](int s, int j) { return stage_a(s, j) + PC::A_BYTES * (X3 ? 2 : 1); };

    if (pair_bad) {
        // nothing to do: both CTAs go straight to the teardown
    } else if (warp == 0) {
        if (lane == 0) {
            // ---------------- producer: this CTA's halves of each k-block ----------------
            int s = 0;
            uint32_t ph = 0;
            uint32_t issued_parity[S];
            bool issued[S];
            for (int k = 0; k < S; ++k) issued[k] = false, issued_parity[k] = 0;
            for (int64_t u = blockIdx.x >> 1; u < p.nunits && !abort_flag; u += gridDim.x >> 1) {
                const P2Unit w = p2_unit(u, p);
                const int64_t mt = w.tile % p.tiles_m, nt = w.tile / p.tiles_m;
                const int bh = w.half ? 64 : 128;  // this CTA's rows of B^T
                const int32_t m0 = (int32_t)(p.row_lb + mt * P2_TILE + 128 * (int64_t)rank);
                const int32_t n0 = (int32_t)(nt * P2_TILE + (w.half == 2 ? 128 : 0) + bh * (int64_t)rank);
                const CUtensorMap* mbh = w.half ? &tm_bh64 : &tm_bh;
                const CUtensorMap* mbl = w.half ? &tm_bl64 : &tm_bl;
                const uint32_t bytes =
                    2u * KS * (uint32_t)((X3 ? 2 : 1) * (PC::A_BYTES + (w.half ? PC::B_BYTES / 2 : PC::B_BYTES)));
                for (int kst = 0; kst < nst; ++kst) {
                    if (!p2_wait(&empty[s], ph ^ 1u, p, &abort_flag)) break;
                    const uint32_t fb = pair_addr(&full[s], 0);
                    if (leader) mbar_arrive_expect_tx(&full[s], bytes);
#pragma unroll
                    for (int j = 0; j < KS; ++j) {
                        const int32_t k0 = (kst * KS + j) * PC::BK;
                        unsigned char* a = stage_a(s, j);
                        unsigned char* b = stage_b(s, j);
                        tma_load_2d_pair(a, &tm_ah, fb, k0, m0);
                        tma_load_2d_pair(b, mbh, fb, k0, n0);
                        if (X3) {
                            tma_load_2d_pair(a + PC::A_BYTES, &tm_al, fb, k0, m0);
                            tma_load_2d_pair(b + PC::B_BYTES, mbl, fb, k0, n0);
                        }
                    }
                    issued[s] = true;
                    issued_parity[s] = ph;
                    if (++s == S) s = 0, ph ^= 1u;
                }
            }
            if (abort_flag && leader) {
                // copies in flight get a bounded chance to land before the ring is released
                for (int k = 0; k < S; ++k)
                    if (issued[k]) mbar_wait_bounded(&full[k], issued_parity[k], p.spin_limit, nullptr);
            }
        }
    } else if (warp == 1) {
        if (lane == 0 && leader) {
            // ---------------- MMA issuer (leading CTA) ----------------
            constexpr uint32_t idesc_full = pair_idesc(), idesc_half = pair_idesc(P2_TILE / 2);
            int s = 0, acc = 0;
            uint32_t ph = 0, aph = 0;
            bool issued_any = false, ok = true;
            for (int64_t u = blockIdx.x >> 1; u < p.nunits && ok && !abort_flag; u += gridDim.x >> 1) {
                const uint32_t idesc = p2_unit(u, p).half ? idesc_half : idesc_full;
                for (int kb0 = 0; kb0 < nst && ok; kb0 += seg_st) {
                    // one K segment into a fresh accumulator buffer
                    if (!p2_wait(&tempty[acc], aph ^ 1u, p, &abort_flag, true)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d_tmem = tmem_base + (uint32_t)(acc * TC_BN);
                    const int kb1 = min(kb0 + seg_st, nst);
                    for (int kb = kb0; kb < kb1; ++kb) {
                        if (!p2_wait(&full[s], ph, p, &abort_flag, true)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
#pragma unroll
                        for (int j = 0; j < KS; ++j) {
                            const uint32_t a = smem_u32(stage_a(s, j)), b = smem_u32(stage_b(s, j));
#pragma unroll
                            for (int k = 0; k < PC::BK / 16; ++k) {
                                const uint32_t koff = (uint32_t)k * 32u;  // 16 bfloat16 along K
                                mma_pair(d_tmem, smem_desc<Cfg>(a + koff), smem_desc<Cfg>(b + koff), idesc,
                                         (kb > kb0 || j > 0 || k > 0) ? 1u : 0u);
                                if (X3) {
                                    mma_pair(d_tmem, smem_desc<Cfg>(a + koff),
                                             smem_desc<Cfg>(b + PC::B_BYTES + koff), idesc, 1u);
                                    mma_pair(d_tmem, smem_desc<Cfg>(a + PC::A_BYTES + koff),
                                             smem_desc<Cfg>(b + koff), idesc, 1u);
                                }
                            }
                        }
                        issued_any = true;
                        commit_both(&empty[s]);  // both CTAs' stage s is free once these MMAs have read it
                        if (++s == S) s = 0, ph ^= 1u;
                    }
                    if (!ok) break;
                    commit_both(&tfull[acc]);
                    if (++acc == NACC) acc = 0, aph ^= 1u;
                }
            }
            if (abort_flag && issued_any) {
                // MMAs in flight must finish before either CTA frees its TMEM
                commit_own(&mma_done);
                mbar_wait_bounded(&mma_done, 0, p.spin_limit, nullptr);
            }
        }
    } else {
        // ---------------- epilogue: this CTA's 128 accumulator rows -> C ----------------
        const int q = warp & 3;               // TMEM lane quadrant this warp may access
        const int quarter = (warp - 2) >> 2;  // which quarter of the tile's columns
        int acc = 0;
        uint32_t aph = 0;
        const bool v8_ok = (p.N % 8) == 0 && (reinterpret_cast<uintptr_t>(p.C) & 31) == 0;
        const uint32_t te0 = pair_addr(&tempty[0], 0), te1 = pair_addr(&tempty[NACC - 1], 0);
        const int nseg = (nst + seg_st - 1) / seg_st;
        bool ok = true;
        for (int64_t u = blockIdx.x >> 1; u < p.nunits && ok && !abort_flag; u += gridDim.x >> 1) {
            const P2Unit w = p2_unit(u, p);
            const int cw = w.half ? TC_EPI_COLS / 2 : TC_EPI_COLS;  // columns of this warp
            const int64_t mt = w.tile % p.tiles_m, nt = w.tile / p.tiles_m;
            const int64_t row = p.row_lb + mt * P2_TILE + 128 * (int64_t)rank + 32 * q + lane;
            const int64_t n0 = nt * P2_TILE + (w.half == 2 ? 128 : 0) + quarter * cw;
            float* crow = row < p.row_ub ? p.C + row * p.N : nullptr;
            const bool full_row = v8_ok && n0 + cw <= p.N;
            float sum[MSEG ? TC_EPI_COLS : 1];  // running sum of the earlier K segments
            for (int seg = 0; seg < nseg; ++seg) {
                if (!p2_wait(&tfull[acc], aph, p, &abort_flag)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t ta = tmem_base + ((uint32_t)(32 * q) << 16) + (uint32_t)(quarter * cw) +
                                    (uint32_t)(acc * TC_BN);
                if (MSEG && seg + 1 < nseg) {
#pragma unroll
                    for (int c = 0; c < TC_EPI_COLS; c += 16) {
                        if (c < cw) {
                            float v[16];
                            tmem_ld16(ta + (uint32_t)c, v);
#pragma unroll
                            for (int j = 0; j < 16; ++j)
                                sum[MSEG ? c + j : 0] = seg ? __fadd_rn(sum[MSEG ? c + j : 0], v[j]) : v[j];
                        }
                    }
                } else {
                    // the last segment goes straight out, 32 columns at a time
#pragma unroll
                    for (int h = 0; h < TC_EPI_COLS; h += 32) {
                        if (h < cw) {
                            float v[32];
                            tmem_ld32(ta + (uint32_t)h, v);
                            if (MSEG && seg) {
#pragma unroll
                                for (int j = 0; j < 32; ++j) v[j] = __fadd_rn(sum[MSEG ? h + j : 0], v[j]);
                            }
                            if (crow) store_row(crow, n0 + h, p.N, full_row, v, 32);
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive_remote(acc ? te1 : te0);
                if (++acc == NACC) acc = 0, aph ^= 1u;
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    // neither CTA frees its TMEM or leaves while the pair's MMAs, copies or
    // arrivals may still reach it
    cluster_sync_all();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;"
                     ::"r"(tmem_base), "r"(kCols) : "memory");
    }
}

// The large shared-memory window, set once per instantiation; returns the
// result of that one call.
template <bool X3, bool MSEG, int KS>
cudaError_t p2_configure() {
    static cudaError_t state = cudaFuncSetAttribute(gemm_tc2_kernel<X3, MSEG, KS>,
                                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P2_SMEM);
    return state;
}

// Two k-blocks per stage unless K segments of an odd number of k-blocks
// would split a stage.
template <bool X3, bool MSEG>
cudaError_t p2_launch(const TcParams& tp, int ctas, const CUtensorMap* m, cudaStream_t s) {
    if (MSEG && tp.seg_kb % 2) {
        const cudaError_t e = p2_configure<X3, MSEG, 1>();
        if (e != cudaSuccess) return e;
        gemm_tc2_kernel<X3, MSEG, 1><<<ctas, TC_THREADS, P2_SMEM, s>>>(tp, m[0], m[1], m[2], m[3], m[4], m[5]);
    } else {
        const cudaError_t e = p2_configure<X3, MSEG, 2>();
        if (e != cudaSuccess) return e;
        gemm_tc2_kernel<X3, MSEG, 2><<<ctas, TC_THREADS, P2_SMEM, s>>>(tp, m[0], m[1], m[2], m[3], m[4], m[5]);
    }
    return cudaGetLastError();
}

}  // namespace

size_t gemm_tc2_smem_bytes() { return P2_SMEM; }

int gemm_tc2_max_clusters() {
    static int cached = -1;
    if (cached >= 0) return cached;
    if (cudaFuncSetAttribute(gemm_tc2_plain_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P2_SMEM) !=
        cudaSuccess) {
        cudaGetLastError();
        return cached = 0;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kNumSMs);
    cfg.blockDim = dim3(TC_THREADS);
    cfg.dynamicSmemBytes = P2_SMEM;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, gemm_tc2_plain_kernel, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return cached = 0;
    }
    return cached = n;
}

// m: A_hi, A_lo, B_hi and B_lo (128-row boxes), then B_hi and B_lo with
// 64-row boxes for half tiles; the plain form uses A_hi, B_hi and B_hi64.
cudaError_t launch_gemm_tc2(const TcParams& tp, int ctas, bool x3, bool mseg, const CUtensorMap* m, cudaStream_t s) {
    if (x3) return mseg ? p2_launch<true, true>(tp, ctas, m, s) : p2_launch<true, false>(tp, ctas, m, s);
    if (mseg) return p2_launch<false, true>(tp, ctas, m, s);
    static const cudaError_t conf = cudaFuncSetAttribute(gemm_tc2_plain_kernel,
                                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P2_SMEM);
    if (conf != cudaSuccess) return conf;
    gemm_tc2_plain_kernel<<<ctas, TC_THREADS, P2_SMEM, s>>>(tp, m[0], m[2], m[4]);
    return cudaGetLastError();
}

}  // namespace upir
