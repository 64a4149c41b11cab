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
//               K segment (or tile) overlap this epilogue work; each thread
//               writes its row of C with 32-byte stores (one full sector).
// A last, partial wave of tiles is cut into 128-column halves (N = 128 MMAs)
// so that the teams it would leave idle take a share; with fewer tiles than
// SMs the tiles are cut along K instead, the last-finishing part of each
// tile adding all parts in part order.
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

#include "tc_common.cuh"

namespace upir {

namespace {

// MSEG: K may span several accumulation segments (a running sum is kept);
// without it every unit is one segment and goes straight from TMEM out.
template <bool X3, bool MSEG>
__global__ void __launch_bounds__(TC_THREADS, 1)
gemm_tc_kernel(const TcParams p, const __grid_constant__ CUtensorMap tm_ah,
               const __grid_constant__ CUtensorMap tm_al, const __grid_constant__ CUtensorMap tm_bh,
               const __grid_constant__ CUtensorMap tm_bl, const __grid_constant__ CUtensorMap tm_bh2,
               const __grid_constant__ CUtensorMap tm_bl2) {
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
                const int32_t m0 = (int32_t)(p.row_lb + mt * TC_BM);
                const int32_t n0 = (int32_t)(nt * TC_BN + (w.half == 2 ? TC_BN / 2 : 0));
                // half tiles load 128 rows of B^T through the maps with the 128-row box
                const CUtensorMap* mbh = w.half ? &tm_bh2 : &tm_bh;
                const CUtensorMap* mbl = w.half ? &tm_bl2 : &tm_bl;
                const uint32_t bytes = w.half ? Cfg::HALF_STAGE_BYTES : Cfg::STAGE_BYTES;
                for (int kb = w.kb0; kb < w.kb1; ++kb) {
                    if (!tc_wait(&empty[s], ph ^ 1u, p, &abort_flag)) break;
                    mbar_arrive_expect_tx(&full[s], bytes);
                    const int32_t k0 = kb * Cfg::BK;
                    unsigned char* a = stage_a(s);
                    unsigned char* b = stage_b(s);
                    tma_load_2d(a, &tm_ah, &full[s], k0, m0);
                    tma_load_2d(b, mbh, &full[s], k0, n0);
                    if (X3) {
                        tma_load_2d(a + Cfg::A_BYTES, &tm_al, &full[s], k0, m0);
                        tma_load_2d(b + Cfg::B_BYTES, mbl, &full[s], k0, n0);
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
            constexpr uint32_t idesc_full = tc_idesc(), idesc_half = tc_idesc(TC_BN / 2);
            TcTiles it = tc_first(p);
            int s = 0, acc = 0;
            uint32_t ph = 0, aph = 0;
            bool issued_any = false, ok = true;
            for (int64_t u = tc_next_tile(it, p); u >= 0 && ok && !abort_flag; u = tc_next_tile(it, p)) {
                const TcUnit w = tc_unit(u, p, nkb);
                const uint32_t idesc = w.half ? idesc_half : idesc_full;
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
        const int sub = quarter * (TC_BM / 32) + q;
        TcTiles it = tc_first(p);
        int acc = 0;
        uint32_t aph = 0;
        // rows of C start on 32-byte boundaries, so 8 columns go in one store
        const bool v8_ok = (p.N % 8) == 0 && (reinterpret_cast<uintptr_t>(p.C) & 31) == 0;
        bool ok = true;
        for (int64_t u = tc_next_tile(it, p); u >= 0 && ok && !abort_flag; u = tc_next_tile(it, p)) {
            const TcUnit w = tc_unit(u, p, nkb);
            const int nseg = (w.kb1 - w.kb0 + p.seg_kb - 1) / p.seg_kb;
            // each warp holds 32 rows x cw columns: 64 of a whole tile, 32 of a half
            const int cw = w.half ? TC_EPI_COLS / 2 : TC_EPI_COLS;
            const int64_t mt = w.tile % p.tiles_m, nt = w.tile / p.tiles_m;
            const int64_t row = p.row_lb + mt * TC_BM + 32 * q + lane;
            const int64_t n0 = nt * TC_BN + (w.half == 2 ? TC_BN / 2 : 0) + quarter * cw;
            float* crow = row < p.row_ub ? p.C + row * p.N : nullptr;
            const bool full_row = v8_ok && n0 + cw <= p.N;
            const uint32_t tq = tmem_base + ((uint32_t)(32 * q) << 16) + (uint32_t)(quarter * cw);
            // One K part of a split tile publishes its 32 x 64 block to the
            // workspace instead of writing C.
            const bool split = w.split_idx >= 0;
            const int64_t part_stride = (int64_t)TC_SUBS * 32 * TC_EPI_COLS;
            float* const work =
                split ? p.work + ((w.split_idx * p.parts * TC_SUBS + sub) * 32 + lane) * TC_EPI_COLS : nullptr;
            float sum[MSEG ? TC_EPI_COLS : 1];  // running sum of the earlier K segments
            for (int seg = 0; seg < nseg; ++seg) {
                if (!tc_wait(&tfull[acc], aph, p, &abort_flag)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t ta = tq + (uint32_t)(acc * TC_BN);
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
                            if (split) {
#pragma unroll
                                for (int c = 0; c < 32; c += 8) st_v8_cg(work + w.part * part_stride + h + c, v + c);
                            } else if (crow) {
                                store_row(crow, n0 + h, p.N, full_row, v, 32);
                            }
                        }
                    }
                }
                tc_fence_before();
                mbar_arrive(&tempty[acc]);
                if (++acc == 2) acc = 0, aph ^= 1u;
            }
            if (!ok) break;
            if (!split) continue;
            // Each warp takes a ticket for its block once its part is
            // published; the warp holding the last ticket sums every part
            // (its own included, from the workspace) in part order and writes
            // C.  No barrier spans warps, so an aborting warp cannot strand
            // the others.  The warp barrier orders every lane's stores before
            // lane 0's release, and lane 0's acquire before the lanes' loads.
            __syncwarp();
            unsigned int last = 0;
            if (lane == 0) {
                unsigned int* ctr = p.tile_count + w.split_idx * TC_SUBS + sub;
                last = atomic_add_acq_rel(ctr, 1u) == (unsigned int)(p.parts - 1) ? 1u : 0u;
                if (last) atomicExch(ctr, 0u);  // every part has arrived: ready for the next launch
            }
            if (!__shfl_sync(0xffffffffu, last, 0)) continue;
            __syncwarp();
            if (p.parts == 2) {
                // 32 columns of both parts per round trip
#pragma unroll
                for (int h = 0; h < TC_EPI_COLS; h += 32) {
                    float a[32], b[32];
#pragma unroll
                    for (int c = 0; c < 32; c += 8) {
                        ld_v8_cg(work + h + c, a + c);
                        ld_v8_cg(work + part_stride + h + c, b + c);
                    }
#pragma unroll
                    for (int j = 0; j < 32; ++j) a[j] = __fadd_rn(a[j], b[j]);
                    if (crow) store_row(crow, n0 + h, p.N, full_row, a, 32);
                }
            } else {
                // 16 columns of every part per round trip
#pragma unroll
                for (int c = 0; c < TC_EPI_COLS; c += 16) {
                    float v[TC_MAX_PARTS][16];
#pragma unroll
                    for (int j = 0; j < TC_MAX_PARTS; ++j)
                        if (j < p.parts) {
                            ld_v8_cg(work + j * part_stride + c, v[j]);
                            ld_v8_cg(work + j * part_stride + c + 8, v[j] + 8);
                        }
#pragma unroll
                    for (int j = 1; j < TC_MAX_PARTS; ++j)
                        if (j < p.parts) {
#pragma unroll
                            for (int i = 0; i < 16; ++i) v[0][i] = __fadd_rn(v[0][i], v[j][i]);
                        }
                    if (crow) store_row(crow, n0 + c, p.N, full_row, v[0], 16);
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

template <bool X3, bool MSEG>
cudaError_t tc_launch(const TcParams& tp, int teams, const CUtensorMap* m, cudaStream_t s) {
    static bool configured = false;
    if (!configured) {
        const cudaError_t e = cudaFuncSetAttribute(gemm_tc_kernel<X3, MSEG>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TcCfg<X3>::SMEM);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    gemm_tc_kernel<X3, MSEG><<<teams, TC_THREADS, TcCfg<X3>::SMEM, s>>>(tp, m[0], m[1], m[2], m[3], m[4], m[5]);
    return cudaGetLastError();
}

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace

// The planned parameters live in the loop record's tc_params bytes; the four
// tensor maps in its tmap[] array (A_hi, A_lo, B_hi, B_lo, then B_hi and
// B_lo again with a 128-row box for half tiles).
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
        // The planner sizes the grid.  The whole waves of tiles go one tile
        // per team.  When a last, partial wave would leave at least half of
        // the teams idle, its tiles are cut into two 128-column halves (N =
        // 128 MMAs; a half takes about 2/3 of a whole tile's time, its
        // operand traffic per flop being higher).  With fewer tiles than
        // teams, every tile is cut into P contiguous K parts instead, P
        // minimising the length of the wave (in tiles) plus a small charge
        // per extra part for publishing and summing the partial tiles, with
        // at least two k-blocks per part.  Without a split the grid is the
        // fewest teams that give every team the same number of tiles (less
        // L2 contention at equal wave count).  Units are dealt round-robin
        // (static, chunk 1), so the pieces of one tile run side by side on
        // neighbouring teams at the end.
        const int64_t T = kNumSMs;
        const int64_t whole = tp.ntiles / T, rem = tp.ntiles % T;
        int best_p = 1;
        if (whole == 0) {
            const int pmax = (int)std::min<int64_t>(TC_MAX_PARTS, std::max<int64_t>(nkb0 / 2, 1));
            double best = 1.0;
            for (int P = 2; P <= pmax; ++P) {
                const double t = (double)ceil_div(rem * P, T) / P + 0.02 * (P - 1);
                if (t < best - 1e-9) best = t, best_p = P;
            }
        }
        if (whole > 0 && rem > 0 && 2 * rem <= T) {
            tp.half_tiles = rem;
            tp.full_tiles = whole * T;
            tp.nunits = tp.full_tiles + 2 * rem;
            lp.teams = (int)std::min<int64_t>(T, tp.nunits);
        } else if (best_p > 1) {
            tp.split_tiles = rem;
            tp.full_tiles = 0;
            tp.parts = best_p;
            tp.nunits = rem * best_p;
            lp.teams = (int)std::min<int64_t>(T, tp.nunits);
        } else {
            lp.teams = (int)ceil_div(tp.ntiles, ceil_div(tp.ntiles, T));
        }
        chunk_eff = 1;
    }
    // The CTA-pair kernel (planner geometry) when its 256 x 256 tiles give
    // every resident cluster at least one; UPIR_HINT_VARIANT 1 keeps the
    // one-SM kernel, 2 asks for pairs.
    if (lp.variant == 2 && (r->teams || lp.chunk != 0))
        return fail(ctx, UPIR_EUNSUPPORTED, "upir_loop: the CTA-pair GEMM takes planner teams and chunk 0");
    if (!r->teams && lp.chunk == 0 && lp.variant != 1 && tp.ntiles > 0) {
        const int64_t tm2 = ceil_div(lp.trip, 256), tn2 = ceil_div(N, 256), nt2 = tm2 * tn2;
        const int maxc = gemm_tc2_max_clusters();
        if (maxc <= 0 && lp.variant == 2)
            return fail(ctx, UPIR_EUNSUPPORTED, "upir_loop: no cluster of two 576-thread teams fits this GPU");
        if (maxc > 0 && (nt2 >= maxc || lp.variant == 2)) {
            // units dealt round-robin to the clusters; a last wave that would
            // leave at least half of them idle is cut into 128-column halves
            const int64_t C = maxc, whole = nt2 / C, rem = nt2 % C;
            tp.pair = 1;
            tp.tiles_m = tm2;
            tp.tiles_n = tn2;
            tp.ntiles = nt2;
            tp.full_tiles = nt2;
            tp.half_tiles = tp.split_tiles = 0;
            if (whole > 0 && rem > 0 && 2 * rem <= C) {
                tp.full_tiles = whole * C;
                tp.half_tiles = rem;
            }
            tp.nunits = tp.full_tiles + 2 * tp.half_tiles;
            tp.parts = 1;
            lp.teams = (int)(2 * std::min<int64_t>(C, tp.nunits));
            chunk_eff = 1;
        }
    }
    tp.chunk = chunk_eff;
    tp.sk = make_sched_const(tp.nunits, chunk_eff, tp.pair ? lp.teams / 2 : lp.teams);
    if (tp.parts > 1) {
        // partial tiles of every part, then one arrival counter per 32 x 64 block
        const size_t work_bytes = (size_t)tp.split_tiles * tp.parts * TC_BM * TC_BN * sizeof(float);
        const size_t count_bytes = (size_t)tp.split_tiles * TC_SUBS * sizeof(unsigned int);
        const size_t bytes = work_bytes + count_bytes;
        lp.scratch = dev_alloc(ctx, bytes);
        if (!lp.scratch) return fail(ctx, UPIR_ENOMEM, "upir_loop: GEMM split-K workspace of %zu bytes", bytes);
        lp.scratch_bytes = bytes;
        lp.counter_off = work_bytes;
        lp.counter_bytes = count_bytes;
        tp.work = static_cast<float*>(lp.scratch);
        tp.tile_count = reinterpret_cast<unsigned int*>(static_cast<unsigned char*>(lp.scratch) + work_bytes);
        const cudaError_t e = cudaMemsetAsync(tp.tile_count, 0, count_bytes, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "upir_loop: clearing the GEMM split-K counters");
    }
    memcpy(lp.tc_params, &tp, sizeof(tp));
    lp.skip = lp.trip == 0 || N == 0;
    if (lp.skip || K == 0) {
        if (K == 0 && !lp.skip)
            return fail(ctx, UPIR_EUNSUPPORTED, "upir_loop: tensor-core GEMM needs K > 0");
        return UPIR_OK;
    }
    const void* bases[6] = {lp.bufs[0]->dev, lp.bufs[x3 ? 1 : 0]->dev, lp.bufs[na]->dev,
                            lp.bufs[x3 ? na + 1 : na]->dev, lp.bufs[na]->dev, lp.bufs[x3 ? na + 1 : na]->dev};
    const uint64_t rows[6] = {(uint64_t)M, (uint64_t)M, (uint64_t)N, (uint64_t)N, (uint64_t)N, (uint64_t)N};
    const uint32_t box_rows[6] = {TC_BM, TC_BM, TC_BN, TC_BN, TC_BN / 2, TC_BN / 2};
    // the CTA-pair kernel: every operand box is 128 rows (a CTA's share),
    // the last two maps 64 rows of B^T for half tiles
    const uint32_t pair_rows[6] = {128, 128, 128, 128, 64, 64};
    for (int i = 0; i < 6; ++i) {
        const uint32_t br = tp.pair ? pair_rows[i] : box_rows[i];
        upir_status s2 = encode_tmap_2d(ctx, &lp.tmap[i], bases[i], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                                        (uint64_t)K, rows[i], (uint32_t)bk, br, bk * 2);
        if (s2 != UPIR_OK) return s2;
    }
    return UPIR_OK;
}

cudaError_t launch_gemm_tc_loop(upir_ctx, LoopRec& lp, cudaStream_t s) {
    TcParams tp;
    memcpy(&tp, lp.tc_params, sizeof(tp));
    CUtensorMap m[6];
    memcpy(m, lp.tmap, sizeof(m));
    const int nkb = (int)((tp.K + (lp.body == UPIR_BODY_GEMM_BF16X3 ? TcCfg<true>::BK : TcCfg<false>::BK) - 1) /
                          (lp.body == UPIR_BODY_GEMM_BF16X3 ? TcCfg<true>::BK : TcCfg<false>::BK));
    const bool mseg = tp.seg_kb < nkb;
    if (tp.pair) return launch_gemm_tc2(tp, lp.teams, lp.body == UPIR_BODY_GEMM_BF16X3, mseg, m, s);
    if (lp.body == UPIR_BODY_GEMM_BF16X3)
        return mseg ? tc_launch<true, true>(tp, lp.teams, m, s) : tc_launch<true, false>(tp, lp.teams, m, s);
    return mseg ? tc_launch<false, true>(tp, lp.teams, m, s) : tc_launch<false, false>(tp, lp.teams, m, s);
}

}  // namespace upir
