// Tiled 5-point Jacobi sweep (the 2D stencil workload of §6, 5-point form).
// The canonical loop collapse(2) over the interior is tiled by the runtime
// (tiling is one of the loop transformations the separation of loop and
// loop_parallel allows, §3.2) and the tile loop is workshared over teams.
//
// Each team walks its tiles through an S-deep shared-memory ring: one thread
// issues the TMA copy of the (TM + 2) x (TN + 8) halo box of the tile S - 1
// positions ahead, while all threads compute the current tile (TM x TN points,
// 128-bit shared loads, 128-bit streaming global stores).  The per-sweep
// max-norm residual is folded into the reduction variable with one atomic per
// team; max/min are exact in any order, so the result does not depend on
// which team finishes first.
//
// While the two grids fit the L2 (KEEP), the 2D-box kernel reads its input
// with an evict-first L2 policy and stores its output with normal priority
// (otherwise streaming stores): the L2 then keeps the output, which the next
// sweep reads, rather than the input, which the next sweep overwrites.
//
// Under a blocked static schedule a sweep over the previous sweep's output
// walks each team's run of tiles descending (the planner sets `reverse` on
// every other sweep of such a chain): the tiles the previous sweep wrote
// last, still in L2, are read first.  The order is not observable in the
// result.
//
// Grids whose width is not a multiple of 4 have rows that do not start on a
// 16-byte boundary, which a 2D tensor map cannot describe (its row pitch must
// be a multiple of 16 bytes).  jacobi_rows_kernel views such a grid as one
// dimension and copies each halo row on its own, from the 16-byte boundary at
// or before the row's first column; a row then sits in shared memory shifted
// by 0-3 columns, the same shift for the whole row.  Its lanes take the
// tile's columns cyclically (lane q: columns q, q + TN/4, ...), so 32-bit
// shared loads from any shift and 32-bit global stores stay unit-stride.
#include <cstring>

#include "device_common.cuh"
#include "tile_iter.cuh"

namespace upir {

namespace {

// Under a blocked static schedule the team owns tiles [f, f + n); walking
// them descending maps the ascending sequence's tile t to 2 f + n - 1 - t.
__device__ __forceinline__ int64_t tile_reverse_sum(const JacobiParams& p) {
    const int64_t w = blockIdx.x;
    const int64_t f = w * p.sk.base + min(w, p.sk.extra);
    return 2 * f + p.sk.base + (w < p.sk.extra ? 1 : 0) - 1;
}

template <int S, int ROP, bool KEEP>
__global__ void __launch_bounds__(1024) jacobi_tma_kernel(const JacobiParams p,
                                                         const __grid_constant__ CUtensorMap tmap) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar[S];
    __shared__ int2 stage_rc[S];  // (first row, first column) of the tile in each stage; x < 0: none
    __shared__ int last_team;
    const int TM = p.tile_m, TN = p.tile_n, SW = TN + 8;
    const int stage_floats = ((TM + 2) * SW + 255) / 256 * 256;  // 1 KB multiples
    // stage 0 starts on a 1024-byte boundary (the launch adds 1 KB of slack)
    float* ring = smem_align1k<float>(smem_raw);
    const int tpr = TN / 4;                    // threads per tile row (4 columns each)
    const int tx = threadIdx.x % tpr, ty = threadIdx.x / tpr;
    const int nty = blockDim.x / tpr;          // thread rows
    const bool active = threadIdx.x < nty * tpr;
    const uint32_t box_bytes = (uint32_t)((TM + 2) * SW * sizeof(float));
    const int cols = (int)p.cols, r_ub = (int)p.r_ub;
    float racc = ROP == UPIR_RED_MIN ? __int_as_float(0x7f800000) : -__int_as_float(0x7f800000);

    TileIter it = tile_iter_begin(p);
    const int64_t rev_sum = tile_reverse_sum(p);
    const uint64_t in_policy = KEEP ? l2_evict_first_policy() : 0;
    // producer side (one thread): next tile -> (row, column), then its copy
    auto issue_next = [&](int s) {
        int64_t t = tile_iter_next(it, p);
        if (t >= 0 && p.reverse) t = rev_sum - t;
        if (t < 0) {
            stage_rc[s] = make_int2(-1, -1);
            return;
        }
        const int tr = (int)(t / p.tiles_c), tc = (int)(t - (int64_t)tr * p.tiles_c);
        const int r0 = (int)p.r_lb + tr * TM, c0 = tc * TN;
        stage_rc[s] = make_int2(r0, c0);
        mbar_arrive_expect_tx(&bar[s], box_bytes);
        if (KEEP) tma_load_2d_hint(ring + s * stage_floats, &tmap, &bar[s], c0 - 4, r0 - 1, in_policy);
        else tma_load_2d(ring + s * stage_floats, &tmap, &bar[s], c0 - 4, r0 - 1);
    };

    if (threadIdx.x == 0) {
        prefetch_tmap(&tmap);
#pragma unroll
        for (int s = 0; s < S; ++s) mbar_init(&bar[s], 1);
        fence_mbar_init();
    }
    // the previous sweep's output is this sweep's input: wait for it
    griddep_wait_prior(p.wait_prior);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int s = 0; s < S; ++s) issue_next(s);
    }
    __syncthreads();
    griddep_launch_dependents();

    bool failed = false;
    int s = 0, prev = -1;
    uint32_t parity = 0;
    for (;;) {
        const int2 rc = stage_rc[s];
        if (rc.x < 0) break;
        if (!__syncthreads_and(mbar_wait_bounded(&bar[s], parity, p.spin_limit, p.err_word))) {
            failed = true;
            break;
        }
        // with three or more stages, every thread has finished the previous
        // stage once it passes this barrier: its refill goes out now, and its
        // stage_rc entry is next read two barriers later
        if (S >= 3 && threadIdx.x == 0 && prev >= 0) issue_next(prev);
        if (active) {
            const float* cen = ring + s * stage_floats + (ty + 1) * SW + 4 + 4 * tx;
            const int c = rc.y + 4 * tx;
            const bool full = c >= 1 && c + 3 <= cols - 2;
            const int nrows = min(TM, r_ub - rc.x);
            float* out = p.uout + (size_t)(rc.x + ty) * cols + c;
            const size_t out_step = (size_t)nty * cols;
#pragma unroll 4
            for (int i2 = ty; i2 < nrows; i2 += nty, cen += nty * SW, out += out_step) {
                const float4 C = *reinterpret_cast<const float4*>(cen);
                const float4 N = *reinterpret_cast<const float4*>(cen - SW);
                const float4 Sv = *reinterpret_cast<const float4*>(cen + SW);
                const float Wl = cen[-1], Er = cen[4];
                float4 v;
                v.x = __fmul_rn(0.25f, __fadd_rn(__fadd_rn(N.x, Sv.x), __fadd_rn(Wl, C.y)));
                v.y = __fmul_rn(0.25f, __fadd_rn(__fadd_rn(N.y, Sv.y), __fadd_rn(C.x, C.z)));
                v.z = __fmul_rn(0.25f, __fadd_rn(__fadd_rn(N.z, Sv.z), __fadd_rn(C.y, C.w)));
                v.w = __fmul_rn(0.25f, __fadd_rn(__fadd_rn(N.w, Sv.w), __fadd_rn(C.z, Er)));
                if (full) {
                    if (KEEP) *reinterpret_cast<float4*>(out) = v;
                    else __stcs(reinterpret_cast<float4*>(out), v);
                    if (ROP) {
                        racc = fold(racc, fabsf(__fsub_rn(v.x, C.x)), ROP);
                        racc = fold(racc, fabsf(__fsub_rn(v.y, C.y)), ROP);
                        racc = fold(racc, fabsf(__fsub_rn(v.z, C.z)), ROP);
                        racc = fold(racc, fabsf(__fsub_rn(v.w, C.w)), ROP);
                    }
                } else {
                    const float vs[4] = {v.x, v.y, v.z, v.w};
                    const float cs[4] = {C.x, C.y, C.z, C.w};
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        if (c + j >= 1 && c + j <= cols - 2) {
                            out[j] = vs[j];
                            if (ROP) racc = fold(racc, fabsf(__fsub_rn(vs[j], cs[j])), ROP);
                        }
                    }
                }
            }
        }
        if (S < 3) {
            __syncthreads();  // every thread is done with stage s
            if (threadIdx.x == 0) issue_next(s);
            __syncthreads();  // stage_rc[s] is read again (at once when S == 1)
        }
        prev = s;
        if (++s == S) {
            s = 0;
            parity ^= 1u;
        }
    }

    if (ROP && !failed) {
        const float b = block_fold(racc, ROP);
        if (threadIdx.x == 0) atomic_fold_minmax(p.rvar, b, ROP);
    }
    tile_iter_reset(p, &last_team);
    if (failed && threadIdx.x == 0) {
        // copies still in flight get a bounded chance to land before the
        // shared memory is released
        for (int k = 0; k < S; ++k) {
            if (stage_rc[k].x < 0) continue;
            if (!mbar_wait_bounded(&bar[k], 0, p.spin_limit, nullptr))
                mbar_wait_bounded(&bar[k], 1, p.spin_limit, nullptr);
        }
    }
}

// The row-copy variant (widths that are not a multiple of 4).  Per stage,
// thread 0 takes the next tile and arms the stage's barrier while the team
// computes; after the barrier that opens the following stage (the team is
// then done with this one), threads 0 .. TM + 1 issue one halo-row copy each,
// so the copies cost every thread at most one instruction and a tile costs
// one team barrier.  TNC: the tile width fixed at compile time (0: taken from
// the parameters), so that a thread's column offsets fold into the shared
// loads and global stores; tiles whose columns are all interior skip the
// per-point column test.
template <int S, int ROP, int TNC>
__global__ void __launch_bounds__(1024) jacobi_rows_kernel(const JacobiParams p,
                                                          const __grid_constant__ CUtensorMap tmap) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar[S];
    __shared__ int2 stage_rc[S];  // (first row, first column) of the tile in each stage; x < 0: none
    __shared__ int last_team;
    const int TM = p.tile_m, TN = TNC ? TNC : p.tile_n;
    const int SW = jacobi_rt_pitch(TN);  // every row copy lands on a 128-byte boundary
    const int stage_floats = ((TM + 2) * SW + 255) / 256 * 256;
    float* ring = smem_align1k<float>(smem_raw);
    const int tpr = TN / 4;
    const int tx = threadIdx.x % tpr, ty = threadIdx.x / tpr;
    const int nty = blockDim.x / tpr;
    const bool active = threadIdx.x < nty * tpr;
    const uint32_t box_bytes = (uint32_t)((TM + 2) * (TN + 8) * sizeof(float));
    const int cols = (int)p.cols, r_ub = (int)p.r_ub;
    const uint32_t cq = (uint32_t)cols & 3u;
    float racc = ROP == UPIR_RED_MIN ? __int_as_float(0x7f800000) : -__int_as_float(0x7f800000);

    TileIter it = tile_iter_begin(p);
    const int64_t rev_sum = tile_reverse_sum(p);
    // thread 0: the team's next tile into stage s, arming the stage's barrier
    auto take_next = [&](int s) {
        int64_t t = tile_iter_next(it, p);
        if (t >= 0 && p.reverse) t = rev_sum - t;
        if (t < 0) {
            stage_rc[s] = make_int2(-1, -1);
            return;
        }
        const int tr = (int)(t / p.tiles_c), tc = (int)(t - (int64_t)tr * p.tiles_c);
        stage_rc[s] = make_int2((int)p.r_lb + tr * TM, tc * TN);
        mbar_arrive_expect_tx(&bar[s], box_bytes);
    };
    // halo row i of the tile in stage s, from the 16-byte boundary at or
    // before its grid column c0 - 4 (a multiple of 4 elements of the 1D view)
    auto copy_rows = [&](int s) {
        const int2 rc = stage_rc[s];
        if (rc.x < 0) return;
        for (int i = threadIdx.x; i < TM + 2; i += blockDim.x) {
            const int64_t g = (int64_t)(rc.x - 1 + i) * cols + rc.y - 4;
            tma_load_1d(ring + s * stage_floats + i * SW, &tmap, &bar[s], (int32_t)(g & ~(int64_t)3));
        }
    };

    if (threadIdx.x == 0) {
        prefetch_tmap(&tmap);
#pragma unroll
        for (int s = 0; s < S; ++s) mbar_init(&bar[s], 1);
        fence_mbar_init();
    }
    // the previous sweep's output is this sweep's input: wait for it
    griddep_wait_prior(p.wait_prior);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int s = 0; s < S; ++s) take_next(s);
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < S; ++s) copy_rows(s);
    griddep_launch_dependents();

    bool failed = false;
    int s = 0, prev = -1;
    uint32_t parity = 0;
    for (;;) {
        const int2 rc = stage_rc[s];
        if (rc.x < 0) break;
        if (!__syncthreads_and(mbar_wait_bounded(&bar[s], parity, p.spin_limit, p.err_word))) {
            failed = true;
            break;
        }
        // past this barrier every thread has left the previous stage, whose
        // next tile thread 0 took an iteration ago: its row copies go out
        if (prev >= 0) copy_rows(prev);
        // every thread has read stage_rc[s] and the stage's phase is complete:
        // the stage's next tile can be taken and its barrier re-armed
        if (threadIdx.x == 0) take_next(s);
        if (active) {
            const float* st = ring + s * stage_floats;
            const int nrows = min(TM, r_ub - rc.x);
            // halo row h sits shifted by ((r0 - 1 + h) * cols + c0) mod 4 columns
            const uint32_t sh0 = ((uint32_t)(rc.x - 1) * cq + (uint32_t)rc.y) & 3u;
            // every column of the tile interior: no per-point column test
            const bool full = rc.y >= 1 && rc.y + TN <= cols - 1;
            // grid column c0 of the rows above, at and below the thread's
            // first output row, offset by its first column.  Its rows are nty
            // apart; with nty a multiple of 4 they all have the same shifts
            const int dn = (int)((sh0 + (uint32_t)ty * cq) & 3u);
            const int dm = (int)((sh0 + (uint32_t)(ty + 1) * cq) & 3u);
            const int ds = (int)((sh0 + (uint32_t)(ty + 2) * cq) & 3u);
            const bool same_shift = (nty & 3) == 0;
            const float* rn = st + ty * SW + dn + 4 + tx;
            const float* rm = st + (ty + 1) * SW + dm + 4 + tx;
            const float* rs = st + (ty + 2) * SW + ds + 4 + tx;
            float* orow = p.uout + ((size_t)(rc.x + ty) * cols + rc.y + tx);
            const size_t ostep = (size_t)nty * cols;
#pragma unroll 2
            for (int i2 = ty; i2 < nrows; i2 += nty, rn += nty * SW, rm += nty * SW, rs += nty * SW, orow += ostep) {
                if (!same_shift) {
                    rn = st + i2 * SW + ((sh0 + (uint32_t)i2 * cq) & 3u) + 4 + tx;
                    rm = st + (i2 + 1) * SW + ((sh0 + (uint32_t)(i2 + 1) * cq) & 3u) + 4 + tx;
                    rs = st + (i2 + 2) * SW + ((sh0 + (uint32_t)(i2 + 2) * cq) & 3u) + 4 + tx;
                }
                if (full) {
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int q = tpr * j;
                        const float cv = rm[q];
                        const float v = __fmul_rn(0.25f, __fadd_rn(__fadd_rn(rn[q], rs[q]),
                                                                   __fadd_rn(rm[q - 1], rm[q + 1])));
                        __stcs(orow + q, v);
                        if (ROP) racc = fold(racc, fabsf(__fsub_rn(v, cv)), ROP);
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int q = tpr * j;
                        const int c = rc.y + tx + q;
                        const float cv = rm[q];
                        const float v = __fmul_rn(0.25f, __fadd_rn(__fadd_rn(rn[q], rs[q]),
                                                                   __fadd_rn(rm[q - 1], rm[q + 1])));
                        if (c >= 1 && c <= cols - 2) {
                            __stcs(orow + q, v);
                            if (ROP) racc = fold(racc, fabsf(__fsub_rn(v, cv)), ROP);
                        }
                    }
                }
            }
        }
        prev = s;
        if (++s == S) {
            s = 0;
            parity ^= 1u;
        }
    }

    if (ROP && !failed) {
        const float b = block_fold(racc, ROP);
        if (threadIdx.x == 0) atomic_fold_minmax(p.rvar, b, ROP);
    }
    tile_iter_reset(p, &last_team);
    if (failed && threadIdx.x == 0) {
        // copies still in flight get a bounded chance to land before the
        // shared memory is released
        for (int k = 0; k < S; ++k) {
            if (stage_rc[k].x < 0) continue;
            if (!mbar_wait_bounded(&bar[k], 0, p.spin_limit, nullptr))
                mbar_wait_bounded(&bar[k], 1, p.spin_limit, nullptr);
        }
    }
}

using JacobiKernel = void (*)(const JacobiParams, const CUtensorMap);

template <int S, bool ROWS, int TNC = 0>
JacobiKernel pick_rop(int rop, bool keep) {
    if (ROWS) {
        if (rop == UPIR_RED_MAX) return jacobi_rows_kernel<S, UPIR_RED_MAX, TNC>;
        if (rop == UPIR_RED_MIN) return jacobi_rows_kernel<S, UPIR_RED_MIN, TNC>;
        return jacobi_rows_kernel<S, 0, TNC>;
    }
    if (keep) {
        if (rop == UPIR_RED_MAX) return jacobi_tma_kernel<S, UPIR_RED_MAX, true>;
        if (rop == UPIR_RED_MIN) return jacobi_tma_kernel<S, UPIR_RED_MIN, true>;
        return jacobi_tma_kernel<S, 0, true>;
    }
    if (rop == UPIR_RED_MAX) return jacobi_tma_kernel<S, UPIR_RED_MAX, false>;
    if (rop == UPIR_RED_MIN) return jacobi_tma_kernel<S, UPIR_RED_MIN, false>;
    return jacobi_tma_kernel<S, 0, false>;
}

template <bool ROWS, int TNC = 0>
JacobiKernel pick_stages(int stages, int rop, bool keep) {
    switch (stages) {
        case 1: return pick_rop<1, ROWS, TNC>(rop, keep);
        case 2: return pick_rop<2, ROWS, TNC>(rop, keep);
        case 3: return pick_rop<3, ROWS, TNC>(rop, keep);
        default: return pick_rop<4, ROWS, TNC>(rop, keep);
    }
}

// the row-copy kernel has a fixed-width instantiation for 128-column tiles
// keep: the 2D-box kernel reading its input evict-first and storing with
// normal priority (the row-copy kernel ignores it)
JacobiKernel pick_kernel(int stages, int rop, bool rows, int tile_n, bool keep) {
    if (!rows) return pick_stages<false>(stages, rop, keep);
    return tile_n == 128 ? pick_stages<true, 128>(stages, rop, false) : pick_stages<true>(stages, rop, false);
}

bool configure_jacobi(JacobiKernel k) {
    // each instantiation gets the large dynamic shared memory window once
    static JacobiKernel done[64] = {};
    for (auto& d : done) {
        if (d == k) return true;
        if (!d) {
            if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024) != cudaSuccess)
                return false;
            d = k;
            return true;
        }
    }
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024) == cudaSuccess;
}

}  // namespace

size_t jacobi_tma_smem_bytes(int tile_m, int tile_n, int stages, bool rows) {
    const size_t sw = rows ? (size_t)jacobi_rt_pitch(tile_n) : (size_t)tile_n + 8;
    const size_t stage_floats = ((size_t)(tile_m + 2) * sw + 255) / 256 * 256;
    return stage_floats * sizeof(float) * stages + 1024;
}

int jacobi_tma_max_teams_per_sm(int units, int tile_m, int tile_n, int stages, bool rows, bool keep) {
    JacobiKernel k = pick_kernel(stages, UPIR_RED_MAX, rows, tile_n, keep);
    if (!configure_jacobi(k)) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, units,
                                                      jacobi_tma_smem_bytes(tile_m, tile_n, stages, rows)) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

cudaError_t launch_jacobi_tma(int teams, int units, const JacobiParams& p, const void* tmap,
                              cudaStream_t s) {
    JacobiKernel k = pick_kernel(p.stages, p.rvar ? p.rop : 0, p.rows_tma != 0, p.tile_n, p.keep_l2 != 0);
    if (!configure_jacobi(k)) return cudaGetLastError();
    CUtensorMap m;
    memcpy(&m, tmap, sizeof(m));
    return launch_pdl(k, teams, units, jacobi_tma_smem_bytes(p.tile_m, p.tile_n, p.stages, p.rows_tma != 0), s,
                      p, m);
}

}  // namespace upir
