// Stencil loop nests beyond the single 5-point sweep (the 2D stencil workload
// of §6):
//
//  * JACOBI5_TB: several Jacobi sweeps carried by one loop (the time loop of
//    the stencil nest tiled together with its space loops).  A team loads a
//    tile with a halo as deep as the number of sweeps, runs every sweep in
//    shared memory on a shrinking region, and writes only the last sweep's
//    values: the grid crosses HBM once per `sweeps` sweeps instead of once
//    per sweep.  Each sweep does exactly the arithmetic of a JACOBI5 sweep, so
//    the field and the per-sweep residuals are bit-identical to running the
//    sweeps one loop at a time.
//  * FILTER7: the size-7 filter, a 7 x 7 weighted window accumulated by fused
//    multiply-adds in row-major tap order.  Each thread streams the input rows
//    of its 4-column, 4-row output block through registers, so every input
//    row is read from shared memory once per block and the weights stay in
//    the kernel parameters.  Two ring stages keep four teams per SM.
//
// Both kernels are persistent teams over the tile loop with TMA copies of the
// halo boxes into a shared-memory ring; every mbarrier wait is bounded.
#include <cstring>

#include "device_common.cuh"
#include "tile_iter.cuh"

namespace upir {

namespace {

constexpr float kInf = __builtin_huge_valf();

// ----------------------------------------------------------------------------
// JACOBI5_TB
// ----------------------------------------------------------------------------

// Plane = (tile_m + 2 sweeps) rows x (tile_n + 2 halo_c) columns, rounded up
// to 1 KB so that every plane starts where a TMA copy may land.
__host__ __device__ inline size_t tb_plane_floats(int tm, int tn, int sweeps, int hc) {
    return ((size_t)(tm + 2 * sweeps) * (tn + 2 * hc) + 255) / 256 * 256;
}

// What one lane needs to sweep its columns of a strip of box rows.
// A box row is 32 lanes x 4 columns (TB_BC floats).
constexpr int TB_BC = 128;

struct TbLane {
    int lane;
    int ulo, uhi;      // box rows the loop updates
    int own_lo, own_hi;  // box rows the tile owns
    bool ucol[4];      // the lane's columns that the loop updates
    bool own_c;        // the lane's columns belong to the tile
};

// One 5-point row update of a lane's four points, 0.25 * ((N + S) + (W + E))
// with every operation rounded (JACOBI5's arithmetic), two points per paired
// instruction; points the loop does not update keep their value when EDGE.
template <bool EDGE>
__device__ __forceinline__ float4 tb_point4(const TbLane& L, int i, const float4& N, const float4& C,
                                            const float4& S) {
    // box edges: lane 0's west and the last lane's east neighbour are not
    // copied in; they only feed points outside the valid region
    const float Wl = __shfl_up_sync(0xffffffffu, C.w, 1);
    const float Er = __shfl_down_sync(0xffffffffu, C.x, 1);
    const F2 q = f2(0.25f, 0.25f);
    const F2 ns0 = f2_add(f2(N.x, N.y), f2(S.x, S.y)), ns1 = f2_add(f2(N.z, N.w), f2(S.z, S.w));
    const F2 we0 = f2_add(f2(Wl, C.x), f2(C.y, C.z)), we1 = f2_add(f2(C.y, C.z), f2(C.w, Er));
    const F2 v0 = f2_mul(q, f2_add(ns0, we0)), v1 = f2_mul(q, f2_add(ns1, we1));
    float4 v;
    f2_split(v0, v.x, v.y);
    f2_split(v1, v.z, v.w);
    if (EDGE) {
        const bool urow = i >= L.ulo && i < L.uhi;
        v.x = urow && L.ucol[0] ? v.x : C.x;
        v.y = urow && L.ucol[1] ? v.y : C.y;
        v.z = urow && L.ucol[2] ? v.z : C.z;
        v.w = urow && L.ucol[3] ? v.w : C.w;
    }
    return v;
}

// Largest |v - C| of a lane's four points.
__device__ __forceinline__ float tb_absdiff_max(const float4& v, const float4& C) {
    float d0, d1, d2, d3;
    f2_split(f2_sub(f2(v.x, v.y), f2(C.x, C.y)), d0, d1);
    f2_split(f2_sub(f2(v.z, v.w), f2(C.z, C.w)), d2, d3);
    return fmaxf(fmaxf(fabsf(d0), fabsf(d1)), fmaxf(fabsf(d2), fabsf(d3)));
}

// Smallest |v - C| over the owned points the loop updates (min reductions).
template <bool EDGE>
__device__ __forceinline__ void tb_resid_min(const TbLane& L, int i, const float4& v, const float4& C,
                                             float& rk) {
    const bool urow = !EDGE || (i >= L.ulo && i < L.uhi);
    if (urow && L.own_c && i >= L.own_lo && i < L.own_hi) {
        if (!EDGE || L.ucol[0]) rk = fminf(rk, fabsf(__fsub_rn(v.x, C.x)));
        if (!EDGE || L.ucol[1]) rk = fminf(rk, fabsf(__fsub_rn(v.y, C.y)));
        if (!EDGE || L.ucol[2]) rk = fminf(rk, fabsf(__fsub_rn(v.z, C.z)));
        if (!EDGE || L.ucol[3]) rk = fminf(rk, fabsf(__fsub_rn(v.w, C.w)));
    }
}

// One row of a lane's four points: update, store, residual.  Residuals: for
// max, every row folds into rk unmasked (the caller keeps rk only for lanes
// whose columns are valid: points the loop does not update give 0 and halo
// points repeat a neighbour tile's values, neither of which changes a
// maximum); for min, exactly the owned, updated points.
template <int ROP, bool EDGE>
__device__ __forceinline__ void tb_row(const TbLane& L, int i, const float4& N, const float4& C, const float4& S,
                                       float* out, float& rk) {
    const float4 v = tb_point4<EDGE>(L, i, N, C, S);
    *reinterpret_cast<float4*>(out) = v;
    if (ROP == UPIR_RED_MAX) rk = fmaxf(rk, tb_absdiff_max(v, C));
    else if (ROP == UPIR_RED_MIN) tb_resid_min<EDGE>(L, i, v, C, rk);
}

// Rows [i0, i1) of one sweep, src -> dst, two per step, so that the rows
// above and below rotate through registers.
template <int ROP, bool EDGE>
__device__ __forceinline__ void tb_strip(const TbLane& L, const float* src, float* dst, int i0, int i1,
                                              float& rk) {
    const float* in = src + (i0 + 1) * TB_BC + 4 * L.lane;  // row below the current one
    float* out = dst + i0 * TB_BC + 4 * L.lane;
    float4 N = *reinterpret_cast<const float4*>(in - 2 * TB_BC);
    float4 C = *reinterpret_cast<const float4*>(in - TB_BC);
    int i = i0;
    for (; i + 1 < i1; i += 2, in += 2 * TB_BC, out += 2 * TB_BC) {
        const float4 S = *reinterpret_cast<const float4*>(in);
        const float4 S2 = *reinterpret_cast<const float4*>(in + TB_BC);
        tb_row<ROP, EDGE>(L, i, N, C, S, out, rk);
        tb_row<ROP, EDGE>(L, i + 1, C, S, S2, out + TB_BC, rk);
        N = S;
        C = S2;
    }
    if (i < i1) tb_row<ROP, EDGE>(L, i, N, C, *reinterpret_cast<const float4*>(in), out, rk);
}


// Smem: two input planes (the tile being swept and the next tile's copy) and
// one scratch plane for the ping-pong of the sweeps.
template <int T, int ROP>
__global__ void __launch_bounds__(1024, 1) jacobi_tb_kernel(const JacobiTBParams p,
                                                           const __grid_constant__ CUtensorMap tmap) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ int2 stage_rc[2];
    __shared__ int last_team;
    float* base = smem_align1k<float>(smem_raw);
    const int TM = p.tile_m, TN = p.tile_n, HC = p.halo_c;
    const int BR = TM + 2 * T, BC = TB_BC;  // box rows and columns (TN + 2 HC == TB_BC)
    const size_t plane = tb_plane_floats(TM, TN, T, HC);
    // stage t of the copy ring (computed, not indexed, so that the compiler
    // keeps these as shared-memory addresses)
    auto ring = [&](int t) { return base + (size_t)t * plane; };
    float* const scratch = base + 2 * plane;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const uint32_t box_bytes = (uint32_t)(BR * BC * sizeof(float));
    const int64_t cols = p.cols, r_lb = p.r_lb, r_ub = p.r_ub;
    // per-warp residual of each sweep, folded over the team's tiles
    __shared__ float racc[T][32];
    const float ident = ROP == UPIR_RED_MIN ? kInf : -kInf;
    for (int t = threadIdx.x; t < T * 32; t += blockDim.x) racc[t >> 5][t & 31] = ident;
    // warp w sweeps box rows [1 + w h0, 1 + (w + 1) h0), clipped to the rows
    // that are valid after each sweep
    const int h0 = (BR - 2 + nwarps - 1) / nwarps;
    const int w_lo = 1 + warp * h0, w_hi = w_lo + h0;

    TileIter it = tile_iter_begin(p);
    auto issue = [&](int s) {  // thread 0: the next tile's box into stage s
        const int64_t t = tile_iter_next(it, p);
        if (t < 0) {
            stage_rc[s] = make_int2(-1, -1);
            return;
        }
        const int tr = (int)(t / p.tiles_c), tc = (int)(t - (int64_t)tr * p.tiles_c);
        const int r0 = (int)r_lb + tr * TM, c0 = tc * TN;
        stage_rc[s] = make_int2(r0, c0);
        mbar_arrive_expect_tx(&bar[s], box_bytes);
        tma_load_2d(ring(s), &tmap, &bar[s], c0 - HC, r0 - T);
    };

    if (threadIdx.x == 0) {
        prefetch_tmap(&tmap);
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    griddep_wait_prior(p.wait_prior);
    if (threadIdx.x == 0) issue(0);
    __syncthreads();
    griddep_launch_dependents();

    bool failed = false;
    int s = 0;
    uint32_t parities = 0;  // bit t: phase parity of stage t's barrier
    for (;;) {
        const int2 rc = stage_rc[s];
        if (rc.x < 0) break;
        if (!__syncthreads_and(mbar_wait_bounded(&bar[s], (parities >> s) & 1u, p.spin_limit, p.err_word))) {
            failed = true;
            break;
        }
        parities ^= 1u << s;
        // the other stage was released by the previous tile: copy the next tile into it
        if (threadIdx.x == 0) issue(s ^ 1);
        // this lane's four columns: updated by the loop, and owned by the tile;
        // the box rows [ulo, uhi) are the loop's rows
        TbLane L;
        L.lane = lane;
        const int64_t gc0 = (int64_t)rc.y - HC + 4 * lane;
#pragma unroll
        for (int j = 0; j < 4; ++j) L.ucol[j] = gc0 + j >= 1 && gc0 + j <= cols - 2;
        L.own_c = 4 * lane >= HC && 4 * lane < HC + TN;
        const int64_t row0 = (int64_t)rc.x - T;  // grid row of box row 0
        L.ulo = (int)max((int64_t)0, min((int64_t)BR, r_lb - row0));
        L.uhi = (int)max((int64_t)0, min((int64_t)BR, r_ub - row0));
        L.own_lo = T;
        L.own_hi = T + TM;
        // a tile whose box holds only updated points needs no masks
        const bool edge = L.ulo > 0 || L.uhi < BR || (int64_t)rc.y - HC < 1 || (int64_t)rc.y - HC + BC - 1 > cols - 2;
        // T sweeps: ring(s) -> scratch -> ring(s) -> ...  A warp owns a strip
        // of consecutive box rows, lane l the columns 4l .. 4l + 3, so the
        // west and east neighbours come from the adjacent lanes.
#pragma unroll
        for (int k = 1; k <= T; ++k) {
            const float* src = (k & 1) ? ring(s) : scratch;
            float* dst = (k & 1) ? scratch : ring(s);
            const int i0 = max(w_lo, k), i1 = min(w_hi, BR - k);
            const int gv = (k + 3) / 4;                  // lanes whose columns are all valid
            const bool lane_valid = lane >= gv && lane <= 31 - gv;
            float rk = ROP == UPIR_RED_MIN ? kInf : -kInf;
            if (i0 < i1) {
                if (edge) tb_strip<ROP, true>(L, src, dst, i0, i1, rk);
                else tb_strip<ROP, false>(L, src, dst, i0, i1, rk);
            }
            if (ROP) {
                float r = (ROP == UPIR_RED_MAX && !lane_valid) ? ident : rk;
#pragma unroll
                for (int m = 16; m >= 1; m >>= 1) r = fold(r, __shfl_xor_sync(0xffffffffu, r, m), ROP);
                if (lane == 0) racc[k - 1][warp] = fold(racc[k - 1][warp], r, ROP);
            }
            __syncthreads();
        }
        // the last sweep's owned, updated points go out
        {
            const float* fin = (T & 1) ? scratch : ring(s);
            const int opr = TN / 4;  // float4 groups per owned row
            const int ox = threadIdx.x % opr, oy = threadIdx.x / opr, noy = blockDim.x / opr;
            const int64_t gc = (int64_t)rc.y + 4 * ox;
            const int nrows = (int)min((int64_t)TM, r_ub - rc.x);
            if (oy < noy && gc < cols) {
                const bool full = gc >= 1 && gc + 3 <= cols - 2;
                for (int i = oy; i < nrows; i += noy) {
                    const float4 v = *reinterpret_cast<const float4*>(fin + (T + i) * BC + HC + 4 * ox);
                    float* out = p.uout + (rc.x + i) * cols + gc;
                    if (full) {
                        __stcs(reinterpret_cast<float4*>(out), v);
                    } else {
                        const float vs[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            if (gc + j >= 1 && gc + j <= cols - 2) out[j] = vs[j];
                    }
                }
            }
        }
        // no barrier here: the next tile's opening barrier orders these reads
        // of ring(s) and the scratch plane before the copy into ring(s) and
        // the next sweeps' writes
        s ^= 1;
    }

    if (ROP && !failed) {
        __syncthreads();
        // warp w folds the per-warp values of sweeps w, w + nwarps, ... into
        // the reduction variable
        for (int k = warp; k < T; k += nwarps) {
            float r = lane < nwarps ? racc[k][lane] : ident;
#pragma unroll
            for (int m = 16; m >= 1; m >>= 1) r = fold(r, __shfl_xor_sync(0xffffffffu, r, m), ROP);
            if (lane == 0) atomic_fold_minmax(p.rvar + k, r, ROP);
        }
    }
    tile_iter_reset(p, &last_team);
    if (failed && threadIdx.x == 0) {
        // copies still in flight get a bounded chance to land before the
        // shared memory is released
        for (int k = 0; k < 2; ++k) {
            if (stage_rc[k].x < 0) continue;
            mbar_wait_bounded(&bar[k], (parities >> k) & 1u, p.spin_limit, nullptr);
        }
    }
}

using TBKernel = void (*)(const JacobiTBParams, const CUtensorMap);

template <int T>
TBKernel tb_pick_rop(int rop) {
    if (rop == UPIR_RED_MAX) return jacobi_tb_kernel<T, UPIR_RED_MAX>;
    if (rop == UPIR_RED_MIN) return jacobi_tb_kernel<T, UPIR_RED_MIN>;
    return jacobi_tb_kernel<T, 0>;
}

TBKernel tb_pick(int sweeps, int rop) {
    switch (sweeps) {
        case 1: return tb_pick_rop<1>(rop);
        case 2: return tb_pick_rop<2>(rop);
        case 3: return tb_pick_rop<3>(rop);
        case 4: return tb_pick_rop<4>(rop);
        case 5: return tb_pick_rop<5>(rop);
        case 6: return tb_pick_rop<6>(rop);
        case 7: return tb_pick_rop<7>(rop);
        case 8: return tb_pick_rop<8>(rop);
        default: return nullptr;
    }
}

// ----------------------------------------------------------------------------
// FILTER7
// ----------------------------------------------------------------------------


// Box: (tile_m + 6) x (tile_n + 8) floats (the columns widened to whole
// 16-byte groups), rounded up to 1 KB per stage.
__host__ __device__ inline size_t f7_stage_floats(int tm, int tn) {
    return ((size_t)(tm + 6) * (tn + 8) + 255) / 256 * 256;
}

// S-stage TMA ring (S >= 2) of (TM + 6) x (TN + 8) input boxes; each thread
// computes strips of RS output rows x 4 columns.  A tile costs one team
// barrier: past the barrier that opens stage s every thread has left the
// stage computed before it, whose refill then goes out.  The end of the
// team's tiles also completes its stage's barrier (an arrival without bytes),
// so every thread reads a stage's tile record only after that barrier, and
// the record's next write (the stage's refill) comes a barrier later.
// TMC / TNC fix the tile shape at compile time (0: taken from the
// parameters) so that shared-memory offsets fold into the loads; tiles whose
// outputs are all inside the loop's rows and the interior columns store
// without per-point tests.
// acc (low half: output row 2p of a pair, high half: row 2p + 1) plus the
// weight pair w2 times x in both halves, one rounding per half (the paired
// form of fmaf; subnormals kept)
__device__ __forceinline__ void fma2_bcast(float& lo, float& hi, unsigned long long w2, float x) {
    asm("{\n\t.reg .b64 xx, acc;\n\t"
        "mov.b64 xx, {%2, %2};\n\t"
        "mov.b64 acc, {%0, %1};\n\t"
        "fma.rn.f32x2 acc, %3, xx, acc;\n\t"
        "mov.b64 {%0, %1}, acc;\n\t}"
        : "+f"(lo), "+f"(hi)
        : "f"(x), "l"(w2));
}

// teams per SM each form is built for: four with 4-row strips (64
// registers), three with scalar 8-row strips, two with paired 8-row strips
template <int RS, bool PAIR>
constexpr int f7_min_teams() { return RS == 4 ? 4 : (PAIR ? 2 : 3); }

template <int S, int TMC, int TNC, int RS, bool PAIR>
__global__ void __launch_bounds__(kFilter7Units, f7_min_teams<RS, PAIR>()) filter7_kernel(const Filter7Params p,
                                                                const __grid_constant__ CUtensorMap tmap) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar[S];
    __shared__ int2 stage_rc[S];
    __shared__ int last_team;
    float* ring = smem_align1k<float>(smem_raw);
    const int TM = TMC ? TMC : p.tile_m, TN = TNC ? TNC : p.tile_n, BW = TN + 8;
    const size_t stage = f7_stage_floats(TM, TN);
    const int tpr = TN / 4;
    const int tx = threadIdx.x % tpr, ty = threadIdx.x / tpr;  // 4 columns x RS rows per strip
    const int nty = kFilter7Units / tpr;
    const uint32_t box_bytes = (uint32_t)((TM + 6) * BW * sizeof(float));
    const int64_t cols = p.cols, r_ub = p.r_ub;

    static_assert(S >= 2, "the ring refills a stage while the team computes another");
    TileIter it = tile_iter_begin(p);
    auto issue = [&](int s) {
        const int64_t t = tile_iter_next(it, p);
        if (t < 0) {
            stage_rc[s] = make_int2(-1, -1);
            mbar_arrive(&bar[s]);  // completes the phase: the team sees the end
            return;
        }
        const int tr = (int)(t / p.tiles_c), tc = (int)(t - (int64_t)tr * p.tiles_c);
        const int r0 = (int)p.r_lb + tr * TM, c0 = tc * TN;
        stage_rc[s] = make_int2(r0, c0);
        mbar_arrive_expect_tx(&bar[s], box_bytes);
        tma_load_2d(ring + s * stage, &tmap, &bar[s], c0 - 4, r0 - 3);
    };

    if (threadIdx.x == 0) {
        prefetch_tmap(&tmap);
#pragma unroll
        for (int s = 0; s < S; ++s) mbar_init(&bar[s], 1);
        fence_mbar_init();
    }
    griddep_wait_prior(p.wait_prior);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int s = 0; s < S; ++s) issue(s);
    }
    __syncthreads();
    griddep_launch_dependents();

    bool failed = false;
    int s = 0, prev = -1;
    uint32_t parity = 0;
    for (;;) {
        if (!__syncthreads_and(mbar_wait_bounded(&bar[s], parity, p.spin_limit, p.err_word))) {
            failed = true;
            break;
        }
        const int2 rc = stage_rc[s];
        if (rc.x < 0) break;
        if (threadIdx.x == 0 && prev >= 0) issue(prev);
        // every output of the tile inside the loop's rows and the interior columns
        const bool full_tile = rc.x + TM <= r_ub && rc.y >= 3 && rc.y + TN <= cols - 3;
        // strips of RS output rows, first row q0 within the tile
        for (int q0 = ty * RS; q0 < TM; q0 += nty * RS) {
            // input box row q0 + rho holds grid row r0 + q0 + rho - 3; the
            // 12 floats at box columns 4 tx .. 4 tx + 11 cover grid columns
            // c - 4 .. c + 7 of the outputs c .. c + 3 (c = c0 + 4 tx)
            const float* in = ring + s * stage + (size_t)q0 * BW + 4 * tx;
            float acc[RS][4];
#pragma unroll
            for (int q = 0; q < RS; ++q)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[q][j] = 0.0f;
#pragma unroll
            for (int rho = 0; rho < RS + 6; ++rho) {
                float x[12];
                const float4 a = *reinterpret_cast<const float4*>(in + rho * BW);
                const float4 b = *reinterpret_cast<const float4*>(in + rho * BW + 4);
                const float4 c = *reinterpret_cast<const float4*>(in + rho * BW + 8);
                x[0] = a.x, x[1] = a.y, x[2] = a.z, x[3] = a.w;
                x[4] = b.x, x[5] = b.y, x[6] = b.z, x[7] = b.w;
                x[8] = c.x, x[9] = c.y, x[10] = c.z, x[11] = c.w;
                if (!PAIR) {
                    // input row rho is filter row i = rho - q of output row q
#pragma unroll
                    for (int q = 0; q < RS; ++q) {
                        const int i = rho - q;
                        if (i < 0 || i > 6) continue;
#pragma unroll
                        for (int jj = 0; jj < 7; ++jj)
#pragma unroll
                            for (int j = 0; j < 4; ++j)
                                acc[q][j] = __fmaf_rn(p.w[i * 7 + jj], x[1 + j + jj], acc[q][j]);
                    }
                } else {
                    // output rows 2pp and 2pp + 1 take input row rho as filter
                    // rows i = rho - 2pp and i - 1: one paired FMA for both
                    // while both are in the window, the lone row at its ends
#pragma unroll
                    for (int pp = 0; pp < RS / 2; ++pp) {
                        const int i = rho - 2 * pp;
                        if (i < 0 || i > 7) continue;
#pragma unroll
                        for (int jj = 0; jj < 7; ++jj)
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                float& lo = acc[2 * pp][j];
                                float& hi = acc[2 * pp + 1][j];
                                if (i == 0) lo = __fmaf_rn(p.w[jj], x[1 + j + jj], lo);
                                else if (i == 7) hi = __fmaf_rn(p.w[42 + jj], x[1 + j + jj], hi);
                                else fma2_bcast(lo, hi, p.w2[(i - 1) * 7 + jj], x[1 + j + jj]);
                            }
                    }
                }
            }
            const int64_t c = (int64_t)rc.y + 4 * tx;
            float* out = p.xout + ((int64_t)rc.x + q0) * cols + c;
            if (full_tile) {
#pragma unroll
                for (int q = 0; q < RS; ++q)
                    __stcs(reinterpret_cast<float4*>(out + q * cols),
                           make_float4(acc[q][0], acc[q][1], acc[q][2], acc[q][3]));
            } else {
                const bool full = c >= 3 && c + 3 <= cols - 4;
#pragma unroll
                for (int q = 0; q < RS; ++q) {
                    const int64_t r = (int64_t)rc.x + q0 + q;
                    if (q0 + q >= TM || r >= r_ub) break;
                    float* o = out + q * cols;
                    if (full) {
                        __stcs(reinterpret_cast<float4*>(o), make_float4(acc[q][0], acc[q][1], acc[q][2], acc[q][3]));
                    } else {
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            if (c + j >= 3 && c + j <= cols - 4) o[j] = acc[q][j];
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
    tile_iter_reset(p, &last_team);
    if (failed && threadIdx.x == 0) {
        for (int k = 0; k < S; ++k) {
            if (stage_rc[k].x < 0) continue;
            if (!mbar_wait_bounded(&bar[k], 0, p.spin_limit, nullptr))
                mbar_wait_bounded(&bar[k], 1, p.spin_limit, nullptr);
        }
    }
}

using F7Kernel = void (*)(const Filter7Params, const CUtensorMap);

template <int S, int RS, bool PAIR>
F7Kernel filter7_pick_shape(int tile_m, int tile_n) {
    if (tile_m == 32 && tile_n == 128) return filter7_kernel<S, 32, 128, RS, PAIR>;
    if (tile_m == 64 && tile_n == 128) return filter7_kernel<S, 64, 128, RS, PAIR>;
    return filter7_kernel<S, 0, 0, RS, PAIR>;
}

template <int S, bool PAIR>
F7Kernel filter7_pick_rs(int tile_m, int tile_n, int rs) {
    return rs == 8 ? filter7_pick_shape<S, 8, PAIR>(tile_m, tile_n) : filter7_pick_shape<S, 4, PAIR>(tile_m, tile_n);
}

// 32 x 128 and 64 x 128 tiles have their own instantiations; other shapes
// (hints) run the runtime-shape kernel.  rs: output rows per thread strip
// (4 or 8); stages: 2 or 3; pair: paired-row FMAs.
F7Kernel filter7_pick(int stages, int tile_m, int tile_n, int rs, int pair) {
    if (pair) return stages >= 3 ? filter7_pick_rs<3, true>(tile_m, tile_n, rs) : filter7_pick_rs<2, true>(tile_m, tile_n, rs);
    return stages >= 3 ? filter7_pick_rs<3, false>(tile_m, tile_n, rs) : filter7_pick_rs<2, false>(tile_m, tile_n, rs);
}

template <class K>
bool configure_once(K k, size_t smem) {
    static K done[64] = {};
    for (auto& d : done) {
        if (d == k) return true;
        if (!d) {
            if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
                return false;
            d = k;
            return true;
        }
    }
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess;
}

// dynamic shared memory the kernels may ask for (227 KB per block minus room
// for their static shared memory)
constexpr size_t kMaxDynSmem = kStencilSmemBudget;

}  // namespace

size_t jacobi_tb_plane_floats(int tile_m, int tile_n, int sweeps, int halo_c) {
    return tb_plane_floats(tile_m, tile_n, sweeps, halo_c);
}

size_t jacobi_tb_smem_bytes(int tile_m, int tile_n, int sweeps, int halo_c) {
    return 3 * tb_plane_floats(tile_m, tile_n, sweeps, halo_c) * sizeof(float) + 1024;
}

cudaError_t launch_jacobi_tb(int teams, int units, const JacobiTBParams& p, const void* tmap, cudaStream_t s) {
    TBKernel k = tb_pick(p.sweeps, p.rvar ? p.rop : 0);
    if (!k) return cudaErrorInvalidValue;
    if (!configure_once(k, kMaxDynSmem)) return cudaGetLastError();
    CUtensorMap m;
    memcpy(&m, tmap, sizeof(m));
    return launch_pdl(k, teams, units, jacobi_tb_smem_bytes(p.tile_m, p.tile_n, p.sweeps, p.halo_c), s, p, m);
}

size_t filter7_smem_bytes(int tile_m, int tile_n, int stages) {
    return (size_t)stages * f7_stage_floats(tile_m, tile_n) * sizeof(float) + 1024;
}

int filter7_max_teams_per_sm(int tile_m, int tile_n, int stages, int rs, int pair) {
    F7Kernel k = filter7_pick(stages, tile_m, tile_n, rs, pair);
    if (!configure_once(k, kMaxDynSmem)) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, kFilter7Units, filter7_smem_bytes(tile_m, tile_n, stages)) !=
        cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

cudaError_t launch_filter7(int teams, const Filter7Params& p, const void* tmap, cudaStream_t s) {
    F7Kernel k = filter7_pick(p.stages, p.tile_m, p.tile_n, p.rs, p.pair);
    if (!configure_once(k, kMaxDynSmem)) return cudaGetLastError();
    CUtensorMap m;
    memcpy(&m, tmap, sizeof(m));
    return launch_pdl(k, teams, kFilter7Units, filter7_smem_bytes(p.tile_m, p.tile_n, p.stages), s, p, m);
}

}  // namespace upir
