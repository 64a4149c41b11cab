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
    // the region's fields, read once (the stores to y could alias them)
    const float a = R.a;
    const int fop = R.fop;
    const int64_t e0 = R.lb + t * P.axpy_tile;
    const int64_t e1 = min(e0 + (int64_t)P.axpy_tile, R.lb + R.trip);
    FAcc f = facc_identity(fop);
    const bool red = fop != 0;
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
    const uintptr_t al = reinterpret_cast<uintptr_t>(x + e0) | reinterpret_cast<uintptr_t>(y + e0);
    if ((al & 31) == 0) {
        // groups of eight iterations on 256-bit accesses, two groups per
        // unit in flight; the reduction terms go to paired accumulators
        FAcc2 acc2 = facc2_zero();
        const int64_t n8 = (e1 - e0) / 8;
        const int B = blockDim.x;
        auto group = [&](const float* xv, float* yv, int64_t g) {
#pragma unroll
            for (int j = 0; j < 8; ++j) yv[j] = __fmaf_rn(a, xv[j], yv[j]);
            st_v8_cs_f(y + e0 + 8 * g, yv);
            if (red) {
#pragma unroll
                for (int j = 0; j < 8; j += 2) {
                    if (xy) facc2_add_prod(acc2, f2(xv[j], xv[j + 1]), f2(yv[j], yv[j + 1]));
                    else facc2_add(acc2, f2(yv[j], yv[j + 1]));
                }
            }
        };
        int64_t g = threadIdx.x;
        for (; g + B < n8; g += 2 * B) {
            float x0[8], y0[8], x1[8], y1[8];
            ld_v8_cs(x + e0 + 8 * g, x0);
            ld_v8_cs(y + e0 + 8 * g, y0);
            ld_v8_cs(x + e0 + 8 * (g + B), x1);
            ld_v8_cs(y + e0 + 8 * (g + B), y1);
            group(x0, y0, g);
            group(x1, y1, g + B);
        }
        if (g < n8) {
            float x0[8], y0[8];
            ld_v8_cs(x + e0 + 8 * g, x0);
            ld_v8_cs(y + e0 + 8 * g, y0);
            group(x0, y0, g);
        }
        for (int64_t e = e0 + 8 * n8 + threadIdx.x; e < e1; e += B) {
            const float yn = __fmaf_rn(a, x[e], y[e]);
            y[e] = yn;
            term(x[e], yn);
        }
        if (red) f = facc_merge2(f, acc2);
    } else if ((al & 15) == 0) {
        const int64_t n4 = (e1 - e0) / 4;
#pragma unroll 4
        for (int64_t g = threadIdx.x; g < n4; g += blockDim.x) {
            const float4 xv = __ldcs(reinterpret_cast<const float4*>(x + e0) + g);
            const float4 yv = __ldcs(reinterpret_cast<const float4*>(y + e0) + g);
            float4 yn;
            yn.x = __fmaf_rn(a, xv.x, yv.x);
            yn.y = __fmaf_rn(a, xv.y, yv.y);
            yn.z = __fmaf_rn(a, xv.z, yv.z);
            yn.w = __fmaf_rn(a, xv.w, yv.w);
            __stcs(reinterpret_cast<float4*>(y + e0) + g, yn);
            term(xv.x, yn.x);
            term(xv.y, yn.y);
            term(xv.z, yn.z);
            term(xv.w, yn.w);
        }
        for (int64_t e = e0 + 4 * n4 + threadIdx.x; e < e1; e += blockDim.x) {
            const float yn = __fmaf_rn(a, x[e], y[e]);
            y[e] = yn;
            term(x[e], yn);
        }
    } else {
        for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
            const float yn = __fmaf_rn(a, x[e], y[e]);
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

// shared row: 4 + 128 + 4 columns, and up to 3 more for a row copied from
// the 16-byte boundary before its first column
constexpr int kHaloW = kBatchJacCols + 12;
constexpr int kHaloFloats = (kBatchMaxJacRows + 2) * kHaloW;

// Rows whose width is a multiple of 4 and 16-byte aligned buffers take the
// 128-bit paths, including the asynchronous halo copy.
__device__ __forceinline__ bool jacobi_vec(const BatchRegion& R) {
    return (R.cols & 3) == 0 && ((reinterpret_cast<uintptr_t>(R.in0) | reinterpret_cast<uintptr_t>(R.out)) & 15) == 0;
}

// Other widths with a 16-byte aligned input grid: each halo row is copied in
// 16-byte pieces from the boundary at or before its first column, so the row
// sits in shared memory shifted by ((row * cols + c0) mod 4) columns.
__device__ __forceinline__ bool jacobi_shifted(const BatchRegion& R) {
    return !jacobi_vec(R) && (reinterpret_cast<uintptr_t>(R.in0) & 15) == 0;
}

// Issue the asynchronous copy of tile t's halo into `halo` and commit it as
// one group: 16-byte copies for 128-bit-capable regions and for shifted rows,
// 4-byte copies for the others; columns outside the grid are zero-filled.
// Unshifted, shared column j holds grid column c0 - 4 + j, so the tile's
// first column sits on a 16-byte boundary.
__device__ __forceinline__ void jacobi_halo_async(const BatchParams& P, const BatchRegion& R, int64_t t,
                                                  float* halo) {
    const int64_t band = t / R.tiles_c, tc = t - band * R.tiles_c;
    const int64_t r0 = R.lb + band * P.jac_rows;
    const int nr = (int)min((int64_t)P.jac_rows, R.lb + R.trip - r0);
    const int64_t c0 = tc * kBatchJacCols, cols = R.cols;
    // a warp per halo row; a lane's columns advance by 32 copies at a time
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = kBatchUnits / 32;
    const int64_t cfirst = c0 - 4;  // grid column of shared column 0
    if (jacobi_shifted(R)) {
        const int64_t total = R.rows * cols;  // elements of the grid
        for (int i = warp; i < nr + 2; i += nw) {
            const int64_t g = (r0 - 1 + i) * cols + cfirst;  // grid column c0 - 4 of halo row i
            const int64_t base = g & ~(int64_t)3;
            const uint32_t srow = smem_u32(halo + i * kHaloW);
            for (int q = lane; q < kHaloW / 4; q += 32) {
                const int64_t idx = base + 4 * q;
                const int64_t nv = idx < 0 ? 0 : min(max(total - idx, (int64_t)0), (int64_t)4);
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;"
                             ::"r"(srow + 16u * q), "l"(nv ? R.in0 + idx : R.in0), "r"((int)(4 * nv)) : "memory");
            }
        }
    } else if (jacobi_vec(R)) {
        for (int i = warp; i < nr + 2; i += nw) {
            const float* grow = R.in0 + (r0 - 1 + i) * cols;
            const uint32_t srow = smem_u32(halo + i * kHaloW);
            for (int q = lane; q < kHaloW / 4; q += 32) {
                const int64_t cc = cfirst + 4 * q;
                const bool in = cc >= 0 && cc + 3 < cols;
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;"
                             ::"r"(srow + 16u * q), "l"(in ? grow + cc : R.in0), "r"(in ? 16 : 0) : "memory");
            }
        }
    } else {
        for (int i = warp; i < nr + 2; i += nw) {
            const float* grow = R.in0 + (r0 - 1 + i) * cols;
            const uint32_t srow = smem_u32(halo + i * kHaloW);
#pragma unroll
            for (int j = lane; j < kHaloW; j += 32) {
                const int64_t cc = cfirst + j;
                const bool in = cc >= 0 && cc < cols;
                asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;"
                             ::"r"(srow + 4u * j), "l"(in ? grow + cc : R.in0), "r"(in ? 4 : 0) : "memory");
            }
        }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// One Jacobi tile.  `staged`: its halo copy was issued into `halo` while the
// previous item ran.  `next` (may be null): a following Jacobi item whose
// halo copy is issued into `halo_next` before this tile computes, so that its
// DRAM latency overlaps this tile's work.
// The rows i = i0, i0 + step, ... < nr of one lane's four columns, from the
// staged halo to the output (5-point stencil, JACOBI5's arithmetic), folding
// |new - old| of the updated points into the residual (FOP 0: none).
template <int FOP>
__device__ __forceinline__ float jacobi_rows(const float* cen, float* out, int i0, int nr, int step, int64_t ostep,
                                             bool inside, bool full, int64_t c, int64_t cols) {
    constexpr int HW = kHaloW;
    float racc = FOP == UPIR_RED_MIN ? __int_as_float(0x7f800000) : -__int_as_float(0x7f800000);
    for (int i = i0; i < nr; i += step, cen += step * HW, out += ostep) {
        const float4 C = *reinterpret_cast<const float4*>(cen);
        const float4 N = *reinterpret_cast<const float4*>(cen - HW);
        const float4 S = *reinterpret_cast<const float4*>(cen + HW);
        const float Wl = cen[-1], Er = cen[4];
        float4 v;
        v.x = __fmul_rn(0.25f, __fadd_rn(__fadd_rn(N.x, S.x), __fadd_rn(Wl, C.y)));
        v.y = __fmul_rn(0.25f, __fadd_rn(__fadd_rn(N.y, S.y), __fadd_rn(C.x, C.z)));
        v.z = __fmul_rn(0.25f, __fadd_rn(__fadd_rn(N.z, S.z), __fadd_rn(C.y, C.w)));
        v.w = __fmul_rn(0.25f, __fadd_rn(__fadd_rn(N.w, S.w), __fadd_rn(C.z, Er)));
        if (inside) {
            if (full) {
                __stcs(reinterpret_cast<float4*>(out), v);
            } else {
                __stcs(out, v.x);
                __stcs(out + 1, v.y);
                __stcs(out + 2, v.z);
                __stcs(out + 3, v.w);
            }
            if (FOP) {
                const float a = fold(fabsf(__fsub_rn(v.x, C.x)), fabsf(__fsub_rn(v.y, C.y)), FOP);
                const float b = fold(fabsf(__fsub_rn(v.z, C.z)), fabsf(__fsub_rn(v.w, C.w)), FOP);
                racc = fold(racc, fold(a, b, FOP), FOP);
            }
        } else {
            const float vs[4] = {v.x, v.y, v.z, v.w}, cs[4] = {C.x, C.y, C.z, C.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (c + j >= 1 && c + j <= cols - 2) {
                    out[j] = vs[j];
                    if (FOP) racc = fold(racc, fabsf(__fsub_rn(vs[j], cs[j])), FOP);
                }
            }
        }
    }
    return racc;
}

// A Jacobi region's max (min) residual over its tiles, kept as an unsigned
// key in the region's slot with a fire-and-forget atomic max: the key of a
// non-NaN float orders like the float (sign bit flipped for non-negative
// values, all bits flipped for negative ones), complemented for min; 0 means
// no tile has reported.  The last team to finish folds each slot into the
// reduction variable (maxNum / minNum, NaN residuals ignored) and clears it.
__device__ __forceinline__ unsigned resid_key(float v, int op) {
    const unsigned b = __float_as_uint(v);
    const unsigned k = (b & 0x80000000u) ? ~b : (b | 0x80000000u);
    return op == UPIR_RED_MIN ? ~k : k;
}

__device__ __forceinline__ float resid_value(unsigned key, int op) {
    const unsigned k = op == UPIR_RED_MIN ? ~key : key;
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// The shifted-row form: lane tx takes columns c0 + tx + 32 j (j = 0..3), so
// 32-bit shared loads from rows of any shift and the 32-bit global stores
// stay unit-stride across the warp.
template <int FOP>
__device__ __forceinline__ float jacobi_rows_shifted(const float* halo, float* outb, int64_t r0, int nr, int ty,
                                                     int nty, int tx, int64_t c0, int64_t cols) {
    constexpr int HW = kHaloW;
    float racc = FOP == UPIR_RED_MIN ? __int_as_float(0x7f800000) : -__int_as_float(0x7f800000);
    const uint32_t cq = (uint32_t)cols & 3u;
    const uint32_t sh0 = ((uint32_t)(r0 - 1) * cq + (uint32_t)c0) & 3u;  // shift of halo row 0
    for (int i = ty; i < nr; i += nty) {
        const float* rn = halo + i * HW + ((sh0 + (uint32_t)i * cq) & 3u) + 4;
        const float* rm = halo + (i + 1) * HW + ((sh0 + (uint32_t)(i + 1) * cq) & 3u) + 4;
        const float* rs = halo + (i + 2) * HW + ((sh0 + (uint32_t)(i + 2) * cq) & 3u) + 4;
        float* orow = outb + (r0 + i) * cols + c0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int q = tx + 32 * j;
            const int64_t c = c0 + q;
            const float cv = rm[q];
            const float v = __fmul_rn(0.25f, __fadd_rn(__fadd_rn(rn[q], rs[q]), __fadd_rn(rm[q - 1], rm[q + 1])));
            if (c >= 1 && c <= cols - 2) {
                __stcs(orow + q, v);
                if (FOP) racc = fold(racc, fabsf(__fsub_rn(v, cv)), FOP);
            }
        }
    }
    return racc;
}

__device__ __forceinline__ void jacobi_tile(const BatchParams& P, const BatchRegion& R, int64_t t, float* halo,
                                            bool staged, const BatchRegion* next, int64_t tn, float* halo_next) {
    constexpr int HW = kHaloW;
    // the region's fields, read once (the output stores could alias them)
    const int64_t cols = R.cols, tiles_c = R.tiles_c, lb = R.lb, trip = R.trip;
    float* const outb = R.out;
    unsigned* const rslot = R.ticket;
    const int fop = R.fop;
    const bool vec = jacobi_vec(R);
    const int64_t band = t / tiles_c, tc = t - band * tiles_c;
    const int64_t r0 = lb + band * P.jac_rows;
    const int nr = (int)min((int64_t)P.jac_rows, lb + trip - r0);
    const int64_t c0 = tc * kBatchJacCols;
    if (!staged) jacobi_halo_async(P, R, t, halo);
    if (next) {
        jacobi_halo_async(P, *next, tn, halo_next);
        asm volatile("cp.async.wait_group 1;" ::: "memory");
    } else {
        asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    __syncthreads();
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5, nty = blockDim.x >> 5;
    const int64_t c = c0 + 4 * tx;
    const bool inside = c >= 1 && c + 3 <= cols - 2;  // all four points are updated
    const bool full = vec && inside;
    const float* cen = halo + (ty + 1) * HW + 4 + 4 * tx;
    float* out = outb + (r0 + ty) * cols + c;
    const int64_t ostep = (int64_t)nty * cols;
    if (jacobi_shifted(R)) {
        if (fop == UPIR_RED_MAX || fop == UPIR_RED_MIN) {
            const float r = fop == UPIR_RED_MAX
                                ? jacobi_rows_shifted<UPIR_RED_MAX>(halo, outb, r0, nr, ty, nty, tx, c0, cols)
                                : jacobi_rows_shifted<UPIR_RED_MIN>(halo, outb, r0, nr, ty, nty, tx, c0, cols);
            const float b = block_fold(r, fop);
            if (threadIdx.x == 0 && !isnan(b)) atomicMax(rslot, resid_key(b, fop));
        } else {
            jacobi_rows_shifted<0>(halo, outb, r0, nr, ty, nty, tx, c0, cols);
        }
    } else if (fop == UPIR_RED_MAX) {
        const float r = jacobi_rows<UPIR_RED_MAX>(cen, out, ty, nr, nty, ostep, inside, full, c, cols);
        const float b = block_fold(r, UPIR_RED_MAX);
        if (threadIdx.x == 0 && !isnan(b)) atomicMax(rslot, resid_key(b, UPIR_RED_MAX));
    } else if (fop == UPIR_RED_MIN) {
        const float r = jacobi_rows<UPIR_RED_MIN>(cen, out, ty, nr, nty, ostep, inside, full, c, cols);
        const float b = block_fold(r, UPIR_RED_MIN);
        if (threadIdx.x == 0 && !isnan(b)) atomicMax(rslot, resid_key(b, UPIR_RED_MIN));
    } else {
        jacobi_rows<0>(cen, out, ty, nr, nty, ostep, inside, full, c, cols);
    }
    __syncthreads();  // the halo buffer is reused by a later item
}

__device__ __forceinline__ void matvec_tile(const BatchParams& P, const BatchRegion& R, int64_t t) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    // the region's fields, read once (the stores to y could alias them)
    const float* const A = R.in0;
    const float* const x = R.in1;
    float* const y = R.out;
    const int64_t cols = R.cols;
    const int64_t r0 = R.lb + t * P.mv_rows;
    const int64_t r1 = min(r0 + (int64_t)P.mv_rows, R.lb + R.trip);
    for (int64_t r = r0 + warp; r < r1; r += nw) {
        const float v = row_dot(A + r * cols, x, cols, lane);
        if (lane == 0) y[r] = v;
    }
}

__global__ void __launch_bounds__(kBatchUnits, 4) batch_persistent_kernel(const BatchParams P) {
    // two halo buffers: the current Jacobi tile's and the next one's, whose
    // asynchronous copy runs while the current item is processed
    __shared__ __align__(16) float halo[2][kHaloFloats];
    __shared__ int64_t cur_item, next_item, after_next;
    __shared__ int last_team;
    griddep_wait();
    if (threadIdx.x == 0) {
        cur_item = (int64_t)atomicAdd(P.counter, 1ull);
        next_item = (int64_t)atomicAdd(P.counter, 1ull);
    }
    __syncthreads();
    int hb = 0;           // halo buffer of the current item
    bool staged = false;  // its halo copy was issued during the previous item
    for (;;) {
        const int64_t k = cur_item, kn = next_item;
        if (k >= P.nitems) break;
        // claim the item after next now, so the atomic's latency overlaps this one
        if (threadIdx.x == 0) after_next = (int64_t)atomicAdd(P.counter, 1ull);
        const int2 it = P.items[k];
        const BatchRegion& R = P.regions[it.x];
        // a following Jacobi tile gets its halo copied while this item runs
        const BatchRegion* nreg = nullptr;
        int64_t tn = 0;
        if (kn < P.nitems) {
            const int2 itn = P.items[kn];
            const BatchRegion* q = &P.regions[itn.x];
            if (q->op == BOP_JACOBI) nreg = q, tn = itn.y;
        }
        switch (R.op) {
            case BOP_AXPY:
                if (nreg) jacobi_halo_async(P, *nreg, tn, halo[hb ^ 1]);
                axpy_tile(P, R, it.y);
                break;
            case BOP_JACOBI: jacobi_tile(P, R, it.y, halo[hb], staged, nreg, tn, halo[hb ^ 1]); break;
            default:
                if (nreg) jacobi_halo_async(P, *nreg, tn, halo[hb ^ 1]);
                matvec_tile(P, R, it.y);
                break;
        }
        if (nreg) hb ^= 1;
        staged = nreg != nullptr;
        __syncthreads();  // every thread has read the item slots
        if (threadIdx.x == 0) {
            cur_item = next_item;
            next_item = after_next;
        }
        __syncthreads();
    }
    // no copy may still be landing in shared memory when the team exits
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    // the last team returns the work counter to zero for the next launch
    if (threadIdx.x == 0) {
        __threadfence();
        last_team = atomicAdd(P.exit_ticket, 1u) == gridDim.x - 1;
        if (last_team) {
            *P.exit_ticket = 0;
            *P.counter = 0;
        }
    }
    __syncthreads();
    if (last_team) {
        // fold the Jacobi regions' residual keys into their variables
        __threadfence();
        for (int i = threadIdx.x; i < P.nregions; i += blockDim.x) {
            const BatchRegion& R = P.regions[i];
            if (R.op != BOP_JACOBI || !R.fop) continue;
            const unsigned key = atomicExch(R.ticket, 0u);
            if (key) atomic_fold_minmax(R.fvar, resid_value(key, R.fop), R.fop);
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
