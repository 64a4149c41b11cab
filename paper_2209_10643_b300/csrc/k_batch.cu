// Many independent, uneven regions in one persistent launch.  The regions'
// loops are cut into tiles; the (region, tile) work items, largest regions
// first, are claimed one at a time from an atomic counter by persistent teams
// and dispatched on the region's body.  The tile loop of each region is thus
// workshared dynamically over all teams of the GPU (§3.2 schedule(dynamic)).
// An AXPY region's reduction is finalized by its last tile, the tile partials
// folded in tile order, so the result does not depend on which team ran which
// tile; a Jacobi region's max/min residual (exact in any order) is gathered
// with atomics and folded into its variable by the last team to finish.
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

// Rows whose width is a multiple of 4 and 16-byte aligned grids take the
// 128-bit loads and stores.
__device__ __forceinline__ bool jacobi_vec(const BatchRegion& R) {
    return (R.cols & 3) == 0 && ((reinterpret_cast<uintptr_t>(R.in0) | reinterpret_cast<uintptr_t>(R.out)) & 15) == 0;
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

// One Jacobi tile, straight from global memory: warp w of the team takes a
// band of the tile's rows and each lane 4 of its 128 columns; the lane issues
// the loads of all rows it needs (its output rows and the ones above and
// below) at once, so a team keeps up to six row segments per warp in flight
// with no shared-memory staging (which leaves the SM's shared memory to the
// L1 cache, where the rows that neighbouring warps share meet).  West and east
// neighbours come from the adjacent lanes by shuffles, the tile's edge columns
// by one extra load in lanes 0 and 31.  VEC: 128-bit loads and stores; else
// (rows off the 16-byte grid) four 32-bit ones.
template <bool VEC>
__device__ __forceinline__ void jacobi_tile_direct(const BatchParams& P, const BatchRegion& R, int64_t t) {
    constexpr int kMaxR = kBatchMaxJacRows / (kBatchUnits / 32) + 2;  // rows a warp loads at most
    const int64_t cols = R.cols, tiles_c = R.tiles_c, lb = R.lb, trip = R.trip;
    const float* const inb = R.in0;
    float* const outb = R.out;
    unsigned* const rslot = R.ticket;
    const int fop = R.fop;
    const int64_t band = t / tiles_c, tc = t - band * tiles_c;
    const int64_t r0 = lb + band * P.jac_rows;
    const int nr = (int)min((int64_t)P.jac_rows, lb + trip - r0);
    const int64_t c0 = tc * kBatchJacCols;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int rpw = (nr + nw - 1) / nw;
    const int ra = min(nr, w * rpw), rb = min(nr, ra + rpw);  // this warp's output rows [ra, rb) of the tile
    const int64_t c = c0 + 4 * lane;
    const bool cin = c < cols;                          // the lane's first column is in the grid
    const bool inside = c >= 1 && c + 3 <= cols - 2;    // all four points are updated
    float racc = fop == UPIR_RED_MIN ? __int_as_float(0x7f800000) : -__int_as_float(0x7f800000);
    if (ra < rb) {
        const int nload = rb - ra + 2;
        const float* src = inb + (r0 + ra - 1) * cols + c;
        float4 row[kMaxR];
        float wl[kMaxR - 2], er[kMaxR - 2];
#pragma unroll
        for (int k = 0; k < kMaxR; ++k) {
            if (VEC) {
                row[k] = (k < nload && cin) ? __ldg(reinterpret_cast<const float4*>(src + k * cols))
                                            : make_float4(0.f, 0.f, 0.f, 0.f);
            } else {
                // rows off the 16-byte grid: four 32-bit loads, columns past the edge read as 0
                const bool rk = k < nload;
                const float* q = src + k * cols;
                row[k] = make_float4(rk && c < cols ? __ldg(q) : 0.f, rk && c + 1 < cols ? __ldg(q + 1) : 0.f,
                                     rk && c + 2 < cols ? __ldg(q + 2) : 0.f, rk && c + 3 < cols ? __ldg(q + 3) : 0.f);
            }
        }
#pragma unroll
        for (int k = 0; k < kMaxR - 2; ++k) {
            const bool rk = k < nload - 2;
            wl[k] = (rk && lane == 0 && c0 >= 1) ? __ldg(src + (k + 1) * cols - 1) : 0.0f;
            er[k] = (rk && lane == 31 && c0 + kBatchJacCols < cols) ? __ldg(src + (k + 1) * cols + 4) : 0.0f;
        }
        float* out = outb + (r0 + ra) * cols + c;
#pragma unroll
        for (int k = 0; k < kMaxR - 2; ++k) {
            if (k >= nload - 2) break;
            const float4 N = row[k], C = row[k + 1], S = row[k + 2];
            float Wl = __shfl_up_sync(0xffffffffu, C.w, 1), Er = __shfl_down_sync(0xffffffffu, C.x, 1);
            if (lane == 0) Wl = wl[k];
            if (lane == 31) Er = er[k];
            float4 v;
            v.x = __fmul_rn(0.25f, __fadd_rn(__fadd_rn(N.x, S.x), __fadd_rn(Wl, C.y)));
            v.y = __fmul_rn(0.25f, __fadd_rn(__fadd_rn(N.y, S.y), __fadd_rn(C.x, C.z)));
            v.z = __fmul_rn(0.25f, __fadd_rn(__fadd_rn(N.z, S.z), __fadd_rn(C.y, C.w)));
            v.w = __fmul_rn(0.25f, __fadd_rn(__fadd_rn(N.w, S.w), __fadd_rn(C.z, Er)));
            float* o = out + k * cols;
            if (inside) {
                if (VEC) {
                    __stcs(reinterpret_cast<float4*>(o), v);
                } else {
                    __stcs(o, v.x);
                    __stcs(o + 1, v.y);
                    __stcs(o + 2, v.z);
                    __stcs(o + 3, v.w);
                }
                if (fop) {
                    const float a = fold(fabsf(__fsub_rn(v.x, C.x)), fabsf(__fsub_rn(v.y, C.y)), fop);
                    const float b = fold(fabsf(__fsub_rn(v.z, C.z)), fabsf(__fsub_rn(v.w, C.w)), fop);
                    racc = fold(racc, fold(a, b, fop), fop);
                }
            } else if (cin) {
                const float vs[4] = {v.x, v.y, v.z, v.w}, cs[4] = {C.x, C.y, C.z, C.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (c + j >= 1 && c + j <= cols - 2) {
                        o[j] = vs[j];
                        if (fop) racc = fold(racc, fabsf(__fsub_rn(vs[j], cs[j])), fop);
                    }
                }
            }
        }
    }
    if (fop) {
        const float b = block_fold(racc, fop);
        if (threadIdx.x == 0 && !isnan(b)) atomicMax(rslot, resid_key(b, fop));
    }
}

__device__ __forceinline__ void matvec_tile(const BatchParams& P, const BatchRegion& R, int64_t t) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    // the region's fields, read once (the stores to y could alias them)
    const float* const A = R.in0;
    const float* const x = R.in1;
    float* const y = R.out;
    const int64_t cols = R.cols;
    const int64_t r0 = R.lb + t * R.tile_rows;
    const int64_t r1 = min(r0 + (int64_t)R.tile_rows, R.lb + R.trip);
    // the tile's rows of A are requested into L2 at once, so that a warp's
    // dot product, a chain of a few load rounds per row, waits on L2 rather
    // than on DRAM
    if (threadIdx.x == 0 && r1 > r0) prefetch_l2_range(A + r0 * cols, (size_t)(r1 - r0) * cols * sizeof(float));
    if (cols <= kBatchNarrowCols) {
        // narrow rows: one per unit, its dot product a chain of fused
        // multiply-adds in column order (a warp per row would leave most of
        // its lanes idle and pay a butterfly per row)
        const int64_t r = r0 + threadIdx.x;
        if (r < r1) {
            const float* a = A + r * cols;
            float acc = 0.0f;
#pragma unroll 4
            for (int64_t j = 0; j < cols; ++j) acc = __fmaf_rn(__ldg(a + j), __ldg(x + j), acc);
            y[r] = acc;
        }
        return;
    }
    for (int64_t r = r0 + warp; r < r1; r += nw) {
        const float v = row_dot(A + r * cols, x, cols, lane);
        if (lane == 0) y[r] = v;
    }
}

__global__ void __launch_bounds__(kBatchUnits, 4) batch_persistent_kernel(const BatchParams P) {
    __shared__ int64_t cur_item, next_item, after_next;
    __shared__ int last_team;
    griddep_wait();
    if (threadIdx.x == 0) {
        cur_item = (int64_t)atomicAdd(P.counter, 1ull);
        next_item = (int64_t)atomicAdd(P.counter, 1ull);
    }
    __syncthreads();
    for (;;) {
        const int64_t k = cur_item;
        if (k >= P.nitems) break;
        // claim the item after next now, so the atomic's latency overlaps this one
        if (threadIdx.x == 0) after_next = (int64_t)atomicAdd(P.counter, 1ull);
        const int2 it = P.items[k];
        const BatchRegion& R = P.regions[it.x];
        switch (R.op) {
            case BOP_AXPY: axpy_tile(P, R, it.y); break;
            case BOP_JACOBI:
                if (jacobi_vec(R)) jacobi_tile_direct<true>(P, R, it.y);
                else jacobi_tile_direct<false>(P, R, it.y);
                break;
            default: matvec_tile(P, R, it.y); break;
        }
        __syncthreads();  // every thread has read the item slots
        if (threadIdx.x == 0) {
            cur_item = next_item;
            next_item = after_next;
        }
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
