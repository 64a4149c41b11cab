// Internal types shared by the runtime (host) and the kernels (device).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "upir.h"

namespace upir {

constexpr int kGroup = 1024;             // blocks per first-level group of a static reduction
constexpr int kFinSeg = 2048;            // partial slots folded by one finalize block
constexpr int UPIR_ERR_WAIT_TIMEOUT = 1;  // device error word: a bounded wait ran out
constexpr int kNumSMs = 148;
constexpr double kL2Bytes = 126.0 * 1024 * 1024;  // last-level cache of the GPU

// One reduction partial: FP32 (sum, compensation) and an int64 value.
struct __align__(16) Partial {
    float s, c;
    long long i;
};

struct RedVars {
    float* fvar;       // FP32 reduction variable (nullptr: none)
    long long* ivar;   // int64 reduction variable (nullptr: none)
    int fop, iop;      // upir_red_op of each
    int fterm, iterm;  // upir_term of each
};

// Static-schedule constants, computed on the host for the launched worker
// count W: blocked schedules give worker w [w*base + min(w, extra), +base +
// (w < extra)); chunked ones hand out chunks w, w + W, ... < nchunks.
struct SchedConst {
    int64_t base, extra, nchunks;
};

inline SchedConst make_sched_const(int64_t trip, int64_t chunk, int64_t workers) {
    SchedConst s;
    s.base = workers > 0 ? trip / workers : 0;
    s.extra = workers > 0 ? trip % workers : 0;
    s.nchunks = chunk > 0 ? (trip + chunk - 1) / chunk : 0;
    return s;
}

// Per-loop device scratch for reductions and dynamic schedules.
struct Scratch {
    unsigned long long* chunk_counter;
    unsigned* ticket;
    unsigned* group_tickets;
    Partial* group_partials;
    Partial* partials;
    // guided schedules and taskloops: the starts of the nchunks_tab chunks
    // (and the end of the last), else nullptr for chunks of a fixed size
    const int64_t* chunk_starts;
    int64_t nchunks_tab;
};

// Element-granular loop bodies (AXPY, IMOD, COVERAGE, per-point JACOBI5).
struct ElemParams {
    int64_t lb, step, trip, chunk, nchunks;
    const float* x;
    float* y;
    float a;
    long long* owner;
    unsigned long long* count;
    const float* uin;
    float* uout;
    int64_t rows, cols;
    long long imod_mul, imod_mod, imod_inc;  // imod_inc = (mul * step) mod m, in [0, m)
    unsigned long long imod_minv;            // floor(2^64 / m) for Barrett reduction (m >= 2)
    int imod32;                              // m < 2^28: eight terms sum in 32 bits
    SchedConst sk;
    int wait_prior;                          // 1: implicit barrier; 2: previous loop nowait (griddep_wait_prior)
    int fuse_fin;                            // the last team finishes the reductions (few partials)
    RedVars rv;
    Scratch sc;
};

// Tiled 5-point Jacobi sweep over interior rows [r_lb, r_ub).
struct JacobiParams {
    const float* uin;
    float* uout;
    int64_t rows, cols;
    int64_t r_lb, r_ub;
    int tile_m, tile_n;
    int64_t tiles_r, tiles_c, ntiles;
    int64_t chunk;
    int sched;
    float* rvar;  // reduction variable (max/min of |u_out - u_in|), or nullptr
    int rop;
    int stages;   // shared-memory pipeline depth
    int rows_tma; // one copy per halo row from a 1D view of the grid (width not a multiple of 4)
    int reverse;  // blocked static schedule: the team walks its run of tiles descending
    int keep_l2;  // 2D boxes: inputs read evict-first, outputs stored with normal priority
    long long spin_limit;
    int* err_word;
    SchedConst sk;
    int wait_prior;
    Scratch sc;
};

// Time-blocked Jacobi (JACOBI5_TB): `sweeps` sweeps per tile visit, tiles of
// tile_m x tile_n points with a halo of `sweeps` rows and halo_c columns.
struct JacobiTBParams {
    const float* uin;
    float* uout;
    int64_t rows, cols;
    int64_t r_lb, r_ub;
    int tile_m, tile_n, sweeps, halo_c;
    int64_t tiles_r, tiles_c, ntiles;
    int64_t chunk;
    int sched;
    float* rvar;  // first of `sweeps` reduction variables, or nullptr
    int rop;
    long long spin_limit;
    int* err_word;
    SchedConst sk;
    int wait_prior;
    Scratch sc;
};

// The 7 x 7 filter (FILTER7): tiles of tile_m x tile_n outputs.
struct Filter7Params {
    const float* xin;
    float* xout;
    int64_t rows, cols;
    int64_t r_lb, r_ub;
    int tile_m, tile_n;
    int stages;  // TMA ring depth (2 or 3)
    int rs;      // output rows per thread strip (4 or 8)
    int pair;    // 1: two output rows per paired FMA (fma.rn.f32x2)
    int64_t tiles_r, tiles_c, ntiles;
    int64_t chunk;
    int sched;
    long long spin_limit;
    int* err_word;
    SchedConst sk;
    int wait_prior;
    Scratch sc;
    float w[49];  // weights, row-major over the window
    // weight pairs of the paired-row form: element (i - 1) * 7 + j holds
    // w[i][j] in its low half and w[i - 1][j] in its high half, i = 1..6
    unsigned long long w2[42];
};

struct MatvecParams {
    const float* A;
    const float* x;
    float* y;
    int64_t rows, cols;
    int64_t lb, step, trip, chunk;
    int sched;
    SchedConst sk;
    int wait_prior;
    Scratch sc;
};

struct GemmParams {
    const float* A;
    const float* B;
    float* C;
    int64_t M, N, K;
    int64_t row_lb, row_ub;
    int64_t chunk;
    int sched;
    SchedConst sk;
    Scratch sc;
    // tail split (static default plan only, kparts > 1): teams [0, whole) take
    // whole tiles; the tiles from `whole` on are each taken by kparts teams,
    // one share of the k tiles each, whose sums meet in `work` (kparts 128 x
    // 128 partial tiles per split tile) and are added by the last to finish
    int64_t whole;
    int kparts;
    float* work;
    unsigned* tile_tickets;
    long long spin_limit;  // TMA-fed kernel: bound of each wait for a k tile
    int* err_word;
};

struct SplitParams {
    const float* src;
    uint16_t* hi;
    uint16_t* lo;
    int64_t rows, cols;
    int64_t lb, ub;  // row range
    int transpose;
};

// Persistent execution of a batch of single-loop regions: one entry per
// region, one (region, tile) work item per tile.
enum BatchOp { BOP_AXPY = 0, BOP_JACOBI = 1, BOP_MATVEC = 2 };

struct BatchRegion {
    int op;             // BatchOp
    int fop;            // reduction operator of the FP32 clause, 0 if none
    int fterm;          // AXPY: TERM_Y or TERM_XY
    int tile_rows;      // MATVEC: rows per work item
    const float* in0;   // AXPY x | JACOBI u_in | MATVEC A
    const float* in1;   // MATVEC x
    float* out;         // AXPY y | JACOBI u_out | MATVEC y
    float a;
    int pad2;
    int64_t lb, trip;   // first index and count (AXPY) / first row and rows (JACOBI, MATVEC)
    int64_t rows, cols; // JACOBI grid / MATVEC shape
    int64_t tiles;      // work items of this region
    int64_t tiles_c;    // JACOBI: tiles per row band
    int64_t slot0;      // AXPY: first partial slot
    float* fvar;        // reduction variable, or nullptr
    unsigned* ticket;   // AXPY with a reduction: tiles finished so far; JACOBI: residual key (0: none yet)
};

struct BatchParams {
    const BatchRegion* regions;
    const int2* items;             // (region, tile), largest regions first
    int64_t nitems;
    Partial* partials;
    unsigned long long* counter;   // next work item
    unsigned* exit_ticket;         // teams finished
    int nregions;
    int axpy_tile;                 // AXPY iterations per tile (multiple of 1024)
    int jac_rows;                  // JACOBI rows per tile (tiles are 128 columns wide)
    int mv_rows;                   // MATVEC rows per tile
};

constexpr int kBatchUnits = 256;
constexpr int kBatchJacCols = 128;
constexpr int kBatchMaxJacRows = 32;
constexpr int kBatchNarrowCols = 64;  // MATVEC rows this narrow take one unit each

// Host-side launchers (one per kernel family).
// fop / iop: the loop's FP32 / int64 reduction operator, 0 when it has none.
cudaError_t launch_elem(int body, bool dynamic, int fop, int iop, int teams, int units,
                        const ElemParams& p, cudaStream_t s);
cudaError_t launch_elem_main(int body, bool dynamic, int fop, int iop, int teams, int units,
                             const ElemParams& p, cudaStream_t s);
cudaError_t launch_finalize(const RedVars& rv, const Scratch& sc, int64_t nslots, bool reset_counter,
                            cudaStream_t s);
int64_t finalize_groups(int64_t nslots);
cudaError_t launch_jacobi_tma(int teams, int units, const JacobiParams& p, const void* tmap,
                              cudaStream_t s);
size_t jacobi_tma_smem_bytes(int tile_m, int tile_n, int stages, bool rows);
// shared row pitch (floats) of the row-copy Jacobi variant: the halo box width
// tile_n + 8 rounded up to 128 bytes
__host__ __device__ constexpr int jacobi_rt_pitch(int tile_n) { return (tile_n + 8 + 31) / 32 * 32; }
constexpr int kJacobiTBUnits = 1024, kFilter7Units = 256, kFilter7Stages = 2;
constexpr size_t kStencilSmemBudget = 222 * 1024;  // dynamic shared memory of the stencil kernels
size_t jacobi_tb_plane_floats(int tile_m, int tile_n, int sweeps, int halo_c);
size_t jacobi_tb_smem_bytes(int tile_m, int tile_n, int sweeps, int halo_c);
cudaError_t launch_jacobi_tb(int teams, int units, const JacobiTBParams& p, const void* tmap, cudaStream_t s);
size_t filter7_smem_bytes(int tile_m, int tile_n, int stages);
int filter7_max_teams_per_sm(int tile_m, int tile_n, int stages, int rs, int pair);
cudaError_t launch_filter7(int teams, const Filter7Params& p, const void* tmap, cudaStream_t s);
int jacobi_tma_max_teams_per_sm(int units, int tile_m, int tile_n, int stages, bool rows, bool keep);
cudaError_t launch_matvec(int teams, int units, const MatvecParams& p, cudaStream_t s);
int matvec_max_teams_per_sm(int units);
cudaError_t launch_gemm_f32(int teams, int units, const GemmParams& p, cudaStream_t s);
// tm: the A (K x M, 16 x 128 boxes) and B (N x K, 128 x 16 boxes) tensor maps
cudaError_t launch_gemm_f32_tma(int teams, const GemmParams& p, const CUtensorMap* tm, cudaStream_t s);
cudaError_t launch_split_bf16(int teams, int units, const SplitParams& p, cudaStream_t s);
cudaError_t launch_bounded_wait_selftest(long long spin_limit, int* err_word, cudaStream_t s);
cudaError_t launch_batch_persistent(int teams, const BatchParams& p, cudaStream_t s);
int batch_persistent_teams_per_sm();

}  // namespace upir
