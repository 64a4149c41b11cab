// Internal types shared by the runtime (host) and the kernels (device).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "upir.h"

namespace upir {

constexpr int kGroup = 1024;             // blocks per first-level group of a static reduction
constexpr int UPIR_ERR_WAIT_TIMEOUT = 1;  // device error word: a bounded wait ran out
constexpr int kNumSMs = 148;

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

// Per-loop device scratch for reductions and dynamic schedules.
struct Scratch {
    unsigned long long* chunk_counter;
    unsigned* ticket;
    unsigned* group_tickets;
    Partial* group_partials;
    Partial* partials;
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
    long long spin_limit;
    int* err_word;
    Scratch sc;
};

struct MatvecParams {
    const float* A;
    const float* x;
    float* y;
    int64_t rows, cols;
    int64_t lb, step, trip, chunk;
    int sched;
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
    Scratch sc;
};

struct SplitParams {
    const float* src;
    uint16_t* hi;
    uint16_t* lo;
    int64_t rows, cols;
    int64_t lb, ub;  // row range
    int transpose;
};

// Host-side launchers (one per kernel family).
cudaError_t launch_elem(int body, bool dynamic, bool has_f, bool has_i, int teams, int units,
                        const ElemParams& p, cudaStream_t s);
cudaError_t launch_jacobi_tma(int teams, int units, const JacobiParams& p, const void* tmap,
                              cudaStream_t s);
cudaError_t launch_jacobi_direct(int teams, int units, const JacobiParams& p, cudaStream_t s);
size_t jacobi_tma_smem_bytes(int tile_m, int tile_n);
cudaError_t launch_matvec(int teams, int units, const MatvecParams& p, cudaStream_t s);
cudaError_t launch_gemm_f32(int teams, int units, const GemmParams& p, cudaStream_t s);
cudaError_t launch_split_bf16(int teams, int units, const SplitParams& p, cudaStream_t s);
cudaError_t launch_bounded_wait_selftest(long long spin_limit, int* err_word, cudaStream_t s);

}  // namespace upir
