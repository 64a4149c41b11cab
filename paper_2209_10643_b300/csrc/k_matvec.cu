// Dense matrix-vector product y = A x (the matvec workload of §6).  The
// worksharing loop runs over rows; its worker is a warp, and the inner dot
// product over the row is spread over the warp's lanes (the inner loop is the
// SIMD-parallel one).  Each lane streams 128-bit loads of A with 16 FP32
// accumulators, which are folded in a fixed order and then across the lanes
// with a butterfly: the result is deterministic and its rounding error is
// bounded by about (cols/512 + 9) unit roundoffs of sum_j |A_rj x_j|.
#include "matvec_row.cuh"

namespace upir {

namespace {

__global__ void __launch_bounds__(1024) matvec_kernel(const MatvecParams p) {
    const int lane = threadIdx.x & 31;
    const int64_t wpb = blockDim.x >> 5;
    const int64_t W = (int64_t)gridDim.x * wpb;
    const int64_t w = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5);
    griddep_wait_prior(p.wait_prior);
    griddep_launch_dependents();
    auto rows = [&](int64_t k0, int64_t k1) {
        for (int64_t k = k0; k < k1; ++k) {
            const int64_t r = p.lb + k * p.step;
            const float v = row_dot(p.A + r * p.cols, p.x, p.cols, lane);
            if (lane == 0) p.y[r] = v;
        }
    };
    if (p.sched == UPIR_SCHED_DYNAMIC) {
        for (;;) {
            unsigned long long j = 0;
            if (lane == 0) j = atomicAdd(p.sc.chunk_counter, 1ull);
            j = __shfl_sync(0xffffffffu, j, 0);
            int64_t k0, k1;
            if (!dyn_chunk(p.sc, p.chunk, p.trip, (int64_t)j, k0, k1)) break;
            rows(k0, k1);
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
    } else {
        static_ranges(p.sk, p.trip, p.chunk, W, w, rows);
    }
}

}  // namespace

int matvec_max_teams_per_sm(int units) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, matvec_kernel, units, 0) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return n > 0 ? n : 1;
}

cudaError_t launch_matvec(int teams, int units, const MatvecParams& p, cudaStream_t s) {
    return launch_pdl(matvec_kernel, teams, units, 0, s, p);
}

}  // namespace upir
