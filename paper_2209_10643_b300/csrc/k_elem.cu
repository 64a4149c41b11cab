// Element-granular loop kernels other than AXPY (IMOD, COVERAGE, per-point
// JACOBI5), the reduction finalize kernel and the dispatch of all of them.
#include "elem_kernel.cuh"

namespace upir {

namespace {

// Deterministic finalization of a loop's reductions (the reduction sync fused
// with the loop's closing barrier, §3.1.2): block g folds partial slots
// [g * kFinSeg, (g + 1) * kFinSeg) in a fixed order; with several blocks the
// last one to finish (atomic ticket) folds the group results in index order,
// combines them with the variables' values before the loop and stores them.
// It runs after the loop kernel completes (programmatic dependent launch +
// griddepcontrol.wait) and also returns the dynamic chunk counter to zero.
__global__ void __launch_bounds__(256) finalize_kernel(const RedVars rv, const Scratch sc,
                                                       int64_t nslots, int reset_counter) {
    __shared__ int last;
    griddep_wait();
    const int64_t G = gridDim.x, g = blockIdx.x;
    const int64_t s0 = g * kFinSeg;
    const int64_t rem = nslots - s0;
    const int64_t n = rem <= 0 ? 0 : (rem < kFinSeg ? rem : (int64_t)kFinSeg);
    const Partial gp = block_reduce_slots(sc.partials + s0, n, rv.fop, rv.iop);
    if (G == 1) {
        if (threadIdx.x == 0) {
            write_reduction_vars(rv, gp);
            if (reset_counter) *sc.chunk_counter = 0;
        }
        return;
    }
    if (threadIdx.x == 0) {
        sc.group_partials[g] = gp;
        __threadfence();
        last = atomicAdd(sc.ticket, 1u) == (unsigned)G - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    const Partial fin = block_reduce_slots(sc.group_partials, G, rv.fop, rv.iop);
    if (threadIdx.x == 0) {
        write_reduction_vars(rv, fin);
        *sc.ticket = 0;
        if (reset_counter) *sc.chunk_counter = 0;
    }
}

template <int BODY, bool DYN>
cudaError_t launch_fop(int fop, int iop, int teams, int units, const ElemParams& p, cudaStream_t s) {
    switch (fop) {
        case 0: return launch_elem_iop<BODY, DYN, 0>(iop, teams, units, p, s);
        case UPIR_RED_ADD: return launch_elem_iop<BODY, DYN, UPIR_RED_ADD>(iop, teams, units, p, s);
        case UPIR_RED_MUL: return launch_elem_iop<BODY, DYN, UPIR_RED_MUL>(iop, teams, units, p, s);
        case UPIR_RED_MAX: return launch_elem_iop<BODY, DYN, UPIR_RED_MAX>(iop, teams, units, p, s);
        case UPIR_RED_MIN: return launch_elem_iop<BODY, DYN, UPIR_RED_MIN>(iop, teams, units, p, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_axpy_main(bool dyn, int fop, int iop, int teams, int units, const ElemParams& p,
                             cudaStream_t s);

int64_t finalize_groups(int64_t nslots) { return nslots > 0 ? (nslots + kFinSeg - 1) / kFinSeg : 1; }

cudaError_t launch_finalize(const RedVars& rv, const Scratch& sc, int64_t nslots, bool reset_counter,
                            cudaStream_t s) {
    return launch_pdl(finalize_kernel, (unsigned)finalize_groups(nslots), 256, 0, s, rv, sc, nslots,
                      reset_counter ? 1 : 0);
}

cudaError_t launch_elem_main(int body, bool dyn, int fop, int iop, int teams, int units,
                             const ElemParams& p, cudaStream_t s) {
    switch (body) {
        case UPIR_BODY_AXPY: return launch_axpy_main(dyn, fop, iop, teams, units, p, s);
        case UPIR_BODY_IMOD:
            return dyn ? launch_elem_iop<UPIR_BODY_IMOD, true, 0>(iop, teams, units, p, s)
                       : launch_elem_iop<UPIR_BODY_IMOD, false, 0>(iop, teams, units, p, s);
        case UPIR_BODY_COVERAGE:
            return dyn ? launch_elem_iop<UPIR_BODY_COVERAGE, true, 0>(iop, teams, units, p, s)
                       : launch_elem_iop<UPIR_BODY_COVERAGE, false, 0>(iop, teams, units, p, s);
        case UPIR_BODY_JACOBI5:
            return dyn ? launch_fop<UPIR_BODY_JACOBI5, true>(fop, 0, teams, units, p, s)
                       : launch_fop<UPIR_BODY_JACOBI5, false>(fop, 0, teams, units, p, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_elem(int body, bool dyn, int fop, int iop, int teams, int units,
                        const ElemParams& p, cudaStream_t s) {
    const bool red = fop || iop;
    const int64_t nslots = dyn ? p.nchunks : teams;
    if ((red || dyn) && (!red || (nslots <= kFinSeg && units % 32 == 0))) {
        ElemParams q = p;  // the loop kernel's last team finishes the loop
        q.fuse_fin = 1;
        return launch_elem_main(body, dyn, fop, iop, teams, units, q, s);
    }
    cudaError_t e = launch_elem_main(body, dyn, fop, iop, teams, units, p, s);
    if (e != cudaSuccess) return e;
    if (red) return launch_finalize(p.rv, p.sc, nslots, dyn, s);
    return cudaSuccess;
}

}  // namespace upir
