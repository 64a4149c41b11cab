// AXPY loop kernels (§6, y[i] = y[i] + a * x[i]) for every pair of reduction
// operators; compiled in a file of their own to keep build times short.
#include "elem_kernel.cuh"

namespace upir {

namespace {

template <bool DYN>
cudaError_t launch_axpy_fop(int fop, int iop, int teams, int units, const ElemParams& p, cudaStream_t s) {
    switch (fop) {
        case 0: return launch_elem_iop<UPIR_BODY_AXPY, DYN, 0>(iop, teams, units, p, s);
        case UPIR_RED_ADD: return launch_elem_iop<UPIR_BODY_AXPY, DYN, UPIR_RED_ADD>(iop, teams, units, p, s);
        case UPIR_RED_MUL: return launch_elem_iop<UPIR_BODY_AXPY, DYN, UPIR_RED_MUL>(iop, teams, units, p, s);
        case UPIR_RED_MAX: return launch_elem_iop<UPIR_BODY_AXPY, DYN, UPIR_RED_MAX>(iop, teams, units, p, s);
        case UPIR_RED_MIN: return launch_elem_iop<UPIR_BODY_AXPY, DYN, UPIR_RED_MIN>(iop, teams, units, p, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_axpy_main(bool dyn, int fop, int iop, int teams, int units, const ElemParams& p,
                             cudaStream_t s) {
    return dyn ? launch_axpy_fop<true>(fop, iop, teams, units, p, s)
               : launch_axpy_fop<false>(fop, iop, teams, units, p, s);
}

}  // namespace upir
