// Tensor-core (tcgen05) GEMM bodies: planning and launch.
#include "runtime_internal.h"

namespace upir {

upir_status plan_gemm_tc(upir_region r, LoopRec& lp, int64_t, int64_t, int64_t, upir_status st) {
    if (st != UPIR_OK) return st;
    (void)lp;
    return fail(r->ctx, UPIR_EUNSUPPORTED, "upir_loop: tensor-core GEMM bodies are not built yet");
}

cudaError_t launch_gemm_tc_loop(upir_ctx, LoopRec&, cudaStream_t) { return cudaErrorNotSupported; }

}  // namespace upir
