// Learned cost model kernels (12 -> 64 -> 64 -> 1 ReLU MLP).
#include "runtime_internal.h"

using namespace upir;

extern "C" upir_status upir_mlp_forward(upir_ctx ctx, const float*, const float*, int32_t, float*) {
    return ctx ? fail(ctx, UPIR_EUNSUPPORTED, "MLP kernels are not built yet") : UPIR_EINVAL;
}
extern "C" upir_status upir_mlp_backward(upir_ctx ctx, const float*, const float*, const float*, int32_t,
                                         float*, float*) {
    return ctx ? fail(ctx, UPIR_EUNSUPPORTED, "MLP kernels are not built yet") : UPIR_EINVAL;
}
extern "C" upir_status upir_mlp_sgd(upir_ctx ctx, float*, const float*, float) {
    return ctx ? fail(ctx, UPIR_EUNSUPPORTED, "MLP kernels are not built yet") : UPIR_EINVAL;
}
