// Batches of independent regions (§3.1 SPMD regions submitted together):
// one launch per loop, the same launches captured in one CUDA graph, or one
// persistent launch over a work list.
#include "runtime_internal.h"

struct upir_batch_s {
    upir_ctx ctx = nullptr;
    std::vector<upir_region> regions;
    int mode = UPIR_BATCH_LAUNCHES;
    cudaGraphExec_t gexec = nullptr;
};

namespace upir {

void destroy_batch(upir_batch b) {
    for (upir_region r : b->regions) r->batch_refs--;
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    b->ctx->batches.erase(b);
    delete b;
}

}  // namespace upir

using namespace upir;

extern "C" upir_status upir_batch_create(upir_ctx ctx, const upir_region* regions, int32_t n,
                                         int32_t mode, upir_batch* out) {
    if (!ctx) return UPIR_EINVAL;
    if (!out || n < 0 || (n > 0 && !regions)) return fail(ctx, UPIR_EINVAL, "upir_batch_create: bad arguments");
    *out = nullptr;
    if (mode < UPIR_BATCH_LAUNCHES || mode > UPIR_BATCH_PERSISTENT)
        return fail(ctx, UPIR_EINVAL, "upir_batch_create: unknown mode %d", mode);
    for (int32_t i = 0; i < n; ++i)
        if (!regions[i] || !ctx->regions.count(regions[i]))
            return fail(ctx, UPIR_EINVAL, "upir_batch_create: region %d does not belong to the context", i);
    if (mode == UPIR_BATCH_PERSISTENT)
        return fail(ctx, UPIR_EUNSUPPORTED, "upir_batch_create: persistent batches are not built yet");
    upir_batch b = new upir_batch_s();
    b->ctx = ctx;
    b->mode = mode;
    b->regions.assign(regions, regions + n);
    for (upir_region r : b->regions) r->batch_refs++;
    ctx->batches.insert(b);
    if (mode == UPIR_BATCH_GRAPH) {
        upir_status st = capture_graph(ctx, b->regions, &b->gexec);
        if (st != UPIR_OK) {
            destroy_batch(b);
            return st;
        }
    }
    *out = b;
    return UPIR_OK;
}

extern "C" upir_status upir_batch_submit(upir_batch b) {
    if (!b) return UPIR_EINVAL;
    upir_ctx ctx = b->ctx;
    if (b->mode == UPIR_BATCH_LAUNCHES) {
        for (upir_region r : b->regions) {
            upir_status st = launch_region_loops(r, ctx->timing);
            if (st != UPIR_OK) return st;
        }
        return UPIR_OK;
    }
    return launch_graph_timed(ctx, b->gexec, -2);
}

extern "C" upir_status upir_batch_destroy(upir_batch b) {
    if (!b) return UPIR_EINVAL;
    destroy_batch(b);
    return UPIR_OK;
}
