// Batches of independent regions (§3.1 SPMD regions submitted together):
// one launch per loop, the same launches captured in one CUDA graph, or one
// persistent launch over a work list of (region, tile) items, itself captured
// in a CUDA graph.  The tile shapes of a persistent batch are picked by
// measurement (upir_batch_autotune).
#include <algorithm>
#include <cstring>
#include <numeric>

#include "runtime_internal.h"

struct upir_batch_s {
    upir_ctx ctx = nullptr;
    std::vector<upir_region> regions;
    int mode = UPIR_BATCH_LAUNCHES;
    cudaGraphExec_t gexec = nullptr;
    // persistent mode
    std::vector<upir::BatchRegion> table;  // host copy; device copy in `dev`
    std::vector<double> cost;              // bytes moved by each region
    int axpy_tile = 8192, jac_rows = 16, mv_rows = 16;
    int teams = 0;
    void* dev = nullptr;
    size_t dev_bytes = 0;
    upir::BatchParams params{};
};

namespace upir {

void destroy_batch(upir_batch b) {
    for (upir_region r : b->regions) r->batch_refs--;
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->dev) {
        cudaStreamSynchronize(b->ctx->stream);
        dev_free(b->ctx, b->dev, b->dev_bytes);
    }
    b->ctx->batches.erase(b);
    delete b;
}

}  // namespace upir

using namespace upir;

namespace {

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Describe one region for the persistent executor, or say why it cannot be.
upir_status describe_region(upir_ctx ctx, int idx, upir_region r, BatchRegion* out, double* cost) {
    if (r->loops.size() != 1)
        return fail(ctx, UPIR_EUNSUPPORTED, "persistent batch: region %d must hold exactly one loop", idx);
    const LoopRec& lp = *r->loops[0];
    BatchRegion R;
    memset(&R, 0, sizeof(R));
    const upir_reduction* red = lp.reds.empty() ? nullptr : &lp.reds[0];
    if (lp.reds.size() > 1 || (red && red->dtype != UPIR_F32))
        return fail(ctx, UPIR_EUNSUPPORTED, "persistent batch: region %d may carry one FP32 reduction", idx);
    if (red) {
        R.fop = red->op;
        R.fterm = red->term;
        R.fvar = static_cast<float*>(red->var->dev) + red->index;
    }
    switch (lp.body) {
        case UPIR_BODY_AXPY:
            if (lp.step != 1)
                return fail(ctx, UPIR_EUNSUPPORTED, "persistent batch: region %d: AXPY needs step 1", idx);
            if (red && red->op != UPIR_RED_ADD)
                return fail(ctx, UPIR_EUNSUPPORTED, "persistent batch: region %d: AXPY reductions must be +", idx);
            R.op = BOP_AXPY;
            R.in0 = static_cast<const float*>(lp.bufs[0]->dev);
            R.out = static_cast<float*>(lp.bufs[1]->dev);
            R.a = (float)lp.scalars[0];
            R.lb = lp.lb;
            R.trip = lp.trip;
            *cost = 12.0 * lp.trip;
            break;
        case UPIR_BODY_JACOBI5:
            if (red && red->op != UPIR_RED_MAX && red->op != UPIR_RED_MIN)
                return fail(ctx, UPIR_EUNSUPPORTED, "persistent batch: region %d: Jacobi reductions must be max/min", idx);
            R.op = BOP_JACOBI;
            R.in0 = static_cast<const float*>(lp.bufs[0]->dev);
            R.out = static_cast<float*>(lp.bufs[1]->dev);
            R.rows = (int64_t)lp.scalars[0];
            R.cols = (int64_t)lp.scalars[1];
            R.lb = lp.lb;
            R.trip = lp.ub - lp.lb > 0 ? lp.ub - lp.lb : 0;
            *cost = 8.0 * R.trip * (R.cols - 2);
            break;
        case UPIR_BODY_MATVEC:
            if (lp.step != 1)
                return fail(ctx, UPIR_EUNSUPPORTED, "persistent batch: region %d: matvec needs step 1", idx);
            R.op = BOP_MATVEC;
            R.in0 = static_cast<const float*>(lp.bufs[0]->dev);
            R.in1 = static_cast<const float*>(lp.bufs[1]->dev);
            R.out = static_cast<float*>(lp.bufs[2]->dev);
            R.rows = (int64_t)lp.scalars[0];
            R.cols = (int64_t)lp.scalars[1];
            R.lb = lp.lb;
            R.trip = lp.trip;
            *cost = 4.0 * lp.trip * R.cols;
            break;
        default:
            return fail(ctx, UPIR_EUNSUPPORTED, "persistent batch: region %d: body %d is not supported", idx, lp.body);
    }
    *out = R;
    return UPIR_OK;
}

// (Re)build the work list for the batch's tile shapes, upload it and capture
// the persistent launch in a CUDA graph.
upir_status build_persistent(upir_batch b) {
    upir_ctx ctx = b->ctx;
    const int n = (int)b->table.size();
    // tiles per region and partial slots
    int64_t nitems = 0, nslots = 0;
    for (auto& R : b->table) {
        if (R.op == BOP_AXPY) R.tiles = ceil_div(R.trip, b->axpy_tile);
        else if (R.op == BOP_JACOBI) {
            R.tiles_c = ceil_div(R.cols, kBatchJacCols);
            R.tiles = ceil_div(R.trip, b->jac_rows) * R.tiles_c;
        } else {
            // rows of at most 64 columns go one per unit (a team takes 256 of
            // them); wider rows one per warp, mv_rows to an item
            R.tile_rows = R.cols <= kBatchNarrowCols ? kBatchUnits : b->mv_rows;
            R.tiles = ceil_div(R.trip, R.tile_rows);
        }
        R.slot0 = nslots;
        if (R.op == BOP_AXPY && R.fop) nslots += R.tiles;
        nitems += R.tiles;
    }
    // largest regions first: the small ones fill in behind them
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int i, int j) { return b->cost[i] > b->cost[j]; });
    std::vector<int2> items;
    items.reserve((size_t)nitems);
    for (int i : order)
        for (int64_t t = 0; t < b->table[i].tiles; ++t) items.push_back(make_int2(i, (int)t));

    // device layout: [counter u64, exit ticket u32, pad][tickets u32 x n][regions][items][partials]
    auto align = [](size_t v) { return (v + 255) / 256 * 256; };
    const size_t off_tickets = 256;
    const size_t off_regions = align(off_tickets + 4 * (size_t)n);
    const size_t off_items = align(off_regions + sizeof(BatchRegion) * (size_t)n);
    const size_t off_partials = align(off_items + sizeof(int2) * items.size());
    const size_t bytes = off_partials + sizeof(Partial) * (size_t)nslots;
    if (bytes > b->dev_bytes) {
        if (b->dev) {
            cudaStreamSynchronize(ctx->stream);
            dev_free(ctx, b->dev, b->dev_bytes);
            b->dev = nullptr;
            b->dev_bytes = 0;
        }
        b->dev = dev_alloc(ctx, bytes);
        if (!b->dev) return fail(ctx, UPIR_ENOMEM, "persistent batch: scratch of %zu bytes", bytes);
        b->dev_bytes = bytes;
    }
    char* base = static_cast<char*>(b->dev);
    for (int i = 0; i < n; ++i)
        b->table[i].ticket = reinterpret_cast<unsigned*>(base + off_tickets) + i;
    cudaError_t e = cudaMemsetAsync(base, 0, off_regions, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(base + off_regions, b->table.data(), sizeof(BatchRegion) * n,
                            cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess && !items.empty())
        e = cudaMemcpyAsync(base + off_items, items.data(), sizeof(int2) * items.size(),
                            cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "persistent batch: uploading the work list");

    BatchParams& P = b->params;
    P.regions = reinterpret_cast<const BatchRegion*>(base + off_regions);
    P.items = reinterpret_cast<const int2*>(base + off_items);
    P.nitems = (int64_t)items.size();
    P.partials = reinterpret_cast<Partial*>(base + off_partials);
    P.counter = reinterpret_cast<unsigned long long*>(base);
    P.exit_ticket = reinterpret_cast<unsigned*>(base + 8);
    P.nregions = n;
    P.axpy_tile = b->axpy_tile;
    P.jac_rows = b->jac_rows;
    P.mv_rows = b->mv_rows;
    b->teams = (int)std::max<int64_t>(1, std::min<int64_t>(nitems, (int64_t)kNumSMs * batch_persistent_teams_per_sm()));

    if (b->gexec) {
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
    }
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamBeginCapture");
    cudaError_t le = P.nitems ? launch_batch_persistent(b->teams, P, ctx->stream) : cudaSuccess;
    e = cudaStreamEndCapture(ctx->stream, &g);
    if (le != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(ctx, le, "persistent batch launch");
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&b->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGraphInstantiate");
    return UPIR_OK;
}

}  // namespace

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
    std::vector<BatchRegion> table;
    std::vector<double> cost;
    if (mode == UPIR_BATCH_PERSISTENT) {
        table.resize(n);
        cost.resize(n);
        for (int32_t i = 0; i < n; ++i) {
            upir_status st = describe_region(ctx, i, regions[i], &table[i], &cost[i]);
            if (st != UPIR_OK) return st;
        }
    }
    upir_batch b = new upir_batch_s();
    b->ctx = ctx;
    b->mode = mode;
    b->regions.assign(regions, regions + n);
    for (upir_region r : b->regions) r->batch_refs++;
    ctx->batches.insert(b);
    upir_status st = UPIR_OK;
    if (mode == UPIR_BATCH_GRAPH) {
        st = capture_graph(ctx, b->regions, &b->gexec);
    } else if (mode == UPIR_BATCH_PERSISTENT) {
        b->table = std::move(table);
        b->cost = std::move(cost);
        st = build_persistent(b);
    }
    if (st != UPIR_OK) {
        destroy_batch(b);
        return st;
    }
    *out = b;
    return UPIR_OK;
}

extern "C" upir_status upir_batch_submit(upir_batch b) {
    if (!b) return UPIR_EINVAL;
    upir_ctx ctx = b->ctx;
    for (upir_region r : b->regions)
        if (upir_status st = wait_region_buffers(r)) return st;
    upir_status st = UPIR_OK;
    if (b->mode == UPIR_BATCH_LAUNCHES) {
        for (upir_region r : b->regions) {
            st = launch_region_loops(r, ctx->timing);
            if (st != UPIR_OK) break;
        }
    } else {
        st = launch_graph_timed(ctx, b->gexec, b->mode == UPIR_BATCH_GRAPH ? -2 : -3);
    }
    // record the buffers' last use even after a failed launch: the launches
    // that went out before it still use them (the first error is returned)
    upir_status mst = mark_regions_buffers(b->regions.data(), b->regions.size());
    return st == UPIR_OK ? mst : st;
}

extern "C" upir_status upir_batch_destroy(upir_batch b) {
    if (!b) return UPIR_EINVAL;
    destroy_batch(b);
    return UPIR_OK;
}

extern "C" upir_status upir_batch_autotune(upir_batch b, int32_t reps, int64_t* tiles_out) {
    if (!b) return UPIR_EINVAL;
    upir_ctx ctx = b->ctx;
    if (b->mode != UPIR_BATCH_PERSISTENT)
        return fail(ctx, UPIR_EINVAL, "upir_batch_autotune: only persistent batches have tile shapes");
    if (reps < 1) return fail(ctx, UPIR_EINVAL, "upir_batch_autotune: reps must be >= 1");
    static const int axpy_tiles[] = {4096, 8192, 16384, 32768};
    static const int jac_rows[] = {8, 16, 32};
    static const int mv_rows[] = {8, 16, 32};
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return cuda_fail(ctx, cudaGetLastError(), "cudaEventCreate");
    float best = 1e30f;
    int best_cfg[3] = {b->axpy_tile, b->jac_rows, b->mv_rows};
    upir_status st = UPIR_OK;
    for (int at : axpy_tiles)
        for (int jr : jac_rows)
            for (int mr : mv_rows) {
                b->axpy_tile = at;
                b->jac_rows = jr;
                b->mv_rows = mr;
                if ((st = build_persistent(b)) != UPIR_OK) goto done;
                cudaGraphLaunch(b->gexec, ctx->stream);  // warm-up
                std::vector<float> ts;
                for (int k = 0; k < reps; ++k) {
                    cudaEventRecord(e0, ctx->stream);
                    cudaGraphLaunch(b->gexec, ctx->stream);
                    cudaEventRecord(e1, ctx->stream);
                    if (cudaEventSynchronize(e1) != cudaSuccess) {
                        st = cuda_fail(ctx, cudaGetLastError(), "upir_batch_autotune: timing");
                        goto done;
                    }
                    float ms = 0.0f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    ts.push_back(ms);
                }
                std::nth_element(ts.begin(), ts.begin() + ts.size() / 2, ts.end());
                const float med = ts[ts.size() / 2];
                if (med < best) {
                    best = med;
                    best_cfg[0] = at;
                    best_cfg[1] = jr;
                    best_cfg[2] = mr;
                }
            }
done:
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->axpy_tile = best_cfg[0];
    b->jac_rows = best_cfg[1];
    b->mv_rows = best_cfg[2];
    upir_status st2 = build_persistent(b);
    if (st == UPIR_OK) st = st2;
    // the timing runs used every region's buffers
    if (upir_status st3 = mark_regions_buffers(b->regions.data(), b->regions.size()); st == UPIR_OK) st = st3;
    if (tiles_out) {
        tiles_out[0] = b->axpy_tile;
        tiles_out[1] = b->jac_rows;
        tiles_out[2] = b->mv_rows;
    }
    return st;
}
