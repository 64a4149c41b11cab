// Loop validation and launch planning (§3.2: canonical loop + worksharing;
// §5: reduction clauses).  A loop is checked completely when it is recorded;
// the planner then fixes the kernel variant, the launch geometry, the device
// scratch and the kernel parameters, so submission only launches.
#include <cstring>

#include "runtime_internal.h"

using namespace upir;

namespace {

constexpr int64_t kMaxTrip = 1ll << 62;
constexpr int kResidentThreadsPerSM = 2048;

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// ceil((ub - lb) / step) in 128-bit arithmetic (no overflow for any int64 bounds).
bool compute_trip(int64_t lb, int64_t ub, int64_t step, int64_t* trip) {
    __int128 n = 0;
    if (step > 0 && ub > lb) n = ((__int128)ub - lb + step - 1) / step;
    if (step < 0 && lb > ub) n = ((__int128)lb - ub + (-(__int128)step) - 1) / (-(__int128)step);
    if (n > kMaxTrip) return false;
    *trip = (int64_t)n;
    return true;
}

bool is_int(double v) { return v == (double)(int64_t)v; }

struct Check {
    upir_ctx ctx;
    upir_status st = UPIR_OK;
    bool operator()(bool cond, upir_status code, const char* msg) {
        if (!cond && st == UPIR_OK) st = fail(ctx, code, "upir_loop: %s", msg);
        return cond;
    }
};

// Device scratch: [chunk counter u64][ticket u32][pad][group tickets u32 x G]
// [group partials x G][partials x S][chunk starts i64 x (chunks + 1)], zeroed
// once, then the loop's chunk table (guided schedules, taskloops) copied in.
upir_status alloc_scratch(upir_ctx ctx, LoopRec& lp, int64_t ngroups, int64_t nslots, Scratch* sc) {
    if (lp.dry) {  // planning only: the geometry is wanted, not the scratch
        memset(sc, 0, sizeof(*sc));
        return UPIR_OK;
    }
    const size_t head = 16;
    const size_t gt = ((size_t)ngroups * 4 + 15) / 16 * 16;
    const size_t tab_off = head + gt + (size_t)ngroups * sizeof(Partial) + (size_t)nslots * sizeof(Partial);
    const size_t bytes = tab_off + lp.chunk_table.size() * sizeof(int64_t);
    char* p = static_cast<char*>(dev_alloc(ctx, bytes));
    if (!p) return fail(ctx, UPIR_ENOMEM, "upir_loop: scratch allocation of %zu bytes failed", bytes);
    cudaError_t e = cudaMemsetAsync(p, 0, bytes, ctx->stream);
    if (e != cudaSuccess) {
        dev_free(ctx, p, bytes);
        return cuda_fail(ctx, e, "upir_loop: scratch memset");
    }
    lp.scratch = p;
    lp.scratch_bytes = bytes;
    lp.counter_off = 0;
    lp.counter_bytes = head + gt;
    sc->chunk_counter = reinterpret_cast<unsigned long long*>(p);
    sc->ticket = reinterpret_cast<unsigned*>(p + 8);
    sc->group_tickets = reinterpret_cast<unsigned*>(p + head);
    sc->group_partials = reinterpret_cast<Partial*>(p + head + gt);
    sc->partials = sc->group_partials + ngroups;
    sc->chunk_starts = nullptr;
    sc->nchunks_tab = 0;
    if (!lp.chunk_table.empty()) {
        // the host table lives in the loop record, so the copy may stay in flight
        e = cudaMemcpyAsync(p + tab_off, lp.chunk_table.data(), lp.chunk_table.size() * sizeof(int64_t),
                            cudaMemcpyHostToDevice, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "upir_loop: chunk table copy");
        sc->chunk_starts = reinterpret_cast<const int64_t*>(p + tab_off);
        sc->nchunks_tab = (int64_t)lp.chunk_table.size() - 1;
    }
    return UPIR_OK;
}

bool is_dyn(int sched) {
    return sched == UPIR_SCHED_DYNAMIC || sched == UPIR_SCHED_GUIDED || sched == UPIR_SCHED_TASKLOOP;
}

// Kernels know two ways of handing out work: static ranges, or chunks claimed
// from a counter (of fixed size, or from the chunk table).
int kernel_sched(int sched) { return is_dyn(sched) ? UPIR_SCHED_DYNAMIC : UPIR_SCHED_STATIC; }

constexpr int64_t kDefaultTasks = 8 * kNumSMs;  // taskloop without grainsize / num_tasks

int64_t taskloop_tasks(const LoopRec& lp, int64_t n) {
    if (n <= 0) return 0;
    int64_t t = -1;
    if (lp.num_tasks > 0) t = std::min(lp.num_tasks, n);
    if (lp.grainsize > 0) t = t < 0 ? std::max<int64_t>(1, n / lp.grainsize)
                                    : std::min(t, std::max<int64_t>(1, n / lp.grainsize));
    return t < 0 ? std::min(kDefaultTasks, n) : t;
}

// Number of chunks handed out dynamically over n units, for sizing the grid
// (guided: an upper bound; the table is built once the workers are known).
int64_t dyn_estimate(const LoopRec& lp, int64_t n) {
    if (lp.sched == UPIR_SCHED_TASKLOOP) return taskloop_tasks(lp, n);
    return ceil_div(n, lp.chunk > 0 ? lp.chunk : 1);
}

// The chunk table of a guided schedule or a taskloop over n units with W
// workers (§3.2; see upir_sched); returns the number of chunks handed out
// dynamically, also kept in lp.nchunks.
int64_t build_chunk_table(LoopRec& lp, int64_t n, int64_t workers) {
    lp.chunk_table.clear();
    if (lp.sched == UPIR_SCHED_GUIDED) {
        const int64_t c = lp.chunk > 0 ? lp.chunk : 1, W = std::max<int64_t>(workers, 1);
        int64_t s = 0;
        lp.chunk_table.push_back(0);
        while (s < n) {
            s += std::min(n - s, std::max(c, ceil_div(n - s, W)));
            lp.chunk_table.push_back(s);
        }
    } else if (lp.sched == UPIR_SCHED_TASKLOOP) {
        const int64_t t = taskloop_tasks(lp, n);
        lp.chunk_table.push_back(0);
        for (int64_t k = 0, s = 0; k < t; ++k) {
            s += n / t + (k < n % t ? 1 : 0);
            lp.chunk_table.push_back(s);
        }
    }
    lp.nchunks = lp.chunk_table.empty() ? ceil_div(n, lp.chunk > 0 ? lp.chunk : 1)
                                        : (int64_t)lp.chunk_table.size() - 1;
    return lp.nchunks;
}

int default_teams_for_chunks(int64_t nchunks, int units) {
    const int64_t resident = (int64_t)kNumSMs * (kResidentThreadsPerSM / units);
    return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(nchunks, units), resident));
}

}  // namespace

namespace upir {

using PFN_encodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                     const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                     const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                     CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static PFN_encodeTiled encode_fn(upir_ctx ctx) {
    static PFN_encodeTiled fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void* f = nullptr;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000,
                                                         cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !f) {
            fail(ctx, UPIR_ECUDA, "cuTensorMapEncodeTiled entry point unavailable");
            return nullptr;
        }
        fn = reinterpret_cast<PFN_encodeTiled>(f);
    }
    return fn;
}

upir_status encode_tmap_1d(upir_ctx ctx, CUtensorMap* m, const void* base, int dtype_code, uint64_t n,
                           uint32_t box) {
    PFN_encodeTiled fn = encode_fn(ctx);
    if (!fn) return UPIR_ECUDA;
    const cuuint64_t dims[1] = {n};
    const cuuint64_t strides[1] = {0};  // a rank-1 map has no strides; the array is not read
    const cuuint32_t boxd[1] = {box};
    const cuuint32_t estr[1] = {1};
    CUresult r = fn(m, (CUtensorMapDataType)dtype_code, 1, const_cast<void*>(base), dims, strides, boxd, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(ctx, UPIR_ECUDA, "cuTensorMapEncodeTiled (1D) failed (%d)", (int)r);
    return UPIR_OK;
}

upir_status encode_tmap_2d(upir_ctx ctx, CUtensorMap* m, const void* base, int dtype_code,
                           int elem_bytes, uint64_t cols, uint64_t rows, uint32_t box_cols,
                           uint32_t box_rows, int swizzle_bytes) {
    PFN_encodeTiled fn = encode_fn(ctx);
    if (!fn) return UPIR_ECUDA;
    const cuuint64_t dims[2] = {cols, rows};
    const cuuint64_t strides[1] = {cols * (uint64_t)elem_bytes};
    const cuuint32_t box[2] = {box_cols, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, (CUtensorMapDataType)dtype_code, 2, const_cast<void*>(base), dims, strides,
                    box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    swizzle_bytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B
                    : swizzle_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B
                    : swizzle_bytes == 32 ? CU_TENSOR_MAP_SWIZZLE_32B : CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(ctx, UPIR_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return UPIR_OK;
}

void release_loop(upir_ctx ctx, LoopRec& lp) {
    if (lp.scratch) {
        cudaStreamSynchronize(ctx->stream);
        dev_free(ctx, lp.scratch, lp.scratch_bytes);
        lp.scratch = nullptr;
    }
    if (lp.holds_refs) {
        for (upir_buf b : lp.bufs) b->refs--;
        for (auto& red : lp.reds) red.var->refs--;
        lp.holds_refs = false;
    }
}

upir_status plan_loop(upir_region r, const upir_loop_desc* d, LoopRec& lp) {
    upir_ctx ctx = r->ctx;
    Check ok{ctx};
    if (!ok(d != nullptr, UPIR_EINVAL, "descriptor is NULL")) return ok.st;
    ok(d->step != 0, UPIR_EINVAL, "step must be non-zero");
    ok(d->chunk >= 0, UPIR_EINVAL, "chunk must be >= 0");
    ok(d->sched >= UPIR_SCHED_STATIC && d->sched <= UPIR_SCHED_TASKLOOP, UPIR_EINVAL, "unknown schedule");
    ok(d->body >= UPIR_BODY_AXPY && d->body <= UPIR_BODY_FILTER7, UPIR_EINVAL, "unknown body");
    ok(d->nbufs >= 0 && (d->nbufs == 0 || d->bufs), UPIR_EINVAL, "bad buffer list");
    ok(d->nscalars >= 0 && (d->nscalars == 0 || d->scalars), UPIR_EINVAL, "bad scalar list");
    ok(d->nreductions >= 0 && d->nreductions <= 2 && (d->nreductions == 0 || d->reductions),
       UPIR_EINVAL, "0..2 reductions per loop");
    ok(d->nhints >= 0 && (d->nhints == 0 || d->hints), UPIR_EINVAL, "bad hint list");
    ok(d->collapse == 1 || d->collapse == 2, UPIR_EINVAL, "collapse must be 1 or 2");
    if (ok.st) return ok.st;
    if (!ok(compute_trip(d->lb, d->ub, d->step, &lp.trip), UPIR_EINVAL, "trip count overflows"))
        return ok.st;

    lp.lb = d->lb;
    lp.ub = d->ub;
    lp.step = d->step;
    lp.chunk = d->chunk;
    lp.collapse = d->collapse;
    lp.sched = d->sched;
    lp.body = d->body;
    lp.nowait = d->nowait;
    for (int i = 0; i < d->nbufs; ++i) {
        if (!d->bufs[i] || !ctx->all_bufs.count(d->bufs[i]) || !d->bufs[i]->live)
            return fail(ctx, UPIR_ENOTMAPPED, "upir_loop: buffer %d is not mapped", i);
        lp.bufs.push_back(d->bufs[i]);
    }
    lp.scalars.assign(d->scalars, d->scalars + d->nscalars);
    for (int i = 0; i < d->nhints; ++i) {
        const int64_t k = d->hints[2 * i], v = d->hints[2 * i + 1];
        if (k == UPIR_HINT_VARIANT) ok(v >= 0 && v <= 3, UPIR_EINVAL, "variant hint out of range"), lp.variant = (int)v;
        else if (k == UPIR_HINT_TILE_M) ok(v >= 1 && v <= 254, UPIR_EINVAL, "tile_m hint out of range"), lp.tile_m = (int)v;
        else if (k == UPIR_HINT_TILE_N) ok(v >= 4 && v <= 248 && v % 4 == 0, UPIR_EINVAL, "tile_n hint must be a multiple of 4 in [4, 248]"), lp.tile_n = (int)v;
        else if (k == UPIR_HINT_VEC) ok(v == 1 || v == 4 || v == 8 || v == 16 || v == 32, UPIR_EINVAL, "vec hint must be 1, 4, 8, 16 or 32"), lp.vec = (int)v;
        else if (k == UPIR_HINT_STAGES) ok(v >= 1 && v <= 4, UPIR_EINVAL, "stages hint must be in [1, 4]"), lp.stages = (int)v;
        else if (k == UPIR_HINT_GRAINSIZE) ok(v >= 1, UPIR_EINVAL, "grainsize hint must be >= 1"), lp.grainsize = v;
        else if (k == UPIR_HINT_NUM_TASKS) ok(v >= 1, UPIR_EINVAL, "num_tasks hint must be >= 1"), lp.num_tasks = v;
        else if (k == UPIR_HINT_TILE_ORDER) ok(v >= 0 && v <= 2, UPIR_EINVAL, "tile order hint must be 0, 1 or 2"), lp.tile_order = (int)v;
        else ok(false, UPIR_EINVAL, "unknown hint key");
    }
    if (ok.st) return ok.st;

    // Schedule: RUNTIME takes the context's run schedule, AUTO the cost
    // model's pick (§3.2 schedule policies; see upir_sched).
    if (lp.sched == UPIR_SCHED_RUNTIME) {
        lp.sched = ctx->run_sched;
        lp.chunk = ctx->run_chunk;
    }
    int auto_units = 0;
    if (lp.sched == UPIR_SCHED_AUTO) {
        int s2 = UPIR_SCHED_STATIC;
        int64_t c2 = 0;
        auto_schedule(ctx, r, d, lp.trip, &s2, &c2, &auto_units);
        lp.sched = s2;
        lp.chunk = c2;
    }
    ok(lp.sched != UPIR_SCHED_TASKLOOP || lp.chunk == 0, UPIR_EINVAL,
       "taskloop takes no chunk (GRAINSIZE / NUM_TASKS hints set its tasks)");
    ok(lp.sched == UPIR_SCHED_TASKLOOP || (lp.grainsize == 0 && lp.num_tasks == 0), UPIR_EINVAL,
       "GRAINSIZE / NUM_TASKS hints need the TASKLOOP schedule");
    if (ok.st) return ok.st;

    // Reductions: at most one FP32 and one int64 clause.
    RedVars rv{nullptr, nullptr, UPIR_RED_NONE, UPIR_RED_NONE, 0, 0};
    for (int i = 0; i < d->nreductions; ++i) {
        const upir_reduction& red = d->reductions[i];
        ok(red.op >= UPIR_RED_ADD && red.op <= UPIR_RED_MIN, UPIR_EINVAL, "unknown reduction op");
        ok(red.dtype == UPIR_F32 || red.dtype == UPIR_I64, UPIR_EINVAL, "unknown reduction dtype");
        ok(red.term >= UPIR_TERM_Y && red.term <= UPIR_TERM_RESID, UPIR_EINVAL, "unknown reduction term");
        if (ok.st) return ok.st;
        if (!red.var || !ctx->all_bufs.count(red.var) || !red.var->live)
            return fail(ctx, UPIR_ENOTMAPPED, "upir_loop: reduction variable %d is not mapped", i);
        const size_t esz = red.dtype == UPIR_F32 ? 4 : 8;
        if (!ok(red.index >= 0 && (size_t)(red.index + 1) * esz <= red.var->bytes, UPIR_EINVAL,
                "reduction index outside its buffer"))
            return ok.st;
        if (red.dtype == UPIR_F32) {
            if (!ok(rv.fvar == nullptr, UPIR_EINVAL, "at most one FP32 reduction per loop")) return ok.st;
            rv.fvar = static_cast<float*>(red.var->dev) + red.index;
            rv.fop = red.op;
            rv.fterm = red.term;
        } else {
            if (!ok(rv.ivar == nullptr, UPIR_EINVAL, "at most one int64 reduction per loop")) return ok.st;
            rv.ivar = static_cast<long long*>(red.var->dev) + red.index;
            rv.iop = red.op;
            rv.iterm = red.term;
        }
        lp.reds.push_back(red);
    }
    const bool has_f = rv.fvar != nullptr, has_i = rv.ivar != nullptr;
    const bool has_red = has_f || has_i;
    const int64_t first_iv = lp.lb;
    const int64_t last_iv = lp.trip ? lp.lb + (lp.trip - 1) * lp.step : lp.lb;
    const int64_t min_iv = std::min(first_iv, last_iv), max_iv = std::max(first_iv, last_iv);
    auto buf_floats = [&](int i) { return (int64_t)(lp.bufs[i]->bytes / 4); };

    // int64 terms over the induction value
    long long imod_mul = 0, imod_mod = 1, imod_inc = 0;
    auto check_int_terms = [&](int scalar_base) {
        if (!has_i) return;
        ok(rv.iterm == UPIR_TERM_IMOD || rv.iterm == UPIR_TERM_IV, UPIR_EINVAL,
           "int64 reductions take TERM_IMOD or TERM_IV");
        if (rv.iterm != UPIR_TERM_IMOD) return;
        if (!ok((int)lp.scalars.size() >= scalar_base + 2, UPIR_EINVAL, "TERM_IMOD needs scalars mul, mod"))
            return;
        const double mu = lp.scalars[scalar_base], mo = lp.scalars[scalar_base + 1];
        ok(is_int(mu) && is_int(mo) && mo >= 1 && mo < 4.6e18 && std::abs(mu) < 9.2e18, UPIR_EINVAL,
           "TERM_IMOD needs integer mul and a modulus in [1, 2^62)");
        if (ok.st) return;
        imod_mul = (long long)mu;
        imod_mod = (long long)mo;
        const __int128 big = (__int128)1 << 62;
        const __int128 pm = (__int128)imod_mul * std::max<__int128>(-(__int128)min_iv, (__int128)max_iv);
        ok(pm < big && pm > -big, UPIR_EINVAL, "(mul * iv) overflows int64 for this loop");
        const __int128 inc = ((__int128)imod_mul * lp.step) % imod_mod;
        imod_inc = (long long)(inc < 0 ? inc + imod_mod : inc);
    };

    const int U0 = r->units, T0 = r->teams;
    // implicit barrier after the previous loop of the region (1), or, when
    // that loop was nowait, run beside it but complete only after it (2)
    const int wait_prior = (r->loops.empty() || !r->loops.back()->nowait) ? 1 : 2;
    lp.units = U0 ? U0 : (auto_units ? auto_units : 256);
    lp.kind = LK_ELEM;
    ElemParams& ep = lp.ep;
    memset(&ep, 0, sizeof(ep));
    ep.lb = lp.lb;
    ep.step = lp.step;
    ep.trip = lp.trip;
    ep.chunk = lp.chunk;
    ep.rv = rv;
    ep.imod_mod = 1;
    ep.wait_prior = wait_prior;

    switch (lp.body) {
        case UPIR_BODY_AXPY: {
            ok(lp.bufs.size() == 2, UPIR_EINVAL, "AXPY takes bufs x, y");
            ok(lp.scalars.size() >= 1, UPIR_EINVAL, "AXPY takes scalar a");
            ok(lp.collapse == 1, UPIR_EINVAL, "AXPY is a collapse(1) loop");
            if (ok.st) return ok.st;
            if (lp.trip)
                ok(min_iv >= 0 && max_iv < buf_floats(0) && max_iv < buf_floats(1), UPIR_EINVAL,
                   "AXPY iterations index outside x or y");
            if (has_f) ok(rv.fterm == UPIR_TERM_Y || rv.fterm == UPIR_TERM_XY, UPIR_EINVAL,
                          "AXPY FP32 reductions take TERM_Y or TERM_XY");
            check_int_terms(1);
            ep.x = static_cast<const float*>(lp.bufs[0]->dev);
            ep.y = static_cast<float*>(lp.bufs[1]->dev);
            ep.a = (float)lp.scalars[0];
            break;
        }
        case UPIR_BODY_IMOD: {
            ok(lp.bufs.empty(), UPIR_EINVAL, "IMOD takes no buffers");
            ok(!has_f, UPIR_EINVAL, "IMOD has no FP32 terms");
            check_int_terms(0);
            break;
        }
        case UPIR_BODY_COVERAGE: {
            ok(lp.bufs.size() == 2, UPIR_EINVAL, "COVERAGE takes bufs owner, count");
            ok(!has_f, UPIR_EINVAL, "COVERAGE has no FP32 terms");
            if (ok.st) return ok.st;
            ok((int64_t)(lp.bufs[0]->bytes / 8) >= lp.trip && (int64_t)(lp.bufs[1]->bytes / 8) >= lp.trip,
               UPIR_EINVAL, "COVERAGE buffers need trip int64 elements");
            check_int_terms(0);
            ep.owner = static_cast<long long*>(lp.bufs[0]->dev);
            ep.count = static_cast<unsigned long long*>(lp.bufs[1]->dev);
            break;
        }
        case UPIR_BODY_JACOBI5: {
            ok(lp.bufs.size() == 2, UPIR_EINVAL, "JACOBI5 takes bufs u_in, u_out");
            ok(lp.scalars.size() >= 2, UPIR_EINVAL, "JACOBI5 takes scalars rows, cols");
            ok(lp.collapse == 2, UPIR_EINVAL, "JACOBI5 is a collapse(2) loop");
            if (ok.st) return ok.st;
            const double rows = lp.scalars[0], cols = lp.scalars[1];
            ok(is_int(rows) && is_int(cols) && rows >= 3 && cols >= 3 && rows < 2e9 && cols < 2e9,
               UPIR_EINVAL, "JACOBI5 grid must be at least 3 x 3");
            if (ok.st) return ok.st;
            const int64_t R = (int64_t)rows, C = (int64_t)cols;
            ok(lp.bufs[0] != lp.bufs[1], UPIR_EINVAL, "JACOBI5 needs distinct u_in and u_out");
            ok(buf_floats(0) >= R * C && buf_floats(1) >= R * C, UPIR_EINVAL, "JACOBI5 buffers smaller than the grid");
            ok(lp.step == 1 && (lp.trip == 0 || (lp.lb >= 1 && lp.ub <= R - 1)), UPIR_EINVAL,
               "JACOBI5 rows must be a unit-step range inside [1, rows-1)");
            ok(!has_i, UPIR_EINVAL, "JACOBI5 has no int64 terms");
            if (has_f) ok(rv.fterm == UPIR_TERM_RESID, UPIR_EINVAL, "JACOBI5 reductions take TERM_RESID");
            if (ok.st) return ok.st;
            const float* uin = static_cast<const float*>(lp.bufs[0]->dev);
            float* uout = static_cast<float*>(lp.bufs[1]->dev);
            const bool aligned = (reinterpret_cast<uintptr_t>(uin) & 15) == 0 &&
                                 (reinterpret_cast<uintptr_t>(uout) & 15) == 0 &&
                                 (!has_f || rv.fop == UPIR_RED_MAX || rv.fop == UPIR_RED_MIN);
            // widths that are not a multiple of 4: one copy per halo row from a
            // 1D view of the grid (its element indices must fit 32 bits, and
            // the view holds at least one box of up to 256 elements)
            const bool rows_tma = C % 4 != 0 && R * C < (1ll << 31) - 4096 && R * C >= 256;
            if (lp.variant == 0 && aligned && (C % 4 == 0 || rows_tma)) {
                lp.kind = LK_JACOBI_TMA;
                JacobiParams& jp = lp.jp;
                memset(&jp, 0, sizeof(jp));
                jp.rows_tma = rows_tma ? 1 : 0;
                // 2D boxes on a grid whose two buffers outgrow the L2 by more
                // than a quarter stream every sweep from HBM; there 64-column
                // tiles run faster (5120^2 .. 16384^2: 0.86-0.94 of HBM
                // against 0.82-0.88 with 128 columns), while at 4096^2, where
                // part of the pair stays in L2, 128 columns are faster (21.4
                // against 24.5 us per sweep)
                const bool beyond_l2 = !rows_tma && 2.0 * 4.0 * (double)R * (double)C > 1.25 * kL2Bytes;
                // while they fit it, the L2 is left to the output, which the
                // next sweep reads: input read evict-first, output stored with
                // normal priority (4096^2: 7 % less time per sweep; beyond the
                // L2, 6144^2 and 8192^2, the same policy runs 20-45 % slower)
                jp.keep_l2 = !rows_tma && !beyond_l2 ? 1 : 0;
                // 2D boxes: 64 x 128 tiles, three stages, two teams per SM;
                // teams of 256 units (eight rows per thread) while the grids
                // fit the L2 (4096^2 grid, 100 sweeps with alternating tile
                // order: 20.48 us per sweep; 512 units 20.74 us, 384 units
                // 20.43 us), 512 beyond it.  Row copies: two stages, teams of
                // 256 units on 40 x 128 tiles (4095^2 grid: 24.7 us per
                // sweep; 32 rows 25.0 us, 64 rows and 512 units 25.7 us,
                // three stages 27.9 us)
                if (!U0 && !auto_units) lp.units = (rows_tma || !beyond_l2) ? 256 : 512;
                lp.tile_m = lp.tile_m ? lp.tile_m : (rows_tma ? 40 : 64);
                lp.tile_n = lp.tile_n ? lp.tile_n : (beyond_l2 ? 64 : 128);
                lp.tile_n = (int)std::min<int64_t>(lp.tile_n, 4 * (int64_t)lp.units);
                jp.stages = lp.stages ? lp.stages : (rows_tma ? 2 : 3);
                while (jp.stages > 1 && jacobi_tma_smem_bytes(lp.tile_m, lp.tile_n, jp.stages, rows_tma) > 220 * 1024)
                    --jp.stages;
                lp.smem = jacobi_tma_smem_bytes(lp.tile_m, lp.tile_n, jp.stages, rows_tma);
                if (!ok(lp.smem <= 220 * 1024, UPIR_EINVAL, "Jacobi tile too large for shared memory"))
                    return ok.st;
                jp.uin = uin;
                jp.uout = uout;
                jp.rows = R;
                jp.cols = C;
                jp.r_lb = lp.lb;
                jp.r_ub = lp.lb + lp.trip;
                jp.tile_m = lp.tile_m;
                jp.tile_n = lp.tile_n;
                jp.tiles_r = ceil_div(lp.trip, lp.tile_m);
                jp.tiles_c = ceil_div(C, lp.tile_n);
                jp.ntiles = jp.tiles_r * jp.tiles_c;
                jp.chunk = lp.chunk;
                jp.sched = kernel_sched(lp.sched);
                jp.rvar = rv.fvar;
                jp.rop = rv.fop == UPIR_RED_MIN ? UPIR_RED_MIN : UPIR_RED_MAX;
                jp.spin_limit = ctx->spin_limit;
                jp.err_word = ctx->err_word;
                jp.wait_prior = wait_prior;
                if (lp.trip) {
                    upir_status st =
                        rows_tma ? encode_tmap_1d(ctx, &lp.tmap[0], uin, CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                                                  (uint64_t)(R * C), (uint32_t)(lp.tile_n + 8))
                                 : encode_tmap_2d(ctx, &lp.tmap[0], uin, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4,
                                                  (uint64_t)C, (uint64_t)R, (uint32_t)(lp.tile_n + 8),
                                                  (uint32_t)(lp.tile_m + 2), 0);
                    if (st != UPIR_OK) return st;
                }
                // persistent teams: as many as are resident at once, balanced so
                // every team gets the same number of tiles (to within one)
                const int per_sm =
                    std::max(1, jacobi_tma_max_teams_per_sm(lp.units, lp.tile_m, lp.tile_n, jp.stages, rows_tma,
                                                              jp.keep_l2 != 0));
                const int64_t slots = (int64_t)kNumSMs * per_sm;
                if (T0) lp.teams = T0;
                else if (lp.sched == UPIR_SCHED_STATIC && lp.chunk == 0) {
                    const int64_t per = std::max<int64_t>(1, ceil_div(jp.ntiles, slots));
                    lp.teams = (int)std::max<int64_t>(1, ceil_div(jp.ntiles, per));
                } else {
                    lp.teams = (int)std::max<int64_t>(1, std::min<int64_t>(dyn_estimate(lp, jp.ntiles), slots));
                }
                jp.sk = make_sched_const(jp.ntiles, lp.chunk, lp.teams);
                // a sweep over the previous sweep's output walks its tiles the
                // other way, so that it starts where that sweep ended, when a
                // good part of that sweep's data can still be in L2 (the two
                // grids within three L2s; 4096^2: 20.9 against 21.5 us per
                // sweep, 4095^2: 24.9 against 25.9 us, 6144^2: 52.7 against
                // 53.6 us; 8192^2: 92.0 against 91.5 us, so not there)
                const bool l2_reuse = 2.0 * 4.0 * (double)R * (double)C <= 3.0 * kL2Bytes;
                const bool blocked = lp.sched == UPIR_SCHED_STATIC && lp.chunk == 0;
                if (lp.tile_order == 0 && l2_reuse && blocked && !r->loops.empty()) {
                    const LoopRec& prev = *r->loops.back();
                    jp.reverse = prev.kind == LK_JACOBI_TMA && prev.jp.uout == uin && !prev.jp.reverse ? 1 : 0;
                }
                if (lp.tile_order == 2 && blocked) jp.reverse = 1;
                if (is_dyn(lp.sched)) {
                    build_chunk_table(lp, jp.ntiles, lp.teams);
                    upir_status st = alloc_scratch(ctx, lp, 0, 0, &jp.sc);
                    if (st != UPIR_OK) return st;
                }
                lp.skip = lp.trip == 0;
                return UPIR_OK;
            }
            // per-point variant (worker = unit, iteration = point)
            ep.uin = uin;
            ep.uout = uout;
            ep.rows = R;
            ep.cols = C;
            ep.trip = lp.trip * (C - 2);
            ep.step = 1;
            if (!lp.vec) lp.vec = 4;
            lp.trip = ep.trip;
            break;
        }
        case UPIR_BODY_JACOBI5_TB: {
            ok(lp.bufs.size() == 2, UPIR_EINVAL, "JACOBI5_TB takes bufs u_in, u_out");
            ok(lp.scalars.size() >= 3, UPIR_EINVAL, "JACOBI5_TB takes scalars rows, cols, sweeps");
            ok(lp.collapse == 2, UPIR_EINVAL, "JACOBI5_TB is a collapse(2) loop");
            if (ok.st) return ok.st;
            const double rows = lp.scalars[0], cols = lp.scalars[1], sw = lp.scalars[2];
            ok(is_int(rows) && is_int(cols) && rows >= 3 && cols >= 3 && rows < 2e9 && cols < 2e9,
               UPIR_EINVAL, "JACOBI5_TB grid must be at least 3 x 3");
            ok(is_int(sw) && sw >= 1 && sw <= 8, UPIR_EINVAL, "JACOBI5_TB sweeps must be an integer in [1, 8]");
            if (ok.st) return ok.st;
            const int64_t R = (int64_t)rows, C = (int64_t)cols;
            const int T = (int)sw;
            ok(lp.bufs[0] != lp.bufs[1], UPIR_EINVAL, "JACOBI5_TB needs distinct u_in and u_out");
            ok(buf_floats(0) >= R * C && buf_floats(1) >= R * C, UPIR_EINVAL,
               "JACOBI5_TB buffers smaller than the grid");
            ok(lp.step == 1 && (lp.trip == 0 || (lp.lb >= 1 && lp.ub <= R - 1)), UPIR_EINVAL,
               "JACOBI5_TB rows must be a unit-step range inside [1, rows-1)");
            ok(!has_i, UPIR_EINVAL, "JACOBI5_TB has no int64 terms");
            if (has_f) {
                ok(rv.fterm == UPIR_TERM_RESID, UPIR_EINVAL, "JACOBI5_TB reductions take TERM_RESID");
                ok(rv.fop == UPIR_RED_MAX || rv.fop == UPIR_RED_MIN, UPIR_EUNSUPPORTED,
                   "JACOBI5_TB reduces with max or min");
                const upir_reduction& red = lp.reds[0];
                ok((size_t)(red.index + T) * 4 <= red.var->bytes, UPIR_EINVAL,
                   "JACOBI5_TB needs `sweeps` reduction elements from the index on");
            }
            if (ok.st) return ok.st;
            const float* uin = static_cast<const float*>(lp.bufs[0]->dev);
            float* uout = static_cast<float*>(lp.bufs[1]->dev);
            ok(C % 4 == 0 && (reinterpret_cast<uintptr_t>(uin) & 15) == 0 &&
                   (reinterpret_cast<uintptr_t>(uout) & 15) == 0,
               UPIR_EUNSUPPORTED, "JACOBI5_TB needs cols % 4 == 0 and 16-byte aligned buffers");
            ok(U0 == 0 || (U0 % 32 == 0 && U0 <= kJacobiTBUnits), UPIR_EUNSUPPORTED,
               "JACOBI5_TB runs with num_units a multiple of 32 up to 1024 (or 0)");
            if (ok.st) return ok.st;
            lp.kind = LK_JACOBI_TB;
            lp.units = U0 ? U0 : kJacobiTBUnits;
            JacobiTBParams& tp = lp.tb;
            memset(&tp, 0, sizeof(tp));
            // halo: T rows; T columns rounded up to whole 16-byte groups (the
            // copy's first column must be 16-byte aligned)
            const int hc = (T + 3) / 4 * 4;
            // a box row is 32 groups of 4 columns, one per lane of a warp
            ok(lp.tile_n == 0 || lp.tile_n == 128 - 2 * hc, UPIR_EINVAL,
               "JACOBI5_TB tiles are 128 - 2 x column halo (4 or 8) columns wide");
            lp.tile_n = 128 - 2 * hc;
            // three planes (two copies in flight, one for the ping-pong)
            const int64_t plane_rows = (int64_t)(kStencilSmemBudget - 1024) / 3 / 4 / (lp.tile_n + 2 * hc);
            const int tm_max = (int)std::min<int64_t>(128, plane_rows - 2 * T) / 8 * 8;
            lp.tile_m = lp.tile_m ? lp.tile_m : tm_max;
            ok(lp.tile_m >= 1 && jacobi_tb_smem_bytes(lp.tile_m, lp.tile_n, T, hc) <= kStencilSmemBudget &&
                   lp.tile_m + 2 * T <= 256 && lp.tile_n + 2 * hc <= 256,
               UPIR_EINVAL, "JACOBI5_TB tile too large for shared memory");
            if (ok.st) return ok.st;
            lp.smem = jacobi_tb_smem_bytes(lp.tile_m, lp.tile_n, T, hc);
            tp.uin = uin;
            tp.uout = uout;
            tp.rows = R;
            tp.cols = C;
            tp.r_lb = lp.lb;
            tp.r_ub = lp.lb + lp.trip;
            tp.tile_m = lp.tile_m;
            tp.tile_n = lp.tile_n;
            tp.sweeps = T;
            tp.halo_c = hc;
            tp.tiles_r = ceil_div(lp.trip, lp.tile_m);
            tp.tiles_c = ceil_div(C, lp.tile_n);
            tp.ntiles = tp.tiles_r * tp.tiles_c;
            tp.chunk = lp.chunk;
            tp.sched = kernel_sched(lp.sched);
            tp.rvar = rv.fvar;
            tp.rop = rv.fop == UPIR_RED_MIN ? UPIR_RED_MIN : UPIR_RED_MAX;
            tp.spin_limit = ctx->spin_limit;
            tp.err_word = ctx->err_word;
            tp.wait_prior = wait_prior;
            if (lp.trip) {
                upir_status st = encode_tmap_2d(ctx, &lp.tmap[0], uin, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4,
                                                (uint64_t)C, (uint64_t)R, (uint32_t)(lp.tile_n + 2 * hc),
                                                (uint32_t)(lp.tile_m + 2 * T), 0);
                if (st != UPIR_OK) return st;
            }
            // one persistent team per SM, tiles balanced to within one
            if (T0) lp.teams = T0;
            else if (lp.sched == UPIR_SCHED_STATIC && lp.chunk == 0) {
                const int64_t per = std::max<int64_t>(1, ceil_div(tp.ntiles, kNumSMs));
                lp.teams = (int)std::max<int64_t>(1, ceil_div(tp.ntiles, per));
            } else {
                lp.teams = (int)std::max<int64_t>(1, std::min<int64_t>(dyn_estimate(lp, tp.ntiles), kNumSMs));
            }
            tp.sk = make_sched_const(tp.ntiles, lp.chunk, lp.teams);
            if (is_dyn(lp.sched)) {
                build_chunk_table(lp, tp.ntiles, lp.teams);
                upir_status st = alloc_scratch(ctx, lp, 0, 0, &tp.sc);
                if (st != UPIR_OK) return st;
            }
            lp.skip = lp.trip == 0;
            return UPIR_OK;
        }
        case UPIR_BODY_FILTER7: {
            ok(lp.bufs.size() == 2, UPIR_EINVAL, "FILTER7 takes bufs x_in, x_out");
            ok(lp.scalars.size() >= 51, UPIR_EINVAL, "FILTER7 takes scalars rows, cols and 49 weights");
            ok(lp.collapse == 2, UPIR_EINVAL, "FILTER7 is a collapse(2) loop");
            ok(!has_red, UPIR_EINVAL, "FILTER7 takes no reduction clause");
            if (ok.st) return ok.st;
            const double rows = lp.scalars[0], cols = lp.scalars[1];
            ok(is_int(rows) && is_int(cols) && rows >= 7 && cols >= 7 && rows < 2e9 && cols < 2e9,
               UPIR_EINVAL, "FILTER7 grid must be at least 7 x 7");
            if (ok.st) return ok.st;
            const int64_t R = (int64_t)rows, C = (int64_t)cols;
            ok(lp.bufs[0] != lp.bufs[1], UPIR_EINVAL, "FILTER7 needs distinct x_in and x_out");
            ok(buf_floats(0) >= R * C && buf_floats(1) >= R * C, UPIR_EINVAL, "FILTER7 buffers smaller than the grid");
            ok(lp.step == 1 && (lp.trip == 0 || (lp.lb >= 3 && lp.ub <= R - 3)), UPIR_EINVAL,
               "FILTER7 rows must be a unit-step range inside [3, rows-3)");
            const float* xin = static_cast<const float*>(lp.bufs[0]->dev);
            float* xout = static_cast<float*>(lp.bufs[1]->dev);
            ok(C % 4 == 0 && (reinterpret_cast<uintptr_t>(xin) & 15) == 0 &&
                   (reinterpret_cast<uintptr_t>(xout) & 15) == 0,
               UPIR_EUNSUPPORTED, "FILTER7 needs cols % 4 == 0 and 16-byte aligned buffers");
            ok(U0 == 0 || U0 == kFilter7Units, UPIR_EUNSUPPORTED, "FILTER7 runs with num_units 256 (or 0)");
            if (ok.st) return ok.st;
            lp.kind = LK_FILTER7;
            lp.units = kFilter7Units;
            Filter7Params& fp = lp.fp;
            memset(&fp, 0, sizeof(fp));
            lp.tile_m = lp.tile_m ? lp.tile_m : 32;
            lp.tile_n = lp.tile_n ? lp.tile_n : 128;
            ok(lp.tile_n / 4 <= kFilter7Units && kFilter7Units % (lp.tile_n / 4) == 0, UPIR_EINVAL,
               "FILTER7 tile_n / 4 must divide 256");
            // Two output rows per paired FMA (fma.rn.f32x2) with strips of 4
            // output rows per thread by default (4096^2: 36.8-37.3 us against
            // 39.6-40.7 us with one FMA per output; a third fewer
            // instructions, the FMA pipe then the busiest unit).  VARIANT 1:
            // paired, 8-row strips; 2: one FMA per output, 4-row strips; 3:
            // one FMA per output, 8-row strips.  STAGES: TMA ring depth 2
            // (default) or 3; either takes one team barrier per tile
            const int f7_rs = (lp.variant == 1 || lp.variant == 3) ? 8 : 4;
            const int f7_pair = lp.variant <= 1 ? 1 : 0;
            const int f7_stages = lp.stages ? lp.stages : kFilter7Stages;
            ok(f7_stages == 2 || f7_stages == 3, UPIR_EINVAL, "FILTER7 stages must be 2 or 3");
            ok(lp.tile_m % f7_rs == 0, UPIR_EINVAL, "FILTER7 tile_m must be a multiple of the strip rows (4; variants 1 and 3: 8)");
            ok(lp.tile_m + 6 <= 256 && lp.tile_n + 8 <= 256 &&
                   filter7_smem_bytes(lp.tile_m, lp.tile_n, f7_stages) <= kStencilSmemBudget,
               UPIR_EINVAL, "FILTER7 tile too large");
            if (ok.st) return ok.st;
            lp.smem = filter7_smem_bytes(lp.tile_m, lp.tile_n, f7_stages);
            fp.stages = f7_stages;
            fp.rs = f7_rs;
            fp.pair = f7_pair;
            fp.xin = xin;
            fp.xout = xout;
            fp.rows = R;
            fp.cols = C;
            fp.r_lb = lp.lb;
            fp.r_ub = lp.lb + lp.trip;
            fp.tile_m = lp.tile_m;
            fp.tile_n = lp.tile_n;
            fp.tiles_r = ceil_div(lp.trip, lp.tile_m);
            fp.tiles_c = ceil_div(C, lp.tile_n);
            fp.ntiles = fp.tiles_r * fp.tiles_c;
            fp.chunk = lp.chunk;
            fp.sched = kernel_sched(lp.sched);
            fp.spin_limit = ctx->spin_limit;
            fp.err_word = ctx->err_word;
            fp.wait_prior = wait_prior;
            for (int k = 0; k < 49; ++k) fp.w[k] = (float)lp.scalars[2 + k];
            for (int k = 0; k < 42; ++k) {
                uint32_t lo, hi;
                memcpy(&lo, &fp.w[k + 7], 4);  // w[i][j], i = k / 7 + 1
                memcpy(&hi, &fp.w[k], 4);      // w[i - 1][j]
                fp.w2[k] = (unsigned long long)hi << 32 | lo;
            }
            if (lp.trip) {
                upir_status st = encode_tmap_2d(ctx, &lp.tmap[0], xin, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4,
                                                (uint64_t)C, (uint64_t)R, (uint32_t)(lp.tile_n + 8),
                                                (uint32_t)(lp.tile_m + 6), 0);
                if (st != UPIR_OK) return st;
            }
            const int per_sm = std::max(1, filter7_max_teams_per_sm(lp.tile_m, lp.tile_n, f7_stages, f7_rs, f7_pair));
            const int64_t slots = (int64_t)kNumSMs * per_sm;
            if (T0) lp.teams = T0;
            else if (lp.sched == UPIR_SCHED_STATIC && lp.chunk == 0) {
                const int64_t per = std::max<int64_t>(1, ceil_div(fp.ntiles, slots));
                lp.teams = (int)std::max<int64_t>(1, ceil_div(fp.ntiles, per));
            } else {
                lp.teams = (int)std::max<int64_t>(1, std::min<int64_t>(dyn_estimate(lp, fp.ntiles), slots));
            }
            fp.sk = make_sched_const(fp.ntiles, lp.chunk, lp.teams);
            if (is_dyn(lp.sched)) {
                build_chunk_table(lp, fp.ntiles, lp.teams);
                upir_status st = alloc_scratch(ctx, lp, 0, 0, &fp.sc);
                if (st != UPIR_OK) return st;
            }
            lp.skip = lp.trip == 0;
            return UPIR_OK;
        }
        case UPIR_BODY_MATVEC: {
            ok(lp.bufs.size() == 3, UPIR_EINVAL, "MATVEC takes bufs A, x, y");
            ok(lp.scalars.size() >= 2, UPIR_EINVAL, "MATVEC takes scalars rows, cols");
            ok(!has_red, UPIR_EINVAL, "MATVEC takes no reduction clause");
            ok(lp.collapse == 1, UPIR_EINVAL, "MATVEC is a collapse(1) loop over rows");
            if (ok.st) return ok.st;
            const double rows = lp.scalars[0], cols = lp.scalars[1];
            ok(is_int(rows) && is_int(cols) && rows >= 0 && cols >= 0, UPIR_EINVAL, "bad matvec shape");
            if (ok.st) return ok.st;
            const int64_t R = (int64_t)rows, C = (int64_t)cols;
            ok(buf_floats(0) >= R * C && buf_floats(1) >= C && buf_floats(2) >= R, UPIR_EINVAL,
               "MATVEC buffers smaller than the shape");
            if (lp.trip) ok(min_iv >= 0 && max_iv < R, UPIR_EINVAL, "MATVEC rows outside [0, rows)");
            ok(lp.units % 32 == 0, UPIR_EINVAL, "MATVEC needs num_units a multiple of 32 (worker = warp)");
            if (ok.st) return ok.st;
            lp.kind = LK_MATVEC;
            MatvecParams& mp = lp.mp;
            memset(&mp, 0, sizeof(mp));
            mp.A = static_cast<const float*>(lp.bufs[0]->dev);
            mp.x = static_cast<const float*>(lp.bufs[1]->dev);
            mp.y = static_cast<float*>(lp.bufs[2]->dev);
            mp.rows = R;
            mp.cols = C;
            mp.lb = lp.lb;
            mp.step = lp.step;
            mp.trip = lp.trip;
            mp.chunk = lp.chunk;
            mp.sched = kernel_sched(lp.sched);
            const int64_t wpb = lp.units / 32;
            // the warps that fit at once (the kernel's registers, not the
            // thread limit, bound them): a static plan gives each the same
            // number of rows and launches no second wave
            const int64_t resident_warps = (int64_t)kNumSMs * matvec_max_teams_per_sm(lp.units) * wpb;
            if (T0) lp.teams = T0;
            else if (lp.sched == UPIR_SCHED_STATIC && lp.chunk == 0) {
                const int64_t per = std::max<int64_t>(1, ceil_div(lp.trip, resident_warps));
                lp.teams = (int)std::max<int64_t>(1, ceil_div(ceil_div(lp.trip, per), wpb));
            } else {
                lp.teams = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(dyn_estimate(lp, lp.trip), wpb),
                                                                       resident_warps / wpb));
            }
            mp.sk = make_sched_const(lp.trip, lp.chunk, (int64_t)lp.teams * wpb);
            mp.wait_prior = wait_prior;
            if (is_dyn(lp.sched)) {
                build_chunk_table(lp, lp.trip, (int64_t)lp.teams * wpb);
                upir_status st = alloc_scratch(ctx, lp, 0, 0, &mp.sc);
                if (st != UPIR_OK) return st;
            }
            lp.skip = lp.trip == 0;
            return UPIR_OK;
        }
        case UPIR_BODY_GEMM_F32:
        case UPIR_BODY_GEMM_BF16:
        case UPIR_BODY_GEMM_BF16X3: {
            const bool tc = lp.body != UPIR_BODY_GEMM_F32;
            const size_t nb = lp.body == UPIR_BODY_GEMM_BF16X3 ? 5 : 3;
            ok(lp.bufs.size() == nb, UPIR_EINVAL, "GEMM buffer count (F32: A B C; BF16: A Bt C; BF16X3: Ah Al Bth Btl C)");
            ok(lp.scalars.size() >= 3, UPIR_EINVAL, "GEMM takes scalars M, N, K");
            ok(!has_red, UPIR_EINVAL, "GEMM takes no reduction clause");
            ok(lp.collapse == 2, UPIR_EINVAL, "GEMM is a collapse(2) loop");
            if (ok.st) return ok.st;
            const double Md = lp.scalars[0], Nd = lp.scalars[1], Kd = lp.scalars[2];
            ok(is_int(Md) && is_int(Nd) && is_int(Kd) && Md >= 0 && Nd >= 0 && Kd >= 0 && Md < 2e9 && Nd < 2e9 && Kd < 2e9,
               UPIR_EINVAL, "bad GEMM shape");
            if (ok.st) return ok.st;
            const int64_t M = (int64_t)Md, N = (int64_t)Nd, K = (int64_t)Kd;
            ok(lp.step == 1 && (lp.trip == 0 || (lp.lb >= 0 && lp.ub <= M)), UPIR_EINVAL,
               "GEMM rows must be a unit-step range inside [0, M)");
            if (ok.st) return ok.st;
            if (!tc) {
                ok((int64_t)(lp.bufs[0]->bytes / 4) >= M * K && (int64_t)(lp.bufs[1]->bytes / 4) >= K * N &&
                   (int64_t)(lp.bufs[2]->bytes / 4) >= M * N, UPIR_EINVAL, "GEMM buffers smaller than the shape");
                ok(lp.units == 256, UPIR_EUNSUPPORTED, "GEMM_F32 runs with num_units 256");
                if (ok.st) return ok.st;
                lp.kind = LK_GEMM_F32;
                GemmParams& gp = lp.gp;
                memset(&gp, 0, sizeof(gp));
                gp.A = static_cast<const float*>(lp.bufs[0]->dev);
                gp.B = static_cast<const float*>(lp.bufs[1]->dev);
                gp.C = static_cast<float*>(lp.bufs[2]->dev);
                gp.M = M;
                gp.N = N;
                gp.K = K;
                gp.row_lb = lp.lb;
                gp.row_ub = lp.lb + lp.trip;
                gp.chunk = lp.chunk;
                gp.sched = kernel_sched(lp.sched);
                const int64_t ntiles = ceil_div(lp.trip, 128) * ceil_div(N, 128);
                gp.whole = ntiles;
                gp.kparts = 1;
                if (T0) lp.teams = T0;
                else if (lp.sched == UPIR_SCHED_STATIC && lp.chunk == 0) {
                    // one tile per team; when the last wave of resident teams
                    // (two per SM) would be at most half full, its tiles are
                    // split in k over the idle slots, each share at least 8 k tiles
                    const int64_t slots = 2 * kNumSMs, rem = ntiles % slots;
                    const int64_t q = rem ? std::min<int64_t>(std::min<int64_t>(slots / rem, 4), ceil_div(K, 16) / 8) : 1;
                    if (ntiles > slots && q >= 2) {
                        gp.whole = ntiles - rem;
                        gp.kparts = (int)q;
                        upir_status st = alloc_scratch(ctx, lp, rem, rem * q * 128 * 128 / 4, &gp.sc);
                        if (st != UPIR_OK) return st;
                        gp.tile_tickets = gp.sc.group_tickets;
                        gp.work = reinterpret_cast<float*>(gp.sc.partials);
                    }
                    lp.teams = (int)std::max<int64_t>(1, std::min<int64_t>(gp.whole + (ntiles - gp.whole) * gp.kparts,
                                                                           0x7fffffff));
                } else
                    lp.teams = (int)std::max<int64_t>(1, std::min<int64_t>(dyn_estimate(lp, ntiles), kNumSMs * 2));
                gp.sk = make_sched_const(ntiles, lp.chunk, lp.teams);
                if (is_dyn(lp.sched)) {
                    build_chunk_table(lp, ntiles, lp.teams);
                    upir_status st = alloc_scratch(ctx, lp, 0, 0, &gp.sc);
                    if (st != UPIR_OK) return st;
                }
                // TMA boxes need rows of A and B (and C's float4 stores) that
                // start on 16-byte boundaries; VARIANT 1 keeps the register-
                // staged kernel
                const auto al16 = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15) == 0; };
                lp.gemm_tma = lp.variant != 1 && lp.trip > 0 && N > 0 && K > 0 && K % 4 == 0 && N % 4 == 0 &&
                              al16(gp.A) && al16(gp.B) && al16(gp.C);
                if (lp.gemm_tma) {
                    gp.spin_limit = ctx->spin_limit;
                    gp.err_word = ctx->err_word;
                    upir_status st = encode_tmap_2d(ctx, &lp.tmap[0], gp.A, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4,
                                                    (uint64_t)K, (uint64_t)M, 16, 128, 0);
                    if (st == UPIR_OK)
                        st = encode_tmap_2d(ctx, &lp.tmap[1], gp.B, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4,
                                            (uint64_t)N, (uint64_t)K, 128, 16, 0);
                    if (st != UPIR_OK) return st;
                }
                lp.skip = lp.trip == 0 || N == 0;
                return UPIR_OK;
            }
            return plan_gemm_tc(r, lp, M, N, K, ok.st);
        }
        case UPIR_BODY_SPLIT_BF16: {
            ok(lp.bufs.size() == 3, UPIR_EINVAL, "SPLIT_BF16 takes bufs src, hi, lo");
            ok(lp.scalars.size() >= 3, UPIR_EINVAL, "SPLIT_BF16 takes scalars rows, cols, transpose");
            ok(!has_red, UPIR_EINVAL, "SPLIT_BF16 takes no reduction clause");
            if (ok.st) return ok.st;
            const double rows = lp.scalars[0], cols = lp.scalars[1];
            ok(is_int(rows) && is_int(cols) && rows >= 0 && cols >= 0, UPIR_EINVAL, "bad split shape");
            if (ok.st) return ok.st;
            const int64_t R = (int64_t)rows, C = (int64_t)cols;
            ok(buf_floats(0) >= R * C && (int64_t)(lp.bufs[1]->bytes / 2) >= R * C &&
               (int64_t)(lp.bufs[2]->bytes / 2) >= R * C, UPIR_EINVAL, "SPLIT_BF16 buffers smaller than the shape");
            ok(lp.step == 1 && (lp.trip == 0 || (lp.lb >= 0 && lp.ub <= R)), UPIR_EINVAL,
               "SPLIT_BF16 rows must be a unit-step range inside [0, rows)");
            ok(lp.units == 256, UPIR_EUNSUPPORTED, "SPLIT_BF16 runs with num_units 256");
            if (ok.st) return ok.st;
            lp.kind = LK_SPLIT;
            SplitParams& sp = lp.sp;
            sp.src = static_cast<const float*>(lp.bufs[0]->dev);
            sp.hi = static_cast<uint16_t*>(lp.bufs[1]->dev);
            sp.lo = static_cast<uint16_t*>(lp.bufs[2]->dev);
            sp.rows = R;
            sp.cols = C;
            sp.lb = lp.lb;
            sp.ub = lp.lb + lp.trip;
            sp.transpose = lp.scalars[2] != 0.0;
            const int64_t ntiles = ceil_div(lp.trip, 32) * ceil_div(C, 32);
            lp.teams = T0 ? T0 : (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, kNumSMs * 8));
            lp.skip = lp.trip == 0 || C == 0;
            return UPIR_OK;
        }
        default:
            return fail(ctx, UPIR_EINVAL, "upir_loop: unknown body");
    }
    if (ok.st) return ok.st;

    // element engine geometry and scratch
    ep.imod_mul = imod_mul;
    ep.imod_mod = imod_mod;
    ep.imod_inc = imod_inc;
    ep.imod_minv = imod_mod >= 2 ? (unsigned long long)(((unsigned __int128)1 << 64) / (unsigned long long)imod_mod) : 0;
    ep.imod32 = imod_mod < (1ll << 28) ? 1 : 0;
    const int64_t trip = lp.trip;
    // iterations per worker the blocked schedule aims for.  Without
    // reductions: 4 (one 128-bit access), 8 once every SM's thread slots stay
    // busy at 8 per worker.  With reductions: 8 (one 256-bit access), 16 once
    // the slots stay busy at 16 (the reduction tree and the range set-up
    // amortised over twice the iterations).  Longer ranges spread a warp's
    // accesses over more DRAM pages: measured on 2^28 iterations, 32 per
    // worker ran 30 % slower than 16.
    const int64_t slots = (int64_t)kNumSMs * 2048;
    const int64_t vdef = !has_red ? (trip >= 8 * slots ? 8 : 4) : (trip >= 16 * slots ? 16 : 8);
    // reducing element loops run better in smaller teams (more, shorter-lived
    // blocks overlap their block-level reduction trees with other blocks' loads)
    if (!U0 && !auto_units && has_red && lp.body == UPIR_BODY_AXPY) lp.units = 128;
    const int U = lp.units;
    // per-point Jacobi: 4 consecutive points per worker (one division per range;
    // on a 4095^2 grid 4 points take 93 us per sweep, 8 points 115 us, 16 points 214 us)
    const int64_t V = (lp.body == UPIR_BODY_AXPY && lp.step == 1) ? (lp.vec ? lp.vec : vdef)
                      : lp.body == UPIR_BODY_IMOD ? vdef : lp.body == UPIR_BODY_JACOBI5 ? lp.vec : 1;
    if (lp.sched == UPIR_SCHED_STATIC) {
        if (T0) lp.teams = T0;
        else if (lp.chunk == 0) lp.teams = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(trip, U * V), 0x7fffffff));
        else lp.teams = default_teams_for_chunks(ceil_div(trip, lp.chunk), U);
        ep.sk = make_sched_const(trip, lp.chunk, (int64_t)lp.teams * U);
        if (has_red) {
            upir_status st = alloc_scratch(ctx, lp, finalize_groups(lp.teams), lp.teams, &ep.sc);
            if (st != UPIR_OK) return st;
        }
    } else {
        // dynamic, guided or taskloop: chunks claimed from a counter
        const int64_t est = dyn_estimate(lp, trip);
        if (has_red && !ok(est <= (1ll << 27), UPIR_EUNSUPPORTED,
                           "dynamic reductions need at most 2^27 chunks (raise the chunk)"))
            return ok.st;
        lp.teams = T0 ? T0 : default_teams_for_chunks(est, U);
        ep.nchunks = build_chunk_table(lp, trip, (int64_t)lp.teams * U);
        const int64_t nslots = has_red ? ep.nchunks : 0;
        upir_status st = alloc_scratch(ctx, lp, finalize_groups(nslots), nslots, &ep.sc);
        if (st != UPIR_OK) return st;
    }
    lp.skip = trip == 0;
    return UPIR_OK;
}

cudaError_t launch_loop(upir_ctx ctx, LoopRec& lp, cudaStream_t s) {
    switch (lp.kind) {
        case LK_ELEM:
            return launch_elem(lp.body, is_dyn(lp.sched), lp.ep.rv.fvar ? lp.ep.rv.fop : 0,
                               lp.ep.rv.ivar ? lp.ep.rv.iop : 0, lp.teams, lp.units, lp.ep, s);
        case LK_JACOBI_TMA: return launch_jacobi_tma(lp.teams, lp.units, lp.jp, &lp.tmap[0], s);
        case LK_MATVEC: return launch_matvec(lp.teams, lp.units, lp.mp, s);
        case LK_GEMM_F32:
            return lp.gemm_tma ? launch_gemm_f32_tma(lp.teams, lp.gp, &lp.tmap[0], s)
                               : launch_gemm_f32(lp.teams, lp.units, lp.gp, s);
        case LK_SPLIT: return launch_split_bf16(lp.teams, lp.units, lp.sp, s);
        case LK_GEMM_TC: return launch_gemm_tc_loop(ctx, lp, s);
        case LK_JACOBI_TB: return launch_jacobi_tb(lp.teams, lp.units, lp.tb, &lp.tmap[0], s);
        case LK_FILTER7: return launch_filter7(lp.teams, lp.fp, &lp.tmap[0], s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace upir
