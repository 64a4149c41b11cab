// schedule(auto) (§3.2 lists auto among the schedule policies; the paper's IR
// keeps several parallelization options so that "the compiler or the runtime
// [can] choose the most performant one"): the runtime scores candidate
// schedules with the learned cost model and takes the one it predicts
// fastest.  Host code only; it runs when a loop is recorded.
//
// The candidate lists and the 12 features are the ones the cost model is
// trained on (paper_2209_10643_b300/costmodel.py takes both from here).
#include <cmath>
#include <cstring>
#include <vector>

#include "runtime_internal.h"

namespace upir {

namespace {

constexpr int NI = UPIR_MLP_IN, NH = UPIR_MLP_HIDDEN;
constexpr int OFF_B1 = NH * NI, OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + NH * NH, OFF_W3 = OFF_B2 + NH,
              OFF_B3 = OFF_W3 + NH;

enum { OP_AXPY = 0, OP_JACOBI = 1, OP_MATVEC = 2, OP_GEMM = 3 };

int body_op(int body) {
    switch (body) {
        case UPIR_BODY_AXPY: return OP_AXPY;
        case UPIR_BODY_JACOBI5: return OP_JACOBI;
        case UPIR_BODY_MATVEC: return OP_MATVEC;
        case UPIR_BODY_GEMM_F32: return OP_GEMM;
        default: return -1;
    }
}

struct Cand {
    int sched;
    int64_t chunk;
    int units;
};

std::vector<Cand> candidate_list(int op) {
    std::vector<Cand> c;
    if (op == OP_AXPY) {
        for (int u : {128, 256, 512, 1024}) {
            for (int64_t ch : {0, 4, 64, 1024}) c.push_back({UPIR_SCHED_STATIC, ch, u});
            for (int64_t ch : {256, 4096, 65536}) c.push_back({UPIR_SCHED_DYNAMIC, ch, u});
        }
    } else if (op == OP_JACOBI) {
        for (int u : {128, 256, 512}) {
            for (int64_t ch : {0, 1, 4}) c.push_back({UPIR_SCHED_STATIC, ch, u});
            for (int64_t ch : {1, 4}) c.push_back({UPIR_SCHED_DYNAMIC, ch, u});
        }
    } else if (op == OP_MATVEC) {
        for (int u : {128, 256, 512, 1024}) {
            for (int64_t ch : {0, 1, 8}) c.push_back({UPIR_SCHED_STATIC, ch, u});
            for (int64_t ch : {1, 8}) c.push_back({UPIR_SCHED_DYNAMIC, ch, u});
        }
    } else if (op == OP_GEMM) {
        // the FP32 tile kernel runs 256-unit teams; the choice is how the
        // 128 x 128 output tiles are shared out (chunk 0: one tile per team,
        // the last wave's tiles split in k)
        for (int64_t ch : {0, 1, 2, 8}) c.push_back({UPIR_SCHED_STATIC, ch, 256});
        for (int64_t ch : {1, 2}) c.push_back({UPIR_SCHED_DYNAMIC, ch, 256});
    }
    return c;
}

// Feature vector of one candidate.  trip counts iterations (JACOBI5:
// interior points of the loop's rows; GEMM_F32: output elements); cols is
// the grid or matrix width (GEMM_F32: the contraction length K).  Bytes per
// iteration of the GEMM: the 128 x 128 tile kernel reads 2 x 128 x K operand
// floats per tile of 128^2 outputs, K / 16 bytes per output.
void features(int op, int64_t trip, int64_t cols, int sched, int64_t chunk, int units, int teams, float* f) {
    for (int i = 0; i < NI; ++i) f[i] = 0.0f;
    f[op] = 1.0f;
    f[4] = (float)std::log2((double)std::max<int64_t>(trip, 1));
    if (op == OP_AXPY) f[5] = 12.0f, f[6] = 4.0f;
    else if (op == OP_JACOBI) f[5] = 8.0f, f[6] = 6.0f;
    else if (op == OP_GEMM) f[5] = (float)cols / 16.0f, f[6] = 2.0f * (float)cols;
    else f[5] = 4.0f * (float)cols, f[6] = 2.0f * (float)cols;
    f[7 + (sched == UPIR_SCHED_DYNAMIC ? 1 : 0)] = 1.0f;
    f[9] = (float)std::log2((double)chunk + 1.0);
    f[10] = (float)std::log2((double)std::max(units, 1));
    f[11] = (float)std::log2((double)std::max(teams, 1));
}

float bf16r(float v) {  // round to nearest even bfloat16
    uint32_t b;
    std::memcpy(&b, &v, 4);
    b += 0x7fffu + ((b >> 16) & 1u);
    b &= 0xffff0000u;
    float r;
    std::memcpy(&r, &b, 4);
    return r;
}

// The MLP on one standardised input, bfloat16-rounded weights, FP32 sums.
float mlp_predict(const float* p, const float* x) {
    float h1[NH], h2[NH];
    for (int j = 0; j < NH; ++j) {
        float z = p[OFF_B1 + j];
        for (int i = 0; i < NI; ++i) z = std::fmaf(bf16r(p[j * NI + i]), x[i], z);
        h1[j] = z > 0.0f ? z : 0.0f;
    }
    for (int j = 0; j < NH; ++j) {
        float z = p[OFF_B2 + j];
        for (int k = 0; k < NH; ++k) z = std::fmaf(bf16r(p[OFF_W2 + j * NH + k]), h1[k], z);
        h2[j] = z > 0.0f ? z : 0.0f;
    }
    float y = p[OFF_B3];
    for (int j = 0; j < NH; ++j) y = std::fmaf(bf16r(p[OFF_W3 + j]), h2[j], y);
    return y;
}

int64_t loop_trip(int op, int64_t trip, int64_t cols) {
    return op == OP_JACOBI ? trip * std::max<int64_t>(cols - 2, 0) : trip;
}

}  // namespace

// The cost model's pick for a loop; `units` fixed by the region (0: free).
// teams_of(candidate) gives the teams feature of a candidate (the teams the
// planner launches it with), or < 0 for a candidate that cannot run the loop.
// Bodies without candidates take STATIC with chunk 0.
template <class TeamsOf>
void auto_pick(const float* params, const float* mean, const float* sdev, int body, int64_t trip, int64_t cols,
               int units, TeamsOf teams_of, int* sched, int64_t* chunk, int* units_out) {
    *sched = UPIR_SCHED_STATIC;
    *chunk = 0;
    *units_out = 0;
    const int op = body_op(body);
    if (!params || op < 0) return;
    std::vector<Cand> cands = candidate_list(op);
    float best = 0.0f;
    bool have = false;
    for (const Cand& c : cands) {
        if (units && c.units != units) continue;
        const int teams = teams_of(c);
        if (teams < 0) continue;
        float f[NI];
        features(op, loop_trip(op, trip, cols), cols, c.sched, c.chunk, c.units, teams, f);
        for (int i = 0; i < NI; ++i) {
            const float sd = sdev && sdev[i] > 0.0f ? sdev[i] : 1.0f;
            f[i] = (f[i] - (mean ? mean[i] : 0.0f)) / sd;
        }
        const float y = mlp_predict(params, f);
        if (!have || y < best) {
            best = y;
            have = true;
            *sched = c.sched;
            *chunk = c.chunk;
            *units_out = units ? 0 : c.units;
        }
    }
}

// The teams the planner launches a loop with under one candidate schedule:
// the loop is planned on a scratch region with the candidate's schedule,
// chunk and units and no device scratch; -1 when the candidate cannot run it.
// The context's last error message is left as it was.
int planned_teams(upir_region r, const upir_loop_desc* d, const Cand& c) {
    upir_ctx ctx = r->ctx;
    const std::string saved = ctx->err;
    upir_region_s tmp;
    tmp.ctx = ctx;
    tmp.teams = r->teams;
    tmp.units = r->units ? r->units : c.units;
    upir_loop_desc dd = *d;
    dd.sched = c.sched;
    dd.chunk = c.chunk;
    LoopRec lp;
    lp.dry = true;
    const upir_status st = plan_loop(&tmp, &dd, lp);
    ctx->err = saved;
    return st == UPIR_OK ? lp.teams : -1;
}

void auto_schedule(upir_ctx ctx, upir_region r, const upir_loop_desc* d, int64_t trip, int* sched, int64_t* chunk,
                   int* units_out) {
    int64_t cols = d->nscalars >= 2 && d->scalars ? (int64_t)d->scalars[1] : 0;
    if (d->body == UPIR_BODY_GEMM_F32) {
        // output elements of the loop's rows, and K
        const int64_t n = cols, k = d->nscalars >= 3 ? (int64_t)d->scalars[2] : 0;
        trip = trip * std::max<int64_t>(n, 0);
        cols = k;
    }
    if (ctx->cm_params.empty()) {
        *sched = UPIR_SCHED_STATIC;
        *chunk = 0;
        *units_out = 0;
        return;
    }
    auto_pick(ctx->cm_params.data(), ctx->cm_mean.data(), ctx->cm_std.data(), d->body, trip, cols, r->units,
              [&](const Cand& c) { return planned_teams(r, d, c); }, sched, chunk, units_out);
}

}  // namespace upir

using namespace upir;

extern "C" upir_status upir_ctx_set_cost_model(upir_ctx ctx, const float* params, const float* feat_mean,
                                               const float* feat_std) {
    if (!ctx) return UPIR_EINVAL;
    if (!params) {
        ctx->cm_params.clear();
        ctx->cm_mean.clear();
        ctx->cm_std.clear();
        return UPIR_OK;
    }
    if (!feat_mean || !feat_std) return fail(ctx, UPIR_EINVAL, "upir_ctx_set_cost_model: feature statistics missing");
    ctx->cm_params.assign(params, params + UPIR_MLP_NPARAM);
    ctx->cm_mean.assign(feat_mean, feat_mean + NI);
    ctx->cm_std.assign(feat_std, feat_std + NI);
    return UPIR_OK;
}

extern "C" upir_status upir_auto_candidates(int32_t body, int32_t* sched, int64_t* chunk, int32_t* units,
                                            int32_t cap, int32_t* count) {
    if (!count || cap < 0) return UPIR_EINVAL;
    const int op = body_op(body);
    const std::vector<Cand> c = op < 0 ? std::vector<Cand>() : candidate_list(op);
    *count = (int32_t)c.size();
    for (int32_t i = 0; i < (int32_t)c.size() && i < cap; ++i) {
        if (sched) sched[i] = c[i].sched;
        if (chunk) chunk[i] = c[i].chunk;
        if (units) units[i] = c[i].units;
    }
    return UPIR_OK;
}

extern "C" upir_status upir_auto_features(int32_t body, int64_t trip, int64_t cols, int32_t sched, int64_t chunk,
                                          int32_t units, int32_t teams, float* out) {
    const int op = body_op(body);
    if (op < 0 || !out || trip < 0 || chunk < 0) return UPIR_EINVAL;
    features(op, loop_trip(op, trip, cols), cols, sched, chunk, units, teams, out);
    return UPIR_OK;
}

extern "C" upir_status upir_auto_pick(const float* params, const float* feat_mean, const float* feat_std,
                                      int32_t body, int64_t trip, int64_t cols, int32_t units, int32_t teams,
                                      int32_t* sched, int64_t* chunk, int32_t* units_out) {
    if (!sched || !chunk || !units_out || trip < 0) return UPIR_EINVAL;
    int s = 0, u = 0;
    int64_t c = 0;
    auto_pick(params, feat_mean, feat_std, body, trip, cols, units, [teams](const Cand&) { return teams; }, &s, &c,
              &u);
    *sched = s;
    *chunk = c;
    *units_out = u;
    return UPIR_OK;
}
