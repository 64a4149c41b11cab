// Host-side runtime objects behind the opaque C ABI handles.
#pragma once

#include <algorithm>
#include <string>
#include <unordered_set>
#include <memory>
#include <vector>

#include "upir_internal.h"

struct upir_buf_s {
    upir_ctx ctx = nullptr;
    void* host = nullptr;
    void* dev = nullptr;
    size_t bytes = 0;
    int kind = UPIR_MAP_TO;
    bool wrapped = false;  // caller-owned device memory
    bool live = true;
    int refs = 0;          // loops of live regions that use this buffer
    cudaEvent_t ready = nullptr;  // end of the last asynchronous copy
    bool pending = false;         // the compute stream has not waited for it yet
    int64_t last_use = 0;         // the compute-stream submission that last used it (0: none)
};

struct upir_event_s {
    cudaEvent_t ev = nullptr;
};

namespace upir {

enum LaunchKind {
    LK_ELEM = 0, LK_JACOBI_TMA = 1, LK_MATVEC = 2, LK_GEMM_F32 = 3, LK_SPLIT = 4, LK_GEMM_TC = 5,
    LK_JACOBI_TB = 6, LK_FILTER7 = 7
};

// A recorded, validated and planned loop.
struct LoopRec {
    int64_t lb = 0, ub = 0, step = 1, chunk = 0, trip = 0;
    int collapse = 1, sched = 0, body = 0, nowait = 0;
    std::vector<upir_buf> bufs;
    std::vector<double> scalars;
    std::vector<upir_reduction> reds;
    int variant = 0, tile_m = 0, tile_n = 0, vec = 0, stages = 0;  // 0: planner default
    int tile_order = 0;  // UPIR_HINT_TILE_ORDER
    bool gemm_tma = false;  // GEMM_F32: the TMA-fed kernel (maps in tmap[0], tmap[1])
    int64_t grainsize = 0, num_tasks = 0;  // taskloop hints
    // guided / taskloop chunk starts (host copy; the device copy is in scratch)
    std::vector<int64_t> chunk_table;
    int64_t nchunks = 0;  // chunks or tasks handed out dynamically (0: static)
    int teams = 0, units = 0;
    int kind = LK_ELEM;
    bool skip = false;       // zero-trip loop: nothing to launch
    bool holds_refs = false;
    bool dry = false;        // planning only (schedule(auto) scoring): no device scratch
    void* scratch = nullptr;
    size_t scratch_bytes = 0;
    // Scratch bytes [counter_off, counter_off + counter_bytes) hold counters
    // and tickets that each launch returns to zero itself; a launch that gave
    // up on a bounded wait may leave them set, so they are cleared again when
    // the context reports the timeout.
    size_t counter_off = 0, counter_bytes = 0;
    size_t smem = 0;
    ElemParams ep{};
    JacobiParams jp{};
    JacobiTBParams tb{};
    Filter7Params fp{};
    MatvecParams mp{};
    GemmParams gp{};
    SplitParams sp{};
    CUtensorMap tmap[6];  // the type carries the alignment TMA needs
    alignas(16) unsigned char tc_params[256];  // tensor-core GEMM parameters
};

struct TimingRec {
    cudaEvent_t a, b;
    int body;
};

}  // namespace upir

struct upir_region_s {
    upir_ctx ctx = nullptr;
    int teams = 0, units = 0;
    std::vector<std::unique_ptr<upir::LoopRec>> loops;
    cudaGraphExec_t gexec = nullptr;
    int batch_refs = 0;
};

struct upir_ctx_s {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    upir_allocator alloc{nullptr, nullptr, nullptr};
    std::string err;
    std::unordered_set<upir_buf> all_bufs;
    std::unordered_set<upir_region> regions;
    std::unordered_set<upir_batch> batches;
    int* err_word = nullptr;
    long long spin_limit = 1ll << 26;
    bool timing = false;
    std::vector<upir::TimingRec> timings;
    std::vector<cudaEvent_t> event_pool;
    void* mlp_scratch = nullptr;      // per-team gradient partials of the cost model
    size_t mlp_scratch_bytes = 0;
    // asynchronous copies, host->device and device->host on separate streams
    // so that both copy directions and the computation overlap (created on
    // first use)
    cudaStream_t copy_stream = nullptr, d2h_stream = nullptr;
    // submissions that use buffers, numbered; submission k records use_ring[k
    // % size] on the compute stream.  A slot re-recorded by a later
    // submission marks a later point of the same stream, so waiting on it
    // stays correct (it only waits for more).
    std::vector<cudaEvent_t> use_ring;
    int64_t submissions = 0;
    int run_sched = UPIR_SCHED_STATIC;  // what UPIR_SCHED_RUNTIME loops take
    int64_t run_chunk = 0;
    std::vector<float> cm_params, cm_mean, cm_std;  // cost model for UPIR_SCHED_AUTO (empty: none)
};

namespace upir {

upir_status fail(upir_ctx ctx, upir_status code, const char* fmt, ...);
upir_status cuda_fail(upir_ctx ctx, cudaError_t e, const char* what);
void* dev_alloc(upir_ctx ctx, size_t bytes);
void dev_free(upir_ctx ctx, void* p, size_t bytes);

upir_status plan_loop(upir_region r, const upir_loop_desc* d, LoopRec& lp);
// schedule(auto): the cost model's schedule, chunk and units for a loop
void auto_schedule(upir_ctx ctx, upir_region r, const upir_loop_desc* d, int64_t trip, int* sched, int64_t* chunk,
                   int* units_out);
void release_loop(upir_ctx ctx, LoopRec& lp);
cudaError_t launch_loop(upir_ctx ctx, LoopRec& lp, cudaStream_t s);
upir_status launch_region_loops(upir_region r, bool timed);
upir_status capture_graph(upir_ctx ctx, const std::vector<upir_region>& regions,
                          cudaGraphExec_t* out);
upir_status launch_graph_timed(upir_ctx ctx, cudaGraphExec_t g, int tag);
void destroy_region(upir_region r);
upir_status plan_gemm_tc(upir_region r, LoopRec& lp, int64_t M, int64_t N, int64_t K, upir_status st);
cudaError_t launch_gemm_tc_loop(upir_ctx ctx, LoopRec& lp, cudaStream_t s);
void destroy_batch(upir_batch b);
// make the compute stream wait for pending asynchronous copies of the
// buffers a region's loops use
upir_status wait_region_buffers(upir_region r);
// Record, on the compute stream, the end of the work submitted so far that
// uses the buffer (or every buffer of the region): asynchronous copies of a
// buffer are ordered after that point, not after all submitted work.
upir_status mark_buffer_use(upir_ctx ctx, upir_buf b);
upir_status mark_region_buffers(upir_region r);
upir_status mark_regions_buffers(const upir_region* rs, size_t n);

// Encode a 2D tiled TMA descriptor (row-major [rows][cols] of `elem_bytes`);
// swizzle_bytes is 0 (none), 32, 64 or 128.
upir_status encode_tmap_1d(upir_ctx ctx, CUtensorMap* m, const void* base, int dtype_code, uint64_t n,
                           uint32_t box);
upir_status encode_tmap_2d(upir_ctx ctx, CUtensorMap* m, const void* base, int dtype_code,
                           int elem_bytes, uint64_t cols, uint64_t rows, uint32_t box_cols,
                           uint32_t box_rows, int swizzle_bytes);

}  // namespace upir
