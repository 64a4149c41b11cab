// The sequence of tiles one team owns under a tiled loop's schedule (§3.2:
// the tile loop of a tiled collapse(2) nest is workshared over teams), produced
// on demand by the single thread that issues the tile copies.  P provides
// sched, chunk, ntiles, sk (static constants) and sc.chunk_counter (dynamic).
#pragma once

#include "device_common.cuh"

namespace upir {

struct TileIter {
    int64_t next, end;  // current contiguous run [next, end)
    int64_t chunk_j;    // static chunked: next chunk index
    bool done;
};

// Blocked static schedules hand each team its whole run up front.
template <class P>
__device__ __forceinline__ TileIter tile_iter_begin(const P& p) {
    TileIter it{0, 0, (int64_t)blockIdx.x, false};
    if (p.sched == UPIR_SCHED_STATIC && p.chunk == 0) {
        const int64_t w = blockIdx.x;
        it.next = w * p.sk.base + min(w, p.sk.extra);
        it.end = it.next + p.sk.base + (w < p.sk.extra ? 1 : 0);
    }
    return it;
}

template <class P>
__device__ __forceinline__ int64_t tile_iter_next(TileIter& it, const P& p) {
    for (;;) {
        if (it.done) return -1;
        if (it.next < it.end) return it.next++;
        if (p.sched == UPIR_SCHED_DYNAMIC) {
            const int64_t j = (int64_t)atomicAdd(p.sc.chunk_counter, 1ull);
            if (!dyn_chunk(p.sc, p.chunk, p.ntiles, j, it.next, it.end)) {
                it.done = true;
                return -1;
            }
        } else if (p.chunk > 0) {
            if (it.chunk_j >= p.sk.nchunks) {
                it.done = true;
                return -1;
            }
            it.next = it.chunk_j * p.chunk;
            it.end = min(it.next + p.chunk, p.ntiles);
            it.chunk_j += gridDim.x;
        } else {
            it.done = true;  // the blocked run was set up front
            return -1;
        }
    }
}

// After a dynamic schedule, the last team to finish returns the tile counter
// (and its own ticket) to zero for the next launch.  Called by every thread.
template <class P>
__device__ __forceinline__ void tile_iter_reset(const P& p, int* last_team_sh) {
    if (p.sched != UPIR_SCHED_DYNAMIC) return;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        *last_team_sh = atomicAdd(p.sc.ticket, 1u) == gridDim.x - 1;
        if (*last_team_sh) {
            *p.sc.ticket = 0;
            *p.sc.chunk_counter = 0;
        }
    }
}

}  // namespace upir
