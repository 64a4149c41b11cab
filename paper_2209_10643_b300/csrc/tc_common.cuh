// Building blocks of the tensor-core GEMM kernels (one-SM and CTA-pair
// forms): tile and ring geometry, tcgen05 instruction and shared-memory
// descriptors, TMEM loads, 32-byte stores and the static schedule of work
// units over teams.
#pragma once

#include "device_common.cuh"
#include "runtime_internal.h"

namespace upir {

constexpr int TC_BM = 128, TC_BN = 256;
constexpr int TC_THREADS = 576;  // producer warp, MMA warp, 16 epilogue warps
constexpr int TC_EPI_THREADS = 512;
constexpr int TC_EPI_COLS = 64;  // accumulator columns per epilogue warp
constexpr int kSegK = 1024;      // default K per accumulation segment of the split form
constexpr uint32_t TC_TMEM_COLS = 512;

struct TcParams {
    float* C;
    int64_t M, N, K;
    int64_t row_lb, row_ub;
    int64_t tiles_m, tiles_n, ntiles;
    int64_t chunk;
    SchedConst sk;
    long long spin_limit;
    int* err_word;
    int seg_kb;  // k-blocks per accumulation segment
    // work units: full tiles first, then either `half_tiles` tiles cut into
    // two 128-column halves (N = 128 MMAs, nothing to add up), or
    // `split_tiles` tiles cut into `parts` contiguous K ranges.  Every part of
    // a K-split tile leaves its partial sums in `work`; the part that finishes
    // last (per 32 x 64 block, counted in `tile_count`) adds all of them in
    // part order and writes C.
    int64_t full_tiles, half_tiles, split_tiles, nunits;
    int parts;
    int pair;  // CTA-pair kernel: 256 x 256 tiles, tiles_m / tiles_n count pair tiles
    float* work;
    unsigned int* tile_count;
};

constexpr int TC_SUBS = (TC_BM / 32) * (TC_BN / TC_EPI_COLS);  // 32 x 64 blocks per tile, one per epilogue warp
constexpr int TC_MAX_PARTS = 4;  // K parts of a split tile

struct TcUnit {
    int64_t tile;
    int kb0, kb1, part;
    int64_t split_idx;
    int half;  // 0: all 256 columns; 1, 2: the first or second 128
};

__device__ __forceinline__ TcUnit tc_unit(int64_t u, const TcParams& p, int nkb) {
    if (u < p.full_tiles) return TcUnit{u, 0, nkb, 0, -1, 0};
    const int64_t v = u - p.full_tiles;
    if (p.half_tiles > 0) return TcUnit{p.full_tiles + (v >> 1), 0, nkb, 0, -1, 1 + (int)(v & 1)};
    const int64_t si = v / p.parts;
    const int part = (int)(v - si * p.parts);
    return TcUnit{p.full_tiles + si, (int)((int64_t)part * nkb / p.parts),
                  (int)((int64_t)(part + 1) * nkb / p.parts), part, si, 0};
}

// Per variant: bfloat16 uses 64-wide k-blocks (one 128-byte swizzled row,
// 4 stages); the split form, three MMAs per k-step, uses 32-wide k-blocks
// (64-byte swizzle, 4 stages of four operand tiles).
template <bool X3>
struct TcCfg {
    static constexpr int BK = X3 ? 32 : 64;
    static constexpr int ROW_BYTES = BK * 2;                 // swizzle width
    static constexpr uint32_t SBO = 8 * ROW_BYTES;           // 8-row swizzle atom
    static constexpr uint64_t LAYOUT = ROW_BYTES == 128 ? 2 : 4;  // 128- or 64-byte swizzle
    static constexpr int A_BYTES = TC_BM * BK * 2;
    static constexpr int B_BYTES = TC_BN * BK * 2;
    static constexpr int STAGES = 4;
    static constexpr int STAGE_BYTES = X3 ? 2 * (A_BYTES + B_BYTES) : (A_BYTES + B_BYTES);
    static constexpr int HALF_STAGE_BYTES = X3 ? 2 * (A_BYTES + B_BYTES / 2) : (A_BYTES + B_BYTES / 2);
    static constexpr size_t SMEM = (size_t)STAGES * STAGE_BYTES + 1024;
};

// kind::f16 instruction descriptor: FP32 accumulator, bfloat16 A and B, both
// K-major, M = 128, N = 256 (or 128 for half tiles).
constexpr uint32_t tc_idesc(int n = TC_BN) {
    return (1u << 4)                        // D format: FP32
           | (1u << 7)                      // A format: BF16
           | (1u << 10)                     // B format: BF16
           | ((uint32_t)(n >> 3) << 17)     // N / 8
           | ((uint32_t)(TC_BM >> 4) << 24);// M / 16
}

// Shared-memory matrix descriptor of a K-major operand tile written by TMA
// with a 64- or 128-byte swizzle: rows of ROW_BYTES, 8-row swizzle atoms
// stacked along M/N, so the stride between atoms is 8 * ROW_BYTES.
template <class Cfg>
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);   // start address
    d |= (uint64_t)(16u >> 4) << 16;            // leading byte offset (unused for these layouts)
    d |= (uint64_t)(Cfg::SBO >> 4) << 32;       // stride byte offset
    d |= (uint64_t)1 << 46;                     // descriptor version
    d |= Cfg::LAYOUT << 61;                     // swizzle mode
    return d;
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                       uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// TMEM -> registers (32 lanes x N columns, one row per thread), with the
// wait in the same statement so that no use of the registers can be moved
// ahead of it.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr) : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr) : "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// 32-byte global accesses (one full sector per thread).
__device__ __forceinline__ void st_v8_cs(float* p, const float* v) {
    asm volatile("st.global.cs.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};"
                 ::"l"(p), "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7])
                 : "memory");
}

__device__ __forceinline__ void st_v8_cg(float* p, const float* v) {
    asm volatile("st.global.cg.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};"
                 ::"l"(p), "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7])
                 : "memory");
}

__device__ __forceinline__ void ld_v8_cg(const float* p, float* v) {
    asm volatile("ld.global.cg.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
                 : "l"(p) : "memory");
}

// Columns [n0, n0 + n) of one row of C from v: 32-byte streaming stores when
// the row segment is whole and aligned, else element by element up to N.
__device__ __forceinline__ void store_row(float* crow, int64_t n0, int64_t N, bool full, const float* v, int n) {
    if (full) {
#pragma unroll
        for (int c = 0; c < n; c += 8) st_v8_cs(crow + n0 + c, v + c);
    } else {
#pragma unroll
        for (int c = 0; c < n; ++c)
            if (n0 + c < N) crow[n0 + c] = v[c];
    }
}

// Device-scope atomic add with acquire-release ordering.
__device__ __forceinline__ unsigned int atomic_add_acq_rel(unsigned int* p, unsigned int v) {
    unsigned int old;
    asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

// Bounded wait that also gives up as soon as another role has given up.
__device__ __forceinline__ bool tc_wait(uint64_t* bar, uint32_t parity, const TcParams& p,
                                        volatile int* abort_flag) {
    for (long long n = 0; n < p.spin_limit; ++n) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((n & 255) == 255 && *abort_flag) return false;
    }
    atomicCAS(p.err_word, 0, UPIR_ERR_WAIT_TIMEOUT);
    *abort_flag = 1;
    return false;
}

// Work units of this team under the loop's static schedule, in order.
struct TcTiles {
    int64_t next, end, chunk_j;
};

__device__ __forceinline__ int64_t tc_next_tile(TcTiles& it, const TcParams& p) {
    if (it.next < it.end) return it.next++;
    if (p.chunk > 0 && it.chunk_j < p.sk.nchunks) {
        it.next = it.chunk_j * p.chunk;
        it.end = min(it.next + p.chunk, p.nunits);
        it.chunk_j += gridDim.x;
        return it.next++;
    }
    return -1;
}

__device__ __forceinline__ TcTiles tc_first(const TcParams& p) {
    TcTiles it{0, 0, (int64_t)blockIdx.x};
    if (p.chunk == 0) {
        const int64_t w = blockIdx.x;
        it.next = w * p.sk.base + min(w, p.sk.extra);
        it.end = it.next + p.sk.base + (w < p.sk.extra ? 1 : 0);
    }
    return it;
}


size_t gemm_tc2_smem_bytes();
int gemm_tc2_max_clusters();
cudaError_t launch_gemm_tc2(const TcParams& tp, int ctas, bool x3, bool mseg, const CUtensorMap* m, cudaStream_t s);

}  // namespace upir
