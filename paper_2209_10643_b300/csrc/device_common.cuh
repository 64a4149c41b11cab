// Device-side building blocks shared by the loop kernels: compensated FP32
// accumulation, reduction combine rules, warp/block trees in a fixed order,
// worksharing schedule iteration, bounded mbarrier waits and TMA copies.
#pragma once

#include <cstdint>
#include <utility>
#include <cuda_runtime.h>
#include "upir_internal.h"

namespace upir {

// ----------------------------------------------------------------------------
// Reductions (§5: a reduction sync combines the units' partial values with the
// clause's operation).  FP32 "+" keeps a (sum, compensation) pair built with
// Knuth's TwoSum, so the result is close to the correctly rounded sum
// whatever the order; the combine order itself is fixed, so results repeat
// bit for bit.
// ----------------------------------------------------------------------------

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bp = __fsub_rn(s, a);
    const float ap = __fsub_rn(s, bp);
    e = __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp));
}

// Paired FP32 arithmetic (two lanes of one 64-bit register pair per
// instruction, each rounded to nearest like its scalar form).
struct F2 {
    unsigned long long v;
};
__device__ __forceinline__ F2 f2(float a, float b) {
    F2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void f2_split(F2 x, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(x.v));
}
__device__ __forceinline__ F2 f2_add(F2 a, F2 b) {
    F2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ F2 f2_sub(F2 a, F2 b) {
    F2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ F2 f2_mul(F2 a, F2 b) {
    F2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}

__device__ __forceinline__ F2 f2_fma(F2 a, F2 b, F2 c) {
    F2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return r;
}

// TwoSum on both lanes of a pair.
__device__ __forceinline__ void two_sum2(F2 a, F2 b, F2& s, F2& e) {
    s = f2_add(a, b);
    const F2 bp = f2_sub(s, a);
    const F2 ap = f2_sub(s, bp);
    e = f2_add(f2_sub(a, ap), f2_sub(b, bp));
}

// 256-bit global accesses: eight FP32 values, one 32-byte sector per lane.
// The address must be 32-byte aligned.  Streaming (evict-first) policy.
__device__ __forceinline__ void ld_v8_cs(const float* p, float* v) {
    asm("ld.global.cs.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
        : "l"(p));
}
__device__ __forceinline__ void st_v8_cs_f(float* p, const float* v) {
    asm volatile("st.global.cs.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};"
                 :: "l"(p), "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7])
                 : "memory");
}

struct FAcc {
    float s, c;
};

// Two compensated (+) accumulators advanced by paired instructions: lane 0
// takes the even terms of a stream, lane 1 the odd ones.
struct FAcc2 {
    F2 s, c;
};

__device__ __forceinline__ FAcc2 facc2_zero() { return FAcc2{f2(0.0f, 0.0f), f2(0.0f, 0.0f)}; }

// acc += v (both lanes), TwoSum error into the compensation.
__device__ __forceinline__ void facc2_add(FAcc2& a, F2 v) {
    F2 s, e;
    two_sum2(a.s, v, s, e);
    a.s = s;
    a.c = f2_add(a.c, e);
}

// acc += x * y (both lanes): TwoProduct by FMA, then TwoSum; both errors go
// to the compensation.
__device__ __forceinline__ void facc2_add_prod(FAcc2& a, F2 x, F2 y) {
    const F2 p = f2_mul(x, y);
    const F2 perr = f2_fma(x, y, f2_sub(f2(0.0f, 0.0f), p));
    F2 s, e;
    two_sum2(a.s, p, s, e);
    a.s = s;
    a.c = f2_add(a.c, f2_add(e, perr));
}

__device__ __forceinline__ FAcc facc_identity(int op) {
    switch (op) {
        case UPIR_RED_MUL: return {1.0f, 0.0f};
        case UPIR_RED_MAX: return {-__int_as_float(0x7f800000), 0.0f};
        case UPIR_RED_MIN: return {__int_as_float(0x7f800000), 0.0f};
        default: return {0.0f, 0.0f};
    }
}

// Add one term.  ``err`` is an exact low-order part of the term (the error of
// a rounded product), folded into the compensation for "+".
__device__ __forceinline__ void facc_add(FAcc& a, float v, int op, float err = 0.0f) {
    switch (op) {
        case UPIR_RED_ADD: {
            float s, e;
            two_sum(a.s, v, s, e);
            a.s = s;
            a.c = __fadd_rn(a.c, __fadd_rn(e, err));
            break;
        }
        case UPIR_RED_MUL: a.s = __fmul_rn(a.s, v); break;
        case UPIR_RED_MAX: a.s = fmaxf(a.s, v); break;
        case UPIR_RED_MIN: a.s = fminf(a.s, v); break;
        default: break;
    }
}

// Commutative combine of two partials (identical bits for (a, b) and (b, a)).
__device__ __forceinline__ FAcc facc_combine(FAcc a, FAcc b, int op) {
    switch (op) {
        case UPIR_RED_ADD: {
            float s, e;
            two_sum(a.s, b.s, s, e);
            return {s, __fadd_rn(__fadd_rn(a.c, b.c), e)};
        }
        case UPIR_RED_MUL: return {__fmul_rn(a.s, b.s), 0.0f};
        case UPIR_RED_MAX: return {fmaxf(a.s, b.s), 0.0f};
        case UPIR_RED_MIN: return {fminf(a.s, b.s), 0.0f};
        default: return a;
    }
}

// Fold both lanes of a paired accumulator into a (+) accumulator: lane 0,
// then lane 1.
__device__ __forceinline__ FAcc facc_merge2(FAcc a, const FAcc2& b) {
    float s0, s1, c0, c1;
    f2_split(b.s, s0, s1);
    f2_split(b.c, c0, c1);
    return facc_combine(facc_combine(a, FAcc{s0, c0}, UPIR_RED_ADD), FAcc{s1, c1}, UPIR_RED_ADD);
}

__device__ __forceinline__ long long iacc_identity(int op) {
    switch (op) {
        case UPIR_RED_MUL: return 1;
        case UPIR_RED_MAX: return (long long)0x8000000000000000ull;
        case UPIR_RED_MIN: return 0x7fffffffffffffffll;
        default: return 0;
    }
}

__device__ __forceinline__ long long iacc_combine(long long a, long long b, int op) {
    switch (op) {
        case UPIR_RED_ADD: return (long long)((unsigned long long)a + (unsigned long long)b);
        case UPIR_RED_MUL: return (long long)((unsigned long long)a * (unsigned long long)b);
        case UPIR_RED_MAX: return a > b ? a : b;
        case UPIR_RED_MIN: return a < b ? a : b;
        default: return a;
    }
}

__device__ __forceinline__ Partial make_partial(FAcc f, long long i) {
    Partial p;
    p.s = f.s;
    p.c = f.c;
    p.i = i;
    return p;
}

__device__ __forceinline__ Partial combine_partial(const Partial& a, const Partial& b,
                                                   int fop, int iop) {
    FAcc f = facc_combine(FAcc{a.s, a.c}, FAcc{b.s, b.c}, fop);
    return make_partial(f, iacc_combine(a.i, b.i, iop));
}

__device__ __forceinline__ Partial identity_partial(int fop, int iop) {
    return make_partial(facc_identity(fop), iacc_identity(iop));
}

__device__ __forceinline__ Partial shfl_xor_partial(const Partial& p, int m, unsigned mask) {
    Partial q;
    q.s = __shfl_xor_sync(mask, p.s, m);
    q.c = __shfl_xor_sync(mask, p.c, m);
    q.i = __shfl_xor_sync(mask, p.i, m);
    return q;
}

// Lanes of the calling thread's warp that exist: 32 except in the last warp
// of a block whose size is not a multiple of 32.
__device__ __forceinline__ int warp_lanes() {
    const int rest = (int)blockDim.x - (int)(threadIdx.x & ~31u);
    return rest < 32 ? rest : 32;
}

__device__ __forceinline__ unsigned lanes_mask(int n) { return n >= 32 ? 0xffffffffu : (1u << n) - 1u; }

// Butterfly over the warp's lanes: every lane ends with the same combined
// value.  In a partial warp the missing partners contribute the identity.
__device__ __forceinline__ Partial warp_reduce_partial(Partial p, int fop, int iop) {
    const int n = warp_lanes(), lane = threadIdx.x & 31;
    const unsigned mask = lanes_mask(n);
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) {
        Partial q = shfl_xor_partial(p, m, mask);
        if ((lane ^ m) >= n) q = identity_partial(fop, iop);
        p = combine_partial(p, q, fop, iop);
    }
    return p;
}

// Fixed-shape block tree; the result is valid in every thread.  All threads of
// the block must call it.
__device__ __forceinline__ Partial block_reduce_partial(Partial p, int fop, int iop) {
    __shared__ Partial warp_part[32];
    __shared__ Partial result;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
    p = warp_reduce_partial(p, fop, iop);
    __syncthreads();  // warp_part may still be read by a previous call
    if (lane == 0) warp_part[warp] = p;
    __syncthreads();
    if (warp == 0) {
        Partial q = lane < nwarps ? warp_part[lane] : identity_partial(fop, iop);
        q = warp_reduce_partial(q, fop, iop);
        if (lane == 0) result = q;
    }
    __syncthreads();
    return result;
}

// Partials written by other blocks are read through L2 (L1 is not coherent).
__device__ __forceinline__ Partial load_partial_cg(const Partial* src) {
    const float4 v = __ldcg(reinterpret_cast<const float4*>(src));
    Partial p;
    p.s = v.x;
    p.c = v.y;
    p.i = (long long)(((unsigned long long)__float_as_uint(v.w) << 32) | __float_as_uint(v.z));
    return p;
}

// Reduce slots [0, n) in a fixed order: thread t folds t, t + B, t + 2B, ...
// sequentially, then the block tree.  Every thread of the block must call it.
// Fold slots v, v + stride, v + 2 stride, ... below n into the identity in
// that order; the loads are issued four at a time so that one L2 round trip
// covers four slots.
__device__ __forceinline__ Partial fold_strided_slots(const Partial* slots, int64_t n, int64_t v,
                                                      int64_t stride, int fop, int iop) {
    Partial acc = identity_partial(fop, iop);
    int64_t k = v;
    for (; k + 3 * stride < n; k += 4 * stride) {
        const Partial a0 = load_partial_cg(slots + k), a1 = load_partial_cg(slots + k + stride);
        const Partial a2 = load_partial_cg(slots + k + 2 * stride), a3 = load_partial_cg(slots + k + 3 * stride);
        acc = combine_partial(acc, a0, fop, iop);
        acc = combine_partial(acc, a1, fop, iop);
        acc = combine_partial(acc, a2, fop, iop);
        acc = combine_partial(acc, a3, fop, iop);
    }
    for (; k < n; k += stride) acc = combine_partial(acc, load_partial_cg(slots + k), fop, iop);
    return acc;
}

__device__ __forceinline__ Partial block_reduce_slots(const Partial* slots, int64_t n,
                                                      int fop, int iop) {
    const Partial acc = fold_strided_slots(slots, n, threadIdx.x, blockDim.x, fop, iop);
    return block_reduce_partial(acc, fop, iop);
}

// The same fold as block_reduce_slots run by a block of 256 threads, computed
// by a block of any size that is a multiple of 32: 256 virtual threads fold
// their strided slots into shared memory, then the eight virtual warps and the
// final warp take the same butterflies.  A loop's last team finishes the
// reduction with it, giving the value the separate finalize kernel would.
// Every thread of the block must call it, and the block size must be a
// multiple of 32.
__device__ __forceinline__ Partial block_reduce_slots_v256(const Partial* slots, int64_t n,
                                                           int fop, int iop) {
    __shared__ Partial vpart[256];
    __shared__ Partial vwarp[8];
    __shared__ Partial vresult;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (int)(blockDim.x >> 5);  // >= 1: the block size is a multiple of 32
    for (int v = threadIdx.x; v < 256; v += blockDim.x) vpart[v] = fold_strided_slots(slots, n, v, 256, fop, iop);
    __syncthreads();
    for (int vw = warp; vw < 8; vw += nwarps) {
        const Partial q = warp_reduce_partial(vpart[vw * 32 + lane], fop, iop);
        if (lane == 0) vwarp[vw] = q;
    }
    __syncthreads();
    if (warp == 0) {
        Partial q = lane < 8 ? vwarp[lane] : identity_partial(fop, iop);
        q = warp_reduce_partial(q, fop, iop);
        if (lane == 0) vresult = q;
    }
    __syncthreads();
    return vresult;
}

// Combine the reduction variables' values before the loop with the final
// partial and store them (one thread).
__device__ __forceinline__ void write_reduction_vars(const RedVars& rv, const Partial& fin) {
    if (rv.fvar) {
        const float init = *rv.fvar;
        FAcc r = facc_combine(FAcc{init, 0.0f}, FAcc{fin.s, fin.c}, rv.fop);
        *rv.fvar = rv.fop == UPIR_RED_ADD ? __fadd_rn(r.s, r.c) : r.s;
    }
    if (rv.ivar) *rv.ivar = iacc_combine(*rv.ivar, fin.i, rv.iop);
}

// ----------------------------------------------------------------------------
// max / min folds (exact in any order), used where one atomic per team folds
// a team result into the reduction variable.
// ----------------------------------------------------------------------------

// maxNum / minNum folded into *addr; NaN operands are ignored.
__device__ __forceinline__ void atomic_fold_minmax(float* addr, float v, int op) {
    if (isnan(v)) return;
    int* ai = reinterpret_cast<int*>(addr);
    int old = *reinterpret_cast<volatile int*>(ai);
    for (;;) {
        const float of = __int_as_float(old);
        const bool better = op == UPIR_RED_MAX ? (v > of) : (v < of);
        if (!isnan(of) && !better) return;
        const int prev = atomicCAS(ai, old, __float_as_int(v));
        if (prev == old) return;
        old = prev;
    }
}

__device__ __forceinline__ float fold(float a, float b, int op) {
    return op == UPIR_RED_MIN ? fminf(a, b) : fmaxf(a, b);
}

// max / min over the warp's lanes; in a partial warp a missing partner
// stands in with the lane's own value (the fold is idempotent).
__device__ __forceinline__ float warp_fold(float v, int op) {
    const int n = warp_lanes(), lane = threadIdx.x & 31;
    const unsigned mask = lanes_mask(n);
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) {
        const float q = __shfl_xor_sync(mask, v, m);
        v = fold(v, (lane ^ m) < n ? q : v, op);
    }
    return v;
}

__device__ __forceinline__ float block_fold(float v, int op) {
    __shared__ float part[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_fold(v, op);
    if (lane == 0) part[warp] = v;
    __syncthreads();
    if (warp == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        v = warp_fold(lane < nw ? part[lane] : v, op);
    }
    return v;  // valid in thread 0
}

// Dynamically handed-out chunk j of a loop over n logical units: [b, e) of
// fixed size c (0 means 1), or from the planner's table of chunk starts
// (guided schedules, taskloops).  False once j is past the last chunk.
__device__ __forceinline__ bool dyn_chunk(const Scratch& sc, int64_t c, int64_t n, int64_t j, int64_t& b,
                                          int64_t& e) {
    if (sc.chunk_starts) {
        if (j >= sc.nchunks_tab) return false;
        b = sc.chunk_starts[j];
        e = sc.chunk_starts[j + 1];
        return true;
    }
    const int64_t cc = c > 0 ? c : 1;
    if (j >= (n + cc - 1) / cc) return false;
    b = j * cc;
    e = min(b + cc, n);
    return true;
}

// Warp-aggregated claim of the next dynamic chunk: the active lanes take
// consecutive tickets with one atomic.
__device__ __forceinline__ unsigned long long claim_chunk(unsigned long long* counter) {
    const unsigned mask = __activemask();
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(counter, (unsigned long long)__popc(mask));
    base = __shfl_sync(mask, base, leader);
    return base + __popc(mask & ((1u << lane) - 1u));
}

// ----------------------------------------------------------------------------
// Worksharing (§3.2, schedule(static[, chunk])): call f(k0, k1) for each
// contiguous range of logical iterations worker w owns.
//   chunk > 0 : chunks j = w, w + W, ... ([j c, min((j+1) c, trip)))
//   chunk = 0 : one block of ceil/floor(trip / W), the longer ones first.
// ----------------------------------------------------------------------------

template <class F>
__device__ __forceinline__ void static_ranges(const SchedConst& sk, int64_t trip, int64_t chunk,
                                              int64_t W, int64_t w, F&& f) {
    if (chunk > 0) {
        for (int64_t j = w; j < sk.nchunks; j += W) {
            const int64_t k0 = j * chunk;
            f(k0, min(k0 + chunk, trip));
        }
    } else {
        const int64_t start = w * sk.base + min(w, sk.extra);
        const int64_t len = sk.base + (w < sk.extra ? 1 : 0);
        if (len > 0) f(start, start + len);
    }
}

// Programmatic dependent launch (PTX griddepcontrol): a kernel launched with
// programmatic stream serialization may start while the previous kernel of
// the stream drains; ``griddep_wait`` blocks until that kernel has completed
// and its memory is visible (the implicit barrier after a worksharing loop).
__device__ __forceinline__ void griddep_wait() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// The start of a loop's kernel.  mode 1: the implicit barrier after the
// previous loop, every thread waits for it.  mode 2: the previous loop was
// nowait, so this one may run beside it; one thread still waits for it, so
// this loop completes only after the previous one, and the implicit barrier
// after this loop covers both (a barrier waits for all earlier work).
// mode 0: nothing to wait for.
__device__ __forceinline__ void griddep_wait_prior(int mode) {
    if (mode == 1 || (mode == 2 && blockIdx.x == 0 && threadIdx.x == 0)) griddep_wait();
}

__device__ __forceinline__ void griddep_launch_dependents() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Launch with programmatic stream serialization, so the kernel's launch and
// prologue overlap the tail of the previous kernel on the stream.
template <typename... Exp, typename... Act>
inline cudaError_t launch_pdl(void (*kern)(Exp...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t s, Act&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Act>(args)...);
}

// ----------------------------------------------------------------------------
// mbarrier and TMA (PTX ISA: mbarrier.*, cp.async.bulk.tensor).  Every wait is
// bounded: after ``limit`` polls it records UPIR_ERR_WAIT_TIMEOUT in the
// device error word and returns false; callers then skip the dependent work.
// ----------------------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// The first 1024-byte aligned address at or after `raw` (dynamic shared
// memory), formed by pointer arithmetic on the shared array rather than an
// integer round trip, so that accesses through it stay shared-memory
// instructions instead of generic ones.
template <class T>
__device__ __forceinline__ T* smem_align1k(unsigned char* raw) {
    const uint32_t a = smem_u32(raw);
    return reinterpret_cast<T*>(raw + ((1024u - (a & 1023u)) & 1023u));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}

// Bounded wait for phase ``parity`` of ``bar``.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  long long limit, int* err_word) {
    for (long long n = 0; n < limit; ++n)
        if (mbar_try_wait(bar, parity)) return true;
    if (err_word) atomicCAS(err_word, 0, UPIR_ERR_WAIT_TIMEOUT);
    return false;
}

__device__ __forceinline__ void tma_load_2d(void* smem_dst, const void* tmap, uint64_t* bar,
                                            int32_t x, int32_t y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(smem_dst)), "l"(tmap), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// An L2 access policy that marks the lines it touches first to evict.
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// tma_load_2d with an L2 cache policy for the lines it reads.
__device__ __forceinline__ void tma_load_2d_hint(void* smem_dst, const void* tmap, uint64_t* bar,
                                                 int32_t x, int32_t y, uint64_t pol) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1, {%2, %3}], [%4], %5;"
        ::"r"(smem_u32(smem_dst)), "l"(tmap), "r"(x), "r"(y), "r"(smem_u32(bar)), "l"(pol)
        : "memory");
}

// One-dimensional tiled copy of box elements starting at element x (x times
// the element size a multiple of 16 bytes; elements past either end of the
// tensor read as zero).  The destination must be 128-byte aligned.
__device__ __forceinline__ void tma_load_1d(void* smem_dst, const void* tmap, uint64_t* bar, int32_t x) {
    asm volatile(
        "cp.async.bulk.tensor.1d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2}], [%3];"
        ::"r"(smem_u32(smem_dst)), "l"(tmap), "r"(x), "r"(smem_u32(bar))
        : "memory");
}

// Ask for [p, p + bytes) to be brought into L2 (a bulk prefetch: no
// registers, no completion to wait for).  The range is shrunk to whole
// 16-byte units inside it, as the instruction requires.
__device__ __forceinline__ void prefetch_l2_range(const void* p, size_t bytes) {
    const uintptr_t a = (reinterpret_cast<uintptr_t>(p) + 15) & ~uintptr_t(15);
    const uintptr_t e = (reinterpret_cast<uintptr_t>(p) + bytes) & ~uintptr_t(15);
    if (e > a)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"((uint32_t)(e - a)) : "memory");
}

__device__ __forceinline__ void prefetch_tmap(const void* tmap) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(tmap) : "memory");
}

}  // namespace upir
