// Element-granular worksharing loops: the worker is one SPMD unit (a thread),
// the work item one iteration of the canonical loop (§3.2).  Bodies: AXPY
// (§6), the empty IMOD body (reduction terms only), the COVERAGE
// instrumentation body and the per-point 5-point Jacobi sweep.
//
// The kernel template is specialised on the body, the schedule kind and the
// two reduction operators (FOP for the FP32 clause, IOP for the int64 one; 0
// when the loop has none), so the per-iteration accumulation compiles to
// straight-line code.  Each team leaves one partial per team (static) or per
// chunk (dynamic) in scratch; the last team to finish folds them when they
// fit one fold, finalize_kernel afterwards otherwise.
#pragma once

#include "device_common.cuh"

namespace upir {

// (mul * iv) mod m with a non-negative remainder.  |mul * iv| < 2^62 (checked
// when the loop is recorded); the remainder uses Barrett reduction with the
// host-computed minv = floor(2^64 / m): q = hi64(x * minv) undershoots
// floor(x / m) by at most 2, so two conditional subtractions finish it.
__device__ __forceinline__ long long imod_first(const ElemParams& p, long long iv) {
    const unsigned long long m = (unsigned long long)p.imod_mod;
    if (m == 1) return 0;
    const long long prod = p.imod_mul * iv;
    const unsigned long long x = prod < 0 ? (unsigned long long)(-prod) : (unsigned long long)prod;
    unsigned long long r = x - __umul64hi(x, p.imod_minv) * m;
    if (r >= m) r -= m;
    if (r >= m) r -= m;
    return (prod < 0 && r) ? (long long)(m - r) : (long long)r;
}

// The next iteration's term from the current one: add (mul * step) mod m.
__device__ __forceinline__ long long imod_next(long long t, long long inc, long long m) {
    t += inc;
    return t >= m ? t - m : t;
}

// Per-thread accumulation state of the loop's reduction clauses.
struct Terms {
    FAcc f;
    long long i;
    long long imod;  // (mul * iv) mod m of the current iteration
};

template <int IOP>
__device__ __forceinline__ void add_int_term(const ElemParams& p, Terms& t, int64_t iv) {
    if (IOP) {
        const bool imod = p.rv.iterm == UPIR_TERM_IMOD;
        t.i = iacc_combine(t.i, imod ? t.imod : (long long)iv, IOP);
        if (imod) t.imod = imod_next(t.imod, p.imod_inc, p.imod_mod);
    }
}

template <int FOP>
__device__ __forceinline__ void add_axpy_term(const ElemParams& p, Terms& t, float xv, float yn) {
    if (FOP) {
        if (p.rv.fterm == UPIR_TERM_Y) {
            facc_add(t.f, yn, FOP);
        } else {  // x * y, with the exact product error (TwoProduct via FMA)
            const float pr = __fmul_rn(xv, yn);
            facc_add(t.f, pr, FOP, __fmaf_rn(xv, yn, -pr));
        }
    }
}

template <int FOP, int IOP>
__device__ __forceinline__ void axpy_one(const ElemParams& p, Terms& t, int64_t iv) {
    const float xv = p.x[iv];
    const float yn = __fmaf_rn(p.a, xv, p.y[iv]);
    p.y[iv] = yn;
    add_axpy_term<FOP>(p, t, xv, yn);
    add_int_term<IOP>(p, t, iv);
}

// The AXPY iterations [i, iend) of one worker, 32-byte aligned x + i and
// y + i, in groups of eight with 256-bit accesses; leaves i at the first
// iteration not done (fewer than eight remain).  PAIR: reduction(+) over y
// with two compensated accumulators, one per lane of paired FP32
// instructions (even and odd iterations), merged into t at the end.  IMOD32:
// reduction(+) over (mul * iv) mod m with m < 2^28, the eight terms of a
// group summed in 32 bits before the 64-bit accumulation.
template <int FOP, int IOP, bool PAIR, bool IMOD32>
__device__ __forceinline__ void axpy_v8(const ElemParams& p, Terms& t, int64_t& i, int64_t iend) {
    FAcc2 acc2 = facc2_zero();
    uint32_t tm = (uint32_t)t.imod;
    const uint32_t inc = (uint32_t)p.imod_inc, m = (uint32_t)p.imod_mod;
    auto group = [&](const float* xv, float* yv, int64_t i0) {
#pragma unroll
        for (int j = 0; j < 8; ++j) yv[j] = __fmaf_rn(p.a, xv[j], yv[j]);
        st_v8_cs_f(p.y + i0, yv);
        if (PAIR) {
#pragma unroll
            for (int j = 0; j < 8; j += 2) facc2_add(acc2, f2(yv[j], yv[j + 1]));
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) add_axpy_term<FOP>(p, t, xv[j], yv[j]);
        }
        if (IMOD32) {
            uint32_t g = 0;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                g += tm;
                tm += inc;
                tm = min(tm, tm - m);  // tm - m wraps above tm when tm < m
            }
            t.i = (long long)((unsigned long long)t.i + g);
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) add_int_term<IOP>(p, t, i0 + j);
        }
    };
    for (; i + 16 <= iend; i += 16) {
        float x0[8], y0[8], x1[8], y1[8];
        ld_v8_cs(p.x + i, x0);
        ld_v8_cs(p.y + i, y0);
        ld_v8_cs(p.x + i + 8, x1);
        ld_v8_cs(p.y + i + 8, y1);
        group(x0, y0, i);
        group(x1, y1, i + 8);
    }
    if (i + 8 <= iend) {
        float x0[8], y0[8];
        ld_v8_cs(p.x + i, x0);
        ld_v8_cs(p.y + i, y0);
        group(x0, y0, i);
        i += 8;
    }
    if (IMOD32) t.imod = tm;
    if (PAIR) t.f = facc_merge2(t.f, acc2);
}

template <int FOP, int IOP>
__device__ __forceinline__ void axpy_range(const ElemParams& p, Terms& t, int64_t k0, int64_t k1) {
    if (p.step != 1) {
        for (int64_t k = k0; k < k1; ++k) axpy_one<FOP, IOP>(p, t, p.lb + k * p.step);
        return;
    }
    int64_t i = p.lb + k0;
    const int64_t iend = p.lb + k1;
    const uintptr_t phase = reinterpret_cast<uintptr_t>(p.x + i) ^ reinterpret_cast<uintptr_t>(p.y + i);
    // loops without reductions keep the 128-bit path (one access per worker
    // by default, and fewer registers)
    constexpr bool kV8 = FOP != 0 || IOP != 0;
    if (kV8 && (phase & 31) == 0 && iend - i >= 8) {
        while (i < iend && (reinterpret_cast<uintptr_t>(p.x + i) & 31)) axpy_one<FOP, IOP>(p, t, i++);
        constexpr bool kPairOk = FOP == UPIR_RED_ADD;
        constexpr bool kImodOk = IOP == UPIR_RED_ADD;
        const bool pair = kPairOk && p.rv.fterm == UPIR_TERM_Y;
        const bool im32 = kImodOk && p.rv.iterm == UPIR_TERM_IMOD && p.imod32;
        if (pair && im32) axpy_v8<FOP, IOP, kPairOk, kImodOk>(p, t, i, iend);
        else if (pair) axpy_v8<FOP, IOP, kPairOk, false>(p, t, i, iend);
        else if (im32) axpy_v8<FOP, IOP, false, kImodOk>(p, t, i, iend);
        else axpy_v8<FOP, IOP, false, false>(p, t, i, iend);
    } else if ((phase & 15) == 0) {
        while (i < iend && (reinterpret_cast<uintptr_t>(p.x + i) & 15)) axpy_one<FOP, IOP>(p, t, i++);
#pragma unroll 2
        for (; i + 4 <= iend; i += 4) {
            const float4 xv = __ldcs(reinterpret_cast<const float4*>(p.x + i));
            const float4 yv = __ldcs(reinterpret_cast<const float4*>(p.y + i));
            float4 yn;
            yn.x = __fmaf_rn(p.a, xv.x, yv.x);
            yn.y = __fmaf_rn(p.a, xv.y, yv.y);
            yn.z = __fmaf_rn(p.a, xv.z, yv.z);
            yn.w = __fmaf_rn(p.a, xv.w, yv.w);
            __stcs(reinterpret_cast<float4*>(p.y + i), yn);
            add_axpy_term<FOP>(p, t, xv.x, yn.x);
            add_axpy_term<FOP>(p, t, xv.y, yn.y);
            add_axpy_term<FOP>(p, t, xv.z, yn.z);
            add_axpy_term<FOP>(p, t, xv.w, yn.w);
            add_int_term<IOP>(p, t, i);
            add_int_term<IOP>(p, t, i + 1);
            add_int_term<IOP>(p, t, i + 2);
            add_int_term<IOP>(p, t, i + 3);
        }
    }
    while (i < iend) axpy_one<FOP, IOP>(p, t, i++);
}

template <int FOP>
__device__ __forceinline__ void jacobi_point(const ElemParams& p, Terms& t, int64_t r, int64_t c) {
    const float* u = p.uin;
    const int64_t at = r * p.cols + c;
    const float ns = __fadd_rn(u[at - p.cols], u[at + p.cols]);
    const float we = __fadd_rn(u[at - 1], u[at + 1]);
    const float v = __fmul_rn(0.25f, __fadd_rn(ns, we));
    p.uout[at] = v;
    if (FOP) facc_add(t.f, fabsf(__fsub_rn(v, u[at])), FOP);
}

template <int BODY, int FOP, int IOP>
__device__ __forceinline__ void body_range(const ElemParams& p, Terms& t, int64_t k0, int64_t k1,
                                           int64_t worker) {
    if (k0 >= k1) return;
    if (IOP && p.rv.iterm == UPIR_TERM_IMOD) t.imod = imod_first(p, p.lb + k0 * p.step);
    if (BODY == UPIR_BODY_AXPY) {
        axpy_range<FOP, IOP>(p, t, k0, k1);
    } else if (BODY == UPIR_BODY_JACOBI5) {
        // iteration k is interior point (lb + k / (cols - 2), 1 + k % (cols - 2)):
        // one division per range, then the column advances
        const int64_t inner = p.cols - 2;
        int64_t r = p.lb + k0 / inner, c = 1 + k0 % inner;
        for (int64_t k = k0; k < k1; ++k) {
            jacobi_point<FOP>(p, t, r, c);
            if (++c == p.cols - 1) c = 1, ++r;
        }
    } else if (BODY == UPIR_BODY_COVERAGE) {
        for (int64_t k = k0; k < k1; ++k) {
            p.owner[k] = worker;
            atomicAdd(p.count + k, 1ull);
            add_int_term<IOP>(p, t, p.lb + k * p.step);
        }
    } else {  // IMOD: reduction terms only
        for (int64_t k = k0; k < k1; ++k) add_int_term<IOP>(p, t, p.lb + k * p.step);
    }
}

// The closing barrier of a loop whose partials fit one fold (§3.1.2): every
// team takes a ticket once its partials are written; the team holding the
// last one folds them (block_reduce_slots_v256, so the value equals the
// separate finalize kernel's), stores the reduction variables and returns the
// ticket and the dynamic chunk counter to zero.  Saves a launch per loop.
template <bool DYN, int FOP, int IOP>
__device__ __forceinline__ void elem_finish(const ElemParams& p) {
    constexpr bool HR = FOP != 0 || IOP != 0;
    __shared__ int last;
    // the team's partial slots, written by any of its threads, are ordered
    // before the ticket by the barrier and thread 0's device-scope fence
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(p.sc.ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (HR) {
        const int64_t nslots = DYN ? p.nchunks : (int64_t)gridDim.x;
        const Partial fin = block_reduce_slots_v256(p.sc.partials, nslots, FOP, IOP);
        if (threadIdx.x == 0) write_reduction_vars(p.rv, fin);
    }
    if (threadIdx.x == 0) {
        *p.sc.ticket = 0;
        if (DYN) *p.sc.chunk_counter = 0;
    }
}

template <int BODY, bool DYN, int FOP, int IOP>
__global__ void __launch_bounds__(1024, 1) elem_kernel(const ElemParams p) {
    constexpr bool HR = FOP != 0 || IOP != 0;
    const int64_t W = (int64_t)gridDim.x * blockDim.x;
    const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    griddep_wait_prior(p.wait_prior);
    griddep_launch_dependents();
    if (!DYN) {
        Terms t{facc_identity(FOP), iacc_identity(IOP), 0};
        static_ranges(p.sk, p.trip, p.chunk, W, w,
                      [&](int64_t k0, int64_t k1) { body_range<BODY, FOP, IOP>(p, t, k0, k1, w); });
        if (HR) {
            const Partial bp = block_reduce_partial(make_partial(t.f, t.i), FOP, IOP);
            if (threadIdx.x == 0) p.sc.partials[blockIdx.x] = bp;
        }
    } else {
        for (;;) {
            const int64_t k = (int64_t)claim_chunk(p.sc.chunk_counter);
            int64_t k0, k1;
            if (!dyn_chunk(p.sc, p.chunk, p.trip, k, k0, k1)) break;
            Terms t{facc_identity(FOP), iacc_identity(IOP), 0};
            body_range<BODY, FOP, IOP>(p, t, k0, k1, w);
            if (HR) p.sc.partials[k] = make_partial(t.f, t.i);
        }
    }
    if (p.fuse_fin) elem_finish<DYN, FOP, IOP>(p);
}

template <int BODY, bool DYN, int FOP>
cudaError_t launch_elem_iop(int iop, int teams, int units, const ElemParams& p, cudaStream_t s) {
    switch (iop) {
        case 0: return launch_pdl(elem_kernel<BODY, DYN, FOP, 0>, teams, units, 0, s, p);
        case UPIR_RED_ADD: return launch_pdl(elem_kernel<BODY, DYN, FOP, UPIR_RED_ADD>, teams, units, 0, s, p);
        case UPIR_RED_MUL: return launch_pdl(elem_kernel<BODY, DYN, FOP, UPIR_RED_MUL>, teams, units, 0, s, p);
        case UPIR_RED_MAX: return launch_pdl(elem_kernel<BODY, DYN, FOP, UPIR_RED_MAX>, teams, units, 0, s, p);
        case UPIR_RED_MIN: return launch_pdl(elem_kernel<BODY, DYN, FOP, UPIR_RED_MIN>, teams, units, 0, s, p);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace upir
