// Element-granular worksharing loops: the worker is one SPMD unit (a thread),
// the work item one iteration of the canonical loop (§3.2).  Bodies: AXPY
// (§6), the empty IMOD body (reduction terms only), the COVERAGE
// instrumentation body and the per-point 5-point Jacobi sweep.
#include "device_common.cuh"

namespace upir {

namespace {

__device__ __forceinline__ long long imod_first(long long mul, long long iv, long long m) {
    const long long r = (mul * iv) % m;  // the runtime rejects products that overflow
    return r < 0 ? r + m : r;
}

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

template <bool HI>
__device__ __forceinline__ void add_int_term(const ElemParams& p, Terms& t, int64_t iv) {
    if (HI) {
        const long long v = p.rv.iterm == UPIR_TERM_IMOD ? t.imod : (long long)iv;
        t.i = iacc_combine(t.i, v, p.rv.iop);
        if (p.rv.iterm == UPIR_TERM_IMOD) t.imod = imod_next(t.imod, p.imod_inc, p.imod_mod);
    }
}

template <bool HF, bool HI>
__device__ __forceinline__ void axpy_one(const ElemParams& p, Terms& t, int64_t iv) {
    const float xv = p.x[iv];
    const float yn = __fmaf_rn(p.a, xv, p.y[iv]);
    p.y[iv] = yn;
    if (HF) {
        if (p.rv.fterm == UPIR_TERM_Y) {
            facc_add(t.f, yn, p.rv.fop);
        } else {  // x * y, with the exact product error (TwoProduct via FMA)
            const float pr = __fmul_rn(xv, yn);
            facc_add(t.f, pr, p.rv.fop, __fmaf_rn(xv, yn, -pr));
        }
    }
    add_int_term<HI>(p, t, iv);
}

template <bool HF, bool HI>
__device__ __forceinline__ void axpy_range(const ElemParams& p, Terms& t, int64_t k0, int64_t k1) {
    if (p.step != 1) {
        for (int64_t k = k0; k < k1; ++k) axpy_one<HF, HI>(p, t, p.lb + k * p.step);
        return;
    }
    int64_t i = p.lb + k0;
    const int64_t iend = p.lb + k1;
    const bool same_phase =
        ((reinterpret_cast<uintptr_t>(p.x + i) ^ reinterpret_cast<uintptr_t>(p.y + i)) & 15) == 0;
    if (same_phase) {
        while (i < iend && (reinterpret_cast<uintptr_t>(p.x + i) & 15)) axpy_one<HF, HI>(p, t, i++);
        for (; i + 4 <= iend; i += 4) {
            const float4 xv = __ldcs(reinterpret_cast<const float4*>(p.x + i));
            const float4 yv = __ldcs(reinterpret_cast<const float4*>(p.y + i));
            float4 yn;
            yn.x = __fmaf_rn(p.a, xv.x, yv.x);
            yn.y = __fmaf_rn(p.a, xv.y, yv.y);
            yn.z = __fmaf_rn(p.a, xv.z, yv.z);
            yn.w = __fmaf_rn(p.a, xv.w, yv.w);
            __stcs(reinterpret_cast<float4*>(p.y + i), yn);
            if (HF) {
                const float xs[4] = {xv.x, xv.y, xv.z, xv.w};
                const float ys[4] = {yn.x, yn.y, yn.z, yn.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (p.rv.fterm == UPIR_TERM_Y) {
                        facc_add(t.f, ys[j], p.rv.fop);
                    } else {
                        const float pr = __fmul_rn(xs[j], ys[j]);
                        facc_add(t.f, pr, p.rv.fop, __fmaf_rn(xs[j], ys[j], -pr));
                    }
                }
            }
            if (HI) {
#pragma unroll
                for (int j = 0; j < 4; ++j) add_int_term<HI>(p, t, i + j);
            }
        }
    }
    while (i < iend) axpy_one<HF, HI>(p, t, i++);
}

template <bool HF>
__device__ __forceinline__ void jacobi_point(const ElemParams& p, Terms& t, int64_t k) {
    const int64_t inner = p.cols - 2;
    const int64_t r = p.lb + k / inner, c = 1 + k % inner;
    const float* u = p.uin;
    const int64_t at = r * p.cols + c;
    const float ns = __fadd_rn(u[at - p.cols], u[at + p.cols]);
    const float we = __fadd_rn(u[at - 1], u[at + 1]);
    const float v = __fmul_rn(0.25f, __fadd_rn(ns, we));
    p.uout[at] = v;
    if (HF) facc_add(t.f, fabsf(__fsub_rn(v, u[at])), p.rv.fop);
}

template <int BODY, bool HF, bool HI>
__device__ __forceinline__ void body_range(const ElemParams& p, Terms& t, int64_t k0, int64_t k1,
                                           int64_t worker) {
    if (k0 >= k1) return;
    if (HI && p.rv.iterm == UPIR_TERM_IMOD)
        t.imod = imod_first(p.imod_mul, p.lb + k0 * p.step, p.imod_mod);
    if (BODY == UPIR_BODY_AXPY) {
        axpy_range<HF, HI>(p, t, k0, k1);
    } else if (BODY == UPIR_BODY_JACOBI5) {
        for (int64_t k = k0; k < k1; ++k) jacobi_point<HF>(p, t, k);
    } else if (BODY == UPIR_BODY_COVERAGE) {
        for (int64_t k = k0; k < k1; ++k) {
            p.owner[k] = worker;
            atomicAdd(p.count + k, 1ull);
            add_int_term<HI>(p, t, p.lb + k * p.step);
        }
    } else {  // IMOD: reduction terms only
        for (int64_t k = k0; k < k1; ++k) add_int_term<HI>(p, t, p.lb + k * p.step);
    }
}

template <int BODY, bool DYN, bool HF, bool HI>
__global__ void __launch_bounds__(1024, 1) elem_kernel(const ElemParams p) {
    constexpr bool HR = HF || HI;
    const int64_t W = (int64_t)gridDim.x * blockDim.x;
    const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (!DYN) {
        Terms t{facc_identity(p.rv.fop), iacc_identity(p.rv.iop), 0};
        static_ranges(p.trip, p.chunk, W, w,
                      [&](int64_t k0, int64_t k1) { body_range<BODY, HF, HI>(p, t, k0, k1, w); });
        if (HR) {
            const Partial bp = block_reduce_partial(make_partial(t.f, t.i), p.rv.fop, p.rv.iop);
            finish_static(p.rv, p.sc, bp);
        }
    } else {
        const int64_t c = p.chunk > 0 ? p.chunk : 1;
        for (;;) {
            const int64_t k = (int64_t)claim_chunk(p.sc.chunk_counter);
            if (k >= p.nchunks) break;
            Terms t{facc_identity(p.rv.fop), iacc_identity(p.rv.iop), 0};
            body_range<BODY, HF, HI>(p, t, k * c, min(k * c + c, p.trip), w);
            if (HR) p.sc.partials[k] = make_partial(t.f, t.i);
        }
        finish_dynamic(p.rv, p.sc, p.nchunks, HR);
    }
}

template <int BODY, bool DYN>
cudaError_t launch_3(bool hf, bool hi, int teams, int units, const ElemParams& p, cudaStream_t s) {
    if (hf && hi) elem_kernel<BODY, DYN, true, true><<<teams, units, 0, s>>>(p);
    else if (hf) elem_kernel<BODY, DYN, true, false><<<teams, units, 0, s>>>(p);
    else if (hi) elem_kernel<BODY, DYN, false, true><<<teams, units, 0, s>>>(p);
    else elem_kernel<BODY, DYN, false, false><<<teams, units, 0, s>>>(p);
    return cudaGetLastError();
}

template <int BODY>
cudaError_t launch_2(bool dyn, bool hf, bool hi, int teams, int units, const ElemParams& p,
                     cudaStream_t s) {
    return dyn ? launch_3<BODY, true>(hf, hi, teams, units, p, s)
               : launch_3<BODY, false>(hf, hi, teams, units, p, s);
}

}  // namespace

cudaError_t launch_elem(int body, bool dyn, bool hf, bool hi, int teams, int units,
                        const ElemParams& p, cudaStream_t s) {
    switch (body) {
        case UPIR_BODY_AXPY: return launch_2<UPIR_BODY_AXPY>(dyn, hf, hi, teams, units, p, s);
        case UPIR_BODY_IMOD: return launch_2<UPIR_BODY_IMOD>(dyn, hf, hi, teams, units, p, s);
        case UPIR_BODY_COVERAGE: return launch_2<UPIR_BODY_COVERAGE>(dyn, hf, hi, teams, units, p, s);
        case UPIR_BODY_JACOBI5: return launch_2<UPIR_BODY_JACOBI5>(dyn, hf, false, teams, units, p, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace upir
