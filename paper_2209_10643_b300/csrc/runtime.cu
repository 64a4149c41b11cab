// The host side of the C ABI: contexts, data mappings (§4.1), SPMD regions
// (§3.1), worksharing loops with their validation and launch planning
// (§3.2), syncs (§5), region submission, batches, timing and diagnostics.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <string>
#include <unordered_set>
#include <vector>

#include "runtime_internal.h"

using namespace upir;

// ---------------------------------------------------------------- helpers --

upir_status upir::fail(upir_ctx ctx, upir_status code, const char* fmt, ...) {
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return code;
}

upir_status upir::cuda_fail(upir_ctx ctx, cudaError_t e, const char* what) {
    cudaGetLastError();  // clear a non-sticky error
    return fail(ctx, UPIR_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

void* upir::dev_alloc(upir_ctx ctx, size_t bytes) {
    if (bytes == 0) return nullptr;
    if (ctx->alloc.alloc) return ctx->alloc.alloc(bytes, ctx->stream, ctx->alloc.user);
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void upir::dev_free(upir_ctx ctx, void* p, size_t bytes) {
    if (!p) return;
    if (ctx->alloc.free) ctx->alloc.free(p, bytes, ctx->stream, ctx->alloc.user);
    else cudaFree(p);
}

static bool buf_ok(upir_ctx ctx, upir_buf b) {
    return b && ctx->all_bufs.count(b) && b->live;
}

// ------------------------------------------------------------------ status --

extern "C" const char* upir_status_string(upir_status s) {
    switch (s) {
        case UPIR_OK: return "UPIR_OK";
        case UPIR_EINVAL: return "UPIR_EINVAL: invalid argument";
        case UPIR_ENOTMAPPED: return "UPIR_ENOTMAPPED: buffer is not mapped";
        case UPIR_EBUSY: return "UPIR_EBUSY: object still in use";
        case UPIR_ENOMEM: return "UPIR_ENOMEM: device allocation failed";
        case UPIR_ECUDA: return "UPIR_ECUDA: CUDA runtime error";
        case UPIR_ETIMEDOUT: return "UPIR_ETIMEDOUT: a bounded device wait ran out";
        case UPIR_EUNSUPPORTED: return "UPIR_EUNSUPPORTED: not supported by this library";
        default: return "unknown upir_status";
    }
}

extern "C" const char* upir_last_error(upir_ctx ctx) {
    return ctx ? ctx->err.c_str() : "no context";
}

// ----------------------------------------------------------------- context --

extern "C" upir_status upir_init(upir_ctx* out, int32_t device, void* cuda_stream,
                                 const upir_allocator* allocator) {
    if (!out) return UPIR_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
        cudaGetLastError();
        return UPIR_ECUDA;
    }
    if (device < 0 || device >= ndev) return UPIR_EINVAL;
    if (allocator && (!allocator->alloc || !allocator->free)) return UPIR_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return UPIR_ECUDA;
    }
    std::unique_ptr<upir_ctx_s> c(new upir_ctx_s());
    c->device = device;
    if (allocator) c->alloc = *allocator;
    if (cuda_stream) {
        c->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            return UPIR_ECUDA;
        }
        c->own_stream = true;
    }
    const char* env = getenv("UPIR_SPIN_LIMIT");
    if (env && atoll(env) > 0) c->spin_limit = atoll(env);
    // run schedule of UPIR_SCHED_RUNTIME loops: "static|dynamic|guided[,chunk]"
    if (const char* rs = getenv("UPIR_SCHEDULE")) {
        const std::string v(rs);
        const size_t comma = v.find(',');
        const std::string kind = v.substr(0, comma);
        const long long ch = comma == std::string::npos ? 0 : atoll(v.c_str() + comma + 1);
        const int k = kind == "static" ? UPIR_SCHED_STATIC : kind == "dynamic" ? UPIR_SCHED_DYNAMIC
                      : kind == "guided" ? UPIR_SCHED_GUIDED : -1;
        if (k >= 0 && ch >= 0) {
            c->run_sched = k;
            c->run_chunk = ch;
        }
    }
    c->err_word = static_cast<int*>(dev_alloc(c.get(), 256));
    if (!c->err_word) {
        if (c->own_stream) cudaStreamDestroy(c->stream);
        return UPIR_ENOMEM;
    }
    if (cudaMemsetAsync(c->err_word, 0, 256, c->stream) != cudaSuccess) {
        cudaGetLastError();
        return UPIR_ECUDA;
    }
    *out = c.release();
    return UPIR_OK;
}

extern "C" upir_status upir_finalize(upir_ctx ctx) {
    if (!ctx) return UPIR_OK;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    if (ctx->copy_stream) cudaStreamSynchronize(ctx->copy_stream);
    if (ctx->d2h_stream) cudaStreamSynchronize(ctx->d2h_stream);
    cudaGetLastError();
    for (upir_batch b : std::vector<upir_batch>(ctx->batches.begin(), ctx->batches.end()))
        destroy_batch(b);
    for (upir_region r : std::vector<upir_region>(ctx->regions.begin(), ctx->regions.end()))
        destroy_region(r);
    for (upir_buf b : ctx->all_bufs) {
        if (b->live && !b->wrapped) dev_free(ctx, b->dev, b->bytes);
        if (b->ready) cudaEventDestroy(b->ready);
        delete b;
    }
    ctx->all_bufs.clear();
    for (auto& t : ctx->timings) {
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    for (cudaEvent_t e : ctx->event_pool) cudaEventDestroy(e);
    for (cudaEvent_t e : ctx->use_ring) cudaEventDestroy(e);
    dev_free(ctx, ctx->mlp_scratch, ctx->mlp_scratch_bytes);
    dev_free(ctx, ctx->err_word, 256);
    cudaStreamSynchronize(ctx->stream);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
    if (ctx->d2h_stream) cudaStreamDestroy(ctx->d2h_stream);
    cudaGetLastError();
    delete ctx;
    return UPIR_OK;
}

extern "C" upir_status upir_ctx_wait(upir_ctx ctx) {
    if (!ctx) return UPIR_EINVAL;
    cudaError_t e = ctx->copy_stream ? cudaStreamSynchronize(ctx->copy_stream) : cudaSuccess;
    if (e == cudaSuccess && ctx->d2h_stream) e = cudaStreamSynchronize(ctx->d2h_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamSynchronize");
    int word = 0;
    e = cudaMemcpyAsync(&word, ctx->err_word, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "reading the device error word");
    if (word != 0) {
        cudaMemsetAsync(ctx->err_word, 0, sizeof(int), ctx->stream);
        // a launch that gave up may have left its self-clearing counters set
        for (upir_region r : ctx->regions)
            for (auto& lp : r->loops)
                if (lp->scratch && lp->counter_bytes)
                    cudaMemsetAsync(static_cast<char*>(lp->scratch) + lp->counter_off, 0, lp->counter_bytes,
                                    ctx->stream);
        cudaStreamSynchronize(ctx->stream);
        return fail(ctx, UPIR_ETIMEDOUT, "a bounded device-side wait ran out (error word %d)", word);
    }
    return UPIR_OK;
}

extern "C" upir_status upir_ctx_set_spin_limit(upir_ctx ctx, int64_t spin_limit) {
    if (!ctx || spin_limit <= 0) return UPIR_EINVAL;
    ctx->spin_limit = spin_limit;
    return UPIR_OK;
}

extern "C" upir_status upir_selftest_bounded_wait(upir_ctx ctx, int64_t spin_limit) {
    if (!ctx || spin_limit <= 0) return UPIR_EINVAL;
    cudaError_t e = launch_bounded_wait_selftest(spin_limit, ctx->err_word, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "bounded-wait self test launch");
    return UPIR_OK;
}

// ------------------------------------------------------------ data mapping --

extern "C" upir_status upir_data_map(upir_ctx ctx, void* host, size_t bytes, int32_t kind,
                                     upir_buf* out) {
    if (!ctx) return UPIR_EINVAL;
    if (!out) return fail(ctx, UPIR_EINVAL, "upir_data_map: out is NULL");
    *out = nullptr;
    if (kind < UPIR_MAP_TO || kind > UPIR_MAP_ALLOC)
        return fail(ctx, UPIR_EINVAL, "upir_data_map: unknown map kind %d", kind);
    if (!host && bytes > 0 && kind != UPIR_MAP_ALLOC)
        return fail(ctx, UPIR_EINVAL, "upir_data_map: NULL host pointer for a copied mapping");
    void* dev = dev_alloc(ctx, bytes);
    if (bytes > 0 && !dev) return fail(ctx, UPIR_ENOMEM, "upir_data_map: allocation of %zu bytes failed", bytes);
    if (bytes > 0 && (kind == UPIR_MAP_TO || kind == UPIR_MAP_TOFROM)) {
        cudaError_t e = cudaMemcpyAsync(dev, host, bytes, cudaMemcpyHostToDevice, ctx->stream);
        if (e != cudaSuccess) {
            dev_free(ctx, dev, bytes);
            return cuda_fail(ctx, e, "upir_data_map: host->device copy");
        }
    }
    upir_buf b = new upir_buf_s();
    b->ctx = ctx;
    b->host = host;
    b->dev = dev;
    b->bytes = bytes;
    b->kind = kind;
    ctx->all_bufs.insert(b);
    if (bytes > 0 && (kind == UPIR_MAP_TO || kind == UPIR_MAP_TOFROM)) {
        // the copy went out on the compute stream
        if (upir_status st = mark_buffer_use(ctx, b)) {
            *out = b;
            return st;
        }
    }
    *out = b;
    return UPIR_OK;
}

extern "C" upir_status upir_data_map_device(upir_ctx ctx, void* device_ptr, size_t bytes,
                                            upir_buf* out) {
    if (!ctx) return UPIR_EINVAL;
    if (!out || (!device_ptr && bytes > 0))
        return fail(ctx, UPIR_EINVAL, "upir_data_map_device: bad arguments");
    upir_buf b = new upir_buf_s();
    b->ctx = ctx;
    b->dev = device_ptr;
    b->bytes = bytes;
    b->kind = UPIR_MAP_ALLOC;
    b->wrapped = true;
    ctx->all_bufs.insert(b);
    *out = b;
    return UPIR_OK;
}

extern "C" upir_status upir_data_update(upir_ctx ctx, upir_buf b, int32_t direction) {
    if (!ctx) return UPIR_EINVAL;
    if (!buf_ok(ctx, b)) return fail(ctx, UPIR_ENOTMAPPED, "upir_data_update: buffer not mapped");
    if (b->wrapped || !b->host) return fail(ctx, UPIR_EINVAL, "upir_data_update: no host copy");
    if (b->bytes == 0) return UPIR_OK;
    cudaError_t e;
    if (direction == UPIR_MAP_TO) {
        e = cudaMemcpyAsync(b->dev, b->host, b->bytes, cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess) return mark_buffer_use(ctx, b);
    } else if (direction == UPIR_MAP_FROM) {
        e = cudaMemcpyAsync(b->host, b->dev, b->bytes, cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    } else {
        return fail(ctx, UPIR_EINVAL, "upir_data_update: direction must be TO or FROM");
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "upir_data_update");
    return UPIR_OK;
}

extern "C" upir_status upir_data_unmap(upir_ctx ctx, upir_buf b) {
    if (!ctx) return UPIR_EINVAL;
    if (!buf_ok(ctx, b)) return fail(ctx, UPIR_ENOTMAPPED, "upir_data_unmap: buffer not mapped");
    if (b->refs > 0)
        return fail(ctx, UPIR_EBUSY, "upir_data_unmap: %d live region loop(s) use this buffer", b->refs);
    cudaError_t e = cudaSuccess;
    if (b->ready) {
        // a pending asynchronous copy finishes first (and the compute stream
        // is ordered after it, for the copy back below)
        e = cudaStreamWaitEvent(ctx->stream, b->ready, 0);
        b->pending = false;
    }
    if (!b->wrapped && b->bytes > 0 && (b->kind == UPIR_MAP_FROM || b->kind == UPIR_MAP_TOFROM))
        e = cudaMemcpyAsync(b->host, b->dev, b->bytes, cudaMemcpyDeviceToHost, ctx->stream);
    cudaError_t e2 = cudaStreamSynchronize(ctx->stream);
    if (e == cudaSuccess) e = e2;
    if (!b->wrapped) dev_free(ctx, b->dev, b->bytes);
    if (b->ready) cudaEventDestroy(b->ready);
    b->ready = nullptr;
    b->last_use = 0;
    b->live = false;
    b->dev = nullptr;
    if (e != cudaSuccess) return cuda_fail(ctx, e, "upir_data_unmap: device->host copy");
    return UPIR_OK;
}

extern "C" upir_status upir_buf_device_ptr(upir_buf b, void** device_ptr, size_t* bytes) {
    if (!b || !b->live) return UPIR_ENOTMAPPED;
    if (device_ptr) *device_ptr = b->dev;
    if (bytes) *bytes = b->bytes;
    return UPIR_OK;
}

// ----------------------------------------------- asynchronous data movement --

namespace {

// The copy stream of one direction, created on first use, ordered after the
// buffer's previous copy and, with after_compute, after the submitted work
// that uses the buffer (its last use on the compute stream: region and batch
// submissions, device-side copies and copies issued on the compute stream
// record it; work that does not touch the buffer is not waited for).
upir_status copy_stream_for(upir_ctx ctx, upir_buf b, bool to_device, bool after_compute, cudaStream_t* out) {
    cudaStream_t& cs = to_device ? ctx->copy_stream : ctx->d2h_stream;
    if (!cs && cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess)
        return cuda_fail(ctx, cudaGetLastError(), "creating a copy stream");
    cudaError_t e = cudaSuccess;
    if (after_compute && b->last_use > 0)
        e = cudaStreamWaitEvent(cs, ctx->use_ring[(size_t)(b->last_use % (int64_t)ctx->use_ring.size())], 0);
    if (e == cudaSuccess && b->ready) e = cudaStreamWaitEvent(cs, b->ready, 0);
    *out = cs;
    return e == cudaSuccess ? UPIR_OK : cuda_fail(ctx, e, "ordering a copy stream");
}

// Record the end of a buffer's copy on the stream that carried it.
upir_status mark_pending(upir_ctx ctx, upir_buf b, cudaStream_t cs) {
    cudaError_t e = cudaSuccess;
    if (!b->ready) e = cudaEventCreateWithFlags(&b->ready, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(b->ready, cs);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "recording a copy event");
    b->pending = true;
    return UPIR_OK;
}

}  // namespace

namespace {

// Number a new submission and record its ring event on the compute stream.
upir_status record_submission(upir_ctx ctx, int64_t* k) {
    constexpr size_t kRing = 64;
    if (ctx->use_ring.empty()) {
        ctx->use_ring.assign(kRing, nullptr);
        for (cudaEvent_t& e : ctx->use_ring)
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
                return cuda_fail(ctx, cudaGetLastError(), "creating the buffer-use events");
    }
    *k = ++ctx->submissions;
    const cudaError_t e = cudaEventRecord(ctx->use_ring[(size_t)(*k % (int64_t)kRing)], ctx->stream);
    return e == cudaSuccess ? UPIR_OK : cuda_fail(ctx, e, "recording a submission's end");
}

}  // namespace

upir_status upir::mark_buffer_use(upir_ctx ctx, upir_buf b) {
    int64_t k = 0;
    if (upir_status st = record_submission(ctx, &k)) return st;
    b->last_use = k;
    return UPIR_OK;
}

upir_status upir::mark_regions_buffers(const upir_region* rs, size_t n) {
    if (n == 0) return UPIR_OK;
    int64_t k = 0;
    if (upir_status st = record_submission(rs[0]->ctx, &k)) return st;
    for (size_t i = 0; i < n; ++i)
        for (auto& lp : rs[i]->loops) {
            for (upir_buf b : lp->bufs) b->last_use = k;
            for (auto& red : lp->reds) red.var->last_use = k;
        }
    return UPIR_OK;
}

upir_status upir::mark_region_buffers(upir_region r) { return mark_regions_buffers(&r, 1); }

upir_status upir::wait_region_buffers(upir_region r) {
    upir_ctx ctx = r->ctx;
    for (auto& lp : r->loops) {
        auto wait = [&](upir_buf b) -> cudaError_t {
            if (!b->pending) return cudaSuccess;
            b->pending = false;
            return cudaStreamWaitEvent(ctx->stream, b->ready, 0);
        };
        for (upir_buf b : lp->bufs)
            if (cudaError_t e = wait(b)) return cuda_fail(ctx, e, "waiting for a buffer's copy");
        for (auto& red : lp->reds)
            if (cudaError_t e = wait(red.var)) return cuda_fail(ctx, e, "waiting for a buffer's copy");
    }
    return UPIR_OK;
}

extern "C" upir_status upir_data_map_async(upir_ctx ctx, void* host, size_t bytes, int32_t kind,
                                           upir_buf* out) {
    if (!ctx) return UPIR_EINVAL;
    if (!out) return fail(ctx, UPIR_EINVAL, "upir_data_map_async: out is NULL");
    *out = nullptr;
    if (kind < UPIR_MAP_TO || kind > UPIR_MAP_ALLOC)
        return fail(ctx, UPIR_EINVAL, "upir_data_map_async: unknown map kind %d", kind);
    if (!host && bytes > 0 && kind != UPIR_MAP_ALLOC)
        return fail(ctx, UPIR_EINVAL, "upir_data_map_async: NULL host pointer for a copied mapping");
    void* dev = dev_alloc(ctx, bytes);
    if (bytes > 0 && !dev) return fail(ctx, UPIR_ENOMEM, "upir_data_map_async: allocation of %zu bytes failed", bytes);
    upir_buf b = new upir_buf_s();
    b->ctx = ctx;
    b->host = host;
    b->dev = dev;
    b->bytes = bytes;
    b->kind = kind;
    ctx->all_bufs.insert(b);
    if (bytes > 0 && (kind == UPIR_MAP_TO || kind == UPIR_MAP_TOFROM)) {
        // A fresh buffer: the copy need not wait for earlier work, only for
        // a caller allocator's stream-ordered allocation on the context stream
        // (cudaMalloc's memory is usable at once); then it runs beside the
        // computation.
        cudaStream_t cs = nullptr;
        upir_status st = copy_stream_for(ctx, b, true, ctx->alloc.alloc != nullptr, &cs);
        cudaError_t e = st == UPIR_OK ? cudaMemcpyAsync(dev, host, bytes, cudaMemcpyHostToDevice, cs)
                                      : cudaErrorUnknown;
        if (st == UPIR_OK && e != cudaSuccess) st = cuda_fail(ctx, e, "upir_data_map_async: host->device copy");
        if (st == UPIR_OK) st = mark_pending(ctx, b, cs);
        if (st != UPIR_OK) {
            if (ctx->copy_stream) cudaStreamSynchronize(ctx->copy_stream);
            dev_free(ctx, dev, bytes);
            if (b->ready) cudaEventDestroy(b->ready);
            ctx->all_bufs.erase(b);
            delete b;
            return st;
        }
    }
    *out = b;
    return UPIR_OK;
}

extern "C" upir_status upir_data_update_async(upir_ctx ctx, upir_buf b, int32_t direction) {
    if (!ctx) return UPIR_EINVAL;
    if (!buf_ok(ctx, b)) return fail(ctx, UPIR_ENOTMAPPED, "upir_data_update_async: buffer not mapped");
    if (b->wrapped || !b->host) return fail(ctx, UPIR_EINVAL, "upir_data_update_async: no host copy");
    if (direction != UPIR_MAP_TO && direction != UPIR_MAP_FROM)
        return fail(ctx, UPIR_EINVAL, "upir_data_update_async: direction must be TO or FROM");
    if (b->bytes == 0) return UPIR_OK;
    // after the work submitted so far (which may read or write the buffer)
    // and after the buffer's previous copy (the copy stream is in order)
    cudaStream_t cs = nullptr;
    upir_status st = copy_stream_for(ctx, b, direction == UPIR_MAP_TO, true, &cs);
    if (st != UPIR_OK) return st;
    cudaError_t e = direction == UPIR_MAP_TO
                        ? cudaMemcpyAsync(b->dev, b->host, b->bytes, cudaMemcpyHostToDevice, cs)
                        : cudaMemcpyAsync(b->host, b->dev, b->bytes, cudaMemcpyDeviceToHost, cs);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "upir_data_update_async");
    return mark_pending(ctx, b, cs);
}

extern "C" upir_status upir_buf_wait(upir_ctx ctx, upir_buf b) {
    if (!ctx) return UPIR_EINVAL;
    if (!buf_ok(ctx, b)) return fail(ctx, UPIR_ENOTMAPPED, "upir_buf_wait: buffer not mapped");
    if (!b->ready) return UPIR_OK;
    cudaError_t e = cudaEventSynchronize(b->ready);
    return e == cudaSuccess ? UPIR_OK : cuda_fail(ctx, e, "upir_buf_wait");
}

extern "C" upir_status upir_buf_copy(upir_ctx ctx, upir_buf dst, upir_buf src) {
    if (!ctx) return UPIR_EINVAL;
    if (!buf_ok(ctx, dst) || !buf_ok(ctx, src)) return fail(ctx, UPIR_ENOTMAPPED, "upir_buf_copy: buffer not mapped");
    if (dst->bytes < src->bytes)
        return fail(ctx, UPIR_EINVAL, "upir_buf_copy: destination (%zu bytes) smaller than the source (%zu bytes)",
                    dst->bytes, src->bytes);
    if (src->bytes == 0 || dst == src) return UPIR_OK;
    // a pending copy into src (or out of dst) finishes first; the compute
    // stream orders everything after this copy behind it
    for (upir_buf b : {src, dst}) {
        if (!b->pending) continue;
        const cudaError_t e = cudaStreamWaitEvent(ctx->stream, b->ready, 0);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "upir_buf_copy: waiting for a buffer's copy");
        b->pending = false;
    }
    const cudaError_t e = cudaMemcpyAsync(dst->dev, src->dev, src->bytes, cudaMemcpyDeviceToDevice, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "upir_buf_copy");
    upir_status st = mark_buffer_use(ctx, dst);
    src->last_use = dst->last_use;
    return st;
}

// ------------------------------------------------------- two-step sync steps --

extern "C" upir_status upir_ctx_arrive(upir_ctx ctx, upir_event* out) {
    if (!ctx) return UPIR_EINVAL;
    if (!out) return fail(ctx, UPIR_EINVAL, "upir_ctx_arrive: out is NULL");
    upir_event ev = new upir_event_s();
    cudaError_t e = cudaEventCreateWithFlags(&ev->ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ev->ev, ctx->stream);
    if (e != cudaSuccess) {
        if (ev->ev) cudaEventDestroy(ev->ev);
        delete ev;
        return cuda_fail(ctx, e, "upir_ctx_arrive");
    }
    *out = ev;
    return UPIR_OK;
}

extern "C" upir_status upir_event_query(upir_event ev) {
    if (!ev) return UPIR_EINVAL;
    const cudaError_t e = cudaEventQuery(ev->ev);
    if (e == cudaSuccess) return UPIR_OK;
    if (e == cudaErrorNotReady) {
        cudaGetLastError();
        return UPIR_EBUSY;
    }
    return UPIR_ECUDA;
}

extern "C" upir_status upir_event_wait(upir_event ev) {
    if (!ev) return UPIR_EINVAL;
    return cudaEventSynchronize(ev->ev) == cudaSuccess ? UPIR_OK : UPIR_ECUDA;
}

extern "C" upir_status upir_ctx_wait_event(upir_ctx ctx, upir_event ev) {
    if (!ctx || !ev) return UPIR_EINVAL;
    const cudaError_t e = cudaStreamWaitEvent(ctx->stream, ev->ev, 0);
    return e == cudaSuccess ? UPIR_OK : cuda_fail(ctx, e, "upir_ctx_wait_event");
}

extern "C" upir_status upir_event_destroy(upir_event ev) {
    if (!ev) return UPIR_EINVAL;
    cudaEventDestroy(ev->ev);
    delete ev;
    return UPIR_OK;
}

// ----------------------------------------------------------------- regions --

extern "C" upir_status upir_spmd_region(upir_ctx ctx, int32_t num_teams, int32_t num_units,
                                        upir_region* out) {
    if (!ctx) return UPIR_EINVAL;
    if (!out) return fail(ctx, UPIR_EINVAL, "upir_spmd_region: out is NULL");
    *out = nullptr;
    if (num_teams < 0) return fail(ctx, UPIR_EINVAL, "num_teams must be >= 0 (0 = planner)");
    if (num_units < 0 || num_units > 1024)
        return fail(ctx, UPIR_EINVAL, "num_units must be in [0, 1024] (0 = planner)");
    upir_region r = new upir_region_s();
    r->ctx = ctx;
    r->teams = num_teams;
    r->units = num_units;
    ctx->regions.insert(r);
    *out = r;
    return UPIR_OK;
}

void upir::destroy_region(upir_region r) {
    upir_ctx ctx = r->ctx;
    for (auto& lp : r->loops) release_loop(ctx, *lp);
    r->loops.clear();
    if (r->gexec) cudaGraphExecDestroy(r->gexec);
    ctx->regions.erase(r);
    delete r;
}

extern "C" upir_status upir_region_destroy(upir_region r) {
    if (!r) return UPIR_EINVAL;
    if (r->batch_refs > 0)
        return fail(r->ctx, UPIR_EBUSY, "upir_region_destroy: a batch still uses this region");
    destroy_region(r);
    return UPIR_OK;
}

extern "C" upir_status upir_loop(upir_region r, const upir_loop_desc* d) {
    if (!r) return UPIR_EINVAL;
    if (r->batch_refs > 0)
        return fail(r->ctx, UPIR_EBUSY, "upir_loop: the region belongs to a batch");
    std::unique_ptr<LoopRec> lp(new LoopRec());
    upir_status st = plan_loop(r, d, *lp);
    if (st != UPIR_OK) {
        release_loop(r->ctx, *lp);
        return st;
    }
    for (upir_buf b : lp->bufs) b->refs++;
    for (auto& red : lp->reds) red.var->refs++;
    lp->holds_refs = true;
    r->loops.push_back(std::move(lp));
    if (r->gexec) {
        cudaGraphExecDestroy(r->gexec);
        r->gexec = nullptr;
    }
    return UPIR_OK;
}

extern "C" upir_status upir_sync(upir_region r, int32_t kind) {
    if (!r) return UPIR_EINVAL;
    if (kind == UPIR_SYNC_BARRIER) {
        // Work on one stream is ordered, so an explicit barrier after a loop
        // is already implied by its implicit one and is elided; after a
        // nowait loop it restores the ordering (also implied on one stream).
        if (!r->loops.empty()) r->loops.back()->nowait = 0;
        return UPIR_OK;
    }
    if (kind == UPIR_SYNC_TASKWAIT) return upir_ctx_wait(r->ctx);
    return fail(r->ctx, UPIR_EINVAL, "upir_sync: unknown kind %d", kind);
}

extern "C" upir_status upir_region_loop_schedule(upir_region r, int32_t i, int32_t* sched, int64_t* chunk,
                                                 int64_t* nchunks) {
    if (!r) return UPIR_EINVAL;
    if (i < 0 || i >= (int32_t)r->loops.size()) return fail(r->ctx, UPIR_EINVAL, "loop index out of range");
    const LoopRec& lp = *r->loops[i];
    if (sched) *sched = lp.sched;
    if (chunk) *chunk = lp.chunk;
    if (nchunks) *nchunks = lp.sched == UPIR_SCHED_STATIC ? 0 : lp.nchunks;
    return UPIR_OK;
}

extern "C" upir_status upir_ctx_set_run_schedule(upir_ctx ctx, int32_t sched, int64_t chunk) {
    if (!ctx) return UPIR_EINVAL;
    if ((sched != UPIR_SCHED_STATIC && sched != UPIR_SCHED_DYNAMIC && sched != UPIR_SCHED_GUIDED) || chunk < 0)
        return fail(ctx, UPIR_EINVAL, "upir_ctx_set_run_schedule: STATIC, DYNAMIC or GUIDED with chunk >= 0");
    ctx->run_sched = sched;
    ctx->run_chunk = chunk;
    return UPIR_OK;
}

extern "C" upir_status upir_region_loop_geometry(upir_region r, int32_t i, int32_t* teams,
                                                 int32_t* units) {
    if (!r) return UPIR_EINVAL;
    if (i < 0 || i >= (int32_t)r->loops.size()) return fail(r->ctx, UPIR_EINVAL, "loop index out of range");
    if (teams) *teams = r->loops[i]->teams;
    if (units) *units = r->loops[i]->units;
    return UPIR_OK;
}

// ------------------------------------------------------------------ submit --

static upir_status record_timed(upir_ctx ctx, int body, cudaEvent_t* a) {
    if (!ctx->timing) return UPIR_OK;
    cudaEvent_t e;
    if (!ctx->event_pool.empty()) {
        e = ctx->event_pool.back();
        ctx->event_pool.pop_back();
    } else if (cudaEventCreate(&e) != cudaSuccess) {
        return cuda_fail(ctx, cudaGetLastError(), "cudaEventCreate");
    }
    cudaEventRecord(e, ctx->stream);
    *a = e;
    (void)body;
    return UPIR_OK;
}

upir_status upir::launch_region_loops(upir_region r, bool timed) {
    upir_ctx ctx = r->ctx;
    for (auto& lp : r->loops) {
        if (lp->skip) continue;
        cudaEvent_t a = nullptr, b = nullptr;
        if (timed && record_timed(ctx, lp->body, &a) != UPIR_OK) return UPIR_ECUDA;
        cudaError_t e = launch_loop(ctx, *lp, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "kernel launch");
        if (timed) {
            if (record_timed(ctx, lp->body, &b) != UPIR_OK) return UPIR_ECUDA;
            ctx->timings.push_back({a, b, lp->body});
        }
    }
    return UPIR_OK;
}

upir_status upir::capture_graph(upir_ctx ctx, const std::vector<upir_region>& regions,
                                cudaGraphExec_t* out) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamBeginCapture");
    upir_status st = UPIR_OK;
    for (upir_region r : regions) {
        st = launch_region_loops(r, false);
        if (st != UPIR_OK) break;
    }
    e = cudaStreamEndCapture(ctx->stream, &g);
    if (st != UPIR_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGraphInstantiate");
    return UPIR_OK;
}

upir_status upir::launch_graph_timed(upir_ctx ctx, cudaGraphExec_t g, int tag) {
    cudaEvent_t a = nullptr, b = nullptr;
    if (ctx->timing && record_timed(ctx, tag, &a) != UPIR_OK) return UPIR_ECUDA;
    cudaError_t e = cudaGraphLaunch(g, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGraphLaunch");
    if (ctx->timing) {
        if (record_timed(ctx, tag, &b) != UPIR_OK) return UPIR_ECUDA;
        ctx->timings.push_back({a, b, tag});
    }
    return UPIR_OK;
}

extern "C" upir_status upir_region_submit(upir_region r, int32_t flags) {
    if (!r) return UPIR_EINVAL;
    upir_ctx ctx = r->ctx;
    if (flags & ~UPIR_SUBMIT_GRAPH) return fail(ctx, UPIR_EINVAL, "upir_region_submit: unknown flags");
    if (upir_status st = wait_region_buffers(r)) return st;
    upir_status st = UPIR_OK;
    if (!(flags & UPIR_SUBMIT_GRAPH)) {
        st = launch_region_loops(r, ctx->timing);
    } else {
        if (!r->gexec) st = capture_graph(ctx, {r}, &r->gexec);
        if (st == UPIR_OK) st = launch_graph_timed(ctx, r->gexec, -1);
    }
    // The loops that did launch still use the buffers even when a later one
    // failed: record their last use whatever the status, so that an
    // asynchronous copy waits for them; the first error is returned.
    upir_status mst = mark_region_buffers(r);
    return st == UPIR_OK ? mst : st;
}

// ------------------------------------------------------------------ timing --

extern "C" upir_status upir_ctx_set_timing(upir_ctx ctx, int32_t enable) {
    if (!ctx) return UPIR_EINVAL;
    ctx->timing = enable != 0;
    return UPIR_OK;
}

extern "C" upir_status upir_ctx_timings(upir_ctx ctx, float* ms, int32_t* body, int32_t cap,
                                        int32_t* count) {
    if (!ctx || cap < 0 || (cap > 0 && !ms)) return UPIR_EINVAL;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamSynchronize");
    int32_t n = 0;
    for (auto& t : ctx->timings) {
        if (n < cap) {
            float v = 0.0f;
            cudaEventElapsedTime(&v, t.a, t.b);
            ms[n] = v;
            if (body) body[n] = t.body;
            ++n;
        }
        ctx->event_pool.push_back(t.a);
        ctx->event_pool.push_back(t.b);
    }
    ctx->timings.clear();
    if (count) *count = n;
    return UPIR_OK;
}
