// AXPY with its FP32 sum and int64 (mul*i mod m) reductions for callers that
// cannot allocate device memory.  It runs the same kernels as an AXPY loop
// recorded through upir_loop with a static schedule, on teams of 256 units
// with 8 iterations per unit, but takes its reduction scratch from one fixed
// array that lives in the library's device image instead of from an
// allocator.
#include <cstring>
#include <mutex>

#include "elem_kernel.cuh"

namespace upir {

namespace {

constexpr int kNoAllocUnits = 256;                   // threads per team
constexpr int64_t kNoAllocPerWorker = 8;             // iterations per thread (planner default with reductions)
constexpr int64_t kNoAllocMaxTeams = 32768;          // one partial slot per team
constexpr int64_t kNoAllocMaxGroups = (kNoAllocMaxTeams + kFinSeg - 1) / kFinSeg;
constexpr int64_t kNoAllocMaxN = kNoAllocMaxTeams * kNoAllocUnits * kNoAllocPerWorker;  // 2^26

// Slot 0 holds the finalize ticket and the (unused) chunk counter, then the
// group partials, then one partial per team: (1 + 16 + 32768) x 16 B, about
// 512 KiB, present on every device that loads the library.
static __device__ __align__(256) Partial g_noalloc_scratch[1 + kNoAllocMaxGroups + kNoAllocMaxTeams];

constexpr int kMaxDevices = 64;

std::mutex g_noalloc_mu;
void* g_noalloc_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  The array's name
// is only a host-side stand-in, so the address is looked up once per device
// (with that device current) and cached.  The cache lives as long as the
// process: a device reset (cudaDeviceReset, or a reset of the primary
// context) reloads the module elsewhere and leaves the cached address
// dangling, so this entry point must not be used across such a reset.
upir_status noalloc_scratch(Partial** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return UPIR_ECUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return UPIR_EUNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return UPIR_ECUDA;
        }
        g_noalloc_addr[dev] = p;
    }
    *out = static_cast<Partial*>(g_noalloc_addr[dev]);
    return UPIR_OK;
}

}  // namespace

}  // namespace upir

using namespace upir;

extern "C" upir_status upir_axpy_reduce_noalloc(const float* x, float* y, int64_t n, float a,
                                                int64_t imod_mul, int64_t imod_mod, float* sum_y,
                                                int64_t* imod_sum, void* cuda_stream) {
    if (n < 0 || n > kNoAllocMaxN) return UPIR_EINVAL;
    if ((n > 0 && (!x || !y)) || !sum_y || !imod_sum) return UPIR_EINVAL;
    if (imod_mod < 1 || imod_mod >= (1ll << 62)) return UPIR_EINVAL;
    const __int128 big = (__int128)1 << 62;
    const __int128 pm = (__int128)imod_mul * (n > 0 ? n - 1 : 0);
    if (pm >= big || pm <= -big) return UPIR_EINVAL;
    if (n == 0) return UPIR_OK;  // no iteration: the variables keep their values

    Partial* scratch = nullptr;
    upir_status st = noalloc_scratch(&scratch);
    if (st != UPIR_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const int64_t teams = (n + kNoAllocUnits * kNoAllocPerWorker - 1) / (kNoAllocUnits * kNoAllocPerWorker);

    ElemParams p;
    memset(&p, 0, sizeof(p));
    p.lb = 0;
    p.step = 1;
    p.trip = n;
    p.chunk = 0;
    p.x = x;
    p.y = y;
    p.a = a;
    p.imod_mul = imod_mul;
    p.imod_mod = imod_mod;
    const __int128 inc = (__int128)imod_mul % imod_mod;
    p.imod_inc = (long long)(inc < 0 ? inc + imod_mod : inc);
    p.imod_minv = imod_mod >= 2 ? (unsigned long long)(((unsigned __int128)1 << 64) / (unsigned long long)imod_mod) : 0;
    p.imod32 = imod_mod < (1ll << 28) ? 1 : 0;
    p.sk = make_sched_const(n, 0, teams * kNoAllocUnits);
    p.wait_prior = 1;
    p.rv = RedVars{sum_y, reinterpret_cast<long long*>(imod_sum), UPIR_RED_ADD, UPIR_RED_ADD,
                   UPIR_TERM_Y, UPIR_TERM_IMOD};
    p.sc.chunk_counter = reinterpret_cast<unsigned long long*>(scratch);
    p.sc.ticket = reinterpret_cast<unsigned*>(reinterpret_cast<char*>(scratch) + 8);
    p.sc.group_tickets = nullptr;
    p.sc.group_partials = scratch + 1;
    p.sc.partials = scratch + 1 + kNoAllocMaxGroups;

    // the finalize ticket must start at zero (an earlier call may have been cut short)
    if (cudaMemsetAsync(scratch, 0, sizeof(Partial), s) != cudaSuccess) {
        cudaGetLastError();
        return UPIR_ECUDA;
    }
    if (launch_elem(UPIR_BODY_AXPY, false, UPIR_RED_ADD, UPIR_RED_ADD, (int)teams, kNoAllocUnits, p, s) !=
        cudaSuccess) {
        cudaGetLastError();
        return UPIR_ECUDA;
    }
    return UPIR_OK;
}
