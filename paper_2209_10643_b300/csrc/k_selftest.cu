// Bounded-wait self test.  One thread initialises an mbarrier and waits for a
// phase that nothing will complete, through the same bounded wait the
// TMA/tensor-core kernels use.  The wait gives up after ``spin_limit`` polls,
// records UPIR_ERR_WAIT_TIMEOUT in the device error word and the kernel
// returns normally, so the context stays usable.
#include "device_common.cuh"

namespace upir {

namespace {

__global__ void bounded_wait_selftest_kernel(long long spin_limit, int* err_word) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        mbar_wait_bounded(&bar, 0, spin_limit, err_word);
    }
}

}  // namespace

cudaError_t launch_bounded_wait_selftest(long long spin_limit, int* err_word, cudaStream_t s) {
    bounded_wait_selftest_kernel<<<1, 32, 0, s>>>(spin_limit, err_word);
    return cudaGetLastError();
}

}  // namespace upir
