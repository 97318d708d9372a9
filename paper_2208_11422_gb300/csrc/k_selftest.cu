// Test hooks: host-side allocation-failure injection and a self-test of the
// bounded mbarrier wait the tensor-core kernels use (a wait that can never
// complete must give up, report its error word and leave the context usable).
#include <algorithm>

#include "lfd_internal.h"
#include "tc_ptx.h"

namespace lfd {
namespace {

// one thread waits for phase 0 of a barrier that nothing arrives at
__global__ void k_wait_selftest(unsigned long long limit_ns, int* err) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        tcx::mbar_init(&bar, 1);
        abort_flag = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) tcx::mbar_wait(&bar, 0, &abort_flag, err, 77, limit_ns);
}

}  // namespace
}  // namespace lfd

using namespace lfd;

extern "C" {

void lfd_debug_fail_allocs(int n) { g_fail_allocs.store(n > 0 ? n : 0); }

lfd_status lfd_selftest_bounded_wait(int64_t limit_ns, int* code) {
    if (!code || limit_ns < 1000000 || limit_ns > (int64_t)tcx::kTimeoutNs) return LFD_EINVAL;
    *code = 0;
    int* err = nullptr;
    if (cudaMalloc((void**)&err, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return LFD_ENOMEM;
    }
    cudaError_t e = cudaMemset(err, 0, sizeof(int));
    if (e == cudaSuccess) {
        k_wait_selftest<<<1, 32>>>((unsigned long long)limit_ns, err);
        count_launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(code, err, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(err);
    if (e != cudaSuccess) return LFD_ECUDA;
    return *code != 0 ? LFD_ETIMEDOUT : LFD_OK;
}

}  // extern "C"
