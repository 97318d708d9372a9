// Test hooks: host-side allocation-failure injection and a self-test of the
// bounded mbarrier wait the tensor-core kernels use (a wait that can never
// complete must give up, report its error word and leave the context usable).
#include <algorithm>
#include <random>
#include <vector>

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

lfd_status lfd_selftest_freelist(int seed, int steps) {
    if (steps < 1) return LFD_EINVAL;
    const int64_t cap = 1 << 20;
    FreeList fl;
    fl.reset(cap);
    std::vector<char> owner(cap, 0);  // brute-force model: byte -> taken
    std::vector<std::pair<int64_t, int64_t>> live;  // (offset, size)
    std::mt19937_64 rng((uint64_t)seed);
    int64_t used = 0;
    for (int i = 0; i < steps; ++i) {
        const bool do_alloc = live.empty() || rng() % 3 != 0;
        if (do_alloc) {
            const int64_t want = 1 + (int64_t)(rng() % 40000);
            const int64_t off = fl.alloc(want);
            const int64_t size = align256(want);
            // a first-fit allocator fails only when no free run of `size` exists
            int64_t run = 0, best = 0;
            for (int64_t b = 0; b < cap; ++b) {
                run = owner[b] ? 0 : run + 1;
                best = std::max(best, run);
            }
            if (off < 0) {
                if (best >= size) return LFD_EINTERNAL;
                continue;
            }
            if (off % 256 != 0 || off + size > cap) return LFD_EINTERNAL;
            for (int64_t b = off; b < off + size; ++b) {
                if (owner[b]) return LFD_EINTERNAL;  // overlap
                owner[b] = 1;
            }
            live.emplace_back(off, size);
            used += size;
        } else {
            const size_t k = rng() % live.size();
            const auto blk = live[k];
            live[k] = live.back();
            live.pop_back();
            if (!fl.release(blk.first)) return LFD_EINTERNAL;
            for (int64_t b = blk.first; b < blk.first + blk.second; ++b) owner[b] = 0;
            used -= blk.second;
        }
        if (fl.used != used) return LFD_EINTERNAL;
    }
    if (fl.release(cap + 256)) return LFD_EINTERNAL;  // never handed out
    for (const auto& blk : live)
        if (!fl.release(blk.first)) return LFD_EINTERNAL;
    // everything coalesces back into one free run
    if (fl.used != 0 || fl.free_blocks() != 1 || fl.alloc(cap) != 0) return LFD_EINTERNAL;
    return LFD_OK;
}

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
