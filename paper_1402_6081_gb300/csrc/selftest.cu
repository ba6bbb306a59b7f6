// Diagnostic: the bounded device wait the library's kernels use, exercised
// on purpose.  One CTA waits on an mbarrier phase.  With complete != 0 a
// thread arrives and the wait ends at once; with complete == 0 nothing
// completes the phase, so the wait gives up after limit_us microseconds of
// %globaltimer, records the timeout in a status word and returns.  No trap,
// no fault: the context stays usable, which the tests check.
#include <cuda_runtime.h>

#include <cstdint>

#include "lgf_internal.h"

namespace lgf {
namespace {

__global__ void k_wait_selftest(int complete, long long limit_ns, int* status) {
    __shared__ __align__(8) uint64_t bar;
    const uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(&bar));
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(a) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (complete && threadIdx.x == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
    unsigned long long t0, t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    while (true) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a)
            : "memory");
        if (done) break;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (static_cast<long long>(t - t0) > limit_ns) {
            if (threadIdx.x == 0) atomicExch(status, 1);
            return;
        }
    }
    if (threadIdx.x == 0) atomicCAS(status, -1, 0);
}

}  // namespace
}  // namespace lgf

extern "C" lgf_status lgf_selftest_bounded_wait(int32_t complete, int32_t limit_us) {
    if (limit_us < 1 || limit_us > 2000000)
        return lgf::fail(LGF_ERR_INVALID_ARG, "lgf_selftest_bounded_wait: need 1 <= limit_us <= 2e6");
    int* d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(int));
    if (e != cudaSuccess) return lgf::fail(LGF_ERR_CUDA, std::string("selftest: ") + cudaGetErrorString(e));
    const int init = -1;
    int status = -1;
    e = cudaMemcpy(d, &init, sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        lgf::k_wait_selftest<<<1, 64>>>(complete, static_cast<long long>(limit_us) * 1000, d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&status, d, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return lgf::fail(LGF_ERR_CUDA, std::string("selftest: ") + cudaGetErrorString(e));
    if (status == 1) return lgf::fail(LGF_ERR_TIMEOUT, "lgf_selftest_bounded_wait: the wait ran out (as asked)");
    if (status != 0) return lgf::fail(LGF_ERR_CUDA, "lgf_selftest_bounded_wait: no status written");
    return lgf::ok();
}
