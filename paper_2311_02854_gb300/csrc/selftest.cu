// Check of the bounded mbarrier wait of the warp-specialised kernels: a wait
// on a barrier that nothing arrives on gives up after its limit and reports
// through an error word; the context stays usable.
#include "engine.h"
#include "ptx.h"

namespace dmrg {
namespace {

__global__ void wait_selftest_kernel(int* err, uint64_t limit_ns, int arrive) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    ptx::mbar_init(ptx::smem_u32(&bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    if (arrive) ptx::mbar_arrive(ptx::smem_u32(&bar));
    if (!ptx::mbar_wait(ptx::smem_u32(&bar), 0, limit_ns)) atomicExch(err, 1);
}

}  // namespace

bool wait_selftest(double seconds, bool arrive, cudaStream_t st) {
    int* d_err = nullptr;
    DMRG_CHECK_CUDA(cudaMalloc(&d_err, sizeof(int)));
    int err = 0;
    cudaError_t e = cudaMemsetAsync(d_err, 0, sizeof(int), st);
    if (e == cudaSuccess) {
        wait_selftest_kernel<<<1, 32, 0, st>>>(d_err, (uint64_t)(seconds * 1e9), arrive ? 1 : 0);
        ++launch_counter();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err, d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d_err);
    DMRG_CHECK_CUDA(e);
    return err == 0;
}

}  // namespace dmrg
