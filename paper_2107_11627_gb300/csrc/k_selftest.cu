// Self-test of the stall detection every tensor-core kernel relies on: one
// CTA waits on an mbarrier that nothing will ever complete, through the same
// bounded wait the kernels use (here with a 0.1 s limit instead of 2 s).  The
// wait gives up, flags the CTA and sets the context's status word, which the
// host reads with p2s_check.  No GPU fault, trap or hang is involved.
#include "p2s_internal.h"
#include "tc_common.cuh"
#include "tc_ptx.cuh"

namespace p2s {
namespace {

constexpr int kStallCode = 0x100;

__global__ void stall_kernel(int *status, long long limit) {
    __shared__ uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        abort_flag = 0;
        ptx::mbar_init(ptx::smem_u32(&bar), 1);
        ptx::mbar_fence_init();
    }
    __syncthreads();
    tcc::Ctl ctl{(volatile int *)&abort_flag, status};
    // phase 0 never completes: no thread arrives
    tcc::wait_bar(ptx::smem_u32(&bar), 0, ctl, kStallCode, limit);
    __syncthreads();
}

}  // namespace
}  // namespace p2s

extern "C" p2s_status p2s_selftest_stall(p2s_ctx *ctx, void *stream) {
    if (!ctx) {
        p2s::set_error("ctx must be non-NULL");
        return P2S_EINVAL;
    }
    p2s::stall_kernel<<<1, 64, 0, (cudaStream_t)stream>>>(ctx->d_status, 200000000ll);  // ~0.1 s at 2 GHz
    P2S_CUDA(cudaGetLastError());
    return P2S_OK;
}
