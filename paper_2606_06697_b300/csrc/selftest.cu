// Self-test of the bounded waits (failure detection without a GPU fault): one warp runs
// the guard's own mbarrier wait on a barrier that expects 16 bytes no copy will deliver,
// and polls a device flag that nothing sets. Both waits give up after their time limit
// (0.25 s for the barrier, the caller's for the flag); each sets the log's TIMEOUT status,
// and the kernel returns. No copy is in flight when it exits, so the context stays usable.
#include <cuda_runtime.h>

#include "agile_internal.h"
#include "guard_device.cuh"

namespace {

__global__ void k_selftest_waits(agile::LogDev *log, const volatile uint32_t *flag,
                                 unsigned long long flag_ns, uint32_t *waits_out) {
    __shared__ unsigned long long s_bar;
    if (threadIdx.x != 0) return;
    const uint32_t bar = agile::smem_addr(&s_bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], 16;" ::"r"(bar) : "memory");
    uint32_t gave_up = 0;
    if (!agile::mbar_wait(bar, 0)) {                 // no copy will complete the phase
        atomicOr(&log->status, AGILE_LOG_STATUS_TIMEOUT);
        gave_up |= 1u;
    }
    const unsigned long long t0 = agile::global_ns();
    bool seen = false;
    for (uint32_t it = 0; it < (1u << 26) && !seen; ++it) {
        seen = *flag != 0;
        if ((it & 255) == 255 && agile::global_ns() - t0 > flag_ns) break;
    }
    if (!seen) {
        atomicOr(&log->status, AGILE_LOG_STATUS_TIMEOUT);
        gave_up |= 2u;
    }
    *waits_out = gave_up;
}

}  // namespace

extern "C" int agile_selftest_bounded_waits(void *d_log, const uint32_t *d_flag, uint32_t flag_us,
                                            uint32_t *d_result, void *stream) {
    if (d_log == nullptr || d_flag == nullptr || d_result == nullptr || flag_us == 0 ||
        flag_us > 1000000)
        return AGILE_ERR_INVALID_ARG;
    if (((uintptr_t)d_log & 15) != 0 || ((uintptr_t)d_flag & 3) != 0 || ((uintptr_t)d_result & 3) != 0)
        return AGILE_ERR_ALIGN;
    k_selftest_waits<<<1, 32, 0, (cudaStream_t)stream>>>((agile::LogDev *)d_log, d_flag,
                                                          (unsigned long long)flag_us * 1000ull, d_result);
    AGILE_CUDA_TRY(cudaGetLastError());
    return AGILE_OK;
}
