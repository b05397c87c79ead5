// Batched guard check: one verdict per (address, width) pair, the Sec. IV-E rule applied
// as the kernel guard of Sec. V-E applies it, with the first violation (smallest index)
// and the violation count in the log.
//
// Launch shape: 512 threads, two blocks per SM, a grid-stride loop. Each lane
// handles VEC consecutive accesses: VEC = 8 reads 64 address bytes as four 16-byte loads,
// 8 width bytes as one 8-byte load and writes 8 verdict bytes as one 8-byte store. The
// page map is staged into shared memory with one bulk copy when it fits. Each thread keeps
// its smallest violation in registers; the block reduces them once at the end.
#include <cuda_runtime.h>

#include "agile_internal.h"
#include "guard_device.cuh"

namespace {

using agile::LaneLog;
using agile::LogDev;

constexpr int kThreads = 512;
constexpr uint32_t kSmemMax = 48 * 1024;

__device__ __forceinline__ bool legal_width(uint32_t w) {
    return w != 0 && w <= 16 && (w & (w - 1)) == 0;
}

__device__ __forceinline__ uint8_t check_one(const agile_dev_table_t &T, const uint32_t *pg,
                                             uint64_t a, uint32_t w, size_t i, LaneLog &ll) {
    uint32_t rid = agile::kNoRange;
    uint32_t v = legal_width(w) ? agile::classify(T, pg, a, w, &rid) : (uint32_t)AGILE_DENY_INVALID;
    if (v != AGILE_ALLOW) ll.note(i, agile::pack_info(0, v, w, rid), a);
    return (uint8_t)v;
}

template <bool SMEM, int VEC>
__global__ void __launch_bounds__(kThreads, 2)
k_check_batch(const agile_dev_table_t T, const uint64_t *__restrict__ addr,
              const uint8_t *__restrict__ width, uint8_t *__restrict__ verdict, size_t n,
              LogDev *log) {
    extern __shared__ __align__(16) uint32_t s_page[];
    __shared__ unsigned long long s_bar;
    const uint32_t *pg = T.page;
    if constexpr (SMEM) pg = agile::stage_page_map(T, s_page, &s_bar, log);

    const uint32_t lane = threadIdx.x & 31;
    const size_t warp = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const size_t nwarps = ((size_t)gridDim.x * blockDim.x) >> 5;
    const size_t ngroups = n / VEC;

    LaneLog ll;
    for (size_t g = warp * 32 + lane; g < ngroups; g += nwarps * 32) {
        {
            if constexpr (VEC == 8) {
                const uint4 *pa = reinterpret_cast<const uint4 *>(addr + g * 8);
                uint4 q[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) q[k] = __ldg(pa + k);
                const uint64_t wv = __ldg(reinterpret_cast<const unsigned long long *>(width + g * 8));
                uint64_t out = 0;
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const uint4 &h = q[k >> 1];
                    uint64_t a = (k & 1) ? ((uint64_t)h.w << 32 | h.z) : ((uint64_t)h.y << 32 | h.x);
                    uint32_t w = (uint32_t)(wv >> (8 * k)) & 0xFFu;
                    out |= (uint64_t)check_one(T, pg, a, w, g * 8 + k, ll) << (8 * k);
                }
                *reinterpret_cast<unsigned long long *>(verdict + g * 8) = out;
            } else {
                verdict[g] = check_one(T, pg, __ldg(addr + g), __ldg(width + g), g, ll);
            }
        }
    }
    if (VEC > 1 && blockIdx.x == 0 && threadIdx.x < 32) {    // the last n % VEC accesses
        const size_t i = ngroups * VEC + lane;
        if (i < n) verdict[i] = check_one(T, pg, __ldg(addr + i), __ldg(width + i), i, ll);
    }
    agile::block_log_flush(log, ll);
}

template <bool SMEM, int VEC>
int launch(const agile_dev_table_t &T, const uint64_t *a, const uint8_t *w, size_t n,
           uint8_t *v, LogDev *log, cudaStream_t st, uint32_t smem) {
    size_t groups = n / VEC;
    size_t want = (groups + kThreads - 1) / kThreads;
    size_t cap = (size_t)agile::sm_count() * 2;
    unsigned blocks = (unsigned)(want < 1 ? 1 : want > cap ? cap : want);
    k_check_batch<SMEM, VEC><<<blocks, kThreads, SMEM ? smem : 0, st>>>(T, a, w, v, n, log);
    AGILE_CUDA_TRY(cudaGetLastError());
    return AGILE_OK;
}

}  // namespace

extern "C" int agile_guard_check_batch(const agile_dev_table_t *tbl, const uint64_t *d_addr,
                                       const uint8_t *d_width, size_t n, uint8_t *d_verdict,
                                       void *d_log, void *stream) {
    if (tbl == nullptr) return AGILE_ERR_INVALID_ARG;
    if (n == 0) return AGILE_OK;
    if (d_addr == nullptr || d_width == nullptr || d_verdict == nullptr) return AGILE_ERR_INVALID_ARG;
    if (d_log != nullptr && ((uintptr_t)d_log & 15) != 0) return AGILE_ERR_ALIGN;
    const bool vec = ((uintptr_t)d_addr & 15) == 0 && ((uintptr_t)d_width & 7) == 0 &&
                     ((uintptr_t)d_verdict & 7) == 0;
    const uint64_t map_bytes = ((tbl->npages + 1) * 4 + 15) & ~15ull;
    const bool smem = tbl->npages > 0 && map_bytes <= kSmemMax;
    LogDev *log = (LogDev *)d_log;
    cudaStream_t st = (cudaStream_t)stream;
    const uint32_t sb = (uint32_t)map_bytes;
    if (smem) return vec ? launch<true, 8>(*tbl, d_addr, d_width, n, d_verdict, log, st, sb)
                         : launch<true, 1>(*tbl, d_addr, d_width, n, d_verdict, log, st, sb);
    return vec ? launch<false, 8>(*tbl, d_addr, d_width, n, d_verdict, log, st, 0)
               : launch<false, 1>(*tbl, d_addr, d_width, n, d_verdict, log, st, 0);
}
