// Batched guard check: one verdict per (address, width) pair, the Sec. IV-E rule applied
// as the kernel guard of Sec. V-E applies it, with the first violation (smallest index)
// and the violation count in the log.
//
// Launch shape: 512 threads, two blocks per SM, a grid-stride loop. Each lane handles
// VEC consecutive accesses: VEC = 8 reads 64 address bytes as four 16-byte loads, 8 width
// bytes as one 8-byte load and writes 8 verdict bytes as one 8-byte store. The whole
// table (page map and range arrays) is staged into shared memory by bulk copies when it
// fits in 96 KiB, so the classification -- page lookup, and a short binary search on
// mixed pages -- runs inline on shared memory. Each thread keeps its smallest violation
// in registers; the block reduces them once at the end.
#include <cuda_runtime.h>

#include "agile_internal.h"
#include "guard_device.cuh"

namespace {

using agile::LaneLog;
using agile::LogDev;
using agile::TView;

constexpr int kThreads = 512;

__device__ __forceinline__ uint32_t check_one(const TView &V, uint64_t a, uint32_t w, size_t i,
                                              LaneLog &ll) {
    uint32_t rid = agile::kNoRange;
    const bool legal = w != 0 && w <= 16 && (w & (w - 1)) == 0;
    const uint32_t v = legal ? agile::classify(V, a, w, &rid) : (uint32_t)AGILE_DENY_INVALID;
    if (v != AGILE_ALLOW) ll.note(i, agile::pack_info(0, v, w, rid), a);
    return v;
}

template <int MODE, int VEC>
__global__ void __launch_bounds__(kThreads, 2)
k_check_batch(const agile_dev_table_t T, const uint64_t *__restrict__ addr,
              const uint8_t *__restrict__ width, uint8_t *__restrict__ verdict, size_t n,
              LogDev *log) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned long long s_bar;
    const TView V = agile::stage_table<MODE>(T, smem, &s_bar, log);

    const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t nthreads = (size_t)gridDim.x * blockDim.x;
    const size_t ngroups = n / VEC;

    LaneLog ll;
    for (size_t g = tid; g < ngroups; g += nthreads) {
        if constexpr (VEC == 8) {
            const uint4 *pa = reinterpret_cast<const uint4 *>(addr + g * 8);
            uint4 q[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) q[k] = __ldcs(pa + k);
            const uint64_t wv = __ldcs(reinterpret_cast<const unsigned long long *>(width + g * 8));
            uint64_t out = 0;
#pragma unroll 2
            for (int k = 0; k < 8; ++k) {
                const uint4 &h = q[k >> 1];
                const uint64_t a = (k & 1) ? ((uint64_t)h.w << 32 | h.z) : ((uint64_t)h.y << 32 | h.x);
                const uint32_t w = (uint32_t)(wv >> (8 * k)) & 0xFFu;
                out |= (uint64_t)check_one(V, a, w, g * 8 + k, ll) << (8 * k);
            }
            __stcs(reinterpret_cast<unsigned long long *>(verdict + g * 8), (unsigned long long)out);
        } else {
            verdict[g] = (uint8_t)check_one(V, addr[g], width[g], g, ll);
        }
    }
    if (VEC > 1 && blockIdx.x == 0 && threadIdx.x < 32) {    // the last n % VEC accesses
        const size_t i = ngroups * VEC + threadIdx.x;
        if (i < n) verdict[i] = (uint8_t)check_one(V, addr[i], width[i], i, ll);
    }
    agile::block_log_flush(log, ll);
}

template <int MODE, int VEC>
int launch(const agile_dev_table_t &T, const uint64_t *a, const uint8_t *w, size_t n,
           uint8_t *v, LogDev *log, cudaStream_t st) {
    const uint32_t smem = agile::stage_bytes(T, MODE);
    if (smem > 48 * 1024) {
        AGILE_CUDA_TRY(cudaFuncSetAttribute(k_check_batch<MODE, VEC>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024));
    }
    size_t groups = n / VEC;
    size_t want = (groups + kThreads - 1) / kThreads;
    size_t cap = (size_t)agile::sm_count() * 2;
    unsigned blocks = (unsigned)(want < 1 ? 1 : want > cap ? cap : want);
    k_check_batch<MODE, VEC><<<blocks, kThreads, smem, st>>>(T, a, w, v, n, log);
    AGILE_CUDA_TRY(cudaGetLastError());
    return AGILE_OK;
}

template <int VEC>
int launch_mode(const agile_dev_table_t &T, const uint64_t *a, const uint8_t *w, size_t n,
                uint8_t *v, LogDev *log, cudaStream_t st) {
    switch (agile::stage_mode(T, true)) {
        case agile::STAGE_ALL: return launch<agile::STAGE_ALL, VEC>(T, a, w, n, v, log, st);
        case agile::STAGE_PAGES: return launch<agile::STAGE_PAGES, VEC>(T, a, w, n, v, log, st);
        default: return launch<agile::STAGE_NONE, VEC>(T, a, w, n, v, log, st);
    }
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
    LogDev *log = (LogDev *)d_log;
    cudaStream_t st = (cudaStream_t)stream;
    return vec ? launch_mode<8>(*tbl, d_addr, d_width, n, d_verdict, log, st)
               : launch_mode<1>(*tbl, d_addr, d_width, n, d_verdict, log, st);
}
