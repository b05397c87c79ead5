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

// Branch-light form of the rule for random access streams: every lane reads its page
// entry and runs the same fixed number of binary-search steps over its page's range
// slice, and the allow decision is made with selects, so a warp stays converged on the
// common path. An access allowed by its page entry (all-user page) or by the range the
// search lands on is decided here; everything else -- denials, accesses across the
// window edge, illegal widths -- takes the full classification out of line.
__device__ __forceinline__ bool allow_uniform(const TView &V, uint64_t a, uint32_t w) {
    const uint64_t off = a - V.lo;
    const bool inwin = (off >> V.lg) < V.npages;
    const uint32_t p = inwin ? (uint32_t)(off >> V.lg) : 0u;
    const uint32_t e = V.page[p], e2 = V.page[p + 1];
    const uint32_t f = e & agile::kIdxMask, f2 = e2 & agile::kIdxMask;
    const bool fast = inwin && (e >> 30) == agile::PG_USER && (off & V.gmask) + w <= V.gmask + 1;
    const uint32_t hi = f2 + 1 < V.n ? f2 + 1 : V.n;
    uint32_t b = f, len = (inwin && hi > f) ? hi - f : 0u;
    for (uint32_t it = 0; it < V.steps; ++it) {
        const uint32_t half = len >> 1;
        const uint32_t probe = b + half < V.n ? b + half : (V.n ? V.n - 1 : 0u);
        const bool le = len > 0 && V.base[probe] <= a;
        b = le ? b + half + 1 : b;
        len = le ? len - half - 1 : half;
    }
    const uint32_t j = b > f ? b - 1 : 0u;          // index 0 exists (npages > 0 implies n > 0)
    const bool hit = b > f && V.kind[j] == AGILE_USER && V.end[j] >= a + w;   // base[j] <= a
    return fast || hit;
}

__device__ __forceinline__ uint32_t check_one(const TView &V, uint64_t a, uint32_t w, size_t i,
                                              LaneLog &ll) {
    const bool legal = w != 0 && w <= 16 && (w & (w - 1)) == 0 && a <= ~0ull - w;
    if (legal && V.npages > 0 && allow_uniform(V, a, w)) return AGILE_ALLOW;
    uint32_t rid = agile::kNoRange;
    const uint32_t v = (w != 0 && w <= 16 && (w & (w - 1)) == 0)
                           ? agile::classify_slow(V, a, w, &rid) : (uint32_t)AGILE_DENY_INVALID;
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
            uint64_t av[8];
#pragma unroll
            for (int k = 0; k < 4; ++k) {              // registers only: no indexed arrays
                const uint4 q = __ldcs(pa + k);
                av[2 * k] = (uint64_t)q.y << 32 | q.x;
                av[2 * k + 1] = (uint64_t)q.w << 32 | q.z;
            }
            const uint64_t wv = __ldcs(reinterpret_cast<const unsigned long long *>(width + g * 8));
            uint64_t out = 0;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const uint32_t w = (uint32_t)(wv >> (8 * k)) & 0xFFu;
                out |= (uint64_t)check_one(V, av[k], w, g * 8 + k, ll) << (8 * k);
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
