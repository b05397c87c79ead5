// Irregular kernels with the guard fused in by hand (Sec. V-E) and their unguarded
// twins; the per-group bodies live in irregular_body.cuh.
#include <cuda_runtime.h>

#include "agile_internal.h"
#include "irregular_body.cuh"

namespace {

using agile::LaneLog;
using agile::LogDev;
using agile::TView;

// One 1024-thread block per SM: the staged bitmap is held once per SM, leaving the rest
// of the unified L1/shared storage to L1, which caches the hot set of skewed gathers.
constexpr int kThreads = 1024;

template <int KIND, bool GUARD, int MODE, int POLICY, int FAST>
__global__ void __launch_bounds__(kThreads, 1)
k_irregular(const agile_dev_table_t T, const int64_t *__restrict__ idx, float *base,
            float *__restrict__ out, size_t n, LogDev *log) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned long long s_bar;
    TView V{};
    if constexpr (GUARD) V = agile::stage_table<MODE>(T, smem, &s_bar, log);
    const size_t warp = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const size_t nwarps = ((size_t)gridDim.x * blockDim.x) >> 5;
    const size_t n4 = n >> 2;
    LaneLog ll;
    ll.log = log;
    for (size_t u0 = warp * 32; u0 < n4; u0 += nwarps * 32)      // warp-uniform trip count
        agile::irregular_group<KIND, GUARD, POLICY, FAST>(V, T, idx, base, out, u0, n4, ll, true);
    if (blockIdx.x == 0 && threadIdx.x < 32 && (n & 3))
        agile::irregular_tail<KIND, GUARD, POLICY>(V, T, idx, base, out, n, ll);
    if constexpr (GUARD) agile::block_log_flush(log, ll);
}

template <int KIND, bool GUARD, int MODE, int POLICY, int FAST = agile::FAST_BITMAP>
int launch(const agile_dev_table_t &T, const int64_t *idx, void *base, float *out, size_t n,
           LogDev *log, cudaStream_t st) {
    const uint32_t smem = GUARD ? (uint32_t)agile::stage_bytes(T, MODE) : 0;
    if (smem > 48 * 1024) {
        AGILE_CUDA_TRY(cudaFuncSetAttribute(k_irregular<KIND, GUARD, MODE, POLICY, FAST>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024));
    }
    size_t want = ((n >> 2) + kThreads - 1) / kThreads;
    size_t cap = (size_t)agile::sm_count();
    unsigned blocks = (unsigned)(want < 1 ? 1 : want > cap ? cap : want);
    k_irregular<KIND, GUARD, MODE, POLICY, FAST><<<blocks, kThreads, smem, st>>>(
        T, idx, reinterpret_cast<float *>(base), out, n, log);
    AGILE_CUDA_TRY(cudaGetLastError());
    return AGILE_OK;
}

template <int KIND, int POLICY, int FAST = agile::FAST_BITMAP>
int by_mode(const agile_dev_table_t &T, const int64_t *idx, void *base, float *out, size_t n,
            LogDev *log, cudaStream_t st) {
    // Only the all-user bitmap is staged (at most 32 KiB): it decides nearly every access,
    // and the page map and ranges, used on the slow path, are read through L1.
    if (T.npages != 0 && agile::stage_bytes(T, agile::STAGE_BITS) <= 48 * 1024)
        return launch<KIND, true, agile::STAGE_BITS, POLICY, FAST>(T, idx, base, out, n, log, st);
    return launch<KIND, true, agile::STAGE_NONE, POLICY, FAST>(T, idx, base, out, n, log, st);
}

template <int KIND>
int dispatch(const agile_dev_table_t *tbl, const int64_t *idx, void *base, float *out, size_t n,
             int policy, LogDev *log, cudaStream_t st) {
    if (tbl == nullptr) {
        agile_dev_table_t none = {};
        return launch<KIND, false, agile::STAGE_NONE, AGILE_POLICY_REPORT>(none, idx, base, out, n, nullptr, st);
    }
    switch (policy) {
        case AGILE_POLICY_POISON: return by_mode<KIND, AGILE_POLICY_POISON>(*tbl, idx, base, out, n, log, st);
        case AGILE_POLICY_SINK: return by_mode<KIND, AGILE_POLICY_SINK>(*tbl, idx, base, out, n, log, st);
        case AGILE_POLICY_REPORT: return by_mode<KIND, AGILE_POLICY_REPORT>(*tbl, idx, base, out, n, log, st);
        case AGILE_POLICY_REMAP_OR: return by_mode<KIND, AGILE_POLICY_REMAP_OR>(*tbl, idx, base, out, n, log, st);
        default: return AGILE_ERR_INVALID_ARG;
    }
}

int irregular_args(int kind, int policy, const int64_t *d_idx, void *d_base, float *d_out,
                   void *d_log) {
    if (kind < AGILE_IRR_GATHER || kind > AGILE_IRR_HIST) return AGILE_ERR_INVALID_ARG;
    if (policy < AGILE_POLICY_POISON || policy > AGILE_POLICY_REMAP_OR || policy == AGILE_POLICY_TRAP)
        return AGILE_ERR_INVALID_ARG;
    if (d_idx == nullptr || d_base == nullptr || (kind == AGILE_IRR_GATHER && d_out == nullptr))
        return AGILE_ERR_INVALID_ARG;
    if (((uintptr_t)d_idx & 15) || ((uintptr_t)d_base & 3) ||
        (kind == AGILE_IRR_GATHER && ((uintptr_t)d_out & 15)))
        return AGILE_ERR_ALIGN;
    if (d_log != nullptr && ((uintptr_t)d_log & 15) != 0) return AGILE_ERR_ALIGN;
    return AGILE_OK;
}

}  // namespace

extern "C" int agile_irregular_launch_fastpath(int kind, const agile_dev_table_t *tbl,
                                               const int64_t *d_idx, void *d_base, float *d_out,
                                               size_t n, int policy, void *d_log, int fast_path,
                                               void *stream) {
    if (fast_path == AGILE_FAST_BITMAP)
        return agile_irregular_launch(kind, tbl, d_idx, d_base, d_out, n, policy, d_log, stream);
    if (fast_path != AGILE_FAST_MATCH || tbl == nullptr || policy != AGILE_POLICY_POISON)
        return AGILE_ERR_INVALID_ARG;
    if (kind < AGILE_IRR_GATHER || kind > AGILE_IRR_HIST) return AGILE_ERR_INVALID_ARG;
    if (n == 0) return AGILE_OK;
    if (int rc = irregular_args(kind, policy, d_idx, d_base, d_out, d_log)) return rc;
    LogDev *log = (LogDev *)d_log;
    cudaStream_t st = (cudaStream_t)stream;
    constexpr int P = AGILE_POLICY_POISON, M = agile::FAST_MATCH;
    switch (kind) {
        case AGILE_IRR_GATHER: return by_mode<AGILE_IRR_GATHER, P, M>(*tbl, d_idx, d_base, d_out, n, log, st);
        case AGILE_IRR_SCATTER: return by_mode<AGILE_IRR_SCATTER, P, M>(*tbl, d_idx, d_base, d_out, n, log, st);
        default: return by_mode<AGILE_IRR_HIST, P, M>(*tbl, d_idx, d_base, d_out, n, log, st);
    }
}

extern "C" int agile_irregular_launch(int kind, const agile_dev_table_t *tbl, const int64_t *d_idx,
                                      void *d_base, float *d_out, size_t n, int policy,
                                      void *d_log, void *stream) {
    if (kind < AGILE_IRR_GATHER || kind > AGILE_IRR_HIST) return AGILE_ERR_INVALID_ARG;
    if (policy < AGILE_POLICY_POISON || policy > AGILE_POLICY_REMAP_OR || policy == AGILE_POLICY_TRAP)
        return AGILE_ERR_INVALID_ARG;
    if (n == 0) return AGILE_OK;
    if (int rc = irregular_args(kind, policy, d_idx, d_base, d_out, d_log)) return rc;
    LogDev *log = (LogDev *)d_log;
    cudaStream_t st = (cudaStream_t)stream;
    switch (kind) {
        case AGILE_IRR_GATHER: return dispatch<AGILE_IRR_GATHER>(tbl, d_idx, d_base, d_out, n, policy, log, st);
        case AGILE_IRR_SCATTER: return dispatch<AGILE_IRR_SCATTER>(tbl, d_idx, d_base, d_out, n, policy, log, st);
        default: return dispatch<AGILE_IRR_HIST>(tbl, d_idx, d_base, d_out, n, policy, log, st);
    }
}
