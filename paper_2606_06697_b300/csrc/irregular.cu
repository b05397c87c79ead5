// Irregular kernels with the guard fused in by hand (Sec. V-E): gather out[i] = T[idx[i]],
// scatter T[idx[i]] = (float)(idx[i] & 0xFFFFFF), histogram bins[idx[i]] += 1, with int64
// element offsets that an untrusted kernel could aim anywhere. Unguarded twins share the
// code shape.
//
// Each thread takes four consecutive elements per step: the index array is read as two
// 16-byte loads (sites 0 and 1) and output stored as one 16-byte store (site 3), both
// contiguous across the warp, so one warp-uniform page check decides them; the four
// element accesses (site 2) go to data-dependent addresses and are checked per lane --
// a page-map lookup, and a binary search only on mixed pages, on a shared-memory copy of
// the table when it fits (the page map alone otherwise). The n mod 4
// tail elements use an 8-byte index load, the element access and a 4-byte store.
#include <cuda_runtime.h>

#include "agile_internal.h"
#include "guard_device.cuh"

namespace {

using agile::LaneLog;
using agile::LogDev;
using agile::TView;

constexpr int kThreads = 512;

__device__ __forceinline__ bool lane_check(const TView &V, uint64_t a, uint32_t w, uint32_t site,
                                           LaneLog &ll) {
    uint32_t rid;
    uint32_t v = agile::classify(V, a, w, &rid);
    if (v == AGILE_ALLOW) return true;
    ll.note(a, agile::pack_info(site, v, w, rid), a);
    return false;
}

template <int KIND, int POLICY>
__device__ __forceinline__ float element(float *addr, bool ok, int64_t e, const agile_dev_table_t &T) {
    constexpr bool kAlways = POLICY == AGILE_POLICY_REPORT;
    if constexpr (KIND == AGILE_IRR_GATHER) {
        return __ldg((ok || kAlways) ? addr : reinterpret_cast<const float *>(T.zero_page));
    } else if constexpr (KIND == AGILE_IRR_SCATTER) {
        const float f = (float)((uint64_t)e & 0xFFFFFFu);
        if (ok || kAlways) *addr = f;
        else if constexpr (POLICY == AGILE_POLICY_SINK) *reinterpret_cast<float *>(T.sink_page) = f;
        return 0.f;
    } else {
        if (ok || kAlways) atomicAdd(reinterpret_cast<unsigned int *>(addr), 1u);
        else if constexpr (POLICY == AGILE_POLICY_SINK)
            atomicAdd(reinterpret_cast<unsigned int *>(T.sink_page), 1u);
        return 0.f;
    }
}

template <int KIND, bool GUARD, int MODE, int POLICY>
__global__ void __launch_bounds__(kThreads, 2)
k_irregular(const agile_dev_table_t T, const int64_t *__restrict__ idx, float *base,
            float *__restrict__ out, size_t n, LogDev *log) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned long long s_bar;
    TView V{};
    if constexpr (GUARD) V = agile::stage_table<MODE>(T, smem, &s_bar, log);
    constexpr bool kAlways = POLICY == AGILE_POLICY_REPORT;
    constexpr bool kGather = KIND == AGILE_IRR_GATHER;

    const uint32_t lane = threadIdx.x & 31;
    const size_t warp = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const size_t nwarps = ((size_t)gridDim.x * blockDim.x) >> 5;
    const size_t n4 = n >> 2;
    const longlong2 *idx2 = reinterpret_cast<const longlong2 *>(idx);
    const longlong2 *zero2 = reinterpret_cast<const longlong2 *>(T.zero_page);
    const float4 *zero4 = reinterpret_cast<const float4 *>(T.zero_page);
    float4 *out4 = reinterpret_cast<float4 *>(out);
    (void)zero4;
    LaneLog ll;

    for (size_t u0 = warp * 32; u0 < n4; u0 += nwarps * 32) {      // warp-uniform trip count
        const size_t u = u0 + lane;
        const bool act = u < n4;
        bool ok0 = true, ok1 = true, oko = true;
        if constexpr (GUARD) {
            const bool full = u0 + 32 <= n4;
            const bool fast_i = full && agile::span_allowed(V, (uint64_t)(idx2 + 2 * u0), 1024);
            if (!fast_i && act) {
                ok0 = lane_check(V, (uint64_t)(idx2 + 2 * u), 16, 0, ll);
                ok1 = lane_check(V, (uint64_t)(idx2 + 2 * u + 1), 16, 1, ll);
            }
            if constexpr (kGather) {
                const bool fast_o = full && agile::span_allowed(V, (uint64_t)(out4 + u0), 512);
                if (!fast_o && act) oko = lane_check(V, (uint64_t)(out4 + u), 16, 3, ll);
            }
        }
        if (!act) continue;                  // no collective below: lanes may leave
        const longlong2 p0 = __ldg((ok0 || kAlways) ? idx2 + 2 * u : zero2);
        const longlong2 p1 = __ldg((ok1 || kAlways) ? idx2 + 2 * u + 1 : zero2);
        const int64_t e[4] = {p0.x, p0.y, p1.x, p1.y};
        float v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float *addr = reinterpret_cast<float *>((uint64_t)base + 4 * (uint64_t)e[k]);
            const bool ok = !GUARD || lane_check(V, (uint64_t)addr, 4, 2, ll);
            v[k] = element<KIND, POLICY>(addr, ok, e[k], T);
        }
        if constexpr (kGather) {
            const float4 o = make_float4(v[0], v[1], v[2], v[3]);
            if (oko || kAlways) __stcs(out4 + u, o);
            else if constexpr (POLICY == AGILE_POLICY_SINK) __stcs(reinterpret_cast<float4 *>(T.sink_page), o);
        }
    }

    if (blockIdx.x == 0 && threadIdx.x < 32 && (n & 3)) {          // tail elements
        const size_t i = n4 * 4 + lane;
        if (i < n) {
            const bool oki = !GUARD || lane_check(V, (uint64_t)(idx + i), 8, 0, ll);
            const int64_t e = *((oki || kAlways) ? idx + i : reinterpret_cast<const int64_t *>(T.zero_page));
            float *addr = reinterpret_cast<float *>((uint64_t)base + 4 * (uint64_t)e);
            const bool ok = !GUARD || lane_check(V, (uint64_t)addr, 4, 2, ll);
            const float v = element<KIND, POLICY>(addr, ok, e, T);
            if constexpr (kGather) {
                const bool oko = !GUARD || lane_check(V, (uint64_t)(out + i), 4, 3, ll);
                if (oko || kAlways) out[i] = v;
                else if constexpr (POLICY == AGILE_POLICY_SINK) *reinterpret_cast<float *>(T.sink_page) = v;
            }
        }
    }
    if constexpr (GUARD) agile::block_log_flush(log, ll);
}

template <int KIND, bool GUARD, int MODE, int POLICY>
int launch(const agile_dev_table_t &T, const int64_t *idx, void *base, float *out, size_t n,
           LogDev *log, cudaStream_t st) {
    const uint32_t smem = GUARD ? agile::stage_bytes(T, MODE) : 0;
    if (smem > 48 * 1024) {
        AGILE_CUDA_TRY(cudaFuncSetAttribute(k_irregular<KIND, GUARD, MODE, POLICY>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024));
    }
    size_t want = ((n >> 2) + kThreads - 1) / kThreads;
    size_t cap = (size_t)agile::sm_count() * 2;
    unsigned blocks = (unsigned)(want < 1 ? 1 : want > cap ? cap : want);
    k_irregular<KIND, GUARD, MODE, POLICY><<<blocks, kThreads, smem, st>>>(
        T, idx, reinterpret_cast<float *>(base), out, n, log);
    AGILE_CUDA_TRY(cudaGetLastError());
    return AGILE_OK;
}

template <int KIND, int POLICY>
int by_mode(const agile_dev_table_t &T, const int64_t *idx, void *base, float *out, size_t n,
            LogDev *log, cudaStream_t st) {
    switch (agile::stage_mode(T, true)) {
        case agile::STAGE_ALL: return launch<KIND, true, agile::STAGE_ALL, POLICY>(T, idx, base, out, n, log, st);
        case agile::STAGE_PAGES: return launch<KIND, true, agile::STAGE_PAGES, POLICY>(T, idx, base, out, n, log, st);
        default: return launch<KIND, true, agile::STAGE_NONE, POLICY>(T, idx, base, out, n, log, st);
    }
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
        default: return AGILE_ERR_INVALID_ARG;
    }
}

}  // namespace

extern "C" int agile_irregular_launch(int kind, const agile_dev_table_t *tbl, const int64_t *d_idx,
                                      void *d_base, float *d_out, size_t n, int policy,
                                      void *d_log, void *stream) {
    if (kind < AGILE_IRR_GATHER || kind > AGILE_IRR_HIST) return AGILE_ERR_INVALID_ARG;
    if (policy < AGILE_POLICY_POISON || policy > AGILE_POLICY_REPORT) return AGILE_ERR_INVALID_ARG;
    if (n == 0) return AGILE_OK;
    if (d_idx == nullptr || d_base == nullptr || (kind == AGILE_IRR_GATHER && d_out == nullptr))
        return AGILE_ERR_INVALID_ARG;
    if (((uintptr_t)d_idx & 15) || ((uintptr_t)d_base & 3) ||
        (kind == AGILE_IRR_GATHER && ((uintptr_t)d_out & 15)))
        return AGILE_ERR_ALIGN;
    if (d_log != nullptr && ((uintptr_t)d_log & 15) != 0) return AGILE_ERR_ALIGN;
    LogDev *log = (LogDev *)d_log;
    cudaStream_t st = (cudaStream_t)stream;
    switch (kind) {
        case AGILE_IRR_GATHER: return dispatch<AGILE_IRR_GATHER>(tbl, d_idx, d_base, d_out, n, policy, log, st);
        case AGILE_IRR_SCATTER: return dispatch<AGILE_IRR_SCATTER>(tbl, d_idx, d_base, d_out, n, policy, log, st);
        default: return dispatch<AGILE_IRR_HIST>(tbl, d_idx, d_base, d_out, n, policy, log, st);
    }
}
