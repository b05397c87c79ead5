// Streaming kernels with the guard fused in by hand: COPY a = b, SCALE a = s*b, TRIAD
// a = b + s*c (one fused multiply-add), fp32, 16-byte vector accesses (Sec. V-E: an
// address-range check before every global access, ordinary user-allocation accesses left
// on the normal path), and their unguarded twins.
//
// Guard placement. A warp's k-th unit covers 32 consecutive 16-byte vectors, i.e. one
// contiguous 512-byte span per array. When that span lies inside one all-user page of the
// map, every access in it is allowed: one shared-memory broadcast read decides the whole
// warp (the warp-uniform fast path). Otherwise each lane classifies its own access and
// the policy applies per access: POISON and SINK redirect denied loads to the table's
// zero page; POISON drops denied stores, SINK sends them to the sink page; REPORT lets
// every access through. Denied accesses are logged with key (address, site).
#include <cuda_runtime.h>

#include "agile_internal.h"
#include "guard_device.cuh"

namespace {

using agile::LaneLog;
using agile::LogDev;

constexpr int kThreads = 512;
constexpr int kUnroll = 4;
constexpr uint32_t kSmemMax = 48 * 1024;

template <int OP>
__device__ __forceinline__ float4 op4(float s, float4 b, float4 c) {
    if constexpr (OP == AGILE_OP_COPY) return b;
    if constexpr (OP == AGILE_OP_SCALE) return make_float4(s * b.x, s * b.y, s * b.z, s * b.w);
    return make_float4(__fmaf_rn(s, c.x, b.x), __fmaf_rn(s, c.y, b.y), __fmaf_rn(s, c.z, b.z),
                       __fmaf_rn(s, c.w, b.w));
}

template <int OP>
__device__ __forceinline__ float op1(float s, float b, float c) {
    if constexpr (OP == AGILE_OP_COPY) return b;
    if constexpr (OP == AGILE_OP_SCALE) return s * b;
    return __fmaf_rn(s, c, b);
}

// Per-lane check of one access; notes a violation. Returns whether it is allowed.
__device__ __forceinline__ bool lane_check(const agile_dev_table_t &T, const uint32_t *pg,
                                           uint64_t a, uint32_t w, uint32_t site, LaneLog &ll) {
    uint32_t rid;
    uint32_t v = agile::classify(T, pg, a, w, &rid);
    if (v == AGILE_ALLOW) return true;
    ll.note(a, agile::pack_info(site, v, w, rid), a);
    return false;
}

// The per-lane path, out of line so the common path keeps few registers: called when some
// unit k of this warp (bit k clear in `fast`) is not decided by the warp-uniform check.
// Returns ok bits: bit 3k+0 b, 3k+1 c, 3k+2 a; violations go to the thread's LaneLog.
template <int OP>
__device__ __noinline__ uint32_t slow_units(const agile_dev_table_t &T, const uint32_t *pg,
                                            const float4 *a4, const float4 *b4, const float4 *c4,
                                            size_t first, size_t stride, size_t n4, uint32_t fast,
                                            LaneLog &ll) {
    constexpr bool kTriad = OP == AGILE_OP_TRIAD;
    constexpr uint32_t kSiteB = 0, kSiteC = 1, kSiteA = kTriad ? 2 : 1;
    uint32_t ok = ~0u;
#pragma unroll 1
    for (int k = 0; k < kUnroll; ++k) {
        const size_t i = first + k * stride;
        if ((fast >> k) & 1 || i >= n4) continue;
        if (!lane_check(T, pg, (uint64_t)(b4 + i), 16, kSiteB, ll)) ok &= ~(1u << (3 * k));
        if (kTriad && !lane_check(T, pg, (uint64_t)(c4 + i), 16, kSiteC, ll)) ok &= ~(2u << (3 * k));
        if (!lane_check(T, pg, (uint64_t)(a4 + i), 16, kSiteA, ll)) ok &= ~(4u << (3 * k));
    }
    return ok;
}

template <int OP, bool GUARD, bool SMEM, int POLICY>
__global__ void __launch_bounds__(kThreads, 2)
k_stream(const agile_dev_table_t T, float *__restrict__ a, const float *__restrict__ b,
         const float *__restrict__ c, size_t n, float s, LogDev *log) {
    extern __shared__ __align__(16) uint32_t s_page[];
    __shared__ unsigned long long s_bar;
    const uint32_t *pg = T.page;
    if constexpr (GUARD && SMEM) pg = agile::stage_page_map(T, s_page, &s_bar, log);

    constexpr bool kTriad = OP == AGILE_OP_TRIAD;
    constexpr uint32_t kSiteB = 0, kSiteC = 1, kSiteA = kTriad ? 2 : 1;
    constexpr bool kLoadAlways = POLICY == AGILE_POLICY_REPORT;

    const size_t n4 = n >> 2;
    const float4 *b4 = reinterpret_cast<const float4 *>(b);
    const float4 *c4 = reinterpret_cast<const float4 *>(c);
    float4 *a4 = reinterpret_cast<float4 *>(a);
    const float4 *zero4 = reinterpret_cast<const float4 *>(T.zero_page);
    float4 *sink4 = reinterpret_cast<float4 *>(T.sink_page);

    const uint32_t lane = threadIdx.x & 31;
    const size_t gtid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t wbase = gtid - lane;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    LaneLog ll;

    for (size_t chunk = 0; chunk < n4; chunk += stride * kUnroll) {
        size_t idx[kUnroll];
        bool act[kUnroll];
        uint32_t ok = ~0u;                  // bit 3k+0 b, 3k+1 c, 3k+2 a
#pragma unroll
        for (int k = 0; k < kUnroll; ++k) {
            idx[k] = chunk + k * stride + gtid;
            act[k] = idx[k] < n4;
        }
        if constexpr (GUARD) {
            uint32_t fast = 0;              // warp-uniform
#pragma unroll
            for (int k = 0; k < kUnroll; ++k) {
                const size_t w0 = chunk + k * stride + wbase;
                bool f = w0 + 32 <= n4 &&
                         agile::span_in_user_page(T, pg, (uint64_t)(b4 + w0), 512) &&
                         agile::span_in_user_page(T, pg, (uint64_t)(a4 + w0), 512);
                if constexpr (kTriad) f = f && agile::span_in_user_page(T, pg, (uint64_t)(c4 + w0), 512);
                fast |= (uint32_t)f << k;
            }
            if (fast != (1u << kUnroll) - 1)
                ok = slow_units<OP>(T, pg, a4, b4, c4, chunk + gtid, stride, n4, fast, ll);
        }
    float4 vb[kUnroll], vc[kUnroll];
#pragma unroll
        for (int k = 0; k < kUnroll; ++k) {
            if (act[k]) {
                const bool okb = (ok >> (3 * k)) & 1, okc = (ok >> (3 * k + 1)) & 1;
                vb[k] = __ldcs((okb || kLoadAlways) ? b4 + idx[k] : zero4);
                if constexpr (kTriad) vc[k] = __ldcs((okc || kLoadAlways) ? c4 + idx[k] : zero4);
                else vc[k] = vb[k];
            }
        }
#pragma unroll
        for (int k = 0; k < kUnroll; ++k) {
            if (act[k]) {
                float4 out = op4<OP>(s, vb[k], vc[k]);
                const bool oka = (ok >> (3 * k + 2)) & 1;
                if (oka || kLoadAlways) __stcs(a4 + idx[k], out);
                else if constexpr (POLICY == AGILE_POLICY_SINK) __stcs(sink4, out);
            }
        }
    }

    // Elements past the last whole 16-byte unit: 4-byte accesses, same sites and policy.
    if (blockIdx.x == 0 && threadIdx.x < 32 && (n & 3)) {
        const size_t i = n4 * 4 + lane;
        const bool on = i < n;
        bool ob = true, oc = true, oa = true;
        if constexpr (GUARD) {
            if (on) {
                ob = lane_check(T, pg, (uint64_t)(b + i), 4, kSiteB, ll);
                if constexpr (kTriad) oc = lane_check(T, pg, (uint64_t)(c + i), 4, kSiteC, ll);
                oa = lane_check(T, pg, (uint64_t)(a + i), 4, kSiteA, ll);
            }
        }
        if (on) {
            const float *zero = reinterpret_cast<const float *>(T.zero_page);
            float vb1 = *((ob || kLoadAlways) ? b + i : zero);
            float vc1 = kTriad ? *((oc || kLoadAlways) ? c + i : zero) : 0.f;
            float out = op1<OP>(s, vb1, vc1);
            if (oa || kLoadAlways) a[i] = out;
            else if constexpr (POLICY == AGILE_POLICY_SINK) *reinterpret_cast<float *>(T.sink_page) = out;
        }
    }
    if constexpr (GUARD) agile::block_log_flush(log, ll);
}

template <int OP, bool GUARD, bool SMEM, int POLICY>
int launch(const agile_dev_table_t &T, float *a, const float *b, const float *c, size_t n,
           float s, LogDev *log, cudaStream_t st, uint32_t smem) {
    size_t n4 = n >> 2;
    size_t want = (n4 + kThreads - 1) / kThreads;
    size_t cap = (size_t)agile::sm_count() * 2;
    unsigned blocks = (unsigned)(want < 1 ? 1 : want > cap ? cap : want);
    k_stream<OP, GUARD, SMEM, POLICY><<<blocks, kThreads, (GUARD && SMEM) ? smem : 0, st>>>(
        T, a, b, c, n, s, log);
    AGILE_CUDA_TRY(cudaGetLastError());
    return AGILE_OK;
}

template <int OP>
int dispatch(const agile_dev_table_t *tbl, float *a, const float *b, const float *c, size_t n,
             float s, int policy, LogDev *log, cudaStream_t st) {
    if (tbl == nullptr) {
        agile_dev_table_t none = {};
        return launch<OP, false, false, AGILE_POLICY_REPORT>(none, a, b, c, n, s, nullptr, st, 0);
    }
    const uint64_t map_bytes = ((tbl->npages + 1) * 4 + 15) & ~15ull;
    const bool smem = tbl->npages > 0 && map_bytes <= kSmemMax;
    const uint32_t sb = (uint32_t)map_bytes;
    switch (policy) {
        case AGILE_POLICY_POISON:
            return smem ? launch<OP, true, true, AGILE_POLICY_POISON>(*tbl, a, b, c, n, s, log, st, sb)
                        : launch<OP, true, false, AGILE_POLICY_POISON>(*tbl, a, b, c, n, s, log, st, 0);
        case AGILE_POLICY_SINK:
            return smem ? launch<OP, true, true, AGILE_POLICY_SINK>(*tbl, a, b, c, n, s, log, st, sb)
                        : launch<OP, true, false, AGILE_POLICY_SINK>(*tbl, a, b, c, n, s, log, st, 0);
        case AGILE_POLICY_REPORT:
            return smem ? launch<OP, true, true, AGILE_POLICY_REPORT>(*tbl, a, b, c, n, s, log, st, sb)
                        : launch<OP, true, false, AGILE_POLICY_REPORT>(*tbl, a, b, c, n, s, log, st, 0);
        default:
            return AGILE_ERR_INVALID_ARG;
    }
}

}  // namespace

extern "C" int agile_stream_launch(int op, const agile_dev_table_t *tbl, float *d_a,
                                   const float *d_b, const float *d_c, size_t n, float s,
                                   int policy, void *d_log, void *stream) {
    if (op < AGILE_OP_COPY || op > AGILE_OP_TRIAD) return AGILE_ERR_INVALID_ARG;
    if (policy < AGILE_POLICY_POISON || policy > AGILE_POLICY_REPORT) return AGILE_ERR_INVALID_ARG;
    if (n == 0) return AGILE_OK;
    if (d_a == nullptr || d_b == nullptr || (op == AGILE_OP_TRIAD && d_c == nullptr))
        return AGILE_ERR_INVALID_ARG;
    if (((uintptr_t)d_a & 15) || ((uintptr_t)d_b & 15) || (op == AGILE_OP_TRIAD && ((uintptr_t)d_c & 15)))
        return AGILE_ERR_ALIGN;
    if (d_log != nullptr && ((uintptr_t)d_log & 15) != 0) return AGILE_ERR_ALIGN;
    LogDev *log = (LogDev *)d_log;
    cudaStream_t st = (cudaStream_t)stream;
    const float *c = op == AGILE_OP_TRIAD ? d_c : d_b;
    switch (op) {
        case AGILE_OP_COPY: return dispatch<AGILE_OP_COPY>(tbl, d_a, d_b, c, n, s, policy, log, st);
        case AGILE_OP_SCALE: return dispatch<AGILE_OP_SCALE>(tbl, d_a, d_b, c, n, s, policy, log, st);
        default: return dispatch<AGILE_OP_TRIAD>(tbl, d_a, d_b, c, n, s, policy, log, st);
    }
}
