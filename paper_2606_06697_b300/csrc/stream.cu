// Streaming kernels with the guard fused in by hand: COPY a = b, SCALE a = s*b, TRIAD
// a = b + s*c (one fused multiply-add), fp32, 16-byte vector accesses (Sec. V-E: an
// address-range check before every global access, ordinary user-allocation accesses left
// on the normal path), and their unguarded twins.
//
// Guard placement. Work is cut into warp tiles of 128 16-byte units (2 KiB per array);
// lane l handles units l, l+32, l+64, l+96, so every access is coalesced. Before a tile,
// the warp checks each array's 2 KiB span once: if the pages of its first and last byte
// are all-user pages of the same allocation, the whole span lies inside that allocation
// and every access in it is allowed; otherwise the span is classified as one access.
// Only when a span is not allowed does the warp take the per-access path (out of line),
// where each lane classifies its own accesses and the policy applies: POISON and SINK
// send denied loads to the table's zero page; POISON drops denied stores, SINK sends
// them to the sink page; REPORT lets every access through. Denied accesses are logged
// with key (address, site) into per-warp shared-memory slots, reduced once per block.
#include <cuda_runtime.h>

#include "agile_internal.h"
#include "guard_device.cuh"

namespace {

using agile::LaneLog;
using agile::LogDev;
using agile::TView;
using agile::WarpSlots;

constexpr int kThreads = 512;
constexpr int kU = 4;                        // units per lane per tile
constexpr uint32_t kTileUnits = 32 * kU;     // 128 units = 2 KiB per array

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

__device__ __forceinline__ bool lane_ok(const TView &V, uint64_t a, uint32_t w, uint32_t site,
                                        LaneLog &ll) {
    uint32_t rid;
    const uint32_t v = agile::classify(V, a, w, &rid);
    if (v == AGILE_ALLOW) return true;
    ll.note(a, agile::pack_info(site, v, w, rid), a);
    return false;
}

// Per-access path for one warp tile (units u0 .. u0+127 clipped to n4; for the n mod 4
// tail, the lane's element is 4*n4 + lane with 4-byte accesses). Warp-collective.
// Applies the policy and logs into the warp's slot.
template <int OP, int POLICY, bool TAIL>
__device__ __noinline__ void slow_tile(const TView &V, const agile_dev_table_t &T, float *a,
                                       const float *b, const float *c, size_t u0, size_t n4,
                                       size_t n, float s, WarpSlots &S) {
    constexpr bool kTriad = OP == AGILE_OP_TRIAD;
    constexpr uint32_t kSiteB = 0, kSiteC = 1, kSiteA = kTriad ? 2 : 1;
    constexpr bool kAlways = POLICY == AGILE_POLICY_REPORT;
    const uint32_t lane = threadIdx.x & 31;
    LaneLog ll;
    if constexpr (!TAIL) {
        const float4 *b4 = reinterpret_cast<const float4 *>(b);
        const float4 *c4 = reinterpret_cast<const float4 *>(c);
        float4 *a4 = reinterpret_cast<float4 *>(a);
        const float4 *zero4 = reinterpret_cast<const float4 *>(T.zero_page);
#pragma unroll 1
        for (int k = 0; k < kU; ++k) {
            const size_t u = u0 + 32 * k + lane;
            if (u >= n4) continue;
            const bool okb = lane_ok(V, (uint64_t)(b4 + u), 16, kSiteB, ll);
            const bool okc = !kTriad || lane_ok(V, (uint64_t)(c4 + u), 16, kSiteC, ll);
            const bool oka = lane_ok(V, (uint64_t)(a4 + u), 16, kSiteA, ll);
            const float4 vb = __ldcs((okb || kAlways) ? b4 + u : zero4);
            const float4 vc = kTriad ? __ldcs((okc || kAlways) ? c4 + u : zero4) : vb;
            const float4 o = op4<OP>(s, vb, vc);
            if (oka || kAlways) __stcs(a4 + u, o);
            else if constexpr (POLICY == AGILE_POLICY_SINK) __stcs(reinterpret_cast<float4 *>(T.sink_page), o);
        }
    } else {
        const size_t i = 4 * n4 + lane;
        if (i < n) {
            const float *zero = reinterpret_cast<const float *>(T.zero_page);
            const bool okb = lane_ok(V, (uint64_t)(b + i), 4, kSiteB, ll);
            const bool okc = !kTriad || lane_ok(V, (uint64_t)(c + i), 4, kSiteC, ll);
            const bool oka = lane_ok(V, (uint64_t)(a + i), 4, kSiteA, ll);
            const float vb = *((okb || kAlways) ? b + i : zero);
            const float vc = kTriad ? *((okc || kAlways) ? c + i : zero) : 0.f;
            const float o = op1<OP>(s, vb, vc);
            if (oka || kAlways) a[i] = o;
            else if constexpr (POLICY == AGILE_POLICY_SINK) *reinterpret_cast<float *>(T.sink_page) = o;
        }
    }
    agile::warp_note(S, ll);
}

template <int OP, bool GUARD, int MODE, int POLICY>
__global__ void __launch_bounds__(kThreads, 2)
k_stream(const agile_dev_table_t T, float *__restrict__ a, const float *__restrict__ b,
         const float *__restrict__ c, size_t n, float s, LogDev *log) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned long long s_bar;
    __shared__ WarpSlots S;
    constexpr bool kTriad = OP == AGILE_OP_TRIAD;
    TView V{};
    if constexpr (GUARD) {
        agile::slots_init(S);
        __syncthreads();
        V = agile::stage_table<MODE>(T, smem, &s_bar, log);
    }

    const size_t n4 = n >> 2;
    const float4 *b4 = reinterpret_cast<const float4 *>(b);
    const float4 *c4 = reinterpret_cast<const float4 *>(c);
    float4 *a4 = reinterpret_cast<float4 *>(a);
    const uint32_t lane = threadIdx.x & 31;
    const size_t warp = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const size_t nwarps = ((size_t)gridDim.x * blockDim.x) >> 5;
    const size_t full_tiles = n4 / kTileUnits;
    const size_t tiles = (n4 + kTileUnits - 1) / kTileUnits;

    for (size_t t = warp; t < tiles; t += nwarps) {          // warp-uniform
        const size_t u0 = t * kTileUnits;
        bool fast = t < full_tiles;
        if constexpr (GUARD) {
            fast = fast && agile::span_allowed(V, (uint64_t)(b4 + u0), 16 * kTileUnits) &&
                   agile::span_allowed(V, (uint64_t)(a4 + u0), 16 * kTileUnits);
            if constexpr (kTriad)
                fast = fast && agile::span_allowed(V, (uint64_t)(c4 + u0), 16 * kTileUnits);
            if (!fast) {
                slow_tile<OP, POLICY, false>(V, T, a, b, c, u0, n4, n, s, S);
                continue;
            }
        } else if (!fast) {                                   // unguarded partial tile
#pragma unroll
            for (int k = 0; k < kU; ++k) {
                const size_t u = u0 + 32 * k + lane;
                if (u < n4) __stcs(a4 + u, op4<OP>(s, __ldcs(b4 + u), kTriad ? __ldcs(c4 + u) : float4{}));
            }
            continue;
        }
        float4 vb[kU], vc[kU];
#pragma unroll
        for (int k = 0; k < kU; ++k) {
            vb[k] = __ldcs(b4 + u0 + 32 * k + lane);
            if constexpr (kTriad) vc[k] = __ldcs(c4 + u0 + 32 * k + lane);
            else vc[k] = vb[k];
        }
#pragma unroll
        for (int k = 0; k < kU; ++k) __stcs(a4 + u0 + 32 * k + lane, op4<OP>(s, vb[k], vc[k]));
    }

    // Elements past the last whole 16-byte unit: 4-byte accesses by the last warp.
    if ((n & 3) && blockIdx.x == gridDim.x - 1 && (threadIdx.x >> 5) == (blockDim.x >> 5) - 1) {
        if constexpr (GUARD) {
            slow_tile<OP, POLICY, true>(V, T, a, b, c, n4, n4, n, s, S);
        } else {
            const size_t i = 4 * n4 + lane;
            if (i < n) a[i] = op1<OP>(s, b[i], kTriad ? c[i] : 0.f);
        }
    }
    if constexpr (GUARD) agile::slots_flush(log, S);
}

template <int OP, bool GUARD, int MODE, int POLICY>
int launch(const agile_dev_table_t &T, float *a, const float *b, const float *c, size_t n,
           float s, LogDev *log, cudaStream_t st) {
    const uint32_t smem = GUARD ? agile::stage_bytes(T, MODE) : 0;
    if (smem > 48 * 1024) {
        AGILE_CUDA_TRY(cudaFuncSetAttribute(k_stream<OP, GUARD, MODE, POLICY>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024));
    }
    const size_t tiles = ((n >> 2) + kTileUnits - 1) / kTileUnits;
    const size_t want = (tiles * 32 + kThreads - 1) / kThreads;
    const size_t cap = (size_t)agile::sm_count() * 2;
    const unsigned blocks = (unsigned)(want < 1 ? 1 : want > cap ? cap : want);
    k_stream<OP, GUARD, MODE, POLICY><<<blocks, kThreads, smem, st>>>(T, a, b, c, n, s, log);
    AGILE_CUDA_TRY(cudaGetLastError());
    return AGILE_OK;
}

template <int OP, int POLICY>
int by_mode(const agile_dev_table_t &T, float *a, const float *b, const float *c, size_t n,
            float s, LogDev *log, cudaStream_t st) {
    switch (agile::stage_mode(T, false)) {
        case agile::STAGE_PAGES: return launch<OP, true, agile::STAGE_PAGES, POLICY>(T, a, b, c, n, s, log, st);
        default: return launch<OP, true, agile::STAGE_NONE, POLICY>(T, a, b, c, n, s, log, st);
    }
}

template <int OP>
int dispatch(const agile_dev_table_t *tbl, float *a, const float *b, const float *c, size_t n,
             float s, int policy, LogDev *log, cudaStream_t st) {
    if (tbl == nullptr) {
        agile_dev_table_t none = {};
        return launch<OP, false, agile::STAGE_NONE, AGILE_POLICY_REPORT>(none, a, b, c, n, s, nullptr, st);
    }
    switch (policy) {
        case AGILE_POLICY_POISON: return by_mode<OP, AGILE_POLICY_POISON>(*tbl, a, b, c, n, s, log, st);
        case AGILE_POLICY_SINK: return by_mode<OP, AGILE_POLICY_SINK>(*tbl, a, b, c, n, s, log, st);
        case AGILE_POLICY_REPORT: return by_mode<OP, AGILE_POLICY_REPORT>(*tbl, a, b, c, n, s, log, st);
        default: return AGILE_ERR_INVALID_ARG;
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
