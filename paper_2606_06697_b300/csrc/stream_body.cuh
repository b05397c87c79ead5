// Guarded streaming bodies shared by the standalone kernels and the batched persistent
// kernel: COPY a = b, SCALE a = s*b, TRIAD a = b + s*c (one fused multiply-add).
//
// Work is cut into warp tiles of 32*U 16-byte units (U = 4: 2 KiB per array); lane l
// handles units l, l+32, ..., l+32(U-1), so every access is coalesced. Before a tile the warp checks each
// array's 2 KiB span once (span_allowed: first and last byte in all-user pages of the
// same allocation, else the span classified as one access). Only a tile whose spans are
// not all allowed takes the per-access path (slow_tile, out of line), where each lane
// classifies its own accesses and the policy applies: POISON and SINK send denied loads
// to the table's zero page; POISON drops denied stores, SINK sends them to the sink page;
// REPORT lets every access through. Violations (key = (address, site)) go to per-warp
// shared-memory slots.
#pragma once

#include "guard_device.cuh"

namespace agile {

constexpr int kStreamU = 4;                         // default units per lane per warp tile
constexpr uint32_t kStreamTileUnits = 32 * kStreamU;

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
    const uint32_t v = classify(V, a, w, &rid);
    if (v == AGILE_ALLOW) return true;
    ll.note(a, pack_info(site, v, w, rid), a);
    return false;
}

// Per-access path for one warp tile (units u0 .. u0+32U-1 clipped to n4; for the n mod 4
// tail, the lane's element is 4*n4 + lane with 4-byte accesses). Warp-collective.
// Applies the policy and logs into the warp's slot.
template <int OP, int POLICY, bool TAIL, int U = kStreamU>
static __device__ __noinline__ void slow_tile(const TView &V, const agile_dev_table_t &T, float *a,
                                       const float *b, const float *c, size_t u0, size_t n4,
                                       size_t n, float s, WarpSlots &S) {
    constexpr bool kTriad = OP == AGILE_OP_TRIAD;
    constexpr uint32_t kSiteB = 0, kSiteC = 1, kSiteA = kTriad ? 2 : 1;
    constexpr bool kAlways = POLICY == AGILE_POLICY_REPORT;
    const uint32_t lane = threadIdx.x & 31;
    LaneLog ll;
    ll.log = S.log;
    if constexpr (!TAIL) {
        const float4 *b4 = reinterpret_cast<const float4 *>(b);
        const float4 *c4 = reinterpret_cast<const float4 *>(c);
        float4 *a4 = reinterpret_cast<float4 *>(a);
        const float4 *zero4 = reinterpret_cast<const float4 *>(T.zero_page);
#pragma unroll 1
        for (int k = 0; k < U; ++k) {
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
    warp_note(S, ll);
}

// One warp tile t (units t*32U .. t*32U+32U-1, clipped to n4): the span checks when
// `spans` is set, else straight to the per-access path. Warp-collective.
template <int OP, bool GUARD, int POLICY, int U = kStreamU>
__device__ __forceinline__ void stream_warp_tile(const TView &V, const agile_dev_table_t &T,
                                                 float *a, const float *b, const float *c,
                                                 size_t t, size_t n4, size_t n, float s,
                                                 WarpSlots &S, bool spans) {
    constexpr bool kTriad = OP == AGILE_OP_TRIAD;
    const float4 *b4 = reinterpret_cast<const float4 *>(b);
    const float4 *c4 = reinterpret_cast<const float4 *>(c);
    float4 *a4 = reinterpret_cast<float4 *>(a);
    const uint32_t lane = threadIdx.x & 31;
    constexpr uint32_t kTile = 32 * U;
    const size_t u0 = t * kTile;
    bool fast = u0 + kTile <= n4;
    if constexpr (GUARD) {
        fast = fast && spans && span_allowed(V, (uint64_t)(b4 + u0), 16 * kTile) &&
               span_allowed(V, (uint64_t)(a4 + u0), 16 * kTile);
        if constexpr (kTriad)
            fast = fast && span_allowed(V, (uint64_t)(c4 + u0), 16 * kTile);
        if (!fast) {
            slow_tile<OP, POLICY, false, U>(V, T, a, b, c, u0, n4, n, s, S);
            return;
        }
    } else if (!fast) {                               // unguarded partial tile
#pragma unroll
        for (int k = 0; k < U; ++k) {
            const size_t u = u0 + 32 * k + lane;
            if (u < n4) __stcs(a4 + u, op4<OP>(s, __ldcs(b4 + u), kTriad ? __ldcs(c4 + u) : float4{}));
        }
        return;
    }
    float4 vb[U], vc[U];
#pragma unroll
    for (int k = 0; k < U; ++k) {
        vb[k] = __ldcs(b4 + u0 + 32 * k + lane);
        if constexpr (kTriad) vc[k] = __ldcs(c4 + u0 + 32 * k + lane);
        else vc[k] = vb[k];
    }
#pragma unroll
    for (int k = 0; k < U; ++k) __stcs(a4 + u0 + 32 * k + lane, op4<OP>(s, vb[k], vc[k]));
}

// The n mod 4 tail elements (4-byte accesses), by one warp.
template <int OP, bool GUARD, int POLICY>
__device__ __forceinline__ void stream_tail(const TView &V, const agile_dev_table_t &T, float *a,
                                            const float *b, const float *c, size_t n, float s,
                                            WarpSlots &S) {
    constexpr bool kTriad = OP == AGILE_OP_TRIAD;
    const size_t n4 = n >> 2;
    if constexpr (GUARD) {
        slow_tile<OP, POLICY, true>(V, T, a, b, c, n4, n4, n, s, S);
    } else {
        const size_t i = 4 * n4 + (threadIdx.x & 31);
        if (i < n) a[i] = op1<OP>(s, b[i], kTriad ? c[i] : 0.f);
    }
}

}  // namespace agile
