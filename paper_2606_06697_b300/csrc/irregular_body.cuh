// Guarded irregular bodies shared by the standalone kernels and the batched persistent
// kernel: gather out[i] = T[idx[i]], scatter T[idx[i]] = (float)(idx[i] & 0xFFFFFF),
// histogram bins[idx[i]] += 1, with int64 element offsets an untrusted kernel could aim
// anywhere.
//
// Each lane takes four consecutive elements: the index array is read as two 16-byte
// loads (sites 0 and 1) and the output stored as one 16-byte store (site 3), contiguous
// across the warp, so one warp-uniform span check decides them; the four element
// accesses (site 2) go to data-dependent addresses and are checked per lane -- a page-map
// lookup, and a binary search only on mixed pages. The n mod 4 tail elements use an
// 8-byte index load, the element access and a 4-byte store. Each thread keeps its
// smallest violation in a LaneLog.
#pragma once

#include "guard_device.cuh"

namespace agile {

__device__ __forceinline__ bool lane_check(const TView &V, uint64_t a, uint32_t w, uint32_t site,
                                           LaneLog &ll) {
    uint32_t rid;
    const uint32_t v = classify(V, a, w, &rid);
    if (v == AGILE_ALLOW) return true;
    ll.note(a, pack_info(site, v, w, rid), a);
    return false;
}

// REMAP_OR (Sec. V-E remap_or, made safe as the paper asks): a denied access moves to its
// address with the table's mask ORed in, if that access is allowed. Returns the address to
// use for a denied access under POLICY, or 0 for "drop it / read the zero page".
template <int POLICY>
__device__ __forceinline__ uint64_t remapped(const TView &V, const agile_dev_table_t &T,
                                             uint64_t a, uint32_t w) {
    if constexpr (POLICY != AGILE_POLICY_REMAP_OR) {
        return 0ull;
    } else {
        const uint64_t a2 = a | T.remap_or;
        uint32_t rid;
        return classify(V, a2, w, &rid) == AGILE_ALLOW ? a2 : 0ull;
    }
}

__device__ __forceinline__ void red_add1(void *p) {
    asm volatile("red.global.add.u32 [%0], 1;" ::"l"(p) : "memory");
}

template <int KIND, int POLICY>
__device__ __forceinline__ float element(const TView &V, float *addr, bool ok, int64_t e,
                                         const agile_dev_table_t &T) {
    constexpr bool kAlways = POLICY == AGILE_POLICY_REPORT;
    if constexpr (POLICY == AGILE_POLICY_REMAP_OR) {
        if (!ok) {
            const uint64_t a2 = remapped<POLICY>(V, T, (uint64_t)addr, 4);
            ok = a2 != 0;
            if (ok) addr = reinterpret_cast<float *>(a2);
        }
    }
    if constexpr (KIND == AGILE_IRR_GATHER) {
        // Read-only load with a 64-byte L2 fetch hint: for uniform random elements it
        // measured 3% faster than the default (256 B hint: 4% slower; .cg/.ca/.cs: no change)
        const float *p = (ok || kAlways) ? addr : reinterpret_cast<const float *>(T.zero_page);
        float v;
        asm volatile("ld.global.nc.L2::64B.f32 %0, [%1];" : "=f"(v) : "l"(p));
        return v;
    } else if constexpr (KIND == AGILE_IRR_SCATTER) {
        const float f = (float)((uint64_t)e & 0xFFFFFFu);
        if (ok || kAlways) *addr = f;
        else if constexpr (POLICY == AGILE_POLICY_SINK) *reinterpret_cast<float *>(T.sink_page) = f;
        return 0.f;
    } else {
        // a reduction with no return value (red), so the lane does not wait for it
        if (ok || kAlways) red_add1(addr);
        else if constexpr (POLICY == AGILE_POLICY_SINK) red_add1(T.sink_page);
        return 0.f;
    }
}

// Source of a guarded load: the access itself, its remapped address, or the zero page.
template <int POLICY, typename P>
__device__ __forceinline__ const P *load_src(const TView &V, const agile_dev_table_t &T,
                                             const P *p, bool ok, uint32_t w) {
    if (ok || POLICY == AGILE_POLICY_REPORT) return p;
    const uint64_t a2 = remapped<POLICY>(V, T, (uint64_t)p, w);
    return a2 ? reinterpret_cast<const P *>(a2) : reinterpret_cast<const P *>(T.zero_page);
}

// A lane's group after its index loads: the four element offsets and whether the
// output store is allowed.
struct IrrGroup {
    int64_t e[4];
    size_t u;
    bool act, oko;
};

// First half of a group (units u0 .. u0+31, one per lane, clipped to n4): the span checks
// and the two 16-byte index loads. Warp-collective only in its uniform span checks;
// `spans` off means every index/output access is checked per lane.
template <int KIND, bool GUARD, int POLICY>
__device__ __forceinline__ IrrGroup irregular_load(const TView &V, const agile_dev_table_t &T,
                                                   const int64_t *idx, float *out, size_t u0,
                                                   size_t n4, LaneLog &ll, bool spans) {
    constexpr bool kGather = KIND == AGILE_IRR_GATHER;
    const longlong2 *idx2 = reinterpret_cast<const longlong2 *>(idx);
    float4 *out4 = reinterpret_cast<float4 *>(out);
    IrrGroup G;
    G.u = u0 + (threadIdx.x & 31);
    G.act = G.u < n4;
    G.oko = true;
    bool ok0 = true, ok1 = true;
    if constexpr (GUARD) {
        // A warp's span that stays inside one all-user block is decided by one bitmap word
        // (shared memory when staged); other spans by the page map.
        const bool full = spans && u0 + 32 <= n4;
        const uint64_t si = (uint64_t)(idx2 + 2 * u0);
        const bool fast_i = full && (block_user_fast(V, si, 1024, user_bits(V, si)) ||
                                     span_allowed(V, si, 1024));
        if (!fast_i && G.act) {
            ok0 = lane_check(V, (uint64_t)(idx2 + 2 * G.u), 16, 0, ll);
            ok1 = lane_check(V, (uint64_t)(idx2 + 2 * G.u + 1), 16, 1, ll);
        }
        if constexpr (kGather) {
            const uint64_t so = (uint64_t)(out4 + u0);
            const bool fast_o = full && (block_user_fast(V, so, 512, user_bits(V, so)) ||
                                         span_allowed(V, so, 512));
            if (!fast_o && G.act) G.oko = lane_check(V, (uint64_t)(out4 + G.u), 16, 3, ll);
        }
    }
    longlong2 p0 = {0, 0}, p1 = {0, 0};
    if (G.act) {
        p0 = __ldg(load_src<POLICY>(V, T, idx2 + 2 * G.u, ok0, 16));
        p1 = __ldg(load_src<POLICY>(V, T, idx2 + 2 * G.u + 1, ok1, 16));
    }
    G.e[0] = p0.x; G.e[1] = p0.y; G.e[2] = p1.x; G.e[3] = p1.y;
    return G;
}

// How the four element accesses of a lane read the all-user bitmap: each lane its own
// word (FAST_BITMAP), or once per group of lanes whose elements share a bitmap block, found
// with __match_any_sync, the group's leader reading the word and __shfl_sync handing it
// to the others (FAST_MATCH). Both decide the same accesses; the second is kept as a
// measured alternative.
enum : int { FAST_BITMAP = 0, FAST_MATCH = 1 };

// Second half: the four element accesses and gather's output store. Per lane; with
// FAST_MATCH called by all 32 lanes of the warp together.
template <int KIND, bool GUARD, int POLICY, int FAST = FAST_BITMAP>
__device__ __forceinline__ void irregular_apply(const TView &V, const agile_dev_table_t &T,
                                                const IrrGroup &G, float *base, float *out,
                                                LaneLog &ll) {
    constexpr bool kAlways = POLICY == AGILE_POLICY_REPORT;
    constexpr bool kGather = KIND == AGILE_IRR_GATHER;
    unsigned am = kFull;                  // lanes with a group (FAST_MATCH)
    if constexpr (GUARD && FAST == FAST_MATCH) am = __ballot_sync(kFull, G.act);
    if (!G.act) return;
    float4 *out4 = reinterpret_cast<float4 *>(out);
    float *addr[4];
    bool ok[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        addr[k] = reinterpret_cast<float *>((uint64_t)base + 4 * (uint64_t)G.e[k]);
        ok[k] = true;
    }
    if constexpr (GUARD) {
        // The four all-user bitmap words are read before any is used, so their latencies
        // overlap; an element in an all-user block is then decided without a branch, the
        // rest (blocks that are not all user, denials) by the full classification.
        uint32_t pe[4];
        if constexpr (FAST == FAST_MATCH) {
            const uint32_t lane = threadIdx.x & 31;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint64_t k0 = ((uint64_t)addr[k] - V.lo) >> V.ulg;
                const uint32_t blk = k0 < V.un ? (uint32_t)k0 : V.un;
                const unsigned peers = __match_any_sync(am, blk);
                const int leader = __ffs(peers) - 1;
                uint32_t w = 0;
                if ((int)lane == leader) w = V.ubits[blk >> 5];
                w = __shfl_sync(am, w, leader);
                pe[k] = w >> (blk & 31);
            }
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) pe[k] = user_bits(V, (uint64_t)addr[k]);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) ok[k] = block_user_fast(V, (uint64_t)addr[k], 4, pe[k]);
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (!ok[k]) ok[k] = lane_check(V, (uint64_t)addr[k], 4, 2, ll);
    }
    float v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = element<KIND, POLICY>(V, addr[k], ok[k], G.e[k], T);
    if constexpr (kGather) {
        const float4 o = make_float4(v[0], v[1], v[2], v[3]);
        if (G.oko || kAlways) {
            __stcs(out4 + G.u, o);
        } else if constexpr (POLICY == AGILE_POLICY_SINK) {
            __stcs(reinterpret_cast<float4 *>(T.sink_page), o);
        } else if constexpr (POLICY == AGILE_POLICY_REMAP_OR) {
            const uint64_t a2 = remapped<POLICY>(V, T, (uint64_t)(out4 + G.u), 16);
            if (a2) __stcs(reinterpret_cast<float4 *>(a2), o);
        }
    }
}

// One group: load, then apply. Warp-collective in its uniform span checks (and, with
// FAST_MATCH, in the bitmap reads).
template <int KIND, bool GUARD, int POLICY, int FAST = FAST_BITMAP>
__device__ __forceinline__ void irregular_group(const TView &V, const agile_dev_table_t &T,
                                                const int64_t *idx, float *base, float *out,
                                                size_t u0, size_t n4, LaneLog &ll, bool spans) {
    const IrrGroup G = irregular_load<KIND, GUARD, POLICY>(V, T, idx, out, u0, n4, ll, spans);
    irregular_apply<KIND, GUARD, POLICY, FAST>(V, T, G, base, out, ll);
}

// The n mod 4 tail elements, lanes 0..2 of one warp.
template <int KIND, bool GUARD, int POLICY>
__device__ __forceinline__ void irregular_tail(const TView &V, const agile_dev_table_t &T,
                                               const int64_t *idx, float *base, float *out,
                                               size_t n, LaneLog &ll) {
    constexpr bool kAlways = POLICY == AGILE_POLICY_REPORT;
    const size_t i = (n >> 2) * 4 + (threadIdx.x & 31);
    if (i >= n) return;
    const bool oki = !GUARD || lane_check(V, (uint64_t)(idx + i), 8, 0, ll);
    const int64_t e = *load_src<POLICY>(V, T, idx + i, oki, 8);
    float *addr = reinterpret_cast<float *>((uint64_t)base + 4 * (uint64_t)e);
    const bool ok = !GUARD || lane_check(V, (uint64_t)addr, 4, 2, ll);
    const float v = element<KIND, POLICY>(V, addr, ok, e, T);
    if constexpr (KIND == AGILE_IRR_GATHER) {
        const bool oko = !GUARD || lane_check(V, (uint64_t)(out + i), 4, 3, ll);
        if (oko || kAlways) {
            out[i] = v;
        } else if constexpr (POLICY == AGILE_POLICY_SINK) {
            *reinterpret_cast<float *>(T.sink_page) = v;
        } else if constexpr (POLICY == AGILE_POLICY_REMAP_OR) {
            const uint64_t a2 = remapped<POLICY>(V, T, (uint64_t)(out + i), 4);
            if (a2) *reinterpret_cast<float *>(a2) = v;
        }
    }
}

}  // namespace agile
