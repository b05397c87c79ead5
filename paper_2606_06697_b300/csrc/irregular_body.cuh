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

// Source of a guarded load: the access itself, its remapped address, or the zero page.
template <int POLICY, typename P>
__device__ __forceinline__ const P *load_src(const TView &V, const agile_dev_table_t &T,
                                             const P *p, bool ok, uint32_t w) {
    if (ok || POLICY == AGILE_POLICY_REPORT) return p;
    const uint64_t a2 = remapped<POLICY>(V, T, (uint64_t)p, w);
    return a2 ? reinterpret_cast<const P *>(a2) : reinterpret_cast<const P *>(T.zero_page);
}

// Units u0 .. u0+31 (one per lane, clipped to n4). Warp-collective only in its uniform
// span checks; `spans` off means every index/output access is checked per lane.
template <int KIND, bool GUARD, int POLICY>
__device__ __forceinline__ void irregular_group(const TView &V, const agile_dev_table_t &T,
                                                const int64_t *idx, float *base, float *out,
                                                size_t u0, size_t n4, LaneLog &ll, bool spans) {
    constexpr bool kAlways = POLICY == AGILE_POLICY_REPORT;
    constexpr bool kGather = KIND == AGILE_IRR_GATHER;
    const longlong2 *idx2 = reinterpret_cast<const longlong2 *>(idx);
    const longlong2 *zero2 = reinterpret_cast<const longlong2 *>(T.zero_page);
    float4 *out4 = reinterpret_cast<float4 *>(out);
    const size_t u = u0 + (threadIdx.x & 31);
    const bool act = u < n4;
    bool ok0 = true, ok1 = true, oko = true;
    if constexpr (GUARD) {
        // A warp's span that stays inside one all-user block is decided by one bitmap word
        // (shared memory when staged); other spans by the page map.
        const bool full = spans && u0 + 32 <= n4;
        const uint64_t si = (uint64_t)(idx2 + 2 * u0);
        const bool fast_i = full && (block_user_fast(V, si, 1024, user_bits(V, si)) ||
                                     span_allowed(V, si, 1024));
        if (!fast_i && act) {
            ok0 = lane_check(V, (uint64_t)(idx2 + 2 * u), 16, 0, ll);
            ok1 = lane_check(V, (uint64_t)(idx2 + 2 * u + 1), 16, 1, ll);
        }
        if constexpr (kGather) {
            const uint64_t so = (uint64_t)(out4 + u0);
            const bool fast_o = full && (block_user_fast(V, so, 512, user_bits(V, so)) ||
                                         span_allowed(V, so, 512));
            if (!fast_o && act) oko = lane_check(V, (uint64_t)(out4 + u), 16, 3, ll);
        }
    }
    if (!act) return;
    const longlong2 p0 = __ldg(load_src<POLICY>(V, T, idx2 + 2 * u, ok0, 16));
    const longlong2 p1 = __ldg(load_src<POLICY>(V, T, idx2 + 2 * u + 1, ok1, 16));
    (void)zero2;
    const int64_t e[4] = {p0.x, p0.y, p1.x, p1.y};
    float *addr[4];
    bool ok[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        addr[k] = reinterpret_cast<float *>((uint64_t)base + 4 * (uint64_t)e[k]);
        ok[k] = true;
    }
    if constexpr (GUARD) {
        // The four all-user bitmap words are read before any is used, so their latencies
        // overlap; an element in an all-user block is then decided without a branch, the
        // rest (blocks that are not all user, denials) by the full classification.
        uint32_t pe[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) pe[k] = user_bits(V, (uint64_t)addr[k]);
#pragma unroll
        for (int k = 0; k < 4; ++k) ok[k] = block_user_fast(V, (uint64_t)addr[k], 4, pe[k]);
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (!ok[k]) ok[k] = lane_check(V, (uint64_t)addr[k], 4, 2, ll);
    }
    float v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = element<KIND, POLICY>(V, addr[k], ok[k], e[k], T);
    if constexpr (kGather) {
        const float4 o = make_float4(v[0], v[1], v[2], v[3]);
        if (oko || kAlways) {
            __stcs(out4 + u, o);
        } else if constexpr (POLICY == AGILE_POLICY_SINK) {
            __stcs(reinterpret_cast<float4 *>(T.sink_page), o);
        } else if constexpr (POLICY == AGILE_POLICY_REMAP_OR) {
            const uint64_t a2 = remapped<POLICY>(V, T, (uint64_t)(out4 + u), 16);
            if (a2) __stcs(reinterpret_cast<float4 *>(a2), o);
        }
    }
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
