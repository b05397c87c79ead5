// Device core of the kernel memory guard (Sec. V-E: an address-range check before every
// global access; Sec. IV-E: the user / protected / MMIO classification rule).
//
// Table layout in device memory (one caller-owned buffer, written by the upload):
//   [0, 128)    agile_dev_table_t header (absolute device pointers)
//   [128, 192)  zero page: denied loads under SINK/POISON read these 64 zero bytes
//   [192, 256)  sink page: denied stores under SINK land here
//   [256, ...)  page map, npages + 1 u32 entries, padded to 256 bytes
//   then base[n] u64, end[n] u64, kind[n] u32, id[n] u32 (ascending base), each 256-aligned
//
// Two-level lookup. The window [lo, lo + npages*G) is cut into pages of G bytes. Entry p
// holds in bits 0-29 the index f_p of the first range whose end lies above the page's
// first byte (n if none) and in bits 30-31 what the page holds:
//   USER  - every byte of the page is inside user range f_p
//   HOLE  - no range touches the page
//   DENY  - every byte of the page is inside protected/MMIO range f_p
//   MIXED - anything else
// An access that stays inside one USER/HOLE/DENY page is decided from the entry alone.
// Otherwise the last range starting at or below the access is found by a branchless
// binary search over base[f_p, f_{p+1} + 1) -- only those ranges can start at or below
// an address inside page p and still reach it -- and the ranges the access touches are
// walked in address order (at most `width` of them), applying the class order
// MMIO > PROTECTED > STRADDLE. Accesses outside the window search the whole table.
#pragma once

#include <stdint.h>

#include "agile_guard.h"

namespace agile {

enum : uint32_t { PG_MIXED = 0, PG_USER = 1, PG_HOLE = 2, PG_DENY = 3 };
constexpr uint32_t kIdxMask = 0x3FFFFFFFu;
constexpr uint32_t kNoRange = 0xFFFFFFFFu;
constexpr unsigned kFull = 0xFFFFFFFFu;

constexpr size_t kHeaderBytes = 128;
constexpr size_t kZeroOff = 128;
constexpr size_t kSinkOff = 192;
constexpr size_t kPageOff = 256;

// Device log, AGILE_LOG_BYTES bytes, 16-byte aligned. Two 128-bit words are kept at their
// lexicographic minimum by compare-and-swap: first = (key, info) and where = (key, addr),
// so both hold the fields of the violation with the smallest key whatever the schedule.
struct LogDev {
    unsigned long long first_key, first_info;
    unsigned long long where_key, where_addr;
    unsigned long long count;
    uint32_t client, status;
    unsigned long long pad[2];
};
static_assert(sizeof(LogDev) == AGILE_LOG_BYTES, "log layout");

__host__ __device__ inline unsigned long long pack_info(uint32_t site, uint32_t verdict,
                                                        uint32_t width, uint32_t rid) {
    return ((unsigned long long)(site & 0xFFFFu) << 48) |
           ((unsigned long long)(verdict & 0xFFu) << 40) |
           ((unsigned long long)(width & 0xFFu) << 32) | rid;
}

// ------------------------------------------------------------------ classification

__device__ __forceinline__ uint32_t deny_of_kind(uint32_t kind) {
    return kind == AGILE_MMIO ? AGILE_DENY_MMIO
         : kind == AGILE_PROTECTED ? AGILE_DENY_PROTECTED : AGILE_DENY_STRADDLE;
}

// Search ranges [lo_i, hi_i) for the last one starting at or below a, then walk.
static __device__ __noinline__ uint32_t classify_search(const agile_dev_table_t &T, uint32_t lo_i,
                                                 uint32_t hi_i, uint64_t a, uint64_t w,
                                                 uint32_t *rid) {
    uint32_t b = lo_i, len = hi_i - lo_i;
    while (len > 0) {                       // b = first index in [lo_i, hi_i) with base > a
        uint32_t half = len >> 1;
        bool le = __ldg(T.base + b + half) <= a;
        b = le ? b + half + 1 : b;
        len = le ? len - half - 1 : half;
    }
    uint32_t first = b;
    if (b > lo_i) {
        uint32_t j = b - 1;
        uint64_t e = __ldg(T.end + j);
        if (e > a) {
            if (__ldg(T.kind + j) == AGILE_USER && a + w <= e) {
                *rid = __ldg(T.id + j);
                return AGILE_ALLOW;
            }
            first = j;
        }
    }
    uint32_t best = 3, bj = 0;              // rank: 0 MMIO, 1 PROTECTED, 2 USER
    for (uint32_t k = first; k < T.n; ++k) {
        if (__ldg(T.base + k) >= a + w) break;
        uint32_t kd = __ldg(T.kind + k);
        uint32_t r = kd == AGILE_MMIO ? 0u : kd == AGILE_PROTECTED ? 1u : 2u;
        if (r < best) { best = r; bj = k; }
    }
    if (best == 3) { *rid = kNoRange; return AGILE_DENY_UNMAPPED; }
    *rid = __ldg(T.id + bj);
    return best == 0 ? AGILE_DENY_MMIO : best == 1 ? AGILE_DENY_PROTECTED : AGILE_DENY_STRADDLE;
}

// Verdict of [a, a + w) for 1 <= w; pg is the page map (shared or global memory).
__device__ __forceinline__ uint32_t classify(const agile_dev_table_t &T, const uint32_t *pg,
                                             uint64_t a, uint64_t w, uint32_t *rid) {
    if (w == 0 || a > ~0ull - w) { *rid = kNoRange; return AGILE_DENY_INVALID; }
    uint64_t off = a - T.lo;
    uint64_t p = off >> T.log2_page;
    uint32_t lo_i = 0, hi_i = T.n;
    if (p < T.npages) {
        uint32_t e = pg[p];
        uint32_t f = e & kIdxMask, ty = e >> 30;
        uint64_t G = 1ull << T.log2_page;
        if ((off & (G - 1)) + w <= G) {
            if (ty == PG_USER) { *rid = kNoRange; return AGILE_ALLOW; }
            if (ty == PG_HOLE) { *rid = kNoRange; return AGILE_DENY_UNMAPPED; }
            if (ty == PG_DENY) { *rid = __ldg(T.id + f); return deny_of_kind(__ldg(T.kind + f)); }
        }
        uint32_t f2 = pg[p + 1] & kIdxMask;
        lo_i = f;
        hi_i = f2 + 1 < T.n ? f2 + 1 : T.n;
    }
    return classify_search(T, lo_i, hi_i, a, w, rid);
}

// True when [a, a + bytes) lies inside one USER page: every access inside it is allowed.
__device__ __forceinline__ bool span_in_user_page(const agile_dev_table_t &T, const uint32_t *pg,
                                                  uint64_t a, uint64_t bytes) {
    uint64_t off = a - T.lo;
    uint64_t p = off >> T.log2_page;
    if (p >= T.npages) return false;
    uint64_t G = 1ull << T.log2_page;
    return (pg[p] >> 30) == PG_USER && (off & (G - 1)) + bytes <= G;
}

// ------------------------------------------------------------------ violation log

__device__ __forceinline__ void cas128(unsigned long long *p, unsigned long long cmp_lo,
                                       unsigned long long cmp_hi, unsigned long long new_lo,
                                       unsigned long long new_hi, unsigned long long &old_lo,
                                       unsigned long long &old_hi) {
    asm volatile(
        "{\n\t.reg .b128 c, s, d;\n\t"
        "mov.b128 c, {%2, %3};\n\t"
        "mov.b128 s, {%4, %5};\n\t"
        "atom.global.cas.b128 d, [%6], c, s;\n\t"
        "mov.b128 {%0, %1}, d;\n\t}"
        : "=l"(old_lo), "=l"(old_hi)
        : "l"(cmp_lo), "l"(cmp_hi), "l"(new_lo), "l"(new_hi), "l"(p)
        : "memory");
}

// Lower the 128-bit word at p to (k, v) if that is lexicographically smaller. Each failed
// exchange sees a strictly smaller word, so the loop ends; the bound is a backstop.
__device__ inline void cas_min128(unsigned long long *p, unsigned long long k,
                                  unsigned long long v, uint32_t *status) {
    unsigned long long ok = *(volatile unsigned long long *)p;
    unsigned long long ov = *(volatile unsigned long long *)(p + 1);
    for (int it = 0; it < (1 << 16); ++it) {
        if (!(k < ok || (k == ok && v < ov))) return;
        unsigned long long rk, rv;
        cas128(p, ok, ov, k, v, rk, rv);
        if (rk == ok && rv == ov) return;
        ok = rk;
        ov = rv;
    }
    atomicOr(status, AGILE_LOG_STATUS_TIMEOUT);
}

// Per-thread running minimum of the violations it has seen.
struct LaneLog {
    uint32_t cnt = 0;
    unsigned long long key = ~0ull, info = ~0ull, addr = 0;
    __device__ __forceinline__ void note(unsigned long long k, unsigned long long i,
                                         unsigned long long a) {
        ++cnt;
        if (k < key || (k == key && i < info)) { key = k; info = i; addr = a; }
    }
};

__device__ __forceinline__ void min3_shfl(unsigned long long &k, unsigned long long &v,
                                          unsigned long long &a) {
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        unsigned long long k2 = __shfl_xor_sync(kFull, k, o);
        unsigned long long v2 = __shfl_xor_sync(kFull, v, o);
        unsigned long long a2 = __shfl_xor_sync(kFull, a, o);
        if (k2 < k || (k2 == k && v2 < v)) { k = k2; v = v2; a = a2; }
    }
}

// Block-collective, called once by every thread at the end of a kernel: the block's
// violations are reduced to one count and one smallest record in shared memory, and one
// thread updates the log. One global update per block keeps the log address cold.
__device__ inline void block_log_flush(LogDev *L, const LaneLog &ll) {
    __shared__ unsigned long long s_key[32], s_info[32], s_addr[32];
    __shared__ uint32_t s_cnt[32];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long k = ll.cnt ? ll.key : ~0ull, v = ll.cnt ? ll.info : ~0ull, a = ll.addr;
    min3_shfl(k, v, a);
    uint32_t c = __reduce_add_sync(kFull, ll.cnt);
    if (lane == 0) { s_key[warp] = k; s_info[warp] = v; s_addr[warp] = a; s_cnt[warp] = c; }
    __syncthreads();
    if (warp == 0) {
        const uint32_t nw = (blockDim.x + 31) >> 5;
        k = lane < nw ? s_key[lane] : ~0ull;
        v = lane < nw ? s_info[lane] : ~0ull;
        a = lane < nw ? s_addr[lane] : 0;
        unsigned long long total = lane < nw ? s_cnt[lane] : 0;
        min3_shfl(k, v, a);
#pragma unroll
        for (int o = 16; o; o >>= 1) total += __shfl_xor_sync(kFull, total, o);
        if (lane == 0 && total != 0 && L != nullptr) {
            atomicAdd(&L->count, total);
            cas_min128(&L->first_key, k, v, &L->status);
            cas_min128(&L->where_key, k, a, &L->status);
        }
    }
}

// ------------------------------------------------------------------ page-map staging

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait on an mbarrier phase: gives up after ~0.25 s or 2^24 polls.
__device__ inline bool mbar_wait(uint32_t bar, uint32_t phase) {
    unsigned long long t0 = global_ns();
    for (uint32_t it = 0; it < (1u << 24); ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(phase)
            : "memory");
        if (done) return true;
        if ((it & 255) == 255 && global_ns() - t0 > 250000000ull) return false;
    }
    return false;
}

// Copy the page map into shared memory with one bulk copy (TMA, non-multicast) completed
// on an mbarrier. Every thread of the block calls it. Returns the map to use: the shared
// copy, or -- if the wait gave up -- the global one (results stay exact; the log, when
// present, is flagged).
__device__ inline const uint32_t *stage_page_map(const agile_dev_table_t &T, uint32_t *s_page,
                                                 unsigned long long *s_bar, LogDev *log) {
    uint32_t bytes = (uint32_t)(((T.npages + 1) * 4 + 15) & ~15ull);
    uint32_t bar = smem_addr(s_bar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                     : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
            ::"r"(smem_addr(s_page)), "l"(T.page), "r"(bytes), "r"(bar)
            : "memory");
    }
    if (mbar_wait(bar, 0)) return s_page;
    if (log != nullptr && threadIdx.x == 0) atomicOr(&log->status, AGILE_LOG_STATUS_TIMEOUT);
    mbar_wait(bar, 0);                      // let the copy in flight land before moving on
    return T.page;
}

}  // namespace agile
