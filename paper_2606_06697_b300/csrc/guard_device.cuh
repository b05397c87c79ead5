// Device core of the kernel memory guard (Sec. V-E: an address-range check before every
// global access; Sec. IV-E: the user / protected / MMIO classification rule).
//
// Table layout in device memory (one caller-owned buffer, written by the upload):
//   [0, 256)    agile_dev_table_t header (absolute device pointers)
//   [256, 320)  zero page: denied loads under SINK/POISON read these 64 zero bytes
//   [320, 384)  sink page: denied stores under SINK land here
//   [384, ...)  page map, npages + 1 u32 entries, padded to 256 bytes
//   then base[n] u64, end[n] u64, kind[n] u32, id[n] u32 (ascending base), each 256-aligned,
//   the packed records (windows under 4 GiB), the all-user bitmap and the block class map
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

// Device log, AGILE_LOG_BYTES bytes, 16-byte aligned. Two 128-bit words are kept at their
// lexicographic minimum by compare-and-swap: first = (key, info) and where = (key, addr),
// so both hold the fields of the violation with the smallest key whatever the schedule.
// `list` is the device address of an attached bounded list (0: none) and `list_next` the
// list slots taken since it was attached.
struct LogDev {
    unsigned long long first_key, first_info;
    unsigned long long where_key, where_addr;
    unsigned long long count;
    uint32_t client, status;
    unsigned long long list, list_next;
};
static_assert(sizeof(LogDev) == AGILE_LOG_BYTES, "log layout");
static_assert(AGILE_LIST_HEADER_BYTES == 16 && AGILE_LIST_ENTRY_BYTES == 32, "list layout");

// Append one violation record to the log's bounded list, if one is attached: the slot
// comes from list_next, and the entry {key, addr, info, 0} is written when the slot is
// below the capacity in the list's header (later violations are only counted). Called on
// violation paths only.
__device__ __forceinline__ void list_append(LogDev *L, unsigned long long key,
                                            unsigned long long info, unsigned long long addr) {
    if (L == nullptr) return;
    const unsigned long long list = L->list;
    if (list == 0) return;
    const unsigned long long slot = atomicAdd(&L->list_next, 1ull);
    if (slot >= *reinterpret_cast<const unsigned long long *>(list)) return;
    ulonglong2 *e = reinterpret_cast<ulonglong2 *>(list + AGILE_LIST_HEADER_BYTES +
                                                   slot * AGILE_LIST_ENTRY_BYTES);
    e[0] = make_ulonglong2(key, addr);
    e[1] = make_ulonglong2(info, 0ull);
}


__host__ __device__ inline unsigned long long pack_info(uint32_t site, uint32_t verdict,
                                                        uint32_t width, uint32_t rid) {
    return ((unsigned long long)(site & 0xFFFFu) << 48) |
           ((unsigned long long)(verdict & 0xFFu) << 40) |
           ((unsigned long long)(width & 0xFFu) << 32) | rid;
}

// ------------------------------------------------------------------ classification

// The table as a kernel sees it: pointers into shared memory (staged copies) or global.
struct TView {
    uint64_t lo, npages;
    uint64_t gmask;             // page size - 1
    uint64_t last;              // last byte of the window (lo + npages*G - 1)
    uint32_t lg, n, steps;
    const uint32_t *page;
    const uint64_t *base, *end;
    const uint32_t *kind, *id;
    const uint4 *crange;        // {start - lo, last - lo, rank, id} (windows under 4 GiB), or NULL
    const uint32_t *ubits;      // all-user block bitmap (un + 1 bits, the last clear)
    uint32_t ulg, un;           // block size 2^ulg, blocks in the window
    const uint32_t *cmap;       // block class map (2 bits per block, cn + 1 blocks)
    uint32_t clg, cn;           // block size 2^clg, blocks in the window
    const uint2 *cdesc;         // open-block descriptors {block, payload}, 2^dlg slots, or NULL
    uint32_t dlg, dk1, dk2;     // their slot count (log2) and hash multipliers
};

__device__ __forceinline__ TView view_of(const agile_dev_table_t &T) {
    const uint64_t G = 1ull << T.log2_page;
    return TView{T.lo, T.npages, G - 1, T.lo + (T.npages << T.log2_page) - 1, T.log2_page, T.n,
                 T.search_steps, T.page, T.base, T.end, T.kind, T.id,
                 reinterpret_cast<const uint4 *>(T.crange), T.ubits, T.ubits_log2, T.ubits_n,
                 T.cmap, T.cmap_log2, T.cmap_n, reinterpret_cast<const uint2 *>(T.cdesc),
                 T.cdesc_log2, T.cdesc_k1, T.cdesc_k2};
}

__device__ __forceinline__ uint32_t deny_of_kind(uint32_t kind) {
    return kind == AGILE_MMIO ? AGILE_DENY_MMIO
         : kind == AGILE_PROTECTED ? AGILE_DENY_PROTECTED : AGILE_DENY_STRADDLE;
}

// After the search: b = first index with base > a among the slice that starts at lo_i.
// Decide from range b-1 (allowed if it is a user range holding all of [a, a+w)), else
// walk the ranges [a, a + w) touches in address order for the deny class.
__device__ __forceinline__ uint32_t decide(const TView &V, uint32_t lo_i, uint32_t b, uint64_t a,
                                          uint64_t w, uint32_t *rid) {
    uint32_t first = b;
    if (b > lo_i) {
        const uint32_t j = b - 1;
        const uint64_t e = V.end[j];
        if (e > a) {
            if (V.kind[j] == AGILE_USER && a + w <= e) { *rid = V.id[j]; return AGILE_ALLOW; }
            first = j;
        }
    }
    uint32_t best = 3, bj = 0;              // rank: 0 MMIO, 1 PROTECTED, 2 USER
    for (uint32_t k = first; k < V.n; ++k) {
        if (V.base[k] >= a + w) break;
        const uint32_t kd = V.kind[k];
        const uint32_t r = kd == AGILE_MMIO ? 0u : kd == AGILE_PROTECTED ? 1u : 2u;
        if (r < best) { best = r; bj = k; }
    }
    if (best == 3) { *rid = kNoRange; return AGILE_DENY_UNMAPPED; }
    *rid = V.id[bj];
    return best == 0 ? AGILE_DENY_MMIO : best == 1 ? AGILE_DENY_PROTECTED : AGILE_DENY_STRADDLE;
}

// Variable-length search over [lo_i, hi_i) (any slice; used outside the window).
__device__ __forceinline__ uint32_t search(const TView &V, uint32_t lo_i, uint32_t hi_i,
                                          uint64_t a, uint64_t w, uint32_t *rid) {
    uint32_t b = lo_i, len = hi_i - lo_i;
    while (len > 0) {                       // b = first index in [lo_i, hi_i) with base > a
        const uint32_t half = len >> 1;
        const bool le = V.base[b + half] <= a;
        b = le ? b + half + 1 : b;
        len = le ? len - half - 1 : half;
    }
    return decide(V, lo_i, b, a, w, rid);
}

// Verdict of [a, a + w), w >= 1 any size, fully inline. Inside the window the search
// runs a fixed number of branchless steps (the table's search_steps covers every page's
// slice), so lanes of a warp stay together; accesses wholly outside the window touch no
// range.
__device__ __forceinline__ uint32_t classify(const TView &V, uint64_t a, uint64_t w, uint32_t *rid) {
    if (w == 0 || a > ~0ull - w) { *rid = kNoRange; return AGILE_DENY_INVALID; }
    const uint64_t off = a - V.lo;
    const uint64_t p = off >> V.lg;
    if (p < V.npages) {
        const uint32_t e = V.page[p];
        const uint32_t f = e & kIdxMask, ty = e >> 30;
        if ((off & V.gmask) + w <= V.gmask + 1) {
            if (ty == PG_USER) { *rid = kNoRange; return AGILE_ALLOW; }
            if (ty == PG_HOLE) { *rid = kNoRange; return AGILE_DENY_UNMAPPED; }
            if (ty == PG_DENY) { *rid = V.id[f]; return deny_of_kind(V.kind[f]); }
        }
        const uint32_t f2 = V.page[p + 1] & kIdxMask;
        const uint32_t hi_i = f2 + 1 < V.n ? f2 + 1 : V.n;
        uint32_t b = f, len = hi_i > f ? hi_i - f : 0;
        for (uint32_t it = 0; it < V.steps; ++it) {
            const uint32_t half = len >> 1;
            const uint32_t probe = b + half < V.n ? b + half : V.n - 1;
            const bool le = len > 0 && V.base[probe] <= a;
            b = le ? b + half + 1 : b;
            len = le ? len - half - 1 : half;
        }
        return decide(V, f, b, a, w, rid);
    }
    if (a + w <= V.lo || a > V.last) { *rid = kNoRange; return AGILE_DENY_UNMAPPED; }
    return search(V, 0, V.n, a, w, rid);
}

// Out-of-line form for paths where the common case is decided elsewhere.
static __device__ __noinline__ uint32_t classify_slow(const TView &V, uint64_t a, uint64_t w, uint32_t *rid) {
    return classify(V, a, w, rid);
}

// Page of a byte, or ~0u outside the window.
__device__ __forceinline__ uint32_t page_entry(const TView &V, uint64_t a) {
    const uint64_t p = (a - V.lo) >> V.lg;
    return p < V.npages ? V.page[p] : ~0u;
}

// Word of the all-user bitmap that holds a's block, shifted so that bit 0 is that block's
// bit; addresses outside the window read the last (always clear) bit.
__device__ __forceinline__ uint32_t user_bits(const TView &V, uint64_t a) {
    const uint64_t k0 = (a - V.lo) >> V.ulg;
    const uint32_t k = k0 < V.un ? (uint32_t)k0 : V.un;
    return V.ubits[k >> 5] >> (k & 31);
}

// [a, a + w) lies inside one user allocation when its block is all-user (bits =
// user_bits(V, a)) and the access does not run past that block's end. Branch-free; false
// means "not decided here".
__device__ __forceinline__ bool block_user_fast(const TView &V, uint64_t a, uint32_t w, uint32_t bits) {
    const uint64_t m = (1ull << V.ulg) - 1;
    return (bits & 1u) && ((a - V.lo) & m) + w <= m + 1;
}

// [a, a + bytes) lies inside one user allocation when the pages of its first and last
// byte are both all-user pages of the same range: the range is an interval holding
// both. Inline, two page reads; false means "not decided here".
__device__ __forceinline__ bool span_fast(const TView &V, uint64_t a, uint64_t bytes) {
    const uint32_t e0 = page_entry(V, a), e1 = page_entry(V, a + bytes - 1);
    return (e0 >> 30) == PG_USER && e0 == e1;
}

// Whole-span check: the fast test, else the full classification of the span as one
// access (allowed iff inside one user allocation).
__device__ __forceinline__ bool span_allowed(const TView &V, uint64_t a, uint64_t bytes) {
    if (span_fast(V, a, bytes)) return true;
    uint32_t rid;
    return classify_slow(V, a, bytes, &rid) == AGILE_ALLOW;
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

// Completion of a block's smallest record before it goes into the log: none for kernels
// that note whole records.
struct RecordWhole {
    __device__ void operator()(unsigned long long, unsigned long long &, unsigned long long &) const {}
};

// Lower the log's two first-record words, (key, info) and (key, addr), to the block's
// (k, v) and (k, a) where those are smaller. Blocks of one launch end at nearly the same
// time, so their updates meet on one L2 line. Each block first lowers where_key alone
// with a 64-bit atomic minimum, which that line takes at the L2's atomic rate; a block
// whose key is above the value it gets back has lost and stops. Only the few that lowered
// it (or tied) complete their record -- a kernel that keys its violations uniquely may
// reduce them by key alone and leave (v, a) to `complete` -- and take the 128-bit
// exchanges: the (key, info) word by lexicographic minimum, and the address beside
// where_key while where_key still holds their key (a smaller key's block writes its own).
// Each failed exchange sees a different word, and the loops are bounded as a backstop.
template <typename Complete = RecordWhole>
__device__ inline void log_min_first(LogDev *L, unsigned long long k, unsigned long long v,
                                     unsigned long long a, Complete complete = Complete()) {
    if (k > atomicMin(&L->where_key, k)) return;
    complete(k, v, a);
    unsigned long long fk = ~0ull, fv = ~0ull;         // first guess: an empty log
    int it = 0;
    for (; it < (1 << 16) && (k < fk || (k == fk && v < fv)); ++it) {
        unsigned long long rk, rv;
        cas128(&L->first_key, fk, fv, k, v, rk, rv);
        if (rk == fk && rv == fv) break;
        fk = rk;
        fv = rv;
    }
    unsigned long long wa = ~0ull;
    for (; it < (1 << 16); ++it) {
        unsigned long long rk, ra;
        cas128(&L->where_key, k, wa, k, a, rk, ra);
        if (rk != k || ra == wa || ra == a) break;    // a smaller key came, or ours is in
        wa = ra;
    }
    if (it >= (1 << 16)) atomicOr(&L->status, AGILE_LOG_STATUS_TIMEOUT);
}

// Per-thread running minimum of the violations it has seen; each is also appended to the
// bounded list of `log`, when it has one.
struct LaneLog {
    uint32_t cnt = 0;
    unsigned long long key = ~0ull, info = ~0ull, addr = 0;
    LogDev *log = nullptr;
    __device__ __forceinline__ void note(unsigned long long k, unsigned long long i,
                                         unsigned long long a) {
        ++cnt;
        if (k < key || (k == key && i < info)) { key = k; info = i; addr = a; }
        list_append(log, k, i, a);
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
// thread updates the log (completing the record first, see log_min_first). One global
// update per block keeps the log address cold.
template <typename Complete = RecordWhole>
__device__ inline void block_log_flush(LogDev *L, const LaneLog &ll, Complete complete = Complete()) {
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
            log_min_first(L, k, v, a, complete);
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

// Shared-memory staging, chosen by the host as a set of sections: the page map, the
// range arrays, the packed records, the all-user bitmap, the block class map, the
// open-block descriptors. Laid out in that order.
enum : int { ST_PAGES = 1, ST_RANGES = 2, ST_COMPACT = 4, ST_BITS = 8, ST_CMAP = 16, ST_CDESC = 32 };
enum : int {
    STAGE_NONE = 0, STAGE_PAGES = ST_PAGES, STAGE_ALL = ST_PAGES | ST_RANGES,
    STAGE_COMPACT = ST_PAGES | ST_COMPACT, STAGE_BITS = ST_BITS
};

__host__ __device__ inline uint32_t round16(uint64_t x) { return (uint32_t)((x + 15) & ~15ull); }

__host__ __device__ inline uint32_t ubits_bytes(const agile_dev_table_t &T) {
    return round16(((uint64_t)T.ubits_n + 1 + 31) / 32 * 4);
}

__host__ __device__ inline uint32_t cmap_bytes(const agile_dev_table_t &T) {
    return round16(((uint64_t)T.cmap_n + 1 + 15) / 16 * 4);
}

__host__ __device__ inline uint32_t cdesc_bytes(const agile_dev_table_t &T) {
    return T.cdesc != nullptr ? 8u << T.cdesc_log2 : 0u;
}

// Bytes of shared memory a staging mode needs for table T (saturating: a map too large
// for shared memory reports more than any budget).
__host__ __device__ inline uint64_t stage_bytes(const agile_dev_table_t &T, int mode) {
    uint64_t b = 0;
    if (mode & ST_PAGES) b += ((T.npages + 1) * 4 + 15) & ~15ull;
    if (mode & ST_RANGES) b += 2 * round16(T.n * 8ull) + 2 * round16(T.n * 4ull);
    if (mode & ST_COMPACT) b += round16(T.n * 16ull);       // packed records
    if (mode & ST_BITS) b += ubits_bytes(T);
    if (mode & ST_CMAP) b += cmap_bytes(T);
    if (mode & ST_CDESC) b += cdesc_bytes(T);
    return b;
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

// Copy the table sections the mode asks for into shared memory with bulk copies (TMA,
// non-multicast) completed on one mbarrier; every thread of the block calls it and
// waits (bounded). Sections in the device buffer are 256-byte aligned and padded, so
// 16-byte rounded copies stay inside them. If the wait gives up, the thread copies the
// sections with plain loads instead (results stay exact) and the log, when present, is
// flagged.
template <int MODE>
__device__ inline TView stage_table(const agile_dev_table_t &T, unsigned char *smem,
                                    unsigned long long *s_bar, LogDev *log) {
    TView V = view_of(T);
    if constexpr (MODE == STAGE_NONE) return V;
    constexpr bool kPages = MODE & ST_PAGES, kRanges = MODE & ST_RANGES;
    constexpr bool kCompact = MODE & ST_COMPACT, kBits = MODE & ST_BITS, kCmap = MODE & ST_CMAP;
    constexpr bool kDesc = MODE & ST_CDESC;
    const uint32_t pb = kPages ? round16((T.npages + 1) * 4) : 0;
    const uint32_t bb = round16(T.n * 8ull), kb = round16(T.n * 4ull);
    const uint32_t rb = kRanges ? 2 * bb + 2 * kb : 0;
    const uint32_t cb = kCompact ? round16(T.n * 16ull) : 0;
    const uint32_t ub = kBits ? ubits_bytes(T) : 0;
    const uint32_t mb = kCmap ? cmap_bytes(T) : 0;
    const uint32_t db = kDesc ? cdesc_bytes(T) : 0;
    uint32_t *s_page = reinterpret_cast<uint32_t *>(smem);
    uint64_t *s_base = reinterpret_cast<uint64_t *>(smem + pb);
    uint64_t *s_end = reinterpret_cast<uint64_t *>(smem + pb + bb);
    uint32_t *s_kind = reinterpret_cast<uint32_t *>(smem + pb + 2 * bb);
    uint32_t *s_id = reinterpret_cast<uint32_t *>(smem + pb + 2 * bb + kb);
    uint4 *s_cr = reinterpret_cast<uint4 *>(smem + pb + rb);
    uint32_t *s_bits = reinterpret_cast<uint32_t *>(smem + pb + rb + cb);
    uint32_t *s_cmap = reinterpret_cast<uint32_t *>(smem + pb + rb + cb + ub);
    uint2 *s_desc = reinterpret_cast<uint2 *>(smem + pb + rb + cb + ub + mb);
    const uint32_t bar = smem_addr(s_bar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t total = pb + (T.n > 0 ? rb + cb : 0) + ub + mb + db;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(total)
                     : "memory");
        if (kPages) bulk_g2s(s_page, T.page, pb, bar);
        if (kRanges && T.n > 0) {
            bulk_g2s(s_base, T.base, bb, bar);
            bulk_g2s(s_end, T.end, bb, bar);
            bulk_g2s(s_kind, T.kind, kb, bar);
            bulk_g2s(s_id, T.id, kb, bar);
        }
        if (kCompact && T.n > 0) bulk_g2s(s_cr, T.crange, cb, bar);
        if (kBits) bulk_g2s(s_bits, T.ubits, ub, bar);
        if (kCmap) bulk_g2s(s_cmap, T.cmap, mb, bar);
        if (kDesc && db) bulk_g2s(s_desc, T.cdesc, db, bar);
    }
    if (!mbar_wait(bar, 0)) {               // (block-uniform only by timing: any thread may)
        if (log != nullptr && threadIdx.x == 0) atomicOr(&log->status, AGILE_LOG_STATUS_TIMEOUT);
        mbar_wait(bar, 0);                  // let copies in flight land, then copy by hand:
        if (kPages)
            for (uint32_t i = threadIdx.x; i < pb / 4; i += blockDim.x) s_page[i] = T.page[i];
        if (kRanges)                        // identical bytes, so a late bulk write is harmless
            for (uint32_t i = threadIdx.x; i < T.n; i += blockDim.x) {
                s_base[i] = T.base[i]; s_end[i] = T.end[i]; s_kind[i] = T.kind[i]; s_id[i] = T.id[i];
            }
        if (kCompact)
            for (uint32_t i = threadIdx.x; i < T.n; i += blockDim.x)
                s_cr[i] = reinterpret_cast<const uint4 *>(T.crange)[i];
        if (kBits)
            for (uint32_t i = threadIdx.x; i < ub / 4; i += blockDim.x) s_bits[i] = T.ubits[i];
        if (kCmap)
            for (uint32_t i = threadIdx.x; i < mb / 4; i += blockDim.x) s_cmap[i] = T.cmap[i];
        if (kDesc)
            for (uint32_t i = threadIdx.x; i < db / 8; i += blockDim.x)
                s_desc[i] = reinterpret_cast<const uint2 *>(T.cdesc)[i];
    }
    __syncthreads();
    if constexpr (kPages) V.page = s_page;
    if constexpr (kRanges) {
        V.base = s_base; V.end = s_end; V.kind = s_kind; V.id = s_id;
    }
    if constexpr (kCompact) V.crange = s_cr;
    if constexpr (kBits) V.ubits = s_bits;
    if constexpr (kCmap) V.cmap = s_cmap;
    if constexpr (kDesc) V.cdesc = s_desc;
    return V;
}

// Per-warp violation slots in shared memory, written only by slow paths, and the log
// whose bounded list the slow paths append to.
struct WarpSlots {
    unsigned long long key[32], info[32], addr[32];
    uint32_t cnt[32];
    LogDev *log;
};

__device__ inline void slots_init(WarpSlots &S) {
    if (threadIdx.x < 32) {
        S.key[threadIdx.x] = ~0ull; S.info[threadIdx.x] = ~0ull;
        S.addr[threadIdx.x] = 0; S.cnt[threadIdx.x] = 0;
    }
}

// Warp-collective: fold every lane's LaneLog into this warp's slot.
__device__ inline void warp_note(WarpSlots &S, const LaneLog &ll) {
    unsigned long long k = ll.cnt ? ll.key : ~0ull, v = ll.cnt ? ll.info : ~0ull, a = ll.addr;
    min3_shfl(k, v, a);
    const uint32_t c = __reduce_add_sync(kFull, ll.cnt);
    const uint32_t w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0 && c) {
        S.cnt[w] += c;
        if (k < S.key[w] || (k == S.key[w] && v < S.info[w])) {
            S.key[w] = k; S.info[w] = v; S.addr[w] = a;
        }
    }
    __syncwarp();
}

// Block-collective at kernel end: reduce the warp slots, one log update per block.
__device__ inline void slots_flush(LogDev *L, WarpSlots &S) {
    __syncthreads();
    if (threadIdx.x < 32) {
        const uint32_t lane = threadIdx.x, nw = (blockDim.x + 31) >> 5;
        unsigned long long k = lane < nw ? S.key[lane] : ~0ull;
        unsigned long long v = lane < nw ? S.info[lane] : ~0ull;
        unsigned long long a = lane < nw ? S.addr[lane] : 0;
        unsigned long long total = lane < nw ? S.cnt[lane] : 0;
        min3_shfl(k, v, a);
#pragma unroll
        for (int o = 16; o; o >>= 1) total += __shfl_xor_sync(kFull, total, o);
        if (lane == 0 && total != 0 && L != nullptr) {
            atomicAdd(&L->count, total);
            log_min_first(L, k, v, a);
        }
    }
}

// Host side: pick the staging mode for a table (96 KiB for everything -- 104 KiB for the
// packed records with the bitmap, two blocks of 512 threads still fitting on an SM --
// 48 KiB for pages alone). want_compact: the kernel has a 32-bit path and the table carries the compact
// arrays; want_bits: the kernel tests single accesses against the all-user bitmap, staged
// with the page map (within 96 KiB) or alone (within 48 KiB) when the map does not fit.
inline int stage_mode(const agile_dev_table_t &T, bool want_ranges, bool want_compact = false,
                      bool want_bits = false) {
    if (T.npages == 0) return STAGE_NONE;
    const int b = want_bits ? ST_BITS : 0;
    if (want_compact && T.crange != nullptr) {
        if (b && stage_bytes(T, STAGE_COMPACT | b) <= 104 * 1024) return STAGE_COMPACT | b;
        if (stage_bytes(T, STAGE_COMPACT) <= 96 * 1024) return STAGE_COMPACT;
    }
    if (want_ranges && stage_bytes(T, STAGE_ALL | b) <= 96 * 1024) return STAGE_ALL | b;
    if (stage_bytes(T, STAGE_PAGES | b) <= (want_bits ? 96 : 48) * 1024) return STAGE_PAGES | b;
    if (want_bits && stage_bytes(T, STAGE_BITS) <= 48 * 1024) return STAGE_BITS;
    return STAGE_NONE;
}

}  // namespace agile
