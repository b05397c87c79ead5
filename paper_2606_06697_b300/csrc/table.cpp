// Guard table: build (sort, validate, page map), upload into a caller-owned device buffer,
// and the host form of the check used for API-time pointer validation (Sec. V-C: the
// worker records each user allocation's base and requested size and resolves pointers
// against that table; Sec. IV-E: protected and MMIO ranges are never valid targets).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <numeric>

#include "agile_internal.h"

namespace {

constexpr uint32_t PG_MIXED = 0, PG_USER = 1, PG_HOLE = 2, PG_DENY = 3;
constexpr uint32_t kIdxMask = 0x3FFFFFFFu;
constexpr uint64_t kMaxPages = 1ull << 26;
using agile::kTableHeaderBytes, agile::kTableZeroOff, agile::kTableSinkOff, agile::kTablePageOff;

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Pages of the window [lo, lo + npages * G) that covers every range.
void window(const agile_guard_table &t, uint32_t lg, uint64_t *lo, uint64_t *np) {
    if (t.n == 0) { *lo = 0; *np = 0; return; }
    uint64_t first = t.base.front() >> lg;
    uint64_t last = (t.end.back() - 1) >> lg;   // end >= 1 since sizes are >= 1
    *lo = first << lg;
    *np = last - first + 1;
}

void build_pages(agile_guard_table &t) {
    const uint64_t G = 1ull << t.log2_page;
    t.page.assign(t.npages + 1, 0);
    uint32_t j = 0;
    for (uint64_t p = 0; p < t.npages; ++p) {
        uint64_t ps = t.lo + p * G, pe = ps + G;   // pe may wrap to 0 at the very top
        while (j < t.n && t.end[j] <= ps) ++j;
        uint32_t type;
        if (j == t.n || (pe != 0 && t.base[j] >= pe)) {
            type = PG_HOLE;
        } else if (t.base[j] <= ps && (pe == 0 ? t.end[j] == 0 : t.end[j] >= pe)) {
            type = t.kind[j] == AGILE_USER ? PG_USER : PG_DENY;
        } else {
            type = PG_MIXED;
        }
        t.page[p] = (type << 30) | j;
    }
    t.page[t.npages] = (PG_HOLE << 30) | t.n;
    // A search inside page p runs over base[f_p, min(f_{p+1} + 1, n)); a slice of L ranges
    // needs floor(log2 L) + 1 halving steps.
    uint32_t steps = 0;
    for (uint64_t p = 0; p < t.npages; ++p) {
        const uint32_t f = t.page[p] & kIdxMask, f2 = t.page[p + 1] & kIdxMask;
        const uint32_t hi = f2 + 1 < t.n ? f2 + 1 : t.n;
        const uint32_t len = hi > f ? hi - f : 0;
        uint32_t k = 0;
        while ((len >> k) != 0) ++k;
        if (k > steps) steps = k;
    }
    t.search_steps = steps;
}

// Class of every block of C = 2^cmap_log2 bytes from lo: 1 inside one user range, 3 inside
// one protected range, 2 touched by no range, 0 otherwise (an MMIO block, a block holding a
// range boundary). The entry past the last block is 2: every range lies inside the
// window, so an access wholly beyond the map's end, or wholly below lo (its offset wraps),
// touches none. A block that ends at 2^64 stays 0, so an access ending there reaches the
// full rule, which finds its end unrepresentable.
void build_cmap(const agile_guard_table &t, uint32_t *map, uint64_t window) {
    const uint64_t C = 1ull << t.cmap_log2, nb = t.cmap_n;
    auto set = [&](uint64_t k, uint32_t code) {
        map[k >> 4] = (map[k >> 4] & ~(3u << (2 * (k & 15)))) | (code << (2 * (k & 15)));
    };
    for (uint64_t k = 0; k < nb; ++k) set(k, 2);
    for (uint32_t i = 0; i < t.n; ++i) {
        const uint64_t b = t.base[i] - t.lo, e = t.end[i] - t.lo;   // e <= window
        const uint64_t k0 = b >> t.cmap_log2, k1 = (e - 1) >> t.cmap_log2;
        const uint64_t f0 = (b & (C - 1)) ? k0 + 1 : k0;              // first full block
        const uint64_t f1 = e >> t.cmap_log2;                         // past the last full one
        const uint32_t code = t.kind[i] == AGILE_USER ? 1u : t.kind[i] == AGILE_PROTECTED ? 3u : 0u;
        for (uint64_t k = f0; k < f1 && k < nb; ++k) set(k, code);
        if (k0 < f0) set(k0, 0);                                      // partial first block
        if (k1 >= f1 && k1 < nb) set(k1, 0);                          // partial last block
    }
    set(nb, 2);
    if (window != 0 && t.lo + window == 0 && nb > 0) set(nb - 1, 0);  // window ends at 2^64
}

// Descriptors of open blocks for the batch check's second pass (windows under 4 GiB, so
// block indices and offsets are 32-bit). An open block (class 0) holding at most one
// range boundary strictly inside it -- or none, inside one MMIO range -- is described by
// that boundary's offset b in the block (C when there is none) and three verdicts of the
// rule: for an access wholly before b, wholly at or after b, and across b (it overlaps
// both regions; the rule's order MMIO, protected, user gives MMIO, PROTECTED, STRADDLE).
// Payload: b in bits 0-13, the three verdicts in bits 16-18, 20-22, 24-26. The block
// that ends at 2^64 is left out: an access ending there is INVALID.
struct Desc { uint32_t block, payload; };

uint32_t region_verdict(const agile_guard_table &t, uint64_t a) {   // the range holding byte a
    const size_t j = std::upper_bound(t.base.begin(), t.base.end(), a) - t.base.begin();
    if (j == 0 || t.end[j - 1] <= a) return AGILE_DENY_UNMAPPED;
    const uint32_t k = t.kind[j - 1];
    return k == AGILE_USER ? AGILE_ALLOW : k == AGILE_PROTECTED ? AGILE_DENY_PROTECTED : AGILE_DENY_MMIO;
}

uint32_t across_verdict(uint32_t vl, uint32_t vr) {
    if (vl == AGILE_DENY_MMIO || vr == AGILE_DENY_MMIO) return AGILE_DENY_MMIO;
    if (vl == AGILE_DENY_PROTECTED || vr == AGILE_DENY_PROTECTED) return AGILE_DENY_PROTECTED;
    if (vl == AGILE_ALLOW || vr == AGILE_ALLOW) return AGILE_DENY_STRADDLE;
    return AGILE_DENY_UNMAPPED;
}

std::vector<Desc> open_block_descs(const agile_guard_table &t, const uint32_t *map, uint64_t window) {
    std::vector<Desc> out;
    const uint64_t C = 1ull << t.cmap_log2;
    for (uint64_t k = 0; k < t.cmap_n; ++k) {
        if ((map[k >> 4] >> (2 * (k & 15)) & 3u) != 0) continue;
        const uint64_t s = t.lo + k * C;               // block [s, s + C)
        if (s + C == 0 || (k + 1 == t.cmap_n && t.lo + window == 0)) continue;
        // distinct range edges strictly inside the block
        uint64_t pts[3];
        int np = 0;
        for (const std::vector<uint64_t> *edges : {&t.base, &t.end}) {
            auto it = std::upper_bound(edges->begin(), edges->end(), s);
            for (; it != edges->end() && *it < s + C && np < 3; ++it) {
                bool seen = false;
                for (int q = 0; q < np; ++q) seen |= pts[q] == *it;
                if (!seen) pts[np++] = *it;
            }
        }
        if (np > 1) continue;
        const uint64_t b = np ? pts[0] : s + C;
        const uint32_t vl = region_verdict(t, s), vr = np ? region_verdict(t, b) : vl;
        out.push_back({(uint32_t)k, (uint32_t)(b - s) | vl << 16 | vr << 20 | across_verdict(vl, vr) << 24});
    }
    return out;
}

// Two-choice hash of the descriptors: block k sits in slot h1(k) or h2(k) of 2^lg slots,
// h(k) = (k * K mod 2^32) >> (32 - lg), empty slots hold block 0xFFFFFFFF. Slots: the
// smallest power of two >= 4 per descriptor (a load of 1/4 or less, well inside what two
// choices place), 64 to 4096. Descriptors that find no slot are left out (their accesses
// reach the full rule). The multiplier pair placing the most descriptors is kept.
void hash_descs(const std::vector<Desc> &d, uint32_t *lg_out, uint32_t *k1_out, uint32_t *k2_out,
                std::vector<Desc> *slots_out) {
    static const uint32_t kMul[16] = {0x9E3779B1u, 0x85EBCA77u, 0xC2B2AE3Du, 0x27D4EB2Fu,
                                      0x165667B1u, 0xD3A2646Du, 0xFD7046C5u, 0xB55A4F09u,
                                      0x7FEB352Du, 0x846CA68Bu, 0x2C1B3C6Du, 0x297A2D39u,
                                      0xCC9E2D51u, 0x1B873593u, 0xE6546B65u, 0x68E31DA5u};
    uint32_t lg = 6;
    while (lg < 12 && (1ull << lg) < 4 * d.size()) ++lg;
    const uint32_t S = 1u << lg;
    size_t best = 0;
    for (int t = 0; t < 8; ++t) {
        const uint32_t k1 = kMul[2 * t], k2 = kMul[2 * t + 1];
        auto h = [&](uint32_t k, uint32_t K) { return (uint32_t)(k * K) >> (32 - lg); };
        std::vector<Desc> slot(S, Desc{0xFFFFFFFFu, 0});
        size_t placed = 0;
        // at most 64 moves per slot in all: a table with far more open blocks than slots
        // fills them and stops, instead of failing every remaining insertion at length
        uint64_t moves = 64ull * S;
        for (const Desc &x : d) {
            if (moves == 0 || placed == S) break;
            Desc cur = x;
            uint32_t pos = h(cur.block, k1);
            bool ok = false;
            for (int kick = 0; kick < 64 && moves > 0; ++kick, --moves) {
                if (slot[pos].block == 0xFFFFFFFFu) { slot[pos] = cur; ok = true; break; }
                std::swap(cur, slot[pos]);
                const uint32_t a1 = h(cur.block, k1);
                pos = pos == a1 ? h(cur.block, k2) : a1;
            }
            placed += ok;                              // else `cur`, whichever it is, is left out
        }
        if (t == 0 || placed > best) {
            best = placed;
            *lg_out = lg; *k1_out = k1; *k2_out = k2;
            *slots_out = slot;
        }
        if (placed == d.size()) break;
    }
}

// Page size for AGILE_PAGE_AUTO: the largest page, from 2 MiB down to 4 KiB, at which at
// least 95% of the user bytes lie in pages that are all one user range (the accesses the
// page map decides alone), keeping the map within 2^24 entries; failing that, the page
// size with the largest such share.
uint32_t auto_page(const agile_guard_table &t) {
    uint64_t user = 0;
    for (uint32_t i = 0; i < t.n; ++i)
        if (t.kind[i] == AGILE_USER) user += t.end[i] - t.base[i];
    if (user == 0) return 21;
    uint32_t best = 21;
    double best_share = -1.0;
    for (uint32_t lg = 21; lg >= 12; --lg) {
        uint64_t lo, np;
        window(t, lg, &lo, &np);
        if (np > (1ull << 24)) break;
        uint64_t pure = 0;
        for (uint32_t i = 0; i < t.n; ++i) {
            if (t.kind[i] != AGILE_USER) continue;
            const uint64_t first = (t.base[i] >> lg) + ((t.base[i] & ((1ull << lg) - 1)) != 0);
            const uint64_t past = t.end[i] >> lg;                            // pages ending in it
            if (past > first) pure += (past - first) << lg;
        }
        const double share = (double)pure / (double)user;
        if (share > best_share) { best_share = share; best = lg; }
        if (share >= 0.95) return lg;
    }
    return best;
}

}  // namespace

namespace agile {

uint32_t classify_host(const agile_guard_table &t, uint64_t a, uint64_t w, uint32_t *rid) {
    *rid = AGILE_NO_RANGE;
    if (w == 0 || a > ~0ull - w) return AGILE_DENY_INVALID;
    // last range starting at or below a
    size_t b = std::upper_bound(t.base.begin(), t.base.end(), a) - t.base.begin();
    size_t first = b;
    if (b > 0 && t.end[b - 1] > a) {
        if (t.kind[b - 1] == AGILE_USER && a + w <= t.end[b - 1]) {
            *rid = t.id[b - 1];
            return AGILE_ALLOW;
        }
        first = b - 1;
    }
    int best = 3;
    for (size_t k = first; k < t.n && t.base[k] < a + w; ++k) {
        int r = t.kind[k] == AGILE_MMIO ? 0 : t.kind[k] == AGILE_PROTECTED ? 1 : 2;
        if (r < best) { best = r; *rid = t.id[k]; }
    }
    static const uint32_t v[3] = {AGILE_DENY_MMIO, AGILE_DENY_PROTECTED, AGILE_DENY_STRADDLE};
    return best == 3 ? (uint32_t)AGILE_DENY_UNMAPPED : v[best];
}

}  // namespace agile

extern "C" {

int agile_guard_table_build(const agile_range_t *h_ranges, size_t n, uint32_t log2_page,
                            agile_guard_table_t **out) {
    if (out == nullptr || (n > 0 && h_ranges == nullptr)) return AGILE_ERR_INVALID_ARG;
    *out = nullptr;
    if (log2_page != AGILE_PAGE_AUTO && (log2_page < 12 || log2_page > 40)) return AGILE_ERR_INVALID_ARG;
    if (n > AGILE_MAX_RANGES) return AGILE_ERR_TOO_LARGE;
    for (size_t i = 0; i < n; ++i) {
        if (h_ranges[i].kind > AGILE_MMIO) return AGILE_ERR_BAD_KIND;
        if (h_ranges[i].size == 0) return AGILE_ERR_ZERO_SIZE;
        if (h_ranges[i].base > ~0ull - h_ranges[i].size) return AGILE_ERR_RANGE_OVERFLOW;
    }
    agile_guard_table *t = new (std::nothrow) agile_guard_table;
    if (t == nullptr) return AGILE_ERR_NOMEM;
    try {
        std::vector<uint32_t> ord(n);
        std::iota(ord.begin(), ord.end(), 0u);
        std::stable_sort(ord.begin(), ord.end(), [&](uint32_t x, uint32_t y) {
            return h_ranges[x].base < h_ranges[y].base;
        });
        t->n = (uint32_t)n;
        t->base.resize(n); t->end.resize(n); t->kind.resize(n); t->id.resize(n);
        for (size_t i = 0; i < n; ++i) {
            const agile_range_t &r = h_ranges[ord[i]];
            t->base[i] = r.base;
            t->end[i] = r.base + r.size;
            t->kind[i] = r.kind;
            t->id[i] = r.id;
            if (i > 0 && t->base[i] < t->end[i - 1]) { delete t; return AGILE_ERR_OVERLAP; }
        }
        uint32_t lg = log2_page == AGILE_PAGE_AUTO ? auto_page(*t) : log2_page;
        window(*t, lg, &t->lo, &t->npages);
        while (t->npages > kMaxPages) {
            ++lg;
            window(*t, lg, &t->lo, &t->npages);
        }
        t->log2_page = lg;
        build_pages(*t);
        size_t off = kTablePageOff + align256((t->npages + 1) * 4);
        t->off_base = off; off += align256(n * 8);
        t->off_end = off;  off += align256(n * 8);
        t->off_kind = off; off += align256(n * 4);
        t->off_id = off;   off += align256(n * 4);
        // Windows under 4 GiB also get one packed 16-byte record per range -- start and
        // last byte as 32-bit offsets from lo, kind, id -- so a kernel can decide in 32 bits
        // with one 128-bit load per range.
        t->compact = n > 0 && lg <= 31 && t->npages <= ((1ull << 32) - 1) >> lg;
        if (t->compact) {
            t->off_crange = off;
            off += align256(n * 16);
        }
        // All-user block bitmap for single-access fast tests: blocks of B = 2^ubits_log2
        // bytes from lo (at least 4 KiB, as small as keeps the bitmap within 2^18 bits),
        // a bit set iff its block lies inside one user range.
        const uint64_t window = t->npages << lg;            // < 2^64: lo + window - 1 fits
        uint32_t ulg = 12;
        while (ulg < 63 && (window >> ulg) + ((window & ((1ull << ulg) - 1)) != 0) > (1ull << 18)) ++ulg;
        t->ubits_log2 = ulg;
        t->ubits_n = (uint32_t)((window >> ulg) + ((window & ((1ull << ulg) - 1)) != 0));
        t->off_ubits = off;
        off += align256(((uint64_t)t->ubits_n + 1 + 31) / 32 * 4);
        // Block class map for the batch check: 2 bits per block of C = 2^cmap_log2 bytes
        // (at least 256, as small as keeps the map within 2^19 blocks).
        uint32_t clg = 8;
        while (clg < 63 && (window >> clg) + ((window & ((1ull << clg) - 1)) != 0) > (1ull << 19)) ++clg;
        t->cmap_log2 = clg;
        t->cmap_n = (uint32_t)((window >> clg) + ((window & ((1ull << clg) - 1)) != 0));
        t->off_cmap = off;
        off += align256(((uint64_t)t->cmap_n + 1 + 15) / 16 * 4);
        std::vector<uint32_t> cmap_img(((uint64_t)t->cmap_n + 1 + 15) / 16, 0);
        build_cmap(*t, cmap_img.data(), window);
        std::vector<Desc> slots;
        if (t->compact) {
            hash_descs(open_block_descs(*t, cmap_img.data(), window), &t->cdesc_log2, &t->cdesc_k1,
                       &t->cdesc_k2, &slots);
            t->off_cdesc = off;
            off += align256(slots.size() * 8);
        }
        t->total = off;
        t->staging.assign(t->total, 0);
        {
            uint32_t *ub = reinterpret_cast<uint32_t *>(t->staging.data() + t->off_ubits);
            const uint64_t B = 1ull << ulg;
            for (size_t i = 0; i < n; ++i) {
                if (t->kind[i] != AGILE_USER) continue;
                const uint64_t b = t->base[i] - t->lo, e = t->end[i] - t->lo;
                uint64_t k = b / B + (b % B != 0);              // first block starting in it
                const uint64_t k_end = std::min<uint64_t>(e / B, t->ubits_n);  // blocks ending in it
                for (; k < k_end; ++k) ub[k >> 5] |= 1u << (k & 31);
            }
        }
        std::memcpy(t->staging.data() + t->off_cmap, cmap_img.data(), cmap_img.size() * 4);
        if (t->compact) std::memcpy(t->staging.data() + t->off_cdesc, slots.data(), slots.size() * 8);
        std::memcpy(t->staging.data() + kTablePageOff, t->page.data(), t->page.size() * 4);
        if (n) {
            std::memcpy(t->staging.data() + t->off_base, t->base.data(), n * 8);
            std::memcpy(t->staging.data() + t->off_end, t->end.data(), n * 8);
            std::memcpy(t->staging.data() + t->off_kind, t->kind.data(), n * 4);
            std::memcpy(t->staging.data() + t->off_id, t->id.data(), n * 4);
        }
        if (t->compact) {
            uint32_t *cr = reinterpret_cast<uint32_t *>(t->staging.data() + t->off_crange);
            for (size_t i = 0; i < n; ++i) {
                cr[4 * i] = (uint32_t)(t->base[i] - t->lo);
                cr[4 * i + 1] = (uint32_t)(t->end[i] - 1 - t->lo);
                // deny rank of the kind: 0 MMIO, 1 protected, 2 user (also "allowable")
                cr[4 * i + 2] = t->kind[i] == AGILE_MMIO ? 0u : t->kind[i] == AGILE_PROTECTED ? 1u : 2u;
                cr[4 * i + 3] = t->id[i];
            }
        }
    } catch (const std::bad_alloc &) {
        delete t;
        return AGILE_ERR_NOMEM;
    }
    *out = t;
    return AGILE_OK;
}

int agile_guard_table_set_remap(agile_guard_table_t *t, uint64_t remap_or) {
    if (t == nullptr) return AGILE_ERR_INVALID_ARG;
    if (remap_or & 15) return AGILE_ERR_ALIGN;
    t->remap_or = remap_or;
    return AGILE_OK;
}

int agile_guard_table_device_bytes(const agile_guard_table_t *t, size_t *bytes) {
    if (t == nullptr || bytes == nullptr) return AGILE_ERR_INVALID_ARG;
    *bytes = t->total;
    return AGILE_OK;
}

int agile_guard_table_geometry(const agile_guard_table_t *t, uint32_t *log2_page,
                               uint64_t *npages) {
    if (t == nullptr) return AGILE_ERR_INVALID_ARG;
    if (log2_page) *log2_page = t->log2_page;
    if (npages) *npages = t->npages;
    return AGILE_OK;
}

namespace {

// The view of a table image whose buffer starts at `d` (device or host address).
agile_dev_table_t view_at(const agile_guard_table &t, unsigned char *d) {
    agile_dev_table_t h;
    std::memset(&h, 0, sizeof h);
    h.lo = t.lo;
    h.npages = t.npages;
    h.log2_page = t.log2_page;
    h.n = t.n;
    h.page = (const uint32_t *)(d + kTablePageOff);
    h.base = (const uint64_t *)(d + t.off_base);
    h.end = (const uint64_t *)(d + t.off_end);
    h.kind = (const uint32_t *)(d + t.off_kind);
    h.id = (const uint32_t *)(d + t.off_id);
    h.zero_page = d + kTableZeroOff;
    h.sink_page = d + kTableSinkOff;
    h.bytes = t.total;
    h.search_steps = t.search_steps;
    h.remap_or = t.remap_or;
    if (t.compact) h.crange = (const uint32_t *)(d + t.off_crange);
    h.ubits = (const uint32_t *)(d + t.off_ubits);
    h.ubits_log2 = t.ubits_log2;
    h.ubits_n = t.ubits_n;
    h.cmap = (const uint32_t *)(d + t.off_cmap);
    h.cmap_log2 = t.cmap_log2;
    h.cmap_n = t.cmap_n;
    if (t.compact) {
        h.cdesc = (const uint32_t *)(d + t.off_cdesc);
        h.cdesc_log2 = t.cdesc_log2;
        h.cdesc_k1 = t.cdesc_k1;
        h.cdesc_k2 = t.cdesc_k2;
    }
    static_assert(sizeof(agile_dev_table_t) <= kTableHeaderBytes, "header fits");
    return h;
}

}  // namespace

int agile_guard_table_upload(agile_guard_table_t *t, void *d_buf, size_t bytes, void *stream,
                             agile_dev_table_t *out) {
    if (t == nullptr || d_buf == nullptr || out == nullptr) return AGILE_ERR_INVALID_ARG;
    if (bytes < t->total) return AGILE_ERR_TOO_LARGE;
    if (((uintptr_t)d_buf & 255) != 0) return AGILE_ERR_ALIGN;
    const agile_dev_table_t h = view_at(*t, (unsigned char *)d_buf);
    std::memcpy(t->staging.data(), &h, sizeof h);
    std::memset(t->staging.data() + kTableZeroOff, 0, 128);
    AGILE_CUDA_TRY(cudaMemcpyAsync(d_buf, t->staging.data(), t->total, cudaMemcpyHostToDevice,
                                   (cudaStream_t)stream));
    *out = h;
    return AGILE_OK;
}

int agile_guard_table_image(const agile_guard_table_t *t, void *h_buf, size_t bytes,
                            agile_dev_table_t *out) {
    if (t == nullptr || h_buf == nullptr || out == nullptr) return AGILE_ERR_INVALID_ARG;
    if (bytes < t->total) return AGILE_ERR_TOO_LARGE;
    if (((uintptr_t)h_buf & 255) != 0) return AGILE_ERR_ALIGN;
    unsigned char *d = (unsigned char *)h_buf;
    const agile_dev_table_t h = view_at(*t, d);
    std::memcpy(d, t->staging.data(), t->total);
    std::memcpy(d, &h, sizeof h);
    std::memset(d + kTableZeroOff, 0, 128);
    *out = h;
    return AGILE_OK;
}

void agile_guard_table_destroy(agile_guard_table_t *t) { delete t; }

int agile_validate_args(const agile_guard_table_t *t, const uint64_t *h_ptr,
                        const uint64_t *h_bytes, size_t n, uint8_t *h_verdict,
                        uint32_t *h_range_id) {
    if (t == nullptr || (n > 0 && (h_ptr == nullptr || h_bytes == nullptr || h_verdict == nullptr)))
        return AGILE_ERR_INVALID_ARG;
    int any = 0;
    for (size_t i = 0; i < n; ++i) {
        uint32_t rid;
        uint32_t v = agile::classify_host(*t, h_ptr[i], h_bytes[i], &rid);
        h_verdict[i] = (uint8_t)v;
        if (h_range_id) h_range_id[i] = rid;
        any |= v != AGILE_ALLOW;
    }
    return any ? AGILE_VIOLATION : AGILE_OK;
}

int agile_validate_dma(const agile_guard_table_t *t, const uint64_t *h_ptr,
                       const uint64_t *h_bytes, size_t n, uint8_t *h_verdict,
                       uint32_t *h_range_id) {
    if (t == nullptr || (n > 0 && (h_ptr == nullptr || h_bytes == nullptr || h_verdict == nullptr)))
        return AGILE_ERR_INVALID_ARG;
    int any = 0;
    for (size_t i = 0; i < n; ++i) {
        uint32_t rid;
        uint32_t v = agile::classify_host(*t, h_ptr[i], h_bytes[i], &rid);
        if (v == AGILE_ALLOW) {
            // the containing allocation is the last range starting at or below ptr
            const size_t j = std::upper_bound(t->base.begin(), t->base.end(), h_ptr[i]) - t->base.begin() - 1;
            if (!(t->base[j] == h_ptr[i] && t->end[j] - t->base[j] == h_bytes[i])) v = AGILE_DENY_NOT_EXACT;
        }
        h_verdict[i] = (uint8_t)v;
        if (h_range_id) h_range_id[i] = rid;
        any |= v != AGILE_ALLOW;
    }
    return any ? AGILE_VIOLATION : AGILE_OK;
}

}  // extern "C"
