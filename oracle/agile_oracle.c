/*
 * Oracle for the kernel memory guard -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, single-threaded C that states what the guard computes. Only tests/,
 * the smoke check and the benchmark's CPU-baseline leg load it; the CUDA library never
 * does, and this file includes nothing from it.
 *
 * The rule (protected GPU memory model, Sec. IV-E; pointer metadata, Sec. V-C; kernel
 * memory guard and its policies, Sec. V-E):
 *   An access A = [a, a+w) against a table of disjoint ranges [base, base+size), each a
 *   user allocation, protected kernel/module memory, or an MMIO mapping (Table I):
 *   1. w == 0, or a+w not representable in 64 bits            -> INVALID   (5)
 *      (batch entry: w must also be one of 1, 2, 4, 8, 16)
 *   2. some USER range holds all of A ("the requested byte range remains within that
 *      allocation", Sec. IV-E / V-C)                           -> ALLOW     (0)
 *   3. else A shares a byte with an MMIO range                  -> MMIO      (2)
 *   4. else A shares a byte with a PROTECTED range              -> PROTECTED (1)
 *   5. else A shares a byte with a USER range (partly outside it, or across two
 *      abutting allocations)                                    -> STRADDLE  (3)
 *   6. else (hole, freed or unknown address, Sec. V-C)          -> UNMAPPED  (4)
 *   The range reported with a deny is the lowest-based range of the deciding class;
 *   UNMAPPED and INVALID report 0xFFFFFFFF. Steps 3-5 order the deny classes; the
 *   paper gives no order, this is the reading the library documents.
 *
 * Two classifiers: classify_linear (A) scans every range per access and is the
 * definition; classify_sorted (B) finds the last range starting at or below a by binary
 * search over a base-sorted copy and walks forward over the few ranges A can touch.
 * B is pinned to A and is used where A would take hours.
 *
 * Violation log (Sec. V-E: poison "records a violation", report "counts or logs"):
 * the first fault is the violating access with the smallest key, a launch-independent
 * order. Batch check: key = access index. Guarded kernels: key = (address, site), site
 * = the access's position in the kernel body. count = number of violating accesses.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { K_USER = 0, K_PROTECTED = 1, K_MMIO = 2 };
enum { V_ALLOW = 0, V_PROTECTED = 1, V_MMIO = 2, V_STRADDLE = 3, V_UNMAPPED = 4, V_INVALID = 5,
       V_NOT_EXACT = 6 };
enum { P_POISON = 0, P_SINK = 1, P_REPORT = 2, P_REMAP = 4 };
#define NO_RANGE 0xFFFFFFFFu

typedef struct {
    uint64_t key;      /* batch: access index; kernels: faulting address */
    uint64_t addr;
    uint32_t width;
    uint32_t verdict;
    uint32_t site;
    uint32_t range_id;
    uint64_t count;    /* violating accesses; 0 = empty log */
} orc_log;

typedef struct {
    size_t n;
    const uint64_t *base, *size;
    const uint32_t *kind, *id;
} orc_table;

/* ---------------------------------------------------------------- classifiers */

static int end_ok(uint64_t a, uint64_t w) { return w != 0 && a <= UINT64_MAX - w; }

static int overlaps(uint64_t a, uint64_t w, uint64_t b, uint64_t s) {
    /* [a, a+w) and [b, b+s) share a byte; both ends representable */
    return a < b + s && b < a + w;
}

/* Oracle A: the definition, one pass over all ranges. */
static uint32_t classify_linear(const orc_table *t, uint64_t a, uint64_t w, uint32_t *rid) {
    *rid = NO_RANGE;
    if (!end_ok(a, w)) return V_INVALID;
    for (size_t j = 0; j < t->n; ++j)
        if (t->kind[j] == K_USER && t->base[j] <= a && a + w <= t->base[j] + t->size[j]) {
            *rid = t->id[j];
            return V_ALLOW;
        }
    static const uint32_t order[3] = {K_MMIO, K_PROTECTED, K_USER};
    static const uint32_t verdict[3] = {V_MMIO, V_PROTECTED, V_STRADDLE};
    for (int c = 0; c < 3; ++c) {
        int found = 0;
        uint64_t lowest = 0;
        for (size_t j = 0; j < t->n; ++j)
            if (t->kind[j] == order[c] && overlaps(a, w, t->base[j], t->size[j]) &&
                (!found || t->base[j] < lowest)) {
                found = 1;
                lowest = t->base[j];
                *rid = t->id[j];
            }
        if (found) return verdict[c];
    }
    return V_UNMAPPED;
}

/* Oracle B: binary search over a base-sorted copy, then the forward walk. */
typedef struct {
    size_t n;
    uint64_t *base, *end;
    uint32_t *kind, *id;
} orc_sorted;

static const orc_table *sort_ctx;
static int by_base(const void *x, const void *y) {
    uint64_t a = sort_ctx->base[*(const size_t *)x], b = sort_ctx->base[*(const size_t *)y];
    return a < b ? -1 : a > b;
}

static orc_sorted *sorted_new(const orc_table *t) {
    orc_sorted *s = calloc(1, sizeof *s);
    size_t *ix = malloc((t->n ? t->n : 1) * sizeof *ix);
    s->n = t->n;
    s->base = malloc((t->n + 1) * 8);
    s->end = malloc((t->n + 1) * 8);
    s->kind = malloc((t->n + 1) * 4);
    s->id = malloc((t->n + 1) * 4);
    for (size_t j = 0; j < t->n; ++j) ix[j] = j;
    sort_ctx = t;
    qsort(ix, t->n, sizeof *ix, by_base);
    for (size_t j = 0; j < t->n; ++j) {
        s->base[j] = t->base[ix[j]];
        s->end[j] = t->base[ix[j]] + t->size[ix[j]];
        s->kind[j] = t->kind[ix[j]];
        s->id[j] = t->id[ix[j]];
    }
    free(ix);
    return s;
}

static void sorted_free(orc_sorted *s) {
    free(s->base); free(s->end); free(s->kind); free(s->id); free(s);
}

static uint32_t classify_sorted(const orc_sorted *s, uint64_t a, uint64_t w, uint32_t *rid) {
    *rid = NO_RANGE;
    if (!end_ok(a, w)) return V_INVALID;
    /* hi = number of ranges with base <= a */
    size_t lo = 0, hi = s->n;
    while (lo < hi) {
        size_t mid = lo + (hi - lo) / 2;
        if (s->base[mid] <= a) lo = mid + 1; else hi = mid;
    }
    size_t first = lo;                      /* candidates start at lo-1 if it reaches a */
    if (lo > 0 && s->end[lo - 1] > a) {
        first = lo - 1;
        if (s->kind[first] == K_USER && a + w <= s->end[first]) {
            *rid = s->id[first];
            return V_ALLOW;
        }
    }
    int best = -1;                          /* class rank: 0 MMIO, 1 PROTECTED, 2 USER */
    for (size_t j = first; j < s->n && s->base[j] < a + w; ++j) {
        int rank = s->kind[j] == K_MMIO ? 0 : s->kind[j] == K_PROTECTED ? 1 : 2;
        if (best < 0 || rank < best) {      /* ranges arrive in base order: first wins */
            best = rank;
            *rid = s->id[j];
        }
    }
    static const uint32_t verdict[3] = {V_MMIO, V_PROTECTED, V_STRADDLE};
    return best < 0 ? V_UNMAPPED : verdict[best];
}

/* ---------------------------------------------------------------- table rules */

/* 0 = a legal table; 1 = a zero-size range; 2 = base+size not representable;
 * 3 = two ranges share a byte; 4 = unknown kind. Pairwise, by definition. */
int orc_table_check(size_t n, const uint64_t *base, const uint64_t *size, const uint32_t *kind) {
    for (size_t j = 0; j < n; ++j) {
        if (kind[j] > K_MMIO) return 4;
        if (size[j] == 0) return 1;
        if (base[j] > UINT64_MAX - size[j]) return 2;
    }
    for (size_t i = 0; i < n; ++i)
        for (size_t j = i + 1; j < n; ++j)
            if (overlaps(base[i], size[i], base[j], size[j])) return 3;
    return 0;
}

/* ---------------------------------------------------------------- log */

static void log_clear(orc_log *g) {
    memset(g, 0, sizeof *g);
    g->key = UINT64_MAX;
    g->range_id = NO_RANGE;
}

static void log_note(orc_log *g, uint64_t key, uint64_t addr, uint32_t width, uint32_t verdict,
                     uint32_t site, uint32_t rid) {
    g->count += 1;
    if (g->count == 1 || key < g->key || (key == g->key && site < g->site)) {
        g->key = key; g->addr = addr; g->width = width;
        g->verdict = verdict; g->site = site; g->range_id = rid;
    }
}

/* ---------------------------------------------------------------- entry points */

/* Batch check: one verdict per (address, width); method 0 = A, 1 = B. */
void orc_check_batch(size_t n, const uint64_t *base, const uint64_t *size, const uint32_t *kind,
                     const uint32_t *id, size_t m, const uint64_t *addr, const uint8_t *width,
                     uint8_t *verdict, uint32_t *rid_out, orc_log *log, int method) {
    orc_table t = {n, base, size, kind, id};
    orc_sorted *s = method ? sorted_new(&t) : NULL;
    log_clear(log);
    for (size_t i = 0; i < m; ++i) {
        uint64_t w = width[i];
        uint32_t rid = NO_RANGE, v;
        if (!(w == 1 || w == 2 || w == 4 || w == 8 || w == 16)) v = V_INVALID;
        else v = method ? classify_sorted(s, addr[i], w, &rid) : classify_linear(&t, addr[i], w, &rid);
        verdict[i] = (uint8_t)v;
        if (rid_out) rid_out[i] = rid;
        if (v != V_ALLOW) log_note(log, i, addr[i], (uint32_t)w, v, 0, rid);
    }
    if (s) sorted_free(s);
}

/* Aperture rule (Table I; Sec. V-E: the PTX guard tests an access against the protected
 * I/O and kernel/module intervals only, leaving everything else on the normal path).
 * The apertures are protected or MMIO ranges; an access is
 *   INVALID  as in step 1 of the table rule (batch widths 1, 2, 4, 8, 16 only),
 *   MMIO     if it shares a byte with an MMIO aperture,
 *   PROTECTED if it shares a byte with a protected aperture,
 *   ALLOW    otherwise (holes, straddles and freed memory are not seen by this rule),
 * reporting the lowest-based aperture of the deciding kind. */
static uint32_t classify_aperture(const orc_table *t, uint64_t a, uint64_t w, uint32_t *rid) {
    *rid = NO_RANGE;
    if (!end_ok(a, w)) return V_INVALID;
    static const uint32_t order[2] = {K_MMIO, K_PROTECTED};
    static const uint32_t verdict[2] = {V_MMIO, V_PROTECTED};
    for (int c = 0; c < 2; ++c) {
        int found = 0;
        uint64_t lowest = 0;
        for (size_t j = 0; j < t->n; ++j)
            if (t->kind[j] == order[c] && overlaps(a, w, t->base[j], t->size[j]) &&
                (!found || t->base[j] < lowest)) {
                found = 1;
                lowest = t->base[j];
                *rid = t->id[j];
            }
        if (found) return verdict[c];
    }
    return V_ALLOW;
}

/* Aperture batch check: as orc_check_batch under the aperture rule. */
void orc_aperture_batch(size_t n, const uint64_t *base, const uint64_t *size, const uint32_t *kind,
                        const uint32_t *id, size_t m, const uint64_t *addr, const uint8_t *width,
                        uint8_t *verdict, uint32_t *rid_out, orc_log *log) {
    orc_table t = {n, base, size, kind, id};
    log_clear(log);
    for (size_t i = 0; i < m; ++i) {
        uint64_t w = width[i];
        uint32_t rid = NO_RANGE, v;
        if (!(w == 1 || w == 2 || w == 4 || w == 8 || w == 16)) v = V_INVALID;
        else v = classify_aperture(&t, addr[i], w, &rid);
        verdict[i] = (uint8_t)v;
        if (rid_out) rid_out[i] = rid;
        if (v != V_ALLOW) log_note(log, i, addr[i], (uint32_t)w, v, 0, rid);
    }
}

/* API-time pointer validation (Sec. IV-E, V-C): (pointer, byte count) pairs, any size. */
void orc_validate(size_t n, const uint64_t *base, const uint64_t *size, const uint32_t *kind,
                  const uint32_t *id, size_t m, const uint64_t *ptr, const uint64_t *bytes,
                  uint8_t *verdict, uint32_t *rid_out) {
    orc_table t = {n, base, size, kind, id};
    for (size_t i = 0; i < m; ++i) {
        uint32_t rid;
        verdict[i] = (uint8_t)classify_linear(&t, ptr[i], bytes[i], &rid);
        if (rid_out) rid_out[i] = rid;
    }
}

/* DMA registration (Sec. V-C: a module may register a user buffer for device DMA, "but the
 * request is accepted only for an exact live user allocation"): allowed only when
 * (ptr, bytes) is exactly one user range; a byte range strictly inside one is NOT_EXACT;
 * anything else gets the ordinary verdict. */
void orc_validate_exact(size_t n, const uint64_t *base, const uint64_t *size, const uint32_t *kind,
                        const uint32_t *id, size_t m, const uint64_t *ptr, const uint64_t *bytes,
                        uint8_t *verdict, uint32_t *rid_out) {
    orc_table t = {n, base, size, kind, id};
    for (size_t i = 0; i < m; ++i) {
        uint32_t rid = NO_RANGE, v = V_NOT_EXACT;
        int exact = 0;
        for (size_t j = 0; j < n; ++j)
            if (kind[j] == K_USER && base[j] == ptr[i] && size[j] == bytes[i]) {
                exact = 1;
                rid = id[j];
            }
        if (exact) {
            v = V_ALLOW;
        } else {
            v = classify_linear(&t, ptr[i], bytes[i], &rid);
            if (v == V_ALLOW) v = V_NOT_EXACT;
        }
        verdict[i] = (uint8_t)v;
        if (rid_out) rid_out[i] = rid;
    }
}

/* The rule a guarded kernel applies: the table rule (classify_sorted over the table) or
 * the aperture rule (classify_aperture over the apertures, Table I / Sec. V-E). */
typedef struct {
    orc_table t;
    orc_sorted *s;          /* NULL under the aperture rule */
} orc_rule;

static orc_rule rule_new(int aperture, size_t tn, const uint64_t *base, const uint64_t *size,
                         const uint32_t *kind, const uint32_t *id) {
    orc_rule r;
    r.t.n = tn; r.t.base = base; r.t.size = size; r.t.kind = kind; r.t.id = id;
    r.s = aperture ? NULL : sorted_new(&r.t);
    return r;
}

static uint32_t rule_classify(const orc_rule *r, uint64_t a, uint64_t w, uint32_t *rid) {
    return r->s ? classify_sorted(r->s, a, w, rid) : classify_aperture(&r->t, a, w, rid);
}

static void rule_free(orc_rule *r) {
    if (r->s) sorted_free(r->s);
}

/*
 * Guarded streaming kernels: copy a = b, scale a = s*b, triad a = b + s*c (one fused
 * multiply-add, rounded once). Each is a sequence of accesses in this order per unit:
 *   unit u < n/4: 16-byte loads of b (site 0) [and c (site 1) for triad], then a 16-byte
 *                 store of a (site 1 for copy/scale, site 2 for triad), at byte offset 16u;
 *   tail i >= 4*(n/4): the same with 4-byte accesses at byte offset 4i.
 * va_* are the arrays' addresses in the guarded address space; b, c, a hold the data
 * (a holds its prior contents on entry: a suppressed store leaves them).
 * Policy (Sec. V-E): poison -- a denied load reads 0, a denied store is dropped, each is
 * logged; sink -- the same observable data (loads read a zero page, stores land in a
 * write sink), logged; report -- the access proceeds, logged.
 * aperture: 0 checks against the table, 1 against the apertures (the ranges passed).
 */
void orc_stream(int op, size_t n, uint64_t va_a, uint64_t va_b, uint64_t va_c, float s,
                const float *b, const float *c, float *a, int policy, int aperture, size_t tn,
                const uint64_t *base, const uint64_t *size, const uint32_t *kind,
                const uint32_t *id, orc_log *log) {
    orc_rule R = rule_new(aperture, tn, base, size, kind, id);
    log_clear(log);
    size_t units = n / 4;
    size_t total = units + (n - units * 4);
    uint32_t store_site = op == 2 ? 2u : 1u;
    for (size_t u = 0; u < total; ++u) {
        int vec = u < units;
        size_t e0 = vec ? 4 * u : 4 * units + (u - units);
        size_t cnt = vec ? 4 : 1;
        uint64_t w = 4 * cnt, off = 4 * e0;
        float vb[4] = {0, 0, 0, 0}, vc[4] = {0, 0, 0, 0}, out[4];
        uint32_t rid, v;
        v = rule_classify(&R, va_b + off, w, &rid);
        if (v == V_ALLOW || policy == P_REPORT) memcpy(vb, b + e0, 4 * cnt);
        if (v != V_ALLOW) log_note(log, va_b + off, va_b + off, (uint32_t)w, v, 0, rid);
        if (op == 2) {
            v = rule_classify(&R, va_c + off, w, &rid);
            if (v == V_ALLOW || policy == P_REPORT) memcpy(vc, c + e0, 4 * cnt);
            if (v != V_ALLOW) log_note(log, va_c + off, va_c + off, (uint32_t)w, v, 1, rid);
        }
        for (size_t k = 0; k < cnt; ++k)
            out[k] = op == 0 ? vb[k] : op == 1 ? s * vb[k] : fmaf(s, vc[k], vb[k]);
        v = rule_classify(&R, va_a + off, w, &rid);
        if (v == V_ALLOW || policy == P_REPORT) memcpy(a + e0, out, 4 * cnt);
        if (v != V_ALLOW) log_note(log, va_a + off, va_a + off, (uint32_t)w, v, store_site, rid);
    }
    rule_free(&R);
}

/* Unguarded reference kernels: the same arithmetic with no table. */
void orc_stream_plain(int op, size_t n, float s, const float *b, const float *c, float *a) {
    for (size_t i = 0; i < n; ++i)
        a[i] = op == 0 ? b[i] : op == 1 ? s * b[i] : fmaf(s, c[i], b[i]);
}

/*
 * Guarded irregular kernels over one arena (the caller's copy of the device memory that
 * holds every array; arena_va is its address). Sec. V-E: each global access is checked
 * first; the policy decides what a denied access does (as for the streaming kernels).
 * Per unit u < n/4 of four elements:
 *   site 0: 16-byte load of idx[4u], idx[4u+1];  site 1: 16-byte load of idx[4u+2..3]
 *   site 2: for k = 0..3 the element access at T + 4*idx[4u+k] (4 bytes):
 *           gather -- load; scatter -- store (float)(idx & 0xFFFFFF); hist -- atomic +1 (u32)
 *   site 3: gather only -- 16-byte store of out[4u..4u+3]
 * Tail elements i >= 4*(n/4): 8-byte idx load (site 0), the element access (site 2),
 * gather's 4-byte out store (site 3). idx is int64; T + 4*idx wraps modulo 2^64.
 * Returns 0, or -1 if an access that is carried out falls outside the arena.
 */
enum { IR_GATHER = 0, IR_SCATTER = 1, IR_HIST = 2 };

typedef struct {
    uint64_t va;
    uint8_t *mem;
    size_t len;
} orc_arena;

static int in_arena(const orc_arena *A, uint64_t a, uint64_t w) {
    return a >= A->va && w <= A->len && a - A->va <= A->len - w;
}

/* One guarded access: classify, log a deny, and tell whether it is carried out and at
 * which address. REMAP (Sec. V-E remap_or, with the paper's caveat that the target must
 * itself be a live user allocation): a denied access moves to a | remap when that access is
 * allowed, else it is dropped as under poison. */
static int guarded(const orc_rule *R, orc_log *log, int policy, uint64_t remap, uint64_t a,
                   uint64_t w, uint32_t site, uint64_t *at) {
    uint32_t rid, v = rule_classify(R, a, w, &rid);
    *at = a;
    if (v == V_ALLOW) return 1;
    log_note(log, a, a, (uint32_t)w, v, site, rid);
    if (policy == P_REPORT) return 1;
    if (policy == P_REMAP) {
        uint32_t r2;
        if (rule_classify(R, a | remap, w, &r2) == V_ALLOW) { *at = a | remap; return 1; }
    }
    return 0;
}

int orc_irregular(int kind, size_t n, uint64_t arena_va, uint8_t *arena, size_t arena_len,
                  uint64_t va_idx, uint64_t va_t, uint64_t va_out, int policy, uint64_t remap,
                  int aperture, size_t tn, const uint64_t *base, const uint64_t *size,
                  const uint32_t *kindv, const uint32_t *id, orc_log *log) {
    orc_rule R = rule_new(aperture, tn, base, size, kindv, id);
    orc_arena A = {arena_va, arena, arena_len};
    int rc = 0;
    log_clear(log);
    size_t units = n / 4, total = units + (n - 4 * units);
    for (size_t u = 0; u < total && rc == 0; ++u) {
        int vec = u < units;
        size_t e0 = vec ? 4 * u : 4 * units + (u - units), cnt = vec ? 4 : 1;
        int64_t idx[4] = {0, 0, 0, 0};
        /* index loads */
        for (size_t h = 0; h < (vec ? 2u : 1u); ++h) {
            uint64_t a = va_idx + 8 * e0 + 16 * h, w = vec ? 16 : 8, at;
            if (guarded(&R, log, policy, remap, a, w, (uint32_t)h, &at)) {
                if (!in_arena(&A, at, w)) { rc = -1; break; }
                memcpy(idx + 2 * h, arena + (at - A.va), w);
            }
        }
        /* element accesses */
        float out[4] = {0, 0, 0, 0};
        for (size_t k = 0; k < cnt && rc == 0; ++k) {
            uint64_t a = va_t + 4 * (uint64_t)idx[k], at;
            if (!guarded(&R, log, policy, remap, a, 4, 2, &at)) continue;
            if (!in_arena(&A, at, 4)) { rc = -1; break; }
            uint8_t *p = arena + (at - A.va);
            if (kind == IR_GATHER) {
                memcpy(&out[k], p, 4);
            } else if (kind == IR_SCATTER) {
                float f = (float)((uint64_t)idx[k] & 0xFFFFFFu);
                memcpy(p, &f, 4);
            } else {
                uint32_t c;
                memcpy(&c, p, 4);
                c += 1;
                memcpy(p, &c, 4);
            }
        }
        /* gather's output store */
        if (kind == IR_GATHER && rc == 0) {
            uint64_t a = va_out + 4 * e0, w = 4 * cnt, at;
            if (guarded(&R, log, policy, remap, a, w, 3, &at)) {
                if (!in_arena(&A, at, w)) rc = -1;
                else memcpy(arena + (at - A.va), out, w);
            }
        }
    }
    rule_free(&R);
    return rc;
}
