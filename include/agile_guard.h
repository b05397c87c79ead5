/*
 * agile_guard.h -- C ABI of the kernel memory guard (B300 / sm_103a).
 *
 * The guard enforces the protected GPU memory model of AgileOS (Sec. IV-E, Table I):
 * device memory is split into user allocations, protected kernel/module memory and
 * MMIO mappings, and an access -- by a host API call (Sec. V-C) or by an untrusted
 * kernel (Sec. V-E) -- passes only when its whole byte range lies inside one live user
 * allocation. Everything else is denied and, under the poison/sink/report policies of
 * Sec. V-E, logged.
 *
 * Conventions for every entry point:
 *  - Return 0 (AGILE_OK) on success, a negative AGILE_ERR_* on a rejected call, or
 *    AGILE_VIOLATION (> 0) where a call reports that violations were recorded.
 *    Nothing throws across this boundary. A rejected call launches nothing.
 *  - "d_" pointers are device pointers (CUDA device memory the caller owns); "h_"
 *    pointers are host memory. `stream` is a cudaStream_t passed as void* (NULL = the
 *    legacy default stream). Device work is asynchronous on that stream unless stated.
 *  - The library owns only what it returns through agile_guard_table_t and the strings
 *    it hands out (free them with agile_free). Every buffer passed in stays the
 *    caller's, is never freed by the library and must outlive the work queued on it.
 *  - Fail closed (Sec. IV-C: unsupported operations fail closed): unknown kinds,
 *    widths, policies or PTX constructs are rejected or denied, never let through.
 */
#ifndef AGILE_GUARD_H
#define AGILE_GUARD_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define AGILE_API __attribute__((visibility("default")))
#else
#define AGILE_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- constants */

/* Range kinds: Table I's three owners of GPU virtual memory. */
enum { AGILE_USER = 0, AGILE_PROTECTED = 1, AGILE_MMIO = 2 };

/* Verdicts, one byte each. The order of the deny classes (MMIO before protected before
 * straddle) is this library's reading; the paper gives none. */
enum {
    AGILE_ALLOW = 0,          /* inside one user allocation (Sec. IV-E, V-C)          */
    AGILE_DENY_PROTECTED = 1, /* touches protected kernel/module memory               */
    AGILE_DENY_MMIO = 2,      /* touches the protected I/O aperture                   */
    AGILE_DENY_STRADDLE = 3,  /* touches user memory but not inside one allocation    */
    AGILE_DENY_UNMAPPED = 4,  /* touches no range: hole, freed or unknown address     */
    AGILE_DENY_INVALID = 5,   /* zero or illegal width, or end beyond 2^64-1          */
    AGILE_DENY_NOT_EXACT = 6  /* DMA registration: inside an allocation, not all of it */
};

/* Violation policies (Sec. V-E). TRAP exists only as instrumented PTX text. */
enum {
    AGILE_POLICY_POISON = 0,  /* denied loads read 0, denied stores/atomics dropped; logged   */
    AGILE_POLICY_SINK = 1,    /* denied loads read a zero page, stores go to a sink; logged   */
    AGILE_POLICY_REPORT = 2,  /* access proceeds unchanged; logged (audit only, not isolating) */
    AGILE_POLICY_TRAP = 3,    /* emit `trap;` before the access (instrumentation only)        */
    AGILE_POLICY_REMAP_OR = 4 /* a denied address is rewritten as addr | remap_or (the table's
                                 mask, e.g. into Table I's user aperture); the access proceeds
                                 there only if that address is allowed, else as POISON; logged */
};

/* Return codes. */
enum {
    AGILE_OK = 0,
    AGILE_VIOLATION = 1,            /* log holds at least one violation */
    AGILE_ERR_INVALID_ARG = -1,
    AGILE_ERR_OVERLAP = -2,         /* two ranges share a byte */
    AGILE_ERR_ZERO_SIZE = -3,
    AGILE_ERR_RANGE_OVERFLOW = -4,  /* base + size beyond 2^64 - 1 */
    AGILE_ERR_BAD_KIND = -5,
    AGILE_ERR_NOMEM = -6,
    AGILE_ERR_CUDA = -7,            /* a CUDA runtime call failed */
    AGILE_ERR_PTX_PARSE = -8,
    AGILE_ERR_PTX_UNSUPPORTED = -9, /* construct the guard cannot cover: rejected */
    AGILE_ERR_TIMEOUT = -10,        /* a bounded device wait gave up */
    AGILE_ERR_TOO_LARGE = -11,
    AGILE_ERR_ALIGN = -12,          /* pointer alignment the call requires */
    AGILE_ERR_NOT_FOUND = -13
};

#define AGILE_NO_RANGE 0xFFFFFFFFu
#define AGILE_LOG_BYTES 64          /* device bytes of one violation log, 16-byte aligned */
/* Bounded violation list (agile_violation_list_attach): a header, then one entry per
 * recorded violation. */
#define AGILE_LIST_HEADER_BYTES 16
#define AGILE_LIST_ENTRY_BYTES 32
#define AGILE_LIST_BYTES(capacity) (AGILE_LIST_HEADER_BYTES + (size_t)(capacity) * AGILE_LIST_ENTRY_BYTES)
#define AGILE_MAX_RANGES 0x3FFFFFFFu

/* One range of the guard table: [base, base + size), owned by `kind`. `id` is the
 * caller's tag for the range, reported in violation records. Sec. V-C: the worker
 * records each user allocation's base and requested (not rounded) size. */
typedef struct {
    uint64_t base;
    uint64_t size;
    uint32_t kind;
    uint32_t id;
} agile_range_t;

/* Host-side table object (opaque), built once per table version. */
typedef struct agile_guard_table agile_guard_table_t;

/* Device view of an uploaded table: plain data, copied by value into launches. It is
 * also stored at the start of the device buffer, so code that holds only the buffer's
 * address (instrumented PTX) reads the same fields from there. */
typedef struct {
    uint64_t lo;              /* first byte of the paged window (page aligned)          */
    uint64_t npages;          /* pages in the window; page map has npages + 1 entries  */
    uint32_t log2_page;       /* page size G = 2^log2_page bytes                         */
    uint32_t n;               /* ranges                                                  */
    const uint32_t *page;     /* page map (device)                                       */
    const uint64_t *base;     /* n bases, ascending (device)                            */
    const uint64_t *end;      /* n exclusive ends (device)                              */
    const uint32_t *kind;     /* n kinds (device)                                        */
    const uint32_t *id;       /* n caller tags (device)                                  */
    void *zero_page;          /* 64 zero bytes read by denied loads under SINK           */
    void *sink_page;          /* 64 bytes that take denied stores under SINK             */
    uint64_t bytes;           /* size of the device buffer in use                       */
    uint32_t search_steps;    /* binary-search steps that cover any page's range slice  */
    uint32_t reserved;
    const uint32_t *crange;   /* windows under 4 GiB: n records of 4 u32 {start - lo,
                                 last byte - lo, rank (0 MMIO, 1 protected, 2 user), id};
                                 else NULL                                              */
    uint64_t remap_or;        /* mask the REMAP_OR policy ORs into a denied address     */
    const uint32_t *ubits;    /* all-user block bitmap (device): bit k of word k / 32 set
                                 iff bytes [lo + k B, lo + (k+1) B) lie inside one user
                                 range, B = 2^ubits_log2 (chosen so that the bitmap is at
                                 most 32 KiB); ubits_n + 1 bits, the last always clear  */
    uint32_t ubits_log2;
    uint32_t ubits_n;         /* blocks covering the window                             */
    const uint32_t *cmap;     /* block class map (device), 2 bits per block of
                                 C = 2^cmap_log2 bytes from lo, 16 blocks per word, block k
                                 in bits 2(k mod 16)..+1 of word k / 16:
                                   1  the block lies inside one user range
                                   2  no range touches the block
                                   3  the block lies inside one protected range
                                   0  anything else (MMIO, several ranges, a boundary)
                                 C is the smallest power of two >= 256 bytes that keeps the
                                 map at 2^19 blocks (128 KiB) or fewer; cmap_n + 1 entries,
                                 the last always 2: nothing lies outside the window. Used
                                 by the batch check to decide most accesses, denied ones
                                 included, from one 2-bit code, and by the PTX pass's
                                 second inline test (class 1 allows).                   */
    uint32_t cmap_log2;
    uint32_t cmap_n;          /* blocks covering the window                             */
    const uint32_t *cdesc;    /* windows under 4 GiB: descriptors of open blocks (class 0)
                                 for the batch check's second pass, else NULL. A block
                                 with at most one range boundary strictly inside it (none:
                                 inside one MMIO range) is described by a pair of u32
                                 {block index, payload}: the boundary's offset b in the
                                 block (C when there is none) in bits 0-13, and the
                                 verdicts of an access wholly before b, wholly at or after
                                 b, and across b in bits 16-18, 20-22, 24-26. Pairs sit in
                                 2^cdesc_log2 slots, block k in slot h(k, cdesc_k1) or
                                 h(k, cdesc_k2), h(k, K) = (k * K mod 2^32) >> (32 -
                                 cdesc_log2); an empty slot holds block 0xFFFFFFFF. Blocks
                                 left out (more boundaries, or no free slot) are decided
                                 by the full rule.                                      */
    uint32_t cdesc_log2;      /* 6..12 when cdesc is not NULL                           */
    uint32_t cdesc_k1;
    uint32_t cdesc_k2;
    uint32_t cdesc_reserved;
} agile_dev_table_t;

/* Decoded violation log. The first fault is the violating access with the smallest
 * key, an order that does not depend on scheduling: for agile_guard_check_batch the
 * key is the access index; for guarded kernels it is (address, site), site being the
 * access's position in the kernel body. */
typedef struct {
    uint64_t key;
    uint64_t addr;
    uint32_t width;
    uint32_t verdict;
    uint32_t site;
    uint32_t range_id;        /* id of the range that decided the deny, or AGILE_NO_RANGE */
    uint32_t client;          /* tag given to agile_violation_log_init                   */
    uint32_t status;          /* 0, or AGILE_LOG_STATUS_* bits                            */
    uint64_t count;           /* violating accesses; 0 = no violation, other fields 0    */
} agile_violation_record_t;

#define AGILE_LOG_STATUS_TIMEOUT 1u /* a kernel's bounded wait gave up; results incomplete */

/* ---------------------------------------------------------------- table */

/* Build a table from n ranges in any order (Sec. V-A: the worker records every user
 * allocation; Sec. IV-E: protected and MMIO ranges). Ranges must be pairwise disjoint,
 * non-empty, with base + size <= 2^64 - 1 and a known kind; abutting ranges stay
 * separate (an access across two allocations is a straddle). Errors: OVERLAP,
 * ZERO_SIZE, RANGE_OVERFLOW, BAD_KIND, TOO_LARGE (n > AGILE_MAX_RANGES), NOMEM,
 * INVALID_ARG (NULL with n > 0, or log2_page outside [12, 40] and not AGILE_PAGE_AUTO).
 * The page size G is 2^log2_page; it is raised until the page map has at most 2^26
 * entries. AGILE_PAGE_AUTO picks it: the largest page from 2 MiB down to 4 KiB at which
 * at least 95% of the user bytes lie in pages wholly inside one user range (so the page
 * map alone decides accesses there), with at most 2^24 pages; else the page size with the
 * largest such share. agile_guard_table_geometry reports the choice. The caller's array
 * is copied; *out is freed with agile_guard_table_destroy. */
#define AGILE_PAGE_AUTO 0u
AGILE_API int agile_guard_table_build(const agile_range_t *h_ranges, size_t n, uint32_t log2_page,
                            agile_guard_table_t **out);

/* Mask for the REMAP_OR policy (Sec. V-E: "rewrite protected addresses into the user
 * range"), used by uploads that follow; a multiple of 16 (ALIGN otherwise) so remapped
 * vector accesses stay aligned. 0 (the default) remaps nothing. */
AGILE_API int agile_guard_table_set_remap(agile_guard_table_t *t, uint64_t remap_or);

/* Device bytes needed by agile_guard_table_upload for this table. */
AGILE_API int agile_guard_table_device_bytes(const agile_guard_table_t *t, size_t *bytes);

/* Page size actually used (log2), and the number of pages in the map. */
AGILE_API int agile_guard_table_geometry(const agile_guard_table_t *t, uint32_t *log2_page,
                               uint64_t *npages);

/* Copy the table into a caller-owned device buffer of at least device_bytes bytes,
 * 256-byte aligned (ALIGN otherwise), queued on `stream`; fills *out (host) with the
 * device view. The buffer is read-only to launches afterwards (only the 64-byte sink
 * page is written, under SINK); a new table version goes to a new buffer. The host
 * staging copy is owned by `t`, so `t` must stay alive until the stream has run it. */
AGILE_API int agile_guard_table_upload(agile_guard_table_t *t, void *d_buf, size_t bytes, void *stream,
                             agile_dev_table_t *out);

/* The same image as agile_guard_table_upload, written synchronously into a caller-owned
 * host buffer of at least device_bytes bytes, 256-byte aligned (ALIGN otherwise), with
 * *out's pointers into that buffer: for inspecting or storing a table on the host. No
 * GPU is used. */
AGILE_API int agile_guard_table_image(const agile_guard_table_t *t, void *h_buf, size_t bytes,
                                      agile_dev_table_t *out);

AGILE_API void agile_guard_table_destroy(agile_guard_table_t *t);

/* ---------------------------------------------------------------- host checks */

/* API-time pointer validation (Sec. IV-E, Sec. V-C): for each (h_ptr[i], h_bytes[i])
 * write the verdict (and, if h_range_id is not NULL, the deciding range id) -- allowed
 * only when [ptr, ptr + bytes) lies inside one live user allocation; bytes == 0 is
 * INVALID. Host only, synchronous. Returns AGILE_VIOLATION if any pair was denied. */
AGILE_API int agile_validate_args(const agile_guard_table_t *t, const uint64_t *h_ptr,
                        const uint64_t *h_bytes, size_t n, uint8_t *h_verdict,
                        uint32_t *h_range_id);

/* DMA-registration check (Sec. V-C: a service-backed module may register a user buffer
 * for device DMA, but only an exact live user allocation is accepted): for each
 * (h_ptr[i], h_bytes[i]) ALLOW only when it is exactly one user range (base and size);
 * AGILE_DENY_NOT_EXACT when it lies strictly inside one; else the verdict of
 * agile_validate_args. Host only, synchronous; AGILE_VIOLATION if any pair was refused. */
AGILE_API int agile_validate_dma(const agile_guard_table_t *t, const uint64_t *h_ptr,
                                 const uint64_t *h_bytes, size_t n, uint8_t *h_verdict,
                                 uint32_t *h_range_id);

/* ---------------------------------------------------------------- violation log */

/* Set a caller-owned AGILE_LOG_BYTES device buffer (16-byte aligned) to the empty log,
 * tagged with `client`, on `stream`. */
AGILE_API int agile_violation_log_init(void *d_log, uint32_t client, void *stream);

/* Wait for `stream`, copy the log to the host and decode it. Returns AGILE_VIOLATION
 * when count > 0 -- the poison policy's "fail at a later synchronization" (Sec. V-E) --
 * and AGILE_ERR_TIMEOUT when a kernel's bounded wait gave up. */
AGILE_API int agile_violation_log_read(const void *d_log, agile_violation_record_t *h_out, void *stream);

/* Attach a bounded violation list to a log (Sec. V-E: report counts or logs would-be
 * violations): from then on every violation recorded in d_log -- by the batch checks, the
 * hand-fused kernels, the batched launches and instrumented modules -- is also appended
 * to d_list, until `capacity` entries are taken; later ones are only counted. d_list is a
 * caller-owned device buffer of AGILE_LIST_BYTES(capacity) bytes, 16-byte aligned, with
 * capacity >= 1. Call after agile_violation_log_init (which detaches any list), on the
 * stream the kernels use; synchronous (it waits for that stream). Entries appear in the
 * order the GPU takes them. */
AGILE_API int agile_violation_list_attach(void *d_log, void *d_list, uint32_t capacity, void *stream);

/* Wait for `stream` and read an attached list: *n_seen = violations recorded since the
 * attach (appended or not), *n_out = min(n_seen, capacity, max) entries decoded into
 * h_out (key, addr, width, verdict, site and range id as in the log's first record;
 * client and status from the log; count 1). INVALID_ARG when d_log has no list or
 * d_list is not the one attached. */
AGILE_API int agile_violation_list_read(const void *d_log, const void *d_list, agile_violation_record_t *h_out,
                                        size_t max, size_t *n_out, uint64_t *n_seen, void *stream);

/* Self-test of the kernels' bounded waits (failure detection without a GPU fault). One
 * warp waits on an mbarrier that expects 16 bytes no copy will deliver -- the guard's
 * staging wait, limited to 0.25 s -- and polls *d_flag (4-byte aligned device memory)
 * for up to flag_us microseconds (1 .. 1e6). Each wait that gives up sets
 * AGILE_LOG_STATUS_TIMEOUT in d_log's status, so agile_violation_log_read then returns
 * AGILE_ERR_TIMEOUT; *d_result gets bit 0 for the barrier and bit 1 for the flag. The
 * kernel always returns; no copy is left in flight. */
AGILE_API int agile_selftest_bounded_waits(void *d_log, const uint32_t *d_flag, uint32_t flag_us,
                                           uint32_t *d_result, void *stream);

/* ---------------------------------------------------------------- device checks */

/* Batched guard check: verdict[i] for the access [d_addr[i], d_addr[i] + d_width[i])
 * (widths 1, 2, 4, 8, 16; anything else is INVALID), by the rule of Sec. IV-E as the
 * kernel guard applies it (Sec. V-E). Violations go to d_log (first fault = smallest
 * index) when d_log is not NULL. Layout: SoA, n entries each; any alignment is
 * accepted (16-byte aligned d_addr and 8-byte aligned d_width/d_verdict take the
 * vector path, unless d_log has a bounded list attached: the per-access path then runs,
 * which appends every denial). A violation is not an error: returns 0 once queued. */
AGILE_API int agile_guard_check_batch(const agile_dev_table_t *tbl, const uint64_t *d_addr,
                            const uint8_t *d_width, size_t n, uint8_t *d_verdict, void *d_log,
                            void *stream);

/* Aperture-only batched check (Table I; Sec. V-E: the paper's PTX guard tests accesses
 * against the protected I/O and kernel/module intervals only, leaving every other access
 * on the normal path). verdict[i] is INVALID as for agile_guard_check_batch; MMIO if the
 * access shares a byte with an MMIO aperture, else PROTECTED if it shares a byte with a
 * protected aperture (the lowest-based such aperture is reported); else ALLOW -- holes,
 * straddles and freed memory are not seen by this rule. h_apertures: host array of at
 * most AGILE_MAX_APERTURES non-empty, pairwise disjoint ranges of kind PROTECTED or MMIO,
 * copied into the launch. Logging, layouts and alignment as for agile_guard_check_batch.
 * Errors: INVALID_ARG, TOO_LARGE, BAD_KIND (a user aperture), ZERO_SIZE, RANGE_OVERFLOW,
 * OVERLAP, ALIGN (d_log). */
#define AGILE_MAX_APERTURES 4
AGILE_API int agile_aperture_check_batch(const agile_range_t *h_apertures, size_t n_apertures,
                                         const uint64_t *d_addr, const uint8_t *d_width, size_t n,
                                         uint8_t *d_verdict, void *d_log, void *stream);

/* ---------------------------------------------------------------- guarded kernels */

enum { AGILE_OP_COPY = 0, AGILE_OP_SCALE = 1, AGILE_OP_TRIAD = 2 };

/* Streaming kernels with the guard fused in by hand (Sec. V-E's check before every
 * global access): COPY a = b, SCALE a = s*b, TRIAD a = b + s*c as one fused
 * multiply-add. fp32, n elements; a, b, c 16-byte aligned (ALIGN otherwise), c ignored
 * unless TRIAD. Access order per 16-byte unit: load b (site 0), load c (site 1, triad),
 * store a (site 1, or 2 for triad); elements past the last whole unit use 4-byte
 * accesses. `policy` is POISON, SINK or REPORT. Violations go to d_log when it is not
 * NULL. tbl == NULL runs the unguarded twin (no checks, same code shape), for
 * measuring the guard's cost. */
AGILE_API int agile_stream_launch(int op, const agile_dev_table_t *tbl, float *d_a, const float *d_b,
                        const float *d_c, size_t n, float s, int policy, void *d_log,
                        void *stream);

/* agile_stream_launch at a chosen launch shape, so that the guard's cost can be measured
 * against the unguarded kernel at the same shape: `units` 16-byte units per lane per warp
 * tile and `blocks_per_sm` blocks of 512 threads per SM, either (8, 1) or (4, 2).
 * agile_stream_launch runs guarded kernels at (8, 1) and unguarded ones (tbl == NULL) at
 * (4, 2); the results are identical at every shape. INVALID_ARG for another shape,
 * otherwise as agile_stream_launch. (Not in the paper: a measurement aid.) */
AGILE_API int agile_stream_launch_shape(int op, const agile_dev_table_t *tbl, float *d_a,
                                        const float *d_b, const float *d_c, size_t n, float s,
                                        int policy, void *d_log, int units, int blocks_per_sm,
                                        void *stream);

/* agile_stream_launch over host arrays: the inputs come from host memory and the result
 * goes back to it, with the copies inside the call. The n elements are cut into chunks of
 * chunk_elems (a multiple of 4; 0 picks 2^24). Chunk k runs on one of three internal
 * streams: copy h_b (and h_c for TRIAD) into d_b (d_c) at the chunk's offset, run the
 * guarded kernel on the chunk, copy d_a back to h_a. So copies in both directions overlap
 * with each other and with other chunks' kernels. A NULL h_b / h_c skips that input's copy
 * (the device array already holds it); a NULL h_a skips the copy out. The kernel makes
 * the same accesses at the same addresses as one launch over all n elements, so outputs
 * and the log match it exactly. The device arrays are the ones the table guards. Pinned
 * host memory is needed for the copies to overlap. Ordered after earlier work on `stream`;
 * later work on `stream` waits for the whole call. Errors as agile_stream_launch, plus
 * INVALID_ARG for chunk_elems not a multiple of 4. Arguments are checked before anything
 * is queued, so a rejected call queues nothing; a CUDA failure part-way returns
 * AGILE_ERR_CUDA after making `stream` wait for the chunks already queued, so buffers
 * may be reused once `stream` has been synchronized. The three streams and four events
 * are created on the first call per device and calling thread and kept until exit. */
AGILE_API int agile_stream_launch_host(int op, const agile_dev_table_t *tbl, float *d_a,
                                       float *d_b, float *d_c, float *h_a, const float *h_b,
                                       const float *h_c, size_t n, float s, int policy,
                                       void *d_log, size_t chunk_elems, void *stream);

enum { AGILE_IRR_GATHER = 0, AGILE_IRR_SCATTER = 1, AGILE_IRR_HIST = 2 };

/* Irregular kernels with the guard fused in by hand (Sec. V-E), n elements, d_idx int64
 * element offsets (16-byte aligned) that the kernel turns into addresses
 * d_base + 4 * d_idx[i] -- the data-dependent addresses the guard exists for:
 *   GATHER  d_out[i] = ((float *)d_base)[d_idx[i]]            (d_out 16-byte aligned)
 *   SCATTER ((float *)d_base)[d_idx[i]] = (float)(d_idx[i] & 0xFFFFFF)
 *   HIST    ((uint32_t *)d_base)[d_idx[i]] += 1 (atomic)
 * Access order per group of four elements: two 16-byte index loads (sites 0, 1), the
 * four element accesses (site 2), gather's 16-byte output store (site 3); elements past
 * the last whole group use an 8-byte index load, the element access and a 4-byte store.
 * Policies and tbl == NULL as for agile_stream_launch, plus REMAP_OR (the table's
 * remap_or mask); under POISON a denied index load reads 0 and a denied element load
 * reads 0.0f. */
AGILE_API int agile_irregular_launch(int kind, const agile_dev_table_t *tbl, const int64_t *d_idx,
                                     void *d_base, float *d_out, size_t n, int policy,
                                     void *d_log, void *stream);

/* How a guarded irregular kernel reads the all-user bitmap for its per-lane element
 * accesses: AGILE_FAST_BITMAP, each lane reads its own word (what agile_irregular_launch
 * does); AGILE_FAST_MATCH, lanes whose elements fall in the same bitmap block are grouped
 * with __match_any_sync, the group's leader reads the word and __shfl_sync hands it on.
 * Both give identical results and logs. (Not in the paper: kept so the two warp-level
 * fast paths can be measured against each other.) AGILE_FAST_MATCH needs a table and the
 * POISON policy, INVALID_ARG otherwise; other arguments as agile_irregular_launch. */
enum { AGILE_FAST_BITMAP = 0, AGILE_FAST_MATCH = 1 };
AGILE_API int agile_irregular_launch_fastpath(int kind, const agile_dev_table_t *tbl,
                                              const int64_t *d_idx, void *d_base, float *d_out,
                                              size_t n, int policy, void *d_log, int fast_path,
                                              void *stream);

/* ---------------------------------------------------------------- batched clients */

/* Kinds of work a batch item runs: the streaming and irregular kernels above. */
enum {
    AGILE_WORK_COPY = 0, AGILE_WORK_SCALE = 1, AGILE_WORK_TRIAD = 2,
    AGILE_WORK_GATHER = 3, AGILE_WORK_SCATTER = 4, AGILE_WORK_HIST = 5
};

/* One client's guarded kernel inside a batch (64 bytes). Streaming kinds: out = a,
 * in0 = b, in1 = c (TRIAD only), s the scalar. Irregular kinds: in0 = int64 offsets,
 * in1 = the table or bins base, out = gather's output. `table` is the device address of
 * the client's uploaded table buffer (256-byte aligned; NULL runs the item unguarded),
 * `log` the client's violation log (may be NULL). Alignment as for the single launches. */
typedef struct {
    uint32_t op;
    uint32_t policy;
    uint64_t n;
    const void *table;
    void *log;
    void *out;
    const void *in0;
    const void *in1;
    float s;
    uint32_t client;
} agile_work_t;

/* Launch shape of a batch. */
typedef struct {
    uint32_t tile;            /* elements per tile, a multiple of 512                      */
    uint32_t span_checks;     /* 1: one check per contiguous warp span; 0: every access    */
    uint32_t blocks_per_sm;   /* 1 or 2 resident 512-thread blocks per SM                  */
    uint32_t reserved;        /* set by the library                                        */
} agile_batch_config_t;

/* Result of agile_batch_autotune. */
typedef struct {
    agile_batch_config_t config;
    uint32_t variant;         /* which of the work-list variants won (e.g. page size)      */
    uint32_t cached;          /* 1 when read from the cache file                          */
    float ms;                 /* mean time of one launch                                   */
} agile_batch_tuning_t;

/* A captured, instantiated CUDA graph (opaque). */
typedef struct agile_graph agile_graph_t;

/* Device bytes of a batch buffer for up to max_items work items. */
AGILE_API size_t agile_batch_device_bytes(size_t max_items);

/* Check the n work items (INVALID_ARG / ALIGN as the single launches would) and copy
 * them, with their tile prefix sums for `tile`, into the caller-owned d_buf (256-byte
 * aligned, >= agile_batch_device_bytes(n)). Synchronous on `stream`. */
AGILE_API int agile_batch_upload(const agile_work_t *h_items, size_t n, uint32_t tile,
                                 void *d_buf, size_t bytes, void *stream);

/* Run an uploaded batch as one persistent launch (Sec. IV-B: one worker runs the CUDA
 * operations of many clients; Sec. V-E: each client's kernel guarded by its own table,
 * logging into its own log). Blocks claim tiles from a counter in d_buf, which this
 * call resets first (a memset, then the kernel, on `stream`). n_items must match the
 * upload. Each client's outputs and log equal those of its single launch. */
AGILE_API int agile_batch_launch(void *d_buf, size_t n_items, const agile_batch_config_t *cfg,
                                 void *stream);

/* Capture agile_batch_launch(d_buf, n_items, cfg) into a CUDA graph and instantiate it.
 * Replays read the work list in d_buf at replay time, so re-uploading a list of the same
 * length (and tile) and replaying runs the new list. */
AGILE_API int agile_batch_graph_create(void *d_buf, size_t n_items, const agile_batch_config_t *cfg,
                                       agile_graph_t **out);
AGILE_API int agile_graph_launch(agile_graph_t *g, void *stream);
AGILE_API void agile_graph_destroy(agile_graph_t *g);

/* Maximum work items of agile_batch_launch_static. */
#define AGILE_BATCH_STATIC_MAX_ITEMS 2048

/* agile_batch_upload + agile_batch_launch without any device allocation: the batch's
 * scratch (work list, tile prefix sums, tile-claim counter) lives in a fixed device
 * array inside the library (about 147 KB, held by every GPU that loads the library).
 * The paper has no counterpart; it is for callers that cannot allocate device memory --
 * a worker whose budget is fully handed out, code that must avoid the implicit
 * synchronization of cudaMalloc/cudaFree, a plugin given no allocator. The caller still
 * provides every input and output. TOO_LARGE above AGILE_BATCH_STATIC_MAX_ITEMS items;
 * other errors as agile_batch_upload. The first call on a device looks up the array's
 * device address, so make it before any stream capture; the address is kept for the
 * process's life, so no call may follow a cudaDeviceReset of that device. All calls share
 * the array: calls that overlap on the GPU race. */
AGILE_API int agile_batch_launch_static(const agile_work_t *h_items, size_t n, uint32_t tile,
                                        const agile_batch_config_t *cfg, void *stream);

/* Pick the fastest launch for a batch: every variant (n_variants work lists of n_items
 * each, back to back in h_variants -- e.g. the same work with tables of different page
 * sizes) x every candidate tile x span checks on/off x 1 or 2 blocks per SM, timed with
 * CUDA events over `reps` launches after one warm-up. The items really run: outputs of
 * non-idempotent kinds (HIST) and the logs must be reset afterwards. With cache_path,
 * a result keyed by the items' kinds and sizes is read from / appended to that file.
 * The winning variant is left uploaded only if it was the last one tried; upload it
 * again before launching. */
AGILE_API int agile_batch_autotune(const agile_work_t *h_variants, size_t n_variants,
                                   size_t n_items, const uint32_t *tiles, size_t n_tiles,
                                   void *d_buf, size_t bytes, int reps, const char *cache_path,
                                   void *stream, agile_batch_tuning_t *best);

/* ---------------------------------------------------------------- serving worker */

#define AGILE_MAX_ARGS 16

/* One client request: validate its pointer arguments, then run its guarded kernel. */
typedef struct {
    uint64_t tag;                       /* caller's id, echoed in the completion            */
    uint32_t client;                    /* client index given to agile_worker_create         */
    uint32_t nargs;                     /* pointer arguments to validate (<= AGILE_MAX_ARGS) */
    uint64_t arg_ptr[AGILE_MAX_ARGS];
    uint64_t arg_bytes[AGILE_MAX_ARGS];
    agile_work_t work;                  /* its kernel; NULL table/log take the client's      */
    uint64_t mem_bytes;                 /* device memory it holds while admitted             */
    uint64_t excl;                      /* nonzero: requests with equal keys never overlap    */
    uint64_t arrival_ns;                /* arrival time on the worker clock (ns from start)  */
} agile_request_t;

/* What happened to a request. */
typedef struct {
    uint64_t tag;
    int32_t status;                     /* AGILE_OK; AGILE_VIOLATION: rejected at validation;
                                           AGILE_ERR_TOO_LARGE: can never fit the budget     */
    uint32_t bad_arg;                   /* first denied argument (rejections)                */
    uint32_t verdict;                   /* its verdict                                       */
    uint32_t launch;                    /* sequence number of the launch that ran it         */
    uint64_t arrival_ns;                /* worker clock: arrival time given with the request  */
    uint64_t admit_ns;                  /* packed into a launch                              */
    uint64_t done_ns;                   /* completed: its kernel's last tile done (the
                                           launch's completion notice), or rejected          */
    uint64_t seen_ns;                   /* taken up and validated by the worker              */
    uint64_t queued_ns;                 /* its launch's copy and kernel queued on the stream  */
} agile_completion_t;

typedef struct {
    uint64_t mem_budget;                /* cap on the sum of admitted requests' mem_bytes    */
    uint32_t max_batch;                 /* requests per launch                               */
    uint32_t max_inflight;              /* launches in flight, one stream each              */
    uint32_t tile;                      /* batch tile (multiple of 512)                      */
    uint32_t continuous;                /* 1: continuous batching; 0: one request at a time  */
} agile_worker_config_t;

typedef struct agile_worker agile_worker_t;

/* Device bytes of the worker's batch buffers (max_inflight of them). */
AGILE_API size_t agile_worker_device_bytes(const agile_worker_config_t *cfg);

/* A worker serving n_clients clients (Sec. IV-B: a trusted worker owns the context and
 * executes the clients' requests; Sec. IV-C / V-C: every pointer argument is validated
 * against the client's live allocations before any launch). h_tables[i] (host, for
 * validation) and d_tables[i] (uploaded, for the guard) are client i's table; d_logs[i]
 * its log. d_buf (256-byte aligned, agile_worker_device_bytes) holds the launches' work
 * lists. The worker thread starts with agile_worker_start; its clock starts there.
 * Tables, logs and d_buf must outlive the worker. */
AGILE_API int agile_worker_create(const agile_worker_config_t *cfg,
                                  const agile_guard_table_t *const *h_tables,
                                  const agile_dev_table_t *const *d_tables, void *const *d_logs,
                                  size_t n_clients, void *d_buf, size_t bytes,
                                  agile_worker_t **out);

/* Queue requests (thread-safe, any time). Each is considered once the worker clock
 * passes its arrival time: validated (a denied argument completes it at once with
 * AGILE_VIOLATION), then admitted in arrival order when the memory budget, a launch slot
 * and its exclusive key allow; admitted requests are packed into the next persistent
 * launch while earlier launches still run (continuous batching). Each request completes
 * on its own: the launch raises a per-request notice in host-mapped memory when the
 * request's last tile is done, and the worker then completes it and returns its memory
 * to the budget, while the rest of that launch may still run. */
AGILE_API int agile_worker_submit(agile_worker_t *w, const agile_request_t *reqs, size_t n);
AGILE_API int agile_worker_start(agile_worker_t *w);

/* Take up to cap completions; waits up to wait_ms for at least one. */
AGILE_API int agile_worker_poll(agile_worker_t *w, agile_completion_t *out, size_t cap,
                                size_t *got, uint32_t wait_ms);

/* Current worker clock (ns since start) and admitted bytes (for tests of the budget). */
AGILE_API int agile_worker_clock(agile_worker_t *w, uint64_t *now_ns, uint64_t *admitted_bytes,
                                 uint64_t *peak_admitted_bytes);

/* Stop after every queued request has completed, then free the worker. */
AGILE_API void agile_worker_destroy(agile_worker_t *w);

/* ---------------------------------------------------------------- PTX guard pass */

typedef struct {
    int policy;                    /* AGILE_POLICY_*                                     */
    const char *const *skip;       /* functions left unguarded (trusted module bodies,   */
    size_t nskip;                  /*   Sec. V-E); may be NULL                            */
    const agile_range_t *apertures; /* with napertures > 0: the aperture rule (Table I;   */
    size_t napertures;             /*   rules as agile_aperture_check_batch) compiled into
                                         the module as constants, in place of the table;
                                         REMAP_OR is then refused                        */
} agile_instrument_opts_t;

typedef struct {
    uint32_t functions;            /* .entry/.func bodies seen                           */
    uint32_t guarded;              /* global accesses given a guard                      */
    uint32_t generic_guarded;      /* generic-space accesses guarded behind isspacep     */
    uint32_t skipped;              /* accesses left alone inside skipped functions       */
} agile_instrument_report_t;

/* Instrument PTX text (Sec. V-E): before every ld/st/atom/red on global memory
 * (and every generic-space one that resolves to global) insert the guard sequence for
 * `policy`; functions named in opts->skip stay unguarded. The table address comes from
 * a module-scope `.global .u64 __agile_guard_table` and the log from
 * `__agile_guard_log`, so kernel signatures do not change. Entry functions count their
 * denials in registers and merge them into the log before each ret and exit, so the log
 * is complete once the kernel has finished; under TRAP, and in modules where a called
 * function can exit the thread, each denial is merged as it happens. Input that already
 * names `__ag` symbols or registers, bulk/tensor copies and other forms the guard cannot
 * cover are rejected (PTX_UNSUPPORTED). *out (NUL terminated, length *out_len) is freed
 * with agile_free. Host only. */
AGILE_API int agile_guard_instrument_ptx(const char *ptx, size_t len, const agile_instrument_opts_t *opts,
                               char **out, size_t *out_len, agile_instrument_report_t *report);

/* A loaded instrumented module (opaque). */
typedef struct agile_module agile_module_t;

/* Load instrumented PTX into the current device's context (JIT for sm_103a). */
AGILE_API int agile_module_load(const char *ptx, agile_module_t **out);

/* Point the module's guard globals at an uploaded table's device buffer and a log
 * (d_log may be NULL: violations then go unrecorded). Synchronous. INVALID_ARG for a
 * module that was not instrumented, or for tbl == NULL unless the module was
 * instrumented with apertures (it then needs only the log). */
AGILE_API int agile_module_bind(agile_module_t *m, const agile_dev_table_t *tbl, void *d_log, void *stream);

/* Launch kernel `name` of the module: grid and block sizes, `args` = array of
 * pointers to each kernel parameter (cudaLaunchKernel convention). An instrumented
 * module is refused (INVALID_ARG) until agile_module_bind has run; NOT_FOUND for an
 * unknown kernel name. */
AGILE_API int agile_module_launch(agile_module_t *m, const char *name, uint32_t grid, uint32_t block,
                        void **args, void *stream);

AGILE_API void agile_module_unload(agile_module_t *m);

/* ---------------------------------------------------------------- misc */

AGILE_API void agile_free(void *p);
AGILE_API const char *agile_strerror(int code);
/* Library version as 0xMMmmpp. */
AGILE_API uint32_t agile_version(void);

#ifdef __cplusplus
}
#endif
#endif /* AGILE_GUARD_H */
