// Batched guard check: one verdict per (address, width) pair, the Sec. IV-E rule applied
// as the kernel guard of Sec. V-E applies it, with the first violation (smallest index)
// and the violation count in the log.
//
// Launch shape: one 1024-thread block per SM, a warp-uniform grid-stride loop. Each lane
// takes kG groups of 8 consecutive accesses per round (four 16-byte address loads, one
// 8-byte width load, one 8-byte verdict store per group). Staged into shared memory by
// bulk copies: the block class map (2 bits per block of 256 B or more) and, where they
// fit beside it, the page map and the packed range records (windows under 4 GiB) or the
// range arrays.
//
// Pass 1 decides each access from its block's 2-bit class alone, without branches: an
// access inside one block of class user, hole or protected gets ALLOW, UNMAPPED or
// PROTECTED. The rest -- blocks holding a boundary, MMIO blocks, accesses that cross a
// block edge, lie below the window in 32-bit mode, illegal widths -- are "open"; accesses
// wholly beyond the window read its last entry, "unmapped". Pass 2 deals the
// warp's open accesses out over its lanes, 32 at a time. Where the table has open-block
// descriptors (windows under 4 GiB), an access inside a described block is decided from
// its block's descriptor: one boundary and three verdicts. The rest go to a per-warp
// queue in shared memory, and each time it holds 32 of them the warp decides those 32
// by the full rule (the 32-bit uniform decision over the packed records where it
// applies). Each thread keeps its smallest violation in registers; the block reduces
// them once at the end.
#include <cuda_runtime.h>

#include "agile_internal.h"
#include "guard_device.cuh"

namespace {

using agile::LaneLog;
using agile::LogDev;
using agile::TView;

constexpr int kThreads = 1024;   // one block per SM

// Dynamic shared memory a launch may stage (the static part -- mbarrier, log reduction --
// takes about 1 KB of the 227 KB an SM gives one block).
constexpr uint64_t kStageBudget = 224 * 1024;

// Uniform decision in 32-bit arithmetic, for tables whose window spans under 4 GiB (the
// packed records hold each range's start and last byte as offsets from the window start,
// its kind and id). Every lane runs the same steps: the page entry, the fixed-step search
// for the last range starting at or below the access, then the three ranges around that
// point -- that range and the next two -- tested with selects. Allowed when the first holds
// the whole access; otherwise the touched ranges' class (MMIO, then protected, then user,
// the lowest-based range of that class reported) or unmapped. Returns false -- leaving the
// full rule to decide -- when a fourth range may be touched or the access crosses the
// window's lower edge. A warp therefore runs one path per access whatever mix of
// verdicts its lanes see.
__device__ __forceinline__ bool decide32(const TView &V, uint64_t a, uint32_t w, uint32_t *v,
                                         uint32_t *rid) {
    const uint64_t off = a - V.lo;
    if (off > V.last - V.lo) {                       // outside the window
        if (a < V.lo && a + w > V.lo) return false;  // reaches into it
        *v = AGILE_DENY_UNMAPPED;
        *rid = agile::kNoRange;
        return true;
    }
    const uint32_t o = (uint32_t)off;
    const uint64_t oe = (uint64_t)o + w - 1;         // last byte, relative
    const uint32_t p = o >> V.lg;
    const uint32_t n = V.n;
    const uint32_t f = V.page[p] & agile::kIdxMask, f2 = V.page[p + 1] & agile::kIdxMask;
    const uint32_t hi = f2 + 1 < n ? f2 + 1 : n;
    uint32_t b = f, len = hi - f;
    for (uint32_t it = 0; it < V.steps; ++it) {
        const uint32_t half = len >> 1;
        const uint32_t probe = b + half < n ? b + half : n - 1;
        const bool le = len > 0 && V.crange[probe].x <= o;
        b = le ? b + half + 1 : b;
        len = le ? len - half - 1 : half;
    }
    const bool v0 = b > 0, v1 = b < n, v2 = b + 1 < n, v3 = b + 2 < n;
    const uint4 r0 = V.crange[v0 ? b - 1 : 0];
    const uint4 r1 = V.crange[v1 ? b : 0];
    const uint4 r2 = V.crange[v2 ? b + 1 : 0];
    const uint32_t s3 = V.crange[v3 ? b + 2 : 0].x;
    if (v3 && (uint64_t)s3 <= oe) return false;      // a fourth range may be touched
    const bool t0 = v0 && r0.y >= o;                 // r0 starts at or below o
    const bool t1 = v1 && (uint64_t)r1.x <= oe;      // r1, r2 start above o
    const bool t2 = v2 && (uint64_t)r2.x <= oe;
    // .z is the deny rank: 0 MMIO, 1 protected, 2 user
    if (t0 && r0.z == 2u && (uint64_t)r0.y >= oe) {
        *v = AGILE_ALLOW;
        *rid = r0.w;
        return true;
    }
    uint32_t best = t0 ? r0.z : 3u, id = r0.w;
    id = (t1 && r1.z < best) ? r1.w : id;
    best = (t1 && r1.z < best) ? r1.z : best;
    id = (t2 && r2.z < best) ? r2.w : id;
    best = (t2 && r2.z < best) ? r2.z : best;
    *v = (0x04030102u >> (8 * best)) & 0xFFu;        // rank 0..3 -> MMIO, PROTECTED, STRADDLE, UNMAPPED
    *rid = best == 3 ? agile::kNoRange : id;
    return true;
}

// x >> s with the PTX rule for shift counts of 32 and more (the result is 0).
__device__ __forceinline__ uint32_t shr_clamped(uint32_t x, uint32_t s) {
    uint32_t r;
    asm("shr.b32 %0, %1, %2;" : "=r"(r) : "r"(x), "r"(s));
    return r;
}

__device__ __forceinline__ bool legal_width(uint32_t w) {
    return shr_clamped(0x10116u, w) & 1u;             // 1, 2, 4, 8, 16
}

// Pass-1 class of one access from the block class map: the 2-bit code of its block (1
// user, 2 hole, 3 protected) when the access is decided here -- it lies inside that block
// and has a legal width; an access wholly beyond the window reads the map's last entry, 2
// -- else 0 ("open": the block holds a boundary or MMIO, the access crosses the block's
// end, lies below the window in 32-bit mode, or has an illegal width). C32: the window
// spans under 4 GiB, so block index and offset are 32-bit.
template <bool C32>
__device__ __forceinline__ uint32_t cmap_code(const TView &V, uint64_t a, uint32_t w) {
    const uint64_t off = a - V.lo;
    uint32_t blk;
    bool ok;
    if constexpr (C32) {
        const uint32_t o = (uint32_t)off;
        const uint32_t k = o >> V.clg;
        blk = k < V.cn ? k : V.cn;                     // past the window: its "unmapped" entry
        const uint32_t m = (1u << V.clg) - 1u;
        // An illegal width gets 2^30 added (a multiply-add, FMA pipe), so that it fails the
        // in-block test: blocks are at most 2^13 bytes here, and the sum cannot wrap.
        const uint32_t bad = ~shr_clamped(0x10116u, w) & 1u;
        uint32_t wf;
        asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(wf) : "r"(bad), "r"(1u << 30), "r"(w));
        ok = (off >> 32) == 0 && (o & m) + wf <= m + 1u;
    } else {
        const uint64_t k = off >> V.clg;
        blk = k < V.cn ? (uint32_t)k : V.cn;
        const uint64_t m = (1ull << V.clg) - 1;
        ok = (off & m) + w <= m + 1;
    }
    // 16 codes per word: rotating the word by 2 * blk (mod 32) brings this block's to bit 0.
    // The doubling is a multiply, so that it issues on the FMA pipe: pass 1 is bound by
    // the integer ALU pipe while the FMA pipe idles.
    const uint32_t word = V.cmap[blk >> 4];
    uint32_t sh;
    asm("mul.lo.u32 %0, %1, 2;" : "=r"(sh) : "r"(blk));
    const uint32_t code = __funnelshift_r(word, word, sh) & 3u;
    if constexpr (C32) return ok ? code : 0u;           // illegal widths failed above
    return ok && legal_width(w) ? code : 0u;
}

// Pass-2 decision from the open-block descriptors (windows under 4 GiB), for an access
// with a legal width: inside one described block, from its descriptor; wholly outside
// the window (which spans less than 4 GiB from lo), UNMAPPED. False otherwise -- no
// descriptor, across a block edge, reaching into the window from below, an end past
// 2^64 - 1 -- and the full rule decides. Branch-free: both slots of the two-choice hash
// are read.
__device__ __forceinline__ bool desc_decide(const TView &V, uint64_t a, uint32_t w, uint32_t *v) {
    const uint64_t off = a - V.lo;
    const uint32_t o = (uint32_t)off;
    const uint32_t k = o >> V.clg;
    const uint32_t oi = o & ((1u << V.clg) - 1u), e = oi + w;
    const uint32_t sh = 32u - V.dlg;                   // dlg >= 6
    const uint2 d1 = V.cdesc[(k * V.dk1) >> sh], d2 = V.cdesc[(k * V.dk2) >> sh];
    const bool hit = d1.x == k || d2.x == k;
    const uint32_t p = d1.x == k ? d1.y : d2.y;
    const uint32_t b = p & 0x3FFFu;                    // the boundary, C when none
    const uint32_t f = e <= b ? 16u : oi >= b ? 20u : 24u;   // before, at or after, across
    const bool outside = (off >> 32) != 0;
    const bool clear = !(a < V.lo && a + w > V.lo) && a <= ~0ull - w;
    *v = outside ? (uint32_t)AGILE_DENY_UNMAPPED : (p >> f) & 7u;
    return legal_width(w) && (outside ? clear : hit && e <= (1u << V.clg));
}

// Full rule for one access (pass 2, the n mod 8 tail, and the misaligned form).
template <bool C32>
__device__ __forceinline__ uint32_t full_rule(const TView &V, uint64_t a, uint32_t w, uint32_t *rid) {
    *rid = agile::kNoRange;
    if (!legal_width(w) || a > ~0ull - w) return AGILE_DENY_INVALID;
    uint32_t v;
    if constexpr (C32) {
        if (decide32(V, a, w, &v, rid)) return v;
        return agile::classify_slow(V, a, w, rid);
    } else {
        return agile::classify(V, a, w, rid);
    }
}

// Per-warp queue of open accesses the descriptors left undecided: fewer than 32 wait
// between rounds, and a round adds at most 32. An entry holds the access itself (its
// index with the width in the top byte, and its address), so that deciding it later
// does not read the inputs again: by then they may have left L2.
constexpr uint32_t kQueue = 64;
constexpr uint32_t kQueueBytes = kThreads / 32 * kQueue * 16;
constexpr uint64_t kIndexMask = (1ull << 56) - 1;   // indices below 2^56
// Per-warp list of a round of groups' open accesses (lane << 5 | bit), written by their
// owners, when they number at most kList.
constexpr uint32_t kList = 256;
constexpr uint32_t kListBytes = kThreads / 32 * kList * 2;

template <int MODE, bool C32, int kG>
__global__ void __launch_bounds__(kThreads, 1)
k_check_batch(const agile_dev_table_t T, const uint64_t *__restrict__ addr,
              const uint8_t *__restrict__ width, uint8_t *__restrict__ verdict, size_t n,
              LogDev *log) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned long long s_bar;
    const TView V = agile::stage_table<MODE>(T, smem, &s_bar, log);
    constexpr bool kDesc = C32 && (MODE & agile::ST_CDESC);
    // the queue and the list follow the staged sections
    const uint32_t staged = (uint32_t)agile::stage_bytes(T, MODE);
    ulonglong2 *s_q = reinterpret_cast<ulonglong2 *>(smem + staged) + (threadIdx.x >> 5) * kQueue;
    uint16_t *s_list = reinterpret_cast<uint16_t *>(smem + staged + kQueueBytes) + (threadIdx.x >> 5) * kList;
    uint32_t qn = 0;                   // queued (warp-uniform)

    const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t nthreads = (size_t)gridDim.x * blockDim.x;
    const size_t ngroups = n / 8;
    const uint32_t lane = threadIdx.x & 31;
    // Pass-2 violations: their count and smallest key (access index). The block's smallest
    // violation gets its record from the full rule at the end (see below), so no lane keeps
    // more than the key.
    LaneLog ll;
    auto note_key = [&](size_t i) {
        ++ll.cnt;
        ll.key = i < ll.key ? i : ll.key;
    };
    // Full rule for access i = (a, w), noting a violation.
    auto decide_at = [&](size_t i, uint64_t a, uint32_t w) {
        uint32_t rid;
        const uint32_t v = full_rule<C32>(V, a, w, &rid);
        if (v != AGILE_ALLOW) {
            note_key(i);
            verdict[i] = (uint8_t)v;
        }
    };
    uint32_t cnt1 = 0;                 // pass-1 denials
    size_t first1 = ~(size_t)0;        // this lane's first pass-1 denial (its smallest)

    // Groups g0 + 32h + lane (h < kG), coalesced across the warp.
    for (size_t g0 = (tid - lane) * kG; g0 < ngroups; g0 += nthreads * kG) {   // warp-uniform
        uint32_t open = 0;             // bit 4k + h: access k of group h not decided in pass 1
#pragma unroll
        for (int h = 0; h < kG; ++h) {
            const size_t g = g0 + 32 * h + lane;
            if (g >= ngroups) continue;
            // Default-cached loads: pass 2 re-reads its open accesses from L1 or L2.
            const uint4 *pa = reinterpret_cast<const uint4 *>(addr + g * 8);
            uint64_t av[8];
#pragma unroll
            for (int k = 0; k < 4; ++k) {              // registers only: no indexed arrays
                const uint4 q = __ldg(pa + k);
                av[2 * k] = (uint64_t)q.y << 32 | q.x;
                av[2 * k + 1] = (uint64_t)q.w << 32 | q.z;
            }
            const uint64_t wv = __ldg(reinterpret_cast<const unsigned long long *>(width + g * 8));
            // The eight codes, access k's in nibble k. A byte permute turns four nibbles into
            // four verdict bytes at once: code c selects byte c of 0x01040000, so 0 (open)
            // and 1 (user) give ALLOW, 2 (hole) UNMAPPED, 3 (protected) PROTECTED.
            uint32_t sel = 0;
#pragma unroll
            for (int k = 0; k < 8; ++k) {           // sel += code << 4k, as a multiply-add (FMA pipe)
                // width byte k by one byte permute
                const uint32_t wk = __byte_perm(k < 4 ? (uint32_t)wv : (uint32_t)(wv >> 32), 0u,
                                                0x4440u | (uint32_t)(k & 3));
                const uint32_t cd = cmap_code<C32>(V, av[k], wk);
                asm("mad.lo.u32 %0, %1, %2, %0;" : "+r"(sel) : "r"(cd), "r"(1u << (4 * k)));
            }
            const uint32_t vlo = __byte_perm(0x01040000u, 0u, sel);
            const uint32_t vhi = __byte_perm(0x01040000u, 0u, sel >> 16);
            __stcs(reinterpret_cast<unsigned long long *>(verdict + g * 8),
                   (unsigned long long)vhi << 32 | vlo);
            const uint32_t nz = (sel | (sel >> 1)) & 0x11111111u;   // nibble k: access k decided
            open |= (~nz & 0x11111111u) << h;
            const uint32_t dn = (sel >> 1) & 0x11111111u;           // decided denials (codes 2, 3)
            cnt1 += __popc(dn);
            if (dn != 0 && first1 == ~(size_t)0) first1 = g * 8 + ((__ffs(dn) - 1) >> 2);
        }
        // Pass 2: the warp's open accesses are dealt out to its lanes, 32 at a time, so
        // the full decision runs ceil(open / 32) times per warp rather than once for
        // every position any lane has open.
        const uint32_t c = __popc(open);
        uint32_t incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(agile::kFull, incl, o);
            if (lane >= (uint32_t)o) incl += t;
        }
        const uint32_t total = __shfl_sync(agile::kFull, incl, 31);
        const uint32_t excl = incl - c;
        // Index of the warp's q-th open access (q < total), called by all lanes: its owner
        // is the first lane whose inclusive count exceeds q, and it is bit 4k + h of the
        // owner's mask, the (q - owner's exclusive count + 1)-th bit set there.
        auto dealt = [&](uint32_t q) -> size_t {
            uint32_t own = 0;                          // lanes whose open accesses all precede q
#pragma unroll
            for (int step = 16; step; step >>= 1) {
                const uint32_t t = __shfl_sync(agile::kFull, incl, own + step - 1);
                own = t <= q ? own + step : own;
            }
            const uint32_t omask = __shfl_sync(agile::kFull, open, own & 31);
            const uint32_t oexcl = __shfl_sync(agile::kFull, excl, own & 31);
            const int b = (int)__fns(omask, 0, (int)(q - oexcl) + 1);
            return (g0 + 32 * (b & 3) + own) * 8 + (b >> 2);
        };
        __syncwarp();                                  // the pass-1 stores above come first
        if constexpr (kDesc) {
            // Where they fit the warp's list, each lane writes out its own open accesses,
            // in order from its exclusive count, and a round reads its access's position
            // there; else the owner search deals them.
            const bool listed = total <= kList;            // warp-uniform
            if (listed) {
                uint32_t m = open, pos = excl;
                while (m != 0) {
                    s_list[pos++] = (uint16_t)(lane << 5 | (uint32_t)(__ffs(m) - 1));
                    m &= m - 1;
                }
                __syncwarp();
            }
            // Two rounds at a time: both rounds' inputs are loaded before either is decided.
            for (uint32_t q0 = 0; q0 < total; q0 += 64) {
                size_t ir[2] = {0, 0};
                uint64_t ar[2] = {0, 0};
                uint32_t wr[2] = {0, 0};
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const uint32_t q = q0 + 32 * r + lane;
                    if (r == 1 && q0 + 32 >= total) break;          // warp-uniform
                    size_t i = 0;
                    if (listed) {
                        if (q < total) {
                            const uint32_t id = s_list[q];          // lane << 5 | (4k + h)
                            i = (g0 + 32 * (id & 3) + (id >> 5)) * 8 + ((id >> 2) & 7);
                        }
                    } else {
                        i = dealt(q);
                    }
                    if (q < total) {
                        ir[r] = i;
                        ar[r] = addr[i];
                        wr[r] = width[i];
                    }
                }
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    bool und = false;
                    if (q0 + 32 * r + lane < total) {
                        uint32_t v;
                        und = !desc_decide(V, ar[r], wr[r], &v);
                        if (!und && v != AGILE_ALLOW) {
                            note_key(ir[r]);
                            verdict[ir[r]] = (uint8_t)v;
                        }
                    }
                    const uint32_t um = __ballot_sync(agile::kFull, und);
                    if (und)
                        s_q[qn + __popc(um & ((1u << lane) - 1u))] =
                            make_ulonglong2(ir[r] | (uint64_t)wr[r] << 56, ar[r]);
                    qn += __popc(um);
                    if (qn >= 32) {                    // a full round of the full rule
                        __syncwarp();
                        const ulonglong2 e = s_q[qn - 32 + lane];
                        decide_at(e.x & kIndexMask, e.y, (uint32_t)(e.x >> 56));
                        qn -= 32;
                        __syncwarp();                  // read before the slots are reused
                    }
                }
            }
            __syncwarp();                              // the list is read before it is rewritten
        } else {
            for (uint32_t q0 = 0; q0 < total; q0 += 32) {
                const uint32_t q = q0 + lane;
                const size_t i = dealt(q);
                if (q < total) decide_at(i, addr[i], width[i]);
            }
        }
    }
    if (kDesc && qn > 0) {                             // what is left in the queue
        __syncwarp();
        if (lane < qn) {
            const ulonglong2 e = s_q[lane];
            decide_at(e.x & kIndexMask, e.y, (uint32_t)(e.x >> 56));
        }
    }
    if (blockIdx.x == 0 && threadIdx.x < 32) {        // the last n % 8 accesses
        const size_t i = ngroups * 8 + threadIdx.x;
        if (i < n) {
            const uint64_t a = addr[i];
            const uint32_t w = width[i];
            uint32_t rid;
            const uint32_t v = full_rule<C32>(V, a, w, &rid);
            if (v != AGILE_ALLOW) note_key(i);
            verdict[i] = (uint8_t)v;
        }
    }
    // Violations are keyed by index, one key per access: the block reduces them by key
    // alone, and its smallest violation's record -- verdict, width, address, range id --
    // comes from the full rule, only once the log shows it lower.
    if (first1 < ll.key) ll.key = first1;
    ll.info = 0;
    ll.addr = 0;
    ll.cnt += cnt1;
    agile::block_log_flush(log, ll, [&](unsigned long long k, unsigned long long &info,
                                        unsigned long long &a) {
        a = addr[k];
        const uint32_t w = width[k];
        uint32_t rid;
        const uint32_t v = full_rule<C32>(V, a, w, &rid);
        info = agile::pack_info(0, v, w, rid);
    });
}

// Inputs not aligned for vector loads, or a log with a bounded list: one access per
// thread per step, full rule, every denial noted (and appended to the list).
template <int MODE, bool C32>
__global__ void __launch_bounds__(kThreads, 1)
k_check_batch_scalar(const agile_dev_table_t T, const uint64_t *__restrict__ addr,
                     const uint8_t *__restrict__ width, uint8_t *__restrict__ verdict, size_t n,
                     LogDev *log) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned long long s_bar;
    const TView V = agile::stage_table<MODE>(T, smem, &s_bar, log);
    LaneLog ll;
    ll.log = log;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const uint64_t a = addr[i];
        const uint32_t w = width[i];
        uint32_t rid;
        const uint32_t v = full_rule<C32>(V, a, w, &rid);
        if (v != AGILE_ALLOW) ll.note(i, agile::pack_info(0, v, w, rid), a);
        verdict[i] = (uint8_t)v;
    }
    agile::block_log_flush(log, ll);
}

template <typename K>
int launch_kernel(K kernel, const agile_dev_table_t &T, const uint64_t *a, const uint8_t *w,
                  size_t n, uint8_t *v, LogDev *log, cudaStream_t st, uint32_t smem, unsigned blocks) {
    if (smem > 48 * 1024)
        AGILE_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kernel<<<blocks, kThreads, smem, st>>>(T, a, w, v, n, log);
    AGILE_CUDA_TRY(cudaGetLastError());
    return AGILE_OK;
}

template <int MODE, bool C32>
int launch(const agile_dev_table_t &T, const uint64_t *a, const uint8_t *w, size_t n,
           uint8_t *v, LogDev *log, cudaStream_t st, bool vec) {
    const size_t units = vec ? n / 8 : n;
    const size_t want = (units + kThreads - 1) / kThreads;
    const size_t cap = (size_t)agile::sm_count();
    const unsigned blocks = (unsigned)(want < 1 ? 1 : want > cap ? cap : want);
    if (!vec) {                                        // the class map serves pass 1 only
        constexpr int kM = MODE & ~(agile::ST_CMAP | agile::ST_CDESC);
        return launch_kernel(k_check_batch_scalar<kM, C32>, T, a, w, n, v, log, st,
                             (uint32_t)agile::stage_bytes(T, kM), blocks);
    }
    const uint32_t smem = (uint32_t)agile::stage_bytes(T, MODE) + (MODE & agile::ST_CDESC ? kQueueBytes + kListBytes : 0);
    // Four (else two) groups per lane per round when the batch gives every lane that many:
    // pass 2 then deals out more open accesses per round and its rounds run fuller. The
    // descriptor form is launched only for such batches.
    if constexpr ((MODE & agile::ST_CDESC) != 0) {
        return launch_kernel(k_check_batch<MODE, C32, 4>, T, a, w, n, v, log, st, smem, blocks);
    } else {
        if (units >= 4 * (size_t)blocks * kThreads)
            return launch_kernel(k_check_batch<MODE, C32, 4>, T, a, w, n, v, log, st, smem, blocks);
        if (units >= 2 * (size_t)blocks * kThreads)
            return launch_kernel(k_check_batch<MODE, C32, 2>, T, a, w, n, v, log, st, smem, blocks);
        return launch_kernel(k_check_batch<MODE, C32, 1>, T, a, w, n, v, log, st, smem, blocks);
    }
}

// Staging: the class map always (at most 128 KiB + 4 bytes); beside it, whatever fits the
// budget of the page map and the packed records (windows under 4 GiB) or the range
// arrays, and the open-block descriptors with the pass-2 queue where they help, in this
// order of preference: everything; descriptors and records without the page map; the
// page map and records; records; ranges; pages. Sections left out are read through L1.
template <bool C32>
int launch_staged(const agile_dev_table_t &T, const uint64_t *a, const uint8_t *w, size_t n,
                  uint8_t *v, LogDev *log, cudaStream_t st, bool vec) {
    using namespace agile;
    constexpr int kMPC = ST_CMAP | ST_PAGES | ST_COMPACT, kMC = ST_CMAP | ST_COMPACT;
    constexpr int kMPCD = kMPC | ST_CDESC, kMCD = kMC | ST_CDESC;
    constexpr int kMA = ST_CMAP | STAGE_ALL, kMP = ST_CMAP | ST_PAGES;
    if (T.npages == 0) return launch<STAGE_NONE, false>(T, a, w, n, v, log, st, vec);
    // Descriptors pay off where every warp runs many rounds: a batch that gives every
    // lane four groups or more. In a shorter one the queue's last, partly filled round of
    // the full rule comes on top of the descriptor rounds.
    const bool many = vec && n / 8 >= 4ull * (uint64_t)sm_count() * kThreads && n < (1ull << 56);
    if (C32 && many && T.cdesc != nullptr && stage_bytes(T, kMPCD) + kQueueBytes + kListBytes <= kStageBudget)
        return launch<kMPCD, C32>(T, a, w, n, v, log, st, vec);
    // the descriptors before the page map: they decide most open accesses without it
    if (C32 && many && T.cdesc != nullptr && stage_bytes(T, kMCD) + kQueueBytes + kListBytes <= kStageBudget)
        return launch<kMCD, C32>(T, a, w, n, v, log, st, vec);
    if (C32 && stage_bytes(T, kMPC) <= kStageBudget) return launch<kMPC, C32>(T, a, w, n, v, log, st, vec);
    if (C32 && stage_bytes(T, kMC) <= kStageBudget) return launch<kMC, C32>(T, a, w, n, v, log, st, vec);
    if (stage_bytes(T, kMA) <= kStageBudget) return launch<kMA, C32>(T, a, w, n, v, log, st, vec);
    if (stage_bytes(T, kMP) <= kStageBudget) return launch<kMP, C32>(T, a, w, n, v, log, st, vec);
    return launch<ST_CMAP, C32>(T, a, w, n, v, log, st, vec);
}

}  // namespace

extern "C" int agile_guard_check_batch(const agile_dev_table_t *tbl, const uint64_t *d_addr,
                                       const uint8_t *d_width, size_t n, uint8_t *d_verdict,
                                       void *d_log, void *stream) {
    if (tbl == nullptr) return AGILE_ERR_INVALID_ARG;
    if (n == 0) return AGILE_OK;
    if (d_addr == nullptr || d_width == nullptr || d_verdict == nullptr) return AGILE_ERR_INVALID_ARG;
    if (d_log != nullptr && ((uintptr_t)d_log & 15) != 0) return AGILE_ERR_ALIGN;
    if (tbl->cmap == nullptr) return AGILE_ERR_INVALID_ARG;
    // the per-access form also when the log has a list, which it appends every denial to
    const bool vec = ((uintptr_t)d_addr & 15) == 0 && ((uintptr_t)d_width & 7) == 0 &&
                     ((uintptr_t)d_verdict & 7) == 0 && !agile::log_has_list(d_log);
    LogDev *log = (LogDev *)d_log;
    cudaStream_t st = (cudaStream_t)stream;
    return tbl->crange != nullptr ? launch_staged<true>(*tbl, d_addr, d_width, n, d_verdict, log, st, vec)
                                  : launch_staged<false>(*tbl, d_addr, d_width, n, d_verdict, log, st, vec);
}
