// Batched guard check: one verdict per (address, width) pair, the Sec. IV-E rule applied
// as the kernel guard of Sec. V-E applies it, with the first violation (smallest index)
// and the violation count in the log.
//
// Launch shape: one 1024-thread block per SM, a warp-uniform grid-stride loop. Each lane
// takes 8 consecutive accesses per round: four 16-byte address loads, one 8-byte width
// load, one 8-byte verdict store. Staged into shared memory by bulk copies: the page map,
// the packed range records (windows under 4 GiB; otherwise the range arrays) and the
// all-user block bitmap. Pass 1 decides the accesses inside all-user blocks from the
// bitmap, without branches; pass 2 deals the warp's remaining accesses out over its lanes
// and decides each by the full rule (the 32-bit uniform decision over the packed records
// where it applies). Each thread keeps its smallest violation in registers; the block
// reduces them once at the end.
#include <cuda_runtime.h>

#include "agile_internal.h"
#include "guard_device.cuh"

namespace {

using agile::LaneLog;
using agile::LogDev;
using agile::TView;

constexpr int kThreads = 1024;   // one block per SM: 250 G checks/s at 2^28 against 231
                                 // for 2 x 512 and 218 for 4 x 256 (same code otherwise)

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

// The bitmap test of pass 1 for windows under 4 GiB (the packed-record tables): one 64-bit
// window check, then 32-bit arithmetic (blocks there are at most 2^14 bytes).
__device__ __forceinline__ bool user_fast32(const TView &V, uint64_t a, uint32_t w) {
    const uint64_t off = a - V.lo;
    const uint32_t o = (uint32_t)off;
    const uint32_t k = off <= V.last - V.lo ? o >> V.ulg : V.un;   // outside: the clear bit
    const uint32_t m = (1u << V.ulg) - 1u;
    return ((V.ubits[k >> 5] >> (k & 31)) & 1u) && (o & m) + w <= m + 1u;
}

__device__ __forceinline__ bool legal_width(uint32_t w) {
    return w <= 16 && ((0x10116u >> w) & 1u);        // 1, 2, 4, 8, 16
}

// Full rule for one access (for the accesses the uniform decision leaves open).
template <bool C32>
__device__ __forceinline__ uint32_t full_one(const TView &V, uint64_t a, uint32_t w, size_t i,
                                             LaneLog &ll) {
    uint32_t rid = agile::kNoRange, v;
    if (!legal_width(w)) v = AGILE_DENY_INVALID;
    else if constexpr (C32) v = agile::classify_slow(V, a, w, &rid);
    else v = agile::classify(V, a, w, &rid);
    if (v != AGILE_ALLOW) ll.note(i, agile::pack_info(0, v, w, rid), a);
    return v;
}

template <int MODE, int VEC, int kG>
__global__ void __launch_bounds__(kThreads, 1)
k_check_batch(const agile_dev_table_t T, const uint64_t *__restrict__ addr,
              const uint8_t *__restrict__ width, uint8_t *__restrict__ verdict, size_t n,
              LogDev *log) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned long long s_bar;
    const TView V = agile::stage_table<MODE>(T, smem, &s_bar, log);

    const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t nthreads = (size_t)gridDim.x * blockDim.x;
    const size_t ngroups = n / VEC;

    constexpr bool kC32 = (MODE & agile::ST_COMPACT) != 0;
    LaneLog ll;
    if constexpr (VEC == 8) {
        // Each lane takes kG groups of 8 accesses per round (groups g0 + 32h + lane,
        // coalesced across the warp). With kG = 2 pass 2 has twice the open accesses to
        // deal out and its 32-lane rounds run fuller (268 -> 285 G checks/s at 2^28);
        // batches too small to give every lane two groups use kG = 1.
        const uint32_t lane = threadIdx.x & 31;
        for (size_t g0 = (tid - lane) * kG; g0 < ngroups; g0 += nthreads * kG) {   // warp-uniform
            // Pass 1, branch-free: an access inside an all-user block of the bitmap is
            // allowed. The others ("open") are decided in pass 2.
            uint32_t open = 0;
#pragma unroll
            for (int h = 0; h < kG; ++h) {
                const size_t g = g0 + 32 * h + lane;
                if (g >= ngroups) continue;
                // Default-cached loads: pass 2 re-reads its accesses, which then hit L1 (with
                // streaming loads they came from DRAM again, 40% more read traffic).
                const uint4 *pa = reinterpret_cast<const uint4 *>(addr + g * 8);
                uint64_t av[8];
#pragma unroll
                for (int k = 0; k < 4; ++k) {          // registers only: no indexed arrays
                    const uint4 q = __ldg(pa + k);
                    av[2 * k] = (uint64_t)q.y << 32 | q.x;
                    av[2 * k + 1] = (uint64_t)q.w << 32 | q.z;
                }
                const uint64_t wv = __ldg(reinterpret_cast<const unsigned long long *>(width + g * 8));
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const uint32_t w = (uint32_t)(wv >> (8 * k)) & 0xFFu;
                    bool inb;
                    if constexpr (kC32) inb = user_fast32(V, av[k], w);
                    else inb = agile::block_user_fast(V, av[k], w, agile::user_bits(V, av[k]));
                    const bool ok = legal_width(w) && av[k] <= ~0ull - w && inb;
                    open |= (uint32_t)!ok << (8 * h + k);
                }
                __stcs(reinterpret_cast<unsigned long long *>(verdict + g * 8), 0ull);
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
            __syncwarp();                              // the zero stores above come first
            for (uint32_t q0 = 0; q0 < total; q0 += 32) {
                const uint32_t q = q0 + lane;
                uint32_t own = 0;                      // lanes whose open accesses all precede q
#pragma unroll
                for (int step = 16; step; step >>= 1) {
                    const uint32_t t = __shfl_sync(agile::kFull, incl, own + step - 1);
                    own = t <= q ? own + step : own;
                }
                const uint32_t omask = __shfl_sync(agile::kFull, open, own & 31);
                const uint32_t oexcl = __shfl_sync(agile::kFull, excl, own & 31);
                if (q < total) {
                    uint32_t m = omask;
                    for (uint32_t r = q - oexcl; r; --r) m &= m - 1;   // drop the earlier ones
                    const int b = __ffs(m) - 1;                       // bit 8h + k
                    const size_t i = (g0 + 32 * (b >> 3) + own) * 8 + (b & 7);
                    const uint64_t a = addr[i];
                    const uint32_t w = width[i];
                    uint32_t v = 0, rid = agile::kNoRange;
                    bool done = false;
                    if constexpr (kC32) done = legal_width(w) && a <= ~0ull - w && decide32(V, a, w, &v, &rid);
                    if (!done) v = full_one<kC32>(V, a, w, i, ll);
                    else if (v != AGILE_ALLOW) ll.note(i, agile::pack_info(0, v, w, rid), a);
                    if (v != AGILE_ALLOW) verdict[i] = (uint8_t)v;
                }
            }
        }
    } else {
        for (size_t g = tid; g < ngroups; g += nthreads)
            verdict[g] = (uint8_t)full_one<kC32>(V, addr[g], width[g], g, ll);
    }
    if (VEC > 1 && blockIdx.x == 0 && threadIdx.x < 32) {    // the last n % VEC accesses
        const size_t i = ngroups * VEC + threadIdx.x;
        if (i < n) verdict[i] = (uint8_t)full_one<kC32>(V, addr[i], width[i], i, ll);
    }
    agile::block_log_flush(log, ll);
}

template <int MODE, int VEC, int kG>
int launch_g(const agile_dev_table_t &T, const uint64_t *a, const uint8_t *w, size_t n,
             uint8_t *v, LogDev *log, cudaStream_t st, uint32_t smem, unsigned blocks) {
    if (smem > 48 * 1024) {
        AGILE_CUDA_TRY(cudaFuncSetAttribute(k_check_batch<MODE, VEC, kG>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    }
    k_check_batch<MODE, VEC, kG><<<blocks, kThreads, smem, st>>>(T, a, w, v, n, log);
    AGILE_CUDA_TRY(cudaGetLastError());
    return AGILE_OK;
}

template <int MODE, int VEC>
int launch(const agile_dev_table_t &T, const uint64_t *a, const uint8_t *w, size_t n,
           uint8_t *v, LogDev *log, cudaStream_t st) {
    const uint32_t smem = agile::stage_bytes(T, MODE);
    size_t groups = n / VEC;
    size_t want = (groups + kThreads - 1) / kThreads;
    size_t cap = (size_t)agile::sm_count();
    unsigned blocks = (unsigned)(want < 1 ? 1 : want > cap ? cap : want);
    if (VEC == 8 && groups >= 2 * (size_t)blocks * kThreads)
        return launch_g<MODE, VEC, 2>(T, a, w, n, v, log, st, smem, blocks);
    return launch_g<MODE, VEC, 1>(T, a, w, n, v, log, st, smem, blocks);
}

template <int VEC>
int launch_mode(const agile_dev_table_t &T, const uint64_t *a, const uint8_t *w, size_t n,
                uint8_t *v, LogDev *log, cudaStream_t st) {
    constexpr int kCB = agile::STAGE_COMPACT | agile::ST_BITS, kAB = agile::STAGE_ALL | agile::ST_BITS;
    constexpr int kPB = agile::STAGE_PAGES | agile::ST_BITS;
    // The bitmap is staged at every size: without it, pass 1 reads it through L1 and the
    // 2^20-access check takes 18.4 us instead of 16.4.
    switch (agile::stage_mode(T, true, true, true)) {
        case kCB: return launch<kCB, VEC>(T, a, w, n, v, log, st);
        case agile::STAGE_COMPACT: return launch<agile::STAGE_COMPACT, VEC>(T, a, w, n, v, log, st);
        case kAB: return launch<kAB, VEC>(T, a, w, n, v, log, st);
        case agile::STAGE_ALL: return launch<agile::STAGE_ALL, VEC>(T, a, w, n, v, log, st);
        case kPB: return launch<kPB, VEC>(T, a, w, n, v, log, st);
        case agile::STAGE_PAGES: return launch<agile::STAGE_PAGES, VEC>(T, a, w, n, v, log, st);
        case agile::STAGE_BITS: return launch<agile::STAGE_BITS, VEC>(T, a, w, n, v, log, st);
        default: return launch<agile::STAGE_NONE, VEC>(T, a, w, n, v, log, st);
    }
}

}  // namespace

extern "C" int agile_guard_check_batch(const agile_dev_table_t *tbl, const uint64_t *d_addr,
                                       const uint8_t *d_width, size_t n, uint8_t *d_verdict,
                                       void *d_log, void *stream) {
    if (tbl == nullptr) return AGILE_ERR_INVALID_ARG;
    if (n == 0) return AGILE_OK;
    if (d_addr == nullptr || d_width == nullptr || d_verdict == nullptr) return AGILE_ERR_INVALID_ARG;
    if (d_log != nullptr && ((uintptr_t)d_log & 15) != 0) return AGILE_ERR_ALIGN;
    const bool vec = ((uintptr_t)d_addr & 15) == 0 && ((uintptr_t)d_width & 7) == 0 &&
                     ((uintptr_t)d_verdict & 7) == 0;
    LogDev *log = (LogDev *)d_log;
    cudaStream_t st = (cudaStream_t)stream;
    return vec ? launch_mode<8>(*tbl, d_addr, d_width, n, d_verdict, log, st)
               : launch_mode<1>(*tbl, d_addr, d_width, n, d_verdict, log, st);
}
