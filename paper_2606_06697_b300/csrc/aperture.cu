// Aperture-only batched check (Table I; Sec. V-E): each access is compared with at most
// four protected/MMIO apertures held in the kernel's parameter space, so the check is a
// few uniform-operand compares and the kernel streams at HBM speed (10 bytes per check).
//
// Launch shape as the table check: one 1024-thread block per SM, grid-stride; each lane
// takes 8 consecutive accesses (four 16-byte address loads, one 8-byte width load, one
// 8-byte verdict store).
#include <cuda_runtime.h>

#include <algorithm>

#include "agile_internal.h"
#include "guard_device.cuh"

namespace {

using agile::LaneLog;
using agile::LogDev;

constexpr int kThreads = 1024;   // one block per SM: 596 G checks/s at 2^28, against 574
                                 // for 2 x 512 and 562 for 4 x 256

// Apertures in decision order: MMIO before protected, then by base. The first aperture
// an access overlaps decides its verdict.
struct Apertures {
    uint64_t lo[AGILE_MAX_APERTURES], end[AGILE_MAX_APERTURES];
    uint32_t verdict[AGILE_MAX_APERTURES], id[AGILE_MAX_APERTURES];
    uint32_t n;
};

__device__ __forceinline__ bool legal_width(uint32_t w) {
    return w <= 16 && ((0x10116u >> w) & 1u);        // 1, 2, 4, 8, 16
}

// x >> s with the PTX rule for shift counts of 32 and more (the result is 0).
__device__ __forceinline__ uint32_t shr_clamped(uint32_t x, uint32_t s) {
    uint32_t r;
    asm("shr.b32 %0, %1, %2;" : "=r"(r) : "r"(x), "r"(s));
    return r;
}

// The verdict alone, for the vector path: a legal width (the clamped shift is 0 for
// widths of 32 and more) and an end that does not wrap past 2^64 - 1, then the first
// aperture the access overlaps.
template <int N>
__device__ __forceinline__ uint32_t verdict_of(const Apertures &A, uint64_t a, uint32_t w) {
    const uint64_t e = a + w;
    uint32_t v = AGILE_ALLOW;
#pragma unroll
    for (int i = N - 1; i >= 0; --i) {                // the lowest i overlapped wins
        const bool hit = a < A.end[i] && e > A.lo[i];
        v = hit ? A.verdict[i] : v;
    }
    return (shr_clamped(0x10116u, w) & 1u) && e > a ? v : (uint32_t)AGILE_DENY_INVALID;
}

// Verdict of one access against the first N apertures (N fixed per launch, so the loop
// unrolls to exactly the apertures there are).
template <int N>
__device__ __forceinline__ uint32_t decide(const Apertures &A, uint64_t a, uint32_t w, uint32_t *rid) {
    if (!legal_width(w) || a > ~0ull - w) { *rid = AGILE_NO_RANGE; return AGILE_DENY_INVALID; }
    const uint64_t e = a + w;
    uint32_t v = AGILE_ALLOW, r = AGILE_NO_RANGE;
#pragma unroll
    for (int i = N - 1; i >= 0; --i) {                // the lowest i overlapped wins
        const bool hit = a < A.end[i] && e > A.lo[i];
        v = hit ? A.verdict[i] : v;
        r = hit ? A.id[i] : r;
    }
    *rid = r;
    return v;
}

// A lane visits its accesses in increasing index order, so its first denial is its
// smallest key: later denials only add to the count.
__device__ __forceinline__ void note_first(LaneLog &ll, size_t i, uint32_t v, uint32_t w, uint32_t rid,
                                           uint64_t a) {
    if (ll.cnt == 0) { ll.key = i; ll.info = agile::pack_info(0, v, w, rid); ll.addr = a; }
    ++ll.cnt;
    agile::list_append(ll.log, i, agile::pack_info(0, v, w, rid), a);
}

template <int N, int VEC>
__global__ void __launch_bounds__(kThreads, 1)
k_aperture_batch(const Apertures A, const uint64_t *__restrict__ addr,
                 const uint8_t *__restrict__ width, uint8_t *__restrict__ verdict, size_t n,
                 LogDev *log) {
    const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t nthreads = (size_t)gridDim.x * blockDim.x;
    const size_t ngroups = n / VEC;
    LaneLog ll;
    ll.log = log;
    for (size_t g = tid; g < ngroups; g += nthreads) {
        if constexpr (VEC == 8) {
            const uint4 *pa = reinterpret_cast<const uint4 *>(addr + g * 8);
            uint64_t av[8];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint4 q = __ldcs(pa + k);
                av[2 * k] = (uint64_t)q.y << 32 | q.x;
                av[2 * k + 1] = (uint64_t)q.w << 32 | q.z;
            }
            const uint64_t wv = __ldcs(reinterpret_cast<const unsigned long long *>(width + g * 8));
            // verdict k into byte k, as multiply-adds (FMA pipe; the compares fill the ALU)
            uint32_t vlo = 0, vhi = 0;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const uint32_t wk = __byte_perm(k < 4 ? (uint32_t)wv : (uint32_t)(wv >> 32), 0u,
                                                0x4440u | (uint32_t)(k & 3));
                const uint32_t v = verdict_of<N>(A, av[k], wk);
                if (k < 4) asm("mad.lo.u32 %0, %1, %2, %0;" : "+r"(vlo) : "r"(v), "r"(1u << (8 * k)));
                else asm("mad.lo.u32 %0, %1, %2, %0;" : "+r"(vhi) : "r"(v), "r"(1u << (8 * (k - 4))));
            }
            const uint64_t out = (uint64_t)vhi << 32 | vlo;
            __stcs(reinterpret_cast<unsigned long long *>(verdict + g * 8), (unsigned long long)out);
            if (out) {                                  // count the group's denials
                uint64_t m = out | (out >> 4);
                m |= m >> 2;
                m |= m >> 1;
                m &= 0x0101010101010101ull;             // bit 8k set iff verdict k is a denial
                // a lane's first denial is its smallest key; its record comes at the end
                if (ll.cnt == 0) ll.key = g * 8 + (__ffsll((long long)m) - 1) / 8;
                ll.cnt += __popcll(m);
            }
        } else {
            uint32_t rid;
            const uint32_t w = width[g];
            const uint32_t v = decide<N>(A, addr[g], w, &rid);
            if (v != AGILE_ALLOW) note_first(ll, g, v, w, rid, addr[g]);
            verdict[g] = (uint8_t)v;
        }
    }
    if (VEC > 1 && blockIdx.x == 0 && threadIdx.x < 32) {    // the last n % VEC accesses
        const size_t i = ngroups * VEC + threadIdx.x;
        if (i < n) {
            uint32_t rid;
            const uint32_t w = width[i];
            const uint32_t v = decide<N>(A, addr[i], w, &rid);
            if (v != AGILE_ALLOW) ll.note(i, agile::pack_info(0, v, w, rid), addr[i]);
            verdict[i] = (uint8_t)v;
        }
    }
    // Keys are access indices, one per access. The vector path keeps only each lane's
    // smallest key: the block's smallest violation gets its record (verdict, width,
    // address, aperture id) here, only once the log shows it lower.
    agile::block_log_flush(log, ll, [&](unsigned long long k, unsigned long long &info,
                                        unsigned long long &a) {
        a = addr[k];
        const uint32_t w = width[k];
        uint32_t rid;
        const uint32_t v = decide<N>(A, a, w, &rid);
        info = agile::pack_info(0, v, w, rid);
    });
}

template <int N, int VEC>
int launch(const Apertures &A, const uint64_t *a, const uint8_t *w, size_t n, uint8_t *v,
           LogDev *log, cudaStream_t st) {
    const size_t want = (n / VEC + kThreads - 1) / kThreads;
    const size_t cap = (size_t)agile::sm_count();
    const unsigned blocks = (unsigned)(want < 1 ? 1 : want > cap ? cap : want);
    k_aperture_batch<N, VEC><<<blocks, kThreads, 0, st>>>(A, a, w, v, n, log);
    AGILE_CUDA_TRY(cudaGetLastError());
    return AGILE_OK;
}

template <int VEC>
int launch_n(const Apertures &A, const uint64_t *a, const uint8_t *w, size_t n, uint8_t *v,
             LogDev *log, cudaStream_t st) {
    switch (A.n) {
        case 0: return launch<0, VEC>(A, a, w, n, v, log, st);
        case 1: return launch<1, VEC>(A, a, w, n, v, log, st);
        case 2: return launch<2, VEC>(A, a, w, n, v, log, st);
        case 3: return launch<3, VEC>(A, a, w, n, v, log, st);
        default: return launch<4, VEC>(A, a, w, n, v, log, st);
    }
}

}  // namespace

extern "C" int agile_aperture_check_batch(const agile_range_t *h_ap, size_t n_ap,
                                          const uint64_t *d_addr, const uint8_t *d_width, size_t n,
                                          uint8_t *d_verdict, void *d_log, void *stream) {
    if (n_ap > AGILE_MAX_APERTURES) return AGILE_ERR_TOO_LARGE;
    if (n_ap > 0 && h_ap == nullptr) return AGILE_ERR_INVALID_ARG;
    agile_range_t r[AGILE_MAX_APERTURES];
    for (size_t i = 0; i < n_ap; ++i) {
        r[i] = h_ap[i];
        if (r[i].kind != AGILE_PROTECTED && r[i].kind != AGILE_MMIO) return AGILE_ERR_BAD_KIND;
        if (r[i].size == 0) return AGILE_ERR_ZERO_SIZE;
        if (r[i].base > ~0ull - r[i].size) return AGILE_ERR_RANGE_OVERFLOW;
    }
    std::sort(r, r + n_ap, [](const agile_range_t &x, const agile_range_t &y) { return x.base < y.base; });
    for (size_t i = 1; i < n_ap; ++i)
        if (r[i].base < r[i - 1].base + r[i - 1].size) return AGILE_ERR_OVERLAP;
    std::stable_sort(r, r + n_ap, [](const agile_range_t &x, const agile_range_t &y) {
        return (x.kind == AGILE_MMIO) > (y.kind == AGILE_MMIO);   // MMIO first, bases ascending
    });
    Apertures A{};
    A.n = (uint32_t)n_ap;
    for (size_t i = 0; i < n_ap; ++i) {
        A.lo[i] = r[i].base;
        A.end[i] = r[i].base + r[i].size;
        A.verdict[i] = r[i].kind == AGILE_MMIO ? AGILE_DENY_MMIO : AGILE_DENY_PROTECTED;
        A.id[i] = r[i].id;
    }
    if (n == 0) return AGILE_OK;
    if (d_addr == nullptr || d_width == nullptr || d_verdict == nullptr) return AGILE_ERR_INVALID_ARG;
    if (d_log != nullptr && ((uintptr_t)d_log & 15) != 0) return AGILE_ERR_ALIGN;
    // the per-access form also when the log has a list, which it appends every denial to
    const bool vec = ((uintptr_t)d_addr & 15) == 0 && ((uintptr_t)d_width & 7) == 0 &&
                     ((uintptr_t)d_verdict & 7) == 0 && !agile::log_has_list(d_log);
    LogDev *log = (LogDev *)d_log;
    cudaStream_t st = (cudaStream_t)stream;
    return vec ? launch_n<8>(A, d_addr, d_width, n, d_verdict, log, st)
               : launch_n<1>(A, d_addr, d_width, n, d_verdict, log, st);
}
