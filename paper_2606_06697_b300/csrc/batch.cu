// Batched guarded launch: many clients' kernels run in one persistent launch, each guarded
// against its own table and logging into its own log (Sec. IV-B: the worker executes the
// CUDA operations of the clients assigned to it in its context; Sec. V-E: the kernel guard
// per client). The launch can be captured once into a CUDA graph and replayed with
// different work lists, and an autotuner picks the tile size, the span-check policy and
// the table page size.
//
// Device buffer (caller-owned, agile_batch_device_bytes):
//   [0, 64)        header: item count, tile count, tile claim counter, tile size, and for a
//                  launch that reports each item's completion, the addresses of the
//                  per-item done counters and of the per-item notice flags
//   [64, ...)      n work items, 64 bytes each
//   then           n + 1 u64 tile prefix sums (tiles of item i are prefix[i] .. prefix[i+1])
// Blocks claim tiles with one atomic on the counter; the launch resets it first.
#include <cuda_runtime.h>

#include <chrono>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <new>
#include <sstream>
#include <string>
#include <vector>

#include "agile_internal.h"
#include "irregular_body.cuh"
#include "stream_body.cuh"

struct agile_graph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

using agile::LaneLog;
using agile::LogDev;
using agile::TView;
using agile::WarpSlots;

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;

struct BatchHdr {
    unsigned long long n_items;
    unsigned long long total_tiles;
    unsigned long long counter;
    uint32_t tile;
    uint32_t pad;
    unsigned int *done;            // per-item count of finished tiles (zeroed), or NULL
    unsigned int *notice;          // per-item flag set to 1 when the item's last tile is done,
                                   // in host-mapped memory, or NULL for no notices
    unsigned long long reserved[2];
};
static_assert(sizeof(BatchHdr) == 64, "header");
static_assert(sizeof(agile_work_t) == 64, "work item");

size_t prefix_offset(size_t n) { return 64 + 64 * n; }

// Elements [e0, e1) of a streaming item, e0 a multiple of 512 (one warp tile = 512 elements).
template <int OP, bool GUARD, int POLICY>
__device__ void stream_tile(const TView &V, const agile_dev_table_t &T, const agile_work_t &W,
                            size_t e0, size_t e1, WarpSlots &S, bool spans) {
    float *a = static_cast<float *>(W.out);
    const float *b = static_cast<const float *>(W.in0);
    const float *c = W.op == AGILE_WORK_TRIAD ? static_cast<const float *>(W.in1) : b;
    const size_t n = W.n, n4 = n >> 2;
    const size_t t0 = e0 / (4 * agile::kStreamTileUnits);
    const size_t u1 = (e1 >= n ? n4 : e1 >> 2);
    const size_t t1 = (u1 + agile::kStreamTileUnits - 1) / agile::kStreamTileUnits;
    for (size_t t = t0 + (threadIdx.x >> 5); t < t1; t += kWarps)
        agile::stream_warp_tile<OP, GUARD, POLICY>(V, T, a, b, c, t, n4, n, W.s, S, spans);
    if (e1 >= n && (n & 3) && (threadIdx.x >> 5) == kWarps - 1)
        agile::stream_tail<OP, GUARD, POLICY>(V, T, a, b, c, n, W.s, S);
}

template <int KIND, bool GUARD, int POLICY>
__device__ void irregular_tile(const TView &V, const agile_dev_table_t &T, const agile_work_t &W,
                               size_t e0, size_t e1, WarpSlots &S, bool spans) {
    const int64_t *idx = static_cast<const int64_t *>(W.in0);
    float *base = static_cast<float *>(const_cast<void *>(W.in1));
    float *out = static_cast<float *>(W.out);
    const size_t n = W.n, n4 = n >> 2;
    const size_t u1 = e1 >= n ? n4 : e1 >> 2;
    LaneLog ll;
    ll.log = S.log;
    for (size_t u0 = (e0 >> 2) + 32 * (threadIdx.x >> 5); u0 < u1; u0 += 32 * kWarps)
        agile::irregular_group<KIND, GUARD, POLICY>(V, T, idx, base, out, u0, u1, ll, spans);
    if (e1 >= n && (n & 3) && (threadIdx.x >> 5) == kWarps - 1)
        agile::irregular_tail<KIND, GUARD, POLICY>(V, T, idx, base, out, n, ll);
    if constexpr (GUARD) agile::warp_note(S, ll);
}

template <bool GUARD, int POLICY>
__device__ void run_tile(const TView &V, const agile_dev_table_t &T, const agile_work_t &W,
                         size_t e0, size_t e1, WarpSlots &S, bool spans) {
    switch (W.op) {
        case AGILE_WORK_COPY: stream_tile<AGILE_OP_COPY, GUARD, POLICY>(V, T, W, e0, e1, S, spans); break;
        case AGILE_WORK_SCALE: stream_tile<AGILE_OP_SCALE, GUARD, POLICY>(V, T, W, e0, e1, S, spans); break;
        case AGILE_WORK_TRIAD: stream_tile<AGILE_OP_TRIAD, GUARD, POLICY>(V, T, W, e0, e1, S, spans); break;
        case AGILE_WORK_GATHER: irregular_tile<AGILE_IRR_GATHER, GUARD, POLICY>(V, T, W, e0, e1, S, spans); break;
        case AGILE_WORK_SCATTER: irregular_tile<AGILE_IRR_SCATTER, GUARD, POLICY>(V, T, W, e0, e1, S, spans); break;
        default: irregular_tile<AGILE_IRR_HIST, GUARD, POLICY>(V, T, W, e0, e1, S, spans); break;
    }
}

__global__ void __launch_bounds__(kThreads, 2)
k_batch(BatchHdr *H, const agile_work_t *__restrict__ items, const uint64_t *__restrict__ prefix,
        int spans) {
    __shared__ unsigned long long s_tile;
    __shared__ uint32_t s_item;
    __shared__ agile_work_t s_work;
    __shared__ agile_dev_table_t s_T;
    __shared__ WarpSlots S;
    agile::slots_init(S);
    const unsigned long long total = H->total_tiles;
    const uint32_t tile = H->tile;
    for (;;) {
        if (threadIdx.x == 0) {
            const unsigned long long t = atomicAdd(&H->counter, 1ull);
            s_tile = t;
            if (t < total) {
                uint32_t lo = 0, hi = (uint32_t)H->n_items;   // last item with prefix <= t
                while (hi - lo > 1) {
                    const uint32_t mid = (lo + hi) >> 1;
                    if (prefix[mid] <= t) lo = mid; else hi = mid;
                }
                s_item = lo;
                s_work = items[lo];
                S.log = static_cast<LogDev *>(s_work.log);
                if (s_work.table != nullptr) s_T = *static_cast<const agile_dev_table_t *>(s_work.table);
            }
        }
        __syncthreads();
        const unsigned long long t = s_tile;
        if (t >= total) break;
        const agile_work_t &W = s_work;
        const size_t e0 = (size_t)(t - prefix[s_item]) * tile;
        const size_t e1 = e0 + tile < W.n ? e0 + tile : W.n;
        if (W.table == nullptr) {
            agile_dev_table_t none = {};
            run_tile<false, AGILE_POLICY_REPORT>(TView{}, none, W, e0, e1, S, true);
        } else {
            const TView V = agile::view_of(s_T);
            switch (W.policy) {
                case AGILE_POLICY_POISON: run_tile<true, AGILE_POLICY_POISON>(V, s_T, W, e0, e1, S, spans); break;
                case AGILE_POLICY_SINK: run_tile<true, AGILE_POLICY_SINK>(V, s_T, W, e0, e1, S, spans); break;
                default: run_tile<true, AGILE_POLICY_REPORT>(V, s_T, W, e0, e1, S, spans); break;
            }
        }
        agile::slots_flush(static_cast<LogDev *>(W.log), S);   // one update per tile
        agile::slots_init(S);
        __syncthreads();
        // Completion notice: the block that finishes an item's last tile tells the host,
        // so a caller can complete that item without waiting for the whole launch. The
        // barrier above orders the tile's writes and log updates before this thread's
        // fence; the count then orders every tile before the notice.
        if (threadIdx.x == 0 && H->notice != nullptr) {
            __threadfence();
            const unsigned int tiles = (unsigned int)(prefix[s_item + 1] - prefix[s_item]);
            if (atomicAdd(&H->done[s_item], 1u) + 1u == tiles) {
                __threadfence_system();
                *(volatile unsigned int *)(H->notice + s_item) = 1u;
            }
        }
    }
}

bool op_ok(uint32_t op) { return op <= AGILE_WORK_HIST; }

int check_item(const agile_work_t &w) {
    if (!op_ok(w.op) || w.policy > AGILE_POLICY_REPORT || w.n == 0) return AGILE_ERR_INVALID_ARG;
    if (w.out == nullptr && (w.op <= AGILE_WORK_TRIAD || w.op == AGILE_WORK_GATHER)) return AGILE_ERR_INVALID_ARG;
    if (w.in0 == nullptr || (w.in1 == nullptr && w.op >= AGILE_WORK_TRIAD)) return AGILE_ERR_INVALID_ARG;
    const uintptr_t a16 = (uintptr_t)w.in0 | (w.op <= AGILE_WORK_TRIAD || w.op == AGILE_WORK_GATHER ? (uintptr_t)w.out : 0) |
                          (w.op == AGILE_WORK_TRIAD ? (uintptr_t)w.in1 : 0);
    if (a16 & 15) return AGILE_ERR_ALIGN;
    if (w.op >= AGILE_WORK_GATHER && ((uintptr_t)w.in1 & 3)) return AGILE_ERR_ALIGN;
    if (w.log != nullptr && ((uintptr_t)w.log & 15)) return AGILE_ERR_ALIGN;
    if (w.table != nullptr && ((uintptr_t)w.table & 255)) return AGILE_ERR_ALIGN;
    return AGILE_OK;
}

int launch_batch(void *d_buf, const agile_batch_config_t *cfg, cudaStream_t st, bool reset = true) {
    BatchHdr *H = static_cast<BatchHdr *>(d_buf);
    unsigned char *base = static_cast<unsigned char *>(d_buf);
    // the item count lives on the device; the prefix follows the largest work list the
    // buffer was sized for, which the kernel finds through the header
    if (reset) AGILE_CUDA_TRY(cudaMemsetAsync(&H->counter, 0, sizeof(unsigned long long), st));
    const int bps = cfg->blocks_per_sm == 1 ? 1 : 2;
    k_batch<<<agile::sm_count() * bps, kThreads, 0, st>>>(
        H, reinterpret_cast<const agile_work_t *>(base + 64),
        reinterpret_cast<const uint64_t *>(base + 64 + 64 * (size_t)cfg->reserved), cfg->span_checks ? 1 : 0);
    AGILE_CUDA_TRY(cudaGetLastError());
    return AGILE_OK;
}

uint64_t fnv1a(const void *p, size_t n, uint64_t h = 1469598103934665603ull) {
    const unsigned char *c = static_cast<const unsigned char *>(p);
    for (size_t i = 0; i < n; ++i) h = (h ^ c[i]) * 1099511628211ull;
    return h;
}

}  // namespace

namespace agile {
int batch_check_item(const agile_work_t &w) { return check_item(w); }

// A launch over a work list whose image -- claim counter zeroed -- was just copied to the
// device on the same stream: no separate reset of the counter.
int batch_launch_fresh(void *d_buf, size_t n_items, const agile_batch_config_t *cfg, void *stream) {
    agile_batch_config_t c = *cfg;
    c.reserved = (uint32_t)n_items;
    return launch_batch(d_buf, &c, (cudaStream_t)stream, false);
}
}  // namespace agile

extern "C" {

size_t agile_batch_device_bytes(size_t max_items) { return agile::batch_device_bytes(max_items); }

int agile_batch_upload(const agile_work_t *h_items, size_t n, uint32_t tile, void *d_buf,
                       size_t bytes, void *stream) {
    if (h_items == nullptr || n == 0 || d_buf == nullptr) return AGILE_ERR_INVALID_ARG;
    if (tile < 512 || (tile & 511) != 0) return AGILE_ERR_INVALID_ARG;
    if (((uintptr_t)d_buf & 255) != 0) return AGILE_ERR_ALIGN;
    if (bytes < agile_batch_device_bytes(n)) return AGILE_ERR_TOO_LARGE;
    for (size_t i = 0; i < n; ++i) {
        const int rc = check_item(h_items[i]);
        if (rc != AGILE_OK) return rc;
    }
    // The prefix sits right after the items of *this* upload; the launch reads its offset
    // from the config (reserved = item count), set by agile_batch_config_for.
    std::vector<unsigned char> img(prefix_offset(n) + 8 * (n + 1));
    BatchHdr h{};
    uint64_t *pre = reinterpret_cast<uint64_t *>(img.data() + prefix_offset(n));
    pre[0] = 0;
    for (size_t i = 0; i < n; ++i) pre[i + 1] = pre[i] + (h_items[i].n + tile - 1) / tile;
    h.n_items = n;
    h.total_tiles = pre[n];
    h.tile = tile;
    std::memcpy(img.data(), &h, sizeof h);
    std::memcpy(img.data() + 64, h_items, 64 * n);
    AGILE_CUDA_TRY(cudaMemcpyAsync(d_buf, img.data(), img.size(), cudaMemcpyHostToDevice,
                                   (cudaStream_t)stream));
    AGILE_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    return AGILE_OK;
}

int agile_batch_launch(void *d_buf, size_t n_items, const agile_batch_config_t *cfg, void *stream) {
    if (d_buf == nullptr || cfg == nullptr || n_items == 0) return AGILE_ERR_INVALID_ARG;
    agile_batch_config_t c = *cfg;
    c.reserved = (uint32_t)n_items;
    return launch_batch(d_buf, &c, (cudaStream_t)stream);
}

int agile_batch_graph_create(void *d_buf, size_t n_items, const agile_batch_config_t *cfg,
                             agile_graph_t **out) {
    if (d_buf == nullptr || cfg == nullptr || out == nullptr || n_items == 0) return AGILE_ERR_INVALID_ARG;
    *out = nullptr;
    agile_graph *g = new (std::nothrow) agile_graph;
    if (g == nullptr) return AGILE_ERR_NOMEM;
    cudaStream_t cs;
    AGILE_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    agile_batch_config_t c = *cfg;
    c.reserved = (uint32_t)n_items;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    int rc = e == cudaSuccess ? launch_batch(d_buf, &c, cs) : AGILE_ERR_CUDA;
    cudaError_t e2 = cudaStreamEndCapture(cs, &g->graph);
    if (rc == AGILE_OK && e2 == cudaSuccess)
        e2 = cudaGraphInstantiate(&g->exec, g->graph, 0);
    cudaStreamDestroy(cs);
    if (rc != AGILE_OK || e2 != cudaSuccess) {
        if (e2 != cudaSuccess) agile::set_cuda_error((int)e2, "graph capture");
        if (g->exec) cudaGraphExecDestroy(g->exec);
        if (g->graph) cudaGraphDestroy(g->graph);
        delete g;
        return rc != AGILE_OK ? rc : AGILE_ERR_CUDA;
    }
    *out = g;
    return AGILE_OK;
}

int agile_graph_launch(agile_graph_t *g, void *stream) {
    if (g == nullptr) return AGILE_ERR_INVALID_ARG;
    AGILE_CUDA_TRY(cudaGraphLaunch(g->exec, (cudaStream_t)stream));
    return AGILE_OK;
}

void agile_graph_destroy(agile_graph_t *g) {
    if (g == nullptr) return;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
}

int agile_batch_autotune(const agile_work_t *h_variants, size_t n_variants, size_t n_items,
                         const uint32_t *tiles, size_t n_tiles, void *d_buf, size_t bytes,
                         int reps, const char *cache_path, void *stream,
                         agile_batch_tuning_t *best) {
    if (h_variants == nullptr || n_variants == 0 || n_items == 0 || tiles == nullptr ||
        n_tiles == 0 || best == nullptr || reps <= 0)
        return AGILE_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    // signature: every item's op, policy and size, per variant, plus the candidate tiles
    uint64_t sig = fnv1a(&n_variants, sizeof n_variants);
    for (size_t v = 0; v < n_variants; ++v)
        for (size_t i = 0; i < n_items; ++i) {
            const agile_work_t &w = h_variants[v * n_items + i];
            sig = fnv1a(&w.op, 8, sig);
            sig = fnv1a(&w.n, 8, sig);
        }
    sig = fnv1a(tiles, 4 * n_tiles, sig);
    if (cache_path != nullptr) {
        std::ifstream f(cache_path);
        std::string line;
        while (std::getline(f, line)) {
            std::istringstream ss(line);
            unsigned long long s;
            agile_batch_tuning_t t{};
            if (ss >> std::hex >> s >> std::dec >> t.config.tile >> t.config.span_checks >>
                    t.config.blocks_per_sm >> t.variant >> t.ms && s == sig) {
                t.cached = 1;
                *best = t;
                return AGILE_OK;
            }
        }
    }
    cudaEvent_t e0, e1;
    AGILE_CUDA_TRY(cudaEventCreate(&e0));
    AGILE_CUDA_TRY(cudaEventCreate(&e1));
    agile_batch_tuning_t top{};
    top.ms = 1e30f;
    int rc = AGILE_OK;
    for (size_t v = 0; v < n_variants && rc == AGILE_OK; ++v)
        for (size_t ti = 0; ti < n_tiles && rc == AGILE_OK; ++ti) {
            rc = agile_batch_upload(h_variants + v * n_items, n_items, tiles[ti], d_buf, bytes, stream);
            for (uint32_t spans = 0; spans < 2 && rc == AGILE_OK; ++spans)
                for (uint32_t bps = 1; bps <= 2 && rc == AGILE_OK; ++bps) {
                    agile_batch_config_t c{tiles[ti], spans, bps, 0};
                    rc = agile_batch_launch(d_buf, n_items, &c, stream);      // warm-up
                    if (rc != AGILE_OK) break;
                    cudaEventRecord(e0, st);
                    for (int r = 0; r < reps && rc == AGILE_OK; ++r)
                        rc = agile_batch_launch(d_buf, n_items, &c, stream);
                    cudaEventRecord(e1, st);
                    if (cudaEventSynchronize(e1) != cudaSuccess) { rc = AGILE_ERR_CUDA; break; }
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    ms /= (float)reps;
                    if (ms < top.ms) { top.config = c; top.variant = (uint32_t)v; top.ms = ms; }
                }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != AGILE_OK) return rc;
    top.cached = 0;
    *best = top;
    if (cache_path != nullptr) {
        std::ofstream f(cache_path, std::ios::app);
        char buf[160];
        std::snprintf(buf, sizeof buf, "%016llx %u %u %u %u %.6f\n", (unsigned long long)sig,
                      top.config.tile, top.config.span_checks, top.config.blocks_per_sm,
                      top.variant, top.ms);
        f << buf;
    }
    return AGILE_OK;
}

}  // extern "C"
