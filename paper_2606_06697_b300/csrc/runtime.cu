// Violation log (Sec. V-E: poison records a violation and fails at a later
// synchronization; report counts or logs would-be violations), error strings, and the
// small runtime helpers the launches share.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <cstdlib>
#include <mutex>
#include <unordered_set>

#include "agile_internal.h"
#include "guard_device.cuh"

namespace {

thread_local char g_cuda_msg[256] = "";

std::mutex g_list_mu;
std::unordered_set<const void *> g_listed;      // logs with a list attached

void set_listed(const void *d_log, bool on) {
    std::lock_guard<std::mutex> g(g_list_mu);
    if (on) g_listed.insert(d_log); else g_listed.erase(d_log);
}

__global__ void k_log_init(agile::LogDev *L, uint32_t client) {
    if (threadIdx.x == 0) {
        L->first_key = ~0ull;
        L->first_info = ~0ull;
        L->where_key = ~0ull;
        L->where_addr = ~0ull;
        L->count = 0;
        L->client = client;
        L->status = 0;
        L->list = 0;
        L->list_next = 0;
    }
}

}  // namespace

namespace agile {

void set_cuda_error(int err, const char *where) {
    std::snprintf(g_cuda_msg, sizeof g_cuda_msg, "%s: %s", where,
                  cudaGetErrorString((cudaError_t)err));
}

bool log_has_list(const void *d_log) {
    if (d_log == nullptr) return false;
    std::lock_guard<std::mutex> g(g_list_mu);
    return g_listed.count(d_log) != 0;
}

int sm_count() {
    static std::mutex mu;
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
    std::lock_guard<std::mutex> g(mu);
    if (cache[dev] == 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0)
            v = 148;
        cache[dev] = v;
    }
    return cache[dev];
}

}  // namespace agile

extern "C" {

int agile_violation_log_init(void *d_log, uint32_t client, void *stream) {
    if (d_log == nullptr || ((uintptr_t)d_log & 15) != 0) return AGILE_ERR_ALIGN;
    k_log_init<<<1, 32, 0, (cudaStream_t)stream>>>((agile::LogDev *)d_log, client);
    AGILE_CUDA_TRY(cudaGetLastError());
    set_listed(d_log, false);
    return AGILE_OK;
}

int agile_violation_log_read(const void *d_log, agile_violation_record_t *h_out, void *stream) {
    if (d_log == nullptr || h_out == nullptr) return AGILE_ERR_INVALID_ARG;
    agile::LogDev L;
    AGILE_CUDA_TRY(cudaMemcpyAsync(&L, d_log, sizeof L, cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    AGILE_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    std::memset(h_out, 0, sizeof *h_out);
    h_out->client = L.client;
    h_out->status = L.status;
    h_out->count = L.count;
    h_out->range_id = AGILE_NO_RANGE;
    if (L.count != 0) {
        h_out->key = L.first_key;
        h_out->addr = L.where_addr;
        h_out->site = (uint32_t)(L.first_info >> 48) & 0xFFFFu;
        h_out->verdict = (uint32_t)(L.first_info >> 40) & 0xFFu;
        h_out->width = (uint32_t)(L.first_info >> 32) & 0xFFu;
        h_out->range_id = (uint32_t)L.first_info;
    }
    if (L.status & AGILE_LOG_STATUS_TIMEOUT) return AGILE_ERR_TIMEOUT;
    return L.count ? AGILE_VIOLATION : AGILE_OK;
}

int agile_violation_list_attach(void *d_log, void *d_list, uint32_t capacity, void *stream) {
    if (d_log == nullptr || d_list == nullptr || capacity == 0) return AGILE_ERR_INVALID_ARG;
    if (((uintptr_t)d_log & 15) != 0 || ((uintptr_t)d_list & 15) != 0) return AGILE_ERR_ALIGN;
    cudaStream_t st = (cudaStream_t)stream;
    // the list's header (its capacity), then the log's list address and slot counter;
    // the stream is synchronized before the host words go out of scope
    const unsigned long long h_hdr[2] = {capacity, 0};
    const unsigned long long h_ref[2] = {(unsigned long long)(uintptr_t)d_list, 0};
    agile::LogDev *L = (agile::LogDev *)d_log;
    AGILE_CUDA_TRY(cudaMemcpyAsync(d_list, h_hdr, sizeof h_hdr, cudaMemcpyHostToDevice, st));
    AGILE_CUDA_TRY(cudaMemcpyAsync(&L->list, h_ref, sizeof h_ref, cudaMemcpyHostToDevice, st));
    AGILE_CUDA_TRY(cudaStreamSynchronize(st));
    set_listed(d_log, true);
    return AGILE_OK;
}

int agile_violation_list_read(const void *d_log, const void *d_list, agile_violation_record_t *h_out,
                              size_t max, size_t *n_out, uint64_t *n_seen, void *stream) {
    if (d_log == nullptr || d_list == nullptr || n_out == nullptr || n_seen == nullptr ||
        (h_out == nullptr && max > 0))
        return AGILE_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    agile::LogDev L;
    unsigned long long hdr[2];
    AGILE_CUDA_TRY(cudaMemcpyAsync(&L, d_log, sizeof L, cudaMemcpyDeviceToHost, st));
    AGILE_CUDA_TRY(cudaMemcpyAsync(hdr, d_list, sizeof hdr, cudaMemcpyDeviceToHost, st));
    AGILE_CUDA_TRY(cudaStreamSynchronize(st));
    if (L.list != (unsigned long long)(uintptr_t)d_list) return AGILE_ERR_INVALID_ARG;
    const unsigned long long taken = L.list_next < hdr[0] ? L.list_next : hdr[0];
    const size_t m = taken < max ? (size_t)taken : max;
    *n_seen = L.list_next;
    *n_out = m;
    if (m == 0) return AGILE_OK;
    unsigned long long *e = static_cast<unsigned long long *>(std::malloc(m * AGILE_LIST_ENTRY_BYTES));
    if (e == nullptr) return AGILE_ERR_NOMEM;
    cudaError_t rc = cudaMemcpyAsync(e, static_cast<const unsigned char *>(d_list) + AGILE_LIST_HEADER_BYTES,
                                     m * AGILE_LIST_ENTRY_BYTES, cudaMemcpyDeviceToHost, st);
    if (rc == cudaSuccess) rc = cudaStreamSynchronize(st);
    if (rc != cudaSuccess) {
        std::free(e);
        agile::set_cuda_error(rc, "agile_violation_list_read");
        return AGILE_ERR_CUDA;
    }
    for (size_t j = 0; j < m; ++j) {
        const unsigned long long *x = e + 4 * j;            // {key, addr, info, 0}
        agile_violation_record_t &r = h_out[j];
        std::memset(&r, 0, sizeof r);
        r.key = x[0];
        r.addr = x[1];
        r.site = (uint32_t)(x[2] >> 48) & 0xFFFFu;
        r.verdict = (uint32_t)(x[2] >> 40) & 0xFFu;
        r.width = (uint32_t)(x[2] >> 32) & 0xFFu;
        r.range_id = (uint32_t)x[2];
        r.client = L.client;
        r.status = L.status;
        r.count = 1;
    }
    std::free(e);
    return AGILE_OK;
}

void agile_free(void *p) { std::free(p); }

uint32_t agile_version(void) { return 0x000100; }

const char *agile_strerror(int code) {
    switch (code) {
        case AGILE_OK: return "ok";
        case AGILE_VIOLATION: return "violations were recorded";
        case AGILE_ERR_INVALID_ARG: return "invalid argument";
        case AGILE_ERR_OVERLAP: return "ranges overlap";
        case AGILE_ERR_ZERO_SIZE: return "zero-size range";
        case AGILE_ERR_RANGE_OVERFLOW: return "range end beyond 2^64-1";
        case AGILE_ERR_BAD_KIND: return "unknown range kind";
        case AGILE_ERR_NOMEM: return "out of host memory";
        case AGILE_ERR_CUDA: return g_cuda_msg[0] ? g_cuda_msg : "CUDA runtime error";
        case AGILE_ERR_PTX_PARSE: return "PTX parse error";
        case AGILE_ERR_PTX_UNSUPPORTED: return "PTX construct the guard cannot cover";
        case AGILE_ERR_TIMEOUT: return "a bounded device wait gave up";
        case AGILE_ERR_TOO_LARGE: return "size beyond the supported maximum";
        case AGILE_ERR_ALIGN: return "pointer not aligned as required";
        case AGILE_ERR_NOT_FOUND: return "not found";
        default: return "unknown error";
    }
}

}  // extern "C"
