// Guarded streaming kernels over host arrays: chunked copies in, the guarded kernel, copy
// out, on three rotating streams, so that the host link's two directions and the kernels
// overlap. Each chunk starts on a 16-byte unit boundary, so the kernels make exactly the
// accesses one launch over the whole arrays would make.
#include <cuda_runtime.h>

#include <map>

#include "agile_internal.h"

namespace {

constexpr int kStreams = 3;

// The pipeline's streams and events, created on first use per device and calling thread
// and kept for the life of the process (a call reuses them instead of creating and
// destroying three streams and four events).
struct Pipeline {
    cudaStream_t st[kStreams] = {};
    cudaEvent_t ev[kStreams + 1] = {};
};

int pipeline_for_current_device(Pipeline **out) {
    thread_local std::map<int, Pipeline> cache;
    int dev = 0;
    AGILE_CUDA_TRY(cudaGetDevice(&dev));
    Pipeline &P = cache[dev];
    for (int i = 0; i < kStreams; ++i)
        if (P.st[i] == nullptr) AGILE_CUDA_TRY(cudaStreamCreateWithFlags(&P.st[i], cudaStreamNonBlocking));
    for (int i = 0; i <= kStreams; ++i)
        if (P.ev[i] == nullptr) AGILE_CUDA_TRY(cudaEventCreateWithFlags(&P.ev[i], cudaEventDisableTiming));
    *out = &P;
    return AGILE_OK;
}

}  // namespace

extern "C" int agile_stream_launch_host(int op, const agile_dev_table_t *tbl, float *d_a,
                                        float *d_b, float *d_c, float *h_a, const float *h_b,
                                        const float *h_c, size_t n, float s, int policy,
                                        void *d_log, size_t chunk_elems, void *stream) {
    if (op < AGILE_OP_COPY || op > AGILE_OP_TRIAD) return AGILE_ERR_INVALID_ARG;
    if (policy < AGILE_POLICY_POISON || policy > AGILE_POLICY_REPORT) return AGILE_ERR_INVALID_ARG;
    if (chunk_elems == 0) chunk_elems = (size_t)1 << 24;
    if (chunk_elems % 4 != 0) return AGILE_ERR_INVALID_ARG;
    if (n == 0) return AGILE_OK;
    const bool triad = op == AGILE_OP_TRIAD;
    if (d_a == nullptr || d_b == nullptr || (triad && d_c == nullptr)) return AGILE_ERR_INVALID_ARG;
    // Every chunk base is the array base plus a multiple of 16 bytes, so the checks that
    // agile_stream_launch makes per chunk hold for all chunks once they hold here: nothing
    // is queued for a call these reject, and a chunk launch can then fail only in CUDA.
    if (((uintptr_t)d_a & 15) || ((uintptr_t)d_b & 15) || (triad && ((uintptr_t)d_c & 15)))
        return AGILE_ERR_ALIGN;
    if (d_log != nullptr && ((uintptr_t)d_log & 15) != 0) return AGILE_ERR_ALIGN;
    cudaStream_t caller = (cudaStream_t)stream;
    Pipeline *P = nullptr;
    if (int rc = pipeline_for_current_device(&P)) return rc;
    AGILE_CUDA_TRY(cudaEventRecord(P->ev[kStreams], caller));     // earlier work first
    for (int i = 0; i < kStreams; ++i) AGILE_CUDA_TRY(cudaStreamWaitEvent(P->st[i], P->ev[kStreams], 0));
    int rc = AGILE_OK;
    size_t k = 0;
    for (size_t e0 = 0; e0 < n && rc == AGILE_OK; e0 += chunk_elems, ++k) {
        const size_t cnt = n - e0 < chunk_elems ? n - e0 : chunk_elems;
        const size_t bytes = cnt * sizeof(float);
        cudaStream_t st = P->st[k % kStreams];
        cudaError_t e = cudaSuccess;
        if (h_b) e = cudaMemcpyAsync(d_b + e0, h_b + e0, bytes, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && triad && h_c)
            e = cudaMemcpyAsync(d_c + e0, h_c + e0, bytes, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) {
            agile::set_cuda_error((int)e, "cudaMemcpyAsync (host to device chunk)");
            rc = AGILE_ERR_CUDA;
            break;
        }
        rc = agile_stream_launch(op, tbl, d_a + e0, d_b + e0, triad ? d_c + e0 : nullptr, cnt, s,
                                 policy, d_log, st);
        if (rc == AGILE_OK && h_a) {
            e = cudaMemcpyAsync(h_a + e0, d_a + e0, bytes, cudaMemcpyDeviceToHost, st);
            if (e != cudaSuccess) {
                agile::set_cuda_error((int)e, "cudaMemcpyAsync (device to host chunk)");
                rc = AGILE_ERR_CUDA;
            }
        }
    }
    // Later work on the caller's stream waits for every chunk queued so far -- also when a
    // chunk failed, so that no copy queued before the failure still runs once the caller
    // reuses or frees its buffers after synchronizing its stream.
    for (int i = 0; i < kStreams; ++i) {
        AGILE_CUDA_TRY(cudaEventRecord(P->ev[i], P->st[i]));
        AGILE_CUDA_TRY(cudaStreamWaitEvent(caller, P->ev[i], 0));
    }
    return rc;
}
