// Guarded streaming kernels over host arrays: chunked copies in, the guarded kernel, copy
// out, on three rotating streams, so that the host link's two directions and the kernels
// overlap. Each chunk starts on a 16-byte unit boundary, so the kernels make exactly the
// accesses one launch over the whole arrays would make.
#include <cuda_runtime.h>

#include "agile_internal.h"

namespace {

constexpr int kStreams = 3;

struct Pipeline {
    cudaStream_t st[kStreams] = {};
    cudaEvent_t ev[kStreams + 1] = {};
    ~Pipeline() {          // destroying streams and events with work pending is allowed
        for (cudaStream_t s : st)
            if (s) cudaStreamDestroy(s);
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
    }
};

}  // namespace

extern "C" int agile_stream_launch_host(int op, const agile_dev_table_t *tbl, float *d_a,
                                        float *d_b, float *d_c, float *h_a, const float *h_b,
                                        const float *h_c, size_t n, float s, int policy,
                                        void *d_log, size_t chunk_elems, void *stream) {
    if (op < AGILE_OP_COPY || op > AGILE_OP_TRIAD) return AGILE_ERR_INVALID_ARG;
    if (chunk_elems == 0) chunk_elems = (size_t)1 << 24;
    if (chunk_elems % 4 != 0) return AGILE_ERR_INVALID_ARG;
    if (n == 0) return AGILE_OK;
    if (d_a == nullptr || d_b == nullptr || (op == AGILE_OP_TRIAD && d_c == nullptr))
        return AGILE_ERR_INVALID_ARG;
    cudaStream_t caller = (cudaStream_t)stream;
    Pipeline P;
    for (int i = 0; i < kStreams; ++i)
        AGILE_CUDA_TRY(cudaStreamCreateWithFlags(&P.st[i], cudaStreamNonBlocking));
    for (int i = 0; i <= kStreams; ++i)
        AGILE_CUDA_TRY(cudaEventCreateWithFlags(&P.ev[i], cudaEventDisableTiming));
    AGILE_CUDA_TRY(cudaEventRecord(P.ev[kStreams], caller));      // earlier work first
    for (int i = 0; i < kStreams; ++i) AGILE_CUDA_TRY(cudaStreamWaitEvent(P.st[i], P.ev[kStreams], 0));
    const bool triad = op == AGILE_OP_TRIAD;
    size_t k = 0;
    for (size_t e0 = 0; e0 < n; e0 += chunk_elems, ++k) {
        const size_t cnt = n - e0 < chunk_elems ? n - e0 : chunk_elems;
        const size_t bytes = cnt * sizeof(float);
        cudaStream_t st = P.st[k % kStreams];
        if (h_b) AGILE_CUDA_TRY(cudaMemcpyAsync(d_b + e0, h_b + e0, bytes, cudaMemcpyHostToDevice, st));
        if (triad && h_c)
            AGILE_CUDA_TRY(cudaMemcpyAsync(d_c + e0, h_c + e0, bytes, cudaMemcpyHostToDevice, st));
        const int rc = agile_stream_launch(op, tbl, d_a + e0, d_b + e0, triad ? d_c + e0 : nullptr,
                                           cnt, s, policy, d_log, st);
        if (rc != AGILE_OK) return rc;
        if (h_a) AGILE_CUDA_TRY(cudaMemcpyAsync(h_a + e0, d_a + e0, bytes, cudaMemcpyDeviceToHost, st));
    }
    for (int i = 0; i < kStreams; ++i) {                          // later work waits for all
        AGILE_CUDA_TRY(cudaEventRecord(P.ev[i], P.st[i]));
        AGILE_CUDA_TRY(cudaStreamWaitEvent(caller, P.ev[i], 0));
    }
    return AGILE_OK;
}
