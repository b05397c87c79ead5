// Streaming kernels with the guard fused in by hand (Sec. V-E: an address-range check
// before every global access, ordinary user-allocation accesses left on the normal path)
// and their unguarded twins; the per-tile bodies live in stream_body.cuh.
#include <cuda_runtime.h>

#include "agile_internal.h"
#include "stream_body.cuh"

namespace {

using agile::LogDev;
using agile::TView;
using agile::WarpSlots;

constexpr int kThreads = 512;

// Launch shapes, measured on the 2^28-element arrays: the guarded kernels run one block of
// 512 threads per SM, each lane keeping 8 units per array in flight (128 registers); the
// unguarded twins run two blocks per SM with 4 units per lane, their best shape. Either
// kind can be launched at either shape (agile_stream_launch_shape), so that the guard's
// cost can be read at equal shapes.
template <int OP, bool GUARD, int POLICY, int U, int BPS>
__global__ void __launch_bounds__(kThreads, BPS)
k_stream(const agile_dev_table_t T, float *__restrict__ a, const float *__restrict__ b,
         const float *__restrict__ c, size_t n, float s, LogDev *log) {
    constexpr uint32_t kTile = 32 * U;
    __shared__ WarpSlots S;
    TView V{};
    if constexpr (GUARD) {
        // The page map is read through L1 rather than staged: a warp checks three spans
        // per tile, and skipping the staging lets every block start streaming at once.
        agile::slots_init(S);
        if (threadIdx.x == 0) S.log = log;
        __syncthreads();
        V = agile::view_of(T);
    }
    const size_t n4 = n >> 2;
    const size_t warp = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const size_t nwarps = ((size_t)gridDim.x * blockDim.x) >> 5;
    const size_t tiles = (n4 + kTile - 1) / kTile;
    for (size_t t = warp; t < tiles; t += nwarps)             // warp-uniform
        agile::stream_warp_tile<OP, GUARD, POLICY, U>(V, T, a, b, c, t, n4, n, s, S, true);
    // Elements past the last whole 16-byte unit: 4-byte accesses by the last warp.
    if ((n & 3) && blockIdx.x == gridDim.x - 1 && (threadIdx.x >> 5) == (blockDim.x >> 5) - 1)
        agile::stream_tail<OP, GUARD, POLICY>(V, T, a, b, c, n, s, S);
    if constexpr (GUARD) agile::slots_flush(log, S);
}

template <int OP, bool GUARD, int POLICY, int U, int BPS>
int launch(const agile_dev_table_t &T, float *a, const float *b, const float *c, size_t n,
           float s, LogDev *log, cudaStream_t st) {
    constexpr uint32_t kTile = 32 * U;
    const size_t tiles = ((n >> 2) + kTile - 1) / kTile;
    const size_t want = (tiles * 32 + kThreads - 1) / kThreads;
    const size_t cap = (size_t)agile::sm_count() * BPS;
    const unsigned blocks = (unsigned)(want < 1 ? 1 : want > cap ? cap : want);
    k_stream<OP, GUARD, POLICY, U, BPS><<<blocks, kThreads, 0, st>>>(T, a, b, c, n, s, log);
    AGILE_CUDA_TRY(cudaGetLastError());
    return AGILE_OK;
}

// Shape 0: 8 units x 1 block per SM; shape 1: 4 units x 2 blocks per SM.
template <int OP, bool GUARD, int POLICY>
int launch_shape(int shape, const agile_dev_table_t &T, float *a, const float *b, const float *c,
                 size_t n, float s, LogDev *log, cudaStream_t st) {
    return shape == 0 ? launch<OP, GUARD, POLICY, 8, 1>(T, a, b, c, n, s, log, st)
                      : launch<OP, GUARD, POLICY, 4, 2>(T, a, b, c, n, s, log, st);
}

template <int OP>
int dispatch(const agile_dev_table_t *tbl, float *a, const float *b, const float *c, size_t n,
             float s, int policy, LogDev *log, int shape, cudaStream_t st) {
    if (tbl == nullptr) {
        agile_dev_table_t none = {};
        return launch_shape<OP, false, AGILE_POLICY_REPORT>(shape < 0 ? 1 : shape, none, a, b, c, n, s,
                                                            nullptr, st);
    }
    if (shape < 0) shape = 0;
    switch (policy) {
        case AGILE_POLICY_POISON:
            return launch_shape<OP, true, AGILE_POLICY_POISON>(shape, *tbl, a, b, c, n, s, log, st);
        case AGILE_POLICY_SINK:
            return launch_shape<OP, true, AGILE_POLICY_SINK>(shape, *tbl, a, b, c, n, s, log, st);
        case AGILE_POLICY_REPORT:
            return launch_shape<OP, true, AGILE_POLICY_REPORT>(shape, *tbl, a, b, c, n, s, log, st);
        default: return AGILE_ERR_INVALID_ARG;
    }
}

// Argument checks and dispatch; shape -1 picks each kind's own shape.
int stream_launch(int op, const agile_dev_table_t *tbl, float *d_a, const float *d_b,
                  const float *d_c, size_t n, float s, int policy, void *d_log, int shape,
                  void *stream) {
    if (op < AGILE_OP_COPY || op > AGILE_OP_TRIAD) return AGILE_ERR_INVALID_ARG;
    if (policy < AGILE_POLICY_POISON || policy > AGILE_POLICY_REPORT) return AGILE_ERR_INVALID_ARG;
    if (n == 0) return AGILE_OK;
    if (d_a == nullptr || d_b == nullptr || (op == AGILE_OP_TRIAD && d_c == nullptr))
        return AGILE_ERR_INVALID_ARG;
    if (((uintptr_t)d_a & 15) || ((uintptr_t)d_b & 15) || (op == AGILE_OP_TRIAD && ((uintptr_t)d_c & 15)))
        return AGILE_ERR_ALIGN;
    if (d_log != nullptr && ((uintptr_t)d_log & 15) != 0) return AGILE_ERR_ALIGN;
    LogDev *log = (LogDev *)d_log;
    cudaStream_t st = (cudaStream_t)stream;
    const float *c = op == AGILE_OP_TRIAD ? d_c : d_b;
    switch (op) {
        case AGILE_OP_COPY: return dispatch<AGILE_OP_COPY>(tbl, d_a, d_b, c, n, s, policy, log, shape, st);
        case AGILE_OP_SCALE: return dispatch<AGILE_OP_SCALE>(tbl, d_a, d_b, c, n, s, policy, log, shape, st);
        default: return dispatch<AGILE_OP_TRIAD>(tbl, d_a, d_b, c, n, s, policy, log, shape, st);
    }
}

}  // namespace

extern "C" int agile_stream_launch(int op, const agile_dev_table_t *tbl, float *d_a,
                                   const float *d_b, const float *d_c, size_t n, float s,
                                   int policy, void *d_log, void *stream) {
    return stream_launch(op, tbl, d_a, d_b, d_c, n, s, policy, d_log, -1, stream);
}

extern "C" int agile_stream_launch_shape(int op, const agile_dev_table_t *tbl, float *d_a,
                                         const float *d_b, const float *d_c, size_t n, float s,
                                         int policy, void *d_log, int units, int blocks_per_sm,
                                         void *stream) {
    int shape;
    if (units == 8 && blocks_per_sm == 1) shape = 0;
    else if (units == 4 && blocks_per_sm == 2) shape = 1;
    else return AGILE_ERR_INVALID_ARG;
    return stream_launch(op, tbl, d_a, d_b, d_c, n, s, policy, d_log, shape, stream);
}
