// Batched guarded launch that allocates nothing.
//
// Some callers cannot call cudaMalloc: a worker whose whole device-memory budget is
// already handed out by its admission accounting, code that must not risk the implicit
// device synchronization an allocation or free can cause, and plugin hosts that give a
// plugin no allocator. For them, agile_batch_launch_static runs the same persistent
// batch kernel with its scratch -- the work list, the tile prefix sums and the tile-claim
// counter -- in a fixed array in this file instead of a caller-provided buffer. The
// caller still owns every input and output buffer named by the work items.
//
// The array is a file-scope __device__ variable of AGILE_BATCH_STATIC_MAX_ITEMS items'
// worth of bytes: every GPU that loads the library holds it until the process exits.
// In host code its name is only a host-side stand-in, so the device address is looked up
// once per device (cudaGetSymbolAddress, with that device current) on the first call
// made on that device, and passed to the kernel. All calls share the array and it keeps
// the last call's contents; the launch clears the claim counter before the kernel runs.
// Calls whose work overlaps on the GPU (different streams, or a new call before the
// previous one finished) race on the array.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "agile_internal.h"

namespace {

constexpr size_t kItems = AGILE_BATCH_STATIC_MAX_ITEMS;
constexpr size_t kBytes = agile::batch_device_bytes(kItems);   // what agile_batch_upload needs
static_assert(kBytes >= 64 + 64 * kItems + 8 * (kItems + 1), "the array holds a full work list");

static __device__ __align__(256) unsigned char g_batch_scratch[kBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_ptr[kMaxDevices] = {};

// Host image of the scratch, built on the calling thread; no heap allocation.
thread_local unsigned char h_image[kBytes];

int scratch_for_current_device(void **out) {
    int dev = 0;
    AGILE_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return AGILE_ERR_TOO_LARGE;
    std::lock_guard<std::mutex> lock(g_mu);
    if (g_ptr[dev] == nullptr) {
        void *p = nullptr;
        AGILE_CUDA_TRY(cudaGetSymbolAddress(&p, g_batch_scratch));
        g_ptr[dev] = p;
    }
    *out = g_ptr[dev];
    return AGILE_OK;
}

}  // namespace

extern "C" int agile_batch_launch_static(const agile_work_t *h_items, size_t n, uint32_t tile,
                                         const agile_batch_config_t *cfg, void *stream) {
    if (h_items == nullptr || cfg == nullptr || n == 0) return AGILE_ERR_INVALID_ARG;
    if (n > kItems) return AGILE_ERR_TOO_LARGE;
    if (tile < 512 || (tile & 511) != 0) return AGILE_ERR_INVALID_ARG;
    for (size_t i = 0; i < n; ++i) {
        const int rc = agile::batch_check_item(h_items[i]);
        if (rc != AGILE_OK) return rc;
    }
    void *d = nullptr;
    const int rc = scratch_for_current_device(&d);
    if (rc != AGILE_OK) return rc;
    // Same image as agile_batch_upload: header, items, tile prefix sums.
    const size_t used = 64 + 64 * n + 8 * (n + 1);
    uint64_t *pre = reinterpret_cast<uint64_t *>(h_image + 64 + 64 * n);
    pre[0] = 0;
    for (size_t i = 0; i < n; ++i) pre[i + 1] = pre[i] + (h_items[i].n + tile - 1) / tile;
    uint64_t hdr[8] = {n, pre[n], 0, tile, 0, 0, 0, 0};   // items, tiles, counter, tile
    std::memcpy(h_image, hdr, 64);
    std::memcpy(h_image + 64, h_items, 64 * n);
    AGILE_CUDA_TRY(cudaMemcpyAsync(d, h_image, used, cudaMemcpyHostToDevice, (cudaStream_t)stream));
    return agile_batch_launch(d, n, cfg, stream);
}
