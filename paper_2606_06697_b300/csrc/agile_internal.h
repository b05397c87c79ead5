// Host-side internals shared by the library's translation units.
#pragma once

#include <stdint.h>

#include <string>
#include <vector>

#include "agile_guard.h"

struct agile_guard_table {
    uint32_t log2_page = 21;
    uint64_t lo = 0;
    uint64_t npages = 0;
    uint32_t n = 0;
    std::vector<uint64_t> base, end;      // ascending base, exclusive end
    std::vector<uint32_t> kind, id;
    std::vector<uint32_t> page;           // npages + 1 entries
    uint32_t search_steps = 0;            // steps covering the largest page slice
    uint64_t remap_or = 0;                // REMAP_OR policy mask
    std::vector<unsigned char> staging;   // host image of the device buffer
    size_t off_base = 0, off_end = 0, off_kind = 0, off_id = 0, total = 0;
    bool compact = false;                 // window < 4 GiB: packed 32-bit records exist
    size_t off_crange = 0;
    size_t off_ubits = 0;
    uint32_t ubits_log2 = 12;
    uint32_t ubits_n = 0;
    size_t off_cmap = 0;                  // block class map (2 bits per block)
    uint32_t cmap_log2 = 8;
    uint32_t cmap_n = 0;
    size_t off_cdesc = 0;                 // open-block descriptors (windows under 4 GiB)
    uint32_t cdesc_log2 = 0, cdesc_k1 = 0, cdesc_k2 = 0;
};

namespace agile {

// Byte layout at the start of an uploaded table's device buffer: the agile_dev_table_t
// header, the 64-byte zero page, the 64-byte sink page, then the page map.
constexpr size_t kTableHeaderBytes = 256, kTableZeroOff = 256, kTableSinkOff = 320,
                 kTablePageOff = 384;

// Device address of the buffer that holds an uploaded table, where its header lives.
inline const unsigned char *table_buffer(const agile_dev_table_t &T) {
    return reinterpret_cast<const unsigned char *>(T.page) - kTablePageOff;
}

// Host form of the rule (same two-level lookup as the device), used by
// agile_validate_args and by the serving loop's admission checks.
uint32_t classify_host(const agile_guard_table &t, uint64_t a, uint64_t w, uint32_t *rid);

// Device bytes of a batch work list of n items: the 64-byte header, the items (64 bytes
// each) and n + 1 tile prefix sums, rounded up to 256 bytes (agile_batch_device_bytes).
constexpr size_t batch_device_bytes(size_t n) { return (64 + 64 * n + 8 * (n + 1) + 255) & ~size_t(255); }

// Validation of one batch work item (kind, policy, size, alignment), as the batch upload
// applies it.
int batch_check_item(const agile_work_t &w);

// agile_batch_launch for a work list image that was copied to the device, claim counter
// zeroed, on the same stream just before (the serving worker's launches).
int batch_launch_fresh(void *d_buf, size_t n_items, const agile_batch_config_t *cfg, void *stream);

// Remember the last CUDA error text for agile_strerror-style diagnostics.
void set_cuda_error(int err, const char *where);

// Logs with a bounded violation list attached through this library (kept on the host, so
// that the batch checks can launch their per-access form, which appends every violation,
// for those logs only); agile_violation_log_init forgets a log.
bool log_has_list(const void *d_log);
int sm_count();
}  // namespace agile

// Internal check for CUDA calls in host code: returns AGILE_ERR_CUDA from the caller.
#define AGILE_CUDA_TRY(call)                                        \
    do {                                                            \
        cudaError_t e_ = (call);                                    \
        if (e_ != cudaSuccess) {                                    \
            agile::set_cuda_error((int)e_, #call);                  \
            return AGILE_ERR_CUDA;                                  \
        }                                                           \
    } while (0)
