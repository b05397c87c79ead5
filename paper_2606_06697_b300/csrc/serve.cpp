// Serving worker: a trusted worker thread that takes client requests as they arrive,
// validates every pointer argument against the client's live allocations before any
// launch (Sec. IV-C: the worker mediates every operation; Sec. V-C: pointers are resolved
// against the allocation table and rejected if not inside one live allocation), admits
// validated requests in arrival order under a device-memory budget, and packs the
// admitted requests into persistent batched launches -- each kernel guarded by its
// client's table (Sec. V-E) -- while earlier launches are still running (continuous
// batching). Requests that carry the same exclusive key never run at the same time, so
// a request's outputs are the same alone and in the mix.
//
// Per launch slot: one stream, one event, one pinned host staging image, one region of the
// caller's device buffer holding the work list and the per-request done counters, and one
// host-mapped array of per-request completion notices. A request completes when its
// notice is raised -- its kernel's last tile is done -- not when its whole launch ends, so
// a small request packed with a large one does not wait for it; the slot itself is reused
// only once its launch's event has completed. The worker clock is steady_clock
// nanoseconds since agile_worker_start.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <queue>
#include <thread>
#include <unordered_set>
#include <vector>

#include "agile_internal.h"

namespace {

// A short busy wait that keeps the core: the worker's latency-critical loop must not give
// its core away for a scheduler tick while launches are in flight or an arrival is near.
inline void spin_pause() {
    for (int i = 0; i < 16; ++i) {
#if defined(__x86_64__) || defined(__i386__)
        __builtin_ia32_pause();
#elif defined(__aarch64__)
        asm volatile("yield");
#endif
    }
}

// A slot's device region: the batch work list of n requests (header, items, tile prefix
// sums), directly followed by one u32 done counter per request, so one copy carries both.
size_t list_bytes(size_t n) { return 64 + 64 * n + 8 * (n + 1); }
size_t slot_bytes(uint32_t max_batch) {
    return (list_bytes(max_batch) + 4 * (size_t)max_batch + 255) & ~size_t(255);
}

struct Slot {
    bool busy = false;
    std::vector<uint32_t> reqs;
    std::vector<char> fin;              // per request of the launch: completed already
    uint32_t open = 0;                  // requests of the launch not yet completed
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    unsigned char *staging = nullptr;   // pinned
    unsigned char *dev = nullptr;
    unsigned int *notice = nullptr;     // pinned, mapped: the host's view
    unsigned int *notice_dev = nullptr; // the same flags as the device addresses them
};

}  // namespace

struct agile_worker {
    agile_worker_config_t cfg{};
    std::vector<const agile_guard_table *> htab;
    std::vector<const agile_dev_table_t *> dtab;
    std::vector<void *> dlog;
    std::vector<Slot> slots;
    int device = 0;

    std::mutex mu_in;
    std::vector<agile_request_t> incoming;
    std::mutex mu_out;
    std::condition_variable cv_out;
    std::deque<agile_completion_t> ready;

    std::thread th;
    std::atomic<bool> stop{false};
    std::atomic<bool> started{false};
    std::chrono::steady_clock::time_point t0;
    std::atomic<uint64_t> admitted_pub{0}, peak_pub{0};
    std::atomic<uint64_t> submitted{0}, completed{0};

    // worker-thread state
    std::vector<agile_request_t> reqs;
    std::vector<agile_completion_t> comp;
    std::priority_queue<std::pair<uint64_t, uint32_t>, std::vector<std::pair<uint64_t, uint32_t>>,
                        std::greater<std::pair<uint64_t, uint32_t>>> arrivals;
    std::deque<uint32_t> waiting;
    std::unordered_set<uint64_t> busy_keys;
    uint64_t admitted = 0;
    uint32_t launches = 0;
    std::vector<uint32_t> batch_buf;             // launch(): reused, so a launch allocates nothing
    std::unordered_set<uint64_t> keys_buf;

    uint64_t now() const {
        return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
                   std::chrono::steady_clock::now() - t0).count();
    }

    void finish(uint32_t id, int32_t status, uint32_t bad_arg, uint32_t verdict, uint64_t t) {
        agile_completion_t &c = comp[id];
        if (c.seen_ns == 0) c.seen_ns = t;
        c.tag = reqs[id].tag;
        c.status = status;
        c.bad_arg = bad_arg;
        c.verdict = verdict;
        c.arrival_ns = reqs[id].arrival_ns;
        c.done_ns = t;
        {
            std::lock_guard<std::mutex> g(mu_out);
            ready.push_back(c);
        }
        completed.fetch_add(1);
        cv_out.notify_all();
    }

    void take_incoming() {
        std::vector<agile_request_t> in;
        {
            std::lock_guard<std::mutex> g(mu_in);
            in.swap(incoming);
        }
        for (const agile_request_t &r : in) {
            const uint32_t id = (uint32_t)reqs.size();
            reqs.push_back(r);
            comp.push_back(agile_completion_t{});
            arrivals.push({r.arrival_ns, id});
        }
    }

    // Validation at arrival: every pointer argument inside one live user allocation of
    // the request's client; the kernel's work item well formed; the request able to fit
    // the budget at all.
    void arrive(uint32_t id, uint64_t t) {
        agile_request_t &r = reqs[id];
        if (r.client >= htab.size() || r.nargs > AGILE_MAX_ARGS) {
            finish(id, AGILE_ERR_INVALID_ARG, 0, 0, t);
            return;
        }
        for (uint32_t k = 0; k < r.nargs; ++k) {
            uint32_t rid;
            const uint32_t v = agile::classify_host(*htab[r.client], r.arg_ptr[k], r.arg_bytes[k], &rid);
            if (v != AGILE_ALLOW) {
                finish(id, AGILE_VIOLATION, k, v, t);
                return;
            }
        }
        if (r.work.table == nullptr) r.work.table = agile::table_buffer(*dtab[r.client]);
        if (r.work.log == nullptr) r.work.log = dlog[r.client];
        const int rc = agile::batch_check_item(r.work);
        if (rc != AGILE_OK) { finish(id, rc, 0, 0, t); return; }
        if (r.mem_bytes > cfg.mem_budget) { finish(id, AGILE_ERR_TOO_LARGE, 0, 0, t); return; }
        comp[id].seen_ns = now();
        waiting.push_back(id);
    }

    // Request k of slot s is done: release its key and memory, complete it.
    void complete(Slot &s, uint32_t k, int32_t status, uint64_t t) {
        const uint32_t id = s.reqs[k];
        s.fin[k] = 1;
        --s.open;
        if (reqs[id].excl) busy_keys.erase(reqs[id].excl);
        admitted -= reqs[id].mem_bytes;
        admitted_pub.store(admitted);
        finish(id, status, 0, 0, t);
    }

    bool any_busy() const {
        for (const Slot &s : slots) if (s.busy) return true;
        return false;
    }

    // Complete every request whose notice is up; free a slot once its launch has ended.
    void reap(uint64_t t) {
        for (Slot &s : slots) {
            if (!s.busy) continue;
            if (s.open != 0)
                for (uint32_t k = 0; k < s.reqs.size(); ++k)
                    if (!s.fin[k] && reinterpret_cast<volatile unsigned int *>(s.notice)[k] != 0)
                        complete(s, k, AGILE_OK, t);
            const cudaError_t q = cudaEventQuery(s.done);
            if (q == cudaErrorNotReady) continue;
            // The launch has ended. A notice that is still down can only mean the launch
            // failed on the device: those requests complete with the error.
            for (uint32_t k = 0; k < s.reqs.size(); ++k)
                if (!s.fin[k]) {
                    const bool up = reinterpret_cast<volatile unsigned int *>(s.notice)[k] != 0;
                    complete(s, k, up && q == cudaSuccess ? AGILE_OK : AGILE_ERR_CUDA, now());
                }
            s.reqs.clear();
            s.fin.clear();
            s.busy = false;
        }
    }

    void launch(Slot &s, uint64_t t) {
        if (!cfg.continuous && any_busy()) return;
        std::vector<uint32_t> &batch = batch_buf;
        std::unordered_set<uint64_t> &keys = keys_buf;
        batch.clear();
        keys.clear();
        uint64_t mem = 0;
        for (auto it = waiting.begin(); it != waiting.end() && batch.size() < cfg.max_batch;) {
            const agile_request_t &r = reqs[*it];
            if (admitted + mem + r.mem_bytes > cfg.mem_budget) break;   // admission in order
            if (r.excl && (busy_keys.count(r.excl) || keys.count(r.excl))) { ++it; continue; }
            batch.push_back(*it);
            mem += r.mem_bytes;
            if (r.excl) keys.insert(r.excl);
            it = waiting.erase(it);
            if (!cfg.continuous) break;
        }
        if (batch.empty()) return;
        const size_t n = batch.size();
        uint64_t *pre = reinterpret_cast<uint64_t *>(s.staging + 64 + 64 * n);
        pre[0] = 0;
        for (size_t i = 0; i < n; ++i) {
            const agile_work_t &w = reqs[batch[i]].work;
            std::memcpy(s.staging + 64 + 64 * i, &w, 64);
            pre[i + 1] = pre[i] + (w.n + cfg.tile - 1) / cfg.tile;
        }
        // header: items, tiles, claim counter (zero), tile, done counters, notices
        const size_t list = list_bytes(n);
        const uint64_t hdr[8] = {n, pre[n], 0, cfg.tile, (uint64_t)(uintptr_t)(s.dev + list),
                                 (uint64_t)(uintptr_t)s.notice_dev, 0, 0};
        std::memcpy(s.staging, hdr, 64);
        std::memset(s.staging + list, 0, 4 * n);
        std::memset(s.notice, 0, 4 * n);
        agile_batch_config_t bc{cfg.tile, 1, 2, 0};
        // one copy: the work list with its zeroed claim counter, and the zeroed done counters
        int rc = cudaMemcpyAsync(s.dev, s.staging, list + 4 * n, cudaMemcpyHostToDevice, s.stream) == cudaSuccess
                     ? agile::batch_launch_fresh(s.dev, n, &bc, s.stream)
                     : AGILE_ERR_CUDA;
        const bool launched = rc == AGILE_OK;
        const bool recorded = cudaEventRecord(s.done, s.stream) == cudaSuccess;
        const uint32_t seq = launches++;
        const uint64_t tq = now();
        for (uint32_t id : batch) {
            comp[id].admit_ns = t;
            comp[id].queued_ns = tq;
            comp[id].launch = seq;
            if (reqs[id].excl) busy_keys.insert(reqs[id].excl);
        }
        admitted += mem;
        admitted_pub.store(admitted);
        if (admitted > peak_pub.load()) peak_pub.store(admitted);
        s.reqs.assign(batch.begin(), batch.end());
        s.fin.assign(n, 0);
        s.open = (uint32_t)n;
        if (!launched || !recorded) {
            // Nothing was launched, or the kernel was launched but its end cannot be
            // observed through the event. Either way wait for the stream, then complete
            // each request by what happened to it: a raised notice means its kernel ran to
            // the end (its outputs and log are written), so it completes normally -- a
            // retry of it would apply non-idempotent work such as histogram increments
            // twice; the others complete with AGILE_ERR_CUDA.
            cudaStreamSynchronize(s.stream);
            const uint64_t tf = now();
            for (uint32_t k = 0; k < n; ++k) {
                const bool up = launched && reinterpret_cast<volatile unsigned int *>(s.notice)[k] != 0;
                complete(s, k, up ? AGILE_OK : AGILE_ERR_CUDA, tf);
            }
            s.reqs.clear();
            s.fin.clear();
            return;
        }
        s.busy = true;
    }

    void run() {
        cudaSetDevice(device);
        for (;;) {
            take_incoming();
            uint64_t t = now();
            reap(t);
            while (!arrivals.empty() && arrivals.top().first <= t) {
                const uint32_t id = arrivals.top().second;
                arrivals.pop();
                arrive(id, t);
            }
            for (Slot &s : slots)
                if (!s.busy && !waiting.empty()) launch(s, now());
            const bool idle = !any_busy() && waiting.empty();
            if (stop.load() && idle && arrivals.empty()) {
                std::lock_guard<std::mutex> g(mu_in);
                if (incoming.empty()) break;
                continue;
            }
            if (any_busy()) {
                spin_pause();
            } else if (!arrivals.empty()) {
                // Sleep only through long gaps, waking 1 ms early: a sleep can overrun by
                // tens of microseconds, which would land on the request's latency. The
                // last stretch is spent polling.
                const uint64_t next = arrivals.top().first;
                const uint64_t t2 = now();
                if (next > t2 + 1500000) std::this_thread::sleep_for(std::chrono::nanoseconds(next - t2 - 1000000));
                else spin_pause();
            } else {
                std::this_thread::sleep_for(std::chrono::microseconds(20));
            }
        }
    }
};

extern "C" {

size_t agile_worker_device_bytes(const agile_worker_config_t *cfg) {
    if (cfg == nullptr || cfg->max_batch == 0 || cfg->max_inflight == 0) return 0;
    return slot_bytes(cfg->max_batch) * cfg->max_inflight;
}

int agile_worker_create(const agile_worker_config_t *cfg, const agile_guard_table_t *const *h_tables,
                        const agile_dev_table_t *const *d_tables, void *const *d_logs,
                        size_t n_clients, void *d_buf, size_t bytes, agile_worker_t **out) {
    if (cfg == nullptr || out == nullptr || h_tables == nullptr || d_tables == nullptr ||
        n_clients == 0 || d_buf == nullptr)
        return AGILE_ERR_INVALID_ARG;
    *out = nullptr;
    if (cfg->max_batch == 0 || cfg->max_inflight == 0 || cfg->max_inflight > 64 ||
        cfg->tile < 512 || (cfg->tile & 511))
        return AGILE_ERR_INVALID_ARG;
    if (((uintptr_t)d_buf & 255) != 0) return AGILE_ERR_ALIGN;
    if (bytes < agile_worker_device_bytes(cfg)) return AGILE_ERR_TOO_LARGE;
    for (size_t i = 0; i < n_clients; ++i)
        if (h_tables[i] == nullptr || d_tables[i] == nullptr) return AGILE_ERR_INVALID_ARG;
    agile_worker *w = new (std::nothrow) agile_worker;
    if (w == nullptr) return AGILE_ERR_NOMEM;
    w->cfg = *cfg;
    w->htab.assign(h_tables, h_tables + n_clients);
    w->dtab.assign(d_tables, d_tables + n_clients);
    w->dlog.assign(n_clients, nullptr);
    if (d_logs) for (size_t i = 0; i < n_clients; ++i) w->dlog[i] = d_logs[i];
    cudaGetDevice(&w->device);
    const size_t sb = slot_bytes(cfg->max_batch);
    w->slots.resize(cfg->max_inflight);
    w->batch_buf.reserve(cfg->max_batch);
    w->keys_buf.reserve(2 * (size_t)cfg->max_batch);
    for (uint32_t k = 0; k < cfg->max_inflight; ++k) {
        Slot &s = w->slots[k];
        s.dev = static_cast<unsigned char *>(d_buf) + k * sb;
        s.reqs.reserve(cfg->max_batch);
        s.fin.reserve(cfg->max_batch);
        cudaError_t e = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void **>(&s.staging), sb);
        if (e == cudaSuccess)
            e = cudaHostAlloc(reinterpret_cast<void **>(&s.notice), 4 * (size_t)cfg->max_batch,
                              cudaHostAllocMapped);
        if (e == cudaSuccess) e = cudaHostGetDevicePointer(reinterpret_cast<void **>(&s.notice_dev), s.notice, 0);
        if (e != cudaSuccess) {
            agile::set_cuda_error((int)e, "worker slot");
            agile_worker_destroy(w);
            return AGILE_ERR_CUDA;
        }
    }
    *out = w;
    return AGILE_OK;
}

int agile_worker_submit(agile_worker_t *w, const agile_request_t *reqs, size_t n) {
    if (w == nullptr || (n > 0 && reqs == nullptr)) return AGILE_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> g(w->mu_in);
        w->incoming.insert(w->incoming.end(), reqs, reqs + n);
    }
    w->submitted.fetch_add(n);
    return AGILE_OK;
}

int agile_worker_start(agile_worker_t *w) {
    if (w == nullptr || w->started.exchange(true)) return AGILE_ERR_INVALID_ARG;
    w->t0 = std::chrono::steady_clock::now();
    w->th = std::thread([w] { w->run(); });
    return AGILE_OK;
}

int agile_worker_poll(agile_worker_t *w, agile_completion_t *out, size_t cap, size_t *got,
                      uint32_t wait_ms) {
    if (w == nullptr || got == nullptr || (cap > 0 && out == nullptr)) return AGILE_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(w->mu_out);
    if (w->ready.empty() && wait_ms > 0)
        w->cv_out.wait_for(lk, std::chrono::milliseconds(wait_ms), [w] { return !w->ready.empty(); });
    size_t k = 0;
    while (k < cap && !w->ready.empty()) {
        out[k++] = w->ready.front();
        w->ready.pop_front();
    }
    *got = k;
    return AGILE_OK;
}

int agile_worker_clock(agile_worker_t *w, uint64_t *now_ns, uint64_t *admitted_bytes,
                       uint64_t *peak_admitted_bytes) {
    if (w == nullptr) return AGILE_ERR_INVALID_ARG;
    if (now_ns) *now_ns = w->started.load() ? w->now() : 0;
    if (admitted_bytes) *admitted_bytes = w->admitted_pub.load();
    if (peak_admitted_bytes) *peak_admitted_bytes = w->peak_pub.load();
    return AGILE_OK;
}

void agile_worker_destroy(agile_worker_t *w) {
    if (w == nullptr) return;
    w->stop.store(true);
    if (w->th.joinable()) w->th.join();
    for (Slot &s : w->slots) {
        if (s.stream) cudaStreamSynchronize(s.stream);
        if (s.done) cudaEventDestroy(s.done);
        if (s.stream) cudaStreamDestroy(s.stream);
        if (s.staging) cudaFreeHost(s.staging);
        if (s.notice) cudaFreeHost(s.notice);
    }
    delete w;
}

}  // extern "C"
