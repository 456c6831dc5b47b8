// pm_server.cu -- request loop with continuous batching on one GPU, built on
// the library's batched C ABI (pmp_hash_batch32/64). Host code only.
//
// A scheduler thread owns K stream slots and one device arena (allocated once
// at creation; the budget). Requests (packed strings in host memory, one
// width each) wait in FIFO order; the head request is admitted as soon as a
// slot is idle and its device memory fits in the arena, so requests that
// arrive while others are running join at once and their work overlaps on
// the device. An admitted request is copied in, hashed by the batched
// kernels, and its results copied back on the slot's stream; an event marks
// the results visible on the host, when the memory and the slot are freed.
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/pmplus.h"

namespace {

uint64_t now_ns() {
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// First-fit allocator over one device range, coalescing on free.
class Arena {
  public:
    void init(uint8_t *base, size_t bytes) {
        base_ = base;
        free_.clear();
        free_[0] = bytes;
    }
    // offset of a block of `bytes`, or SIZE_MAX
    size_t alloc(size_t bytes) {
        bytes = round_up(bytes ? bytes : 1, 256);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                const size_t off = it->first, left = it->second - bytes;
                free_.erase(it);
                if (left) free_[off + bytes] = left;
                used_[off] = bytes;
                return off;
            }
        }
        return SIZE_MAX;
    }
    void release(size_t off) {
        auto u = used_.find(off);
        if (u == used_.end()) return;
        size_t start = off, size = u->second;
        used_.erase(u);
        auto next = free_.lower_bound(start);
        if (next != free_.end() && start + size == next->first) {
            size += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == start) {
                start = prev->first;
                size += prev->second;
                free_.erase(prev);
            }
        }
        free_[start] = size;
    }
    uint8_t *ptr(size_t off) const { return base_ + off; }

  private:
    uint8_t *base_ = nullptr;
    std::map<size_t, size_t> free_;
    std::map<size_t, size_t> used_;
};

struct Request {
    uint64_t ticket;
    int width;
    const uint8_t *host_base;
    const int64_t *host_offsets;
    int64_t n;
    void *host_out;
    uint64_t submit_ns;
};

struct Ticket {
    int state = 0;  // 0 queued, 1 running, 2 done, 3 failed
    int status = PMP_OK;
    uint64_t submit_ns = 0, start_ns = 0, done_ns = 0;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    uint64_t ticket = 0;
    size_t block = SIZE_MAX;
};

}  // namespace

struct pmp_server {
    const pmp_key *key[2];  // [width == 64]
    int device = 0;
    uint8_t *arena_mem = nullptr;
    Arena arena;
    std::vector<Slot> slots;
    std::deque<Request> queue;
    std::unordered_map<uint64_t, Ticket> tickets;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread thread;
    std::atomic<bool> stop{false};
    uint64_t next_ticket = 1;
    int running = 0;
    size_t budget = 0;

    // Device bytes of a request: packed bytes (to align16 of the end),
    // offsets, outputs, scratch.
    static size_t need(const Request &r) {
        const int64_t end = r.n ? r.host_offsets[r.n] : 0;
        return round_up((size_t)((end + 15) & ~(int64_t)15), 256) +
               round_up(sizeof(int64_t) * (size_t)(r.n + 1), 256) +
               round_up((size_t)r.n * (r.width / 8), 256) +
               pmp_batch_scratch_bytes(r.width, r.n, (uint64_t)(end > 0 ? end : 0));
    }

    int launch(Slot &s, const Request &r, size_t block) {
        uint8_t *p = arena.ptr(block);
        const int64_t end = r.n ? r.host_offsets[r.n] : 0;
        const size_t data_bytes = round_up((size_t)((end + 15) & ~(int64_t)15), 256);
        const size_t off_bytes = round_up(sizeof(int64_t) * (size_t)(r.n + 1), 256);
        const size_t out_bytes = round_up((size_t)r.n * (r.width / 8), 256);
        uint8_t *d_base = p;
        int64_t *d_off = reinterpret_cast<int64_t *>(p + data_bytes);
        uint8_t *d_out = p + data_bytes + off_bytes;
        uint8_t *d_scr = d_out + out_bytes;
        const size_t scr_bytes = pmp_batch_scratch_bytes(r.width, r.n, (uint64_t)(end > 0 ? end : 0));
        if (end > 0 && cudaMemcpyAsync(d_base, r.host_base, (size_t)end, cudaMemcpyHostToDevice,
                                       s.stream) != cudaSuccess)
            return PMP_ECUDA;
        if (cudaMemcpyAsync(d_off, r.host_offsets, sizeof(int64_t) * (size_t)(r.n + 1),
                            cudaMemcpyHostToDevice, s.stream) != cudaSuccess)
            return PMP_ECUDA;
        int rc = r.width == 32
                     ? pmp_hash_batch32(key[0], d_base, d_off, r.n, reinterpret_cast<uint32_t *>(d_out),
                                        d_scr, scr_bytes, s.stream)
                     : pmp_hash_batch64(key[1], d_base, d_off, r.n, reinterpret_cast<uint64_t *>(d_out),
                                        d_scr, scr_bytes, s.stream);
        if (rc) return rc;
        if (r.n && cudaMemcpyAsync(r.host_out, d_out, (size_t)r.n * (r.width / 8),
                                   cudaMemcpyDeviceToHost, s.stream) != cudaSuccess)
            return PMP_ECUDA;
        if (cudaEventRecord(s.done, s.stream) != cudaSuccess) return PMP_ECUDA;
        return PMP_OK;
    }

    void loop() {
        cudaSetDevice(device);
        std::unique_lock<std::mutex> lk(mu);
        while (!stop.load()) {
            bool progressed = false;
            // retire finished slots
            for (Slot &s : slots) {
                if (!s.busy) continue;
                const cudaError_t q = cudaEventQuery(s.done);
                if (q == cudaErrorNotReady) continue;
                Ticket &t = tickets[s.ticket];
                t.done_ns = now_ns();
                t.state = q == cudaSuccess ? 2 : 3;
                if (q != cudaSuccess) t.status = PMP_ECUDA;
                arena.release(s.block);
                s.busy = false;
                --running;
                progressed = true;
                cv_done.notify_all();
            }
            // admit the head of the queue while a slot and memory are free
            while (!queue.empty()) {
                Slot *free_slot = nullptr;
                for (Slot &s : slots)
                    if (!s.busy) {
                        free_slot = &s;
                        break;
                    }
                if (!free_slot) break;
                const Request r = queue.front();
                const size_t block = arena.alloc(need(r));
                if (block == SIZE_MAX) break;  // wait for memory to free up
                queue.pop_front();
                Ticket &t = tickets[r.ticket];
                t.state = 1;
                t.start_ns = now_ns();
                const int rc = launch(*free_slot, r, block);
                if (rc != PMP_OK) {
                    t.state = 3;
                    t.status = rc;
                    t.done_ns = now_ns();
                    arena.release(block);
                    cv_done.notify_all();
                    continue;
                }
                free_slot->busy = true;
                free_slot->ticket = r.ticket;
                free_slot->block = block;
                ++running;
                progressed = true;
            }
            if (!progressed) {
                if (running == 0)
                    cv_work.wait(lk, [&] { return stop.load() || !queue.empty(); });
                else {
                    lk.unlock();
                    std::this_thread::sleep_for(std::chrono::microseconds(5));
                    lk.lock();
                }
            }
        }
    }
};

extern "C" {

int pmp_server_create(const pmp_key *key32, const pmp_key *key64, size_t budget_bytes, int slots,
                      pmp_server **out) {
    if (!out || !key32 || !key64 || pmp_key_width(key32) != 32 || pmp_key_width(key64) != 64 ||
        slots < 1 || slots > 64 || budget_bytes < 4096)
        return PMP_EINVAL;
    *out = nullptr;
    pmp_server *s = new pmp_server;
    s->key[0] = key32;
    s->key[1] = key64;
    cudaGetDevice(&s->device);
    if (cudaMalloc(&s->arena_mem, budget_bytes) != cudaSuccess) {
        (void)cudaGetLastError();
        delete s;
        return PMP_ENOMEM;
    }
    s->arena.init(s->arena_mem, budget_bytes);
    s->budget = budget_bytes;
    s->slots.resize((size_t)slots);
    for (Slot &sl : s->slots) {
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess) {
            pmp_server_destroy(s);
            return PMP_ECUDA;
        }
    }
    s->thread = std::thread([s] { s->loop(); });
    *out = s;
    return PMP_OK;
}

int pmp_server_submit(pmp_server *s, int width, const uint8_t *host_base, const int64_t *host_offsets,
                      int64_t n, void *host_out, uint64_t *ticket) {
    if (!s || !ticket || (width != 32 && width != 64) || n < 0 || !host_offsets ||
        (n > 0 && (!host_out || !host_base)))
        return PMP_EINVAL;
    Request r{0, width, host_base, host_offsets, n, host_out, now_ns()};
    if (pmp_server::need(r) > s->budget) return PMP_ENOMEM;  // can never be admitted
    {
        std::lock_guard<std::mutex> lk(s->mu);
        r.ticket = s->next_ticket++;
        Ticket &t = s->tickets[r.ticket];
        t.submit_ns = r.submit_ns;
        s->queue.push_back(r);
    }
    s->cv_work.notify_one();
    *ticket = r.ticket;
    return PMP_OK;
}

int pmp_server_wait(pmp_server *s, uint64_t ticket, double timeout_s, int *done) {
    if (!s || !done) return PMP_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return PMP_EINVAL;
    const auto deadline = std::chrono::steady_clock::now() +
                          std::chrono::nanoseconds((int64_t)(timeout_s * 1e9));
    s->cv_done.wait_until(lk, deadline, [&] { return it->second.state >= 2; });
    *done = it->second.state >= 2;
    return it->second.state == 3 ? it->second.status : PMP_OK;
}

int pmp_server_ticket_times(pmp_server *s, uint64_t ticket, uint64_t *submit_ns, uint64_t *start_ns,
                            uint64_t *done_ns) {
    if (!s) return PMP_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return PMP_EINVAL;
    if (submit_ns) *submit_ns = it->second.submit_ns;
    if (start_ns) *start_ns = it->second.start_ns;
    if (done_ns) *done_ns = it->second.done_ns;
    return it->second.state == 3 ? it->second.status : PMP_OK;
}

int pmp_server_release(pmp_server *s, uint64_t ticket) {
    if (!s) return PMP_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end() || it->second.state < 2) return PMP_EINVAL;
    s->tickets.erase(it);
    return PMP_OK;
}

void pmp_server_destroy(pmp_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop.store(true);
    }
    s->cv_work.notify_all();
    if (s->thread.joinable()) s->thread.join();
    for (Slot &sl : s->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    if (s->arena_mem) cudaFree(s->arena_mem);
    delete s;
}

}  // extern "C"
