// pm_server.cu -- request loop with continuous batching on one GPU, built on
// the library's C ABI (pmp_hash_batch_status, pmp_stream_*). Host code only.
//
// A scheduler thread owns K stream slots and one device arena (allocated once
// at creation; the budget). Requests wait in FIFO order; the head request is
// admitted as soon as a slot is idle and its device memory fits in the
// arena, so requests that arrive while others are running join at once and
// their work overlaps on the device. A request is either a packed batch of
// strings (copied in, hashed by the batched kernels, results copied back) or
// a piece of a string held by the server (a pmp_stream whose tree state
// stays on the device between requests: the piece is copied in and appended,
// and the last piece also yields the hash). The scheduler decides under its
// lock and issues the copies and launches without it; an event on the slot's
// stream marks the results visible on the host, and only then are the slot
// and the memory freed and the request's status (its own device status word
// for batches) reported on its ticket.
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
    int kind;  // 0: batch, 1: piece of a server stream
    int width;
    const uint8_t *host_base;     // batch bytes, or the piece
    const int64_t *host_offsets;  // batch only
    int64_t n;                    // strings (batch) or piece bytes
    void *host_out;               // n results (batch), one result after the last piece
    uint64_t stream_id;           // piece only
    int final;                    // piece only: the string ends with this piece
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
    int *h_status = nullptr;  // pinned: the device status word of the slot's batch
    bool busy = false;
    bool issued = false;      // the launch has returned (its work is queued)
    int fail = PMP_OK;        // error returned while issuing the request
    uint64_t ticket = 0;
    size_t block = SIZE_MAX;
};

// A string hashed from pieces that arrive in separate requests.
struct ServerStream {
    pmp_stream *ps = nullptr;
    cudaEvent_t last = nullptr;  // recorded after the last piece's work
    bool has_last = false;
    int width = 0;
    int pending = 0;             // pieces queued or running
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
    std::unordered_map<uint64_t, ServerStream> streams;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread thread;
    std::atomic<bool> stop{false};
    uint64_t next_ticket = 1, next_stream = 1;
    int running = 0;
    size_t budget = 0;

    // Device bytes of a request: batch: packed bytes (to align16 of the end),
    // offsets, outputs, status word, scratch; piece: its bytes and a result.
    static size_t need(const Request &r) {
        if (r.kind == 1) return round_up((size_t)r.n, 256) + 256;
        const int64_t end = r.n ? r.host_offsets[r.n] : 0;
        return round_up((size_t)((end + 15) & ~(int64_t)15), 256) +
               round_up(sizeof(int64_t) * (size_t)(r.n + 1), 256) +
               round_up((size_t)r.n * (r.width / 8), 256) + 256 +
               pmp_batch_scratch_bytes(r.width, r.n, (uint64_t)(end > 0 ? end : 0));
    }

    // Queue a batch request's work on the slot's stream (no lock held).
    int launch_batch(Slot &s, const Request &r, size_t block) {
        uint8_t *p = arena.ptr(block);
        const int64_t end = r.n ? r.host_offsets[r.n] : 0;
        const size_t data_bytes = round_up((size_t)((end + 15) & ~(int64_t)15), 256);
        const size_t off_bytes = round_up(sizeof(int64_t) * (size_t)(r.n + 1), 256);
        const size_t out_bytes = round_up((size_t)r.n * (r.width / 8), 256);
        uint8_t *d_base = p;
        int64_t *d_off = reinterpret_cast<int64_t *>(p + data_bytes);
        uint8_t *d_out = p + data_bytes + off_bytes;
        int *d_status = reinterpret_cast<int *>(d_out + out_bytes);
        uint8_t *d_scr = d_out + out_bytes + 256;
        const size_t scr_bytes = pmp_batch_scratch_bytes(r.width, r.n, (uint64_t)(end > 0 ? end : 0));
        if (cudaMemsetAsync(d_status, 0, sizeof(int), s.stream) != cudaSuccess) return PMP_ECUDA;
        if (end > 0 && cudaMemcpyAsync(d_base, r.host_base, (size_t)end, cudaMemcpyHostToDevice,
                                       s.stream) != cudaSuccess)
            return PMP_ECUDA;
        if (cudaMemcpyAsync(d_off, r.host_offsets, sizeof(int64_t) * (size_t)(r.n + 1),
                            cudaMemcpyHostToDevice, s.stream) != cudaSuccess)
            return PMP_ECUDA;
        const int rc = pmp_hash_batch_status(key[r.width == 64], d_base, d_off, r.n, d_out, d_status, d_scr,
                                             scr_bytes, s.stream);
        if (rc) return rc;
        if (r.n && cudaMemcpyAsync(r.host_out, d_out, (size_t)r.n * (r.width / 8),
                                   cudaMemcpyDeviceToHost, s.stream) != cudaSuccess)
            return PMP_ECUDA;
        if (cudaMemcpyAsync(s.h_status, d_status, sizeof(int), cudaMemcpyDeviceToHost, s.stream) != cudaSuccess)
            return PMP_ECUDA;
        return PMP_OK;
    }

    // Queue a piece of a server stream on the slot's stream (no lock held;
    // only the scheduler thread touches st.ps between open and close). The
    // piece waits for the previous piece of the same string, whichever slot
    // ran it, so the string's tree state is updated in submission order.
    int launch_piece(Slot &s, const Request &r, size_t block, ServerStream &st) {
        uint8_t *d_piece = arena.ptr(block);
        uint8_t *d_out = d_piece + round_up((size_t)r.n, 256);
        *s.h_status = PMP_OK;
        if (r.n > 0 && cudaMemcpyAsync(d_piece, r.host_base, (size_t)r.n, cudaMemcpyHostToDevice, s.stream) !=
                           cudaSuccess)
            return PMP_ECUDA;
        if (st.has_last && cudaStreamWaitEvent(s.stream, st.last, 0) != cudaSuccess) return PMP_ECUDA;
        int rc = r.n > 0 ? pmp_stream_update(st.ps, d_piece, (uint64_t)r.n, s.stream) : PMP_OK;
        if (rc) return rc;
        if (r.final) {
            rc = pmp_stream_final(st.ps, d_out, nullptr, s.stream);
            if (rc) return rc;
            if (cudaMemcpyAsync(r.host_out, d_out, (size_t)(st.width / 8), cudaMemcpyDeviceToHost, s.stream) !=
                cudaSuccess)
                return PMP_ECUDA;
        }
        if (cudaEventRecord(st.last, s.stream) != cudaSuccess) return PMP_ECUDA;
        st.has_last = true;
        return PMP_OK;
    }

    void loop() {
        cudaSetDevice(device);
        std::unique_lock<std::mutex> lk(mu);
        while (!stop.load()) {
            bool progressed = false;
            // retire slots whose work has completed (or whose issue failed and
            // whose queued work has completed): memory and slot are freed only now
            for (Slot &s : slots) {
                if (!s.busy || !s.issued) continue;
                const cudaError_t q = cudaEventQuery(s.done);
                if (q == cudaErrorNotReady) continue;
                Ticket &t = tickets[s.ticket];
                t.done_ns = now_ns();
                int status = s.fail;
                if (!status && q != cudaSuccess) status = PMP_ECUDA;
                if (!status) status = *s.h_status;  // the request's own device status word
                t.state = status ? 3 : 2;
                t.status = status;
                arena.release(s.block);
                s.busy = false;
                --running;
                progressed = true;
                cv_done.notify_all();
            }
            // admit the head of the queue while a slot and memory are free
            while (!queue.empty()) {
                Slot *slot = nullptr;
                for (Slot &s : slots)
                    if (!s.busy) {
                        slot = &s;
                        break;
                    }
                if (!slot) break;
                const Request r = queue.front();
                const size_t block = arena.alloc(need(r));
                if (block == SIZE_MAX) break;  // wait for memory to free up
                queue.pop_front();
                Ticket &t = tickets[r.ticket];
                t.state = 1;
                t.start_ns = now_ns();
                slot->busy = true;
                slot->issued = false;
                slot->fail = PMP_OK;
                slot->ticket = r.ticket;
                slot->block = block;
                ++running;
                ServerStream *st = nullptr;
                if (r.kind == 1) st = &streams[r.stream_id];  // kept alive by its pending count
                lk.unlock();  // copies and launches without the lock
                int rc = r.kind == 1 ? launch_piece(*slot, r, block, *st) : launch_batch(*slot, r, block);
                // the retirement waits for everything queued so far, also after an error
                if (cudaEventRecord(slot->done, slot->stream) != cudaSuccess) {
                    cudaStreamSynchronize(slot->stream);
                    (void)cudaGetLastError();
                    cudaEventRecord(slot->done, nullptr);  // on the default stream
                    if (!rc) rc = PMP_ECUDA;
                }
                lk.lock();
                if (st) --st->pending;
                slot->fail = rc;
                slot->issued = true;
                progressed = true;
                cv_done.notify_all();
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
            cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess ||
            cudaHostAlloc(reinterpret_cast<void **>(&sl.h_status), sizeof(int), cudaHostAllocDefault) !=
                cudaSuccess) {
            (void)cudaGetLastError();
            pmp_server_destroy(s);
            return PMP_ECUDA;
        }
        *sl.h_status = PMP_OK;
    }
    s->thread = std::thread([s] { s->loop(); });
    *out = s;
    return PMP_OK;
}

static int server_enqueue(pmp_server *s, Request r, uint64_t *ticket) {
    if (pmp_server::need(r) > s->budget) return PMP_ENOMEM;  // can never be admitted
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (r.kind == 1) {
            auto it = s->streams.find(r.stream_id);
            if (it == s->streams.end()) return PMP_EINVAL;
            ++it->second.pending;
        }
        r.ticket = s->next_ticket++;
        Ticket &t = s->tickets[r.ticket];
        t.submit_ns = r.submit_ns;
        s->queue.push_back(r);
    }
    s->cv_work.notify_one();
    *ticket = r.ticket;
    return PMP_OK;
}

int pmp_server_submit(pmp_server *s, int width, const uint8_t *host_base, const int64_t *host_offsets,
                      int64_t n, void *host_out, uint64_t *ticket) {
    if (!s || !ticket || (width != 32 && width != 64) || n < 0 || !host_offsets ||
        (n > 0 && (!host_out || !host_base)))
        return PMP_EINVAL;
    Request r{0, 0, width, host_base, host_offsets, n, host_out, 0, 0, now_ns()};
    return server_enqueue(s, r, ticket);
}

int pmp_server_stream_open(pmp_server *s, int width, uint64_t *stream_id) {
    if (!s || !stream_id || (width != 32 && width != 64)) return PMP_EINVAL;
    int old = 0;
    cudaGetDevice(&old);
    if (cudaSetDevice(s->device) != cudaSuccess) return PMP_ECUDA;
    ServerStream st;
    st.width = width;
    int rc = pmp_stream_create(s->key[width == 64], &st.ps);
    if (!rc && cudaEventCreateWithFlags(&st.last, cudaEventDisableTiming) != cudaSuccess) {
        (void)cudaGetLastError();
        pmp_stream_destroy(st.ps);
        rc = PMP_ECUDA;
    }
    cudaSetDevice(old);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(s->mu);
    *stream_id = s->next_stream++;
    s->streams[*stream_id] = st;
    return PMP_OK;
}

int pmp_server_submit_piece(pmp_server *s, uint64_t stream_id, const void *host_piece, uint64_t len, int final,
                            void *host_out, uint64_t *ticket) {
    if (!s || !ticket || (len > 0 && !host_piece) || (final && !host_out) || len > (1ull << 62))
        return PMP_EINVAL;
    Request r{0, 1, 0, static_cast<const uint8_t *>(host_piece), nullptr, (int64_t)len, host_out,
              stream_id, final ? 1 : 0, now_ns()};
    return server_enqueue(s, r, ticket);
}

int pmp_server_stream_close(pmp_server *s, uint64_t stream_id) {
    if (!s) return PMP_EINVAL;
    ServerStream st;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        auto it = s->streams.find(stream_id);
        if (it == s->streams.end()) return PMP_EINVAL;
        s->cv_done.wait(lk, [&] { return it->second.pending == 0; });  // every piece issued
        st = it->second;
        s->streams.erase(it);
    }
    int old = 0;
    cudaGetDevice(&old);
    cudaSetDevice(s->device);
    pmp_stream_destroy(st.ps);  // synchronizes the device: the pieces' work is done
    cudaEventDestroy(st.last);
    cudaSetDevice(old);
    return PMP_OK;
}

int pmp_server_wait(pmp_server *s, uint64_t ticket, double timeout_s, int *done) {
    if (!s || !done || !(timeout_s >= 0.0)) return PMP_EINVAL;  // also rejects NaN
    if (timeout_s > 1e9) timeout_s = 1e9;
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
    int old = 0;
    cudaGetDevice(&old);
    cudaSetDevice(s->device);
    for (Slot &sl : s->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
        if (sl.h_status) cudaFreeHost(sl.h_status);
    }
    for (auto &kv : s->streams) {
        pmp_stream_destroy(kv.second.ps);
        cudaEventDestroy(kv.second.last);
    }
    if (s->arena_mem) cudaFree(s->arena_mem);
    cudaSetDevice(old);
    delete s;
}

}  // extern "C"
