// Request loop: continuous batching of parse requests on one GPU, in the
// library (a worker thread), so that admission, launch and retirement cost
// no interpreter time per request.
//
// A server owns `slots`; each has a CUDA stream, a device arena and two
// pinned staging buffers (texts in, columns and status words out), allocated
// once.  The worker thread loops: it retires slots whose completion event has
// fired (copying each request's columns and status to the caller's buffers
// and marking its ticket done), then admits waiting requests into the free
// slots.  While no more requests wait than slots are free, each runs alone
// as soon as it arrives; beyond that a free slot takes as many as fit, so
// batches grow with the load; a request joins a slot's batch only while the batch's
// device footprint (texts, columns, workspace, descriptors) fits the arena.
// One request runs as re_parse, several as one re_parse_batch.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_set>
#include <vector>

#include "kernels.cuh"
#include "re_internal.h"

#define CUDA_TRY_SRV(expr)                                                              \
    do {                                                                                \
        const cudaError_t e_ = (expr);                                                  \
        if (e_ != cudaSuccess) {                                                        \
            slpf::set_error(std::string("server set-up: ") + cudaGetErrorString(e_));   \
            return RE_E_CUDA;                                                           \
        }                                                                               \
    } while (0)

namespace slpf {
namespace {

size_t al256(size_t v) { return (v + 255) & ~(size_t)255; }

struct Req {
    uint64_t ticket;
    uint32_t re;
    const uint8_t *text;
    uint64_t len;
    void *cols;
    uint64_t cap;
    int32_t *status;
    size_t dev_bytes, cols_bytes;     // footprint in the arena; column bytes
};

// Copies between the callers' host buffers and the pinned staging buffers,
// spread over a few threads when they are large (one core copies about 10
// GB/s; a loaded server moves texts in and twice as many column bytes out).
class CopyPool {
   public:
    struct Task {
        void *dst;
        const void *src;
        size_t bytes;
    };
    explicit CopyPool(unsigned n) {
        for (unsigned j = 0; j < n; ++j) threads_.emplace_back([this] { loop(); });
    }
    ~CopyPool() {
        {
            std::lock_guard<std::mutex> g(m_);
            stop_ = true;
        }
        cv_.notify_all();
        for (std::thread &t : threads_) t.join();
    }
    // Copy every task; returns when all are done.  Small jobs stay on the caller.
    void run(std::vector<Task> &tasks) {
        size_t total = 0;
        for (const Task &t : tasks) total += t.bytes;
        if (threads_.empty() || total < (4u << 20)) {
            for (const Task &t : tasks) std::memcpy(t.dst, t.src, t.bytes);
            return;
        }
        // cut into pieces of at most 1 MiB so the threads share the work evenly
        std::vector<Task> pieces;
        for (const Task &t : tasks)
            for (size_t o = 0; o < t.bytes; o += (1u << 20))
                pieces.push_back({static_cast<uint8_t *>(t.dst) + o, static_cast<const uint8_t *>(t.src) + o,
                                  std::min<size_t>(1u << 20, t.bytes - o)});
        {
            std::lock_guard<std::mutex> g(m_);                  // a late thread of the last job reads under the lock
            pieces_.swap(pieces);
            next_ = 0;
            left_ = pieces_.size();
            ++job_;
        }
        cv_.notify_all();
        work();                                                   // the caller copies too
        std::unique_lock<std::mutex> lk(m_);
        done_.wait(lk, [&] { return left_ == 0; });
    }

   private:
    void work() {
        for (;;) {
            Task t;
            {
                std::lock_guard<std::mutex> g(m_);
                if (next_ >= pieces_.size()) return;
                t = pieces_[next_++];
            }
            std::memcpy(t.dst, t.src, t.bytes);
            std::lock_guard<std::mutex> g(m_);
            if (--left_ == 0) done_.notify_all();
        }
    }
    void loop() {
        uint64_t seen = 0;
        for (;;) {
            {
                std::unique_lock<std::mutex> lk(m_);
                cv_.wait(lk, [&] { return stop_ || job_ != seen; });
                if (stop_) return;
                seen = job_;
            }
            work();
        }
    }
    std::vector<std::thread> threads_;
    std::vector<Task> pieces_;
    std::mutex m_;
    std::condition_variable cv_, done_;
    size_t next_ = 0, left_ = 0;
    uint64_t job_ = 0;
    bool stop_ = false;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t event = nullptr;
    uint8_t *arena = nullptr, *pin_in = nullptr, *pin_out = nullptr;
    std::vector<Req> reqs;
    std::vector<size_t> out_off;      // per request: columns' offset in pin_out
    size_t status_off = 0;
    re_batch *batch = nullptr;
    bool busy = false;
};

}  // namespace
}  // namespace slpf

using namespace slpf;

struct re_server {
    std::vector<re_handle *> hs;
    std::vector<re_slpf_kind> kind;
    std::vector<uint32_t> cb;
    std::vector<Slot> slots;
    uint64_t arena = 0, staging = 0;
    uint32_t max_batch = 4096;
    int device = 0;
    std::mutex m;
    std::condition_variable cv_work, cv_done;
    std::deque<Req> waiting;
    std::vector<uint64_t> finished;             // completed since the last re_server_poll
    std::vector<uint64_t> finished_ns;          // their completion times on the server clock
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
    uint64_t next_ticket = 1;
    std::unordered_set<uint64_t> pending;       // submitted, not completed
    bool stop = false;
    uint64_t stats[4] = {0, 0, 0, 0};           // batches, requests, largest batch, most slots in flight
    std::unique_ptr<CopyPool> copies;           // used by the worker thread only
    std::thread worker;
    ~re_server() {
        for (Slot &s : slots) {
            if (s.batch) re_batch_free(s.batch);
            if (s.event) cudaEventDestroy(s.event);
            if (s.stream) cudaStreamDestroy(s.stream);
            if (s.arena) cudaFree(s.arena);
            if (s.pin_in) cudaFreeHost(s.pin_in);
            if (s.pin_out) cudaFreeHost(s.pin_out);
        }
    }
};

namespace slpf {
namespace {

// Bytes a request needs in a slot's arena: text, columns, workspace (its own
// re_workspace_size with the batch rule's shortest chunk) and descriptors.
size_t dev_footprint(re_server *S, uint32_t re, uint64_t len) {
    uint64_t ws = 0;
    re_parse_opts o{};
    o.chunk_len = 256;                                         // the shortest chunk a batch picks
    if (len && re_workspace_size(S->hs[re], len, &o, &ws) != RE_OK) ws = 0;
    uint64_t ws_auto = 0;
    if (len) re_workspace_size(S->hs[re], len, nullptr, &ws_auto);
    ws = std::max(ws, ws_auto);
    return al256(len) + al256((len + 1) * S->cb[re]) + al256(ws) + 2048;
}

// Launch the admitted requests of slot s.  Returns false (and marks every
// request's status) when the library refuses the launch.
bool launch(re_server *S, Slot &s) {
    const size_t n = s.reqs.size();
    std::vector<size_t> t_off(n), c_off(n);
    size_t o = 0;
    for (size_t j = 0; j < n; ++j) { t_off[j] = o; o += al256(s.reqs[j].len); }
    const size_t text_end = o;
    for (size_t j = 0; j < n; ++j) { c_off[j] = o; o += al256(s.reqs[j].cols_bytes); }
    s.status_off = o;
    o += al256(4 * n);
    const size_t out_end = o, ws_off = o;
    std::vector<CopyPool::Task> tasks(n);
    for (size_t j = 0; j < n; ++j) tasks[j] = {s.pin_in + t_off[j], s.reqs[j].text, s.reqs[j].len};
    S->copies->run(tasks);
    re_status st = RE_OK;
    cudaStream_t str = s.stream;
    if (text_end) st = cudaMemcpyAsync(s.arena, s.pin_in, text_end, cudaMemcpyHostToDevice, str) == cudaSuccess
                           ? RE_OK : RE_E_CUDA;
    if (st == RE_OK && n == 1) {
        const Req &r = s.reqs[0];
        re_slpf out{S->kind[r.re], S->cb[r.re], 0, s.arena + c_off[0], r.cols_bytes,
                    reinterpret_cast<int32_t *>(s.arena + s.status_off)};
        st = re_parse(S->hs[r.re], r.len ? s.arena + t_off[0] : nullptr, r.len, (re_stream)str, &out,
                      s.arena + ws_off, S->arena - ws_off, nullptr);
    } else if (st == RE_OK) {
        std::vector<re_handle *> hs(n);
        std::vector<uint64_t> lens(n);
        for (size_t j = 0; j < n; ++j) { hs[j] = S->hs[s.reqs[j].re]; lens[j] = s.reqs[j].len; }
        st = re_batch_plan(hs.data(), lens.data(), (uint32_t)n, nullptr, &s.batch);
        uint64_t ws = 0;
        if (st == RE_OK) st = re_batch_workspace_size(s.batch, &ws);
        if (st == RE_OK && ws_off + ws > S->arena) st = RE_E_CAPACITY;
        if (st == RE_OK) {
            std::vector<const uint8_t *> texts(n);
            std::vector<re_slpf> outs(n);
            for (size_t j = 0; j < n; ++j) {
                const Req &r = s.reqs[j];
                texts[j] = r.len ? s.arena + t_off[j] : nullptr;
                outs[j] = re_slpf{S->kind[r.re], S->cb[r.re], 0, s.arena + c_off[j], r.cols_bytes,
                                  reinterpret_cast<int32_t *>(s.arena + s.status_off) + j};
            }
            st = re_parse_batch(s.batch, texts.data(), outs.data(), s.arena + ws_off, ws, (re_stream)str);
        }
    }
    if (st == RE_OK && cudaMemcpyAsync(s.pin_out, s.arena + text_end, out_end - text_end, cudaMemcpyDeviceToHost,
                                       str) != cudaSuccess)
        st = RE_E_CUDA;
    if (st == RE_OK && cudaEventRecord(s.event, str) != cudaSuccess) st = RE_E_CUDA;
    s.out_off.assign(n, 0);
    for (size_t j = 0; j < n; ++j) s.out_off[j] = c_off[j] - text_end;
    s.status_off -= text_end;
    if (st != RE_OK) {
        for (Req &r : s.reqs) *r.status = st;
        return false;
    }
    return true;
}

// Copy a finished slot's results to the callers and report its tickets.
void retire(re_server *S, Slot &s, bool ok, std::vector<uint64_t> &tickets) {
    const int32_t *status = reinterpret_cast<const int32_t *>(s.pin_out + s.status_off);
    if (ok) {
        std::vector<CopyPool::Task> tasks(s.reqs.size());
        for (size_t j = 0; j < s.reqs.size(); ++j) tasks[j] = {s.reqs[j].cols, s.pin_out + s.out_off[j], s.reqs[j].cols_bytes};
        S->copies->run(tasks);
    }
    for (size_t j = 0; j < s.reqs.size(); ++j) {
        Req &r = s.reqs[j];
        if (ok) *r.status = status[j];
        tickets.push_back(r.ticket);
    }
    if (s.batch) { re_batch_free(s.batch); s.batch = nullptr; }
    s.reqs.clear();
    s.busy = false;
}

void worker_loop(re_server *S) {
    cudaSetDevice(S->device);
    std::vector<uint64_t> tickets;
    for (;;) {
        bool idle = true;
        for (Slot &s : S->slots) {                              // retire
            if (!s.busy) continue;
            const cudaError_t q = cudaEventQuery(s.event);
            if (q == cudaErrorNotReady) continue;
            retire(S, s, q == cudaSuccess, tickets);
            idle = false;
        }
        std::unique_lock<std::mutex> lk(S->m);
        if (!tickets.empty()) {
            const uint64_t now = (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
                                     std::chrono::steady_clock::now() - S->t0).count();
            for (uint64_t t : tickets) {
                S->pending.erase(t);
                S->finished.push_back(t);
                S->finished_ns.push_back(now);
            }
            tickets.clear();
            S->cv_done.notify_all();
        }
        size_t free = 0, busy = 0;
        for (Slot &s : S->slots) (s.busy ? busy : free)++;
        for (Slot &s : S->slots) {                              // admit
            if (s.busy || S->waiting.empty()) continue;
            // light load (no more waiting requests than free slots): a slot per
            // request at once; otherwise this slot takes all it can
            const size_t share = S->waiting.size() <= free ? 1 : S->max_batch;
            --free;
            size_t dev = 1 << 20, in = 0, out = 4096;
            while (!S->waiting.empty() && s.reqs.size() < std::min<size_t>(S->max_batch, share)) {
                const Req &r = S->waiting.front();
                if (!s.reqs.empty() && (dev + r.dev_bytes > S->arena || in + al256(r.len) > S->staging ||
                                        out + al256(r.cols_bytes) + 4 > S->staging))
                    break;
                dev += r.dev_bytes; in += al256(r.len); out += al256(r.cols_bytes) + 4;
                s.reqs.push_back(r);
                S->waiting.pop_front();
            }
            s.busy = true;
            ++busy;
            S->stats[0] += 1;
            S->stats[1] += s.reqs.size();
            S->stats[2] = std::max<uint64_t>(S->stats[2], s.reqs.size());
            S->stats[3] = std::max<uint64_t>(S->stats[3], busy);
            lk.unlock();
            if (!launch(S, s)) {                                // refused: let what it enqueued finish first
                cudaStreamSynchronize(s.stream);
                retire(S, s, false, tickets);
            }
            lk.lock();
            idle = false;
        }
        if (S->stop && S->waiting.empty() && busy == 0 && tickets.empty()) return;
        if (idle) {
            if (busy) {                                         // a slot on the GPU: poll its event soon
                lk.unlock();
                std::this_thread::sleep_for(std::chrono::microseconds(5));
            } else {                                            // nothing in flight: sleep until a submission
                S->cv_work.wait_for(lk, std::chrono::milliseconds(50),
                                    [&] { return S->stop || !S->waiting.empty(); });
            }
        }
    }
}

}  // namespace
}  // namespace slpf

extern "C" {

re_status re_server_create(re_handle *const *hs, uint32_t count, const re_server_opts *opts, re_server **out) {
    if (!out || !count || !hs) { set_error("null argument"); return RE_E_INVALID_ARG; }
    *out = nullptr;
    for (uint32_t j = 0; j < count; ++j)
        if (!hs[j] || hs[j]->host_only) { set_error("null or host-only handle"); return RE_E_INVALID_ARG; }
    std::unique_ptr<re_server> S(new (std::nothrow) re_server());
    if (!S) { set_error("host allocation failed"); return RE_E_NOMEM; }
    CUDA_TRY_SRV(cudaGetDevice(&S->device));
    for (uint32_t j = 0; j < count; ++j) {
        if (hs[j]->device != S->device) { set_error("a handle lives on another device"); return RE_E_INVALID_ARG; }
        re_slpf_kind k;
        uint32_t cb;
        uint64_t bytes;
        const re_status st = re_slpf_layout(hs[j], 1, RE_SLPF_AUTO, &k, &cb, &bytes);
        if (st != RE_OK) return st;
        S->hs.push_back(hs[j]);
        S->kind.push_back(k);
        S->cb.push_back(cb);
    }
    const uint32_t nslots = opts && opts->slots ? opts->slots : 4;
    S->arena = opts && opts->arena_bytes ? opts->arena_bytes : (1ull << 30);
    S->staging = opts && opts->staging_bytes ? opts->staging_bytes : S->arena / 2;
    S->max_batch = opts && opts->max_batch ? opts->max_batch : 4096;
    S->slots.resize(nslots);
    for (Slot &s : S->slots) {
        CUDA_TRY_SRV(cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking));
        CUDA_TRY_SRV(cudaEventCreateWithFlags(&s.event, cudaEventDisableTiming));
        CUDA_TRY_SRV(cudaMalloc((void **)&s.arena, S->arena));
        CUDA_TRY_SRV(cudaHostAlloc((void **)&s.pin_in, S->staging, cudaHostAllocDefault));
        CUDA_TRY_SRV(cudaHostAlloc((void **)&s.pin_out, S->staging, cudaHostAllocDefault));
    }
    re_server *raw = S.get();
    try {
        S->copies.reset(new CopyPool(7));                         // with the worker: 8 copying threads
        S->worker = std::thread(worker_loop, raw);
    } catch (...) {
        set_error("cannot start the server thread");
        return RE_E_NOMEM;
    }
    *out = S.release();
    return RE_OK;
}

re_status re_server_submit(re_server *S, uint32_t re_index, const uint8_t *text, uint64_t len, void *cols,
                           uint64_t cols_cap, int32_t *status, uint64_t *ticket) {
    if (!S || !ticket || !status || !cols || (len && !text)) { set_error("null argument"); return RE_E_INVALID_ARG; }
    if (re_index >= S->hs.size()) { set_error("RE index out of range"); return RE_E_INVALID_ARG; }
    Req r{};
    r.re = re_index;
    r.text = text;
    r.len = len;
    r.cols = cols;
    r.cap = cols_cap;
    r.status = status;
    r.cols_bytes = (len + 1) * S->cb[re_index];
    if (cols_cap < r.cols_bytes) { set_error("column buffer too small"); return RE_E_CAPACITY; }
    r.dev_bytes = dev_footprint(S, re_index, len);
    if (r.dev_bytes + (1u << 20) > S->arena || al256(len) > S->staging || al256(r.cols_bytes) + 4096 > S->staging) {
        set_error("request larger than a slot's arena or staging buffers");
        return RE_E_CAPACITY;
    }
    {
        std::lock_guard<std::mutex> g(S->m);
        if (S->stop) { set_error("server is shutting down"); return RE_E_INVALID_ARG; }
        r.ticket = S->next_ticket++;
        S->pending.insert(r.ticket);
        S->waiting.push_back(r);
    }
    S->cv_work.notify_one();
    *ticket = r.ticket;
    return RE_OK;
}

re_status re_server_wait(re_server *S, uint64_t ticket, int32_t timeout_ms) {
    if (!S) { set_error("null argument"); return RE_E_INVALID_ARG; }
    std::unique_lock<std::mutex> lk(S->m);
    if (ticket == 0 || ticket >= S->next_ticket) { set_error("unknown ticket"); return RE_E_INVALID_ARG; }
    auto ready = [&] { return !S->pending.count(ticket); };
    if (timeout_ms < 0) S->cv_done.wait(lk, ready);
    else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) return RE_E_TIMEOUT;
    return RE_OK;
}

re_status re_server_poll(re_server *S, uint64_t *tickets, uint64_t *done_ns, uint32_t cap, uint32_t *n) {
    if (!S || !n || (cap && !tickets)) { set_error("null argument"); return RE_E_INVALID_ARG; }
    std::lock_guard<std::mutex> g(S->m);
    const uint32_t k = (uint32_t)std::min<size_t>(cap, S->finished.size());
    for (uint32_t j = 0; j < k; ++j) {
        tickets[j] = S->finished[j];
        if (done_ns) done_ns[j] = S->finished_ns[j];
    }
    S->finished.erase(S->finished.begin(), S->finished.begin() + k);
    S->finished_ns.erase(S->finished_ns.begin(), S->finished_ns.begin() + k);
    *n = k;
    return RE_OK;
}

uint64_t re_server_clock_ns(const re_server *S) {
    if (!S) return 0;
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now() - S->t0)
        .count();
}

re_status re_server_stats(re_server *S, uint64_t *stats) {
    if (!S || !stats) { set_error("null argument"); return RE_E_INVALID_ARG; }
    std::lock_guard<std::mutex> g(S->m);
    for (int j = 0; j < 4; ++j) stats[j] = S->stats[j];
    return RE_OK;
}

void re_server_destroy(re_server *S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> g(S->m);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->worker.joinable()) S->worker.join();
    delete S;
}

}  // extern "C"
