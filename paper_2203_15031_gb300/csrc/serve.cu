// Serving context: continuous batching of SPMESL requests on one GPU.
//
// A worker thread owns the GPU side.  Requests are queued by spmesl_submit
// and admitted in arrival order while (a) the bytes of all admitted requests
// stay within the context's memory budget and (b) fewer than max_slots
// requests are admitted.  Every admission round turns the requests admitted
// together into one batch (spmesl_batch_*) with its own stream-ordered
// workspace and runs it on a free stream of the context's pool.  Requests
// that arrive while earlier batches are still running are admitted at once
// into a new batch on another stream, so their work overlaps on the device
// with the batches in flight.  When a batch's completion event fires, its
// workspace and slots are released, each request's status and timings are
// recorded, and waiting requests are admitted into the freed room.
//
// Each request's arithmetic does not depend on what it is batched with (the
// batched kernels run the same per-fit and per-column code as a single fit),
// so a result is the same alone and in the mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "gram_tc.cuh"

namespace {

using Clock = std::chrono::steady_clock;

constexpr int kStreams = 8;              // batches in flight at once
constexpr int kMaxPerBatch = 64;         // requests per admission batch
constexpr size_t kPendingLimitFactor = 8;

struct Pending {
    spmesl_problem prob;
    uint64_t ticket;
    size_t bytes;
    Clock::time_point t_submit;
};

struct Done {
    spmesl_status status;
    float ms_queue;                       // submit -> admitted
    float ms_total;                       // submit -> completion seen
    int32_t batch_size;
};

struct Running {
    spmesl_batch* batch = nullptr;
    void* ws = nullptr;
    size_t bytes = 0;
    int stream = -1;
    cudaEvent_t done = nullptr;
    std::vector<uint64_t> tickets;
    std::vector<Clock::time_point> t_submit;
    Clock::time_point t_admit;
    size_t ws_bytes = 0;
};

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

// Device bytes one request needs inside a batch (per-fit arrays, Gram
// output when X is given, the output stays the caller's).
size_t request_bytes(const spmesl_problem& q, int precision) {
    const size_t s = (size_t)spmesl::elem_size(precision);
    const size_t ldp = (size_t)spmesl::padded_ld(q.p);
    size_t b = 256 + 2 * spmesl::align_up((size_t)q.p * 8, 256) + spmesl::align_up((size_t)q.p * 4, 256) * 2 +
               2 * spmesl::align_up((size_t)q.p * s, 256);
    if (q.X) b += spmesl::align_up((size_t)q.p * q.p * s, 256) + spmesl::align_up((size_t)q.p * s, 256);
    if (q.X && precision == SPMESL_MIXED)    // bf16 operands, tensor-map entry, tile-to-fit slots
        b += spmesl::tc_operand_bytes(q.n, q.p) + sizeof(spmesl::TcFit) +
             4 * (size_t)spmesl::tc_tile_grid(q.p, spmesl::TC_BATCH_BN).count() + 512;
    b += 2 * spmesl::align_up((size_t)q.p * ldp * s, 256);
    b += 4096;                            // share of descriptors and queues
    return b;
}

}  // namespace

struct spmesl_ctx {
    int device = 0;
    size_t budget = 0;
    int max_slots = 0;
    spmesl_opts opts{};
    double tol = 1e-6;
    int maxit = 1000;

    std::mutex mu;
    std::condition_variable cv;
    std::thread worker;
    bool stop = false;
    spmesl_status fatal = SPMESL_OK;

    std::deque<Pending> pending;
    std::vector<Running> running;
    std::unordered_map<uint64_t, Done> done;
    std::unordered_map<uint64_t, int> state;   // 0 queued, 1 running
    uint64_t next_ticket = 1;
    size_t in_use = 0;
    int admitted = 0;
    cudaStream_t streams[kStreams] = {};
    bool stream_busy[kStreams] = {};
    cudaMemPool_t pool = nullptr;

    void loop();
    bool reap_locked(std::unique_lock<std::mutex>& lk);
    bool admit_locked(std::unique_lock<std::mutex>& lk);
};

void spmesl_ctx::loop() {
    cudaSetDevice(device);
    spmesl::g_batch_pageable_staging = true;
    std::unique_lock<std::mutex> lk(mu);
    while (!stop) {
        const bool a = reap_locked(lk);
        const bool b = admit_locked(lk);
        if (!a && !b) {
            // nothing changed: wait for a submit or poll the events again soon
            cv.wait_for(lk, std::chrono::microseconds(running.empty() ? 2000 : 20));
        }
    }
    // drain: let every batch in flight finish before the streams go away
    for (Running& r : running) {
        lk.unlock();
        cudaEventSynchronize(r.done);
        lk.lock();
    }
    reap_locked(lk);
}

bool spmesl_ctx::reap_locked(std::unique_lock<std::mutex>& lk) {
    bool any = false;
    for (size_t i = 0; i < running.size();) {
        Running& r = running[i];
        const cudaError_t q = cudaEventQuery(r.done);
        if (q == cudaErrorNotReady) {
            ++i;
            continue;
        }
        const auto t_done = Clock::now();
        std::vector<int32_t> st(r.tickets.size(), SPMESL_ECUDA);
        if (q == cudaSuccess) {
            lk.unlock();
            spmesl_batch_result(r.batch, r.ws, st.data(), nullptr, streams[r.stream]);
            lk.lock();
        }
        for (size_t k = 0; k < r.tickets.size(); ++k) {
            Done d;
            d.status = (spmesl_status)st[k];
            d.ms_queue = (float)ms_between(r.t_submit[k], r.t_admit);
            d.ms_total = (float)ms_between(r.t_submit[k], t_done);
            d.batch_size = (int32_t)r.tickets.size();
            done[r.tickets[k]] = d;
            state.erase(r.tickets[k]);
        }
        cudaFreeAsync(r.ws, streams[r.stream]);
        spmesl_batch_destroy(r.batch);
        cudaEventDestroy(r.done);
        in_use -= r.bytes;
        admitted -= (int)r.tickets.size();
        stream_busy[r.stream] = false;
        running.erase(running.begin() + i);
        any = true;
    }
    return any;
}

bool spmesl_ctx::admit_locked(std::unique_lock<std::mutex>& lk) {
    if (pending.empty()) return false;
    int s = -1;
    for (int k = 0; k < kStreams; ++k)
        if (!stream_busy[k]) { s = k; break; }
    if (s < 0) return false;
    std::vector<Pending> take;
    size_t bytes = 0;
    while (!pending.empty() && (int)take.size() < kMaxPerBatch && admitted + (int)take.size() < max_slots &&
           in_use + bytes + pending.front().bytes <= budget) {
        bytes += pending.front().bytes;
        take.push_back(pending.front());
        pending.pop_front();
    }
    if (take.empty()) return false;
    Running r;
    r.stream = s;
    r.t_admit = Clock::now();
    std::vector<spmesl_problem> probs;
    for (const Pending& p : take) {
        probs.push_back(p.prob);
        r.tickets.push_back(p.ticket);
        r.t_submit.push_back(p.t_submit);
        state[p.ticket] = 1;
    }
    admitted += (int)take.size();
    stream_busy[s] = true;
    lk.unlock();
    spmesl_status st = spmesl_batch_create(probs.data(), (int)probs.size(), tol, maxit, &opts, &r.batch);
    cudaStream_t cs = streams[s];
    if (st == SPMESL_OK) {
        r.ws_bytes = spmesl_batch_workspace_bytes(r.batch);
        if (cudaMallocFromPoolAsync(&r.ws, r.ws_bytes + 256, pool, cs) != cudaSuccess) st = SPMESL_ENOMEM;
    }
    if (st == SPMESL_OK) {
        // 256-byte alignment of the workspace (the pool returns at least that)
        st = spmesl_batch_run(r.batch, r.ws, r.ws_bytes, cs);
    }
    if (st == SPMESL_OK && cudaEventCreateWithFlags(&r.done, cudaEventDisableTiming) != cudaSuccess)
        st = SPMESL_ECUDA;
    if (st == SPMESL_OK) cudaEventRecord(r.done, cs);
    lk.lock();
    if (st != SPMESL_OK) {
        // the whole group fails with this status; nothing of it is in flight
        for (size_t k = 0; k < take.size(); ++k) {
            done[take[k].ticket] = Done{st, 0.f, (float)ms_between(take[k].t_submit, Clock::now()),
                                        (int32_t)take.size()};
            state.erase(take[k].ticket);
        }
        if (r.ws) cudaFreeAsync(r.ws, cs);
        if (r.batch) spmesl_batch_destroy(r.batch);
        admitted -= (int)take.size();
        stream_busy[s] = false;
        return true;
    }
    r.bytes = bytes;
    in_use += bytes;
    running.push_back(r);
    return true;
}

extern "C" {

spmesl_status spmesl_ctx_create(spmesl_ctx** out, size_t mem_budget_bytes, int max_slots,
                                double tol, int maxit, const spmesl_opts* opts) {
    if (!out || mem_budget_bytes == 0 || max_slots < 1 || !(tol > 0.0) || maxit < 1)
        return SPMESL_EINVAL;
    *out = nullptr;
    spmesl_ctx* c = new (std::nothrow) spmesl_ctx();
    if (!c) return SPMESL_ENOMEM;
    if (opts) c->opts = *opts;
    else spmesl_default_opts(&c->opts);
    if (c->opts.precision != SPMESL_FP32 && c->opts.precision != SPMESL_FP64 &&
        c->opts.precision != SPMESL_MIXED) {
        delete c;
        return SPMESL_EINVAL;
    }
    c->opts.use_graph = 0;
    c->opts.record_phase_times = 0;
    c->budget = mem_budget_bytes;
    c->max_slots = max_slots;
    c->tol = tol;
    c->maxit = maxit;
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        delete c;
        return SPMESL_ECUDA;
    }
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = c->device;
    if (cudaMemPoolCreate(&c->pool, &props) != cudaSuccess) {
        delete c;
        return SPMESL_ECUDA;
    }
    // keep freed memory in the pool (up to the budget) instead of returning it
    unsigned long long keep = mem_budget_bytes;
    cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    for (int k = 0; k < kStreams; ++k) {
        if (cudaStreamCreateWithFlags(&c->streams[k], cudaStreamNonBlocking) != cudaSuccess) {
            for (int m = 0; m < k; ++m) cudaStreamDestroy(c->streams[m]);
            cudaMemPoolDestroy(c->pool);
            delete c;
            return SPMESL_ECUDA;
        }
    }
    c->worker = std::thread([c] { c->loop(); });
    *out = c;
    return SPMESL_OK;
}

spmesl_status spmesl_submit(spmesl_ctx* c, const spmesl_problem* req, uint64_t* ticket) {
    if (!c || !req || !ticket) return SPMESL_EINVAL;
    const spmesl_problem& q = *req;
    if (q.p < 2 || q.p > spmesl_max_p(c->opts.precision) || !q.Theta || !q.sigma ||
        (!q.X && !q.S) || (q.X && q.n < 1))
        return SPMESL_EINVAL;
    const size_t need = request_bytes(q, c->opts.precision);
    if (need > c->budget) return SPMESL_ENOMEM;
    std::lock_guard<std::mutex> lk(c->mu);
    if (c->pending.size() >= kPendingLimitFactor * (size_t)c->max_slots) return SPMESL_EBUSY;
    Pending p;
    p.prob = q;
    p.ticket = c->next_ticket++;
    p.bytes = need;
    p.t_submit = Clock::now();
    c->pending.push_back(p);
    c->state[p.ticket] = 0;
    *ticket = p.ticket;
    c->cv.notify_one();
    return SPMESL_OK;
}

spmesl_status spmesl_poll(spmesl_ctx* c, uint64_t ticket, spmesl_stats* stats) {
    if (!c) return SPMESL_EINVAL;
    std::lock_guard<std::mutex> lk(c->mu);
    auto it = c->done.find(ticket);
    if (it == c->done.end()) return c->state.count(ticket) ? SPMESL_EBUSY : SPMESL_ENOTFOUND;
    const Done d = it->second;
    c->done.erase(it);
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        stats->status = d.status;
        stats->ms_queue = d.ms_queue;
        stats->ms_total = d.ms_total;
        stats->batch_size = d.batch_size;
    }
    return d.status;
}

spmesl_status spmesl_ctx_query(spmesl_ctx* c, int32_t* queued, int32_t* running,
                               size_t* bytes_in_use) {
    if (!c) return SPMESL_EINVAL;
    std::lock_guard<std::mutex> lk(c->mu);
    if (queued) *queued = (int32_t)c->pending.size();
    if (running) *running = c->admitted;
    if (bytes_in_use) *bytes_in_use = c->in_use;
    return SPMESL_OK;
}

void spmesl_ctx_destroy(spmesl_ctx* c) {
    if (!c) return;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        c->stop = true;
        c->cv.notify_one();
    }
    if (c->worker.joinable()) c->worker.join();
    for (int k = 0; k < kStreams; ++k) {
        cudaStreamSynchronize(c->streams[k]);
        cudaStreamDestroy(c->streams[k]);
    }
    cudaMemPoolDestroy(c->pool);
    delete c;
}

}  // extern "C"
