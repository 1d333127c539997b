// Serving loop: requests (one query each) against several device-resident
// models arrive at any time; a worker thread packs the pending requests of a
// model into the slot blocks of that model's next graph launch (continuous
// batching: requests that arrive while a launch is on the GPU go into the
// next one), runs up to two launches per model concurrently on their own
// streams, and completes tickets as launches finish.  Evaluation keys,
// model plaintexts and the graphs' memory stay on the device.  Admission is by
// device memory: at creation every launch's reservation is measured (the high-
// water mark of graph-allocated memory while its graph is replayed once), a
// model gets its second concurrent launch only if free memory still holds
// another such reservation plus the admission floor, and creation fails with
// COPSE_EADMIT if even one launch per model does not fit.  While running, a
// request is admitted only if free device memory is at least the floor (by
// default the largest launch reservation: room for one more launch's working
// set, so memory taken by other work on the device stops admission) and the
// pending queue has room; otherwise COPSE_EADMIT.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket;
    std::vector<uint32_t> feats;
};

struct Ticket {
    int model;
    int state;  // 0 queued, 1 running, 2 done
    std::vector<uint8_t> bits;
    Clock::time_point t_submit, t_done;
};

struct Buffer {
    copse_session *sess = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    uint32_t *h_feats = nullptr;  // pinned [per_ct][nf]
    uint8_t *h_bits = nullptr;    // pinned [per_ct][L]
    uint64_t *h_seed = nullptr;   // pinned
    bool busy = false;
    std::vector<uint64_t> tickets;
};

struct ModelSlot {
    copse_model *m = nullptr;
    size_t per_ct = 0, nf = 0, L = 0;
    uint32_t precision = 0;
    int nbuf = 0;  // launches this model runs concurrently (1 or 2, by device memory)
    Buffer buf[2];
    std::deque<Request> pending;
};

}  // namespace

struct copse_server {
    copse_ctx *c = nullptr;
    std::vector<ModelSlot> models;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::unordered_map<uint64_t, Ticket> tickets;
    std::thread worker;
    bool stop = false;
    size_t max_pending = 0, n_pending = 0;
    size_t reserved = 0;    // device bytes the launches reserved at creation
    size_t launch_max = 0;  // the largest single launch's reservation
    size_t mem_floor = 0;   // free device bytes a submit requires
    uint64_t next_ticket = 1, seed = 0;
    copse_status worker_error = COPSE_OK;
    std::string worker_msg;

    void loop();
};

void copse_server::loop() {
    cudaSetDevice(c->device);
    std::unique_lock<std::mutex> lk(mu);
    while (!stop) {
        bool progressed = false;
        // complete finished launches
        for (ModelSlot &ms : models)
            for (int bi = 0; bi < ms.nbuf; bi++) {
                Buffer &b = ms.buf[bi];
                if (!b.busy || cudaEventQuery(b.done) != cudaSuccess) continue;
                const Clock::time_point now = Clock::now();
                for (size_t j = 0; j < b.tickets.size(); j++) {
                    auto it = tickets.find(b.tickets[j]);
                    if (it == tickets.end()) continue;
                    it->second.bits.assign(b.h_bits + j * ms.L, b.h_bits + (j + 1) * ms.L);
                    it->second.state = 2;
                    it->second.t_done = now;
                }
                b.tickets.clear();
                b.busy = false;
                progressed = true;
                cv_done.notify_all();
            }
        // start launches for models with pending requests and a free buffer
        for (ModelSlot &ms : models)
            for (int bi = 0; bi < ms.nbuf; bi++) {
                Buffer &b = ms.buf[bi];
                if (b.busy || ms.pending.empty()) continue;
                const size_t n = std::min(ms.per_ct, ms.pending.size());
                memset(b.h_feats, 0, ms.per_ct * ms.nf * 4);
                for (size_t j = 0; j < n; j++) {
                    Request &r = ms.pending.front();
                    memcpy(b.h_feats + j * ms.nf, r.feats.data(), ms.nf * 4);
                    b.tickets.push_back(r.ticket);
                    tickets[r.ticket].state = 1;
                    ms.pending.pop_front();
                }
                n_pending -= n;
                copse_status st = session_launch(b.sess, b.h_feats, ++seed * 0x9E3779B97F4A7C15ULL, b.h_bits,
                                                 b.stream, b.h_seed);
                if (st == COPSE_OK && cudaEventRecord(b.done, b.stream) != cudaSuccess) st = COPSE_ECUDA;
                if (st != COPSE_OK) {
                    worker_error = st;
                    worker_msg = copse_last_error();
                    stop = true;
                    cv_done.notify_all();
                    return;
                }
                b.busy = true;
                progressed = true;
            }
        if (!progressed) {
            bool any_busy = false;
            for (ModelSlot &ms : models) any_busy |= ms.buf[0].busy || ms.buf[1].busy;
            // poll the GPU briefly while launches are in flight; otherwise sleep until a submit
            if (any_busy)
                cv_work.wait_for(lk, std::chrono::microseconds(50));
            else
                cv_work.wait(lk, [&] { return stop || n_pending > 0; });
        }
    }
}

extern "C" copse_status copse_server_create(copse_ctx *c, const copse_keys *keys, const copse_evk *evk,
                                            copse_model *const *models, size_t n_models, size_t max_pending,
                                            copse_server **out) {
    if (!c || !keys || !evk || !models || !n_models || !out) { set_error("bad argument"); return COPSE_EINVAL; }
    auto S = std::make_unique<copse_server>();
    S->c = c;
    S->models.resize(n_models);
    size_t total_slots = 0;
    for (size_t i = 0; i < n_models; i++) {
        ModelSlot &ms = S->models[i];
        ms.m = models[i];
        if (model_log_n(ms.m) != c->logN) { set_error("model compiled for another ring degree"); return COPSE_EINVAL; }
        ms.per_ct = (size_t)c->N / model_block(ms.m);
        ms.nf = model_features(ms.m);
        ms.L = model_leaves(ms.m);
        ms.precision = model_precision(ms.m);
    }
    auto cleanup = [&](copse_status st) {
        for (ModelSlot &ms : S->models)
            for (Buffer &b : ms.buf) {
                if (b.sess) copse_session_destroy(b.sess);
                if (b.stream) cudaStreamDestroy(b.stream);
                if (b.done) cudaEventDestroy(b.done);
                cudaFreeHost(b.h_feats);
                cudaFreeHost(b.h_bits);
                cudaFreeHost(b.h_seed);
            }
        return st;
    };
    // a failed runtime call releases what the earlier rounds made
    auto cuda_fail = [&](cudaError_t e, const char *what) {
        set_error(std::string(what) + ": " + cudaGetErrorString(e));
        cudaGetLastError();
        return cleanup(COPSE_ECUDA);
    };
    cudaError_t ce = cudaSetDevice(c->device);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaSetDevice");
    // first every model's one launch, then a second per model while device memory allows
    for (int round = 0; round < 2; round++)
        for (ModelSlot &ms : S->models) {
            size_t free0 = 0, total = 0;
            if ((ce = cudaMemGetInfo(&free0, &total)) != cudaSuccess) return cuda_fail(ce, "cudaMemGetInfo");
            if (round == 1 && free0 < S->launch_max + S->launch_max / 8 + S->launch_max) continue;
            Buffer &b = ms.buf[round];
            // the graph's own peak allocation: reset the device's graph-memory high-water mark
            uint64_t zero = 0;
            if ((ce = cudaDeviceSetGraphMemAttribute(c->device, cudaGraphMemAttrUsedMemHigh, &zero)) != cudaSuccess)
                return cuda_fail(ce, "cudaDeviceSetGraphMemAttribute");
            copse_status st = copse_session_create(c, keys, evk, ms.m, ms.per_ct, &b.sess);
            if (st) {
                if (st == COPSE_ENOMEM || st == COPSE_ECUDA) {
                    set_error(std::string("device memory cannot hold the server's launches: ") + copse_last_error());
                    cudaGetLastError();
                    return cleanup(round == 0 ? COPSE_EADMIT : st);
                }
                return cleanup(st);
            }
            if (cudaStreamCreateWithFlags(&b.stream, cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&b.done, cudaEventDisableTiming) != cudaSuccess ||
                cudaMallocHost(&b.h_feats, std::max<size_t>(ms.per_ct * ms.nf, 1) * 4) != cudaSuccess ||
                cudaMallocHost(&b.h_bits, std::max<size_t>(ms.per_ct * ms.L, 1)) != cudaSuccess ||
                cudaMallocHost(&b.h_seed, 8) != cudaSuccess) {
                set_error("server resources could not be created");
                cudaGetLastError();
                return cleanup(COPSE_ENOMEM);
            }
            memset(b.h_feats, 0, ms.per_ct * ms.nf * 4);
            // reserve the graph's device memory now and measure it
            st = session_launch(b.sess, b.h_feats, 1, b.h_bits, b.stream, b.h_seed);
            if (st || cudaStreamSynchronize(b.stream) != cudaSuccess) {
                if (!st) set_error("server warm-up launch failed");
                return cleanup(st ? st : COPSE_ECUDA);
            }
            uint64_t high = 0;
            if ((ce = cudaDeviceGetGraphMemAttribute(c->device, cudaGraphMemAttrUsedMemHigh, &high)) != cudaSuccess)
                return cuda_fail(ce, "cudaDeviceGetGraphMemAttribute");
            const size_t used = (size_t)high;
            S->reserved += used;
            S->launch_max = std::max(S->launch_max, used);
            ms.nbuf = round + 1;
            total_slots += ms.per_ct;
        }
    S->max_pending = max_pending ? max_pending : 4 * total_slots;
    S->mem_floor = S->launch_max;
    copse_server *raw = S.release();
    raw->worker = std::thread([raw] { raw->loop(); });
    *out = raw;
    return COPSE_OK;
}

extern "C" copse_status copse_server_submit(copse_server *S, uint32_t model_id, const uint32_t *feats,
                                            uint64_t *ticket) {
    if (!S || !feats || !ticket) { set_error("bad argument"); return COPSE_EINVAL; }
    if (model_id >= S->models.size()) { set_error("unknown model id"); return COPSE_EINVAL; }
    ModelSlot &ms = S->models[model_id];
    for (size_t k = 0; k < ms.nf; k++)
        if (ms.precision < 32 && feats[k] >= (1u << ms.precision)) { set_error("feature value needs more bits than the precision"); return COPSE_EINVAL; }
    size_t free_b = 0, total_b = 0;
    if (cudaSetDevice(S->c->device) != cudaSuccess || cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        set_error("device memory could not be queried");
        return COPSE_ECUDA;
    }
    std::lock_guard<std::mutex> g(S->mu);
    if (S->worker_error) { set_error("server stopped: " + S->worker_msg); return S->worker_error; }
    if (free_b < S->mem_floor) {
        set_error("free device memory (" + std::to_string(free_b) + " bytes) is below the admission floor (" +
                  std::to_string(S->mem_floor) + " bytes)");
        return COPSE_EADMIT;
    }
    if (S->n_pending >= S->max_pending) { set_error("request queue is full"); return COPSE_EADMIT; }
    const uint64_t t = S->next_ticket++;
    Ticket tk;
    tk.model = (int)model_id;
    tk.state = 0;
    tk.t_submit = Clock::now();
    S->tickets.emplace(t, std::move(tk));
    ms.pending.push_back(Request{t, std::vector<uint32_t>(feats, feats + ms.nf)});
    S->n_pending++;
    S->cv_work.notify_one();
    *ticket = t;
    return COPSE_OK;
}

extern "C" copse_status copse_server_poll(copse_server *S, uint64_t ticket, uint8_t *out_bits, int timeout_ms,
                                          double *latency_ms) {
    if (!S || !out_bits) { set_error("bad argument"); return COPSE_EINVAL; }
    std::unique_lock<std::mutex> lk(S->mu);
    if (S->tickets.find(ticket) == S->tickets.end()) { set_error("unknown ticket"); return COPSE_EINVAL; }
    // looked up afresh on every wake: another thread polling the same ticket may have collected it
    auto done = [&] {
        auto f = S->tickets.find(ticket);
        return S->worker_error != COPSE_OK || f == S->tickets.end() || f->second.state == 2;
    };
    if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms), done)) {
        set_error("result not ready");
        return COPSE_ETIMEOUT;
    }
    if (S->worker_error) { set_error("server stopped: " + S->worker_msg); return S->worker_error; }
    auto it = S->tickets.find(ticket);
    if (it == S->tickets.end()) { set_error("ticket already collected"); return COPSE_EINVAL; }
    Ticket &tk = it->second;
    memcpy(out_bits, tk.bits.data(), tk.bits.size());
    if (latency_ms) latency_ms[0] = std::chrono::duration<double, std::milli>(tk.t_done - tk.t_submit).count();
    S->tickets.erase(it);
    return COPSE_OK;
}

extern "C" copse_status copse_server_memory(copse_server *S, size_t *reserved, size_t *launch_max, size_t *floor,
                                            uint32_t *launches) {
    if (!S) { set_error("bad argument"); return COPSE_EINVAL; }
    std::lock_guard<std::mutex> g(S->mu);
    if (reserved) *reserved = S->reserved;
    if (launch_max) *launch_max = S->launch_max;
    if (floor) *floor = S->mem_floor;
    if (launches) {
        uint32_t n = 0;
        for (const ModelSlot &ms : S->models) n += (uint32_t)ms.nbuf;
        *launches = n;
    }
    return COPSE_OK;
}

extern "C" copse_status copse_server_set_memory_floor(copse_server *S, size_t floor) {
    if (!S) { set_error("bad argument"); return COPSE_EINVAL; }
    std::lock_guard<std::mutex> g(S->mu);
    S->mem_floor = floor;
    return COPSE_OK;
}

extern "C" copse_status copse_server_pending(copse_server *S, size_t *queued, size_t *in_flight) {
    if (!S) { set_error("bad argument"); return COPSE_EINVAL; }
    std::lock_guard<std::mutex> g(S->mu);
    size_t fl = 0;
    for (ModelSlot &ms : S->models)
        for (int bi = 0; bi < ms.nbuf; bi++) fl += ms.buf[bi].tickets.size();
    if (queued) *queued = S->n_pending;
    if (in_flight) *in_flight = fl;
    return COPSE_OK;
}

extern "C" void copse_server_destroy(copse_server *S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->worker.joinable()) S->worker.join();
    cudaSetDevice(S->c->device);
    for (ModelSlot &ms : S->models)
        for (Buffer &b : ms.buf) {
            if (b.stream) cudaStreamSynchronize(b.stream);
            if (b.sess) copse_session_destroy(b.sess);
            if (b.stream) cudaStreamDestroy(b.stream);
            if (b.done) cudaEventDestroy(b.done);
            cudaFreeHost(b.h_feats);
            cudaFreeHost(b.h_bits);
            cudaFreeHost(b.h_seed);
        }
    delete S;
}
