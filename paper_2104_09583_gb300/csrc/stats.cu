// Per-kernel timing: when enabled, every instrumented launch is bracketed by
// two CUDA events recorded on the launch stream, tagged with the kernel
// family and its algorithmic byte count.  copse_stats_get() waits for the
// device and sums event intervals per family.  Events come from a reused pool
// so instrumentation adds no allocation to the timed region after warm-up.
#include <cstring>
#include <map>
#include <mutex>
#include <string>

#include "internal.cuh"

namespace {

struct Rec {
    std::string name;
    int ev;        // index of the event pair
    double bytes;  // algorithmic bytes of the launch
    double ops;    // algorithmic modular products of the launch (0 = not counted)
};
struct Totals {
    uint64_t launches = 0;
    double ms = 0, bytes = 0, ops = 0;
};

std::mutex mu;
bool enabled = false;
std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pool;
size_t used = 0;
std::vector<Rec> pending;
std::map<std::string, Totals> totals;

void drain() {
    // caller holds mu and has synchronised the device
    for (const Rec &r : pending) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, pool[r.ev].first, pool[r.ev].second) == cudaSuccess) {
            Totals &t = totals[r.name];
            t.launches++;
            t.ms += ms;
            t.bytes += r.bytes;
            t.ops += r.ops;
        }
    }
    pending.clear();
    used = 0;
    cudaGetLastError();
}

}  // namespace

// graph capture records no timing events
static thread_local bool suspended = false;
void stats_suspend(bool on) { suspended = on; }

int stats_begin(const char *name, double bytes, cudaStream_t s) { return stats_begin_ops(name, bytes, 0.0, s); }

int stats_begin_ops(const char *name, double bytes, double ops, cudaStream_t s) {
    if (!enabled || suspended) return -1;
    std::lock_guard<std::mutex> g(mu);
    if (used == pool.size()) {
        cudaEvent_t a, b;
        if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return -1;
        pool.push_back({a, b});
    }
    int ev = (int)used++;
    cudaEventRecord(pool[ev].first, s);
    pending.push_back(Rec{name, ev, bytes, ops});
    return ev;
}

void stats_end(int token, cudaStream_t s) {
    if (token < 0) return;
    cudaEventRecord(pool[token].second, s);
}

extern "C" copse_status copse_stats_enable(int on) {
    std::lock_guard<std::mutex> g(mu);
    enabled = on != 0;
    return COPSE_OK;
}

extern "C" copse_status copse_stats_reset(void) {
    CUDA_TRY(cudaDeviceSynchronize());
    std::lock_guard<std::mutex> g(mu);
    drain();
    totals.clear();
    return COPSE_OK;
}

extern "C" copse_status copse_stats_get(const char *name, uint64_t *launches, double *ms, double *bytes) {
    CUDA_TRY(cudaDeviceSynchronize());
    std::lock_guard<std::mutex> g(mu);
    drain();
    Totals t;
    if (name && *name) {
        auto it = totals.find(name);
        if (it != totals.end()) t = it->second;
    } else {
        for (auto &kv : totals) {
            t.launches += kv.second.launches;
            t.ms += kv.second.ms;
            t.bytes += kv.second.bytes;
        }
    }
    if (launches) *launches = t.launches;
    if (ms) *ms = t.ms;
    if (bytes) *bytes = t.bytes;
    return COPSE_OK;
}

extern "C" copse_status copse_stats_get_ops(const char *name, double *ops) {
    if (!ops) { set_error("null output"); return COPSE_EINVAL; }
    CUDA_TRY(cudaDeviceSynchronize());
    std::lock_guard<std::mutex> g(mu);
    drain();
    double v = 0;
    for (auto &kv : totals)
        if (!name || !*name || kv.first == name) v += kv.second.ops;
    *ops = v;
    return COPSE_OK;
}

extern "C" copse_status copse_stats_names(char *buf, size_t cap) {
    CUDA_TRY(cudaDeviceSynchronize());
    std::lock_guard<std::mutex> g(mu);
    drain();
    std::string s;
    for (auto &kv : totals) s += kv.first + "\n";
    if (!buf || cap <= s.size()) { set_error("buffer too small"); return COPSE_EINVAL; }
    memcpy(buf, s.c_str(), s.size() + 1);
    return COPSE_OK;
}
