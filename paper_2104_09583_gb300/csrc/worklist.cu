// Persistent work-list kernel: one resident launch walks a list of elementwise
// ciphertext operations (items), each cut into tiles.  The CTAs -- as many as
// fit on the device at once -- take tiles in list order from a global counter;
// an item that reads another item's output waits for every tile of that item
// first.  Waits are bounded by the global timer: when one runs out the kernel
// raises an error flag, every CTA stops taking tiles, and the host reads
// COPSE_ETIMEOUT.  Because tiles are taken in list order and a CTA only takes
// a tile while it runs, an item's dependency was taken earlier by a CTA that is
// running, so a list whose dependencies point backwards always completes.
//
// Item kinds (x, y, z inputs; o0, o1 outputs; every polynomial [level][N] per
// component, NTT domain, components `comp` words apart):
//   ADD      o0 = x + y                       (2 components)
//   SUB      o0 = x - y                       (2 components)
//   LEAF     o0 = y - z, o1 = 2 z - x + 1 (SecComp leaves with encrypted
//            thresholds, Section 4.1.2: y the threshold plane and x the sum
//            feature + threshold plane, both switched to the level of z = the
//            product of feature and threshold: lt = y - xy, eq = 2xy - (x + y) + 1)
//   TENSOR   (o0, o0 + n, o0 + 2n) = (x0 y0, x0 y1 + x1 y0, x1 y1)
#include <algorithm>
#include <atomic>
#include <memory>

#include "internal.cuh"

namespace {

constexpr int WL_TPB = 256;
constexpr int WL_TILE = 2048;  // elements (one per component position) per tile

struct WlDev {
    int n;
    int tile_off[WL_MAX + 1];  // first global tile of each item, prefix sums
    WlItem it[WL_MAX];
};

__global__ void __launch_bounds__(WL_TPB) k_worklist(const WlDev L, int *counters, int logN,
                                                     const PrimeDev *__restrict__ pr, unsigned long long timeout_ns) {
    // counters: [0] next tile, [1] error flag, [2] item of the failed wait, [2 + 1 + i] tiles done of item i
    int *next = counters, *err = counters + 1, *done = counters + 3;
    __shared__ int s_tile, s_item;
    const int total = L.tile_off[L.n];
    while (true) {
        if (threadIdx.x == 0) {
            s_tile = *(volatile int *)err ? total : atomicAdd(next, 1);
            int lo = 0, hi = L.n - 1;
            while (lo < hi) {  // last item whose first tile is <= s_tile
                const int mid = (lo + hi + 1) >> 1;
                if (L.tile_off[mid] <= s_tile) lo = mid;
                else hi = mid - 1;
            }
            s_item = lo;
        }
        __syncthreads();
        const int tile = s_tile, i = s_item;
        if (tile >= total) return;
        const WlItem &W = L.it[i];
        if (W.dep >= 0 || W.dep2 >= 0) {
            if (threadIdx.x == 0) {
                const unsigned long long t0 = global_ns();
                for (int k = 0; k < 2; k++) {
                    const int d = k == 0 ? W.dep : W.dep2;
                    if (d < 0) continue;
                    const int need = L.tile_off[d + 1] - L.tile_off[d];
                    unsigned ns = 64;
                    while (*(volatile int *)&done[d] < need) {
                        if (*(volatile int *)err) break;
                        if (global_ns() - t0 > timeout_ns) {  // bounded: raise the flag and stop
                            if (atomicExch(err, 1) == 0) counters[2] = i;
                            break;
                        }
                        __nanosleep(ns);
                        ns = min(ns * 2, 4096u);
                    }
                }
                __threadfence();
            }
            __syncthreads();
            if (*(volatile int *)err) return;
        }
        const size_t per = (size_t)W.level << logN;  // elements of one component
        const size_t e0 = (size_t)(tile - L.tile_off[i]) * WL_TILE;
        for (size_t e = e0 + threadIdx.x; e < min(per, e0 + WL_TILE); e += WL_TPB) {
            const PrimeDev P = pr[e >> logN];
            const u64 q = P.q;
            switch (W.kind) {
            case WL_ADD:
            case WL_SUB:
                for (int c = 0; c < 2; c++) {
                    const size_t k = (size_t)c * W.comp + e;
                    W.o0[k] = W.kind == WL_ADD ? add_mod(W.x[k], W.y[k], q) : sub_mod(W.x[k], W.y[k], q);
                }
                break;
            case WL_LEAF:
                for (int c = 0; c < 2; c++) {
                    const size_t k = (size_t)c * W.comp + e;
                    const u64 z = W.z[k];
                    W.o0[k] = sub_mod(W.y[k], z, q);
                    u64 eq = sub_mod(add_mod(z, z, q), W.x[k], q);
                    if (c == 0) eq = add_mod(eq, 1, q);  // + 1: the constant 1 is 1 at every evaluation point
                    W.o1[k] = eq;
                }
                break;
            case WL_TENSOR: {
                const u64 x0 = W.x[e], x1 = W.x[W.comp + e], y0 = W.y[e], y1 = W.y[W.comp + e];
                W.o0[e] = mul_mod(x0, y0, P);
                W.o0[per + e] = add_mod(mul_mod(x0, y1, P), mul_mod(x1, y0, P), q);
                W.o0[2 * per + e] = mul_mod(x1, y1, P);
                break;
            }
            default:
                break;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();  // this tile's stores are visible before it counts as done
            atomicAdd(&done[i], 1);
        }
    }
}

int wl_tiles(const WlItem &w, int logN) {
    const size_t per = (size_t)w.level << logN;
    return (int)((per + WL_TILE - 1) / WL_TILE);
}

}  // namespace

// The persistent grid: CTAs resident on the device at once (queried once per device).
static int wl_grid(int device) {
    static std::atomic<int> cache[64];
    if (device >= 0 && device < 64 && cache[device].load() > 0) return cache[device].load();
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_worklist, WL_TPB, 0);
    const int g = std::max(1, sms * std::max(1, per_sm));
    if (device >= 0 && device < 64) cache[device].store(g);
    return g;
}

copse_status worklist_run(copse_ctx *c, const std::vector<WlItem> &items, int timeout_ms, cudaStream_t s,
                          int *d_counters_out) {
    const size_t n = items.size();
    for (size_t b0 = 0; b0 < n; b0 += WL_MAX) {
        WlDev L{};
        L.n = (int)std::min<size_t>(WL_MAX, n - b0);
        L.tile_off[0] = 0;
        for (int i = 0; i < L.n; i++) {
            L.it[i] = items[b0 + i];
            // a dependency in an earlier launch is already complete (stream order)
            for (int *d : {&L.it[i].dep, &L.it[i].dep2}) {
                if (*d >= (int)(b0 + L.n)) { set_error("work-list dependency on an item of a later launch"); return COPSE_EINVAL; }
                if (*d >= 0) *d = *d < (int)b0 ? -1 : *d - (int)b0;
            }
            L.tile_off[i + 1] = L.tile_off[i] + wl_tiles(L.it[i], c->logN);
        }
        int *cnt = d_counters_out;
        Scratch sc(s);
        if (!cnt) {
            u64 *p = nullptr;
            STATUS_TRY(sc.get(c, &p, (3 + WL_MAX + 1) / 2));
            cnt = (int *)p;
        }
        CUDA_TRY(cudaMemsetAsync(cnt, 0, (3 + WL_MAX) * sizeof(int), s));
        const int grid = std::min(wl_grid(c->device), std::max(1, L.tile_off[L.n]));
        TIMED("worklist", 0.0, s,
              k_worklist<<<grid, WL_TPB, 0, s>>>(L, cnt, c->logN, c->d_prime,
                                                 (unsigned long long)std::max(1, timeout_ms) * 1000000ull));
        LAUNCH_CHECK();
        if (d_counters_out && b0 + WL_MAX < n) {
            // the caller reads the flag of the last launch; stop after a failed one
            int h[3] = {0, 0, 0};
            CUDA_TRY(cudaMemcpyAsync(h, cnt, sizeof(h), cudaMemcpyDeviceToHost, s));
            CUDA_TRY(cudaStreamSynchronize(s));
            if (h[1]) return COPSE_OK;
        }
    }
    return COPSE_OK;
}

// ---------------------------------------------------------------- C ABI
extern "C" copse_status copse_worklist_run(copse_ctx *c, const copse_ctbuf *in, const copse_wl_item *items, size_t n,
                                           int timeout_ms, copse_ctbuf **out, void *stream) {
    if (!c || !in || !out || (n && !items) || timeout_ms < 1) { set_error("bad argument"); return COPSE_EINVAL; }
    if (n > WL_MAX) { set_error("at most " + std::to_string(WL_MAX) + " items per list"); return COPSE_EINVAL; }
    cudaStream_t s = (cudaStream_t)stream;
    const size_t nin = in->cts.size();
    auto buf = std::make_unique<copse_ctbuf>();
    buf->ctx = c;
    buf->stream = s;
    buf->cts.resize(n);
    std::vector<WlItem> wl(n);
    auto operand = [&](uint32_t r, size_t i, const DCt **ct) -> copse_status {
        if (r < nin) { *ct = &in->cts[r]; return COPSE_OK; }
        if (r - nin >= i) { set_error("item " + std::to_string(i) + " reads an output that is not earlier"); return COPSE_EINVAL; }
        *ct = &buf->cts[r - nin];
        return COPSE_OK;
    };
    for (size_t i = 0; i < n; i++) {
        const copse_wl_item &it = items[i];
        const DCt *x = nullptr, *y = nullptr;
        STATUS_TRY(operand(it.a, i, &x));
        STATUS_TRY(operand(it.b, i, &y));
        if (x->level != y->level || x->ncomp != 2 || y->ncomp != 2) { set_error("operands must be two-component ciphertexts at one level"); return COPSE_EINVAL; }
        if (it.kind != COPSE_WL_ADD && it.kind != COPSE_WL_SUB && it.kind != COPSE_WL_TENSOR) { set_error("unknown item kind"); return COPSE_EINVAL; }
        if (it.dep < -1 || it.dep >= (int32_t)n) { set_error("dependency out of range"); return COPSE_EINVAL; }
        DCt &o = buf->cts[i];
        STATUS_TRY(ct_alloc(c, &o, x->level, it.kind == COPSE_WL_TENSOR ? 3 : 2, s));
        WlItem &w = wl[i];
        w.kind = it.kind == COPSE_WL_ADD ? WL_ADD : (it.kind == COPSE_WL_SUB ? WL_SUB : WL_TENSOR);
        w.level = x->level;
        w.comp = (size_t)x->level * c->N;
        w.x = x->data;
        w.y = y->data;
        w.o0 = o.data;
        // the named dependency, and the later of the earlier outputs the item reads
        w.dep = it.dep;
        if (it.a >= nin) w.dep2 = (int)(it.a - nin);
        if (it.b >= nin) w.dep2 = std::max(w.dep2, (int)(it.b - nin));
    }
    u64 *cnt = nullptr;
    STATUS_TRY(dev_alloc(c, (void **)&cnt, (3 + WL_MAX) * sizeof(int), s));
    copse_status st = worklist_run(c, wl, timeout_ms, s, (int *)cnt);
    int h[3] = {0, 0, 0};
    if (st == COPSE_OK && (cudaMemcpyAsync(h, cnt, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                           cudaStreamSynchronize(s) != cudaSuccess)) {
        set_error("work list status could not be read");
        st = COPSE_ECUDA;
    }
    dev_free(cnt, s);
    if (st) return st;
    if (h[1]) {
        set_error("work list: item " + std::to_string(h[2]) + " waited " + std::to_string(timeout_ms) +
                  " ms for its dependency");
        return COPSE_ETIMEOUT;
    }
    *out = buf.release();
    return COPSE_OK;
}
