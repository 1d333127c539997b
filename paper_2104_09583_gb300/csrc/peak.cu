// Measured integer peaks of the modular arithmetic the kernels are built from:
// register-only microbenchmarks, timed with CUDA events, that give the
// denominators of the integer roofline (no spec-sheet rates).
//
//   kind 0  exact products in a lazily reduced sum: x y added to split-28 partial
//           sums (four 32 x 32 -> 64-bit multiply-adds per product, the form of the
//           encrypted-model and key-switching dot products)
//   kind 1  Shoup butterflies: the lazy forward NTT butterfly with a constant
//           twiddle (Harvey 2014), the unit of the transforms
//   kind 2  Barrett products of two data residues (Handbook of Applied
//           Cryptography, Alg. 14.42), fully reduced
//
// Every thread runs CHAINS independent dependency chains so that issue, not
// latency, bounds the rate; the results are folded into one word per thread
// and stored, so nothing is dead code.
#include <algorithm>

#include "internal.cuh"

namespace {

constexpr int CHAINS = 8;
constexpr int PEAK_TPB = 256;

__global__ void __launch_bounds__(PEAK_TPB) k_peak_mac(int iters, u64 seed, u64 *sink) {
    const u64 t = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    Sp28 x[CHAINS];
    Acc3w a[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; c++) {
        x[c] = split28((seed * (t + 1) + 0x9E3779B97F4A7C15ull * (c + 1)) & ((1ull << 55) - 1));
        a[c] = Acc3w{0, 0, 0};
    }
    u64 v = (seed ^ t) & ((1ull << 55) - 1);
    for (int i = 0; i < iters; i++) {
        v = (v + 0x00A3C59AC2F1ull) & ((1ull << 55) - 1);
        const Sp28 y = split28(v);
#pragma unroll
        for (int c = 0; c < CHAINS; c++) mac_sp(a[c], x[c], y);
        // the partial sums hold 64 products exactly; fold them before that bound
        if ((i & 31) == 31) {
#pragma unroll
            for (int c = 0; c < CHAINS; c++) a[c] = Acc3w{a[c].lo >> 8, a[c].mid >> 8, a[c].hi >> 8};
        }
    }
    u64 r = 0;
#pragma unroll
    for (int c = 0; c < CHAINS; c++) r ^= a[c].lo + a[c].mid + a[c].hi;
    sink[t] = r;
}

__global__ void __launch_bounds__(PEAK_TPB) k_peak_butterfly(int iters, u64 q, u64 w, u64 wp, u64 *sink) {
    const u64 t = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    const u64 q2 = 2 * q;
    u64 x[CHAINS], y[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; c++) {
        x[c] = (t * 0x9E3779B97F4A7C15ull + c) % q;
        y[c] = (t * 0xBF58476D1CE4E5B9ull + 3 * c) % q;
    }
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < CHAINS; c++) {
            u64 U = x[c];
            if (U >= q2) U -= q2;
            const u64 V = mul_shoup_lazy(y[c], w, wp, q);
            x[c] = U + V;
            y[c] = U - V + q2;
        }
    }
    u64 r = 0;
#pragma unroll
    for (int c = 0; c < CHAINS; c++) r ^= x[c] + y[c];
    sink[t] = r;
}

__global__ void __launch_bounds__(PEAK_TPB) k_peak_barrett(int iters, PrimeDev P, u64 *sink) {
    const u64 t = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    u64 z[CHAINS], w[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; c++) {
        z[c] = (t * 0x9E3779B97F4A7C15ull + c + 1) % P.q;
        w[c] = (t * 0x94D049BB133111EBull + 7 * c + 2) % P.q;
    }
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < CHAINS; c++) z[c] = mul_mod(z[c], w[c], P);
    }
    u64 r = 0;
#pragma unroll
    for (int c = 0; c < CHAINS; c++) r ^= z[c];
    sink[t] = r;
}

}  // namespace

extern "C" copse_status copse_measure_int_peak(copse_ctx *c, int kind, int reps, double *ops_per_s, float *best_ms) {
    if (!c || !ops_per_s || kind < 0 || kind > 2 || reps < 1) { set_error("bad argument"); return COPSE_EINVAL; }
    int sms = 0;
    CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
    // eight resident CTAs of 256 threads per SM: enough warps to cover every pipe's latency
    const unsigned blocks = (unsigned)sms * 8;
    const size_t threads = (size_t)blocks * PEAK_TPB;
    const int iters = kind == 0 ? 4096 : (kind == 1 ? 2048 : 1024);
    u64 *sink = nullptr;
    CUDA_TRY(cudaMalloc(&sink, threads * sizeof(u64)));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const PrimeDev P = c->hprime[0];
    // a fixed constant and its Shoup quotient modulo the first prime
    const u64 w = (P.q / 3) | 1, wp = (u64)(((unsigned __int128)w << 64) / P.q);
    float best = 1e30f;
    copse_status st = COPSE_OK;
    for (int r = 0; r <= reps && st == COPSE_OK; r++) {  // the first run warms up
        cudaEventRecord(e0, 0);
        if (kind == 0) k_peak_mac<<<blocks, PEAK_TPB>>>(iters, 0x1234567ull + r, sink);
        else if (kind == 1) k_peak_butterfly<<<blocks, PEAK_TPB>>>(iters, P.q, w, wp, sink);
        else k_peak_barrett<<<blocks, PEAK_TPB>>>(iters, P, sink);
        cudaEventRecord(e1, 0);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
            set_error("peak microbenchmark launch failed");
            st = COPSE_ECUDA;
            break;
        }
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r > 0) best = std::min(best, ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (st != COPSE_OK) return st;
    *ops_per_s = (double)threads * iters * CHAINS / (best * 1e-3);
    if (best_ms) *best_ms = best;
    return COPSE_OK;
}
