// Allocation-free negacyclic product: the same result as copse_poly_mul, with
// its two transform buffers in a fixed device array instead of the context's
// memory pool.
//
// Some callers cannot allocate device memory at the moment they need a
// product: serving loops that forbid any allocation after start-up so that
// latency stays flat and memory use stays fixed, and programs whose device
// memory is already fully reserved by another allocator (for example a
// framework's caching allocator that owns the GPU).  This entry point calls no
// cudaMalloc, cudaFree or allocating routine of any library.
//
// The scratch array below lives in device memory on every GPU that loads this
// library, from load until the process exits.  Host code cannot use its name
// as a device address, so the first call on each device looks the address up
// with cudaGetSymbolAddress (that device must be current) and caches it; make
// that first call before any stream capture.  Every call on a device shares
// the same array: calls that overlap on the GPU (different streams, or host
// threads without ordering) race and give wrong results, so order them on one
// stream.  Nothing in the array needs to start at zero: each call overwrites
// the words it reads.
#include <mutex>

#include "internal.cuh"

// per operand: n_res * N words at most (2 MiB), two operands
#define NOALLOC_MAX_WORDS (1u << 18)
#define NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) u64 g_noalloc_scratch[2 * (size_t)NOALLOC_MAX_WORDS];

namespace {

__global__ void k_pointwise_mul(const u64 *a, const u64 *b, u64 *out, int nres, int logN, const PrimeDev *pr) {
    size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ((size_t)nres << logN)) return;
    out[e] = mul_mod(a[e], b[e], pr[e >> logN]);
}

std::mutex scratch_mu;
u64 *scratch_addr[NOALLOC_MAX_DEVICES] = {};

// device address of the scratch array on `device`, which must be the calling thread's
// current device on every call: the cached address belongs to that device's copy of the
// array, and a launch on another device with it would touch memory of the wrong GPU
copse_status scratch_on(int device, u64 **out) {
    if (device < 0 || device >= NOALLOC_MAX_DEVICES) { set_error("device index out of range"); return COPSE_EINVAL; }
    int cur = -1;
    CUDA_TRY(cudaGetDevice(&cur));
    if (cur != device) { set_error("the context's device is not the current device"); return COPSE_EINVAL; }
    std::lock_guard<std::mutex> g(scratch_mu);
    if (!scratch_addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_error(std::string("cudaGetSymbolAddress of the static scratch: ") + cudaGetErrorString(e));
            return COPSE_ECUDA;
        }
        scratch_addr[device] = (u64 *)p;
    }
    *out = scratch_addr[device];
    return COPSE_OK;
}

}  // namespace

extern "C" copse_status copse_poly_mul_noalloc(copse_ctx *c, const uint64_t *a, const uint64_t *b, uint64_t *out,
                                               uint32_t n_res, void *stream) {
    if (!c || !a || !b || !out || n_res < 1 || (int)n_res > c->L) { set_error("bad argument"); return COPSE_EINVAL; }
    const size_t words = (size_t)n_res * c->N;
    if (words > NOALLOC_MAX_WORDS) {
        set_error("n_res * N = " + std::to_string(words) + " words exceeds the static scratch limit of " +
                  std::to_string(NOALLOC_MAX_WORDS) + " words per operand");
        return COPSE_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    u64 *scratch = nullptr;
    STATUS_TRY(scratch_on(c->device, &scratch));
    u64 *fa = scratch, *fb = scratch + NOALLOC_MAX_WORDS;
    const int nr = (int)n_res;
    CUDA_TRY(cudaMemcpyAsync(fa, a, words * 8, cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(fb, b, words * 8, cudaMemcpyDeviceToDevice, s));
    STATUS_TRY(ntt_forward(c, NttBatch{fa, words, 1, 0, nr, nr, -1}, s));
    STATUS_TRY(ntt_forward(c, NttBatch{fb, words, 1, 0, nr, nr, -1}, s));
    k_pointwise_mul<<<(unsigned)((words + 255) / 256), 256, 0, s>>>(fa, fb, out, nr, c->logN, c->d_prime);
    LAUNCH_CHECK();
    return ntt_inverse(c, NttBatch{out, words, 1, 0, nr, nr, -1}, s);
}
