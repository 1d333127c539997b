// Negacyclic NTT over Z_q[X]/(X^N+1), batched over (polynomial, residue).
//
// Forward: Cooley-Tukey, natural coefficient order in, bit-reversed
// evaluation order out: position k holds a(psi^(2*brev(k)+1)).  Inverse:
// Gentleman-Sande back to coefficients, then N^-1.  Twiddles are psi^brev(k)
// (forward) and psi^-brev(k) (inverse) with Shoup quotients (the layout of
// Longa and Naehrig, "Speeding up the Number Theoretic Transform for Faster
// Ideal Lattice-Based Cryptography", CANS 2016).  Butterflies keep values
// lazily in [0, 4q) forward and [0, 2q) inverse (Harvey 2014) and reduce
// once at the end, so outputs are exact residues in [0, q).
//
// One CTA owns one residue polynomial and keeps it in shared memory for all
// log2(N) stages: a single HBM read and write per transform.
#include <atomic>

#include "internal.cuh"

namespace {

__device__ __forceinline__ int ntt_prime(const NttBatch &b, int r, int L) {
    return b.fixed >= 0 ? b.fixed : (r < b.ell ? r : L + (r - b.ell));
}

__global__ void __launch_bounds__(512) k_ntt_fwd(NttBatch b, const PrimeDev *__restrict__ primes,
                                                 const u64 *__restrict__ tw, const u64 *__restrict__ tw_sh,
                                                 int logN, int L) {
    extern __shared__ u64 sm[];
    const int N = 1 << logN, half = N >> 1;
    const int p = blockIdx.x / b.nr, r = b.r0 + blockIdx.x % b.nr;
    const int g = ntt_prime(b, r, L);
    const u64 q = primes[g].q, q2 = 2 * q;
    u64 *data = b.data + (size_t)p * b.stride + (size_t)r * N;
    const u64 *W = tw + (size_t)g * N, *Wp = tw_sh + (size_t)g * N;
    for (int i = threadIdx.x; i < N; i += blockDim.x) sm[i] = data[i];
    __syncthreads();
    for (int m = 1, lt = logN - 1; m < N; m <<= 1, lt--) {
        const int tt = 1 << lt;
        for (int x = threadIdx.x; x < half; x += blockDim.x) {
            const int i = x >> lt, j = x & (tt - 1);
            const int idx = (i << (lt + 1)) + j;
            const u64 w = W[m + i], wp = Wp[m + i];
            u64 U = sm[idx];
            if (U >= q2) U -= q2;
            const u64 V = mul_shoup_lazy(sm[idx + tt], w, wp, q);
            sm[idx] = U + V;
            sm[idx + tt] = U - V + q2;
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        u64 v = sm[i];
        if (v >= q2) v -= q2;
        if (v >= q) v -= q;
        data[i] = v;
    }
}

__global__ void __launch_bounds__(512) k_ntt_inv(NttBatch b, const PrimeDev *__restrict__ primes,
                                                 const u64 *__restrict__ tw, const u64 *__restrict__ tw_sh,
                                                 int logN, int L) {
    extern __shared__ u64 sm[];
    const int N = 1 << logN, half = N >> 1;
    const int p = blockIdx.x / b.nr, r = b.r0 + blockIdx.x % b.nr;
    const int g = ntt_prime(b, r, L);
    const PrimeDev P = primes[g];
    const u64 q = P.q, q2 = 2 * q;
    u64 *data = b.data + (size_t)p * b.stride + (size_t)r * N;
    const u64 *W = tw + (size_t)g * N, *Wp = tw_sh + (size_t)g * N;
    for (int i = threadIdx.x; i < N; i += blockDim.x) sm[i] = data[i];
    __syncthreads();
    for (int m = N, lt = 0; m > 1; m >>= 1, lt++) {
        const int tt = 1 << lt, h = m >> 1;
        for (int x = threadIdx.x; x < half; x += blockDim.x) {
            const int i = x >> lt, j = x & (tt - 1);
            const int idx = (i << (lt + 1)) + j;
            const u64 w = W[h + i], wp = Wp[h + i];
            const u64 U = sm[idx], V = sm[idx + tt];
            u64 s = U + V;
            if (s >= q2) s -= q2;
            sm[idx] = s;
            sm[idx + tt] = mul_shoup_lazy(U - V + q2, w, wp, q);
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < N; i += blockDim.x) data[i] = mul_shoup(sm[i], P.ninv, P.ninv_sh, q);
}

copse_status launch(copse_ctx *ctx, const NttBatch &b, cudaStream_t s, bool inverse) {
    if (b.npoly <= 0 || b.nr <= 0) return COPSE_OK;
    const int N = ctx->N;
    const size_t smem = (size_t)N * sizeof(u64);
    const int threads = N / 2 < 512 ? N / 2 : 512;
    const unsigned grid = (unsigned)b.npoly * (unsigned)b.nr;
    // the kernels' dynamic shared-memory limit only ever grows (contexts of
    // different ring degrees may be alive at the same time)
    static std::atomic<int> smem_limit{0};
    if ((int)smem > smem_limit.load()) {
        CUDA_TRY(cudaFuncSetAttribute(k_ntt_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        CUDA_TRY(cudaFuncSetAttribute(k_ntt_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        smem_limit.store((int)smem);
    }
    const double bytes = (double)grid * N * 16.0;  // one read and one write of each residue polynomial
    if (inverse)
        TIMED("ntt_inv", bytes, s,
              k_ntt_inv<<<grid, threads, smem, s>>>(b, ctx->d_prime, ctx->d_ipsi, ctx->d_ipsi_sh, ctx->logN, ctx->L));
    else
        TIMED("ntt_fwd", bytes, s,
              k_ntt_fwd<<<grid, threads, smem, s>>>(b, ctx->d_prime, ctx->d_psi, ctx->d_psi_sh, ctx->logN, ctx->L));
    LAUNCH_CHECK();
    return COPSE_OK;
}

}  // namespace

copse_status ntt_forward(copse_ctx *ctx, const NttBatch &b, cudaStream_t s) { return launch(ctx, b, s, false); }
copse_status ntt_inverse(copse_ctx *ctx, const NttBatch &b, cudaStream_t s) { return launch(ctx, b, s, true); }
