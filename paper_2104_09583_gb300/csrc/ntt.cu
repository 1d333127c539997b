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
// Large rings (log N >= 12) run in two passes over N = N1 x N2 viewed as N1
// rows of N2 contiguous coefficients.  The first log2(N1) forward stages pair
// coefficients of the same column; the last log2(N2) pair coefficients of the
// same row.  Each pass stages a 16 KB tile (columns x all rows, or rows x all
// columns) in shared memory, so one polynomial spreads over N / 2048 CTAs per
// pass and a launch fills the GPU even for a few dozen polynomials; the
// intermediate round trip stays in L2.  Small rings use one CTA per
// polynomial.
#include "internal.cuh"

namespace {

constexpr int TILE = 2048;  // coefficients per CTA in the two-pass kernels
constexpr int NT2 = 256;    // threads per CTA in the two-pass kernels

__device__ __forceinline__ int ntt_prime(const NttBatch &b, int r, int L) {
    return b.fixed >= 0 ? b.fixed : (r < b.ell ? r : L + (r - b.ell));
}

// residue r of poly p is excluded from this batch (a ModUp digit's own primes)
__device__ __forceinline__ bool ntt_skipped(const NttBatch &b, int p, int r) {
    return b.skip_alpha > 0 && r >= p * b.skip_alpha && r < min((p + 1) * b.skip_alpha, b.ell);
}

// forward butterfly on shared memory, values in [0, 4q)
__device__ __forceinline__ void bf_fwd(u64 *x, u64 *y, u64 w, u64 wp, u64 q, u64 q2) {
    u64 U = *x;
    if (U >= q2) U -= q2;
    const u64 V = mul_shoup_lazy(*y, w, wp, q);
    *x = U + V;
    *y = U - V + q2;
}

// inverse butterfly on shared memory, values in [0, 2q)
__device__ __forceinline__ void bf_inv(u64 *x, u64 *y, u64 w, u64 wp, u64 q, u64 q2) {
    const u64 U = *x, V = *y;
    u64 s = U + V;
    if (s >= q2) s -= q2;
    *x = s;
    *y = mul_shoup_lazy(U - V + q2, w, wp, q);
}

// ---------------------------------------------------------------- one CTA per polynomial
__global__ void __launch_bounds__(512) k_ntt_fwd(NttBatch b, const PrimeDev *__restrict__ primes,
                                                 const u64 *__restrict__ tw, const u64 *__restrict__ tw_sh,
                                                 int logN, int L) {
    extern __shared__ u64 sm[];
    const int N = 1 << logN, half = N >> 1;
    const int p = blockIdx.x / b.nr, r = b.r0 + blockIdx.x % b.nr;
    if (ntt_skipped(b, p, r)) return;
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
            bf_fwd(&sm[idx], &sm[idx + tt], W[m + i], Wp[m + i], q, q2);
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
    if (ntt_skipped(b, p, r)) return;
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
            bf_inv(&sm[idx], &sm[idx + tt], W[h + i], Wp[h + i], q, q2);
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < N; i += blockDim.x) data[i] = mul_shoup(sm[i], P.ninv, P.ninv_sh, q);
}

// ---------------------------------------------------------------- two passes (N = N1 x N2)
// Column pass: tile = C consecutive columns x all N1 rows, stored row-major [row][C].
// Forward: stages 0 .. a-1 (pairs of rows within a column, distance N1/2 .. 1).
__global__ void __launch_bounds__(NT2) k_ntt_fwd_cols(NttBatch b, const PrimeDev *__restrict__ primes,
                                                      const u64 *__restrict__ tw, const u64 *__restrict__ tw_sh,
                                                      int logN, int L, int a) {
    __shared__ u64 sm[TILE];
    const int N = 1 << logN, lb = logN - a, N2 = 1 << lb;
    const int lc = __ffs(TILE) - 1 - a, C = 1 << lc;  // columns per tile
    const int tiles = N2 >> lc;
    const int pr = blockIdx.x / tiles, tile = blockIdx.x % tiles;
    const int p = pr / b.nr, r = b.r0 + pr % b.nr;
    if (ntt_skipped(b, p, r)) return;
    const int g = ntt_prime(b, r, L);
    const u64 q = primes[g].q, q2 = 2 * q;
    u64 *data = b.data + (size_t)p * b.stride + (size_t)r * N + (tile << lc);
    const u64 *W = tw + (size_t)g * N, *Wp = tw_sh + (size_t)g * N;
    for (int e = threadIdx.x; e < TILE; e += NT2) sm[e] = data[((size_t)(e >> lc) << lb) + (e & (C - 1))];
    __syncthreads();
    for (int s = 0; s < a; s++) {
        const int lt = a - 1 - s, tt = 1 << lt, m = 1 << s;
        for (int x = threadIdx.x; x < TILE / 2; x += NT2) {
            const int col = x & (C - 1), j = x >> lc;
            const int i = j >> lt, jj = j & (tt - 1);
            const int row = (i << (lt + 1)) + jj;
            bf_fwd(&sm[(row << lc) + col], &sm[((row + tt) << lc) + col], W[m + i], Wp[m + i], q, q2);
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < TILE; e += NT2) data[((size_t)(e >> lc) << lb) + (e & (C - 1))] = sm[e];
}

// Row pass: tile = R consecutive rows of N2 contiguous coefficients.
// Forward: stages a .. logN-1; the group of a butterfly is row * 2^s' + local group.
__global__ void __launch_bounds__(NT2) k_ntt_fwd_rows(NttBatch b, const PrimeDev *__restrict__ primes,
                                                      const u64 *__restrict__ tw, const u64 *__restrict__ tw_sh,
                                                      int logN, int L, int a) {
    __shared__ u64 sm[TILE];
    const int N = 1 << logN, lb = logN - a;
    const int lr = __ffs(TILE) - 1 - lb;  // rows per tile = 2^lr
    const int tiles = 1 << (a - lr);
    const int pr = blockIdx.x / tiles, tile = blockIdx.x % tiles;
    const int p = pr / b.nr, r = b.r0 + pr % b.nr;
    if (ntt_skipped(b, p, r)) return;
    const int g = ntt_prime(b, r, L);
    const u64 q = primes[g].q, q2 = 2 * q;
    const int row0 = tile << lr;
    u64 *data = b.data + (size_t)p * b.stride + (size_t)r * N + ((size_t)row0 << lb);
    const u64 *W = tw + (size_t)g * N, *Wp = tw_sh + (size_t)g * N;
    for (int e = threadIdx.x; e < TILE; e += NT2) sm[e] = data[e];
    __syncthreads();
    const int lh = lb - 1;  // log2 of butterflies per row
    for (int s = 0; s < lb; s++) {
        const int lt = lb - 1 - s, tt = 1 << lt, m = 1 << (a + s);
        for (int x = threadIdx.x; x < TILE / 2; x += NT2) {
            const int rl = x >> lh, j = x & ((1 << lh) - 1);
            const int il = j >> lt, jj = j & (tt - 1);
            const int idx = (rl << lb) + (il << (lt + 1)) + jj;
            const int gi = m + (((row0 + rl) << s) + il);
            bf_fwd(&sm[idx], &sm[idx + tt], W[gi], Wp[gi], q, q2);
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < TILE; e += NT2) {
        u64 v = sm[e];
        if (v >= q2) v -= q2;
        if (v >= q) v -= q;
        data[e] = v;
    }
}

// Inverse, row pass first: distances 1 .. N2/2; group = row * 2^(lb-1-u) + local group.
__global__ void __launch_bounds__(NT2) k_ntt_inv_rows(NttBatch b, const PrimeDev *__restrict__ primes,
                                                      const u64 *__restrict__ tw, const u64 *__restrict__ tw_sh,
                                                      int logN, int L, int a) {
    __shared__ u64 sm[TILE];
    const int N = 1 << logN, lb = logN - a;
    const int lr = __ffs(TILE) - 1 - lb;
    const int tiles = 1 << (a - lr);
    const int pr = blockIdx.x / tiles, tile = blockIdx.x % tiles;
    const int p = pr / b.nr, r = b.r0 + pr % b.nr;
    if (ntt_skipped(b, p, r)) return;
    const int g = ntt_prime(b, r, L);
    const u64 q = primes[g].q, q2 = 2 * q;
    const int row0 = tile << lr;
    u64 *data = b.data + (size_t)p * b.stride + (size_t)r * N + ((size_t)row0 << lb);
    const u64 *W = tw + (size_t)g * N, *Wp = tw_sh + (size_t)g * N;
    for (int e = threadIdx.x; e < TILE; e += NT2) sm[e] = data[e];
    __syncthreads();
    const int lh = lb - 1;
    for (int u = 0; u < lb; u++) {
        const int tt = 1 << u;
        const int h = 1 << (logN - 1 - u);  // N / (2 tt)
        for (int x = threadIdx.x; x < TILE / 2; x += NT2) {
            const int rl = x >> lh, j = x & ((1 << lh) - 1);
            const int il = j >> u, jj = j & (tt - 1);
            const int idx = (rl << lb) + (il << (u + 1)) + jj;
            const int gi = h + (((row0 + rl) << (lb - 1 - u)) + il);
            bf_inv(&sm[idx], &sm[idx + tt], W[gi], Wp[gi], q, q2);
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < TILE; e += NT2) data[e] = sm[e];
}

// Inverse, column pass: row distances 1 .. N1/2, then the N^-1 scaling.
__global__ void __launch_bounds__(NT2) k_ntt_inv_cols(NttBatch b, const PrimeDev *__restrict__ primes,
                                                      const u64 *__restrict__ tw, const u64 *__restrict__ tw_sh,
                                                      int logN, int L, int a) {
    __shared__ u64 sm[TILE];
    const int N = 1 << logN, lb = logN - a, N2 = 1 << lb;
    const int lc = __ffs(TILE) - 1 - a, C = 1 << lc;
    const int tiles = N2 >> lc;
    const int pr = blockIdx.x / tiles, tile = blockIdx.x % tiles;
    const int p = pr / b.nr, r = b.r0 + pr % b.nr;
    if (ntt_skipped(b, p, r)) return;
    const int g = ntt_prime(b, r, L);
    const PrimeDev P = primes[g];
    const u64 q = P.q, q2 = 2 * q;
    u64 *data = b.data + (size_t)p * b.stride + (size_t)r * N + (tile << lc);
    const u64 *W = tw + (size_t)g * N, *Wp = tw_sh + (size_t)g * N;
    for (int e = threadIdx.x; e < TILE; e += NT2) sm[e] = data[((size_t)(e >> lc) << lb) + (e & (C - 1))];
    __syncthreads();
    for (int v = 0; v < a; v++) {
        const int tt = 1 << v, h = 1 << (a - 1 - v);
        for (int x = threadIdx.x; x < TILE / 2; x += NT2) {
            const int col = x & (C - 1), j = x >> lc;
            const int i = j >> v, jj = j & (tt - 1);
            const int row = (i << (v + 1)) + jj;
            bf_inv(&sm[(row << lc) + col], &sm[((row + tt) << lc) + col], W[h + i], Wp[h + i], q, q2);
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < TILE; e += NT2)
        data[((size_t)(e >> lc) << lb) + (e & (C - 1))] = mul_shoup(sm[e], P.ninv, P.ninv_sh, q);
}

copse_status launch(copse_ctx *ctx, const NttBatch &b, cudaStream_t s, bool inverse) {
    if (b.npoly <= 0 || b.nr <= 0) return COPSE_OK;
    const int N = ctx->N, logN = ctx->logN;
    const double bytes = (double)b.npoly * b.nr * N * 16.0;  // one read and one write of each residue polynomial
    if (logN >= 12) {
        const int a = logN / 2;  // column length 2^a, row length 2^(logN - a)
        const unsigned grid = (unsigned)b.npoly * (unsigned)b.nr * (unsigned)(N / TILE);
        if (inverse) {
            TIMED("ntt_inv", bytes, s, {
                k_ntt_inv_rows<<<grid, NT2, 0, s>>>(b, ctx->d_prime, ctx->d_ipsi, ctx->d_ipsi_sh, logN, ctx->L, a);
                k_ntt_inv_cols<<<grid, NT2, 0, s>>>(b, ctx->d_prime, ctx->d_ipsi, ctx->d_ipsi_sh, logN, ctx->L, a);
            });
        } else {
            TIMED("ntt_fwd", bytes, s, {
                k_ntt_fwd_cols<<<grid, NT2, 0, s>>>(b, ctx->d_prime, ctx->d_psi, ctx->d_psi_sh, logN, ctx->L, a);
                k_ntt_fwd_rows<<<grid, NT2, 0, s>>>(b, ctx->d_prime, ctx->d_psi, ctx->d_psi_sh, logN, ctx->L, a);
            });
        }
        LAUNCH_CHECK();
        return COPSE_OK;
    }
    const size_t smem = (size_t)N * sizeof(u64);
    const int threads = N / 2 < 512 ? N / 2 : 512;
    const unsigned grid = (unsigned)b.npoly * (unsigned)b.nr;
    if (inverse)
        TIMED("ntt_inv", bytes, s,
              k_ntt_inv<<<grid, threads, smem, s>>>(b, ctx->d_prime, ctx->d_ipsi, ctx->d_ipsi_sh, logN, ctx->L));
    else
        TIMED("ntt_fwd", bytes, s,
              k_ntt_fwd<<<grid, threads, smem, s>>>(b, ctx->d_prime, ctx->d_psi, ctx->d_psi_sh, logN, ctx->L));
    LAUNCH_CHECK();
    return COPSE_OK;
}

}  // namespace

copse_status ntt_forward(copse_ctx *ctx, const NttBatch &b, cudaStream_t s) { return launch(ctx, b, s, false); }
copse_status ntt_inverse(copse_ctx *ctx, const NttBatch &b, cudaStream_t s) { return launch(ctx, b, s, true); }
