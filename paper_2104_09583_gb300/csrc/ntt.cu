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
// columns) in shared memory together with every twiddle the tile needs (one
// coalesced load up front instead of a dependent global load per stage), and
// runs two stages per barrier as radix-4 butterflies in registers.  One
// polynomial spreads over N / 2048 CTAs per pass, so a launch fills the GPU
// even for a few dozen polynomials; the intermediate round trip stays in L2.
// Small rings use one CTA per polynomial.
#include <cooperative_groups.h>

#include <atomic>
#include <cstdlib>

#include "internal.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int TILE = 2048;  // coefficients per CTA in the two-pass kernels
constexpr int NT2 = 512;    // threads per CTA in the cluster and most two-pass kernels (radix-4 passes: one unit of 4 per thread)
constexpr int NTT = 256;    // threads per CTA in the forward row passes (radix-8 passes: one unit of 8 per thread)

__device__ __forceinline__ int ntt_prime(const NttBatch &b, int r, int L) {
    return b.fixed >= 0 ? b.fixed : (r < b.ell ? r : L + (r - b.ell));
}

// residue r of poly p is excluded from this batch (a ModUp digit's own primes)
__device__ __forceinline__ bool ntt_skipped(const NttBatch &b, int p, int r) {
    const int j = b.skip_period > 0 ? p % b.skip_period : p;
    return b.skip_alpha > 0 && r >= j * b.skip_alpha && r < min((j + 1) * b.skip_alpha, b.ell);
}

// Forward butterfly without a correction step: the Shoup product V is below 2q for any
// 64-bit input, so x' = U + V and y' = U - V + 2q only grow by 2q per stage.  From inputs
// below q, values stay below (2 log2 N + 1) q <= 31 q < 2^60 for primes below 2^55 (the
// context's limit); the final store reduces them once (fwd_reduce).
__device__ __forceinline__ void bfv_fwd(u64 &x, u64 &y, u64 w, u64 wp, u64 q, u64 q2) {
    const u64 U = x;
    const u64 V = mul_shoup_lazy(y, w, wp, q);
    x = U + V;
    y = U - V + q2;
}

// a forward transform's output value (below 31 q) reduced to [0, q): a Shoup product by 1
__device__ __forceinline__ u64 fwd_reduce(u64 v, u64 q, u64 one_sh) {
    u64 r = mul_shoup_lazy(v, 1, one_sh, q);
    return r >= q ? r - q : r;
}

// inverse butterfly, values in [0, 2q)
__device__ __forceinline__ void bfv_inv(u64 &x, u64 &y, u64 w, u64 wp, u64 q, u64 q2) {
    const u64 U = x, V = y;
    u64 s = U + V;
    if (s >= q2) s -= q2;
    x = s;
    y = mul_shoup_lazy(U - V + q2, w, wp, q);
}

// Inverse butterfly without a correction step, for a stage whose inputs are below c (a
// multiple of q): U - V + c is positive and below 2c, so the product is the same residue,
// x' = U + V < 2c and y' < 2q.  From inputs below q, stage u of a pass takes c = 2^u q and
// its outputs stay below 2^(u+1) q; a pass of at most 8 stages stays below 2^63 for primes
// below 2^55 (the context's limit) and is reduced once before the next pass or the scaling.
__device__ __forceinline__ void bfv_inv_lazy(u64 &x, u64 &y, u64 w, u64 wp, u64 q, u64 c) {
    const u64 U = x, V = y;
    x = U + V;
    y = mul_shoup_lazy(U - V + c, w, wp, q);
}

__device__ __forceinline__ void bf_fwd(u64 *x, u64 *y, u64 w, u64 wp, u64 q, u64 q2) { bfv_fwd(*x, *y, w, wp, q, q2); }
__device__ __forceinline__ void bf_inv(u64 *x, u64 *y, u64 w, u64 wp, u64 q, u64 q2) { bfv_inv(*x, *y, w, wp, q, q2); }

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
        data[i] = fwd_reduce(v, q, primes[g].one_sh);
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
    const Shoup sc = b.scale ? b.scale[r - b.r0] : Shoup{P.ninv, P.ninv_sh};
    for (int i = threadIdx.x; i < N; i += blockDim.x) data[i] = mul_shoup(sm[i], sc, q);
}

// ---------------------------------------------------------------- two passes (N = N1 x N2)
// A tile holds TILE / S independent sequences of length S = 2^ls (columns of a
// column tile, rows of a row tile); element i of sequence g sits at sm[IX(g, i)].
// TW(u, g, il) is the shared-memory index of the twiddle of local stage u and
// local group il of sequence g.

// forward stages 0 .. ls-1 of every sequence: radix-4 pairs of stages, then a radix-2 stage if ls is odd
// work item x -> (sequence g, index j within the sequence's 2^nb items); when the
// sequences are columns of a row-major tile, consecutive threads take consecutive
// columns so that a warp touches consecutive words (no bank conflicts)
template <bool SEQ_FAST>
__device__ __forceinline__ void split_item(int x, int ls, int nb, int &g, int &j) {
    if (SEQ_FAST) {
        const int lg = 11 - ls;  // log2 of the number of sequences in the tile
        g = x & ((1 << lg) - 1);
        j = x >> lg;
    } else {
        g = x >> nb;
        j = x & ((1 << nb) - 1);
    }
}

// One radix-8 pass of the forward transform: stages u, u + 1, u + 2 (half-distances 4 q8, 2 q8,
// q8 with q8 = 2^(ls - 3 - u)) of every sequence, eight coefficients i0 + m q8 in registers;
// the butterflies and twiddles are those of three radix-2 stages.
template <bool SEQ_FAST, int NT, class IX, class TWI>
__device__ __forceinline__ void pass_fwd8(u64 *sm, const u64 *tw, const u64 *twp, int ls, int u, u64 q, u64 q2, IX ix,
                                          TWI twi) {
    const int lt = ls - 1 - u, q8 = 1 << (lt - 2);
    for (int x = threadIdx.x; x < TILE / 8; x += NT) {
        int g, jq;
        split_item<SEQ_FAST>(x, ls, ls - 3, g, jq);
        const int il = jq >> (lt - 2), jj = jq & (q8 - 1);
        const int i0 = (il << (lt + 1)) + jj;
        int a[8];
        u64 v[8];
#pragma unroll
        for (int m = 0; m < 8; m++) {
            a[m] = ix(g, i0 + m * q8);
            v[m] = sm[a[m]];
        }
        {
            const int t = twi(u, g, il);
            const u64 w = tw[t], wp = twp[t];
#pragma unroll
            for (int m = 0; m < 4; m++) bfv_fwd(v[m], v[m + 4], w, wp, q, q2);
        }
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int t = twi(u + 1, g, 2 * il + h);
            const u64 w = tw[t], wp = twp[t];
            bfv_fwd(v[4 * h], v[4 * h + 2], w, wp, q, q2);
            bfv_fwd(v[4 * h + 1], v[4 * h + 3], w, wp, q, q2);
        }
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const int t = twi(u + 2, g, 4 * il + k);
            bfv_fwd(v[2 * k], v[2 * k + 1], tw[t], twp[t], q, q2);
        }
#pragma unroll
        for (int m = 0; m < 8; m++) sm[a[m]] = v[m];
    }
    __syncthreads();
}

// forward stages 0 .. ls-1 of every sequence: radix-8 passes (R8), then radix-4 pairs of stages,
// then a radix-2 stage if one is left; NT threads
template <bool SEQ_FAST, int NT, bool R8, class IX, class TWI>
__device__ __forceinline__ void tile_fwd(u64 *sm, const u64 *tw, const u64 *twp, int ls, u64 q, u64 q2, IX ix,
                                         TWI twi) {
    int u = 0;
    if (R8)
        for (; u + 2 < ls; u += 3) pass_fwd8<SEQ_FAST, NT>(sm, tw, twp, ls, u, q, q2, ix, twi);
#pragma unroll
    for (; u + 1 < ls; u += 2) {
        const int lt = ls - 1 - u, tt = 1 << lt, h2 = tt >> 1;
        for (int x = threadIdx.x; x < TILE / 4; x += NT) {
            int g, jq;
            split_item<SEQ_FAST>(x, ls, ls - 2, g, jq);
            const int il = jq >> (lt - 1), jj = jq & (h2 - 1);
            const int i0 = (il << (lt + 1)) + jj;
            const int a0 = ix(g, i0), a1 = ix(g, i0 + h2), a2 = ix(g, i0 + tt), a3 = ix(g, i0 + tt + h2);
            u64 v0 = sm[a0], v1 = sm[a1], v2 = sm[a2], v3 = sm[a3];
            const int t0 = twi(u, g, il);
            bfv_fwd(v0, v2, tw[t0], twp[t0], q, q2);
            bfv_fwd(v1, v3, tw[t0], twp[t0], q, q2);
            const int ta = twi(u + 1, g, 2 * il), tb = twi(u + 1, g, 2 * il + 1);
            bfv_fwd(v0, v1, tw[ta], twp[ta], q, q2);
            bfv_fwd(v2, v3, tw[tb], twp[tb], q, q2);
            sm[a0] = v0;
            sm[a1] = v1;
            sm[a2] = v2;
            sm[a3] = v3;
        }
        __syncthreads();
    }
    if (u < ls) {  // last stage, distance 1
        for (int x = threadIdx.x; x < TILE / 2; x += NT) {
            int g, il;
            split_item<SEQ_FAST>(x, ls, ls - 1, g, il);
            const int a0 = ix(g, 2 * il), a1 = ix(g, 2 * il + 1);
            const int t0 = twi(u, g, il);
            bf_fwd(&sm[a0], &sm[a1], tw[t0], twp[t0], q, q2);
        }
        __syncthreads();
    }
}

// One radix-8 pass of the inverse transform: stages u, u + 1, u + 2 (distances 2^u, 2^(u+1),
// 2^(u+2)), eight coefficients i0 + m 2^u in registers; stage u + k subtracts against 2^(u+k) q.
template <bool SEQ_FAST, int NT, class IX, class TWI>
__device__ __forceinline__ void pass_inv8(u64 *sm, const u64 *tw, const u64 *twp, int ls, int u, u64 q, IX ix,
                                          TWI twi) {
    const int tt = 1 << u;
    for (int x = threadIdx.x; x < TILE / 8; x += NT) {
        int g, jq;
        split_item<SEQ_FAST>(x, ls, ls - 3, g, jq);
        const int il = jq >> u, jj = jq & (tt - 1);
        const int i0 = (il << (u + 3)) + jj;
        int a[8];
        u64 v[8];
#pragma unroll
        for (int m = 0; m < 8; m++) {
            a[m] = ix(g, i0 + m * tt);
            v[m] = sm[a[m]];
        }
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const int t = twi(u, g, 4 * il + k);
            bfv_inv_lazy(v[2 * k], v[2 * k + 1], tw[t], twp[t], q, q << u);
        }
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int t = twi(u + 1, g, 2 * il + h);
            const u64 w = tw[t], wp = twp[t];
            bfv_inv_lazy(v[4 * h], v[4 * h + 2], w, wp, q, q << (u + 1));
            bfv_inv_lazy(v[4 * h + 1], v[4 * h + 3], w, wp, q, q << (u + 1));
        }
        {
            const int t = twi(u + 2, g, il);
            const u64 w = tw[t], wp = twp[t];
#pragma unroll
            for (int m = 0; m < 4; m++) bfv_inv_lazy(v[m], v[m + 4], w, wp, q, q << (u + 2));
        }
#pragma unroll
        for (int m = 0; m < 8; m++) sm[a[m]] = v[m];
    }
    __syncthreads();
}

// inverse stages (distances 1, 2, .., S/2) of every sequence: radix-8 passes (R8), then radix-4,
// then radix-2; NT threads
template <bool SEQ_FAST, int NT, bool R8, class IX, class TWI>
__device__ __forceinline__ void tile_inv(u64 *sm, const u64 *tw, const u64 *twp, int ls, u64 q, u64 q2, IX ix,
                                         TWI twi) {
    int u = 0;
    if (R8)
        for (; u + 2 < ls; u += 3) pass_inv8<SEQ_FAST, NT>(sm, tw, twp, ls, u, q, ix, twi);
#pragma unroll
    for (; u + 1 < ls; u += 2) {
        const int tt = 1 << u;
        for (int x = threadIdx.x; x < TILE / 4; x += NT) {
            int g, jq;
            split_item<SEQ_FAST>(x, ls, ls - 2, g, jq);
            const int il1 = jq >> u, jj = jq & (tt - 1);
            const int i0 = (il1 << (u + 2)) + jj;
            const int a0 = ix(g, i0), a1 = ix(g, i0 + tt), a2 = ix(g, i0 + 2 * tt), a3 = ix(g, i0 + 3 * tt);
            u64 v0 = sm[a0], v1 = sm[a1], v2 = sm[a2], v3 = sm[a3];
            const int ta = twi(u, g, 2 * il1), tb = twi(u, g, 2 * il1 + 1);
            const u64 c0 = q << u, c1 = q << (u + 1);
            bfv_inv_lazy(v0, v1, tw[ta], twp[ta], q, c0);
            bfv_inv_lazy(v2, v3, tw[tb], twp[tb], q, c0);
            const int t1 = twi(u + 1, g, il1);
            bfv_inv_lazy(v0, v2, tw[t1], twp[t1], q, c1);
            bfv_inv_lazy(v1, v3, tw[t1], twp[t1], q, c1);
            sm[a0] = v0;
            sm[a1] = v1;
            sm[a2] = v2;
            sm[a3] = v3;
        }
        __syncthreads();
    }
    if (u < ls) {  // last stage, distance S/2, one group
        const int tt = 1 << u;
        for (int x = threadIdx.x; x < TILE / 2; x += NT) {
            int g, j;
            split_item<SEQ_FAST>(x, ls, ls - 1, g, j);
            const int a0 = ix(g, j), a1 = ix(g, j + tt);
            const int t0 = twi(u, g, 0);
            bfv_inv_lazy(sm[a0], sm[a1], tw[t0], twp[t0], q, q << u);
        }
        __syncthreads();
    }
}

struct TileCtx {
    int p, r, g, tile;
    u64 q, q2;
};

__device__ __forceinline__ bool tile_ctx(const NttBatch &b, const PrimeDev *primes, int L, int tiles, TileCtx &t) {
    const int pr = blockIdx.x / tiles;
    t.tile = blockIdx.x % tiles;
    t.p = pr / b.nr;
    t.r = b.r0 + pr % b.nr;
    if (ntt_skipped(b, t.p, t.r)) return false;
    t.g = ntt_prime(b, t.r, L);
    t.q = primes[t.g].q;
    t.q2 = 2 * t.q;
    return true;
}

// Column pass: tile = C consecutive columns x all N1 rows, stored row-major [row][C].
__global__ void __launch_bounds__(NT2) k_ntt_fwd_cols(NttBatch b, const PrimeDev *__restrict__ primes,
                                                      const u64 *__restrict__ tw, const u64 *__restrict__ tw_sh,
                                                      int logN, int L, int a) {
    __shared__ u64 sm[TILE], stw[TILE], stwp[TILE];
    const int N = 1 << logN, lb = logN - a, lc = 11 - a, C = 1 << lc;
    TileCtx t;
    if (!tile_ctx(b, primes, L, (1 << lb) >> lc, t)) return;
    u64 *data = b.data + (size_t)t.p * b.stride + (size_t)t.r * N + (t.tile << lc);
    const u64 *W = tw + (size_t)t.g * N, *Wp = tw_sh + (size_t)t.g * N;
    for (int e = threadIdx.x; e < TILE; e += NT2) {
        sm[e] = data[((size_t)(e >> lc) << lb) + (e & (C - 1))];
        if (e < (1 << a)) {
            stw[e] = W[e];
            stwp[e] = Wp[e];
        }
    }
    __syncthreads();
    tile_fwd<true, NT2, false>(sm, stw, stwp, a, t.q, t.q2, [&](int g, int i) { return (i << lc) + g; },
             [&](int u, int, int il) { return (1 << u) + il; });
    for (int e = threadIdx.x; e < TILE; e += NT2) data[((size_t)(e >> lc) << lb) + (e & (C - 1))] = sm[e];
}

// Row pass: tile = R consecutive rows of N2 contiguous coefficients; the twiddle
// of row g, stage u, group il is W[2^(a+u) + ((row0 + g) << u) + il].
__global__ void __launch_bounds__(NTT, 4) k_ntt_fwd_rows(NttBatch b, const PrimeDev *__restrict__ primes,
                                                      const ulonglong2 *__restrict__ stg, int logN, int L, int a) {
    __shared__ u64 sm[TILE], stw[TILE], stwp[TILE];
    const int N = 1 << logN, lb = logN - a, lr = 11 - lb;
    TileCtx t;
    if (!tile_ctx(b, primes, L, 1 << (a - lr), t)) return;
    const int row0 = t.tile << lr;
    u64 *data = b.data + (size_t)t.p * b.stride + (size_t)t.r * N + ((size_t)row0 << lb);
    // stage u needs R << u consecutive twiddles from 2^(a+u) + (row0 << u), stored at R (2^u - 1):
    // pre-staged per tile, loaded together with the data
    const ulonglong2 *st = stg + ((size_t)t.g * (N / TILE) + t.tile) * TILE;
    const int nst = TILE - (1 << lr);
    for (int e = threadIdx.x; e < TILE; e += NTT) {
        sm[e] = data[e];
        if (e < nst) {
            const ulonglong2 v = st[e];
            stw[e] = v.x;
            stwp[e] = v.y;
        }
    }
    __syncthreads();
    tile_fwd<false, NTT, true>(sm, stw, stwp, lb, t.q, t.q2, [&](int g, int i) { return (g << lb) + i; },
             [&](int u, int g, int il) { return ((1 << lr) * ((1 << u) - 1)) + (g << u) + il; });
    for (int e = threadIdx.x; e < TILE; e += NTT) {
        data[e] = fwd_reduce(sm[e], t.q, primes[t.g].one_sh);
    }
}

// Inverse row pass (first): twiddle of row g, stage u, group il is
// W[2^(logN-1-u) + ((row0 + g) << (lb-1-u)) + il].
__global__ void __launch_bounds__(NT2) k_ntt_inv_rows(NttBatch b, const PrimeDev *__restrict__ primes,
                                                      const ulonglong2 *__restrict__ stg, int logN, int L, int a) {
    __shared__ u64 sm[TILE], stw[TILE], stwp[TILE];
    const int N = 1 << logN, lb = logN - a, lr = 11 - lb;
    TileCtx t;
    if (!tile_ctx(b, primes, L, 1 << (a - lr), t)) return;
    const int row0 = t.tile << lr;
    u64 *data = b.data + (size_t)t.p * b.stride + (size_t)t.r * N + ((size_t)row0 << lb);
    // stage u needs R << (lb-1-u) twiddles from 2^(logN-1-u) + (row0 << (lb-1-u)), stored after
    // those of the earlier stages: pre-staged per tile, loaded together with the data
    const ulonglong2 *st = stg + ((size_t)t.g * (N / TILE) + t.tile) * TILE;
    const int nst = TILE - (1 << lr);
    for (int e = threadIdx.x; e < TILE; e += NT2) {
        sm[e] = data[e];
        if (e < nst) {
            const ulonglong2 v = st[e];
            stw[e] = v.x;
            stwp[e] = v.y;
        }
    }
    __syncthreads();
    // offset of stage u: sum_{v<u} R 2^(lb-1-v) = R (2^lb - 2^(lb-u))
    tile_inv<false, NT2, false>(sm, stw, stwp, lb, t.q, t.q2, [&](int g, int i) { return (g << lb) + i; },
             [&](int u, int g, int il) {
                 return (1 << lr) * ((1 << lb) - (1 << (lb - u))) + (g << (lb - 1 - u)) + il;
             });
    const u64 one_sh = primes[t.g].one_sh;
    for (int e = threadIdx.x; e < TILE; e += NT2) data[e] = fwd_reduce(sm[e], t.q, one_sh);
}

// Inverse column pass: twiddle of stage u, group il is W[2^(a-1-u) + il]; then N^-1.
__global__ void __launch_bounds__(NT2) k_ntt_inv_cols(NttBatch b, const PrimeDev *__restrict__ primes,
                                                      const u64 *__restrict__ tw, const u64 *__restrict__ tw_sh,
                                                      int logN, int L, int a) {
    __shared__ u64 sm[TILE], stw[TILE], stwp[TILE];
    const int N = 1 << logN, lb = logN - a, lc = 11 - a, C = 1 << lc;
    TileCtx t;
    if (!tile_ctx(b, primes, L, (1 << lb) >> lc, t)) return;
    const PrimeDev P = primes[t.g];
    u64 *data = b.data + (size_t)t.p * b.stride + (size_t)t.r * N + (t.tile << lc);
    const u64 *W = tw + (size_t)t.g * N, *Wp = tw_sh + (size_t)t.g * N;
    for (int e = threadIdx.x; e < TILE; e += NT2) {
        sm[e] = data[((size_t)(e >> lc) << lb) + (e & (C - 1))];
        if (e < (1 << a)) {
            stw[e] = W[e];
            stwp[e] = Wp[e];
        }
    }
    __syncthreads();
    tile_inv<true, NT2, false>(sm, stw, stwp, a, t.q, t.q2, [&](int g, int i) { return (i << lc) + g; },
             [&](int u, int, int il) { return (1 << (a - 1 - u)) + il; });
    const Shoup sc = b.scale ? b.scale[t.r - b.r0] : Shoup{P.ninv, P.ninv_sh};
    for (int e = threadIdx.x; e < TILE; e += NT2)
        data[((size_t)(e >> lc) << lb) + (e & (C - 1))] = mul_shoup(sm[e], sc, t.q);
}

// ---------------------------------------------------------------- one launch per transform (clusters)
// For 2^12 <= N <= 2^15 a thread-block cluster of CL = N / 2048 CTAs owns one
// residue polynomial.  Each CTA runs the column stages on its column tile;
// after a cluster barrier it gathers its row tile from the other CTAs' shared
// memory (distributed shared memory), a second barrier keeps every tile alive
// until all gathers are done, and it runs the row stages.  One launch and no
// round trip through L2 between the two halves of the transform.
struct ClusterSmem {
    u64 colt[TILE], rowt[TILE];  // column tile [row][C], row tile [row][N2]
    u64 stw[TILE], stwp[TILE];   // row-stage twiddles of this CTA's rows
    u64 ctw[256], ctwp[256];     // column-stage twiddles (the first N1 entries)
};

// finishing arithmetic of a modulus switch for value v = NTT(conversion) at (p, r, k)
__device__ __forceinline__ void ms_store(const MsFuse &f, const PrimeDev *pr, const KsTables &T, int L, int logN,
                                         int p, int r, size_t k, u64 v) {
    const PrimeDev P = pr[r];
    const u64 xv = f.xp[0] ? f.xp[p][((size_t)r << logN) + k] : f.x[(((size_t)p * f.ell + r) << logN) + k];
    const u64 d = mul_shoup(v, P.t_mod, P.t_mod_sh, P.q);
    u64 *o = f.outp[0] ? f.outp[p] + ((size_t)r << logN) + k : f.out + (((size_t)p * (f.ell - 1) + r) << logN) + k;
    *o = mul_shoup(sub_mod(xv, d, P.q), T.ms_qinv[(size_t)f.ell * L + r], P.q);
}

// finishing arithmetic of a ModDown for value v = NTT(conversion) at (p = 2 job + c, r, k)
__device__ __forceinline__ void md_store(const MdFuse &f, const PrimeDev *pr, const KsTables &T, int logN, int p,
                                         int r, size_t k, u64 v) {
    const int job = p >> 1, c = p & 1;
    const PrimeDev P = pr[r];
    const u64 uv = f.U[(size_t)p * f.ustride + ((size_t)r << logN) + k];
    u64 res = mul_shoup(sub_mod(uv, mul_shoup(v, P.t_mod, P.t_mod_sh, P.q), P.q), T.md_Pinv[r], P.q);
    if (c < f.add_comps && f.add[job]) {
        const size_t src = (c == 0 && f.gal[job] != 1) ? galois_src((uint32_t)k, f.gal[job], logN) : k;
        res = add_mod(res, f.add[job][(size_t)c * f.acomp + ((size_t)r << logN) + src], P.q);
    }
    f.out[job][(size_t)c * f.ocomp + ((size_t)r << logN) + k] = res;
}

// conversion of polynomial p's residues ell-1 .. ell+alpha-1 (basis of q_{ell-1} P) to q_r
__device__ __forceinline__ u64 mdd_load(const MddFuse &f, const PrimeDev *pr, const KsTables &T, int L, int alpha,
                                        int logN, int p, int r, size_t n) {
    const int nb = alpha + 1, ell = f.ell;
    const u64 *up = f.U + (size_t)p * f.ustride;
    const u64 qi = pr[r].q;
    u64 acc = 0;
    for (int k = 0; k < nb; k++) {
        const u64 bk = k == 0 ? pr[ell - 1].q : pr[L + k - 1].q;
        const u64 y = up[((size_t)(ell - 1 + k) << logN) + n];  // [U_k (B/b_k)^-1 / t]_{b_k}: scaled by the inverse transform
        u64 v = mul_shoup(y, T.mdd_hat[((size_t)ell * nb + k) * L + r], qi);
        if (y > (bk - 1) / 2) v = sub_mod(v, T.mdd_B[(size_t)ell * L + r], qi);
        acc = add_mod(acc, v, qi);
    }
    return acc;
}

__device__ __forceinline__ void mdd_store(const MddFuse &f, const PrimeDev *pr, const KsTables &T, int L, int logN,
                                          int p, int r, size_t k, u64 v) {
    const PrimeDev P = pr[r];
    const u64 uv = f.U[(size_t)p * f.ustride + ((size_t)r << logN) + k];
    u64 res = mul_shoup(sub_mod(uv, mul_shoup(v, P.t_mod, P.t_mod_sh, P.q), P.q), T.mdd_Binv[(size_t)f.ell * L + r], P.q);
    if (!f.outp[0]) {
        f.out[(((size_t)p * (f.ell - 1) + r) << logN) + k] = res;
        return;
    }
    const size_t at = (((size_t)(p & 1) * (f.ell - 1) + r) << logN) + k;
    if (f.addp[p >> 1]) res = add_mod(res, f.addp[p >> 1][at], P.q);
    f.outp[p >> 1][at] = res;
}

// Load / store of the forward cluster transform: coefficient n of residue r (global
// prime g) of batch polynomial p in; NTT-domain value v (in [0, q)) at position k out.
struct PlainIO {
    u64 *data;
    size_t stride;
    int logN;
    __device__ __forceinline__ u64 load(int p, int r, int, size_t n) const {
        return data[(size_t)p * stride + ((size_t)r << logN) + n];
    }
    __device__ __forceinline__ void store(int p, int r, int, size_t k, u64 v) const {
        data[(size_t)p * stride + ((size_t)r << logN) + k] = v;
    }
    __device__ __forceinline__ void skip(int, int, int, int) const {}
};

// out-of-place transform: residue r of polynomial p from src into dst
struct CopyIO {
    const u64 *src;
    size_t sstride;
    u64 *dst;
    size_t dstride;
    int logN;
    __device__ __forceinline__ u64 load(int p, int r, int, size_t n) const {
        return src[(size_t)p * sstride + ((size_t)r << logN) + n];
    }
    __device__ __forceinline__ void store(int p, int r, int, size_t k, u64 v) const {
        dst[(size_t)p * dstride + ((size_t)r << logN) + k] = v;
    }
    __device__ __forceinline__ void skip(int, int, int, int) const {}
};

// one residue of polynomials at separate addresses in, contiguous residues out
struct GatherIO {
    GatherSrc src;
    u64 *dst;
    int logN;
    __device__ __forceinline__ u64 load(int p, int, int, size_t n) const { return src.p[p][n]; }
    __device__ __forceinline__ void store(int p, int, int, size_t k, u64 v) const {
        dst[((size_t)p << logN) + k] = v;
    }
    __device__ __forceinline__ void skip(int, int, int, int) const {}
};

// ModUp (polynomial p = item nd + digit j, residue r of the extended basis): load the
// centred conversion of the digit's coefficient-form residues, store into
// y [item][nd][ell+alpha][N]; a digit's own residues (skipped by the transform) are
// copied from the input, which already holds them in NTT form
struct MuIO {
    const u64 *xc;     // [item][ell][N] coefficient form
    const u64 *x_ntt;  // item i at x_ntt + i * xs, [ell][N] NTT domain
    size_t xs;
    u64 *y;
    int ell, alpha, nd, L, NP, logN;
    const PrimeDev *pr;
    KsTables T;
    __device__ __forceinline__ u64 load(int p, int, int g, size_t n) const {
        const int item = p / nd, j = p - item * nd;
        const int lo = j * alpha, hi = min(lo + alpha, ell);
        const u64 qg = pr[g].q;
        const u64 *x = xc + (size_t)item * ell * ((size_t)1 << logN);
        u64 acc = 0;
        for (int i = lo; i < hi; i++) {
            const u64 qi = pr[i].q;
            const u64 v = x[((size_t)i << logN) + n];  // already times modup_inv (inverse transform's scale)
            const size_t ti = ((size_t)ell * L + i) * NP + g;
            u64 w = mul_shoup(v, T.modup_hat[ti], qg);
            if (v > (qi - 1) / 2) w = sub_mod(w, T.modup_qhat[ti], qg);
            acc = add_mod(acc, w, qg);
        }
        return acc;
    }
    __device__ __forceinline__ void store(int p, int r, int, size_t k, u64 v) const {
        y[(((size_t)p * (ell + alpha) + r) << logN) + k] = v;
    }
    __device__ __forceinline__ void skip(int p, int r, int rank, int cl) const {
        const int item = p / nd;
        const size_t n = (size_t)1 << logN, part = n / cl, k0 = (size_t)rank * part;
        const u64 *src = x_ntt + (size_t)item * xs + ((size_t)r << logN) + k0;
        u64 *dst = y + (((size_t)p * (ell + alpha) + r) << logN) + k0;
        for (size_t k = threadIdx.x; k < part; k += blockDim.x) dst[k] = src[k];
    }
};

// modulus switch: load the centred conversion of the last prime's residue, store the finish
struct MsIO {
    MsFuse f;
    const PrimeDev *pr;
    KsTables T;
    int L, logN;
    __device__ __forceinline__ u64 load(int p, int r, int, size_t n) const {
        const u64 ql = pr[f.ell - 1].q;
        const u64 w = f.last[((size_t)p << logN) + n];  // already times t^-1 (inverse transform's scale)
        // |centred w| < q_{ell-1}/2 < q_r: the chain is in decreasing order
        return w > (ql - 1) / 2 ? pr[r].q - (ql - w) : w;
    }
    __device__ __forceinline__ void store(int p, int r, int, size_t k, u64 v) const {
        ms_store(f, pr, T, L, logN, p, r, k, v);
    }
    __device__ __forceinline__ void skip(int, int, int, int) const {}
};

// ModDown: load the conversion of the alpha special residues, store the finish
struct MdIO {
    MdFuse f;
    const PrimeDev *pr;
    KsTables T;
    int L, alpha, logN;
    __device__ __forceinline__ u64 load(int p, int r, int, size_t n) const {
        const u64 *up = f.U + (size_t)p * f.ustride;
        const u64 qi = pr[r].q;
        u64 acc = 0;
        for (int k = 0; k < alpha; k++) {
            const u64 pk = pr[L + k].q;
            const u64 y = up[((size_t)(f.ell + k) << logN) + n];  // already times md_inv[k] (inverse transform's scale)
            u64 v = mul_shoup(y, T.md_hat[(size_t)k * L + r], qi);
            if (y > (pk - 1) / 2) v = sub_mod(v, T.md_P[r], qi);
            acc = add_mod(acc, v, qi);
        }
        return acc;
    }
    __device__ __forceinline__ void store(int p, int r, int, size_t k, u64 v) const {
        md_store(f, pr, T, logN, p, r, k, v);
    }
    __device__ __forceinline__ void skip(int, int, int, int) const {}
};

// relinearise-and-drop ModDown: load the conversion from the q_{ell-1} P basis, store the finish
struct MddIO {
    MddFuse f;
    const PrimeDev *pr;
    KsTables T;
    int L, alpha, logN;
    __device__ __forceinline__ u64 load(int p, int r, int, size_t n) const {
        return mdd_load(f, pr, T, L, alpha, logN, p, r, n);
    }
    __device__ __forceinline__ void store(int p, int r, int, size_t k, u64 v) const {
        mdd_store(f, pr, T, L, logN, p, r, k, v);
    }
    __device__ __forceinline__ void skip(int, int, int, int) const {}
};

// ---------------------------------------------------------------- a thread's coefficients of a tile
// A thread of the forward kernels loads K coefficients n0 + i dn (i < K) of one residue
// polynomial and stores K results k0 + i dk.  By default each goes through the functor's
// load / store; the fused conversions and finishes below take all K together, their
// per-tile constants loaded once and every global load of a step in flight at once.
template <int K, class IO>
__device__ __forceinline__ void load_n(const IO &io, int p, int r, int g, size_t n0, size_t dn, u64 (&v)[K]) {
#pragma unroll
    for (int i = 0; i < K; i++) v[i] = io.load(p, r, g, n0 + (size_t)i * dn);
}
template <int K, class IO>
__device__ __forceinline__ void store_n(const IO &io, int p, int r, int g, size_t k0, size_t dk, const u64 (&v)[K]) {
#pragma unroll
    for (int i = 0; i < K; i++) io.store(p, r, g, k0 + (size_t)i * dk, v[i]);
}

// A base conversion sum_k [y_k]_centred * f_k mod q as one lazy sum: with f_k in Montgomery form
// F_k = f_k 2^64 mod q and C = (-c) 2^64 mod q for the correction c of a centred negative digit,
// S = sum_k (y_k F_k + [y_k > (b_k - 1) / 2] C) is summed exactly in 128 bits and reduced once,
// S 2^-64 mod q (Montgomery).  S < m 2^(2 bits) + m q < q 2^64 for m < 2^(63 - bits) terms of
// residues below 2^bits (bits <= 55: any m up to 256).
__device__ __forceinline__ void add128(Acc128 &a, u64 x) {
    a.lo += x;
    a.hi += a.lo < x;
}
template <int K>
__device__ __forceinline__ void conv_term(Acc128 (&s)[K], const u64 (&y)[K], u64 F, u64 C, u64 half) {
#pragma unroll
    for (int i = 0; i < K; i++) {
        mac128(s[i], y[i], F);
        add128(s[i], y[i] > half ? C : 0);
    }
}

template <int K>
__device__ __forceinline__ void load_n(const MuIO &io, int p, int, int g, size_t n0, size_t dn, u64 (&v)[K]) {
    const int item = p / io.nd, j = p - item * io.nd;
    const int lo = j * io.alpha, hi = min(lo + io.alpha, io.ell);
    const u64 *x = io.xc + (size_t)item * io.ell * ((size_t)1 << io.logN) + n0;
    Acc128 s[K];
#pragma unroll
    for (int i = 0; i < K; i++) s[i] = Acc128{0, 0};
    for (int i = lo; i < hi; i++) {
        const size_t ti = ((size_t)io.ell * io.L + i) * io.NP + g;
        const u64 *xi = x + ((size_t)i << io.logN);
        u64 y[K];
#pragma unroll
        for (int k = 0; k < K; k++) y[k] = xi[(size_t)k * dn];  // already times modup_inv (the inverse transform's scale)
        conv_term(s, y, io.T.modup_hat_m[ti], io.T.modup_negq_m[ti], (io.pr[i].q - 1) / 2);
    }
    const PrimeDev P = io.pr[g];
#pragma unroll
    for (int i = 0; i < K; i++) v[i] = mont_reduce(s[i], P);
}

template <int K>
__device__ __forceinline__ void load_n(const MdIO &io, int p, int r, int, size_t n0, size_t dn, u64 (&v)[K]) {
    const u64 *up = io.f.U + (size_t)p * io.f.ustride + ((size_t)io.f.ell << io.logN) + n0;
    const u64 C = io.T.md_negP_m[r];
    Acc128 s[K];
#pragma unroll
    for (int i = 0; i < K; i++) s[i] = Acc128{0, 0};
    for (int k = 0; k < io.alpha; k++) {
        const u64 *yk = up + ((size_t)k << io.logN);
        u64 y[K];
#pragma unroll
        for (int i = 0; i < K; i++) y[i] = yk[(size_t)i * dn];  // already times md_inv[k] (the inverse transform's scale)
        conv_term(s, y, io.T.md_hat_m[(size_t)k * io.L + r], C, (io.pr[io.L + k].q - 1) / 2);
    }
    const PrimeDev P = io.pr[r];
#pragma unroll
    for (int i = 0; i < K; i++) v[i] = mont_reduce(s[i], P);
}

template <int K>
__device__ __forceinline__ void load_n(const MddIO &io, int p, int r, int, size_t n0, size_t dn, u64 (&v)[K]) {
    const int ell = io.f.ell, nb = io.alpha + 1;
    const u64 *up = io.f.U + (size_t)p * io.f.ustride + ((size_t)(ell - 1) << io.logN) + n0;
    const u64 C = io.T.mdd_negB_m[(size_t)ell * io.L + r];
    Acc128 s[K];
#pragma unroll
    for (int i = 0; i < K; i++) s[i] = Acc128{0, 0};
    for (int k = 0; k < nb; k++) {
        const u64 bk = k == 0 ? io.pr[ell - 1].q : io.pr[io.L + k - 1].q;
        const u64 *yk = up + ((size_t)k << io.logN);
        u64 y[K];
#pragma unroll
        for (int i = 0; i < K; i++) y[i] = yk[(size_t)i * dn];  // scaled by the inverse transform
        conv_term(s, y, io.T.mdd_hat_m[((size_t)ell * nb + k) * io.L + r], C, (bk - 1) / 2);
    }
    const PrimeDev P = io.pr[r];
#pragma unroll
    for (int i = 0; i < K; i++) v[i] = mont_reduce(s[i], P);
}

template <int K>
__device__ __forceinline__ void load_n(const MsIO &io, int p, int r, int, size_t n0, size_t dn, u64 (&v)[K]) {
    const u64 ql = io.pr[io.f.ell - 1].q, qr = io.pr[r].q, half = (ql - 1) / 2;
    const u64 *w = io.f.last + ((size_t)p << io.logN) + n0;  // already times t^-1
#pragma unroll
    for (int i = 0; i < K; i++) {
        const u64 x = w[(size_t)i * dn];
        v[i] = x > half ? qr - (ql - x) : x;  // |centred x| < q_{ell-1} / 2 < q_r
    }
}

// the finishes of ms_store, md_store and mdd_store for K positions of one residue
template <int K>
__device__ __forceinline__ void store_n(const MsIO &io, int p, int r, int, size_t k0, size_t dk, const u64 (&v)[K]) {
    const MsFuse &f = io.f;
    const u64 q = io.pr[r].q;
    const Shoup tm{io.pr[r].t_mod, io.pr[r].t_mod_sh}, qinv = io.T.ms_qinv[(size_t)f.ell * io.L + r];
    const u64 *x = (f.xp[0] ? f.xp[p] : f.x + (size_t)p * f.ell * ((size_t)1 << io.logN)) + ((size_t)r << io.logN);
    u64 *o = (f.outp[0] ? f.outp[p] : f.out + (size_t)p * (f.ell - 1) * ((size_t)1 << io.logN)) + ((size_t)r << io.logN);
    u64 xv[K];
#pragma unroll
    for (int i = 0; i < K; i++) xv[i] = x[k0 + (size_t)i * dk];
#pragma unroll
    for (int i = 0; i < K; i++) o[k0 + (size_t)i * dk] = mul_shoup(sub_mod(xv[i], mul_shoup(v[i], tm, q), q), qinv, q);
}

template <int K>
__device__ __forceinline__ void store_n(const MdIO &io, int p, int r, int, size_t k0, size_t dk, const u64 (&v)[K]) {
    const MdFuse &f = io.f;
    const int job = p >> 1, c = p & 1;
    const u64 q = io.pr[r].q;
    const Shoup tm{io.pr[r].t_mod, io.pr[r].t_mod_sh}, pinv = io.T.md_Pinv[r];
    const u64 *U = f.U + (size_t)p * f.ustride + ((size_t)r << io.logN);
    u64 res[K];
#pragma unroll
    for (int i = 0; i < K; i++) res[i] = U[k0 + (size_t)i * dk];
#pragma unroll
    for (int i = 0; i < K; i++) res[i] = mul_shoup(sub_mod(res[i], mul_shoup(v[i], tm, q), q), pinv, q);
    if (c < f.add_comps && f.add[job]) {
        const u64 *a = f.add[job] + (size_t)c * f.acomp + ((size_t)r << io.logN);
        const u64 gal = f.gal[job];
        u64 av[K];
#pragma unroll
        for (int i = 0; i < K; i++) {
            const size_t k = k0 + (size_t)i * dk;
            av[i] = a[(c == 0 && gal != 1) ? (size_t)galois_src((uint32_t)k, gal, io.logN) : k];
        }
#pragma unroll
        for (int i = 0; i < K; i++) res[i] = add_mod(res[i], av[i], q);
    }
    u64 *out = f.out[job] + (size_t)c * f.ocomp + ((size_t)r << io.logN);
#pragma unroll
    for (int i = 0; i < K; i++) out[k0 + (size_t)i * dk] = res[i];
}

template <int K>
__device__ __forceinline__ void store_n(const MddIO &io, int p, int r, int, size_t k0, size_t dk, const u64 (&v)[K]) {
    const MddFuse &f = io.f;
    const u64 q = io.pr[r].q;
    const size_t n = (size_t)1 << io.logN;
    const Shoup tm{io.pr[r].t_mod, io.pr[r].t_mod_sh}, binv = io.T.mdd_Binv[(size_t)f.ell * io.L + r];
    const u64 *U = f.U + (size_t)p * f.ustride + ((size_t)r << io.logN);
    u64 res[K];
#pragma unroll
    for (int i = 0; i < K; i++) res[i] = U[k0 + (size_t)i * dk];
#pragma unroll
    for (int i = 0; i < K; i++) res[i] = mul_shoup(sub_mod(res[i], mul_shoup(v[i], tm, q), q), binv, q);
    u64 *out;
    if (!f.outp[0]) {
        out = f.out + ((size_t)p * (f.ell - 1) + r) * n;
    } else {
        const size_t at = ((size_t)(p & 1) * (f.ell - 1) + r) * n;
        const u64 *add = f.addp[p >> 1];
        if (add) {
            u64 av[K];
#pragma unroll
            for (int i = 0; i < K; i++) av[i] = add[at + k0 + (size_t)i * dk];
#pragma unroll
            for (int i = 0; i < K; i++) res[i] = add_mod(res[i], av[i], q);
        }
        out = f.outp[p >> 1] + at;
    }
#pragma unroll
    for (int i = 0; i < K; i++) out[k0 + (size_t)i * dk] = res[i];
}

template <int CL, class IO>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(NT2)
    k_ntt_fwd_cluster(NttBatch b, const PrimeDev *__restrict__ primes, const u64 *__restrict__ tw,
                      const u64 *__restrict__ tw_sh, const ulonglong2 *__restrict__ stg, int, int L, int, IO io) {
    extern __shared__ __align__(16) u64 dyn_smem[];
    ClusterSmem &S = *reinterpret_cast<ClusterSmem *>(dyn_smem);
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    // the cluster size fixes the ring degree (CL x 2048 coefficients): every tile shape is a
    // compile-time constant, so the radix-4 passes and their index arithmetic unroll
    constexpr int logN = CL == 2 ? 12 : (CL == 4 ? 13 : (CL == 8 ? 14 : 15)), a = logN / 2;
    constexpr int lb = logN - a, N2 = 1 << lb, lc = 11 - a, C = 1 << lc, lr = 11 - lb;
    const int pr = blockIdx.x / CL;
    const int p = pr / b.nr, r = b.r0 + pr % b.nr;
    if (ntt_skipped(b, p, r)) {  // the same for every CTA of the cluster
        io.skip(p, r, rank, CL);
        return;
    }
    const int g = ntt_prime(b, r, L);
    const u64 q = primes[g].q, q2 = 2 * q, one_sh = primes[g].one_sh;
    const size_t N = (size_t)1 << logN;
    const u64 *W = tw + (size_t)g * N, *Wp = tw_sh + (size_t)g * N;
    // the tile, this CTA's row-stage twiddles (pre-staged, one 16-byte load each) and the
    // column-stage twiddles, all loads of a thread in flight together
    const ulonglong2 *st = stg + ((size_t)g * CL + rank) * TILE;
    const int nst = TILE - (1 << lr);
    {
        // coefficient e + i NT2 of the tile is n0 + i dn (NT2 is a multiple of the tile's width C)
        const int e = threadIdx.x;
        u64 v[TILE / NT2];
        load_n(io, p, r, g, (size_t)(rank << lc) + ((size_t)(e >> lc) << lb) + (e & (C - 1)), (size_t)(NT2 >> lc) << lb, v);
#pragma unroll
        for (int i = 0; i < TILE / NT2; i++) S.colt[e + i * NT2] = v[i];
    }
    for (int e = threadIdx.x; e < TILE; e += NT2) {
        if (e < nst) {
            const ulonglong2 v = st[e];
            S.stw[e] = v.x;
            S.stwp[e] = v.y;
        }
        if (e < (1 << a)) {
            S.ctw[e] = W[e];
            S.ctwp[e] = Wp[e];
        }
    }
    const int row0 = rank << lr;
    __syncthreads();
    tile_fwd<true, NT2, false>(S.colt, S.ctw, S.ctwp, a, q, q2, [&](int gg, int i) { return (i << lc) + gg; },
                   [&](int u, int, int il) { return (1 << u) + il; });
    cl.sync();
    for (int e = threadIdx.x; e < TILE; e += NT2) {
        const int row = row0 + (e >> lb), col = e & (N2 - 1);
        const u64 *rc = cl.map_shared_rank(S.colt, col >> lc);
        S.rowt[e] = rc[(row << lc) + (col & (C - 1))];
    }
    cl.sync();
    tile_fwd<false, NT2, false>(S.rowt, S.stw, S.stwp, lb, q, q2, [&](int gg, int i) { return (gg << lb) + i; },
                    [&](int u, int gg, int il) { return ((1 << lr) * ((1 << u) - 1)) + (gg << u) + il; });
    {
        u64 v[TILE / NT2];
#pragma unroll
        for (int i = 0; i < TILE / NT2; i++) v[i] = fwd_reduce(S.rowt[threadIdx.x + i * NT2], q, one_sh);
        store_n(io, p, r, g, ((size_t)row0 << lb) + threadIdx.x, NT2, v);
    }
}

template <int CL, class IO>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(NT2)
    k_ntt_inv_cluster(NttBatch b, const PrimeDev *__restrict__ primes, const u64 *__restrict__ tw,
                      const u64 *__restrict__ tw_sh, const ulonglong2 *__restrict__ stg, int, int L, int, IO io) {
    extern __shared__ __align__(16) u64 dyn_smem[];
    ClusterSmem &S = *reinterpret_cast<ClusterSmem *>(dyn_smem);
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    constexpr int logN = CL == 2 ? 12 : (CL == 4 ? 13 : (CL == 8 ? 14 : 15)), a = logN / 2;
    constexpr int lb = logN - a, lc = 11 - a, C = 1 << lc, lr = 11 - lb, R = 1 << lr;
    const int pr = blockIdx.x / CL;
    const int p = pr / b.nr, r = b.r0 + pr % b.nr;
    if (ntt_skipped(b, p, r)) return;
    const int g = ntt_prime(b, r, L);
    const PrimeDev P = primes[g];
    const u64 q = P.q, q2 = 2 * q;
    const size_t N = (size_t)1 << logN;
    const u64 *W = tw + (size_t)g * N, *Wp = tw_sh + (size_t)g * N;
    const int row0 = rank << lr;
    const ulonglong2 *st = stg + ((size_t)g * CL + rank) * TILE;
    const int nst = TILE - (1 << lr);
    for (int e = threadIdx.x; e < TILE; e += NT2) {
        S.rowt[e] = io.load(p, r, g, ((size_t)row0 << lb) + e);
        if (e < nst) {
            const ulonglong2 v = st[e];
            S.stw[e] = v.x;
            S.stwp[e] = v.y;
        }
        if (e < (1 << a)) {
            S.ctw[e] = W[e];
            S.ctwp[e] = Wp[e];
        }
    }
    __syncthreads();
    tile_inv<false, NT2, false>(S.rowt, S.stw, S.stwp, lb, q, q2, [&](int gg, int i) { return (gg << lb) + i; },
                    [&](int u, int gg, int il) {
                        return (1 << lr) * ((1 << lb) - (1 << (lb - u))) + (gg << (lb - 1 - u)) + il;
                    });
    for (int e = threadIdx.x; e < TILE; e += NT2) S.rowt[e] = fwd_reduce(S.rowt[e], q, P.one_sh);
    cl.sync();
    for (int e = threadIdx.x; e < TILE; e += NT2) {
        const int row = e >> lc, col = (rank << lc) + (e & (C - 1));
        const u64 *rc = cl.map_shared_rank(S.rowt, row >> lr);
        S.colt[e] = rc[((row & (R - 1)) << lb) + col];
    }
    cl.sync();
    tile_inv<true, NT2, false>(S.colt, S.ctw, S.ctwp, a, q, q2, [&](int gg, int i) { return (i << lc) + gg; },
                   [&](int u, int, int il) { return (1 << (a - 1 - u)) + il; });
    const Shoup sc = b.scale ? b.scale[r - b.r0] : Shoup{P.ninv, P.ninv_sh};
    for (int e = threadIdx.x; e < TILE; e += NT2)
        io.store(p, r, g, (size_t)(rank << lc) + ((size_t)(e >> lc) << lb) + (e & (C - 1)),
                 mul_shoup(S.colt[e], sc, q));
}

// The dynamic shared-memory limit is a per-device function attribute: each kernel
// instantiation keeps one bit per device (set after the attribute is raised on that
// device).  Threads that race here both raise it, which is harmless.
inline bool attr_pending(std::atomic<uint64_t> &mask, int device) {
    return device < 0 || device >= 64 || !(mask.load(std::memory_order_acquire) & (1ull << device));
}
inline void attr_done(std::atomic<uint64_t> &mask, int device) {
    if (device >= 0 && device < 64) mask.fetch_or(1ull << device, std::memory_order_release);
}

// the dynamic shared-memory limit, and for 16-CTA clusters (N = 2^15) the opt-in to a
// cluster size above the portable 8
template <class K>
copse_status cluster_attrs(K kernel, int cl) {
    CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(ClusterSmem)));
    if (cl > 8) CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    return COPSE_OK;
}

// butterflies of a batch (N/2 log2 N per transformed residue polynomial): the integer
// roof's unit for the transforms
inline double butterflies(const copse_ctx *ctx, const NttBatch &b) {
    return (double)b.npoly * b.nr * (ctx->N / 2) * ctx->logN;
}

template <int CL>
copse_status launch_cluster(copse_ctx *ctx, const NttBatch &b, cudaStream_t s, bool inverse, double bytes) {
    static std::atomic<uint64_t> attr_devices{0};
    const int smem = (int)sizeof(ClusterSmem);
    if (attr_pending(attr_devices, ctx->device)) {
        STATUS_TRY(cluster_attrs(k_ntt_fwd_cluster<CL, PlainIO>, CL));
        STATUS_TRY(cluster_attrs(k_ntt_inv_cluster<CL, PlainIO>, CL));
        attr_done(attr_devices, ctx->device);
    }
    const unsigned grid = (unsigned)b.npoly * (unsigned)b.nr * CL;
    const int a = ctx->logN / 2;
    if (inverse)
        TIMED_OPS("ntt_inv", bytes, butterflies(ctx, b), s,
              k_ntt_inv_cluster<CL, PlainIO><<<grid, NT2, smem, s>>>(b, ctx->d_prime, ctx->d_ipsi, ctx->d_ipsi_sh,
                                                                     (const ulonglong2 *)ctx->d_stw_i, ctx->logN,
                                                                     ctx->L, a,
                                                                     PlainIO{b.data, b.stride, ctx->logN}));
    else
        TIMED_OPS("ntt_fwd", bytes, butterflies(ctx, b), s,
              k_ntt_fwd_cluster<CL, PlainIO><<<grid, NT2, smem, s>>>(b, ctx->d_prime, ctx->d_psi, ctx->d_psi_sh,
                                                                     (const ulonglong2 *)ctx->d_stw_f, ctx->logN,
                                                                     ctx->L, a,
                                                                     PlainIO{b.data, b.stride, ctx->logN}));
    LAUNCH_CHECK();
    return COPSE_OK;
}

copse_status launch(copse_ctx *ctx, const NttBatch &b, cudaStream_t s, bool inverse) {
    if (b.npoly <= 0 || b.nr <= 0) return COPSE_OK;
    const int N = ctx->N, logN = ctx->logN;
    const double bytes = (double)b.npoly * b.nr * N * 16.0;  // one read and one write of each residue polynomial
    const double bfly = butterflies(ctx, b);
    if (ctx->ntt_clusters && (long)b.npoly * b.nr <= ctx->ntt_cluster_max) {
        if (logN == 12) return launch_cluster<2>(ctx, b, s, inverse, bytes);
        if (logN == 13) return launch_cluster<4>(ctx, b, s, inverse, bytes);
        if (logN == 14) return launch_cluster<8>(ctx, b, s, inverse, bytes);
        if (logN == 15 && ctx->ntt_cluster16) return launch_cluster<16>(ctx, b, s, inverse, bytes);
    }
    if (logN >= 12) {
        const int a = logN / 2;  // column length 2^a, row length 2^(logN - a)
        const unsigned grid = (unsigned)b.npoly * (unsigned)b.nr * (unsigned)(N / TILE);
        if (inverse) {
            TIMED_OPS("ntt_inv", bytes, bfly, s, {
                k_ntt_inv_rows<<<grid, NT2, 0, s>>>(b, ctx->d_prime, (const ulonglong2 *)ctx->d_stw_i, logN, ctx->L, a);
                k_ntt_inv_cols<<<grid, NT2, 0, s>>>(b, ctx->d_prime, ctx->d_ipsi, ctx->d_ipsi_sh, logN, ctx->L, a);
            });
        } else {
            TIMED_OPS("ntt_fwd", bytes, bfly, s, {
                k_ntt_fwd_cols<<<grid, NT2, 0, s>>>(b, ctx->d_prime, ctx->d_psi, ctx->d_psi_sh, logN, ctx->L, a);
                k_ntt_fwd_rows<<<grid, NTT, 0, s>>>(b, ctx->d_prime, (const ulonglong2 *)ctx->d_stw_f, logN, ctx->L, a);
            });
        }
        LAUNCH_CHECK();
        return COPSE_OK;
    }
    const size_t smem = (size_t)N * sizeof(u64);
    const int threads = N / 2 < 512 ? N / 2 : 512;
    const unsigned grid = (unsigned)b.npoly * (unsigned)b.nr;
    if (inverse)
        TIMED_OPS("ntt_inv", bytes, bfly, s,
              k_ntt_inv<<<grid, threads, smem, s>>>(b, ctx->d_prime, ctx->d_ipsi, ctx->d_ipsi_sh, logN, ctx->L));
    else
        TIMED_OPS("ntt_fwd", bytes, bfly, s,
              k_ntt_fwd<<<grid, threads, smem, s>>>(b, ctx->d_prime, ctx->d_psi, ctx->d_psi_sh, logN, ctx->L));
    LAUNCH_CHECK();
    return COPSE_OK;
}

// ---------------------------------------------------------------- two passes fused with the IO
// Where the cluster transform does not run (N = 2^15 by default) the fused transforms take
// the two-pass tiled kernels: the first pass loads through the IO functor (the base
// conversion) and writes its partial transform to scratch [npoly][nr][N]; the second pass
// reads scratch and stores through the functor (the finish).  Residues a batch skips (the
// ModUp digits' own primes) are copied by the first pass, one tile's part each.
template <class IO>
__global__ void __launch_bounds__(NT2) k_ntt_fwd_cols_io(NttBatch b, const PrimeDev *__restrict__ primes,
                                                         const u64 *__restrict__ tw, const u64 *__restrict__ tw_sh,
                                                         int logN, int L, int a, IO io, u64 *scratch) {
    __shared__ u64 sm[TILE], stw[TILE], stwp[TILE];
    const int N = 1 << logN, lb = logN - a, lc = 11 - a, C = 1 << lc, tiles = (1 << lb) >> lc;
    const int pr = blockIdx.x / tiles, tile = blockIdx.x % tiles;
    const int p = pr / b.nr, r = b.r0 + pr % b.nr;
    if (ntt_skipped(b, p, r)) {
        io.skip(p, r, tile, tiles);
        return;
    }
    const int g = ntt_prime(b, r, L);
    const u64 q = primes[g].q, q2 = 2 * q;
    const u64 *W = tw + (size_t)g * N, *Wp = tw_sh + (size_t)g * N;
    {
        // coefficient e + i NT2 of the tile is n0 + i dn (NT2 is a multiple of the tile's width C)
        const int e = threadIdx.x;
        u64 v[TILE / NT2];
        load_n(io, p, r, g, ((size_t)(e >> lc) << lb) + (tile << lc) + (e & (C - 1)), (size_t)(NT2 >> lc) << lb, v);
#pragma unroll
        for (int i = 0; i < TILE / NT2; i++) sm[e + i * NT2] = v[i];
    }
    for (int e = threadIdx.x; e < (1 << a); e += NT2) {
        stw[e] = W[e];
        stwp[e] = Wp[e];
    }
    __syncthreads();
    tile_fwd<true, NT2, false>(sm, stw, stwp, a, q, q2, [&](int gg, int i) { return (i << lc) + gg; },
                   [&](int u, int, int il) { return (1 << u) + il; });
    u64 *out = scratch + ((size_t)pr << logN) + (tile << lc);
    for (int e = threadIdx.x; e < TILE; e += NT2) out[((size_t)(e >> lc) << lb) + (e & (C - 1))] = sm[e];
}

template <class IO>
__global__ void __launch_bounds__(NTT, 4) k_ntt_fwd_rows_io(NttBatch b, const PrimeDev *__restrict__ primes,
                                                         const ulonglong2 *__restrict__ stg, int logN, int L, int a,
                                                         IO io, const u64 *scratch) {
    __shared__ u64 sm[TILE], stw[TILE], stwp[TILE];
    const int N = 1 << logN, lb = logN - a, lr = 11 - lb, tiles = 1 << (a - lr);
    const int pr = blockIdx.x / tiles, tile = blockIdx.x % tiles;
    const int p = pr / b.nr, r = b.r0 + pr % b.nr;
    if (ntt_skipped(b, p, r)) return;
    const int g = ntt_prime(b, r, L);
    const u64 q = primes[g].q, q2 = 2 * q;
    const int row0 = tile << lr;
    const u64 *in = scratch + ((size_t)pr << logN) + ((size_t)row0 << lb);
    const ulonglong2 *st = stg + ((size_t)g * (N / TILE) + tile) * TILE;
    const int nst = TILE - (1 << lr);
    for (int e = threadIdx.x; e < TILE; e += NTT) {
        sm[e] = in[e];
        if (e < nst) {
            const ulonglong2 v = st[e];
            stw[e] = v.x;
            stwp[e] = v.y;
        }
    }
    __syncthreads();
    tile_fwd<false, NTT, true>(sm, stw, stwp, lb, q, q2, [&](int gg, int i) { return (gg << lb) + i; },
                    [&](int u, int gg, int il) { return ((1 << lr) * ((1 << u) - 1)) + (gg << u) + il; });
    const u64 one_sh = primes[g].one_sh;
    u64 v[TILE / NTT];
#pragma unroll
    for (int i = 0; i < TILE / NTT; i++) v[i] = fwd_reduce(sm[threadIdx.x + i * NTT], q, one_sh);
    store_n(io, p, r, g, ((size_t)row0 << lb) + threadIdx.x, NTT, v);
}

template <class IO>
__global__ void __launch_bounds__(NT2) k_ntt_inv_rows_io(NttBatch b, const PrimeDev *__restrict__ primes,
                                                         const ulonglong2 *__restrict__ stg, int logN, int L, int a,
                                                         IO io, u64 *scratch) {
    __shared__ u64 sm[TILE], stw[TILE], stwp[TILE];
    const int N = 1 << logN, lb = logN - a, lr = 11 - lb, tiles = 1 << (a - lr);
    const int pr = blockIdx.x / tiles, tile = blockIdx.x % tiles;
    const int p = pr / b.nr, r = b.r0 + pr % b.nr;
    if (ntt_skipped(b, p, r)) return;
    const int g = ntt_prime(b, r, L);
    const u64 q = primes[g].q, q2 = 2 * q;
    const int row0 = tile << lr;
    const ulonglong2 *st = stg + ((size_t)g * (N / TILE) + tile) * TILE;
    const int nst = TILE - (1 << lr);
    for (int e = threadIdx.x; e < TILE; e += NT2) {
        sm[e] = io.load(p, r, g, ((size_t)row0 << lb) + e);
        if (e < nst) {
            const ulonglong2 v = st[e];
            stw[e] = v.x;
            stwp[e] = v.y;
        }
    }
    __syncthreads();
    tile_inv<false, NT2, false>(sm, stw, stwp, lb, q, q2, [&](int gg, int i) { return (gg << lb) + i; },
                    [&](int u, int gg, int il) {
                        return (1 << lr) * ((1 << lb) - (1 << (lb - u))) + (gg << (lb - 1 - u)) + il;
                    });
    const u64 one_sh = primes[g].one_sh;
    u64 *out = scratch + ((size_t)pr << logN) + ((size_t)row0 << lb);
    for (int e = threadIdx.x; e < TILE; e += NT2) out[e] = fwd_reduce(sm[e], q, one_sh);
}

template <class IO>
__global__ void __launch_bounds__(NT2) k_ntt_inv_cols_io(NttBatch b, const PrimeDev *__restrict__ primes,
                                                         const u64 *__restrict__ tw, const u64 *__restrict__ tw_sh,
                                                         int logN, int L, int a, IO io, const u64 *scratch) {
    __shared__ u64 sm[TILE], stw[TILE], stwp[TILE];
    const int N = 1 << logN, lb = logN - a, lc = 11 - a, C = 1 << lc, tiles = (1 << lb) >> lc;
    const int pr = blockIdx.x / tiles, tile = blockIdx.x % tiles;
    const int p = pr / b.nr, r = b.r0 + pr % b.nr;
    if (ntt_skipped(b, p, r)) return;
    const int g = ntt_prime(b, r, L);
    const PrimeDev P = primes[g];
    const u64 q = P.q, q2 = 2 * q;
    const u64 *W = tw + (size_t)g * N, *Wp = tw_sh + (size_t)g * N;
    const u64 *in = scratch + ((size_t)pr << logN) + (tile << lc);
    for (int e = threadIdx.x; e < TILE; e += NT2) {
        sm[e] = in[((size_t)(e >> lc) << lb) + (e & (C - 1))];
        if (e < (1 << a)) {
            stw[e] = W[e];
            stwp[e] = Wp[e];
        }
    }
    __syncthreads();
    tile_inv<true, NT2, false>(sm, stw, stwp, a, q, q2, [&](int gg, int i) { return (i << lc) + gg; },
                   [&](int u, int, int il) { return (1 << (a - 1 - u)) + il; });
    const Shoup sc = b.scale ? b.scale[r - b.r0] : Shoup{P.ninv, P.ninv_sh};
    for (int e = threadIdx.x; e < TILE; e += NT2)
        io.store(p, r, g, ((size_t)(e >> lc) << lb) + (tile << lc) + (e & (C - 1)), mul_shoup(sm[e], sc, q));
}

// kernel-timer family of each transform variant
template <class IO> constexpr const char *io_family(bool inv) { return inv ? "ntt_inv" : "ntt_fwd"; }
template <> constexpr const char *io_family<CopyIO>(bool) { return "ntt_inv_copy"; }
template <> constexpr const char *io_family<GatherIO>(bool) { return "ntt_inv_copy"; }
template <> constexpr const char *io_family<MsIO>(bool) { return "ntt_fwd_ms"; }
template <> constexpr const char *io_family<MdIO>(bool) { return "ntt_fwd_md"; }
template <> constexpr const char *io_family<MuIO>(bool) { return "ntt_fwd_mu"; }
template <> constexpr const char *io_family<MddIO>(bool) { return "ntt_fwd_mdd"; }

template <int CL, bool INV, class IO>
copse_status launch_cluster_io(copse_ctx *ctx, const NttBatch &b, const IO &io, cudaStream_t s) {
    static std::atomic<uint64_t> attr_devices{0};
    const int smem = (int)sizeof(ClusterSmem);
    if (attr_pending(attr_devices, ctx->device)) {
        if (INV)
            STATUS_TRY(cluster_attrs(k_ntt_inv_cluster<CL, IO>, CL));
        else
            STATUS_TRY(cluster_attrs(k_ntt_fwd_cluster<CL, IO>, CL));
        attr_done(attr_devices, ctx->device);
    }
    const unsigned grid = (unsigned)b.npoly * (unsigned)b.nr * CL;
    const double bytes = (double)b.npoly * b.nr * ctx->N * 16.0;
    if (INV)
        TIMED_OPS(io_family<IO>(true), bytes, butterflies(ctx, b), s,
              k_ntt_inv_cluster<CL, IO><<<grid, NT2, smem, s>>>(b, ctx->d_prime, ctx->d_ipsi, ctx->d_ipsi_sh,
                                                                (const ulonglong2 *)ctx->d_stw_i, ctx->logN, ctx->L,
                                                                ctx->logN / 2, io));
    else
        TIMED_OPS(io_family<IO>(false), bytes, butterflies(ctx, b), s,
              k_ntt_fwd_cluster<CL, IO><<<grid, NT2, smem, s>>>(b, ctx->d_prime, ctx->d_psi, ctx->d_psi_sh,
                                                                (const ulonglong2 *)ctx->d_stw_f, ctx->logN, ctx->L,
                                                                ctx->logN / 2, io));
    LAUNCH_CHECK();
    return COPSE_OK;
}

// the fused transform as two tiled launches through a scratch buffer
template <bool INV, class IO>
copse_status launch_tiled_io(copse_ctx *ctx, const NttBatch &b, const IO &io, cudaStream_t s) {
    const int logN = ctx->logN, a = logN / 2;
    const size_t words = (size_t)b.npoly * b.nr << logN;
    u64 *scratch = nullptr;
    STATUS_TRY(dev_alloc(ctx, (void **)&scratch, words * sizeof(u64), s));
    const unsigned grid = (unsigned)b.npoly * (unsigned)b.nr * (unsigned)(ctx->N / TILE);
    const double bytes = (double)b.npoly * b.nr * ctx->N * 16.0;
    if (INV)
        TIMED_OPS(io_family<IO>(true), bytes, butterflies(ctx, b), s, {
            k_ntt_inv_rows_io<IO><<<grid, NT2, 0, s>>>(b, ctx->d_prime, (const ulonglong2 *)ctx->d_stw_i, logN, ctx->L,
                                                       a, io, scratch);
            k_ntt_inv_cols_io<IO><<<grid, NT2, 0, s>>>(b, ctx->d_prime, ctx->d_ipsi, ctx->d_ipsi_sh, logN, ctx->L, a,
                                                       io, scratch);
        });
    else
        TIMED_OPS(io_family<IO>(false), bytes, butterflies(ctx, b), s, {
            k_ntt_fwd_cols_io<IO><<<grid, NT2, 0, s>>>(b, ctx->d_prime, ctx->d_psi, ctx->d_psi_sh, logN, ctx->L, a,
                                                       io, scratch);
            k_ntt_fwd_rows_io<IO><<<grid, NTT, 0, s>>>(b, ctx->d_prime, (const ulonglong2 *)ctx->d_stw_f, logN, ctx->L,
                                                       a, io, scratch);
        });
    const cudaError_t e = cudaGetLastError();
    dev_free(scratch, s);
    if (e != cudaSuccess) {
        set_error(std::string("fused two-pass transform: ") + cudaGetErrorString(e));
        return COPSE_ECUDA;
    }
    return COPSE_OK;
}

template <bool INV = false, class IO>
copse_status launch_fused(copse_ctx *ctx, const NttBatch &b, const IO &io, cudaStream_t s, bool *done) {
    *done = false;
    if (b.npoly <= 0 || b.nr <= 0) { *done = true; return COPSE_OK; }
    if (!ctx->ntt_clusters) return COPSE_OK;
    if (ctx->logN == 15 && !ctx->ntt_cluster16) {
        // N = 2^15 without 16-CTA clusters: the two-pass transform fused with the IO
        STATUS_TRY((launch_tiled_io<INV, IO>(ctx, b, io, s)));
        *done = true;
        return COPSE_OK;
    }
    if ((long)b.npoly * b.nr > ctx->ntt_fused_max) return COPSE_OK;
    if (ctx->logN == 12) STATUS_TRY((launch_cluster_io<2, INV, IO>(ctx, b, io, s)));
    else if (ctx->logN == 13) STATUS_TRY((launch_cluster_io<4, INV, IO>(ctx, b, io, s)));
    else if (ctx->logN == 14) STATUS_TRY((launch_cluster_io<8, INV, IO>(ctx, b, io, s)));
    else if (ctx->logN == 15) STATUS_TRY((launch_cluster_io<16, INV, IO>(ctx, b, io, s)));
    else return COPSE_OK;
    *done = true;
    return COPSE_OK;
}

__global__ void k_ms_finish_io(const MsFuse f, const u64 *W, int nc, const PrimeDev *pr, KsTables T, int L,
                               int logN) {
    const size_t per = (size_t)(f.ell - 1) << logN;
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)nc * per) return;
    const int p = (int)(e / per);
    const size_t rem = e - p * per;
    ms_store(f, pr, T, L, logN, p, (int)(rem >> logN), rem & ((1ull << logN) - 1), W[e]);
}

__global__ void k_gather_res(const GatherSrc src, int npoly, u64 *dst, int logN) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ((size_t)npoly << logN)) return;
    dst[e] = src.p[e >> logN][e & ((1ull << logN) - 1)];
}

__global__ void k_mdd_conv(const MddFuse f, u64 *W, int npoly, const PrimeDev *pr, KsTables T, int L, int alpha,
                           int logN) {
    const size_t per = (size_t)(f.ell - 1) << logN;
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)npoly * per) return;
    const int p = (int)(e / per);
    const size_t rem = e - p * per;
    W[e] = mdd_load(f, pr, T, L, alpha, logN, p, (int)(rem >> logN), rem & ((1ull << logN) - 1));
}

__global__ void k_mdd_finish(const MddFuse f, const u64 *W, int npoly, const PrimeDev *pr, KsTables T, int L,
                             int logN) {
    const size_t per = (size_t)(f.ell - 1) << logN;
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)npoly * per) return;
    const int p = (int)(e / per);
    const size_t rem = e - p * per;
    mdd_store(f, pr, T, L, logN, p, (int)(rem >> logN), rem & ((1ull << logN) - 1), W[e]);
}

__global__ void k_md_finish_io(const MdFuse f, const u64 *W, int njobs, const PrimeDev *pr, KsTables T, int logN) {
    const size_t per = (size_t)f.ell << logN;
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)2 * njobs * per) return;
    const int p = (int)(e / per);
    const size_t rem = e - p * per;
    md_store(f, pr, T, logN, p, (int)(rem >> logN), rem & ((1ull << logN) - 1), W[e]);
}

}  // namespace

namespace {
// Row-stage twiddles of cluster CTA (or row tile) `rank` in the order the cluster and
// tiled row kernels use them:
// forward stage u of the row pass takes 2^(lr+u) consecutive entries from
// W[2^(a+u) + (row0 << u)], the inverse stage u takes 2^(lr+su) (su = lb-1-u) from
// W[2^(logN-1-u) + (row0 << su)], stages back to back.
__global__ void k_stage_tw(const u64 *W, const u64 *Wp, u64 *out, int np, int logN, int inverse) {
    const int CL = 1 << (logN - 11), a = logN / 2, lb = logN - a, lr = 11 - lb;
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)np * CL * TILE) return;
    const int j = (int)(e % TILE), rank = (int)((e / TILE) % CL);
    const size_t g = e / ((size_t)TILE * CL);
    const int row0 = rank << lr;
    u64 w = 0, wp = 0;
    for (int u = 0, off = 0; u < lb; u++) {
        const int su = inverse ? lb - 1 - u : u, cnt = 1 << (lr + su);
        if (j < off + cnt) {
            const int src = (inverse ? (1 << (logN - 1 - u)) : (1 << (a + u))) + (row0 << su) + (j - off);
            w = W[(g << logN) + src];
            wp = Wp[(g << logN) + src];
            break;
        }
        off += cnt;
    }
    out[2 * e] = w;
    out[2 * e + 1] = wp;
}
}  // namespace

copse_status ntt_stage_tables(copse_ctx *ctx) {
    if (ctx->logN < 12) return COPSE_OK;   // one CTA per transform below 2^12: nothing staged
    if (ctx->logN == 15) {
        // 16-CTA clusters are above the portable size: use them only where the device
        // can place at least one (otherwise N = 2^15 keeps the two-launch transforms)
        STATUS_TRY(cluster_attrs(k_ntt_fwd_cluster<16, PlainIO>, 16));
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(16);
        cfg.blockDim = dim3(NT2);
        cfg.dynamicSmemBytes = sizeof(ClusterSmem);
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 16;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int nclusters = 0;
        const cudaError_t e = cudaOccupancyMaxActiveClusters(&nclusters, k_ntt_fwd_cluster<16, PlainIO>, &cfg);
        // measured slower than the two-launch transforms on GB300 at N = 2^15 (the 16-CTA
        // cluster barriers and cross-SM tile gathers): an option, COPSE_NTT_CLUSTER16=1
        const char *opt = getenv("COPSE_NTT_CLUSTER16");
        ctx->ntt_cluster16 = e == cudaSuccess && nclusters > 0 && opt && opt[0] == '1';
        cudaGetLastError();
    }
    const size_t n = (size_t)ctx->NP * ctx->N;  // NP x (N / TILE) x TILE entries
    for (int inv = 0; inv < 2; inv++) {
        void *p = nullptr;
        CUDA_TRY(cudaMalloc(&p, n * 2 * sizeof(u64)));
        ctx->owned.push_back(p);
        k_stage_tw<<<(unsigned)((n + 255) / 256), 256>>>(inv ? ctx->d_ipsi : ctx->d_psi, inv ? ctx->d_ipsi_sh : ctx->d_psi_sh,
                                                         (u64 *)p, ctx->NP, ctx->logN, inv);
        CUDA_TRY(cudaGetLastError());
        (inv ? ctx->d_stw_i : ctx->d_stw_f) = (u64 *)p;
    }
    CUDA_TRY(cudaDeviceSynchronize());
    return COPSE_OK;
}

copse_status ntt_forward_modswitch(copse_ctx *ctx, const MsFuse &f, int nc, cudaStream_t s, bool *done) {
    NttBatch b{nullptr, 0, nc, 0, f.ell - 1, f.ell - 1, -1};
    return launch_fused(ctx, b, MsIO{f, ctx->d_prime, ctx->ks, ctx->L, ctx->logN}, s, done);
}

copse_status ntt_forward_moddown(copse_ctx *ctx, const MdFuse &f, int njobs, cudaStream_t s, bool *done) {
    if (njobs > MD_JOBS) { set_error("internal: too many ModDown jobs"); return COPSE_EINVAL; }
    NttBatch b{nullptr, 0, 2 * njobs, 0, f.ell, f.ell, -1};
    return launch_fused(ctx, b, MdIO{f, ctx->d_prime, ctx->ks, ctx->L, ctx->alpha, ctx->logN}, s, done);
}

copse_status ntt_inverse_copy(copse_ctx *ctx, const u64 *src, size_t sstride, u64 *dst, size_t dstride, int npoly,
                              int nr, int fixed, cudaStream_t s, bool *done, const Shoup *scale) {
    NttBatch b{nullptr, 0, npoly, 0, nr, nr, fixed};
    b.scale = scale;
    return launch_fused<true>(ctx, b, CopyIO{src, sstride, dst, dstride, ctx->logN}, s, done);
}

copse_status ntt_inverse_gather(copse_ctx *ctx, const GatherSrc &src, int npoly, u64 *dst, int fixed, cudaStream_t s,
                                bool *done, const Shoup *scale) {
    if (npoly > MS_POLYS) { set_error("internal: too many polynomials in one gathered transform"); return COPSE_EINVAL; }
    NttBatch b{nullptr, 0, npoly, 0, 1, 1, fixed};
    b.scale = scale;
    STATUS_TRY(launch_fused<true>(ctx, b, GatherIO{src, dst, ctx->logN}, s, done));
    if (*done) return COPSE_OK;
    // a gather, then the in-place transform
    const size_t n = (size_t)npoly * ctx->N;
    k_gather_res<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(src, npoly, dst, ctx->logN);
    if (cudaGetLastError() != cudaSuccess) { set_error("gather kernel failed to launch"); return COPSE_ECUDA; }
    NttBatch bi{dst, (size_t)ctx->N, npoly, 0, 1, 1, fixed};
    bi.scale = scale;
    STATUS_TRY(launch(ctx, bi, s, true));
    *done = true;
    return COPSE_OK;
}

copse_status ntt_forward_modup(copse_ctx *ctx, const u64 *xc, const u64 *x_ntt, size_t xs, u64 *y, int n_items,
                               int ell, cudaStream_t s, bool *done) {
    const int A = ctx->alpha, nd = (ell + A - 1) / A;
    NttBatch b{nullptr, 0, n_items * nd, 0, ell + A, ell, -1};
    b.skip_alpha = A;
    b.skip_period = nd;
    return launch_fused(ctx, b, MuIO{xc, x_ntt, xs, y, ell, A, nd, ctx->L, ctx->NP, ctx->logN, ctx->d_prime, ctx->ks},
                        s, done);
}

copse_status ntt_forward_moddown_drop(copse_ctx *ctx, const MddFuse &f, int npoly, cudaStream_t s, bool *done) {
    NttBatch b{nullptr, 0, npoly, 0, f.ell - 1, f.ell - 1, -1};
    return launch_fused(ctx, b, MddIO{f, ctx->d_prime, ctx->ks, ctx->L, ctx->alpha, ctx->logN}, s, done);
}

copse_status moddown_drop_unfused(copse_ctx *ctx, const MddFuse &f, int npoly, cudaStream_t s) {
    const size_t n = (size_t)npoly * (f.ell - 1) * ctx->N;
    u64 *W = nullptr;
    STATUS_TRY(dev_alloc(ctx, (void **)&W, n * sizeof(u64), s));
    const unsigned g = (unsigned)((n + 255) / 256);
    TIMED("moddown_conv", 8.0 * (double)n * (ctx->alpha + 2), s,
          k_mdd_conv<<<g, 256, 0, s>>>(f, W, npoly, ctx->d_prime, ctx->ks, ctx->L, ctx->alpha, ctx->logN));
    copse_status st = cudaGetLastError() == cudaSuccess ? COPSE_OK : COPSE_ECUDA;
    if (st == COPSE_OK) st = launch(ctx, NttBatch{W, (size_t)(f.ell - 1) * ctx->N, npoly, 0, f.ell - 1, f.ell - 1, -1},
                                    s, false);
    if (st == COPSE_OK) {
        TIMED("ks_finish", 8.0 * 3.0 * (double)n, s,
              k_mdd_finish<<<g, 256, 0, s>>>(f, W, npoly, ctx->d_prime, ctx->ks, ctx->L, ctx->logN));
        if (cudaGetLastError() != cudaSuccess) st = COPSE_ECUDA;
    }
    dev_free(W, s);
    if (st != COPSE_OK && st != COPSE_ECUDA) return st;
    if (st == COPSE_ECUDA) set_error("moddown-drop kernels failed to launch");
    return st;
}

copse_status modswitch_finish(copse_ctx *ctx, const MsFuse &f, const u64 *W, int nc, cudaStream_t s) {
    const size_t n = (size_t)nc * (f.ell - 1) * ctx->N;
    TIMED("ms_finish", 8.0 * 3.0 * (double)n, s,
          k_ms_finish_io<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(f, W, nc, ctx->d_prime, ctx->ks, ctx->L,
                                                                      ctx->logN));
    LAUNCH_CHECK();
    return COPSE_OK;
}

copse_status moddown_finish(copse_ctx *ctx, const MdFuse &f, const u64 *W, int njobs, cudaStream_t s) {
    if (njobs > MD_JOBS) { set_error("internal: too many ModDown jobs"); return COPSE_EINVAL; }
    const size_t n = (size_t)2 * njobs * f.ell * ctx->N;
    TIMED("ks_finish", 8.0 * 4.0 * (double)n, s,
          k_md_finish_io<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(f, W, njobs, ctx->d_prime, ctx->ks, ctx->logN));
    LAUNCH_CHECK();
    return COPSE_OK;
}

copse_status ntt_forward(copse_ctx *ctx, const NttBatch &b, cudaStream_t s) { return launch(ctx, b, s, false); }
copse_status ntt_inverse(copse_ctx *ctx, const NttBatch &b, cudaStream_t s) { return launch(ctx, b, s, true); }
