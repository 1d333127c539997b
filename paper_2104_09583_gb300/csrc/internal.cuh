// Internal declarations of the GB300 COPSE library: device modular arithmetic,
// the context's device tables, device ciphertexts and the kernel launchers.
//
// Residues are 64-bit words modulo primes q < 2^55 (the transforms and the exact
// split-product sums keep their lazy values below 2^64 under that bound).  Products with a constant
// operand use Shoup's precomputed quotient (V. Shoup, NTL; D. Harvey, "Faster
// arithmetic for number-theoretic transforms", 2014); products of two data
// words use Barrett reduction of the 128-bit product (Handbook of Applied
// Cryptography, Alg. 14.42).  Every kernel leaves its outputs fully reduced to
// [0, q), so device data is bit-comparable with any other exact implementation.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "forest.h"

#include "../../include/copse.h"

typedef uint64_t u64;
typedef int64_t i64;

#define COPSE_MAX_PRIMES 64
#define COPSE_T 65537ULL

// ---------------------------------------------------------------- errors
void set_error(const std::string &msg);
#define CUDA_TRY(expr)                                                                           \
    do {                                                                                         \
        cudaError_t e__ = (expr);                                                                \
        if (e__ != cudaSuccess) {                                                                \
            set_error(std::string(#expr) + ": " + cudaGetErrorString(e__));                      \
            return COPSE_ECUDA;                                                                  \
        }                                                                                        \
    } while (0)
#define STATUS_TRY(expr)                                                                         \
    do {                                                                                         \
        copse_status s__ = (expr);                                                               \
        if (s__ != COPSE_OK) return s__;                                                         \
    } while (0)
// after a kernel launch
#define LAUNCH_CHECK() CUDA_TRY(cudaGetLastError())

// kernel timing (stats.cu): brackets a launch with CUDA events when enabled
int stats_begin(const char *name, double bytes, cudaStream_t s);
int stats_begin_ops(const char *name, double bytes, double ops, cudaStream_t s);
void stats_end(int token, cudaStream_t s);
void stats_suspend(bool on);
#define TIMED(name, bytes, s, ...)                                                               \
    do {                                                                                         \
        int tk__ = stats_begin(name, (double)(bytes), s);                                        \
        __VA_ARGS__;                                                                             \
        stats_end(tk__, s);                                                                      \
    } while (0)
// the same with the launch's algorithmic modular products (the integer roof's unit)
#define TIMED_OPS(name, bytes, ops, s, ...)                                                      \
    do {                                                                                         \
        int tk__ = stats_begin_ops(name, (double)(bytes), (double)(ops), s);                     \
        __VA_ARGS__;                                                                             \
        stats_end(tk__, s);                                                                      \
    } while (0)

// ---------------------------------------------------------------- per-prime constants
struct PrimeDev {
    u64 q;
    u64 mu;       // floor(2^(2*bits) / q): Barrett constant
    u64 ninv;     // N^-1 mod q
    u64 ninv_sh;  // its Shoup quotient floor(ninv * 2^64 / q)
    u64 t_mod;    // t mod q
    u64 t_mod_sh;
    u64 r64;      // 2^64 mod q
    u64 r64_sh;
    uint32_t bits;  // bit length of q
    uint32_t pad;
    u64 one_sh;     // floor(2^64 / q): Shoup quotient of 1 (a reduction of any 64-bit value to [0, 2q))
    u64 qinv_neg;   // -q^-1 mod 2^64 (Montgomery reduction)
};

// value and Shoup quotient of a constant multiplier
struct Shoup {
    u64 w, wp;
};

// ---------------------------------------------------------------- device arithmetic
__device__ __forceinline__ u64 add_mod(u64 a, u64 b, u64 q) {
    u64 s = a + b;
    return s >= q ? s - q : s;
}
__device__ __forceinline__ u64 sub_mod(u64 a, u64 b, u64 q) { return a >= b ? a - b : a + (q - b); }
// a * w mod q in [0, 2q) for any a < 2^64 (w < q, wp = floor(w 2^64 / q))
__device__ __forceinline__ u64 mul_shoup_lazy(u64 a, u64 w, u64 wp, u64 q) {
    u64 h = __umul64hi(a, wp);
    return a * w - h * q;
}
__device__ __forceinline__ u64 mul_shoup(u64 a, u64 w, u64 wp, u64 q) {
    u64 r = mul_shoup_lazy(a, w, wp, q);
    return r >= q ? r - q : r;
}
__device__ __forceinline__ u64 mul_shoup(u64 a, Shoup c, u64 q) { return mul_shoup(a, c.w, c.wp, q); }
// (hi*2^64 + lo) mod q for hi*2^64 + lo < 2^(2*bits)
__device__ __forceinline__ u64 barrett_wide(u64 hi, u64 lo, const PrimeDev &p) {
    const int s = (int)p.bits;
    u64 x1 = (hi << (65 - s)) | (lo >> (s - 1));
    u64 plo = x1 * p.mu, phi = __umul64hi(x1, p.mu);
    u64 qe = (phi << (63 - s)) | (plo >> (s + 1));
    u64 r = lo - qe * p.q;
    if (r >= p.q) r -= p.q;
    if (r >= p.q) r -= p.q;
    return r;
}
// a * b mod q for a, b < q
__device__ __forceinline__ u64 mul_mod(u64 a, u64 b, const PrimeDev &p) {
    return barrett_wide(__umul64hi(a, b), a * b, p);
}
// Lazy sums of products: x * y < 2^120 for residues of primes below 2^60, so a
// 128-bit accumulator holds 256 such products (2^18 at 55 bits); one reduction at
// the end gives the same residue as reducing after every step.
struct Acc128 {
    u64 lo, hi;
};
__device__ __forceinline__ void mac128(Acc128 &a, u64 x, u64 y) {
    const u64 plo = x * y, phi = __umul64hi(x, y);
    a.lo += plo;
    a.hi += phi + (a.lo < plo);
}
__device__ __forceinline__ u64 reduce128(const Acc128 &a, const PrimeDev &P) {
    return add_mod(mul_shoup(barrett_wide(0, a.hi, P), P.r64, P.r64_sh, P.q), barrett_wide(0, a.lo, P), P.q);
}
// Exact sums of products of operands below 2^56 (residues of primes below 2^55 and
// sums of two of them) from 32 x 32 -> 64-bit multiply-adds: x = x1 2^28 + x0 with
// x0, x1 < 2^28, so x y = x1 y1 2^56 + (x1 y0 + x0 y1) 2^28 + x0 y0 and every partial
// product is below 2^56.  Three 64-bit partial sums hold 64 such products exactly
// (lo, hi < 2^62, mid < 2^63); one reduction at the end gives the residue.
struct Sp28 {
    uint32_t lo, hi;
};
__device__ __forceinline__ Sp28 split28(u64 x) { return Sp28{(uint32_t)x & 0x0FFFFFFFu, (uint32_t)(x >> 28)}; }
struct Acc3w {
    u64 lo, mid, hi;
};
__device__ __forceinline__ void mac_sp(Acc3w &a, Sp28 x, Sp28 y) {
    a.lo += (u64)x.lo * y.lo;
    a.mid += (u64)x.lo * y.hi;
    a.mid += (u64)x.hi * y.lo;
    a.hi += (u64)x.hi * y.hi;
}
// lo + mid 2^28 + hi 2^56 (< 2^119) as a 128-bit value
__device__ __forceinline__ Acc128 acc3w_value(const Acc3w &a) {
    Acc128 v{a.lo, 0};
    const u64 m = a.mid << 28;
    v.lo += m;
    v.hi += (a.mid >> 36) + (v.lo < m);
    const u64 h = a.hi << 56;
    v.lo += h;
    v.hi += (a.hi >> 8) + (v.lo < h);
    return v;
}
// Montgomery reduction (P. Montgomery, Math. Comp. 1985) of a 128-bit value x < q 2^64:
// x 2^-64 mod q in [0, q).  Key-switching keys are stored in Montgomery form k 2^64 mod q,
// so a dot product of residues with key words summed exactly in 128 bits (mac128; nd
// products of values below q < 2^58 stay below q 2^64 for nd <= 64) reduces to the plain
// residue sum with one reduction.
__device__ __forceinline__ u64 mont_reduce(const Acc128 &x, const PrimeDev &P) {
    const u64 m = x.lo * P.qinv_neg;
    const u64 t = x.hi + __umul64hi(m, P.q) + (x.lo != 0);
    return t >= P.q ? t - P.q : t;
}
// a signed small integer (|v| < q) as a residue
__device__ __forceinline__ u64 from_signed(i64 v, u64 q) { return v < 0 ? q - (u64)(-v) : (u64)v; }
__device__ __forceinline__ uint32_t bit_reverse(uint32_t x, int logN) { return __brev(x) >> (32 - logN); }
// NTT position whose value lands on position n under X -> X^g (bit-reversed layout:
// position n holds the evaluation at psi^(2 brev(n) + 1))
__device__ __forceinline__ uint32_t galois_src(uint32_t n, u64 g, int logN) {
    uint32_t e = 2u * bit_reverse(n, logN) + 1u;
    uint32_t e2 = (uint32_t)(((u64)e * g) & ((2ull << logN) - 1));
    return bit_reverse((e2 - 1u) >> 1, logN);
}

// SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) in counter form: output number
// (stream * 2^40 + idx + 1) of the sequence whose state starts at `seed`.
__device__ __forceinline__ u64 rng_word(u64 seed, u64 stream, u64 idx) {
    u64 z = seed + 0x9E3779B97F4A7C15ULL * ((stream << 40) + idx + 1ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// Encrypted-model ciphertexts are secret-key encryptions whose mask a is drawn from the
// counter generator in evaluation form: stream MODEL_STREAM + 2 i for model ciphertext i
// (its noise from stream MODEL_STREAM + 2 i + 1).  At NTT position pos of prime r
// (evaluation point psi_r^(2 brev(pos) + 1)) a is the uniform residue number r N + brev(pos)
// of the stream: two 64-bit words hi, lo give (hi 2^64 + lo) mod q.
constexpr u64 MODEL_STREAM = 0x800000ull;
__device__ __forceinline__ u64 seeded_mask(u64 seed, u64 stream, int r, uint32_t pos, int logN, const PrimeDev &P) {
    const u64 j = bit_reverse(pos, logN);
    const u64 idx = 2 * (((u64)r << logN) + j);
    const u64 hi = rng_word(seed, stream, idx), lo = rng_word(seed, stream, idx + 1);
    return add_mod(mul_shoup(barrett_wide(0, hi, P), P.r64, P.r64_sh, P.q), barrett_wide(0, lo, P), P.q);
}

// 16-byte asynchronous copies global -> shared (cp.async, grouped per thread)
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ---------------------------------------------------------------- context
// Base-conversion constants.  Primes are addressed by a global index g:
// 0..L-1 ciphertext primes, L..L+alpha-1 special primes, L+alpha = t.
// At level ell the extended basis lists q_0..q_{ell-1} then p_0..p_{alpha-1};
// ext_prime(r) maps its position r to g.
struct KsTables {
    // ModUp at level ell, source prime i (< ell), digit of i = i / alpha:
    //   modup_inv[ell][i]      = (prod of the other primes of the digit below ell)^-1 mod q_i
    //   modup_hat[ell][i][g]   = (prod of the other primes of the digit below ell) mod prime g
    //   modup_qhat[ell][i][g]  = q_i * modup_hat mod prime g  (correction for a negative centred digit)
    Shoup *modup_inv;   // [(L+1) * L]
    Shoup *modup_hat;   // [(L+1) * L * NP]
    u64 *modup_qhat;    // [(L+1) * L * NP]
    // ModDown: md_inv[k] = t^-1 * Phat_k^-1 mod p_k; md_hat[k][i] = Phat_k mod q_i;
    // md_P[i] = P mod q_i; md_Pinv[i] = P^-1 mod q_i
    Shoup *md_inv;      // [alpha]
    Shoup *md_hat;      // [alpha * L]
    u64 *md_P;          // [L]
    Shoup *md_Pinv;     // [L]
    // modulus switch dropping q_{ell-1}: ms_tinv[ell] = t^-1 mod q_{ell-1};
    // ms_qinv[ell][i] = q_{ell-1}^-1 mod q_i
    Shoup *ms_tinv;     // [L+1]
    Shoup *ms_qinv;     // [(L+1) * L]
    // ModDown over B = q_{ell-1} P (relinearise and drop a prime), basis b_0 = q_{ell-1},
    // b_k = p_{k-1}: mdd_inv[ell][k] = t^-1 (B/b_k)^-1 mod b_k; mdd_hat[ell][k][i] = B/b_k mod q_i;
    // mdd_B[ell][i] = B mod q_i; mdd_Binv[ell][i] = B^-1 mod q_i  (i < ell - 1)
    Shoup *mdd_inv;     // [(L+1) * (alpha+1)]
    // the same first-step factors times N^-1 mod their prime: the scale of the inverse
    // transform whose output the conversion reads (mu_scale [(L+1) * L], md_scale [alpha],
    // ms_scale [L+1], mdd_scale [(L+1) * (alpha+1)], indexed like the factors above)
    Shoup *mu_scale, *md_scale, *ms_scale, *mdd_scale;
    Shoup *mdd_hat;     // [(L+1) * (alpha+1) * L]
    u64 *mdd_B;         // [(L+1) * L]
    Shoup *mdd_Binv;    // [(L+1) * L]
    // The conversion factors in Montgomery form (x 2^64 mod the target prime), indexed like
    // the factors above, for the fused transforms' loads: a conversion sums its products
    // exactly in 128 bits, adds the negated correction of every centred negative digit
    // (modup_negq_m = -modup_qhat, md_negP_m = -P, mdd_negB_m = -B) and reduces once.
    u64 *modup_hat_m, *modup_negq_m, *md_hat_m, *md_negP_m, *mdd_hat_m, *mdd_negB_m;
    // gadget factor of key-switching keys: P mod q_i (i < L)
};

struct copse_ctx {
    uint64_t serial = 0;              // unique per context made in this process
    int device = 0;
    int logN = 0, N = 0;
    u64 t = COPSE_T;
    int L = 0, alpha = 0, ndig = 0, dnum = 0, bits = 0;
    int NP = 0;                       // L + alpha + 1 table entries (t last)
    std::vector<u64> primes;          // L + alpha primes, then t
    std::vector<PrimeDev> hprime;     // host copy of the prime constants
    PrimeDev *d_prime = nullptr;      // [NP]
    u64 *d_psi = nullptr;             // [NP][N] psi^brev(k)
    u64 *d_psi_sh = nullptr;
    u64 *d_ipsi = nullptr;            // [NP][N] psi^-brev(k)
    u64 *d_ipsi_sh = nullptr;
    u64 *d_stw_f = nullptr;           // N >= 2^12: each cluster CTA's / row tile's row-stage twiddles,
    u64 *d_stw_i = nullptr;           //   (w, w') pairs in staging order, [NP][N / 2048][2048][2]
    uint32_t *d_slot_index = nullptr; // [N] NTT(mod t) position of slot s
    KsTables ks{};
    std::vector<void *> owned;        // device allocations freed with the context
    cudaMemPool_t pool = nullptr;
    // side streams for independent operations of one inference (fork/join with events)
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> side_done;
    std::vector<cudaEvent_t> fork_ev;  // one per lane
    // set while a graph is being captured: allocations become graph memory nodes
    bool capturing = false;
    // one-launch cluster NTT for 2^12 <= N <= 2^14 (environment COPSE_NTT_CLUSTERS=0 selects the
    // two-launch form)
    bool ntt_clusters = true;
    // batches of more residue polynomials than this take the two-launch form (autotuned)
    long ntt_cluster_max = 1L << 30;
    long ntt_fused_max = 1L << 30;    // the same crossover for the transforms fused with base conversions
    bool ntt_cluster16 = false;       // N = 2^15: the device places 16-CTA clusters (non-portable size)
    // device status word: kernels whose bounded waits ran out set bits here (COPSE_DEV_*);
    // read and cleared by copse_ctx_device_status
    int *d_status = nullptr;

    int ext_prime(int ell, int r) const { return r < ell ? r : L + (r - ell); }
    int t_index() const { return L + alpha; }
};

// Fork n independent branches off stream s: branch i runs on fork_stream(c, i)
// after everything already queued on s; fork_join makes s wait for all n.
// `lane` selects an independent set of fork streams (one per concurrent inference).
#define COPSE_SIDE_STREAMS 16
#define COPSE_MAX_LANES 32
copse_status ensure_lanes(copse_ctx *c, int lanes);
copse_status fork_begin(copse_ctx *c, cudaStream_t s, int n, int lane = 0);
cudaStream_t fork_stream(copse_ctx *c, int i, int lane = 0);
copse_status fork_join(copse_ctx *c, cudaStream_t s, int n, int lane = 0);
cudaStream_t lane_stream(copse_ctx *c, int lane);  // the lane's own stream
cudaEvent_t lane_event(copse_ctx *c, int lane);

// device memory from the context's stream-ordered pool
copse_status dev_alloc(copse_ctx *ctx, void **p, size_t bytes, cudaStream_t s);
void dev_free(void *p, cudaStream_t s);

// stream-ordered scratch allocations freed (on the same stream) when it goes out of scope
struct Scratch {
    std::vector<void *> ptrs;
    cudaStream_t s;
    explicit Scratch(cudaStream_t st) : s(st) {}
    ~Scratch() {
        for (void *p : ptrs) dev_free(p, s);
    }
    copse_status get(copse_ctx *c, u64 **p, size_t words) {
        STATUS_TRY(dev_alloc(c, (void **)p, words * sizeof(u64), s));
        ptrs.push_back(*p);
        return COPSE_OK;
    }
};

// ---------------------------------------------------------------- ciphertexts
// A ciphertext at level ell with ncomp components, each [ell][N] residues
// (residue r modulo q_r), stored in the bit-reversed NTT (evaluation) domain.
struct DCt {
    int level = 0;
    int ncomp = 2;
    u64 *data = nullptr;
};
// a plaintext polynomial at `level` residues, NTT domain, [level][N]
struct DPt {
    int level = 0;
    u64 *data = nullptr;
};

// ---------------------------------------------------------------- NTT
// Batched NTTs.  Poly p's residue r (r in [r0, r0 + nr)) lives at
// data + p * stride + r * N and is taken modulo prime ext_prime(ell, r), or
// modulo global prime `fixed` when fixed >= 0.
struct NttBatch {
    u64 *data;
    size_t stride;   // words between consecutive polys
    int npoly;
    int r0, nr;
    int ell;
    int fixed;
    int skip_alpha = 0;  // > 0: poly p skips residues [j*skip_alpha, min((j+1)*skip_alpha, ell)),
    int skip_period = 0; //      j = p (skip_period = 0) or p mod skip_period (digits of several inputs)
    // inverse transforms: when set, residue r's result is scaled by scale[r - r0] instead of
    // N^-1 (the first step of the base conversion that reads it folded in: N^-1 * c mod q)
    const Shoup *scale = nullptr;
};
// the staged row twiddles of the cluster transforms (context creation)
copse_status ntt_stage_tables(copse_ctx *ctx);
copse_status ntt_forward(copse_ctx *ctx, const NttBatch &b, cudaStream_t s);
copse_status ntt_inverse(copse_ctx *ctx, const NttBatch &b, cudaStream_t s);

// ---- forward transforms fused with the base conversions around them
// Modulus switch dropping q_{ell-1} (nc components): the transform's input is the
// centred conversion of last ([nc][N], coefficient form, [c_{ell-1} t^-1]) to
// q_0..q_{ell-2}, its output goes straight into
//   out[c][i] = (x[c][i] - t * NTT(conv)) * q_{ell-1}^-1.
#define MS_POLYS 128
struct MsFuse {
    const u64 *last;  // [nc][N] coefficient form
    const u64 *x;     // [nc][ell][N] NTT domain
    u64 *out;         // [nc][ell-1][N], or per polynomial:
    int ell;
    u64 *outp[MS_POLYS];  // when outp[0] is set: polynomial p's result [ell-1][N] at outp[p]
    const u64 *xp[MS_POLYS];  // when xp[0] is set: polynomial p's input [ell][N] at xp[p] (x unused)
};
// ModDown finish of key-switching sums (job j = polys 2j, 2j+1): U (stride ustride
// per poly) holds the extended-basis sum with its alpha special residues in
// coefficient form; the transform's input is their conversion to q_0..q_{ell-1} and
//   out_j[c][i] = (U[c][i] - t * NTT(conv)) * P^-1  + add_j[c] (tau_{gal_j} on c = 0; none
//   when add_comps = 0; component 0 only when add_comps = 1).
#define MD_JOBS 64
struct MdFuse {
    const u64 *U;
    size_t ustride;
    int ell;
    u64 *out[MD_JOBS];        // [2][ell][N] each (components ocomp words apart)
    size_t ocomp;
    const u64 *add[MD_JOBS];  // [2][ell][N] each (components acomp words apart)
    size_t acomp;
    int add_comps;
    u64 gal[MD_JOBS];         // 1 = no permutation
};
// ModDown over B = q_{ell-1} P of npoly polynomials U (stride ustride) whose residues
// ell-1 .. ell+alpha-1 are in coefficient form: the transform's input is their centred
// conversion to q_0..q_{ell-2}, its output goes straight into
//   out[p][i] = (U[p][i] - t * NTT(conv)) * B^-1   (i < ell - 1).
// Products batched together (polys 2j, 2j+1 = product j) may write ciphertext j to
// outp[j] ([2][ell-1][N]) and add the ciphertext addp[j] (same layout) to it.
#define MDD_CTS 32
struct MddFuse {
    const u64 *U;
    size_t ustride;
    int ell;
    u64 *out;         // [npoly][ell-1][N], or per product when outp[0] is set:
    u64 *outp[MDD_CTS];
    const u64 *addp[MDD_CTS];
};
copse_status ntt_forward_moddown_drop(copse_ctx *ctx, const MddFuse &f, int npoly, cudaStream_t s, bool *done);
copse_status moddown_drop_unfused(copse_ctx *ctx, const MddFuse &f, int npoly, cudaStream_t s);
// The fused forms run on the cluster transform (2^12 <= N <= 2^15); *done = false
// (nothing launched) otherwise, and the caller takes the unfused sequence.
copse_status ntt_forward_modswitch(copse_ctx *ctx, const MsFuse &f, int nc, cudaStream_t s, bool *done);
copse_status ntt_forward_moddown(copse_ctx *ctx, const MdFuse &f, int njobs, cudaStream_t s, bool *done);
// out-of-place inverse transform of residues [0, nr) (prime `fixed` when >= 0) of npoly
// polynomials src + p sstride into dst + p dstride
copse_status ntt_inverse_copy(copse_ctx *ctx, const u64 *src, size_t sstride, u64 *dst, size_t dstride, int npoly,
                              int nr, int fixed, cudaStream_t s, bool *done, const Shoup *scale = nullptr);
// the same for one residue (prime `fixed`) of npoly <= MS_POLYS polynomials held at
// separate addresses src[p] ([N] each) into dst + p N
struct GatherSrc {
    const u64 *p[MS_POLYS];
};
copse_status ntt_inverse_gather(copse_ctx *ctx, const GatherSrc &src, int npoly, u64 *dst, int fixed, cudaStream_t s,
                                bool *done, const Shoup *scale = nullptr);
// ModUp of n_items inputs: the transform of every digit's conversion (xc: the inputs in
// coefficient form, [item][ell][N]) into y [item][nd][ell+alpha][N], each digit's own
// residues copied from x_ntt + item * xs
copse_status ntt_forward_modup(copse_ctx *ctx, const u64 *xc, const u64 *x_ntt, size_t xs, u64 *y, int n_items,
                               int ell, cudaStream_t s, bool *done);
// the same finishing arithmetic without a transform (W: the converted sums already in
// NTT form, [2 njobs][ell][N]; last: unused for MdFuse)
copse_status moddown_finish(copse_ctx *ctx, const MdFuse &f, const u64 *W, int njobs, cudaStream_t s);
copse_status modswitch_finish(copse_ctx *ctx, const MsFuse &f, const u64 *W, int nc, cudaStream_t s);

// ---------------------------------------------------------------- keys
struct copse_keys {
    copse_ctx *ctx = nullptr;
    std::vector<i64> s_host;  // ternary secret coefficients
    u64 *s_hat = nullptr;     // [L+alpha][N] NTT domain, every global prime
    u64 *pk = nullptr;        // [2][L][N] NTT domain
};
struct copse_evk {
    copse_ctx *ctx = nullptr;
    u64 *rlk = nullptr;                 // [ndig][2][L+alpha][N] NTT domain, Montgomery form (x 2^64 mod q)
    std::vector<u64> galois;            // Galois elements with a key
    std::vector<u64 *> gk;              // matching keys, same layout as rlk
    const u64 *find(u64 g) const {
        for (size_t i = 0; i < galois.size(); i++)
            if (galois[i] == g) return gk[i];
        return nullptr;
    }
};
struct copse_ctbuf {
    copse_ctx *ctx = nullptr;
    std::vector<DCt> cts;
    cudaStream_t stream = 0;  // the stream whose work produced the ciphertexts; frees are ordered on it
    ~copse_ctbuf();
};

// ---------------------------------------------------------------- BGV operations (ring.cu)
// All allocate outputs from the pool on stream s and enqueue work on s.
size_t ksk_words(const copse_ctx *c);
// a key copy's words from Montgomery form (the stored form) to plain residues, in place
copse_status ksk_from_mont(copse_ctx *c, u64 *k, cudaStream_t s);
copse_status ct_alloc(copse_ctx *c, DCt *ct, int level, int ncomp, cudaStream_t s);
void ct_free(DCt *ct, cudaStream_t s);
copse_status ct_copy(copse_ctx *c, const DCt &in, DCt *out, cudaStream_t s);
copse_status op_modswitch(copse_ctx *c, const DCt &in, DCt *out, cudaStream_t s);
copse_status op_to_level(copse_ctx *c, DCt *ct, int level, cudaStream_t s);  // in place (replaces)
copse_status op_add(copse_ctx *c, const DCt &a, const DCt &b, DCt *out, bool negate_b, cudaStream_t s);
copse_status op_mul(copse_ctx *c, const copse_evk *evk, const DCt &a, const DCt &b, DCt *out, cudaStream_t s);
// Independent products a * b (+ add) run together: one tensor launch, one ModUp, one
// inner-product launch and one relinearise-and-drop ModDown per group of products at
// a common level.  Each result equals op_mul(a, b) (then op_add(add, .) when add is
// set; add must already be at the product's level).
struct MulJob {
    const DCt *a, *b;
    DCt *out;
    const DCt *add = nullptr;
};
// join_lane >= 0: the addends are still being produced on fork branch 0 of that lane
// (fork_begin); s joins it (fork_join) only before the first finishing store.
copse_status op_mul_many(copse_ctx *c, const copse_evk *evk, const std::vector<MulJob> &jobs, cudaStream_t s,
                         int join_lane = -1);
// modulus switch of ciphertexts held at separate addresses, all at one level > 1
copse_status op_modswitch_cts(copse_ctx *c, const std::vector<const DCt *> &in, std::vector<DCt> &out, cudaStream_t s);
copse_status op_affine(copse_ctx *c, const DCt &x, const DPt &mul, const DPt *add, DCt *out, cudaStream_t s);
// x_j * mul_j + add_j (add on component 0, may be null) for independent jobs, one launch
struct AffineJob {
    const DCt *x;
    const u64 *mul, *add;  // plaintexts [>= x.level][N] NTT domain
    DCt *out;
};
copse_status op_affine_many(copse_ctx *c, const std::vector<AffineJob> &jobs, cudaStream_t s);
copse_status op_rotate(copse_ctx *c, const copse_evk *evk, const DCt &a, uint32_t k, DCt *out, cudaStream_t s);
// Diagonal products sharing the rotations of v: for each accumulator a,
//   out[a] = modswitch(ModDown(sum_{k: rots[k] != 0} pt[a][k] * R_k) + pt[a][k0] * v + add[a])
// with R_k the rotation by rots[k] before its ModDown (one ModUp of v serves all k)
// and k0 the zero rotation if present.  pt[a][k] may be null (zero diagonal);
// pt pointers are NTT-domain [v.level + alpha][N] (extended basis), add[a] [v.level][N].
// raw_out set: the sums ModDown(...) + pt[a][k0] * v go to raw_out [nacc][2][v.level][N]
// (no add, no modswitch) and `out` stays empty.
copse_status op_matmul(copse_ctx *c, const copse_evk *evk, const DCt &v, const std::vector<uint32_t> &rots,
                       const std::vector<std::vector<const u64 *>> &pt, const std::vector<const u64 *> &add,
                       std::vector<DCt> &out, cudaStream_t s, u64 *raw_out = nullptr);
// Baby-step / giant-step products: the baby-step sums of every accumulator
// (matrix acc_mat[x], giant step acc_giant[x]) share the rotations of v by the
// baby amounts (op_matmul, raw); then for each matrix a
//   out[a] = modswitch(ModDown(sum_{k != 0} R_k(inner[a, k])) + inner[a, 0] + add[a]),
// R_k the rotation by k before its ModDown; accumulators of one matrix are
// contiguous with giant steps ascending.
// ---------------------------------------------------------------- encrypted models
// The model's ciphertexts in canonical order (threshold planes, reshuffle diagonals,
// level-k diagonals for k = 1..d, masks), each a secret-key encryption at its level
// of use with only c0 stored; c1 is regenerated from (seed, stream of the index).
// words per accumulator row of the element-major diagonal blocks: baby steps rounded up to 16
inline int mac_row(int nb) { return (nb + 15) / 16 * 16; }

struct EncModel {
    uint64_t ctx_serial = 0;
    u64 seed = 0;
    uint32_t g_r = 0, g_l = 0;       // baby-step plan the diagonals were shifted for
    int lvl_D = 0, lvl_B = 0;
    int p = 0, q = 0, b = 0, d = 0;
    u64 *store = nullptr;            // c0 of the threshold planes and the level masks, [ell][N] each
    // The diagonals of the two products (kind 0 reshuffle, 1 levels) in the layout of the
    // tensor-core multiply-accumulate, one block per matrix of the plan: c0 element-major
    // [ell N][nm][mac_row(nb)] (zero where the plan has no diagonal and in the row padding)
    // and the model ciphertext index of each (accumulator, baby step), [nm][nb] (~0u = none),
    // which names its mask stream.
    struct MacMat {
        u64 *c0 = nullptr;
        uint32_t *idx = nullptr;
        int nm = 0, nb = 0, ell = 0;
        int x0 = 0;                  // the matrix's first accumulator in the plan
    };
    std::vector<MacMat> mac[2];
    // where each model ciphertext's c0 lives: kind -1 in `store` at off[i], else in
    // mac[kind][mat] at position pos = x mac_row(nb) + j of every element
    struct DiagAt {
        int kind = -1, mat = 0;
        uint32_t pos = 0;
    };
    std::vector<DiagAt> at;
    // query ciphertexts per rotation group of each product kind, as last sized from free
    // device memory outside graph capture (0 = not sized yet)
    mutable int group_hint[2] = {0, 0};
    std::vector<size_t> off;         // word offset of each stored ciphertext's c0
    std::vector<int> level;
    BsgsGroup grpR, grpL;            // dense plans (every diagonal present)
    int idx_thr(int i) const { return i; }
    int idx_R(int i) const { return p + i; }
    int idx_lvl(int k, int i) const { return p + q + (k - 1) * b + i; }
    int idx_mask(int k) const { return p + q + d * b + (k - 1); }
    const u64 *c0(int idx) const { return store + off[idx]; }
    ~EncModel();
};
copse_status enc_model_build(copse_ctx *c, const copse_keys *keys, const CompiledForest &f, u64 seed, EncModel &E,
                             cudaStream_t s);
// the full ciphertext idx [2][level][N] (c1 regenerated) into a new buffer
copse_status enc_materialize(copse_ctx *c, const EncModel &E, int idx, DCt *out, cudaStream_t s);
// products of each v[i] with the encrypted reshuffle (kind 0) or level matrices and masks
// (kind 1): out[i][matrix]; the query ciphertexts share every diagonal read
copse_status enc_matmul(copse_ctx *c, const copse_evk *evk, const EncModel &E, const std::vector<DCt> &v, int kind,
                        std::vector<std::vector<DCt>> &out, cudaStream_t s);
// Tensor-core multiply-accumulate of one matrix (encmac.cu): for every element e, query
// ciphertext b < nq and accumulator x of M,
//   (acc0, acc1, acc2)[b][x][e] = sum_j (d0 R0, d0 R1 + d1 R0, d1 R1)
// with d the diagonal (x, j) (c0 from M, c1 regenerated from its stream) and R the rotation
// j of query ciphertext b, R element-major [ell N][ceil(nb / 64)][nq][64][2] (baby step j in
// chunk j / 64 at j % 64; each residue v stored as v' + 0x0080808080808080, v' = v or v - q,
// whichever lies in (-q/2, q/2]); acc [nq][nm][3][ell N] (a_ct words per query ciphertext) is
// written (not added to).
copse_status enc_mac_tc(copse_ctx *c, const EncModel::MacMat &M, const u64 *R, int nq, u64 *acc, size_t a_ct,
                        u64 seed, cudaStream_t s);
// rotations [nb][2][ell N] of query ciphertext b into the element-major layout of enc_mac_tc
// f16 multiply-add operations (2 per digit product) the tensor cores issue for one enc_mac_tc
// launch of nq query ciphertexts (padding rows, columns and baby steps included)
double enc_mac_tc_flops(const EncModel::MacMat &M, int nq, int logN);
copse_status rot_to_elements(copse_ctx *c, const u64 *rot, int nb, int nq, int b, int ell, u64 *R, cudaStream_t s);
// c0 of nc model ciphertexts [nc][ell N] into matrix M at positions pos[i] (device array)
copse_status mac_scatter(copse_ctx *c, const u64 *c0, const uint32_t *pos, int nc, const EncModel::MacMat &M,
                         cudaStream_t s);
// c0 [ell N] of the diagonal at position pos of matrix M
copse_status mac_gather(copse_ctx *c, const EncModel::MacMat &M, uint32_t pos, u64 *c0, cudaStream_t s);

// Giant steps over per-accumulator ciphertexts inner [nacc][2][ell][N] (accumulators of
// one matrix contiguous, giant steps ascending): per matrix a
//   out[a] = modswitch(ModDown(sum_{k != 0} R_k(inner_k)) + inner_0 + add_pt[a] + add_ct[a]).
copse_status giant_phase(copse_ctx *c, const copse_evk *evk, const u64 *inner, int ell, const std::vector<int> &acc_mat,
                         const std::vector<uint32_t> &acc_giant, int n_mat, const std::vector<const u64 *> &add_pt,
                         const std::vector<const u64 *> &add_ct, std::vector<DCt> &out, cudaStream_t s);
// rotations of v by each amount (one ModUp shared by all), out [n][2][v.level][N]
copse_status op_rotations(copse_ctx *c, const copse_evk *evk, const DCt &v, const std::vector<uint32_t> &amounts,
                          u64 *out, cudaStream_t s);
// relinearisation of n 3-component ciphertexts d3 [n][3][ell][N] into out [n][2][ell][N]
copse_status relin_batch(copse_ctx *c, const copse_evk *evk, const u64 *d3, int n, int ell, u64 *out, cudaStream_t s);
// c0 += 1 in place
copse_status op_add_one(copse_ctx *c, DCt &x, cudaStream_t s);
copse_status op_matmul_bsgs(copse_ctx *c, const copse_evk *evk, const DCt &v, const std::vector<uint32_t> &baby,
                            const std::vector<std::vector<const u64 *>> &pt, const std::vector<int> &acc_mat,
                            const std::vector<uint32_t> &acc_giant, int n_mat, const std::vector<const u64 *> &add,
                            std::vector<DCt> &out, cudaStream_t s);

// encode host slot patterns: n patterns of `len` values mod t, repeated every
// `period` slots (period divides N; len <= period), into NTT-domain plaintexts
// [n][level + ext_alpha][N] over q_0..q_{level-1} and, when ext_alpha > 0, the
// first ext_alpha special primes
copse_status encode_patterns(copse_ctx *c, const std::vector<uint32_t> &patterns, int n, int len, int period,
                             int level, int ext_alpha, u64 *out, cudaStream_t s);
copse_status keygen_dev(copse_ctx *c, u64 seed, const std::vector<u64> &galois, copse_keys **keys, copse_evk **evk);
// p planes for n queries: feats [n][nf] (device), layout of the model given by
// K, q, pd, block
// (d_seed: when set, the seed is read from that device word instead of `seed`)
copse_status encrypt_planes(copse_ctx *c, const copse_keys *k, const uint32_t *d_feats, int nq, int nf, int K,
                            int q, int pd, int block, int nseg, int p, u64 seed, std::vector<DCt> &out,
                            cudaStream_t s, const u64 *d_seed = nullptr, int index0 = 0);
// decrypt to N slot values (device output, NTT(mod t) order remapped to slot order)
copse_status decrypt_slots_dev(copse_ctx *c, const copse_keys *k, const DCt &ct, u64 *d_slots, cudaStream_t s);
// where each query's result bits sit: query j owns blocks j nseg .. j nseg + nseg - 1; its
// output bits [off[s], off[s] + len[s]) are the first len[s] slots of block j nseg + s
#define COPSE_MAX_SEG 64
struct SegLayout {
    int nseg, block, total;
    int off[COPSE_MAX_SEG + 1];
};
SegLayout seg_layout(const CompiledForest &f);
copse_status extract_bits(copse_ctx *c, const u64 *d_slots, int nq, const SegLayout &lay, uint8_t *d_bits,
                          cudaStream_t s);
// sessions (copse.cu): asynchronous launch with feature/bit buffers in pinned host or
// device memory; seed_slot is pinned host memory holding the run's seed until it completes
copse_status session_launch(copse_session *S, const uint32_t *feats, uint64_t seed, uint8_t *bits, cudaStream_t s,
                            uint64_t *seed_slot);
size_t session_queries(const copse_session *S);
// model accessors for the server (copse.cu)
uint32_t model_block(const copse_model *m);
uint32_t model_features(const copse_model *m);
uint32_t model_leaves(const copse_model *m);
uint32_t model_precision(const copse_model *m);
int model_log_n(const copse_model *m);

// ---------------------------------------------------------------- persistent work lists (worklist.cu)
// Elementwise ciphertext operations walked by one resident launch (see worklist.cu).
// Polynomials are [level][N] per component, `comp` words apart; dep / dep2 = items whose
// every tile must be done first (-1 none).
#define WL_MAX 256
enum { WL_ADD = 0, WL_SUB = 1, WL_LEAF = 2, WL_TENSOR = 3 };
struct WlItem {
    int kind = WL_ADD, level = 0, dep = -1, dep2 = -1;
    size_t comp = 0;
    const u64 *x = nullptr, *y = nullptr, *z = nullptr;
    u64 *o0 = nullptr, *o1 = nullptr;
};
// runs the items in launches of at most WL_MAX; d_status (3 + WL_MAX ints, may be null):
// [1] = 1 if a wait ran out (the launches after it are skipped), [2] = that item
copse_status worklist_run(copse_ctx *c, const std::vector<WlItem> &items, int timeout_ms, cudaStream_t s,
                          int *d_status = nullptr);

// coefficient-form export/import of one ciphertext (device scratch, host buffer)
copse_status ct_to_coeff_host(copse_ctx *c, const DCt &ct, u64 *host, cudaStream_t s);
copse_status ct_from_coeff_host(copse_ctx *c, const u64 *host, int level, DCt *out, cudaStream_t s);
