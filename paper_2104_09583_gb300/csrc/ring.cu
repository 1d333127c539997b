// BGV ring operations on the device: sampling, key generation, encryption,
// decryption, addition, plaintext and ciphertext products, hybrid key
// switching (relinearisation and rotations, with one shared ModUp for all
// rotations of one ciphertext), modulus switching, and slot encoding.
//
// Ciphertexts live in the bit-reversed NTT domain.  Key switching of a
// polynomial x at level ell (primes q_0..q_{ell-1}, special primes
// p_0..p_{alpha-1}, digits of alpha consecutive primes):
//   ModUp:   y_j = sum_{i in digit j} [x_i * Qhat_i^-1]_{q_i} (centred) * Qhat_i
//   inner:   (u0, u1) = sum_j y_j * ksk_j over q_0..q_{ell-1}, p_0..p_{alpha-1}
//   ModDown: W = sum_k [u_k * t^-1 * Phat_k^-1]_{p_k} (centred) * Phat_k,
//            out_i = (u_i - t*W) * P^-1 mod q_i
// A rotation by Galois element g applies tau_g: X -> X^g to the ModUp output;
// because the digits are centred, tau_g commutes with ModUp, so one ModUp
// serves every rotation of the same ciphertext and the result equals
// rotating first and key switching after.
#include <algorithm>
#include <cstring>

#include "internal.cuh"

namespace {

constexpr int TPB = 256;
constexpr int MAX_ALPHA = 40;
constexpr int MAX_ACC = 8;
constexpr int MM_PRECOMPUTE_ACC = 2;  // accumulators from which the rotations are key-switched first
constexpr int CHUNK_ROT = 64;
constexpr int MM_PARTS = 8;  // rotation ranges with their own partial sums in k_mm_fused
constexpr int RS_CHUNK = 32; // giant-step terms per k_rotsum launch

inline unsigned nblk(size_t n) { return (unsigned)((n + TPB - 1) / TPB); }

// Position n of the bit-reversed NTT holds the evaluation at psi^(2 brev(n) + 1);
// tau_g(a) there equals a at psi^((2 brev(n) + 1) g).


__global__ void k_add(const u64 *a, const u64 *b, u64 *out, int ncomp, int level, int logN, int neg,
                      const PrimeDev *pr) {
    size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t n = (size_t)ncomp * level << logN;
    if (e >= n) return;
    int r = (int)((e >> logN) % level);
    u64 q = pr[r].q;
    out[e] = neg ? sub_mod(a[e], b[e], q) : add_mod(a[e], b[e], q);
}

// c0 += p (p: [level][N]) on component 0 only
__global__ void k_add_plain(u64 *ct, const u64 *p, int level, int logN, const PrimeDev *pr) {
    size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ((size_t)level << logN)) return;
    ct[e] = add_mod(ct[e], p[e], pr[e >> logN].q);
}

__global__ void k_affine(const u64 *x, const u64 *m, const u64 *addp, u64 *out, int level, int logN,
                         const PrimeDev *pr) {
    size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t n = (size_t)level << logN;
    if (e >= 2 * n) return;
    size_t k = e < n ? e : e - n;
    const PrimeDev P = pr[k >> logN];
    u64 v = mul_mod(x[e], m[k], P);
    if (addp && e < n) v = add_mod(v, addp[k], P.q);
    out[e] = v;
}

// many products / affine maps in one launch: blockIdx.y picks the job
struct TensorJobs {
    const u64 *a[MDD_CTS];
    const u64 *b[MDD_CTS];
};
__global__ void k_tensor_many(const TensorJobs J, u64 *out, int level, int logN, const PrimeDev *pr) {
    size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t n = (size_t)level << logN;
    if (e >= n) return;
    const u64 *a = J.a[blockIdx.y], *b = J.b[blockIdx.y];
    u64 *o = out + (size_t)blockIdx.y * 3 * n;
    const PrimeDev P = pr[e >> logN];
    u64 a0 = a[e], a1 = a[n + e], b0 = b[e], b1 = b[n + e];
    o[e] = mul_mod(a0, b0, P);
    o[n + e] = add_mod(mul_mod(a0, b1, P), mul_mod(a1, b0, P), P.q);
    o[2 * n + e] = mul_mod(a1, b1, P);
}

#define AFF_JOBS 64
struct AffineJobsDev {
    const u64 *x[AFF_JOBS], *m[AFF_JOBS], *add[AFF_JOBS];
};
__global__ void k_affine_many(const AffineJobsDev J, u64 *out, int level, int logN, const PrimeDev *pr) {
    size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t n = (size_t)level << logN;
    if (e >= 2 * n) return;
    const int j = blockIdx.y;
    size_t k = e < n ? e : e - n;
    const PrimeDev P = pr[k >> logN];
    u64 v = mul_mod(J.x[j][e], J.m[j][k], P);
    if (J.add[j] && e < n) v = add_mod(v, J.add[j][k], P.q);
    out[(size_t)j * 2 * n + e] = v;
}

__global__ void k_mul_elem(const u64 *a, const u64 *b, u64 *out, int nres, int logN, const PrimeDev *pr) {
    size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ((size_t)nres << logN)) return;
    out[e] = mul_mod(a[e], b[e], pr[e >> logN]);
}

__global__ void k_permute(const u64 *src, u64 *dst, int nres, u64 g, int logN) {
    size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ((size_t)nres << logN)) return;
    size_t r = e >> logN;
    uint32_t n = (uint32_t)(e & ((1u << logN) - 1));
    dst[e] = src[(r << logN) + galois_src(n, g, logN)];
}

// ModUp of every digit: x [ell][N] coefficient form -> y [nd][ell+alpha][N] coefficient form, except the
// digit's own primes, which are copied from x_ntt (the same residues in NTT form)
// blockIdx.y = input item: x [item][ell][N] contiguous, x_ntt at item * xs, y [item][nd][nx][N]
__global__ void k_modup(const u64 *x, const u64 *x_ntt, size_t xs, u64 *y, int ell, int alpha, int L, int NP,
                        int logN, const PrimeDev *pr, KsTables T) {
    const int N = 1 << logN;
    const int nd = (ell + alpha - 1) / alpha;
    size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ((size_t)nd << logN)) return;
    const int j = (int)(e >> logN), n = (int)(e & (N - 1));
    const int lo = j * alpha, hi = min((j + 1) * alpha, ell);
    const int nx = ell + alpha;
    x += (size_t)blockIdx.y * ((size_t)ell << logN);
    x_ntt += (size_t)blockIdx.y * xs;
    y += (size_t)blockIdx.y * nd * ((size_t)nx << logN);
    u64 yv[MAX_ALPHA];
    bool neg[MAX_ALPHA];
    for (int i = lo; i < hi; i++) {
        const u64 qi = pr[i].q;
        u64 v = x[((size_t)i << logN) + n];  // already times modup_inv (inverse transform's scale)
        yv[i - lo] = v;
        neg[i - lo] = v > (qi - 1) / 2;
    }
    u64 *yj = y + (size_t)j * nx * N;
    for (int r = 0; r < nx; r++) {
        const int g = r < ell ? r : L + (r - ell);
        u64 out;
        if (g >= lo && g < hi) {
            out = x_ntt[((size_t)g << logN) + n];  // own prime: already in NTT form, not transformed again
        } else {
            const u64 qg = pr[g].q;
            out = 0;
            for (int i = lo; i < hi; i++) {
                const size_t ti = ((size_t)ell * L + i) * NP + g;
                u64 v = mul_shoup(yv[i - lo], T.modup_hat[ti], qg);
                if (neg[i - lo]) v = sub_mod(v, T.modup_qhat[ti], qg);
                out = add_mod(out, v, qg);
            }
        }
        yj[((size_t)r << logN) + n] = out;
    }
}

// sum_j y_j * k_j over the nd key-switching digits of one element and both key
// components: the key words are in Montgomery form (k 2^64 mod q), the products are summed
// exactly in 128 bits and reduced once (mont_reduce).  yh: digit j's value at
// yh[j * ystride]; key component c of digit j at key[(2 j + c) * kstride].
__device__ __forceinline__ void ks_dot(const u64 *yh, size_t ystride, const u64 *key, size_t kstride, int nd,
                                       const PrimeDev &P, u64 &o0, u64 &o1) {
    Acc128 a0{0, 0}, a1{0, 0};
    for (int j = 0; j < nd; j++) {
        const u64 y = yh[(size_t)j * ystride];
        mac128(a0, y, key[(size_t)(2 * j) * kstride]);
        mac128(a1, y, key[(size_t)(2 * j + 1) * kstride]);
    }
    o0 = mont_reduce(a0, P);
    o1 = mont_reduce(a1, P);
}

struct InnerJob {
    const u64 *ksk;          // [ndig][2][L+alpha][N]
    u64 *out;                // [2][ell+alpha][N]
    u64 g;                   // Galois element applied to the ModUp output, 1 = none
    const u64 *y = nullptr;  // this job's own ModUp digits (null = the launch's shared ones)
    const u64 *pd = nullptr; // adds P * (pd[0], pd[1]) ([2][ell][N]) to the sum's q-residues
    const u64 *pc0 = nullptr;// adds P * tau_g(pc0) ([ell][N]) to component 0's q-residues
};
// a launch's jobs, passed by value (kernel parameter space): no host-to-device copy
struct InnerJobs {
    InnerJob j[CHUNK_ROT];
};

// (u0, u1)[r][n] = sum_j yhat[j][r][tau_g n] * ksk[j][c][ext_prime(r)][n]
__global__ void k_ks_inner(const u64 *yhat, const InnerJobs jobs, int ell, int alpha, int L, int logN,
                           const PrimeDev *pr, const u64 *mdP) {
    const int N = 1 << logN;
    const int nx = ell + alpha, nd = (ell + alpha - 1) / alpha;
    const int NB = L + alpha;
    size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ((size_t)nx << logN)) return;
    const InnerJob J = jobs.j[blockIdx.y];
    const int r = (int)(e >> logN);
    const uint32_t n = (uint32_t)(e & (N - 1));
    const int g = r < ell ? r : L + (r - ell);
    const PrimeDev P = pr[g];
    const uint32_t src = J.g == 1 ? n : galois_src(n, J.g, logN);
    const u64 *yh = J.y ? J.y : yhat;
    u64 acc0, acc1;
    ks_dot(yh + ((size_t)r << logN) + src, (size_t)nx << logN, J.ksk + ((size_t)g << logN) + n, (size_t)NB << logN,
           nd, P, acc0, acc1);
    if (J.pd && r < ell) {
        const u64 Pm = mdP[r];
        acc0 = add_mod(acc0, mul_mod(Pm, J.pd[((size_t)r << logN) + n], P), P.q);
        acc1 = add_mod(acc1, mul_mod(Pm, J.pd[((size_t)(ell + r) << logN) + n], P), P.q);
    }
    if (J.pc0 && r < ell) acc0 = add_mod(acc0, mul_mod(mdP[r], J.pc0[((size_t)r << logN) + src], P), P.q);
    J.out[e] = acc0;
    J.out[((size_t)nx << logN) + e] = acc1;
}

// ModDown conversion: u polys (stride ustride) whose residues ell..ell+alpha-1 are in
// coefficient form -> W polys [ell][N] (stride wstride) in coefficient form
__global__ void k_moddown_conv(const u64 *u, size_t ustride, u64 *W, size_t wstride, int npoly, int ell,
                               int alpha, int L, int logN, const PrimeDev *pr, KsTables T) {
    const int N = 1 << logN;
    size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ((size_t)npoly << logN)) return;
    const int p = (int)(e >> logN), n = (int)(e & (N - 1));
    const u64 *up = u + (size_t)p * ustride;
    u64 yv[MAX_ALPHA];
    bool neg[MAX_ALPHA];
    for (int k = 0; k < alpha; k++) {
        const u64 pk = pr[L + k].q;
        u64 v = up[((size_t)(ell + k) << logN) + n];  // already times md_inv[k] (inverse transform's scale)
        yv[k] = v;
        neg[k] = v > (pk - 1) / 2;
    }
    u64 *wp = W + (size_t)p * wstride;
    for (int i = 0; i < ell; i++) {
        const u64 qi = pr[i].q;
        u64 acc = 0;
        for (int k = 0; k < alpha; k++) {
            u64 v = mul_shoup(yv[k], T.md_hat[(size_t)k * L + i], qi);
            if (neg[k]) v = sub_mod(v, T.md_P[i], qi);
            acc = add_mod(acc, v, qi);
        }
        wp[((size_t)i << logN) + n] = acc;
    }
}

// Diagonal products over shared rotations with one ModDown per sum (double
// hoisting).  For every element (r, n) of the extended basis and each rotation k
// of the chunk:
//   R_k = sum_j tau_k(yhat_j) * ksk_k[j]  (+ P * tau_k(c0) on component 0 at q-primes)
//   acc_a += pt[a][k] * R_k
// The key-switched ciphertexts are never written: each key, each diagonal and
// each accumulator is read once per chunk.
struct MmJob {
    const u64 *ksk;  // [ndig][2][L+alpha][N] NTT domain
    u64 g;           // Galois element
    const u64 *R;    // when set: R_k already computed, [2][ell+alpha][N]
};
struct MmTable {
    MmJob job[CHUNK_ROT];
    const u64 *pt[MAX_ACC * CHUNK_ROT];  // [acc][rotation], [ell+alpha][N], null = zero diagonal
    u64 *acc[MAX_ACC];                   // [2][ell+alpha][N]
};

// grid.y splits the chunk's rotations into gridDim.y contiguous ranges; range y
// accumulates into its own partial sums at acc + y * part_stride (summed later).
template <int NA>
__global__ void __launch_bounds__(256) k_mm_fused(const u64 *yhat, const u64 *c0, int nrot, const MmTable tab,
                                                  size_t part_stride, int ell, int alpha, int L, int logN,
                                                  const PrimeDev *pr, KsTables T) {
    const int N = 1 << logN;
    const int nx = ell + alpha, nd = (ell + alpha - 1) / alpha, NB = L + alpha;
    const size_t n_el = (size_t)nx << logN;
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_el) return;
    const int per = (nrot + (int)gridDim.y - 1) / (int)gridDim.y;
    const int k0 = (int)blockIdx.y * per, k1 = min(nrot, k0 + per);
    if (k0 >= k1) return;
    const size_t poff = (size_t)blockIdx.y * part_stride;
    const int r = (int)(e >> logN);
    const uint32_t n = (uint32_t)(e & (N - 1));
    const int g = r < ell ? r : L + (r - ell);
    const PrimeDev P = pr[g];
    const u64 Pm = r < ell ? T.md_P[r] : 0;
    // the accumulators' diagonal products summed lazily (at most CHUNK_ROT terms per
    // launch on a residue < q), reduced once at the end
    u64 a0[NA], a1[NA];
#pragma unroll
    for (int x = 0; x < NA; x++) {
        a0[x] = tab.acc[x][poff + e];
        a1[x] = tab.acc[x][poff + n_el + e];
    }
    for (int k = k0; k < k1; k++) {
        const MmJob J = tab.job[k];
        u64 u0 = 0, u1 = 0;
        if (J.R) {
            u0 = J.R[e];
            u1 = J.R[n_el + e];
        } else {
            const uint32_t src = galois_src(n, J.g, logN);
            ks_dot(yhat + ((size_t)r << logN) + src, (size_t)nx << logN, J.ksk + ((size_t)g << logN) + n,
                   (size_t)NB << logN, nd, P, u0, u1);
            if (r < ell) u0 = add_mod(u0, mul_mod(Pm, c0[((size_t)r << logN) + src], P), P.q);
        }
#pragma unroll
        for (int x = 0; x < NA; x++) {
            const u64 *p = tab.pt[x * nrot + k];
            if (!p) continue;
            const u64 pv = p[e];
            a0[x] = add_mod(a0[x], mul_mod(pv, u0, P), P.q);
            a1[x] = add_mod(a1[x], mul_mod(pv, u1, P), P.q);
        }
    }
#pragma unroll
    for (int x = 0; x < NA; x++) {
        tab.acc[x][poff + e] = a0[x];
        tab.acc[x][poff + n_el + e] = a1[x];
    }
}

// The same accumulation with every R_k precomputed: a streaming multiply-accumulate
// whose loads for rotation k + 1 are issued before the products of rotation k.
template <int NA>
__global__ void __launch_bounds__(256) k_mm_mac(int nrot, const MmTable tab, size_t part_stride, int ell, int alpha,
                                                int L, int logN, const PrimeDev *pr) {
    const int nx = ell + alpha;
    const size_t n_el = (size_t)nx << logN;
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_el) return;
    const int per = (nrot + (int)gridDim.y - 1) / (int)gridDim.y;
    const int k0 = (int)blockIdx.y * per, k1 = min(nrot, k0 + per);
    if (k0 >= k1) return;
    const size_t poff = (size_t)blockIdx.y * part_stride;
    const int r = (int)(e >> logN);
    const PrimeDev P = pr[r < ell ? r : L + (r - ell)];
    u64 a0[NA], a1[NA];
#pragma unroll
    for (int x = 0; x < NA; x++) {
        a0[x] = tab.acc[x][poff + e];
        a1[x] = tab.acc[x][poff + n_el + e];
    }
    u64 r0, r1, pv[NA];
    auto load = [&](int k, u64 &x0, u64 &x1, u64 *v) {
        const u64 *R = tab.job[k].R;
        x0 = R[e];
        x1 = R[n_el + e];
#pragma unroll
        for (int x = 0; x < NA; x++) {
            const u64 *p = tab.pt[x * nrot + k];
            v[x] = p ? p[e] : 0;
        }
    };
    load(k0, r0, r1, pv);
    for (int k = k0; k < k1; k++) {
        u64 n0 = 0, n1 = 0, nv[NA];
#pragma unroll
        for (int x = 0; x < NA; x++) nv[x] = 0;
        if (k + 1 < k1) load(k + 1, n0, n1, nv);
#pragma unroll
        for (int x = 0; x < NA; x++) {
            if (!tab.pt[x * nrot + k]) continue;
            a0[x] = add_mod(a0[x], mul_mod(pv[x], r0, P), P.q);
            a1[x] = add_mod(a1[x], mul_mod(pv[x], r1, P), P.q);
        }
        r0 = n0;
        r1 = n1;
#pragma unroll
        for (int x = 0; x < NA; x++) pv[x] = nv[x];
    }
#pragma unroll
    for (int x = 0; x < NA; x++) {
        tab.acc[x][poff + e] = a0[x];
        tab.acc[x][poff + n_el + e] = a1[x];
    }
}

// Giant steps of a baby-step / giant-step product: for every element (r, n) of
// the extended basis, over the terms t of the chunk (ciphertext c_t, rotation g_t)
//   acc += sum_j tau_t(yhat_t[j]) * ksk_t[j]   (+ P * tau_t(c_t0) on component 0 at q-primes)
// i.e. the key-switched rotation of each term before its ModDown, summed.
struct RsTerm {
    const u64 *yhat;  // ModUp digits of c_t1, [ndig][ell+alpha][N]
    const u64 *c0;    // c_t0, [ell][N]
    const u64 *ksk;   // [ndig][2][L+alpha][N]
    u64 g;            // Galois element
};
struct RsTable {
    RsTerm t[RS_CHUNK];
};

__global__ void __launch_bounds__(256) k_rotsum(const RsTable tab, int nterm, u64 *acc, int ell, int alpha, int L,
                                                int logN, const PrimeDev *pr, KsTables T) {
    const int N = 1 << logN;
    const int nx = ell + alpha, nd = (ell + alpha - 1) / alpha, NB = L + alpha;
    const size_t n_el = (size_t)nx << logN;
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_el) return;
    const int r = (int)(e >> logN);
    const uint32_t n = (uint32_t)(e & (N - 1));
    const int g = r < ell ? r : L + (r - ell);
    const PrimeDev P = pr[g];
    const u64 Pm = r < ell ? T.md_P[r] : 0;
    u64 a0 = acc[e], a1 = acc[n_el + e];
    for (int k = 0; k < nterm; k++) {
        const RsTerm J = tab.t[k];
        const uint32_t src = galois_src(n, J.g, logN);
        u64 t0, t1;
        ks_dot(J.yhat + ((size_t)r << logN) + src, (size_t)nx << logN, J.ksk + ((size_t)g << logN) + n,
               (size_t)NB << logN, nd, P, t0, t1);
        a0 = add_mod(a0, t0, P.q);
        a1 = add_mod(a1, t1, P.q);
        if (r < ell) a0 = add_mod(a0, mul_mod(Pm, J.c0[((size_t)r << logN) + src], P), P.q);
    }
    acc[e] = a0;
    acc[n_el + e] = a1;
}

// out[i] = sum_y part[y * stride + i] over nparts partial sums of extended-basis
// polynomials ([npoly][ell+alpha][N] each)
__global__ void k_sum_parts(const u64 *part, size_t stride, int nparts, u64 *out, size_t words, int ell, int alpha,
                            int L, int logN, const PrimeDev *pr) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= words) return;
    const int r = (int)((i >> logN) % (size_t)(ell + alpha));
    const u64 q = pr[r < ell ? r : L + (r - ell)].q;
    u64 s = part[i];
    for (int y = 1; y < nparts; y++) s = add_mod(s, part[(size_t)y * stride + i], q);
    out[i] = s;
}

// The last step of matrix products for a batch of outputs (blockIdx.y = output a):
// res_a += pt_mul_a * v + ct_add_a + ct_add2_a (+ pt_add_a on component 0), each term optional
#define FIN_MAX 64
struct FinTable {
    u64 *res[FIN_MAX];             // [2][ell][N]
    const u64 *pt_mul[FIN_MAX];    // first ell residues used
    const u64 *ct_add[FIN_MAX];    // [2][ell][N]
    const u64 *ct_add2[FIN_MAX];   // [2][ell][N]
    const u64 *pt_add[FIN_MAX];    // [ell][N]
};

__global__ void k_finish(const FinTable tab, const u64 *v, int ell, int logN, const PrimeDev *pr) {
    const size_t n = (size_t)ell << logN;
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 2 * n) return;
    const int a = blockIdx.y;
    const size_t k = e < n ? e : e - n;
    const PrimeDev P = pr[k >> logN];
    u64 x = tab.res[a][e];
    if (tab.pt_mul[a]) x = add_mod(x, mul_mod(tab.pt_mul[a][k], v[e], P), P.q);
    if (tab.ct_add[a]) x = add_mod(x, tab.ct_add[a][e], P.q);
    if (tab.ct_add2[a]) x = add_mod(x, tab.ct_add2[a][e], P.q);
    if (e < n && tab.pt_add[a]) x = add_mod(x, tab.pt_add[a][k], P.q);
    tab.res[a][e] = x;
}

// modulus switch, conversion step: last [ncomp][N] coefficients of q_{ell-1} ->
// W [ncomp][ell-1][N] = [last * t^-1]_{q_{ell-1}} (centred) mod q_i
__global__ void k_ms_conv(const u64 *last, u64 *W, int ncomp, int ell, int L, int logN, const PrimeDev *pr,
                          KsTables T) {
    const int N = 1 << logN;
    size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ((size_t)ncomp << logN)) return;
    const int c = (int)(e >> logN), n = (int)(e & (N - 1));
    const u64 ql = pr[ell - 1].q;
    const u64 w = last[e];  // already times t^-1 (inverse transform's scale)
    const bool neg = w > (ql - 1) / 2;
    for (int i = 0; i < ell - 1; i++) {
        // |centred w| < q_{ell-1}/2 < q_i: the chain is in decreasing order
        const u64 qi = pr[i].q;
        W[(((size_t)c * (ell - 1) + i) << logN) + n] = neg ? qi - (ql - w) : w;
    }
}

// uniform residues: out[r][j] for global prime g0 + r, (hi 2^64 + lo) mod q with
// hi, lo the words 2 (g N + j) and 2 (g N + j) + 1 of the stream
__global__ void k_sample_uniform(u64 *out, int nres, int g0, u64 seed, u64 stream, int logN, const PrimeDev *pr) {
    size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ((size_t)nres << logN)) return;
    const int g = g0 + (int)(e >> logN);
    const u64 j = e & ((1ull << logN) - 1);
    const PrimeDev P = pr[g];
    const u64 idx = 2 * (((u64)g << logN) + j);
    const u64 hi = rng_word(seed, stream, idx), lo = rng_word(seed, stream, idx + 1);
    const u64 hm = barrett_wide(0, hi, P), lm = barrett_wide(0, lo, P);
    out[e] = add_mod(mul_shoup(hm, P.r64, P.r64_sh, P.q), lm, P.q);
}

__device__ __forceinline__ i64 sample_small(u64 seed, u64 stream, u64 j, int kind) {
    const u64 w = rng_word(seed, stream, j);
    if (kind == 0) return (i64)(w % 3) - 1;  // ternary
    return (i64)__popcll(w & 0x1FFFFFull) - (i64)__popcll((w >> 21) & 0x1FFFFFull);  // centred binomial, eta 21
}

// small samples scaled by `scale`, as residues of global primes 0..nres-1; raw copy optional
__global__ void k_sample_small(u64 *out, int nres, u64 seed, u64 stream, int kind, i64 scale, i64 *raw, int logN,
                               const PrimeDev *pr) {
    size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ((size_t)nres << logN)) return;
    const int r = (int)(e >> logN);
    const u64 j = e & ((1ull << logN) - 1);
    const i64 v = sample_small(seed, stream, j, kind) * scale;
    out[e] = from_signed(v, pr[r].q);
    if (raw && r == 0) raw[j] = v;
}

// pk0 = t e - a s, pk1 = a  (residues 0..L-1)
__global__ void k_pk(const u64 *a, const u64 *s, const u64 *te, u64 *pk, int L, int logN, const PrimeDev *pr) {
    size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t n = (size_t)L << logN;
    if (e >= n) return;
    const PrimeDev P = pr[e >> logN];
    pk[e] = sub_mod(te[e], mul_mod(a[e], s[e], P), P.q);
    pk[n + e] = a[e];
}

// ksk_j = (t e - a s + [r in digit] (P mod q_r) s', a) over all L+alpha primes
__global__ void k_ksk(const u64 *a, const u64 *s, const u64 *te, const u64 *sfrom, u64 *k, int lo, int hi, int L,
                      int alpha, int logN, const PrimeDev *pr, KsTables T) {
    size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t n = (size_t)(L + alpha) << logN;
    if (e >= n) return;
    const int r = (int)(e >> logN);
    const PrimeDev P = pr[r];
    u64 v = sub_mod(te[e], mul_mod(a[e], s[e], P), P.q);
    if (r >= lo && r < hi) v = add_mod(v, mul_mod(T.md_P[r], sfrom[e], P), P.q);
    // stored in Montgomery form (x 2^64 mod q): the key-switch dot products reduce once
    k[e] = mul_shoup(v, P.r64, P.r64_sh, P.q);
    k[n + e] = mul_shoup(a[e], P.r64, P.r64_sh, P.q);
}

// key words back from Montgomery form (x 2^-64 mod q), residue r of NB per polynomial
__global__ void k_from_mont(u64 *k, size_t words, int NB, int logN, const PrimeDev *pr) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= words) return;
    k[e] = mont_reduce(Acc128{k[e], 0}, pr[(e >> logN) % NB]);
}

// slot patterns -> NTT(mod t) order: out[i][slot_index[s]] = pattern_i[s mod period] (0 past len)
__global__ void k_scatter_pattern(const uint32_t *pat, int npat, int len, int period, int logN,
                                  const uint32_t *slot_index, u64 *out) {
    size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ((size_t)npat << logN)) return;
    const int i = (int)(e >> logN);
    const uint32_t s = (uint32_t)(e & ((1u << logN) - 1));
    const int x = (int)(s % (uint32_t)period);
    out[((size_t)i << logN) + slot_index[s]] = x < len ? pat[(size_t)i * len + x] : 0;
}

// coefficients mod t -> centred -> residues over q_0..q_{level-1} then (nres > level)
// p_0..p_{nres-level-1}: out [n][nres][N]
__global__ void k_lift(const u64 *in, u64 *out, int npoly, int level, int nres, int L, int logN, u64 t,
                       const PrimeDev *pr) {
    size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t per = (size_t)nres << logN;
    if (e >= (size_t)npoly * per) return;
    const size_t i = e / per, k = e - i * per;
    const int rr = (int)(k >> logN);
    const int r = rr < level ? rr : L + (rr - level);
    const u64 c = in[(i << logN) + (k & ((1ull << logN) - 1))];
    const i64 m = c > (t - 1) / 2 ? (i64)c - (i64)t : (i64)c;
    out[e] = from_signed(m, pr[r].q);
}

// bit-planes of the replicated, block-periodic feature vectors, NTT(mod t) order
// block beta of the ciphertext belongs to query beta / nseg (its segment beta mod nseg)
__global__ void k_feature_planes(const uint32_t *feats, int nq, int nf, int K, int q, int pd, int block, int nseg,
                                 int p, int logN, const uint32_t *slot_index, u64 *out) {
    size_t s = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= (1ull << logN)) return;
    const int j = (int)(s / block) / nseg, x = (int)(s % block);
    uint32_t val = 0;
    if (j < nq && x < pd) val = feats[(size_t)j * nf + (x % q) / K];
    const uint32_t pos = slot_index[s];
    for (int i = 0; i < p; i++) out[((size_t)i << logN) + pos] = (val >> i) & 1u;
}

// encryption randomness of plane i (stream base 0x1000000 + 3 i):
// u ternary, x0 = t e0 + m, x1 = t e1, as residues mod q_0..q_{L-1}; the seed is
// read from device memory when seed_ptr is set (replayed graphs)
__global__ void k_enc_prep(const u64 *mt, int p, int index0, u64 seed_val, const u64 *seed_ptr, int L, int logN, u64 t,
                           const PrimeDev *pr, u64 *U, u64 *X0, u64 *X1) {
    size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ((size_t)p << logN)) return;
    // replayed graphs: the run's seed from device memory plus the item's offset
    const u64 seed = seed_ptr ? *seed_ptr + seed_val : seed_val;
    const int i = (int)(e >> logN);
    const u64 n = e & ((1ull << logN) - 1);
    // encryption index index0 + i; every stream id stays below 2^24: stream * 2^40 + idx never wraps
    const u64 sb = 0x500000ull + 3ull * (u64)(index0 + i);
    const i64 u = sample_small(seed, sb, n, 0);
    const i64 e0 = sample_small(seed, sb + 1, n, 1), e1 = sample_small(seed, sb + 2, n, 1);
    const u64 c = mt[e];
    const i64 m = c > (t - 1) / 2 ? (i64)c - (i64)t : (i64)c;
    const i64 x0 = (i64)t * e0 + m, x1 = (i64)t * e1;
    for (int r = 0; r < L; r++) {
        const u64 q = pr[r].q;
        const size_t o = (((size_t)i * L + r) << logN) + n;
        U[o] = from_signed(u, q);
        X0[o] = from_signed(x0, q);
        X1[o] = from_signed(x1, q);
    }
}

// ct_i = (pk0 u + x0, pk1 u + x1), out [p][2][L][N]
__global__ void k_enc_combine(const u64 *pk, const u64 *U, const u64 *X0, const u64 *X1, u64 *out, int p, int L,
                              int logN, const PrimeDev *pr) {
    size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t per = (size_t)L << logN;
    if (e >= (size_t)p * per) return;
    const size_t i = e / per, k = e - i * per;
    const PrimeDev P = pr[k >> logN];
    const u64 u = U[e];
    out[(2 * i) * per + k] = add_mod(mul_mod(pk[k], u, P), X0[e], P.q);
    out[(2 * i + 1) * per + k] = add_mod(mul_mod(pk[per + k], u, P), X1[e], P.q);
}

__global__ void k_dec_dot(const u64 *ct, const u64 *s, u64 *x, int logN, const PrimeDev *pr) {
    size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (1ull << logN)) return;
    const PrimeDev P = pr[0];
    x[e] = add_mod(ct[e], mul_mod(ct[(1ull << logN) + e], s[e], P), P.q);
}

__global__ void k_dec_to_t(const u64 *x, u64 *out, int logN, u64 t, const PrimeDev *pr) {
    size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (1ull << logN)) return;
    const u64 q = pr[0].q, v = x[e];
    if (v > (q - 1) / 2) {
        const u64 m = (q - v) % t;  // centred value is -(q - v)
        out[e] = m ? t - m : 0;
    } else {
        out[e] = v % t;
    }
}

__global__ void k_gather_slots(const u64 *ntt_t, const uint32_t *slot_index, u64 *slots, int logN) {
    size_t s = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= (1ull << logN)) return;
    slots[s] = ntt_t[slot_index[s]];
}

// output bit x of query j: segment s with off[s] <= x < off[s] + len[s], slot x - off[s] of
// block j nseg + s
__global__ void k_extract_bits(const u64 *slots, int nq, const SegLayout lay, uint8_t *bits) {
    size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)nq * lay.total) return;
    const size_t j = e / lay.total;
    const int x = (int)(e - j * lay.total);
    int sg = 0;
    while (sg + 1 < lay.nseg && x >= lay.off[sg + 1]) sg++;
    const u64 v = slots[(j * lay.nseg + sg) * lay.block + (x - lay.off[sg])];
    bits[e] = v == 0 ? 0 : (v == 1 ? 1 : 2);
}

// c0 += 1 (the constant polynomial 1 is 1 at every evaluation point)
__global__ void k_add_one(u64 *c0, int ell, int logN, const PrimeDev *pr) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ((size_t)ell << logN)) return;
    const u64 q = pr[e >> logN].q;
    c0[e] = add_mod(c0[e], 1, q);
}

// ---------------------------------------------------------------- helpers
NttBatch batch(u64 *data, size_t stride, int npoly, int r0, int nr, int ell, int fixed = -1) {
    return NttBatch{data, stride, npoly, r0, nr, ell, fixed};
}

// ModUp of x (NTT domain [ell][N]) for every digit; result NTT domain [nd][ell+alpha][N]
// ModUp of n inputs x_ntt + i * xs (NTT domain [ell][N] each); result NTT domain
// [n][nd][ell+alpha][N].  Where the cluster transform applies: an out-of-place inverse
// transform, then one forward transform whose load does the digits' base conversion
// (and whose skipped blocks copy the digits' own residues); else a copy, an in-place
// inverse transform, the conversion kernel and a forward transform.
copse_status ks_modup_batch(copse_ctx *c, const u64 *x_ntt, size_t xs, int n, int ell, Scratch &sc, u64 **yhat,
                            cudaStream_t s) {
    const int N = c->N, A = c->alpha, nx = ell + A, nd = (ell + A - 1) / A;
    u64 *xc = nullptr, *y = nullptr;
    STATUS_TRY(sc.get(c, &xc, (size_t)n * ell * N));
    STATUS_TRY(sc.get(c, &y, (size_t)n * nd * nx * N));
    bool done = false;
    // the inverse transform's output is scaled by modup_inv (the conversion's first step)
    const Shoup *mu = c->ks.mu_scale + (size_t)ell * c->L;
    STATUS_TRY(ntt_inverse_copy(c, x_ntt, xs, xc, (size_t)ell * N, n, ell, -1, s, &done, mu));
    if (!done) {
        if (n == 1)
            CUDA_TRY(cudaMemcpyAsync(xc, x_ntt, (size_t)ell * N * sizeof(u64), cudaMemcpyDeviceToDevice, s));
        else
            CUDA_TRY(cudaMemcpy2DAsync(xc, (size_t)ell * N * sizeof(u64), x_ntt, xs * sizeof(u64),
                                       (size_t)ell * N * sizeof(u64), n, cudaMemcpyDeviceToDevice, s));
        NttBatch ib = batch(xc, (size_t)ell * N, n, 0, ell, ell);
        ib.scale = mu;
        STATUS_TRY(ntt_inverse(c, ib, s));
    }
    STATUS_TRY(ntt_forward_modup(c, xc, x_ntt, xs, y, n, ell, s, &done));
    if (!done) {
        TIMED("modup", 8.0 * N * n * ((double)ell + (double)nd * nx), s,
              k_modup<<<dim3(nblk((size_t)nd * N), n), TPB, 0, s>>>(xc, x_ntt, xs, y, ell, A, c->L, c->NP, c->logN,
                                                                     c->d_prime, c->ks));
        LAUNCH_CHECK();
        // the digit's own primes already hold the input's NTT values: skip them
        NttBatch nb = batch(y, (size_t)nx * N, n * nd, 0, nx, ell);
        nb.skip_alpha = A;
        nb.skip_period = nd;
        STATUS_TRY(ntt_forward(c, nb, s));
    }
    *yhat = y;
    return COPSE_OK;
}

// ModUp of x (NTT domain [ell][N]) for every digit; result NTT domain [nd][ell+alpha][N]
copse_status ks_modup(copse_ctx *c, const u64 *x_ntt, int ell, Scratch &sc, u64 **yhat, cudaStream_t s) {
    return ks_modup_batch(c, x_ntt, 0, 1, ell, sc, yhat, s);
}

// ModDown of nj extended-basis sums U [nj][2][ell+alpha][N] (NTT domain) finished as f
// says (f.U, f.ustride, f.ell filled here): special residues to coefficients, then the
// fused conversion + transform + finish, or conversion, transform and finish
copse_status moddown_apply(copse_ctx *c, u64 *U, int ell, int nj, MdFuse &f, Scratch &sc, cudaStream_t s) {
    const int N = c->N, A = c->alpha, nx = ell + A;
    f.U = U;
    f.ustride = (size_t)nx * N;
    f.ell = ell;
    NttBatch ib = batch(U, (size_t)nx * N, 2 * nj, ell, A, ell);
    ib.scale = c->ks.md_scale;  // the conversion's first step (md_inv) folded in
    STATUS_TRY(ntt_inverse(c, ib, s));
    bool done = false;
    STATUS_TRY(ntt_forward_moddown(c, f, nj, s, &done));
    if (done) return COPSE_OK;
    u64 *W = nullptr;
    STATUS_TRY(sc.get(c, &W, (size_t)nj * 2 * ell * N));
    TIMED("moddown_conv", 8.0 * N * 2.0 * nj * ((double)A + ell), s,
          k_moddown_conv<<<nblk((size_t)2 * nj * N), TPB, 0, s>>>(U, (size_t)nx * N, W, (size_t)ell * N, 2 * nj, ell, A,
                                                                  c->L, c->logN, c->d_prime, c->ks));
    LAUNCH_CHECK();
    STATUS_TRY(ntt_forward(c, batch(W, (size_t)ell * N, 2 * nj, 0, ell, ell), s));
    return moddown_finish(c, f, W, nj, s);
}

// key-switching inner products for jobs (U [nj][2][ell+alpha][N]), then ModDown finished as f
copse_status ks_apply(copse_ctx *c, const u64 *yhat, int ell, const std::vector<InnerJob> &jobs_h, u64 *U, MdFuse &f,
                      Scratch &sc, cudaStream_t s) {
    const int N = c->N, A = c->alpha, nx = ell + A, nj = (int)jobs_h.size();
    if (nj > CHUNK_ROT || nj > MD_JOBS) { set_error("internal: too many key-switch jobs in one launch"); return COPSE_EINVAL; }
    InnerJobs jobs;
    for (int i = 0; i < nj; i++) jobs.j[i] = jobs_h[i];
    dim3 grid(nblk((size_t)nx * N), nj);
    const int ndg = (ell + A - 1) / A;
    // algorithmic bytes: the digits once, per job the two key components of every digit and
    // the output; products: two per digit and element
    TIMED_OPS("ks_inner", 8.0 * N * ((double)ndg * nx + (double)nj * (2.0 * ndg * nx + 2.0 * nx)),
              2.0 * N * (double)nj * ndg * nx, s,
              k_ks_inner<<<grid, TPB, 0, s>>>(yhat, jobs, ell, A, c->L, c->logN, c->d_prime, c->ks.md_P));
    LAUNCH_CHECK();
    return moddown_apply(c, U, ell, nj, f, sc, s);
}

MdFuse md_fuse() {
    MdFuse f;
    memset(&f, 0, sizeof(f));
    for (int i = 0; i < MD_JOBS; i++) f.gal[i] = 1;
    return f;
}

u64 galois_of_rotation(const copse_ctx *c, uint32_t k) {
    u64 m = 2ull * c->N, g = 1, b = 3;
    for (uint32_t e = k % (uint32_t)(c->N / 2); e; e >>= 1, b = b * b % m)
        if (e & 1) g = g * b % m;
    return g;
}

}  // namespace

// the host pinned staging copies in this file are made with the pageable path
// (cudaMemcpyAsync on host memory the caller owns); callers synchronise.

size_t ksk_words(const copse_ctx *c) { return (size_t)c->ndig * 2 * (c->L + c->alpha) * c->N; }

copse_status ksk_from_mont(copse_ctx *c, u64 *k, cudaStream_t s) {
    const size_t n = ksk_words(c);
    k_from_mont<<<nblk(n), TPB, 0, s>>>(k, n, c->L + c->alpha, c->logN, c->d_prime);
    LAUNCH_CHECK();
    return COPSE_OK;
}

copse_ctbuf::~copse_ctbuf() {
    for (auto &ct : cts) ct_free(&ct, stream);
}

copse_status ct_alloc(copse_ctx *c, DCt *ct, int level, int ncomp, cudaStream_t s) {
    ct->level = level;
    ct->ncomp = ncomp;
    return dev_alloc(c, (void **)&ct->data, (size_t)ncomp * level * c->N * sizeof(u64), s);
}
void ct_free(DCt *ct, cudaStream_t s) {
    dev_free(ct->data, s);
    ct->data = nullptr;
}
copse_status ct_copy(copse_ctx *c, const DCt &in, DCt *out, cudaStream_t s) {
    STATUS_TRY(ct_alloc(c, out, in.level, in.ncomp, s));
    CUDA_TRY(cudaMemcpyAsync(out->data, in.data, (size_t)in.ncomp * in.level * c->N * sizeof(u64),
                             cudaMemcpyDeviceToDevice, s));
    return COPSE_OK;
}

copse_status op_modswitch(copse_ctx *c, const DCt &in, DCt *out, cudaStream_t s) {
    const int ell = in.level, nc = in.ncomp, N = c->N;
    if (ell < 2) { set_error("modulus switch below one prime"); return COPSE_ELEVEL; }
    Scratch sc(s);
    u64 *last = nullptr;
    STATUS_TRY(sc.get(c, &last, (size_t)nc * N));
    // the dropped prime's residues in coefficient form: out of place where the cluster
    // transform applies, else a copy and an in-place inverse transform
    bool inv_done = false;
    STATUS_TRY(ntt_inverse_copy(c, in.data + (size_t)(ell - 1) * N, (size_t)ell * N, last, N, nc, 1, ell - 1, s,
                                &inv_done, c->ks.ms_scale + ell));
    if (!inv_done) {
        CUDA_TRY(cudaMemcpy2DAsync(last, (size_t)N * sizeof(u64), in.data + (size_t)(ell - 1) * N,
                                   (size_t)ell * N * sizeof(u64), (size_t)N * sizeof(u64), nc, cudaMemcpyDeviceToDevice,
                                   s));
        NttBatch ib = batch(last, N, nc, 0, 1, ell, ell - 1);
        ib.scale = c->ks.ms_scale + ell;
        STATUS_TRY(ntt_inverse(c, ib, s));
    }
    STATUS_TRY(ct_alloc(c, out, ell - 1, nc, s));
    // conversion of the dropped prime's residue to the others, transform and finish in one
    // launch where the cluster transform applies; else conversion, transform, finish
    const MsFuse f{last, in.data, out->data, ell};
    bool done = false;
    STATUS_TRY(ntt_forward_modswitch(c, f, nc, s, &done));
    if (!done) {
        u64 *W = nullptr;
        STATUS_TRY(sc.get(c, &W, (size_t)nc * (ell - 1) * N));
        TIMED("ms_conv", 8.0 * N * (double)nc * ell, s,
              k_ms_conv<<<nblk((size_t)nc * N), TPB, 0, s>>>(last, W, nc, ell, c->L, c->logN, c->d_prime, c->ks));
        LAUNCH_CHECK();
        STATUS_TRY(ntt_forward(c, batch(W, (size_t)(ell - 1) * N, nc, 0, ell - 1, ell - 1), s));
        STATUS_TRY(modswitch_finish(c, f, W, nc, s));
    }
    return COPSE_OK;
}

// modulus switch of n ciphertexts held contiguously in [n][2][ell][N], into new ciphertexts
copse_status op_modswitch_many(copse_ctx *c, const u64 *in, int n, int ell, std::vector<DCt> &out, cudaStream_t s) {
    const int N = c->N;
    const size_t per = (size_t)2 * ell * N;
    if (ell < 2) { set_error("modulus switch below one prime"); return COPSE_ELEVEL; }
    out.assign(n, DCt());
    for (int a = 0; a < n; a++) STATUS_TRY(ct_alloc(c, &out[a], ell - 1, 2, s));
    for (int a0 = 0; a0 < n; a0 += MS_POLYS / 2) {
        const int na = std::min(MS_POLYS / 2, n - a0), np = 2 * na;
        const u64 *x = in + (size_t)a0 * per;
        Scratch sc(s);
        u64 *last = nullptr;
        STATUS_TRY(sc.get(c, &last, (size_t)np * N));
        bool done = false;
        STATUS_TRY(ntt_inverse_copy(c, x + (size_t)(ell - 1) * N, (size_t)ell * N, last, N, np, 1, ell - 1, s, &done,
                                    c->ks.ms_scale + ell));
        if (!done) {
            CUDA_TRY(cudaMemcpy2DAsync(last, (size_t)N * sizeof(u64), x + (size_t)(ell - 1) * N,
                                       (size_t)ell * N * sizeof(u64), (size_t)N * sizeof(u64), np,
                                       cudaMemcpyDeviceToDevice, s));
            NttBatch ib = batch(last, N, np, 0, 1, ell, ell - 1);
            ib.scale = c->ks.ms_scale + ell;
            STATUS_TRY(ntt_inverse(c, ib, s));
        }
        MsFuse f{last, x, nullptr, ell};
        for (int p = 0; p < np; p++) f.outp[p] = out[a0 + p / 2].data + (size_t)(p & 1) * (ell - 1) * N;
        STATUS_TRY(ntt_forward_modswitch(c, f, np, s, &done));
        if (!done) {
            u64 *W = nullptr;
            STATUS_TRY(sc.get(c, &W, (size_t)np * (ell - 1) * N));
            TIMED("ms_conv", 8.0 * N * (double)np * ell, s,
                  k_ms_conv<<<nblk((size_t)np * N), TPB, 0, s>>>(last, W, np, ell, c->L, c->logN, c->d_prime, c->ks));
            LAUNCH_CHECK();
            STATUS_TRY(ntt_forward(c, batch(W, (size_t)(ell - 1) * N, np, 0, ell - 1, ell - 1), s));
            STATUS_TRY(modswitch_finish(c, f, W, np, s));
        }
    }
    return COPSE_OK;
}

copse_status op_to_level(copse_ctx *c, DCt *ct, int level, cudaStream_t s) {
    while (ct->level > level) {
        DCt nx;
        STATUS_TRY(op_modswitch(c, *ct, &nx, s));
        ct_free(ct, s);
        *ct = nx;
    }
    return COPSE_OK;
}

// copies of a and b at a common level (only the higher one is switched)
static copse_status aligned(copse_ctx *c, const DCt &a, const DCt &b, DCt *ta, DCt *tb, bool *own_a, bool *own_b,
                            cudaStream_t s) {
    *ta = a;
    *tb = b;
    *own_a = *own_b = false;
    if (a.level > b.level) {
        STATUS_TRY(ct_copy(c, a, ta, s));
        *own_a = true;
        STATUS_TRY(op_to_level(c, ta, b.level, s));
    } else if (b.level > a.level) {
        STATUS_TRY(ct_copy(c, b, tb, s));
        *own_b = true;
        STATUS_TRY(op_to_level(c, tb, a.level, s));
    }
    return COPSE_OK;
}

copse_status op_add(copse_ctx *c, const DCt &a, const DCt &b, DCt *out, bool negate_b, cudaStream_t s) {
    DCt ta, tb;
    bool oa, ob;
    STATUS_TRY(aligned(c, a, b, &ta, &tb, &oa, &ob, s));
    if (ta.ncomp != tb.ncomp) { set_error("component mismatch"); return COPSE_EINVAL; }
    STATUS_TRY(ct_alloc(c, out, ta.level, ta.ncomp, s));
    size_t n = (size_t)ta.ncomp * ta.level * c->N;
    TIMED("add", 8.0 * c->N * 3.0 * ta.ncomp * ta.level, s, k_add<<<nblk(n), TPB, 0, s>>>(ta.data, tb.data, out->data, ta.ncomp, ta.level, c->logN, negate_b ? 1 : 0,
                                  c->d_prime));
    LAUNCH_CHECK();
    if (oa) ct_free(&ta, s);
    if (ob) ct_free(&tb, s);
    return COPSE_OK;
}

copse_status op_mul(copse_ctx *c, const copse_evk *evk, const DCt &a, const DCt &b, DCt *out, cudaStream_t s) {
    return op_mul_many(c, evk, {MulJob{&a, &b, out}}, s);
}

// Products at one level ell, at most MDD_CTS: tensor, then relinearised with one prime
// dropped (the canonical policy) in one ModDown over q_{ell-1} P:
// U = KSraw(d2) + P (d0, d1) over the extended basis.
static copse_status mul_group(copse_ctx *c, const copse_evk *evk, const std::vector<const DCt *> &a,
                              const std::vector<const DCt *> &b, const std::vector<MulJob> &jobs,
                              const std::vector<int> &idx, int ell, cudaStream_t s, int &join_lane) {
    const int N = c->N, A = c->alpha, nx = ell + A, nd = (ell + A - 1) / A, nj = (int)idx.size();
    const size_t per3 = (size_t)3 * ell * N;
    if (ell < 2) { set_error("multiplication at one prime: no prime left to drop"); return COPSE_ELEVEL; }
    for (int i : idx) {
        const DCt *ad = jobs[i].add;
        if (ad && (ad->level != ell - 1 || ad->ncomp != 2)) {
            set_error("internal: addend of a product not at the product's level");
            return COPSE_EINVAL;
        }
    }
    Scratch sc(s);
    u64 *d = nullptr, *yhat = nullptr, *U = nullptr;
    STATUS_TRY(sc.get(c, &d, (size_t)nj * per3));
    TensorJobs tj;
    for (int k = 0; k < nj; k++) {
        tj.a[k] = a[idx[k]]->data;
        tj.b[k] = b[idx[k]]->data;
    }
    TIMED("tensor", 8.0 * N * 7.0 * ell * nj, s,
          k_tensor_many<<<dim3(nblk((size_t)ell * N), nj), TPB, 0, s>>>(tj, d, ell, c->logN, c->d_prime));
    LAUNCH_CHECK();
    STATUS_TRY(ks_modup_batch(c, d + (size_t)2 * ell * N, per3, nj, ell, sc, &yhat, s));
    STATUS_TRY(sc.get(c, &U, (size_t)nj * 2 * nx * N));
    InnerJobs ij;
    for (int k = 0; k < nj; k++)
        ij.j[k] = InnerJob{evk->rlk, U + (size_t)k * 2 * nx * N, 1, yhat + (size_t)k * nd * nx * N, d + (size_t)k * per3};
    TIMED_OPS("ks_inner", 8.0 * N * nj * (3.0 * nd * nx + 2.0 * nx + 2.0 * ell), 2.0 * N * (double)nj * nd * nx, s,
              k_ks_inner<<<dim3(nblk((size_t)nx * N), nj), TPB, 0, s>>>(yhat, ij, ell, A, c->L, c->logN, c->d_prime,
                                                                         c->ks.md_P));
    LAUNCH_CHECK();
    // the dropped prime's and the special residues to coefficients, then the fused
    // conversion + transform + finish (or conversion, transform, finish)
    NttBatch ib = batch(U, (size_t)nx * N, 2 * nj, ell - 1, A + 1, ell);
    ib.scale = c->ks.mdd_scale + (size_t)ell * (A + 1);  // the conversion's first step (mdd_inv) folded in
    STATUS_TRY(ntt_inverse(c, ib, s));
    if (join_lane >= 0) {
        STATUS_TRY(fork_join(c, s, 1, join_lane));
        join_lane = -1;
    }
    MddFuse f{U, (size_t)nx * N, ell, nullptr};
    for (int k = 0; k < nj; k++) {
        const MulJob &J = jobs[idx[k]];
        STATUS_TRY(ct_alloc(c, J.out, ell - 1, 2, s));
        f.outp[k] = J.out->data;
        f.addp[k] = J.add ? J.add->data : nullptr;
    }
    bool done = false;
    STATUS_TRY(ntt_forward_moddown_drop(c, f, 2 * nj, s, &done));
    if (!done) STATUS_TRY(moddown_drop_unfused(c, f, 2 * nj, s));
    return COPSE_OK;
}

copse_status op_mul_many(copse_ctx *c, const copse_evk *evk, const std::vector<MulJob> &jobs, cudaStream_t s,
                         int join_lane) {
    const size_t n = jobs.size();
    std::vector<DCt> ta(n), tb(n);
    std::vector<char> oa(n, 0), ob(n, 0);
    std::vector<const DCt *> pa(n), pb(n);
    copse_status st = COPSE_OK;
    for (size_t i = 0; i < n && st == COPSE_OK; i++) {
        bool x = false, y = false;
        st = aligned(c, *jobs[i].a, *jobs[i].b, &ta[i], &tb[i], &x, &y, s);
        oa[i] = x;
        ob[i] = y;
        pa[i] = &ta[i];
        pb[i] = &tb[i];
    }
    // groups of a common level, in the order of first appearance
    std::vector<int> levels;
    for (size_t i = 0; i < n && st == COPSE_OK; i++)
        if (std::find(levels.begin(), levels.end(), ta[i].level) == levels.end()) levels.push_back(ta[i].level);
    for (int ell : levels) {
        std::vector<int> idx;
        for (size_t i = 0; i < n && st == COPSE_OK; i++) {
            if (ta[i].level != ell) continue;
            idx.push_back((int)i);
            if ((int)idx.size() == MDD_CTS) {
                st = mul_group(c, evk, pa, pb, jobs, idx, ell, s, join_lane);
                idx.clear();
            }
        }
        if (st == COPSE_OK && !idx.empty()) st = mul_group(c, evk, pa, pb, jobs, idx, ell, s, join_lane);
    }
    if (st == COPSE_OK && join_lane >= 0) st = fork_join(c, s, 1, join_lane);
    for (size_t i = 0; i < n; i++) {
        if (oa[i]) ct_free(&ta[i], s);
        if (ob[i]) ct_free(&tb[i], s);
    }
    return st;
}

copse_status op_modswitch_cts(copse_ctx *c, const std::vector<const DCt *> &in, std::vector<DCt> &out, cudaStream_t s) {
    const int N = c->N;
    out.assign(in.size(), DCt());
    if (in.empty()) return COPSE_OK;
    const int ell = in[0]->level;
    if (ell < 2) { set_error("modulus switch below one prime"); return COPSE_ELEVEL; }
    std::vector<std::pair<int, int>> polys;  // (ciphertext, component)
    for (size_t a = 0; a < in.size(); a++) {
        if (in[a]->level != ell) { set_error("internal: ciphertexts of a batched modulus switch at several levels"); return COPSE_EINVAL; }
        STATUS_TRY(ct_alloc(c, &out[a], ell - 1, in[a]->ncomp, s));
        for (int k = 0; k < in[a]->ncomp; k++) polys.emplace_back((int)a, k);
    }
    for (size_t p0 = 0; p0 < polys.size(); p0 += MS_POLYS) {
        const int np = (int)std::min<size_t>(MS_POLYS, polys.size() - p0);
        Scratch sc(s);
        u64 *last = nullptr;
        STATUS_TRY(sc.get(c, &last, (size_t)np * N));
        GatherSrc g{};
        MsFuse f{last, nullptr, nullptr, ell};
        for (int p = 0; p < np; p++) {
            const auto [a, k] = polys[p0 + p];
            g.p[p] = in[a]->data + ((size_t)k * ell + ell - 1) * N;
            f.xp[p] = in[a]->data + (size_t)k * ell * N;
            f.outp[p] = out[a].data + (size_t)k * (ell - 1) * N;
        }
        bool done = false;
        STATUS_TRY(ntt_inverse_gather(c, g, np, last, ell - 1, s, &done, c->ks.ms_scale + ell));
        STATUS_TRY(ntt_forward_modswitch(c, f, np, s, &done));
        if (!done) {
            u64 *W = nullptr;
            STATUS_TRY(sc.get(c, &W, (size_t)np * (ell - 1) * N));
            TIMED("ms_conv", 8.0 * N * (double)np * ell, s,
                  k_ms_conv<<<nblk((size_t)np * N), TPB, 0, s>>>(last, W, np, ell, c->L, c->logN, c->d_prime, c->ks));
            LAUNCH_CHECK();
            STATUS_TRY(ntt_forward(c, batch(W, (size_t)(ell - 1) * N, np, 0, ell - 1, ell - 1), s));
            STATUS_TRY(modswitch_finish(c, f, W, np, s));
        }
    }
    return COPSE_OK;
}

copse_status op_affine(copse_ctx *c, const DCt &x, const DPt &mul, const DPt *add, DCt *out, cudaStream_t s) {
    if (mul.level < x.level || (add && add->level < x.level)) { set_error("plaintext level too low"); return COPSE_EINVAL; }
    DCt r;
    STATUS_TRY(ct_alloc(c, &r, x.level, 2, s));
    TIMED("affine", 8.0 * c->N * 6.0 * x.level, s, k_affine<<<nblk((size_t)2 * x.level * c->N), TPB, 0, s>>>(x.data, mul.data, add ? add->data : nullptr, r.data,
                                                              x.level, c->logN, c->d_prime));
    LAUNCH_CHECK();
    copse_status st = op_modswitch(c, r, out, s);
    ct_free(&r, s);
    return st;
}

copse_status op_affine_many(copse_ctx *c, const std::vector<AffineJob> &jobs, cudaStream_t s) {
    const int N = c->N;
    for (size_t j0 = 0; j0 < jobs.size(); j0 += AFF_JOBS) {
        const int nj = (int)std::min<size_t>(AFF_JOBS, jobs.size() - j0);
        const int ell = jobs[j0].x->level;
        AffineJobsDev J;
        for (int k = 0; k < nj; k++) {
            const AffineJob &a = jobs[j0 + k];
            if (a.x->level != ell || a.x->ncomp != 2) { set_error("internal: affine jobs at several levels"); return COPSE_EINVAL; }
            J.x[k] = a.x->data;
            J.m[k] = a.mul;
            J.add[k] = a.add;
        }
        Scratch sc(s);
        u64 *r = nullptr;
        STATUS_TRY(sc.get(c, &r, (size_t)nj * 2 * ell * N));
        TIMED("affine", 8.0 * N * 6.0 * ell * nj, s,
              k_affine_many<<<dim3(nblk((size_t)2 * ell * N), nj), TPB, 0, s>>>(J, r, ell, c->logN, c->d_prime));
        LAUNCH_CHECK();
        std::vector<DCt> o;
        STATUS_TRY(op_modswitch_many(c, r, nj, ell, o, s));
        for (int k = 0; k < nj; k++) *jobs[j0 + k].out = o[k];
    }
    return COPSE_OK;
}

copse_status op_rotate(copse_ctx *c, const copse_evk *evk, const DCt &a, uint32_t k, DCt *out, cudaStream_t s) {
    const int ell = a.level, N = c->N, A = c->alpha;
    const u64 g = galois_of_rotation(c, k);
    if (g == 1) return ct_copy(c, a, out, s);
    const u64 *key = evk->find(g);
    if (!key) { set_error("no rotation key for amount " + std::to_string(k)); return COPSE_ENOKEY; }
    Scratch sc(s);
    u64 *yhat = nullptr, *U = nullptr;
    STATUS_TRY(ks_modup(c, a.data + (size_t)ell * N, ell, sc, &yhat, s));
    STATUS_TRY(sc.get(c, &U, (size_t)2 * (ell + A) * N));
    STATUS_TRY(ct_alloc(c, out, ell, 2, s));
    // (tau_g c0, 0) + ModDown(KSraw(tau_g c1))
    std::vector<InnerJob> jobs{InnerJob{key, U, g}};
    MdFuse f = md_fuse();
    f.out[0] = out->data;
    f.ocomp = (size_t)ell * N;
    f.add[0] = a.data;
    f.add_comps = 1;
    f.gal[0] = g;
    return ks_apply(c, yhat, ell, jobs, U, f, sc, s);
}

// ModDown of n extended-basis ciphertexts acc [n][2][ell+alpha][N] (NTT domain; the
// special-prime residues are transformed in place) into res [n][2][ell][N].
static copse_status moddown_batch(copse_ctx *c, u64 *acc, int n, int ell, u64 *res, cudaStream_t s) {
    const int N = c->N, nx = ell + c->alpha;
    const size_t per = (size_t)2 * ell * N, ext = (size_t)2 * nx * N;
    for (int j0 = 0; j0 < n; j0 += MD_JOBS) {
        const int nj = std::min(MD_JOBS, n - j0);
        Scratch sc(s);
        MdFuse f = md_fuse();
        for (int i = 0; i < nj; i++) f.out[i] = res + (size_t)(j0 + i) * per;
        f.ocomp = (size_t)ell * N;
        STATUS_TRY(moddown_apply(c, acc + (size_t)j0 * ext, ell, nj, f, sc, s));
    }
    return COPSE_OK;
}

copse_status op_matmul(copse_ctx *c, const copse_evk *evk, const DCt &v, const std::vector<uint32_t> &rots,
                       const std::vector<std::vector<const u64 *>> &pt, const std::vector<const u64 *> &add,
                       std::vector<DCt> &out, cudaStream_t s, u64 *raw_out) {
    const int ell = v.level, N = c->N, A = c->alpha, nx = ell + A, nacc = (int)pt.size(), nrot = (int)rots.size();
    const size_t ext = (size_t)2 * nx * N, per = (size_t)2 * ell * N;
    Scratch sc(s);
    std::vector<u64> gal(nrot);
    std::vector<int> ks_idx;  // rotations that need a key switch
    for (int r = 0; r < nrot; r++) {
        gal[r] = galois_of_rotation(c, rots[r]);
        if (gal[r] == 1) continue;
        if (!evk->find(gal[r])) { set_error("no rotation key for amount " + std::to_string(rots[r])); return COPSE_ENOKEY; }
        bool used = false;
        for (int a = 0; a < nacc; a++) used |= pt[a][r] != nullptr;
        if (used) ks_idx.push_back(r);
    }
    // extended-basis accumulators [nacc][2][ell+alpha][N] and the Q-basis results [nacc][2][ell][N]
    u64 *acc = nullptr, *res = raw_out;
    if (!res) STATUS_TRY(sc.get(c, &res, (size_t)nacc * per));
    CUDA_TRY(cudaMemsetAsync(res, 0, (size_t)nacc * per * sizeof(u64), s));
    if (!ks_idx.empty()) {
        // rotations of a chunk are split into `parts` ranges with their own partial sums
        // (more independent threads to hide the gathers' latency), summed before ModDown
        // (with many accumulators the launches over accumulator chunks already fill the GPU)
        const int parts = nacc > MAX_ACC ? 1 : (int)std::min<size_t>(MM_PARTS, (ks_idx.size() + 7) / 8);
        const size_t part_stride = (size_t)nacc * ext;
        u64 *part = nullptr;
        STATUS_TRY(sc.get(c, &acc, (size_t)nacc * ext));
        STATUS_TRY(sc.get(c, &part, (size_t)parts * part_stride));
        CUDA_TRY(cudaMemsetAsync(part, 0, (size_t)parts * part_stride * sizeof(u64), s));
        u64 *yhat = nullptr;
        STATUS_TRY(ks_modup(c, v.data + (size_t)ell * N, ell, sc, &yhat, s));
        const int nd = (ell + A - 1) / A;
        // several accumulators: compute every rotation's key-switched
        // R_k = KSraw(tau_k c1) + (P tau_k c0, 0) once in one wide launch (instead of once
        // per accumulator chunk, inside the accumulation loop), then stream the products
        u64 *Rall = nullptr;
        if (nacc >= MM_PRECOMPUTE_ACC) {
            STATUS_TRY(sc.get(c, &Rall, ks_idx.size() * ext));
            for (size_t k0 = 0; k0 < ks_idx.size(); k0 += CHUNK_ROT) {
                const int nj = (int)std::min<size_t>(CHUNK_ROT, ks_idx.size() - k0);
                InnerJobs jobs;
                for (int i = 0; i < nj; i++) {
                    const int r = ks_idx[k0 + i];
                    jobs.j[i] = InnerJob{evk->find(gal[r]), Rall + (k0 + i) * ext, gal[r], nullptr, nullptr, v.data};
                }
                TIMED_OPS("ks_inner", 8.0 * N * nj * (2.0 * nd * nx + 2.0 * nx + ell), 2.0 * N * (double)nj * nd * nx, s,
                          k_ks_inner<<<dim3(nblk((size_t)nx * N), nj), TPB, 0, s>>>(yhat, jobs, ell, A, c->L, c->logN,
                                                                                     c->d_prime, c->ks.md_P));
                LAUNCH_CHECK();
            }
        }
        for (size_t k0 = 0; k0 < ks_idx.size(); k0 += CHUNK_ROT) {
            const int nr = (int)std::min<size_t>(CHUNK_ROT, ks_idx.size() - k0);
            for (int a0 = 0; a0 < nacc; a0 += MAX_ACC) {
                const int na = std::min(MAX_ACC, nacc - a0);
                MmTable tab;
                memset(&tab, 0, sizeof(tab));
                int nz_pt = 0;
                for (int x = 0; x < nr; x++) {
                    const int r = ks_idx[k0 + x];
                    tab.job[x] = MmJob{evk->find(gal[r]), gal[r], Rall ? Rall + (k0 + x) * ext : nullptr};
                    for (int a = 0; a < na; a++) {
                        tab.pt[a * nr + x] = pt[a0 + a][r];
                        nz_pt += pt[a0 + a][r] != nullptr;
                    }
                }
                for (int a = 0; a < na; a++) tab.acc[a] = part + (size_t)(a0 + a) * ext;
                // algorithmic bytes: keys, diagonals, accumulators in and out, the rotated
                // digits and c0 once (with R_k precomputed: R_k in place of the keys, digits and c0)
                const double bytes = 8.0 * N * (nz_pt * (double)nx + 4.0 * na * nx * parts +
                                                (Rall ? (double)nr * 2 * nx
                                                      : (double)nr * 2 * nd * nx + (double)nd * nx + ell));
                const dim3 grid(nblk((size_t)nx * N), parts);
#define MM_CASE(K)                                                                                        \
    case K:                                                                                               \
        if (Rall)                                                                                         \
            TIMED("mm_fused", bytes, s,                                                                   \
                  k_mm_mac<K><<<grid, TPB, 0, s>>>(nr, tab, part_stride, ell, A, c->L, c->logN, c->d_prime)); \
        else                                                                                              \
            TIMED("mm_fused", bytes, s,                                                                   \
                  k_mm_fused<K><<<grid, TPB, 0, s>>>(yhat, v.data, nr, tab, part_stride, ell, A, c->L,      \
                                                      c->logN, c->d_prime, c->ks));          \
        break;
                switch (na) {
                    MM_CASE(1) MM_CASE(2) MM_CASE(3) MM_CASE(4) MM_CASE(5) MM_CASE(6) MM_CASE(7) MM_CASE(8)
                    default: set_error("internal: accumulator count"); return COPSE_EINVAL;
                }
#undef MM_CASE
                LAUNCH_CHECK();
            }
        }
        TIMED("sum_parts", 8.0 * (double)(parts + 1) * part_stride, s,
              k_sum_parts<<<nblk(part_stride), TPB, 0, s>>>(part, part_stride, parts, acc, part_stride, ell, A,
                                                            c->L, c->logN, c->d_prime));
        LAUNCH_CHECK();
        // one ModDown per accumulator (both components)
        STATUS_TRY(moddown_batch(c, acc, nacc, ell, res, s));
    }
    out.assign(raw_out ? 0 : nacc, DCt());
    // the zero-rotation terms and the addends of every accumulator in one launch, then the
    // modulus switch of all of them together
    int r0 = -1;
    for (int r = 0; r < nrot; r++)
        if (gal[r] == 1) r0 = r;
    for (int a0 = 0; a0 < nacc; a0 += FIN_MAX) {
        const int na = std::min(FIN_MAX, nacc - a0);
        FinTable tab;
        memset(&tab, 0, sizeof(tab));
        bool any = false;
        for (int i = 0; i < na; i++) {
            const int a = a0 + i;
            tab.res[i] = res + (size_t)a * per;
            tab.pt_mul[i] = r0 >= 0 ? pt[a][r0] : nullptr;
            tab.pt_add[i] = (!raw_out && add.size() > (size_t)a) ? add[a] : nullptr;
            any |= tab.pt_mul[i] || tab.pt_add[i];
        }
        if (!any) continue;
        TIMED("mm_finish", 8.0 * N * 5.0 * ell * na, s,
              k_finish<<<dim3(nblk(per), na), TPB, 0, s>>>(tab, v.data, ell, c->logN, c->d_prime));
        LAUNCH_CHECK();
    }
    if (raw_out) return COPSE_OK;
    return op_modswitch_many(c, res, nacc, ell, out, s);
}

copse_status giant_phase(copse_ctx *c, const copse_evk *evk, const u64 *inner, int ell, const std::vector<int> &acc_mat,
                         const std::vector<uint32_t> &acc_giant, int n_mat, const std::vector<const u64 *> &add_pt,
                         const std::vector<const u64 *> &add_ct, std::vector<DCt> &out, cudaStream_t s) {
    const int N = c->N, A = c->alpha, nx = ell + A, nd = (ell + A - 1) / A;
    const int nacc = (int)acc_mat.size();
    const size_t per = (size_t)2 * ell * N, ext = (size_t)2 * nx * N;
    std::vector<u64> gal(nacc);
    bool any_rot = false;
    for (int x = 0; x < nacc; x++) {
        gal[x] = galois_of_rotation(c, acc_giant[x]);
        if (gal[x] == 1) continue;
        any_rot = true;
        if (!evk->find(gal[x])) {
            set_error("no rotation key for amount " + std::to_string(acc_giant[x]));
            return COPSE_ENOKEY;
        }
    }
    Scratch sc(s);
    u64 *acc = nullptr, *res = nullptr;
    STATUS_TRY(sc.get(c, &res, (size_t)n_mat * per));
    if (!any_rot) {
        CUDA_TRY(cudaMemsetAsync(res, 0, (size_t)n_mat * per * sizeof(u64), s));
    } else {
        // per matrix, the rotated accumulators key-switched into one extended-basis sum
        // (the ModUps of a matrix's terms batched), one ModDown for all matrices
        STATUS_TRY(sc.get(c, &acc, (size_t)n_mat * ext));
        CUDA_TRY(cudaMemsetAsync(acc, 0, (size_t)n_mat * ext * sizeof(u64), s));
        for (int a = 0; a < n_mat; a++) {
            int x0 = 0;
            while (x0 < nacc && (acc_mat[x0] != a || gal[x0] == 1)) x0++;
            int x1 = x0;
            while (x1 < nacc && acc_mat[x1] == a && gal[x1] != 1) x1++;
            if (x0 == x1) continue;
            for (int x = x1; x < nacc; x++)
                if (acc_mat[x] == a && gal[x] != 1) {
                    set_error("internal: giant steps of a matrix not contiguous");
                    return COPSE_EINVAL;
                }
            Scratch sk(s);  // this matrix's ModUp digits, freed (stream-ordered) after its launches
            u64 *yhat = nullptr;
            STATUS_TRY(ks_modup_batch(c, inner + (size_t)x0 * per + (size_t)ell * N, per, x1 - x0, ell, sk, &yhat, s));
            for (int k0 = x0; k0 < x1; k0 += RS_CHUNK) {
                const int nt = std::min(RS_CHUNK, x1 - k0);
                RsTable tab;
                memset(&tab, 0, sizeof(tab));
                for (int i = 0; i < nt; i++) {
                    const int x = k0 + i;
                    tab.t[i] = RsTerm{yhat + (size_t)(x - x0) * nd * nx * N, inner + (size_t)x * per,
                                      evk->find(gal[x]), gal[x]};
                }
                const double bytes = 8.0 * N * ((double)nt * (2.0 * nd * nx + (double)nd * nx + ell) + 4.0 * nx);
                TIMED("rotsum", bytes, s,
                      k_rotsum<<<nblk((size_t)nx * N), TPB, 0, s>>>(tab, nt, acc + (size_t)a * ext, ell, A, c->L,
                                                                    c->logN, c->d_prime, c->ks));
                LAUNCH_CHECK();
            }
        }
        STATUS_TRY(moddown_batch(c, acc, n_mat, ell, res, s));
    }
    // + the giant-step-0 sums, + the plaintext or ciphertext addend, in one launch for every
    // matrix, then the modulus switch of all of them together
    for (int a0 = 0; a0 < n_mat; a0 += FIN_MAX) {
        const int na = std::min(FIN_MAX, n_mat - a0);
        FinTable tab;
        memset(&tab, 0, sizeof(tab));
        for (int i = 0; i < na; i++) {
            const int a = a0 + i;
            tab.res[i] = res + (size_t)a * per;
            for (int x = 0; x < nacc; x++)
                if (acc_mat[x] == a && gal[x] == 1) tab.ct_add[i] = inner + (size_t)x * per;
            tab.pt_add[i] = add_pt.size() > (size_t)a ? add_pt[a] : nullptr;
            tab.ct_add2[i] = add_ct.size() > (size_t)a ? add_ct[a] : nullptr;
        }
        TIMED("add", 8.0 * N * 5.0 * ell * na, s,
              k_finish<<<dim3(nblk(per), na), TPB, 0, s>>>(tab, nullptr, ell, c->logN, c->d_prime));
        LAUNCH_CHECK();
    }
    return op_modswitch_many(c, res, n_mat, ell, out, s);
}

copse_status op_matmul_bsgs(copse_ctx *c, const copse_evk *evk, const DCt &v, const std::vector<uint32_t> &baby,
                            const std::vector<std::vector<const u64 *>> &pt, const std::vector<int> &acc_mat,
                            const std::vector<uint32_t> &acc_giant, int n_mat, const std::vector<const u64 *> &add,
                            std::vector<DCt> &out, cudaStream_t s) {
    const int ell = v.level, nacc = (int)pt.size();
    Scratch sc(s);
    // baby steps: inner[x] = sum_j d'_{x,j} * rot(v, j), one ModDown each
    u64 *inner = nullptr;
    STATUS_TRY(sc.get(c, &inner, (size_t)nacc * 2 * ell * c->N));
    std::vector<DCt> none;
    STATUS_TRY(op_matmul(c, evk, v, baby, pt, {}, none, s, inner));
    return giant_phase(c, evk, inner, ell, acc_mat, acc_giant, n_mat, add, {}, out, s);
}

copse_status op_rotations(copse_ctx *c, const copse_evk *evk, const DCt &v, const std::vector<uint32_t> &amounts,
                          u64 *out, cudaStream_t s) {
    const int ell = v.level, N = c->N, A = c->alpha, nx = ell + A;
    const size_t per = (size_t)2 * ell * N;
    std::vector<int> ks;
    std::vector<u64> gal(amounts.size());
    for (size_t x = 0; x < amounts.size(); x++) {
        gal[x] = galois_of_rotation(c, amounts[x]);
        if (gal[x] == 1) {
            CUDA_TRY(cudaMemcpyAsync(out + x * per, v.data, per * sizeof(u64), cudaMemcpyDeviceToDevice, s));
            continue;
        }
        if (!evk->find(gal[x])) { set_error("no rotation key for amount " + std::to_string(amounts[x])); return COPSE_ENOKEY; }
        ks.push_back((int)x);
    }
    if (ks.empty()) return COPSE_OK;
    Scratch sc(s);
    u64 *yhat = nullptr;
    STATUS_TRY(ks_modup(c, v.data + (size_t)ell * N, ell, sc, &yhat, s));
    for (size_t k0 = 0; k0 < ks.size(); k0 += CHUNK_ROT) {
        const int nj = (int)std::min<size_t>(CHUNK_ROT, ks.size() - k0);
        Scratch sk(s);
        u64 *U = nullptr;
        STATUS_TRY(sk.get(c, &U, (size_t)nj * 2 * nx * N));
        std::vector<InnerJob> jobs;
        MdFuse f = md_fuse();
        f.ocomp = (size_t)ell * N;
        f.add_comps = 1;
        for (int i = 0; i < nj; i++) {
            const int x = ks[k0 + i];
            jobs.push_back(InnerJob{evk->find(gal[x]), U + (size_t)i * 2 * nx * N, gal[x]});
            f.out[i] = out + (size_t)x * per;
            f.add[i] = v.data;
            f.gal[i] = gal[x];
        }
        STATUS_TRY(ks_apply(c, yhat, ell, jobs, U, f, sk, s));
    }
    return COPSE_OK;
}

copse_status relin_batch(copse_ctx *c, const copse_evk *evk, const u64 *d3, int n, int ell, u64 *out, cudaStream_t s) {
    const int N = c->N, A = c->alpha, nx = ell + A, nd = (ell + A - 1) / A;
    const size_t per3 = (size_t)3 * ell * N, per = (size_t)2 * ell * N;
    for (int x0 = 0; x0 < n; x0 += CHUNK_ROT) {
        const int nj = std::min(CHUNK_ROT, n - x0);
        Scratch sk(s);
        u64 *yhat = nullptr, *U = nullptr;
        STATUS_TRY(ks_modup_batch(c, d3 + (size_t)x0 * per3 + (size_t)2 * ell * N, per3, nj, ell, sk, &yhat, s));
        STATUS_TRY(sk.get(c, &U, (size_t)nj * 2 * nx * N));
        std::vector<InnerJob> jobs;
        MdFuse f = md_fuse();
        f.ocomp = (size_t)ell * N;
        f.acomp = (size_t)ell * N;
        f.add_comps = 2;
        for (int i = 0; i < nj; i++) {
            jobs.push_back(InnerJob{evk->rlk, U + (size_t)i * 2 * nx * N, 1, yhat + (size_t)i * nd * nx * N});
            f.out[i] = out + (size_t)(x0 + i) * per;
            f.add[i] = d3 + (size_t)(x0 + i) * per3;
        }
        STATUS_TRY(ks_apply(c, yhat, ell, jobs, U, f, sk, s));
    }
    return COPSE_OK;
}

copse_status op_add_one(copse_ctx *c, DCt &x, cudaStream_t s) {
    k_add_one<<<nblk((size_t)x.level * c->N), TPB, 0, s>>>(x.data, x.level, c->logN, c->d_prime);
    LAUNCH_CHECK();
    return COPSE_OK;
}

copse_status encode_patterns(copse_ctx *c, const std::vector<uint32_t> &patterns, int n, int len, int period,
                             int level, int ext_alpha, u64 *out, cudaStream_t s) {
    const int N = c->N, nres = level + ext_alpha;
    if (n <= 0) return COPSE_OK;
    Scratch sc(s);
    u64 *pat = nullptr, *mt = nullptr;
    STATUS_TRY(sc.get(c, &pat, ((size_t)n * len + 1) / 2 + 1));
    STATUS_TRY(sc.get(c, &mt, (size_t)n * N));
    CUDA_TRY(cudaMemcpyAsync(pat, patterns.data(), (size_t)n * len * sizeof(uint32_t), cudaMemcpyHostToDevice, s));
    k_scatter_pattern<<<nblk((size_t)n * N), TPB, 0, s>>>((const uint32_t *)pat, n, len, period, c->logN,
                                                          c->d_slot_index, mt);
    LAUNCH_CHECK();
    STATUS_TRY(ntt_inverse(c, batch(mt, N, n, 0, 1, 0, c->t_index()), s));
    k_lift<<<nblk((size_t)n * nres * N), TPB, 0, s>>>(mt, out, n, level, nres, c->L, c->logN, c->t, c->d_prime);
    LAUNCH_CHECK();
    STATUS_TRY(ntt_forward(c, batch(out, (size_t)nres * N, n, 0, nres, level), s));
    // the pattern staging buffer is read by the device before the caller's vector dies
    CUDA_TRY(cudaStreamSynchronize(s));
    return COPSE_OK;
}

static copse_status make_switch_key(copse_ctx *c, u64 seed, u64 sb, const u64 *s_hat, const u64 *sfrom, u64 *ksk,
                                    Scratch &sc, cudaStream_t s) {
    const int N = c->N, NB = c->L + c->alpha;
    u64 *a = nullptr, *te = nullptr;
    STATUS_TRY(sc.get(c, &a, (size_t)NB * N));
    STATUS_TRY(sc.get(c, &te, (size_t)NB * N));
    for (int j = 0; j < c->ndig; j++) {
        k_sample_uniform<<<nblk((size_t)NB * N), TPB, 0, s>>>(a, NB, 0, seed, sb + 2 * j, c->logN, c->d_prime);
        LAUNCH_CHECK();
        k_sample_small<<<nblk((size_t)NB * N), TPB, 0, s>>>(te, NB, seed, sb + 2 * j + 1, 1, (i64)c->t, nullptr,
                                                            c->logN, c->d_prime);
        LAUNCH_CHECK();
        STATUS_TRY(ntt_forward(c, batch(a, (size_t)NB * N, 1, 0, NB, NB), s));
        STATUS_TRY(ntt_forward(c, batch(te, (size_t)NB * N, 1, 0, NB, NB), s));
        const int lo = j * c->alpha, hi = std::min((j + 1) * c->alpha, c->L);
        k_ksk<<<nblk((size_t)NB * N), TPB, 0, s>>>(a, s_hat, te, sfrom, ksk + (size_t)j * 2 * NB * N, lo, hi, c->L,
                                                   c->alpha, c->logN, c->d_prime, c->ks);
        LAUNCH_CHECK();
    }
    return COPSE_OK;
}

copse_status keygen_dev(copse_ctx *c, u64 seed, const std::vector<u64> &galois, copse_keys **keys_out,
                        copse_evk **evk_out) {
    cudaStream_t s = 0;
    const int N = c->N, L = c->L, NB = c->L + c->alpha;
    copse_keys *K = new copse_keys();
    copse_evk *E = new copse_evk();
    K->ctx = E->ctx = c;
    auto fail = [&](copse_status st) {
        cudaStreamSynchronize(s);
        dev_free(K->s_hat, s);
        dev_free(K->pk, s);
        dev_free(E->rlk, s);
        for (u64 *p : E->gk) dev_free(p, s);
        delete K;
        delete E;
        return st;
    };
    Scratch sc(s);
    copse_status st;
    u64 *raw = nullptr, *a = nullptr, *te = nullptr, *sf = nullptr;
    if ((st = dev_alloc(c, (void **)&K->s_hat, (size_t)NB * N * 8, s)) || (st = dev_alloc(c, (void **)&K->pk, (size_t)2 * L * N * 8, s)) ||
        (st = sc.get(c, &raw, N)) || (st = sc.get(c, &a, (size_t)L * N)) || (st = sc.get(c, &te, (size_t)L * N)) ||
        (st = sc.get(c, &sf, (size_t)NB * N)))
        return fail(st);
    // secret: ternary, stream 1
    k_sample_small<<<nblk((size_t)NB * N), TPB, 0, s>>>(K->s_hat, NB, seed, 1, 0, 1, (i64 *)raw, c->logN, c->d_prime);
    if ((st = ntt_forward(c, batch(K->s_hat, (size_t)NB * N, 1, 0, NB, NB), s))) return fail(st);
    // public key: a from stream 2 (primes 0..L-1), e from stream 3
    k_sample_uniform<<<nblk((size_t)L * N), TPB, 0, s>>>(a, L, 0, seed, 2, c->logN, c->d_prime);
    k_sample_small<<<nblk((size_t)L * N), TPB, 0, s>>>(te, L, seed, 3, 1, (i64)c->t, nullptr, c->logN, c->d_prime);
    if ((st = ntt_forward(c, batch(a, (size_t)L * N, 1, 0, L, L), s))) return fail(st);
    if ((st = ntt_forward(c, batch(te, (size_t)L * N, 1, 0, L, L), s))) return fail(st);
    k_pk<<<nblk((size_t)L * N), TPB, 0, s>>>(a, K->s_hat, te, K->pk, L, c->logN, c->d_prime);
    // relinearisation key: s' = s^2, streams 16 + 2j, 17 + 2j
    const size_t kw = ksk_words(c);
    if ((st = dev_alloc(c, (void **)&E->rlk, kw * 8, s))) return fail(st);
    k_mul_elem<<<nblk((size_t)NB * N), TPB, 0, s>>>(K->s_hat, K->s_hat, sf, NB, c->logN, c->d_prime);
    if ((st = make_switch_key(c, seed, 16, K->s_hat, sf, E->rlk, sc, s))) return fail(st);
    // rotation keys: s' = tau_g(s), streams 0x10000 + 64 g + (2j, 2j + 1)
    for (u64 g : galois) {
        if (g == 1 || E->find(g)) continue;
        u64 *k = nullptr;
        if ((st = dev_alloc(c, (void **)&k, kw * 8, s))) return fail(st);
        E->galois.push_back(g);
        E->gk.push_back(k);
        k_permute<<<nblk((size_t)NB * N), TPB, 0, s>>>(K->s_hat, sf, NB, g, c->logN);
        if ((st = make_switch_key(c, seed, 0x10000ull + 64ull * g, K->s_hat, sf, k, sc, s))) return fail(st);
    }
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
        set_error("key generation kernels failed");
        return fail(COPSE_ECUDA);
    }
    K->s_host.resize(N);
    if (cudaMemcpy(K->s_host.data(), raw, N * sizeof(i64), cudaMemcpyDeviceToHost) != cudaSuccess) {
        set_error("secret key copy failed");
        return fail(COPSE_ECUDA);
    }
    *keys_out = K;
    *evk_out = E;
    return COPSE_OK;
}

copse_status encrypt_planes(copse_ctx *c, const copse_keys *k, const uint32_t *d_feats, int nq, int nf, int K,
                            int q, int pd, int block, int nseg, int p, u64 seed, std::vector<DCt> &out,
                            cudaStream_t s, const u64 *d_seed, int index0) {
    const int N = c->N, L = c->L;
    Scratch sc(s);
    u64 *mt = nullptr, *U = nullptr, *X0 = nullptr, *X1 = nullptr, *cts = nullptr;
    STATUS_TRY(sc.get(c, &mt, (size_t)p * N));
    STATUS_TRY(sc.get(c, &U, (size_t)p * L * N));
    STATUS_TRY(sc.get(c, &X0, (size_t)p * L * N));
    STATUS_TRY(sc.get(c, &X1, (size_t)p * L * N));
    k_feature_planes<<<nblk(N), TPB, 0, s>>>(d_feats, nq, nf, K, q, pd, block, nseg, p, c->logN, c->d_slot_index, mt);
    LAUNCH_CHECK();
    STATUS_TRY(ntt_inverse(c, batch(mt, N, p, 0, 1, 0, c->t_index()), s));
    if (index0 < 0 || index0 + p > 0x100000) { set_error("encryption index out of range"); return COPSE_EINVAL; }
    k_enc_prep<<<nblk((size_t)p * N), TPB, 0, s>>>(mt, p, index0, seed, d_seed, L, c->logN, c->t, c->d_prime, U, X0, X1);
    LAUNCH_CHECK();
    STATUS_TRY(ntt_forward(c, batch(U, (size_t)L * N, p, 0, L, L), s));
    STATUS_TRY(ntt_forward(c, batch(X0, (size_t)L * N, p, 0, L, L), s));
    STATUS_TRY(ntt_forward(c, batch(X1, (size_t)L * N, p, 0, L, L), s));
    STATUS_TRY(dev_alloc(c, (void **)&cts, (size_t)p * 2 * L * N * 8, s));
    k_enc_combine<<<nblk((size_t)p * L * N), TPB, 0, s>>>(k->pk, U, X0, X1, cts, p, L, c->logN, c->d_prime);
    LAUNCH_CHECK();
    // appended to `out`
    for (int i = 0; i < p; i++) {
        DCt ct;
        ct.level = L;
        ct.ncomp = 2;
        STATUS_TRY(ct_alloc(c, &ct, L, 2, s));
        CUDA_TRY(cudaMemcpyAsync(ct.data, cts + (size_t)i * 2 * L * N, (size_t)2 * L * N * 8, cudaMemcpyDeviceToDevice, s));
        out.push_back(ct);
    }
    dev_free(cts, s);
    return COPSE_OK;
}

copse_status decrypt_slots_dev(copse_ctx *c, const copse_keys *k, const DCt &ct, u64 *d_slots, cudaStream_t s) {
    const int N = c->N;
    DCt cur;
    STATUS_TRY(ct_copy(c, ct, &cur, s));
    copse_status st = op_to_level(c, &cur, 1, s);
    if (st) { ct_free(&cur, s); return st; }
    Scratch sc(s);
    u64 *x = nullptr, *xt = nullptr;
    STATUS_TRY(sc.get(c, &x, N));
    STATUS_TRY(sc.get(c, &xt, N));
    k_dec_dot<<<nblk(N), TPB, 0, s>>>(cur.data, k->s_hat, x, c->logN, c->d_prime);
    LAUNCH_CHECK();
    ct_free(&cur, s);
    STATUS_TRY(ntt_inverse(c, batch(x, N, 1, 0, 1, 1), s));
    k_dec_to_t<<<nblk(N), TPB, 0, s>>>(x, xt, c->logN, c->t, c->d_prime);
    LAUNCH_CHECK();
    STATUS_TRY(ntt_forward(c, batch(xt, N, 1, 0, 1, 0, c->t_index()), s));
    k_gather_slots<<<nblk(N), TPB, 0, s>>>(xt, c->d_slot_index, d_slots, c->logN);
    LAUNCH_CHECK();
    return COPSE_OK;
}

copse_status extract_bits(copse_ctx *c, const u64 *d_slots, int nq, const SegLayout &lay, uint8_t *d_bits,
                          cudaStream_t s) {
    if (nq * lay.total == 0) return COPSE_OK;
    k_extract_bits<<<nblk((size_t)nq * lay.total), TPB, 0, s>>>(d_slots, nq, lay, d_bits);
    LAUNCH_CHECK();
    return COPSE_OK;
}

copse_status ct_to_coeff_host(copse_ctx *c, const DCt &ct, u64 *host, cudaStream_t s) {
    const size_t words = (size_t)ct.ncomp * ct.level * c->N;
    Scratch sc(s);
    u64 *tmp = nullptr;
    STATUS_TRY(sc.get(c, &tmp, words));
    CUDA_TRY(cudaMemcpyAsync(tmp, ct.data, words * 8, cudaMemcpyDeviceToDevice, s));
    STATUS_TRY(ntt_inverse(c, batch(tmp, (size_t)ct.level * c->N, ct.ncomp, 0, ct.level, ct.level), s));
    CUDA_TRY(cudaMemcpyAsync(host, tmp, words * 8, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return COPSE_OK;
}

copse_status ct_from_coeff_host(copse_ctx *c, const u64 *host, int level, DCt *out, cudaStream_t s) {
    const size_t words = (size_t)2 * level * c->N;
    STATUS_TRY(ct_alloc(c, out, level, 2, s));
    CUDA_TRY(cudaMemcpyAsync(out->data, host, words * 8, cudaMemcpyHostToDevice, s));
    STATUS_TRY(ntt_forward(c, batch(out->data, (size_t)level * c->N, 2, 0, level, level), s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return COPSE_OK;
}

extern "C" copse_status copse_poly_mul(copse_ctx *c, const uint64_t *a, const uint64_t *b, uint64_t *out,
                                       uint32_t n_res, void *stream) {
    if (!c || !a || !b || !out || n_res < 1 || (int)n_res > c->L) { set_error("bad argument"); return COPSE_EINVAL; }
    cudaStream_t s = (cudaStream_t)stream;
    const int N = c->N, nr = (int)n_res;
    const size_t words = (size_t)nr * N;
    Scratch sc(s);
    u64 *fa = nullptr, *fb = nullptr;
    STATUS_TRY(sc.get(c, &fa, words));
    STATUS_TRY(sc.get(c, &fb, words));
    CUDA_TRY(cudaMemcpyAsync(fa, a, words * 8, cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(fb, b, words * 8, cudaMemcpyDeviceToDevice, s));
    STATUS_TRY(ntt_forward(c, batch(fa, words, 1, 0, nr, nr), s));
    STATUS_TRY(ntt_forward(c, batch(fb, words, 1, 0, nr, nr), s));
    k_mul_elem<<<nblk(words), TPB, 0, s>>>(fa, fb, out, nr, c->logN, c->d_prime);
    LAUNCH_CHECK();
    return ntt_inverse(c, batch(out, words, 1, 0, nr, nr), s);
}
