// Encrypted models: the model owner also owns the data (Maurice = Diane,
// Section 8.3 of the paper), encrypts the threshold planes, every diagonal of
// the reshuffle and level matrices (zero ones included: p + q + d(b+1)
// ciphertexts, Table 1d) and the level masks, and the server evaluates
// Algorithm 1 with ciphertext x ciphertext products.
//
// Layout: each model ciphertext is a secret-key encryption whose mask c1 = a
// is drawn from the counter generator in evaluation form, so only c0 is kept
// in HBM and c1 is regenerated where it is consumed (half the bytes of a full
// ciphertext).  At NTT position k of prime r (evaluation point
// psi_r^(2 brev(k) + 1)) a = uniform residue number (r N + brev(k)) of the
// ciphertext's stream; c0 = m + t e - a s.
#include <algorithm>
#include <cstring>
#include <functional>

#include "internal.cuh"

namespace {

constexpr int TPB = 256;
constexpr int EM_ACC = 8;      // accumulators per MAC launch (the table's capacity)
constexpr int EM_BABY = 16;    // baby steps per MAC launch
constexpr int EM_GROUP = 8;    // query ciphertexts whose rotations are held at once
constexpr int EM_CHUNK = 256;  // model ciphertexts encrypted per batch
constexpr u64 MODEL_STREAM = 0x800000ull;

unsigned nblk(size_t n) { return (unsigned)((n + TPB - 1) / TPB); }

uint32_t clog2u(uint32_t x) {
    uint32_t r = 0;
    while ((1u << r) < x) r++;
    return r;
}

// the mask a at NTT position pos of prime r for a ciphertext's stream
__device__ __forceinline__ u64 seeded_mask(u64 seed, u64 stream, int r, uint32_t pos, int logN, const PrimeDev &P) {
    const u64 j = bit_reverse(pos, logN);
    const u64 idx = 2 * (((u64)r << logN) + j);
    const u64 hi = rng_word(seed, stream, idx), lo = rng_word(seed, stream, idx + 1);
    return add_mod(mul_shoup(barrett_wide(0, hi, P), P.r64, P.r64_sh, P.q), barrett_wide(0, lo, P), P.q);
}

// te[i][r][j] = t * e_i[j] mod q_r, e_i centred binomial (eta 21) from stream stream0 + 2 i + 1
__global__ void k_model_noise(u64 *te, int n, int ell, u64 seed, u64 stream0, int logN, const PrimeDev *pr) {
    const size_t per = (size_t)ell << logN;
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)n * per) return;
    const size_t i = e / per, rem = e - i * per;
    const int r = (int)(rem >> logN);
    const u64 j = rem & ((1ull << logN) - 1);
    const u64 w = rng_word(seed, stream0 + 2 * i + 1, j);
    const i64 v = (i64)__popcll(w & 0x1FFFFFull) - (i64)__popcll((w >> 21) & 0x1FFFFFull);
    const PrimeDev P = pr[r];
    te[e] = mul_shoup(from_signed(v, P.q), P.t_mod, P.t_mod_sh, P.q);
}

// c0 = m + t e - a s for n ciphertexts at level ell (all NTT domain), masks regenerated
__global__ void k_sk_c0(const u64 *mt, const u64 *te, const u64 *s_hat, u64 *c0, int n, int ell, u64 seed,
                        u64 stream0, int logN, const PrimeDev *pr) {
    const size_t per = (size_t)ell << logN;
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)n * per) return;
    const size_t i = e / per, rem = e - i * per;
    const int r = (int)(rem >> logN);
    const uint32_t k = (uint32_t)(rem & ((1ull << logN) - 1));
    const PrimeDev P = pr[r];
    const u64 a = seeded_mask(seed, stream0 + 2 * i, r, k, logN, P);
    const u64 as = mul_mod(a, s_hat[((size_t)r << logN) + k], P);
    c0[e] = sub_mod(add_mod(mt[e], te[e], P.q), as, P.q);
}

// full ciphertext [2][ell][N] from a stored c0 and its stream
__global__ void k_materialize(const u64 *c0, u64 *out, int ell, u64 seed, u64 stream, int logN, const PrimeDev *pr) {
    const size_t per = (size_t)ell << logN;
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= per) return;
    const int r = (int)(e >> logN);
    out[e] = c0[e];
    out[per + e] = seeded_mask(seed, stream, r, (uint32_t)(e & ((1ull << logN) - 1)), logN, pr[r]);
}

// Ciphertext x ciphertext products summed per accumulator, before relinearisation:
// for each element (r, k), every accumulator x and query ciphertext b of the
// thread's tile and every baby step j of the launch,
//   (acc0, acc1, acc2)[b][x] += (d0 R0, d0 R1 + d1 R0, d1 R1),
// d = the encrypted diagonal of (x, j) (c0 read, c1 regenerated once for all
// query ciphertexts), R = rot(v_b, j) (read once for all accumulators).
struct EncMacTable {
    const u64 *c0[EM_ACC * EM_BABY];  // [acc][baby], null = no such diagonal
    u64 stream[EM_ACC * EM_BABY];
};

// 128-bit accumulator: the products of one launch (each < 4 q^2 < 2^122, at most
// EM_BABY of them per accumulator, < 2^126) are summed exactly and reduced once.
// R: rotations [query ct][baby][2][ell][N] from the launch's first baby (r_ct words per
// query ciphertext); acc: [query ct][acc][3][ell][N] from the launch's first accumulator
// (a_ct words per query ciphertext).  A thread holds a register tile of TA
// accumulators x TQ query ciphertexts for one element; blockIdx.y = group of TQ
// query ciphertexts, blockIdx.z = group of TA accumulators.  The next baby step's
// rotations and diagonal words are loaded while the current one is multiplied.
template <int TA, int TQ>
__global__ void __launch_bounds__(128) k_enc_mac(const EncMacTable tab, int na, int nb, int nq, const u64 *R,
                                                 size_t r_ct, u64 *acc, size_t a_ct, int ell, int logN, u64 seed,
                                                 const PrimeDev *pr) {
    const size_t n_el = (size_t)ell << logN;
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_el) return;
    const int q0 = (int)blockIdx.y * TQ, nc = min(TQ, nq - q0);
    const int x0 = (int)blockIdx.z * TA, nx = min(TA, na - x0);
    const int r = (int)(e >> logN);
    const uint32_t k = (uint32_t)(e & ((1ull << logN) - 1));
    const PrimeDev P = pr[r];
    // Karatsuba: P0 = sum d0 R0, P2 = sum d1 R1, S = sum (d0 + d1)(R0 + R1), and the
    // middle component is S - P0 - P2 (sums < 2q, products < 2^122, at most EM_BABY terms)
    Acc128 a[TQ][TA][3];
#pragma unroll
    for (int b = 0; b < TQ; b++)
#pragma unroll
        for (int x = 0; x < TA; x++)
#pragma unroll
            for (int c = 0; c < 3; c++) a[b][x][c] = Acc128{0, 0};
    u64 R0[TQ], R1[TQ], D0[TA];
    auto load = [&](int j, u64 *r0, u64 *r1, u64 *d0) {
#pragma unroll
        for (int b = 0; b < TQ; b++) {
            const u64 *Rb = R + (size_t)(q0 + b) * r_ct + (size_t)j * 2 * n_el;
            r0[b] = b < nc ? Rb[e] : 0;
            r1[b] = b < nc ? Rb[n_el + e] : 0;
        }
#pragma unroll
        for (int x = 0; x < TA; x++) {
            const u64 *p = x < nx ? tab.c0[(x0 + x) * nb + j] : nullptr;
            d0[x] = p ? p[e] : 0;
        }
    };
    load(0, R0, R1, D0);
    for (int j = 0; j < nb; j++) {
        u64 N0[TQ], N1[TQ], ND[TA];
        if (j + 1 < nb) load(j + 1, N0, N1, ND);
        u64 RS[TQ];
#pragma unroll
        for (int b = 0; b < TQ; b++) RS[b] = R0[b] + R1[b];
#pragma unroll
        for (int x = 0; x < TA; x++) {
            if (x >= nx || !tab.c0[(x0 + x) * nb + j]) continue;
            const u64 d0 = D0[x];
            const u64 d1 = seeded_mask(seed, tab.stream[(x0 + x) * nb + j], r, k, logN, P);
            const u64 ds = d0 + d1;
#pragma unroll
            for (int b = 0; b < TQ; b++) {
                mac128(a[b][x][0], d0, R0[b]);
                mac128(a[b][x][1], ds, RS[b]);
                mac128(a[b][x][2], d1, R1[b]);
            }
        }
        if (j + 1 < nb) {
#pragma unroll
            for (int b = 0; b < TQ; b++) {
                R0[b] = N0[b];
                R1[b] = N1[b];
            }
#pragma unroll
            for (int x = 0; x < TA; x++) D0[x] = ND[x];
        }
    }
#pragma unroll
    for (int b = 0; b < TQ; b++)
#pragma unroll
        for (int x = 0; x < TA; x++)
            if (b < nc && x < nx) {
                u64 *o = acc + (size_t)(q0 + b) * a_ct + (size_t)(x0 + x) * 3 * n_el + e;
                const u64 p0 = reduce128(a[b][x][0], P), p2 = reduce128(a[b][x][2], P);
                const u64 mid = sub_mod(sub_mod(reduce128(a[b][x][1], P), p0, P.q), p2, P.q);
                o[0] = add_mod(o[0], p0, P.q);
                o[n_el] = add_mod(o[n_el], mid, P.q);
                o[2 * n_el] = add_mod(o[2 * n_el], p2, P.q);
            }
}

// register tile by the number of query ciphertexts multiplied together
template <int TA, int TQ>
void launch_mac(const EncMacTable &tab, int na, int nb, int nq, const u64 *R, size_t r_ct, u64 *acc, size_t a_ct,
                int ell, int logN, u64 seed, const PrimeDev *pr, cudaStream_t s) {
    const size_t n_el = (size_t)ell << logN;
    const dim3 grid((unsigned)((n_el + 127) / 128), (unsigned)((nq + TQ - 1) / TQ), (unsigned)((na + TA - 1) / TA));
    k_enc_mac<TA, TQ><<<grid, 128, 0, s>>>(tab, na, nb, nq, R, r_ct, acc, a_ct, ell, logN, seed, pr);
}

void enc_mac(const EncMacTable &tab, int na, int nb, int nq, const u64 *R, size_t r_ct, u64 *acc, size_t a_ct,
             int ell, int logN, u64 seed, const PrimeDev *pr, cudaStream_t s) {
    if (nq == 1) launch_mac<4, 1>(tab, na, nb, nq, R, r_ct, acc, a_ct, ell, logN, seed, pr, s);
    else if (nq == 2) launch_mac<2, 2>(tab, na, nb, nq, R, r_ct, acc, a_ct, ell, logN, seed, pr, s);
    else launch_mac<1, 4>(tab, na, nb, nq, R, r_ct, acc, a_ct, ell, logN, seed, pr, s);
}

}  // namespace

EncModel::~EncModel() {
    if (store) cudaFree(store);
}

copse_status enc_model_build(copse_ctx *c, const copse_keys *keys, const CompiledForest &f, u64 seed, EncModel &E,
                             cudaStream_t s) {
    const int N = c->N, L = c->L, B = (int)f.block;
    E.ctx_serial = c->serial;
    E.seed = seed;
    E.g_r = f.g_reshuffle;
    E.g_l = f.g_level;
    E.p = (int)f.precision;
    E.q = (int)f.q;
    E.b = (int)f.b;
    E.d = (int)f.d;
    E.lvl_D = L - 1 - (int)clog2u(f.precision);
    E.lvl_B = E.lvl_D - 1;
    E.grpR = f.group_reshuffle();
    E.grpL = f.group_level();
    const int n_ct = E.p + E.q + E.d * E.b + E.d;
    E.level.assign(n_ct, 0);
    E.off.assign(n_ct, 0);
    size_t words = 0;
    for (int i = 0; i < n_ct; i++) {
        E.level[i] = i < E.p ? L : (i < E.p + E.q ? E.lvl_D : E.lvl_B);
        E.off[i] = words;
        words += (size_t)E.level[i] * N;
    }
    CUDA_TRY(cudaMalloc(&E.store, std::max<size_t>(words, 1) * sizeof(u64)));
    const u64 t = c->t;
    // runs of consecutive indices at one level, encoded and encrypted in batches
    auto run = [&](int idx0, int n, const std::function<void(int, uint32_t *)> &fill) -> copse_status {
        const int ell = E.level[idx0];
        std::vector<uint32_t> pat;
        for (int i0 = 0; i0 < n; i0 += EM_CHUNK) {
            const int nc = std::min(EM_CHUNK, n - i0);
            pat.assign((size_t)nc * B, 0u);
            for (int i = 0; i < nc; i++) fill(i0 + i, pat.data() + (size_t)i * B);
            Scratch sc(s);
            u64 *mt = nullptr, *te = nullptr;
            STATUS_TRY(sc.get(c, &mt, (size_t)nc * ell * N));
            STATUS_TRY(sc.get(c, &te, (size_t)nc * ell * N));
            STATUS_TRY(encode_patterns(c, pat, nc, B, B, ell, 0, mt, s));
            const u64 stream0 = MODEL_STREAM + 2ull * (u64)(idx0 + i0);
            k_model_noise<<<nblk((size_t)nc * ell * N), TPB, 0, s>>>(te, nc, ell, seed, stream0, c->logN, c->d_prime);
            LAUNCH_CHECK();
            STATUS_TRY(ntt_forward(c, NttBatch{te, (size_t)ell * N, nc, 0, ell, ell, -1}, s));
            k_sk_c0<<<nblk((size_t)nc * ell * N), TPB, 0, s>>>(mt, te, keys->s_hat, E.store + E.off[idx0 + i0], nc, ell,
                                                               seed, stream0, c->logN, c->d_prime);
            LAUNCH_CHECK();
        }
        return COPSE_OK;
    };
    // threshold planes (Section 4.2.1), periodic over the decision slots of every block
    STATUS_TRY(run(E.idx_thr(0), E.p, [&](int i, uint32_t *pat) {
        for (uint32_t x = 0; x < f.pd(); x++) pat[x] = (f.thr_slot[x % f.q] >> i) & 1u;
    }));
    // reshuffle diagonals, shifted by their giant step
    std::vector<uint8_t> dg8;
    STATUS_TRY(run(E.idx_R(0), E.q, [&](int i, uint32_t *pat) {
        const uint32_t giant = E.g_r ? (uint32_t)i - (uint32_t)i % E.g_r : 0;
        f.reshuffle_diagonal((uint32_t)i, dg8);
        for (uint32_t x = 0; x < f.m1(); x++) pat[giant + x] = dg8[x];
    }));
    // signed level diagonals (mask folded in), shifted by their giant step
    std::vector<uint64_t> dg64;
    for (int k = 1; k <= E.d; k++)
        STATUS_TRY(run(E.idx_lvl(k, 0), E.b, [&](int i, uint32_t *pat) {
            const uint32_t giant = E.g_l ? (uint32_t)i - (uint32_t)i % E.g_l : 0;
            f.level_diagonal((uint32_t)k, (uint32_t)i, t, dg64);
            for (uint32_t x = 0; x < f.L; x++) pat[giant + x] = (uint32_t)dg64[x];
        }));
    // level masks
    STATUS_TRY(run(E.idx_mask(1), E.d, [&](int k0, uint32_t *pat) {
        for (uint32_t x = 0; x < f.L; x++) pat[x] = f.mask[(size_t)k0 * f.L + x];
    }));
    CUDA_TRY(cudaStreamSynchronize(s));
    return COPSE_OK;
}

copse_status enc_materialize(copse_ctx *c, const EncModel &E, int idx, DCt *out, cudaStream_t s) {
    if (idx < 0 || idx >= (int)E.level.size()) { set_error("model ciphertext index out of range"); return COPSE_EINVAL; }
    const int ell = E.level[idx];
    STATUS_TRY(ct_alloc(c, out, ell, 2, s));
    k_materialize<<<nblk((size_t)ell * c->N), TPB, 0, s>>>(E.c0(idx), out->data, ell, E.seed,
                                                           MODEL_STREAM + 2ull * (u64)idx, c->logN, c->d_prime);
    LAUNCH_CHECK();
    return COPSE_OK;
}

copse_status enc_matmul(copse_ctx *c, const copse_evk *evk, const EncModel &E, const std::vector<DCt> &v, int kind,
                        std::vector<std::vector<DCt>> &out, cudaStream_t s) {
    const BsgsGroup &G = kind == 0 ? E.grpR : E.grpL;
    const int N = c->N, nv = (int)v.size();
    if (nv == 0) return COPSE_OK;
    const int ell = v[0].level;
    for (const DCt &x : v)
        if (x.level != (kind == 0 ? E.lvl_D : E.lvl_B)) { set_error("internal: vector at an unexpected level"); return COPSE_EINVAL; }
    const int nb = (int)G.baby.size(), nacc = (int)G.acc.size(), n_mat = (int)G.n_mat;
    const size_t n_el = (size_t)ell * N, per = 2 * n_el, per3 = 3 * n_el;
    out.assign(nv, std::vector<DCt>(n_mat));
    // encrypted masks of the level products
    std::vector<DCt> masks;
    copse_status st = COPSE_OK;
    if (kind == 1) {
        masks.assign(E.d, DCt());
        for (int k = 1; k <= E.d && st == COPSE_OK; k++) st = enc_materialize(c, E, E.idx_mask(k), &masks[k - 1], s);
    }
    for (int g0 = 0; g0 < nv && st == COPSE_OK; g0 += EM_GROUP) {
        const int ng = std::min(EM_GROUP, nv - g0);
        Scratch sc(s);
        // baby steps: rotations of every query ciphertext of the group (one ModUp each)
        u64 *Rb = nullptr;
        if ((st = sc.get(c, &Rb, (size_t)ng * nb * per))) break;
        for (int q = 0; q < ng && st == COPSE_OK; q++) st = op_rotations(c, evk, v[g0 + q], G.baby, Rb + (size_t)q * nb * per, s);
        // matrix by matrix: products, relinearisation, giant steps (+ mask)
        for (int a = 0; a < n_mat && st == COPSE_OK; a++) {
            int x0 = 0;
            while (x0 < nacc && (int)G.acc[x0].mat != a) x0++;
            int x1 = x0;
            while (x1 < nacc && (int)G.acc[x1].mat == a) x1++;
            const int nm = x1 - x0;
            Scratch sm(s);
            u64 *acc3 = nullptr, *inner = nullptr;
            if ((st = sm.get(c, &acc3, (size_t)ng * nm * per3))) break;
            if ((st = sm.get(c, &inner, (size_t)ng * nm * per))) break;
            if (cudaMemsetAsync(acc3, 0, (size_t)ng * nm * per3 * sizeof(u64), s) != cudaSuccess) {
                set_error("cudaMemsetAsync failed");
                st = COPSE_ECUDA;
                break;
            }
            for (int y0 = 0; y0 < nm; y0 += EM_ACC) {
                const int na = std::min(EM_ACC, nm - y0);
                for (int j0 = 0; j0 < nb; j0 += EM_BABY) {
                    const int nbb = std::min(EM_BABY, nb - j0);
                    EncMacTable tab;
                    memset(&tab, 0, sizeof(tab));
                    int present = 0;
                    for (int y = 0; y < na; y++) {
                        const BsgsGroup::Acc &A = G.acc[x0 + y0 + y];
                        for (int j = 0; j < nbb; j++) {
                            const int i = A.diag[j0 + j];
                            if (i < 0) continue;
                            const int idx = kind == 0 ? E.idx_R(i) : E.idx_lvl((int)A.mat + 1, i);
                            tab.c0[y * nbb + j] = E.c0(idx);
                            tab.stream[y * nbb + j] = MODEL_STREAM + 2ull * (u64)idx;
                            present++;
                        }
                    }
                    if (!present) continue;
                    TIMED("enc_mac", 8.0 * (double)n_el * ((double)present + 2.0 * nbb * ng + 6.0 * na * ng), s,
                          enc_mac(tab, na, nbb, ng, Rb + (size_t)j0 * per, (size_t)nb * per, acc3 + (size_t)y0 * per3,
                                  (size_t)nm * per3, ell, c->logN, E.seed, c->d_prime, s));
                    LAUNCH_CHECK();
                }
            }
            // one relinearisation per (query ciphertext, accumulator), then the giant steps
            if ((st = relin_batch(c, evk, acc3, ng * nm, ell, inner, s))) break;
            std::vector<int> acc_mat(nm, 0);
            std::vector<uint32_t> acc_giant(nm);
            for (int y = 0; y < nm; y++) acc_giant[y] = G.acc[x0 + y].giant;
            std::vector<const u64 *> add_ct;
            if (kind == 1) add_ct.push_back(masks[a].data);
            for (int q = 0; q < ng && st == COPSE_OK; q++) {
                std::vector<DCt> o;
                st = giant_phase(c, evk, inner + (size_t)q * nm * per, ell, acc_mat, acc_giant, 1, {}, add_ct, o, s);
                if (st == COPSE_OK) out[g0 + q][a] = o[0];
            }
        }
    }
    for (DCt &m : masks)
        if (m.data) ct_free(&m, s);
    return st;
}
