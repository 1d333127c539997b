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
constexpr int EM_ACC = 8;      // accumulators per MAC launch
constexpr int EM_BABY = 16;    // baby steps per MAC launch
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
// for each element (r, k) and every (accumulator x, baby step j) of the launch,
//   (acc0, acc1, acc2) += (d0 R0, d0 R1 + d1 R0, d1 R1),
// d = the encrypted diagonal (c0 read, c1 regenerated), R = rot(v, j).
struct EncMacTable {
    const u64 *c0[EM_ACC * EM_BABY];  // [acc][baby], null = no such diagonal
    u64 stream[EM_ACC * EM_BABY];
    const u64 *R[EM_BABY];            // [2][ell][N]
    u64 *acc[EM_ACC];                 // [3][ell][N]
};

__global__ void __launch_bounds__(256) k_enc_mac(const EncMacTable tab, int na, int nb, int ell, int logN, u64 seed,
                                                 const PrimeDev *pr) {
    const size_t n_el = (size_t)ell << logN;
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_el) return;
    const int r = (int)(e >> logN);
    const uint32_t k = (uint32_t)(e & ((1ull << logN) - 1));
    const PrimeDev P = pr[r];
    u64 a0[EM_ACC], a1[EM_ACC], a2[EM_ACC];
    for (int x = 0; x < na; x++) {
        a0[x] = tab.acc[x][e];
        a1[x] = tab.acc[x][n_el + e];
        a2[x] = tab.acc[x][2 * n_el + e];
    }
    for (int j = 0; j < nb; j++) {
        const u64 R0 = tab.R[j][e], R1 = tab.R[j][n_el + e];
        for (int x = 0; x < na; x++) {
            const u64 *p = tab.c0[x * nb + j];
            if (!p) continue;
            const u64 d0 = p[e];
            const u64 d1 = seeded_mask(seed, tab.stream[x * nb + j], r, k, logN, P);
            a0[x] = add_mod(a0[x], mul_mod(d0, R0, P), P.q);
            a1[x] = add_mod(a1[x], add_mod(mul_mod(d0, R1, P), mul_mod(d1, R0, P), P.q), P.q);
            a2[x] = add_mod(a2[x], mul_mod(d1, R1, P), P.q);
        }
    }
    for (int x = 0; x < na; x++) {
        tab.acc[x][e] = a0[x];
        tab.acc[x][n_el + e] = a1[x];
        tab.acc[x][2 * n_el + e] = a2[x];
    }
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

copse_status enc_matmul(copse_ctx *c, const copse_evk *evk, const EncModel &E, const DCt &v, int kind,
                        std::vector<DCt> &out, cudaStream_t s) {
    const BsgsGroup &G = kind == 0 ? E.grpR : E.grpL;
    const int ell = v.level, N = c->N;
    if (ell != (kind == 0 ? E.lvl_D : E.lvl_B)) { set_error("internal: vector at an unexpected level"); return COPSE_EINVAL; }
    const int nb = (int)G.baby.size(), nacc = (int)G.acc.size();
    const size_t per = (size_t)2 * ell * N, per3 = (size_t)3 * ell * N;
    Scratch sc(s);
    // baby steps: rotations of v (one ModUp shared by all)
    u64 *Rb = nullptr, *acc3 = nullptr, *inner = nullptr;
    STATUS_TRY(sc.get(c, &Rb, (size_t)nb * per));
    STATUS_TRY(op_rotations(c, evk, v, G.baby, Rb, s));
    // per (matrix, giant step): sum_j Enc(d'_{k, j}) x rot(v, j), three components
    STATUS_TRY(sc.get(c, &acc3, (size_t)nacc * per3));
    CUDA_TRY(cudaMemsetAsync(acc3, 0, (size_t)nacc * per3 * sizeof(u64), s));
    for (int a0 = 0; a0 < nacc; a0 += EM_ACC) {
        const int na = std::min(EM_ACC, nacc - a0);
        for (int x0 = 0; x0 < nb; x0 += EM_BABY) {
            const int nbb = std::min(EM_BABY, nb - x0);
            EncMacTable tab;
            memset(&tab, 0, sizeof(tab));
            int present = 0;
            for (int x = 0; x < nbb; x++) tab.R[x] = Rb + (size_t)(x0 + x) * per;
            for (int a = 0; a < na; a++) {
                const BsgsGroup::Acc &A = G.acc[a0 + a];
                tab.acc[a] = acc3 + (size_t)(a0 + a) * per3;
                for (int x = 0; x < nbb; x++) {
                    const int i = A.diag[x0 + x];
                    if (i < 0) continue;
                    const int idx = kind == 0 ? E.idx_R(i) : E.idx_lvl((int)A.mat + 1, i);
                    tab.c0[a * nbb + x] = E.c0(idx);
                    tab.stream[a * nbb + x] = MODEL_STREAM + 2ull * (u64)idx;
                    present++;
                }
            }
            if (!present) continue;
            TIMED("enc_mac", 8.0 * N * ell * ((double)present + 2.0 * nbb + 6.0 * na), s,
                  k_enc_mac<<<nblk((size_t)ell * N), TPB, 0, s>>>(tab, na, nbb, ell, c->logN, E.seed, c->d_prime));
            LAUNCH_CHECK();
        }
    }
    // one relinearisation per accumulator, then the giant steps (+ the encrypted masks)
    STATUS_TRY(sc.get(c, &inner, (size_t)nacc * per));
    STATUS_TRY(relin_batch(c, evk, acc3, nacc, ell, inner, s));
    std::vector<DCt> masks;
    std::vector<const u64 *> add_ct;
    copse_status st = COPSE_OK;
    if (kind == 1) {
        masks.assign(E.d, DCt());
        for (int k = 1; k <= E.d && st == COPSE_OK; k++) {
            st = enc_materialize(c, E, E.idx_mask(k), &masks[k - 1], s);
            add_ct.push_back(masks[k - 1].data);
        }
    }
    std::vector<int> acc_mat(nacc);
    std::vector<uint32_t> acc_giant(nacc);
    for (int x = 0; x < nacc; x++) {
        acc_mat[x] = (int)G.acc[x].mat;
        acc_giant[x] = G.acc[x].giant;
    }
    if (st == COPSE_OK) st = giant_phase(c, evk, inner, ell, acc_mat, acc_giant, (int)G.n_mat, {}, add_ct, out, s);
    for (DCt &m : masks)
        if (m.data) ct_free(&m, s);
    return st;
}
