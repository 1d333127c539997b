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
#include <atomic>
#include <cstring>
#include <functional>

#include "internal.cuh"

namespace {

constexpr int TPB = 256;
constexpr int EM_GROUP = 8;    // query ciphertexts per rotation group while no free-memory sizing is known
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
// for each element, every accumulator x, query ciphertext b and baby step j,
//   (acc0, acc1, acc2)[b][x] += (d0 R0, d0 R1 + d1 R0, d1 R1)
// with d the encrypted diagonal of (x, j) (c0 read, c1 regenerated) and R = rot(v_b, j),
// by Karatsuba: P0 = sum d0 R0, P2 = sum d1 R1, S = sum (d0 + d1)(R0 + R1), middle S - P0 - P2.
// One CTA per tile of 32 elements (one per lane) and
// TA accumulators, its W warps covering W * TQ query ciphertexts.  The CTA regenerates the
// masks of its accumulators' diagonals once (shared memory) for every query ciphertext it
// covers; the rotations stream through a STAGES-deep cp.async pipeline of shared-memory
// tiles (32 elements x 2 components per query ciphertext and baby step); each thread
// keeps TA x TQ Karatsuba triples as exact split-28 partial sums (Acc3w) in registers.
// Baby steps are taken in runs of RUN (the partial sums' exact capacity); after each run
// the sums are reduced and added to the accumulators in memory.  CTAs with the same
// element tile and different accumulators are adjacent in the grid, so a tile of
// rotations read from HBM is reused from L2 by the others.
constexpr int MAC_TA = 2;
constexpr int MAC_TQ = 4;
constexpr int MAC_RUN = 64;
constexpr int MAC_STAGES = 4;

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <int W>
constexpr size_t mac_smem() {
    return (size_t)(2 * MAC_TA * MAC_RUN * 32 + MAC_STAGES * W * MAC_TQ * 2 * 32) * sizeof(u64);
}

// tab: [nm][nb] diagonal entries of this launch's accumulators; R: [query ct][nb][2][ell][N]
// (r_ct words per query ciphertext); acc: [query ct][nm][3][ell][N] (a_ct words per query
// ciphertext), added to.
template <int W>
__global__ void __launch_bounds__(W * 32, 1)
    k_enc_mac(const EncModel::MacEntry *__restrict__ tab, int nm, int nb, int nq, const u64 *__restrict__ R,
               size_t r_ct, u64 *__restrict__ acc, size_t a_ct, int ell, int logN, u64 seed,
               const PrimeDev *__restrict__ pr, int n_ag) {
    constexpr int NT = W * 32, CQ = W * MAC_TQ, STAGE = CQ * 2 * 32;
    extern __shared__ __align__(16) u64 sm2[];
    u64 *d0s = sm2, *d1s = sm2 + MAC_TA * MAC_RUN * 32, *rb = sm2 + 2 * MAC_TA * MAC_RUN * 32;
    const size_t n_el = (size_t)ell << logN;
    const uint32_t nmask = (1u << logN) - 1;
    const int ag = (int)(blockIdx.x % (unsigned)n_ag);
    const size_t e0 = (size_t)(blockIdx.x / (unsigned)n_ag) * 32;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int q0 = (int)blockIdx.y * CQ;
    const int x0 = ag * MAC_TA, nx = min(MAC_TA, nm - x0);
    const size_t e = e0 + lane;
    const bool valid = e < n_el, full = e0 + 32 <= n_el;
    const PrimeDev P = pr[valid ? (int)(e >> logN) : 0];

    // rotation tile of baby step j into stage buffer `st`: rows (query ct, component) of 32 words
    auto issue = [&](int j, int st) {
        u64 *dst = rb + (size_t)st * STAGE;
        for (int c = threadIdx.x; c < CQ * 2 * 16; c += NT) {
            const int row = c >> 4, part = c & 15, ct = q0 + (row >> 1), comp = row & 1;
            u64 *d = dst + row * 32 + part * 2;
            const u64 *src = R + (size_t)ct * r_ct + ((size_t)j * 2 + comp) * n_el + e0 + part * 2;
            if (ct < nq && full) {
                cp_async16(d, src);
            } else {
                d[0] = (ct < nq && e0 + part * 2 < n_el) ? src[0] : 0;
                d[1] = (ct < nq && e0 + part * 2 + 1 < n_el) ? src[1] : 0;
            }
        }
        cp_async_commit();
    };

    Acc3w a[MAC_TA][MAC_TQ][3];
    for (int jr = 0; jr < nb; jr += MAC_RUN) {
        const int nr = min(MAC_RUN, nb - jr);
#pragma unroll
        for (int x = 0; x < MAC_TA; x++)
#pragma unroll
            for (int c = 0; c < MAC_TQ; c++)
#pragma unroll
                for (int k = 0; k < 3; k++) a[x][c][k] = Acc3w{0, 0, 0};
        for (int st = 0; st < MAC_STAGES - 1; st++) {
            if (st < nr) issue(jr + st, st);
            else cp_async_commit();
        }
        // the run's diagonal words and regenerated masks for the CTA's accumulators
        for (int i = threadIdx.x; i < MAC_TA * nr * 32; i += NT) {
            const int x = i / (nr * 32), rem = i - x * nr * 32, j = rem >> 5, l = rem & 31;
            const size_t ee = e0 + l;
            u64 v0 = 0, v1 = 0;
            if (x < nx && ee < n_el) {
                const EncModel::MacEntry te = tab[(size_t)(x0 + x) * nb + jr + j];
                if (te.c0) {
                    const int rr = (int)(ee >> logN);
                    v0 = te.c0[ee];
                    v1 = seeded_mask(seed, te.stream, rr, (uint32_t)(ee & nmask), logN, pr[rr]);
                }
            }
            d0s[(x * MAC_RUN + j) * 32 + l] = v0;
            d1s[(x * MAC_RUN + j) * 32 + l] = v1;
        }
        for (int j = 0; j < nr; j++) {
            cp_async_wait<MAC_STAGES - 2>();
            __syncthreads();  // stage j (and the masks) visible; stage j-1 no longer read
            if (j + MAC_STAGES - 1 < nr) issue(jr + j + MAC_STAGES - 1, (j + MAC_STAGES - 1) % MAC_STAGES);
            else cp_async_commit();
            const u64 *st = rb + (size_t)(j % MAC_STAGES) * STAGE + (size_t)w * MAC_TQ * 64 + lane;
            Sp28 r0[MAC_TQ], r1[MAC_TQ], rs[MAC_TQ];
#pragma unroll
            for (int c = 0; c < MAC_TQ; c++) {
                const u64 v0 = st[c * 64], v1 = st[c * 64 + 32];
                r0[c] = split28(v0);
                r1[c] = split28(v1);
                rs[c] = split28(v0 + v1);
            }
#pragma unroll
            for (int x = 0; x < MAC_TA; x++) {
                const u64 d0 = d0s[(x * MAC_RUN + j) * 32 + lane], d1 = d1s[(x * MAC_RUN + j) * 32 + lane];
                const Sp28 s0 = split28(d0), s1 = split28(d1), ss = split28(d0 + d1);
#pragma unroll
                for (int c = 0; c < MAC_TQ; c++) {
                    mac_sp(a[x][c][0], s0, r0[c]);
                    mac_sp(a[x][c][1], ss, rs[c]);
                    mac_sp(a[x][c][2], s1, r1[c]);
                }
            }
        }
        cp_async_wait<0>();
        __syncthreads();  // every read of this run's buffers is done before the next run refills them
#pragma unroll
        for (int x = 0; x < MAC_TA; x++)
#pragma unroll
            for (int c = 0; c < MAC_TQ; c++) {
                const int ct = q0 + w * MAC_TQ + c;
                if (!valid || x >= nx || ct >= nq) continue;
                u64 *o = acc + (size_t)ct * a_ct + (size_t)(x0 + x) * 3 * n_el + e;
                const u64 p0 = reduce128(acc3w_value(a[x][c][0]), P);
                const u64 sv = reduce128(acc3w_value(a[x][c][1]), P);
                const u64 p2 = reduce128(acc3w_value(a[x][c][2]), P);
                o[0] = add_mod(o[0], p0, P.q);
                o[n_el] = add_mod(o[n_el], sub_mod(sub_mod(sv, p0, P.q), p2, P.q), P.q);
                o[2 * n_el] = add_mod(o[2 * n_el], p2, P.q);
            }
    }
}

// per-device raise of the dynamic shared-memory limit of each instantiation
template <int W>
copse_status mac_attr(int device) {
    static std::atomic<uint64_t> done{0};
    if (device >= 0 && device < 64 && (done.load(std::memory_order_acquire) & (1ull << device))) return COPSE_OK;
    CUDA_TRY(cudaFuncSetAttribute(k_enc_mac<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mac_smem<W>()));
    if (device >= 0 && device < 64) done.fetch_or(1ull << device, std::memory_order_release);
    return COPSE_OK;
}

template <int W>
copse_status launch_mac(int device, const EncModel::MacEntry *tab, int nm, int nb, int nq, const u64 *R, size_t r_ct,
                         u64 *acc, size_t a_ct, int ell, int logN, u64 seed, const PrimeDev *pr, cudaStream_t s) {
    STATUS_TRY(mac_attr<W>(device));
    const size_t n_el = (size_t)ell << logN;
    const int n_ag = (nm + MAC_TA - 1) / MAC_TA;
    const size_t tiles = (n_el + 31) / 32;
    const dim3 grid((unsigned)(tiles * n_ag), (unsigned)((nq + W * MAC_TQ - 1) / (W * MAC_TQ)));
    k_enc_mac<W><<<grid, W * 32, mac_smem<W>(), s>>>(tab, nm, nb, nq, R, r_ct, acc, a_ct, ell, logN, seed, pr, n_ag);
    LAUNCH_CHECK();
    return COPSE_OK;
}

copse_status enc_mac(int device, const EncModel::MacEntry *tab, int nm, int nb, int nq, const u64 *R, size_t r_ct,
                      u64 *acc, size_t a_ct, int ell, int logN, u64 seed, const PrimeDev *pr, cudaStream_t s) {
    if (nq > 4 * MAC_TQ) return launch_mac<8>(device, tab, nm, nb, nq, R, r_ct, acc, a_ct, ell, logN, seed, pr, s);
    if (nq > 2 * MAC_TQ) return launch_mac<4>(device, tab, nm, nb, nq, R, r_ct, acc, a_ct, ell, logN, seed, pr, s);
    if (nq > MAC_TQ) return launch_mac<2>(device, tab, nm, nb, nq, R, r_ct, acc, a_ct, ell, logN, seed, pr, s);
    return launch_mac<1>(device, tab, nm, nb, nq, R, r_ct, acc, a_ct, ell, logN, seed, pr, s);
}

}  // namespace

EncModel::~EncModel() {
    if (store) cudaFree(store);
    for (MacEntry *t : d_tab)
        if (t) cudaFree(t);
}

copse_status enc_model_build(copse_ctx *c, const copse_keys *keys, const CompiledForest &f, u64 seed, EncModel &E,
                             cudaStream_t s) {
    const int N = c->N, L = c->L, B = (int)f.block, SP = (int)f.span(), NS = (int)f.n_seg;
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
            pat.assign((size_t)nc * SP, 0u);
            for (int i = 0; i < nc; i++) fill(i0 + i, pat.data() + (size_t)i * SP);
            Scratch sc(s);
            u64 *mt = nullptr, *te = nullptr;
            STATUS_TRY(sc.get(c, &mt, (size_t)nc * ell * N));
            STATUS_TRY(sc.get(c, &te, (size_t)nc * ell * N));
            STATUS_TRY(encode_patterns(c, pat, nc, SP, SP, ell, 0, mt, s));
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
    // threshold planes (Section 4.2.1), periodic over the decision slots of every block; each
    // slot pattern covers the n_seg blocks of one query (block s: segment s)
    STATUS_TRY(run(E.idx_thr(0), E.p, [&](int i, uint32_t *pat) {
        for (int sg = 0; sg < NS; sg++)
            for (uint32_t x = 0; x < f.pd(); x++) pat[(size_t)sg * B + x] = f.thr_bit((uint32_t)sg, x, (uint32_t)i);
    }));
    // reshuffle diagonals, shifted by their giant step
    std::vector<uint8_t> dg8;
    STATUS_TRY(run(E.idx_R(0), E.q, [&](int i, uint32_t *pat) {
        const uint32_t giant = E.g_r ? (uint32_t)i - (uint32_t)i % E.g_r : 0;
        for (int sg = 0; sg < NS; sg++) {
            f.reshuffle_diagonal((uint32_t)i, dg8, (uint32_t)sg);
            for (uint32_t x = 0; x < f.m1(); x++) pat[(size_t)sg * B + giant + x] = dg8[x];
        }
    }));
    // signed level diagonals (mask folded in), shifted by their giant step
    std::vector<uint64_t> dg64;
    for (int k = 1; k <= E.d; k++)
        STATUS_TRY(run(E.idx_lvl(k, 0), E.b, [&](int i, uint32_t *pat) {
            const uint32_t giant = E.g_l ? (uint32_t)i - (uint32_t)i % E.g_l : 0;
            for (int sg = 0; sg < NS; sg++) {
                f.level_diagonal((uint32_t)k, (uint32_t)i, t, dg64, (uint32_t)sg);
                for (uint32_t x = 0; x < f.L; x++) pat[(size_t)sg * B + giant + x] = (uint32_t)dg64[x];
            }
        }));
    // level masks
    STATUS_TRY(run(E.idx_mask(1), E.d, [&](int k0, uint32_t *pat) {
        for (int sg = 0; sg < NS; sg++)
            for (uint32_t x = 0; x < f.L; x++) pat[(size_t)sg * B + x] = f.mask_at((uint32_t)k0 + 1, x, (uint32_t)sg);
    }));
    // the MAC kernels' shared-memory limit, raised here so that no attribute call falls inside
    // a graph recording
    STATUS_TRY(mac_attr<1>(c->device));
    STATUS_TRY(mac_attr<2>(c->device));
    STATUS_TRY(mac_attr<4>(c->device));
    STATUS_TRY(mac_attr<8>(c->device));
    // diagonal tables of the two products, [accumulator][baby step] in plan order
    for (int kind = 0; kind < 2; kind++) {
        const BsgsGroup &G = kind == 0 ? E.grpR : E.grpL;
        const size_t nb = G.baby.size();
        std::vector<EncModel::MacEntry> h(G.acc.size() * nb, EncModel::MacEntry{nullptr, 0});
        for (size_t x = 0; x < G.acc.size(); x++)
            for (size_t j = 0; j < nb; j++) {
                const int i = G.acc[x].diag[j];
                if (i < 0) continue;
                const int idx = kind == 0 ? E.idx_R(i) : E.idx_lvl((int)G.acc[x].mat + 1, i);
                h[x * nb + j] = EncModel::MacEntry{E.c0(idx), MODEL_STREAM + 2ull * (u64)idx};
            }
        CUDA_TRY(cudaMalloc(&E.d_tab[kind], std::max<size_t>(h.size(), 1) * sizeof(EncModel::MacEntry)));
        CUDA_TRY(cudaMemcpy(E.d_tab[kind], h.data(), h.size() * sizeof(EncModel::MacEntry), cudaMemcpyHostToDevice));
    }
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
    // query ciphertexts whose rotations are held at once: up to 32 (the MAC kernel's CTA covers
    // 32), bounded by the device memory the group's buffers take
    int group = 32;
    if (c->capturing) {
        // memory queries are not allowed while a graph is recorded: the last sizing
        group = E.group_hint[kind] > 0 ? E.group_hint[kind] : EM_GROUP;
    } else {
        size_t free_b = 0, total_b = 0;
        CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
        size_t pool_idle = 0;
        if (c->pool) {
            uint64_t res = 0, used = 0;
            cudaMemPoolGetAttribute(c->pool, cudaMemPoolAttrReservedMemCurrent, &res);
            cudaMemPoolGetAttribute(c->pool, cudaMemPoolAttrUsedMemCurrent, &used);
            pool_idle = res > used ? (size_t)(res - used) : 0;
        }
        size_t max_acc = 1;
        for (int a = 0; a < n_mat; a++) {
            size_t n = 0;
            for (const BsgsGroup::Acc &A : G.acc) n += (int)A.mat == a;
            max_acc = std::max(max_acc, n);
        }
        const size_t per_ct = ((size_t)nb * per + max_acc * (per3 + per)) * sizeof(u64);
        const size_t budget = (free_b + pool_idle) / 10 * 7;
        while (group > 1 && (size_t)group * per_ct > budget) group /= 2;
        E.group_hint[kind] = group;
    }
    for (int g0 = 0; g0 < nv && st == COPSE_OK; g0 += group) {
        const int ng = std::min(group, nv - g0);
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
            {
                // every accumulator and baby step of the matrix in one launch
                size_t present = 0;
                for (int y = 0; y < nm; y++)
                    for (int j = 0; j < nb; j++) present += G.acc[x0 + y].diag[j] >= 0;
                const double bytes = 8.0 * (double)n_el * ((double)present + 2.0 * nb * ng + 3.0 * nm * ng);
                TIMED_OPS("enc_mac", bytes, 4.0 * (double)present * ng * n_el, s,
                          st = enc_mac(c->device, E.d_tab[kind] + (size_t)x0 * nb, nm, nb, ng, Rb, (size_t)nb * per,
                                        acc3, (size_t)nm * per3, ell, c->logN, E.seed, c->d_prime, s));
                if (st) break;
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
