// Encrypted models: the model owner also owns the data (Maurice = Diane,
// Section 8.3 of the paper), encrypts the threshold planes, every diagonal of
// the reshuffle and level matrices (zero ones included: p + q + d(b+1)
// ciphertexts, Table 1d) and the level masks, and the server evaluates
// Algorithm 1 with ciphertext x ciphertext products.
//
// Layout: each model ciphertext is a secret-key encryption whose mask c1 = a
// is drawn from the counter generator in evaluation form (seeded_mask), so only
// c0 is kept in HBM and c1 is regenerated where it is consumed (half the bytes of
// a full ciphertext); c0 = m + t e - a s.  The threshold planes and the level
// masks are stored one after another ([ell][N] each); the diagonals are stored
// element-major per matrix of the baby-step / giant-step plan ([ell N][accumulator]
// [baby step]), the layout of the tensor-core multiply-accumulate (encmac.cu).
#include <algorithm>
#include <atomic>
#include <cstring>
#include <functional>

#include "internal.cuh"

namespace {

constexpr int TPB = 256;
constexpr int EM_GROUP = 8;    // query ciphertexts per rotation group while no free-memory sizing is known
constexpr int EM_CHUNK = 256;  // model ciphertexts encrypted per batch
constexpr int EM_GROUP_MAX = 64;  // query ciphertexts per rotation group at most

unsigned nblk(size_t n) { return (unsigned)((n + TPB - 1) / TPB); }

uint32_t clog2u(uint32_t x) {
    uint32_t r = 0;
    while ((1u << r) < x) r++;
    return r;
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

}  // namespace

EncModel::~EncModel() {
    if (store) cudaFree(store);
    for (auto &mats : mac)
        for (MacMat &M : mats) {
            if (M.c0) cudaFree(M.c0);
            if (M.idx) cudaFree(M.idx);
        }
}

copse_status enc_mac_tc_attr(int device);

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
    E.at.assign(n_ct, EncModel::DiagAt{});
    for (int i = 0; i < n_ct; i++) E.level[i] = i < E.p ? L : (i < E.p + E.q ? E.lvl_D : E.lvl_B);
    // the diagonals' blocks: one per matrix of each plan, [ell N][nm][nb]
    for (int kind = 0; kind < 2; kind++) {
        const BsgsGroup &G = kind == 0 ? E.grpR : E.grpL;
        const int nb = (int)G.baby.size(), ell = kind == 0 ? E.lvl_D : E.lvl_B;
        E.mac[kind].assign(G.n_mat, EncModel::MacMat{});
        for (int x = 0; x < (int)G.acc.size(); x++) {
            EncModel::MacMat &M = E.mac[kind][G.acc[x].mat];
            if (M.nm == 0) M.x0 = x;
            M.nm++;
        }
        for (int a = 0; a < (int)G.n_mat; a++) {
            EncModel::MacMat &M = E.mac[kind][a];
            M.nb = nb;
            M.ell = ell;
            if (M.nm == 0 || nb == 0) continue;
            std::vector<uint32_t> idx((size_t)M.nm * nb, ~0u);
            for (int y = 0; y < M.nm; y++)
                for (int j = 0; j < nb; j++) {
                    const int i = G.acc[M.x0 + y].diag[j];
                    if (i < 0) continue;
                    const int id = kind == 0 ? E.idx_R(i) : E.idx_lvl(a + 1, i);
                    idx[(size_t)y * nb + j] = (uint32_t)id;
                    E.at[id] = EncModel::DiagAt{kind, a, (uint32_t)(y * mac_row(nb) + j)};
                }
            const size_t words = ((size_t)ell * N) * M.nm * mac_row(nb);
            CUDA_TRY(cudaMalloc(&M.c0, words * sizeof(u64)));
            CUDA_TRY(cudaMemsetAsync(M.c0, 0, words * sizeof(u64), s));
            CUDA_TRY(cudaMalloc(&M.idx, idx.size() * sizeof(uint32_t)));
            CUDA_TRY(cudaMemcpy(M.idx, idx.data(), idx.size() * sizeof(uint32_t), cudaMemcpyHostToDevice));
        }
    }
    for (int i = 0; i < n_ct; i++)
        if (E.at[i].kind < 0 && i >= E.p && i < E.p + E.q + E.d * E.b) {
            set_error("internal: a diagonal outside the baby-step / giant-step plan");
            return COPSE_EINVAL;
        }
    size_t words = 0;
    for (int i = 0; i < n_ct; i++) {
        if (E.at[i].kind >= 0) continue;
        E.off[i] = words;
        words += (size_t)E.level[i] * N;
    }
    CUDA_TRY(cudaMalloc(&E.store, std::max<size_t>(words, 1) * sizeof(u64)));
    const u64 t = c->t;
    // runs of consecutive indices at one level, encoded and encrypted in batches; diagonals are
    // scattered from the batch into their matrix's block
    auto run = [&](int idx0, int n, const std::function<void(int, uint32_t *)> &fill) -> copse_status {
        const int ell = E.level[idx0];
        std::vector<uint32_t> pat, pos;
        for (int i0 = 0; i0 < n; i0 += EM_CHUNK) {
            const int nc = std::min(EM_CHUNK, n - i0);
            pat.assign((size_t)nc * SP, 0u);
            for (int i = 0; i < nc; i++) fill(i0 + i, pat.data() + (size_t)i * SP);
            Scratch sc(s);
            u64 *mt = nullptr, *te = nullptr, *c0 = nullptr;
            STATUS_TRY(sc.get(c, &mt, (size_t)nc * ell * N));
            STATUS_TRY(sc.get(c, &te, (size_t)nc * ell * N));
            STATUS_TRY(encode_patterns(c, pat, nc, SP, SP, ell, 0, mt, s));
            const u64 stream0 = MODEL_STREAM + 2ull * (u64)(idx0 + i0);
            k_model_noise<<<nblk((size_t)nc * ell * N), TPB, 0, s>>>(te, nc, ell, seed, stream0, c->logN, c->d_prime);
            LAUNCH_CHECK();
            STATUS_TRY(ntt_forward(c, NttBatch{te, (size_t)ell * N, nc, 0, ell, ell, -1}, s));
            const EncModel::DiagAt &at = E.at[idx0 + i0];
            if (at.kind < 0) {
                c0 = E.store + E.off[idx0 + i0];
            } else {
                STATUS_TRY(sc.get(c, &c0, (size_t)nc * ell * N));
            }
            k_sk_c0<<<nblk((size_t)nc * ell * N), TPB, 0, s>>>(mt, te, keys->s_hat, c0, nc, ell, seed, stream0,
                                                               c->logN, c->d_prime);
            LAUNCH_CHECK();
            if (at.kind >= 0) {
                pos.resize(nc);
                for (int i = 0; i < nc; i++) {
                    const EncModel::DiagAt &ai = E.at[idx0 + i0 + i];
                    if (ai.kind != at.kind || ai.mat != at.mat) {
                        set_error("internal: a batch of diagonals spans two matrices");
                        return COPSE_EINVAL;
                    }
                    pos[i] = ai.pos;
                }
                u64 *pw = nullptr;
                STATUS_TRY(sc.get(c, &pw, (size_t)(nc + 1) / 2));
                uint32_t *d_pos = (uint32_t *)pw;
                CUDA_TRY(cudaMemcpyAsync(d_pos, pos.data(), nc * sizeof(uint32_t), cudaMemcpyHostToDevice, s));
                STATUS_TRY(mac_scatter(c, c0, d_pos, nc, E.mac[at.kind][at.mat], s));
                CUDA_TRY(cudaStreamSynchronize(s));  // pos is reused by the next batch
            }
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
    // the multiply-accumulate kernel's shared-memory limit, raised here so that no attribute call
    // falls inside a graph recording
    STATUS_TRY(enc_mac_tc_attr(c->device));
    CUDA_TRY(cudaStreamSynchronize(s));
    return COPSE_OK;
}

copse_status enc_materialize(copse_ctx *c, const EncModel &E, int idx, DCt *out, cudaStream_t s) {
    if (idx < 0 || idx >= (int)E.level.size()) { set_error("model ciphertext index out of range"); return COPSE_EINVAL; }
    const int ell = E.level[idx];
    STATUS_TRY(ct_alloc(c, out, ell, 2, s));
    const EncModel::DiagAt &at = E.at[idx];
    Scratch sc(s);
    const u64 *c0 = nullptr;
    if (at.kind < 0) {
        c0 = E.c0(idx);
    } else {
        u64 *g = nullptr;
        STATUS_TRY(sc.get(c, &g, (size_t)ell * c->N));
        STATUS_TRY(mac_gather(c, E.mac[at.kind][at.mat], at.pos, g, s));
        c0 = g;
    }
    k_materialize<<<nblk((size_t)ell * c->N), TPB, 0, s>>>(c0, out->data, ell, E.seed, MODEL_STREAM + 2ull * (u64)idx,
                                                           c->logN, c->d_prime);
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
    const int nb64 = (nb + 63) / 64 * 64;  // the element-major rotations hold baby steps in chunks of 64
    const size_t n_el = (size_t)ell * N, per = 2 * n_el, per3 = 3 * n_el;
    out.assign(nv, std::vector<DCt>(n_mat));
    // encrypted masks of the level products
    std::vector<DCt> masks;
    copse_status st = COPSE_OK;
    if (kind == 1) {
        masks.assign(E.d, DCt());
        for (int k = 1; k <= E.d && st == COPSE_OK; k++) st = enc_materialize(c, E, E.idx_mask(k), &masks[k - 1], s);
    }
    // query ciphertexts whose rotations are held at once: up to EM_GROUP_MAX (every diagonal and
    // its regenerated mask is read once per group), bounded by the device memory the group's
    // buffers take
    int group = EM_GROUP_MAX;
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
        const size_t per_ct = ((size_t)nb64 * per + max_acc * (per3 + per)) * sizeof(u64);
        const size_t rot_tmp = (size_t)nb * per * sizeof(u64);  // one query ciphertext's rotations
        const size_t budget = (free_b + pool_idle) / 10 * 7;
        while (group > 1 && (size_t)group * per_ct + rot_tmp > budget) group /= 2;
        E.group_hint[kind] = group;
    }
    for (int g0 = 0; g0 < nv && st == COPSE_OK; g0 += group) {
        const int ng = std::min(group, nv - g0);
        Scratch sc(s);
        // baby steps: rotations of every query ciphertext of the group (one ModUp each), moved
        // into the element-major layout [ell N][nb / 64][ng][64][2] of the multiply-accumulate
        u64 *Rb = nullptr, *rot = nullptr;
        if ((st = sc.get(c, &Rb, (size_t)ng * nb64 * per))) break;
        {
            Scratch sr(s);
            if ((st = sr.get(c, &rot, (size_t)nb * per))) break;
            for (int q = 0; q < ng && st == COPSE_OK; q++) {
                st = op_rotations(c, evk, v[g0 + q], G.baby, rot, s);
                if (st == COPSE_OK) st = rot_to_elements(c, rot, nb, ng, q, ell, Rb, s);
            }
        }
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
            {
                // every accumulator and baby step of the matrix in one launch
                const EncModel::MacMat &M = E.mac[kind][a];
                if (M.nm != nm || M.x0 != x0 || M.ell != ell) {
                    set_error("internal: diagonal block does not match the plan");
                    st = COPSE_EINVAL;
                    break;
                }
                size_t present = 0;
                for (int y = 0; y < nm; y++)
                    for (int j = 0; j < nb; j++) present += G.acc[x0 + y].diag[j] >= 0;
                const double bytes = 8.0 * (double)n_el * ((double)present + 2.0 * nb * ng + 3.0 * nm * ng);
                TIMED_OPS("enc_mac", bytes, enc_mac_tc_flops(M, ng, c->logN), s,
                          st = enc_mac_tc(c, M, Rb, ng, acc3, (size_t)nm * per3, E.seed, s));
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
