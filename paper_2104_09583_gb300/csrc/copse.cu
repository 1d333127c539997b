// C-ABI entry points: models (compile, upload of the plaintext structures),
// keys, feature encryption, Algorithm 1 of the paper (Section 4.3) on the
// device, decryption, buffers and single ring operations.
#include <algorithm>
#include <cstring>
#include <functional>
#include <memory>

#include "forest.h"
#include "internal.cuh"

namespace {

uint32_t clog2u(uint32_t x) {
    uint32_t r = 0;
    while ((1u << r) < x) r++;
    return r;
}

cudaStream_t as_stream(void *s) { return (cudaStream_t)s; }

}  // namespace

// Plaintext structures of one model encoded for one context (NTT domain, device).
struct DeviceModel {
    copse_ctx *ctx = nullptr;
    uint64_t ctx_serial = 0;           // the context it was encoded for (addresses can be reused)
    int lvl_D = 0, lvl_B = 0;          // levels of Decisions and of Branches
    u64 *store = nullptr;              // one allocation for every plaintext
    // SecComp leaves, plane i: lt = x * lt_mul + lt_add, eq = x * eq_mul + eq_add (level L)
    std::vector<const u64 *> lt_mul, lt_add, eq_mul, eq_add;
    // matrix products: baby-step amounts, per accumulator (matrix, giant step) the
    // diagonal plaintexts per baby step (null = zero), extended basis
    struct Group {
        BsgsGroup plan;
        std::vector<std::vector<const u64 *>> pt;  // [acc][baby]
        std::vector<int> acc_mat;
        std::vector<uint32_t> acc_giant;
    };
    Group R, Lv;                                    // reshuffle; levels (d matrices)
    std::vector<const u64 *> mask;                  // [d]
    ~DeviceModel() {
        if (store) cudaFree(store);
    }
};

// The label shuffle's diagonal plaintexts (extended basis, at the level of the result)
struct ShuffleDev {
    uint64_t ctx_serial = 0;
    std::vector<uint32_t> rots;
    std::vector<std::vector<const u64 *>> pt;  // [1][rot]
    u64 *store = nullptr;
    ~ShuffleDev() {
        if (store) cudaFree(store);
    }
};

struct copse_model {
    CompiledForest f;
    std::unique_ptr<DeviceModel> dev;
    std::unique_ptr<EncModel> enc;       // set by copse_encrypt_model
    std::unique_ptr<ShuffleDev> shuf;    // set on first use of a shuffled model
};

// level of Algorithm 1's result before the shuffle: Branches at lvl_D - 1, the level
// products drop one more prime, MultAll ceil(log2 d)
static int result_level(const copse_ctx *c, const CompiledForest &f) {
    return c->L - 1 - (int)clog2u(f.precision) - (f.fused ? 1 : 2) - (int)clog2u(f.d);
}

static copse_status upload_shuffle(copse_ctx *c, copse_model *m, cudaStream_t s) {
    if (m->shuf && m->shuf->ctx_serial == c->serial) return COPSE_OK;
    const CompiledForest &f = m->f;
    auto S = std::make_unique<ShuffleDev>();
    S->ctx_serial = c->serial;
    f.shuffle_rotations(S->rots);
    const int ell = result_level(c, f), A = c->alpha, N = c->N;
    const size_t w = (size_t)(ell + A) * N, nr = S->rots.size();
    CUDA_TRY(cudaMalloc(&S->store, std::max<size_t>(nr * w, 1) * sizeof(u64)));
    const uint32_t n_out = f.n_out();
    std::vector<uint32_t> pat(nr * (size_t)n_out), dg;
    S->pt.assign(1, std::vector<const u64 *>());
    for (size_t r = 0; r < nr; r++) {
        f.shuffle_diagonal(S->rots[r], dg);
        std::copy(dg.begin(), dg.end(), pat.begin() + r * n_out);
        S->pt[0].push_back(S->store + r * w);
    }
    STATUS_TRY(encode_patterns(c, pat, (int)nr, (int)n_out, (int)f.block, ell, A, S->store, s));
    m->shuf = std::move(S);
    return COPSE_OK;
}

// ---------------------------------------------------------------- model upload
static copse_status upload_model(copse_ctx *c, copse_model *m, cudaStream_t s) {
    if (m->dev && m->dev->ctx_serial == c->serial) return COPSE_OK;
    const CompiledForest &f = m->f;
    if ((int)f.log_n != c->logN) { set_error("model compiled for another ring degree"); return COPSE_EINVAL; }
    if ((uint32_t)c->L <= f.levels_used()) {
        set_error("prime chain of " + std::to_string(c->L) + " is too short: the circuit drops " +
                  std::to_string(f.levels_used()) + " primes");
        return COPSE_ELEVEL;
    }
    auto D = std::make_unique<DeviceModel>();
    D->ctx = c;
    D->ctx_serial = c->serial;
    const int N = c->N, L = c->L, A = c->alpha, p = (int)f.precision, B = (int)f.block;
    const int SP = (int)f.span(), NS = (int)f.n_seg;  // slot patterns cover the n_seg blocks of a query
    D->lvl_D = L - 1 - (int)clog2u(f.precision);
    D->lvl_B = D->lvl_D - 1;
    const u64 t = c->t;
    const size_t nleaf = 4 * (size_t)p;
    D->R.plan = f.group_reshuffle();
    D->Lv.plan = f.group_level();
    auto count_pt = [](const BsgsGroup &G) {
        size_t n = 0;
        for (const auto &a : G.acc)
            for (int32_t i : a.diag) n += i >= 0;
        return n;
    };
    const size_t nR = count_pt(D->R.plan), nLv = count_pt(D->Lv.plan);
    const size_t words = (nleaf * L + nR * (D->lvl_D + A) + nLv * (D->lvl_D + A) + f.d * D->lvl_D) * (size_t)N;
    CUDA_TRY(cudaMalloc(&D->store, std::max<size_t>(words, 1) * sizeof(u64)));
    u64 *cur = D->store;
    // SecComp leaf plaintexts over whole blocks (threshold bit 0 past the decisions)
    {
        std::vector<uint32_t> pat(nleaf * SP);
        for (int i = 0; i < p; i++) {
            for (int x = 0; x < SP; x++) {
                const uint32_t y = f.thr_bit((uint32_t)(x / B), (uint32_t)(x % B), (uint32_t)i);
                pat[(0 * p + i) * (size_t)SP + x] = y ? (uint32_t)(t - 1) : 0;    // lt: x * (-y) + y
                pat[(1 * p + i) * (size_t)SP + x] = y;
                pat[(2 * p + i) * (size_t)SP + x] = y ? 1u : (uint32_t)(t - 1);   // eq: x * (2y - 1) + (1 - y)
                pat[(3 * p + i) * (size_t)SP + x] = y ? 0u : 1u;
            }
        }
        STATUS_TRY(encode_patterns(c, pat, (int)nleaf, SP, SP, L, 0, cur, s));
        for (int i = 0; i < p; i++) {
            D->lt_mul.push_back(cur + ((size_t)(0 * p + i) * L) * N);
            D->lt_add.push_back(cur + ((size_t)(1 * p + i) * L) * N);
            D->eq_mul.push_back(cur + ((size_t)(2 * p + i) * L) * N);
            D->eq_add.push_back(cur + ((size_t)(3 * p + i) * L) * N);
        }
        cur += nleaf * L * (size_t)N;
    }
    // Diagonal plaintexts of a group, in the extended basis (the products are summed
    // before the key switch's ModDown): diagonal giant + baby of matrix a, shifted by
    // the giant step inside the block; encoded in chunks to bound the staging memory.
    auto encode_group = [&](DeviceModel::Group &G, int level, int rows,
                            const std::function<void(uint32_t, uint32_t, uint32_t, std::vector<uint32_t> &)> &diag) {
        const size_t w = (size_t)(level + A) * N;
        const size_t nacc = G.plan.acc.size(), nb = G.plan.baby.size();
        G.pt.assign(nacc, std::vector<const u64 *>(nb, nullptr));
        G.acc_mat.resize(nacc);
        G.acc_giant.resize(nacc);
        std::vector<std::pair<size_t, size_t>> items;  // (acc, baby) with a nonzero diagonal
        for (size_t a = 0; a < nacc; a++) {
            G.acc_mat[a] = (int)G.plan.acc[a].mat;
            G.acc_giant[a] = G.plan.acc[a].giant;
            for (size_t j = 0; j < nb; j++)
                if (G.plan.acc[a].diag[j] >= 0) items.push_back({a, j});
        }
        const size_t CH = 256;
        std::vector<uint32_t> pat, dg;
        for (size_t i0 = 0; i0 < items.size(); i0 += CH) {
            const size_t n = std::min(CH, items.size() - i0);
            pat.assign(n * (size_t)SP, 0u);
            for (size_t x = 0; x < n; x++) {
                const auto &A_ = G.plan.acc[items[i0 + x].first];
                const uint32_t giant = A_.giant, i = (uint32_t)A_.diag[items[i0 + x].second];
                for (int sg = 0; sg < NS; sg++) {
                    diag(A_.mat, i, (uint32_t)sg, dg);
                    for (int r = 0; r < rows; r++) pat[x * SP + (size_t)sg * B + giant + r] = dg[r];
                }
                G.pt[items[i0 + x].first][items[i0 + x].second] = cur + (i0 + x) * w;
            }
            STATUS_TRY(encode_patterns(c, pat, (int)n, SP, SP, level, A, cur + i0 * w, s));
        }
        cur += items.size() * w;
        return COPSE_OK;
    };
    for (const auto &a : D->R.plan.acc)
        if (a.giant + f.m1() > (uint32_t)B) { set_error("internal: shifted reshuffle diagonal leaves the block"); return COPSE_EINVAL; }
    for (const auto &a : D->Lv.plan.acc)
        if (a.giant + f.L > (uint32_t)B) { set_error("internal: shifted level diagonal leaves the block"); return COPSE_EINVAL; }
    // fused level products (reshuffle folded in) act on Decisions, one level higher
    const int lvl_lv = f.fused ? D->lvl_D : D->lvl_B;
    // reshuffle diagonals at the level of Decisions
    {
        std::vector<uint8_t> dg8;
        STATUS_TRY(encode_group(D->R, D->lvl_D, (int)f.m1(), [&](uint32_t, uint32_t i, uint32_t sg, std::vector<uint32_t> &out) {
            f.reshuffle_diagonal(i, dg8, sg);
            out.assign(dg8.begin(), dg8.end());
        }));
    }
    // level diagonals (signed, mask folded in) and masks at the level of Branches
    {
        std::vector<uint64_t> dg64;
        STATUS_TRY(encode_group(D->Lv, lvl_lv, (int)f.L, [&](uint32_t k, uint32_t i, uint32_t sg, std::vector<uint32_t> &out) {
            if (f.fused) f.fused_diagonal(k + 1, i, t, dg64, sg);
            else f.level_diagonal(k + 1, i, t, dg64, sg);
            out.assign(dg64.begin(), dg64.end());
        }));
        std::vector<uint32_t> mpat((size_t)f.d * SP, 0u);
        for (uint32_t k = 1; k <= f.d; k++) {
            for (int sg = 0; sg < NS; sg++)
                for (uint32_t x = 0; x < f.L; x++) mpat[(size_t)(k - 1) * SP + (size_t)sg * B + x] = f.mask_at(k, x, (uint32_t)sg);
            D->mask.push_back(cur + (size_t)(k - 1) * lvl_lv * N);
        }
        STATUS_TRY(encode_patterns(c, mpat, (int)f.d, SP, SP, lvl_lv, 0, cur, s));
    }
    CUDA_TRY(cudaStreamSynchronize(s));
    m->dev = std::move(D);
    return COPSE_OK;
}

// ---------------------------------------------------------------- models
extern "C" copse_status copse_compile_forest(const char *text, size_t len, uint32_t precision, uint32_t n_features,
                                             uint32_t log_n, copse_model **out) {
    if (!out) { set_error("null output"); return COPSE_EINVAL; }
    *out = nullptr;
    auto m = std::make_unique<copse_model>();
    std::string err;
    int st = compile_forest(text, len, precision, n_features, log_n, m->f, err);
    if (st) { set_error(err); return st; }
    *out = m.release();
    return COPSE_OK;
}

extern "C" void copse_model_destroy(copse_model *m) { delete m; }

uint32_t model_block(const copse_model *m) { return m->f.span(); }

SegLayout seg_layout(const CompiledForest &f) {
    SegLayout lay{};
    lay.nseg = (int)f.n_seg;
    lay.block = (int)f.block;
    lay.off[0] = 0;
    if (f.n_seg == 1) {
        lay.off[1] = (int)f.n_out();
    } else {
        for (uint32_t sg = 0; sg < f.n_seg; sg++) lay.off[sg + 1] = lay.off[sg] + (int)f.seg[sg].L;
    }
    lay.total = lay.off[lay.nseg];
    return lay;
}
uint32_t model_features(const copse_model *m) { return m->f.n_features; }
uint32_t model_leaves(const copse_model *m) { return m->f.n_out(); }
uint32_t model_precision(const copse_model *m) { return m->f.precision; }
int model_log_n(const copse_model *m) { return (int)m->f.log_n; }

extern "C" copse_status copse_model_info_get(const copse_model *m, copse_model_info *info) {
    if (!m || !info) { set_error("null argument"); return COPSE_EINVAL; }
    const CompiledForest &f = m->f;
    info->n_features = f.n_features;
    info->precision = f.precision;
    info->K = f.K;
    info->q = f.q;
    info->b = f.b_total;
    info->n_leaves = f.L_total;
    info->depth = f.d;
    info->n_trees = (uint32_t)f.roots.size();
    info->n_classes = (uint32_t)f.classes.size();
    info->block = f.block;
    std::vector<uint32_t> rs, ls;
    f.group_reshuffle().rotations(rs);
    f.group_level().rotations(ls);
    info->n_rot_reshuffle = (uint32_t)rs.size();
    info->n_rot_level = (uint32_t)ls.size();
    info->levels_used = f.levels_used();
    info->n_out = f.n_out();
    info->n_segments = f.n_seg;
    info->block_branches = f.b;
    info->block_leaves = f.L;
    return COPSE_OK;
}

extern "C" copse_status copse_model_export(const copse_model *m, uint32_t *thr_slot, int32_t *slot_branch,
                                           uint8_t *R, uint8_t *lvl, uint8_t *mask, uint32_t *br_level) {
    if (!m) { set_error("null model"); return COPSE_EINVAL; }
    const CompiledForest &f = m->f;
    if (f.n_seg > 1) { set_error("the model is compiled in row segments: its structures are per segment"); return COPSE_EINVAL; }
    if (thr_slot) std::copy(f.thr_slot.begin(), f.thr_slot.end(), thr_slot);
    if (slot_branch) std::copy(f.slot_branch.begin(), f.slot_branch.end(), slot_branch);
    if (R) std::copy(f.R.begin(), f.R.end(), R);
    if (lvl) std::copy(f.lvl.begin(), f.lvl.end(), lvl);
    if (mask) std::copy(f.mask.begin(), f.mask.end(), mask);
    if (br_level)
        for (uint32_t i = 0; i < f.b; i++) br_level[i] = (uint32_t)f.br_level[i];
    return COPSE_OK;
}

extern "C" copse_status copse_model_rotations(const copse_model *m, uint32_t *reshuffle, uint32_t *level) {
    if (!m) { set_error("null model"); return COPSE_EINVAL; }
    std::vector<uint32_t> rs, ls;
    m->f.group_reshuffle().rotations(rs);
    m->f.group_level().rotations(ls);
    if (reshuffle) std::copy(rs.begin(), rs.end(), reshuffle);
    if (level) std::copy(ls.begin(), ls.end(), level);
    return COPSE_OK;
}

extern "C" copse_status copse_model_set_bsgs(copse_model *m, uint32_t g_reshuffle, uint32_t g_level) {
    if (!m) { set_error("null model"); return COPSE_EINVAL; }
    CompiledForest &f = m->f;
    // a giant step k g must keep the shifted diagonal inside the query block
    auto fits = [&](const BsgsGroup &G, uint32_t rows) {
        for (const auto &a : G.acc)
            if (a.giant + rows > f.block) return false;
        return true;
    };
    const bool ok = f.fused ? fits(bsgs_group(f.fused_nonzero, g_reshuffle), f.L)
                            : fits(bsgs_group({f.rot_reshuffle}, g_reshuffle), f.m1()) &&
                                  fits(bsgs_group(f.lvl_nonzero, g_level), f.L);
    if (!ok) {
        set_error("baby-step size moves a diagonal out of the query block");
        return COPSE_EINVAL;
    }
    if (f.g_reshuffle != g_reshuffle || f.g_level != g_level) {
        f.g_reshuffle = g_reshuffle;
        f.g_level = g_level;
        if (m->dev || m->enc) {
            cudaDeviceSynchronize();
            m->dev.reset();
            m->enc.reset();
        }
    }
    return COPSE_OK;
}

extern "C" copse_status copse_model_set_fused(copse_model *m, int on) {
    if (!m) { set_error("null model"); return COPSE_EINVAL; }
    CompiledForest &f = m->f;
    if (on && f.encrypted) { set_error("fused level matrices are a plaintext-model option"); return COPSE_EINVAL; }
    if (f.fused != (on != 0)) {
        if (on && f.fused_nonzero.empty()) f.build_fused();
        f.fused = on != 0;
        if (m->dev || m->shuf) {
            cudaDeviceSynchronize();
            m->dev.reset();
            m->shuf.reset();
        }
    }
    return COPSE_OK;
}

extern "C" int copse_model_is_fused(const copse_model *m) { return m && m->f.fused ? 1 : 0; }

extern "C" copse_status copse_model_set_encrypted(copse_model *m, int on) {
    if (!m) { set_error("null model"); return COPSE_EINVAL; }
    if (on && m->f.fused) { set_error("the encrypted model keeps the reshuffle and level matrices apart (Table 1d)"); return COPSE_EINVAL; }
    if (m->f.encrypted != (on != 0)) {
        m->f.encrypted = on != 0;
        if (m->dev || m->enc) {
            cudaDeviceSynchronize();
            m->dev.reset();
            m->enc.reset();
        }
    }
    return COPSE_OK;
}

extern "C" int copse_model_is_encrypted(const copse_model *m) { return m && m->f.encrypted ? 1 : 0; }

extern "C" copse_status copse_model_set_shuffle(copse_model *m, const int32_t *src, size_t n_out,
                                                const uint32_t *codebook) {
    if (!m || (n_out && (!src || !codebook))) { set_error("null argument"); return COPSE_EINVAL; }
    CompiledForest &f = m->f;
    if (n_out && f.n_seg > 1) { set_error("label shuffle needs a model in one query block (not in row segments)"); return COPSE_EINVAL; }
    if (n_out) {
        if (n_out < f.L || n_out > f.block) { set_error("shuffle output must hold every leaf and fit the query block"); return COPSE_EINVAL; }
        std::vector<char> seen(f.L, 0);
        for (size_t j = 0; j < n_out; j++) {
            if (src[j] < -1 || src[j] >= (int32_t)f.L || (src[j] >= 0 && seen[src[j]]++)) {
                set_error("shuffle source is not a padded permutation of the leaves");
                return COPSE_EINVAL;
            }
            if (codebook[j] >= f.classes.size()) { set_error("codebook class out of range"); return COPSE_EINVAL; }
            if (src[j] >= 0 && (int)codebook[j] != f.leaf_class[src[j]]) {
                set_error("codebook does not carry each leaf's class");
                return COPSE_EINVAL;
            }
        }
        for (char x : seen)
            if (!x) { set_error("shuffle source misses a leaf"); return COPSE_EINVAL; }
    }
    cudaDeviceSynchronize();
    f.shuffle_src.assign(src, src + n_out);
    f.codebook.assign(codebook, codebook + n_out);
    m->shuf.reset();
    return COPSE_OK;
}

extern "C" copse_status copse_model_codebook(const copse_model *m, uint32_t *classes) {
    if (!m || !classes) { set_error("null argument"); return COPSE_EINVAL; }
    const CompiledForest &f = m->f;
    if (f.shuffle_src.empty())
        for (uint32_t j = 0; j < f.L_total; j++) classes[j] = (uint32_t)f.leaf_class[j];
    else
        std::copy(f.codebook.begin(), f.codebook.end(), classes);
    return COPSE_OK;
}

extern "C" copse_status copse_encrypt_model(copse_ctx *c, const copse_keys *k, copse_model *m, uint64_t seed) {
    if (!c || !k || !m) { set_error("null argument"); return COPSE_EINVAL; }
    const CompiledForest &f = m->f;
    if (!f.encrypted) { set_error("model is not in encrypted mode (copse_model_set_encrypted)"); return COPSE_EINVAL; }
    if ((int)f.log_n != c->logN) { set_error("model compiled for another ring degree"); return COPSE_EINVAL; }
    if ((uint32_t)c->L <= f.levels_used()) {
        set_error("prime chain of " + std::to_string(c->L) + " is too short: the circuit drops " +
                  std::to_string(f.levels_used()) + " primes");
        return COPSE_ELEVEL;
    }
    CUDA_TRY(cudaSetDevice(c->device));
    auto E = std::make_unique<EncModel>();
    STATUS_TRY(enc_model_build(c, k, f, seed, *E, 0));
    m->enc = std::move(E);
    return COPSE_OK;
}

extern "C" copse_status copse_encmodel_export(copse_ctx *c, const copse_model *m, size_t index, uint64_t *out,
                                             size_t words) {
    if (!c || !m || !out) { set_error("null argument"); return COPSE_EINVAL; }
    if (!m->enc || m->enc->ctx_serial != c->serial) { set_error("model not encrypted on this context"); return COPSE_EINVAL; }
    const EncModel &E = *m->enc;
    if (index >= E.level.size()) { set_error("model ciphertext index out of range"); return COPSE_EINVAL; }
    if (words < (size_t)2 * E.level[index] * c->N) { set_error("output buffer too small"); return COPSE_EINVAL; }
    DCt ct;
    STATUS_TRY(enc_materialize(c, E, (int)index, &ct, 0));
    copse_status st = ct_to_coeff_host(c, ct, out, 0);
    ct_free(&ct, 0);
    CUDA_TRY(cudaStreamSynchronize(0));
    return st;
}

extern "C" copse_status copse_model_get_bsgs(const copse_model *m, uint32_t *g_reshuffle, uint32_t *g_level) {
    if (!m || !g_reshuffle || !g_level) { set_error("null argument"); return COPSE_EINVAL; }
    *g_reshuffle = m->f.g_reshuffle;
    *g_level = m->f.g_level;
    return COPSE_OK;
}

extern "C" copse_status copse_classify_plain(const copse_model *m, const uint32_t *feats, size_t n,
                                             uint8_t *out_bits) {
    if (!m || (n && (!feats || !out_bits))) { set_error("null argument"); return COPSE_EINVAL; }
    for (size_t j = 0; j < n; j++) classify_plain(m->f, feats + j * m->f.n_features, out_bits + j * m->f.L_total);
    return COPSE_OK;
}

// ---------------------------------------------------------------- keys
extern "C" copse_status copse_keygen(copse_ctx *c, uint64_t seed, const copse_model *const *models, size_t n_models,
                                     copse_keys **keys, copse_evk **evk) {
    if (!c || !keys || !evk || (n_models && !models)) { set_error("null argument"); return COPSE_EINVAL; }
    std::vector<u64> gal;
    const u64 m2 = 2ull * c->N;
    for (size_t i = 0; i < n_models; i++) {
        const CompiledForest &f = models[i]->f;
        if ((int)f.log_n != c->logN) { set_error("model compiled for another ring degree"); return COPSE_EINVAL; }
        std::vector<uint32_t> rs, ls;
        std::vector<uint32_t> sr;
        f.group_reshuffle().rotations(rs);
        f.group_level().rotations(ls);
        f.shuffle_rotations(sr);
        rs.insert(rs.end(), ls.begin(), ls.end());
        rs.insert(rs.end(), sr.begin(), sr.end());
        for (uint32_t r : rs) {
            if (!r) continue;
            u64 g = 1, b = 3;
            for (uint32_t e = r; e; e >>= 1, b = b * b % m2)
                if (e & 1) g = g * b % m2;
            if (std::find(gal.begin(), gal.end(), g) == gal.end()) gal.push_back(g);
        }
    }
    std::sort(gal.begin(), gal.end());
    CUDA_TRY(cudaSetDevice(c->device));
    return keygen_dev(c, seed, gal, keys, evk);
}

extern "C" void copse_keys_destroy(copse_keys *k) {
    if (!k) return;
    cudaStreamSynchronize(0);
    dev_free(k->s_hat, 0);
    dev_free(k->pk, 0);
    delete k;
}

extern "C" void copse_evk_destroy(copse_evk *e) {
    if (!e) return;
    cudaStreamSynchronize(0);
    dev_free(e->rlk, 0);
    for (u64 *p : e->gk) dev_free(p, 0);
    delete e;
}

extern "C" copse_status copse_keys_export_secret(const copse_keys *k, int64_t *s) {
    if (!k || !s) { set_error("null argument"); return COPSE_EINVAL; }
    std::copy(k->s_host.begin(), k->s_host.end(), s);
    return COPSE_OK;
}

extern "C" copse_status copse_evk_export(const copse_evk *e, uint64_t galois, uint64_t *out, size_t words) {
    if (!e || !out) { set_error("null argument"); return COPSE_EINVAL; }
    copse_ctx *c = e->ctx;
    const u64 *key = galois == 0 ? e->rlk : e->find(galois);
    if (!key) { set_error("no key for that Galois element"); return COPSE_ENOKEY; }
    const size_t n = ksk_words(c);
    if (words < n) { set_error("buffer too small"); return COPSE_EINVAL; }
    u64 *tmp = nullptr;
    STATUS_TRY(dev_alloc(c, (void **)&tmp, n * 8, 0));
    CUDA_TRY(cudaMemcpyAsync(tmp, key, n * 8, cudaMemcpyDeviceToDevice, 0));
    STATUS_TRY(ksk_from_mont(c, tmp, 0));
    const int NB = c->L + c->alpha;
    STATUS_TRY(ntt_inverse(c, NttBatch{tmp, (size_t)NB * c->N, 2 * c->ndig, 0, NB, NB, -1}, 0));
    CUDA_TRY(cudaMemcpy(out, tmp, n * 8, cudaMemcpyDeviceToHost));
    dev_free(tmp, 0);
    CUDA_TRY(cudaStreamSynchronize(0));
    return COPSE_OK;
}

// ---------------------------------------------------------------- data
extern "C" copse_status copse_encrypt_features(copse_ctx *c, const copse_keys *k, copse_model *m,
                                               const uint32_t *feats, size_t nq, int on_device, uint64_t seed,
                                               copse_ctbuf **out, void *stream) {
    if (!c || !k || !m || !out || (nq && !feats)) { set_error("null argument"); return COPSE_EINVAL; }
    const CompiledForest &f = m->f;
    if ((int)f.log_n != c->logN) { set_error("model compiled for another ring degree"); return COPSE_EINVAL; }
    const size_t per_ct = (size_t)(c->N / f.span());
    if (nq > per_ct * 64) { set_error("more than 64 ciphertexts of queries"); return COPSE_EINVAL; }
    cudaStream_t s = as_stream(stream);
    const uint32_t *d_feats = feats;
    uint32_t *tmp = nullptr;
    const size_t nfe = nq * f.n_features;
    if (!on_device) {
        for (size_t i = 0; i < nfe; i++)
            if (f.precision < 32 && feats[i] >= (1u << f.precision)) { set_error("feature value needs more bits than the precision"); return COPSE_EINVAL; }
        STATUS_TRY(dev_alloc(c, (void **)&tmp, std::max<size_t>(nfe, 1) * 4, s));
        if (nfe) CUDA_TRY(cudaMemcpyAsync(tmp, feats, nfe * 4, cudaMemcpyHostToDevice, s));
        d_feats = tmp;
    }
    auto buf = std::make_unique<copse_ctbuf>();
    buf->ctx = c;
    buf->stream = s;
    // query ciphertext q holds queries [q per_ct, (q + 1) per_ct); its plane i is encryption q p + i
    copse_status st = COPSE_OK;
    for (size_t j0 = 0, q = 0; st == COPSE_OK && (j0 < nq || (nq == 0 && q == 0)); j0 += per_ct, q++) {
        const size_t n = std::min(per_ct, nq - j0);
        st = encrypt_planes(c, k, d_feats + j0 * f.n_features, (int)n, (int)f.n_features, (int)f.K, (int)f.q,
                            (int)f.pd(), (int)f.block, (int)f.n_seg, (int)f.precision, seed, buf->cts, s, nullptr,
                            (int)(q * f.precision));
        if (nq == 0) break;
    }
    if (tmp) dev_free(tmp, s);
    if (st) return st;
    *out = buf.release();
    return COPSE_OK;
}

// The products of one vector with a group of matrices: the plain diagonal method,
// or its baby-step / giant-step form.
static copse_status group_matmul(copse_ctx *c, const copse_evk *evk, const DCt &v, const DeviceModel::Group &G,
                                 const std::vector<const u64 *> &add, std::vector<DCt> &out, cudaStream_t s) {
    if (G.plan.plain()) return op_matmul(c, evk, v, G.plan.baby, G.pt, add, out, s);
    return op_matmul_bsgs(c, evk, v, G.plan.baby, G.pt, G.acc_mat, G.acc_giant, (int)G.plan.n_mat, add, out, s);
}

// SecComp (Section 4.1.2) of nct query ciphertexts, p feature planes each (x[q p + i]):
// the decision vectors Dc[q] = [x < thresholds] at level lvl_D.  The leaves of all
// query ciphertexts, and then each level of their combine trees, run as one batch.
static copse_status seccomp(copse_ctx *c, const copse_evk *evk, copse_model *m, const DCt *x, int nct,
                            std::vector<DCt> &Dc, cudaStream_t s, int lane) {
    const bool enc = m->f.encrypted;
    const DeviceModel *D = m->dev.get();
    const int p = (int)m->f.precision;
    struct Node { DCt lt, eq; };
    // SecComp leaves, most significant plane first: lt = (1 - x) y, eq = [x == y]
    std::vector<std::vector<Node>> nodes(nct, std::vector<Node>(p));
    if (!enc) {
        // plaintext thresholds: both leaves are affine in x
        std::vector<AffineJob> lj;
        for (int q = 0; q < nct; q++)
            for (int k = 0; k < p; k++) {
                const int i = p - 1 - k;
                const DCt *xi = &x[(size_t)q * p + i];
                lj.push_back(AffineJob{xi, D->lt_mul[i], D->lt_add[i], &nodes[q][k].lt});
                lj.push_back(AffineJob{xi, D->eq_mul[i], D->eq_add[i], &nodes[q][k].eq});
            }
        STATUS_TRY(op_affine_many(c, lj, s));
    } else {
        // encrypted thresholds y: xy = x * y (every plane together), lt = y - xy,
        // eq = 2 xy - (x + y) + 1, where a binary operation first switches its higher
        // operand down (y and x + y to the level of xy).  The elementwise steps of every
        // (query ciphertext, plane) run as items of persistent work-list launches.
        const int top = x[0].level, ell = top - 1, N = c->N;
        std::vector<DCt> Y(p), XY((size_t)nct * p), S((size_t)nct * p), Yd, Sd;
        std::vector<MulJob> mj;
        for (int k = 0; k < p; k++) STATUS_TRY(enc_materialize(c, *m->enc, m->enc->idx_thr(p - 1 - k), &Y[k], s));
        for (int q = 0; q < nct; q++)
            for (int k = 0; k < p; k++)
                mj.push_back(MulJob{&x[(size_t)q * p + p - 1 - k], &Y[k], &XY[(size_t)q * p + k]});
        STATUS_TRY(op_mul_many(c, evk, mj, s));
        // y at the products' level, once per plane
        std::vector<const DCt *> yp;
        for (int k = 0; k < p; k++) yp.push_back(&Y[k]);
        STATUS_TRY(op_modswitch_cts(c, yp, Yd, s));
        // x + y at the top level, then switched down together
        std::vector<WlItem> wl;
        std::vector<const DCt *> sp;
        for (int q = 0; q < nct; q++)
            for (int k = 0; k < p; k++) {
                const size_t j = (size_t)q * p + k;
                const DCt &xi = x[(size_t)q * p + p - 1 - k];
                if (xi.level != top || Y[k].level != top || XY[j].level != ell) {
                    set_error("internal: unexpected levels in the comparison leaves");
                    return COPSE_EINVAL;
                }
                STATUS_TRY(ct_alloc(c, &S[j], top, 2, s));
                WlItem w;
                w.kind = WL_ADD;
                w.level = top;
                w.comp = (size_t)top * N;
                w.x = xi.data;
                w.y = Y[k].data;
                w.o0 = S[j].data;
                wl.push_back(w);
                sp.push_back(&S[j]);
            }
        STATUS_TRY(worklist_run(c, wl, 1000, s));
        STATUS_TRY(op_modswitch_cts(c, sp, Sd, s));
        // the leaves: lt = y - xy, eq = 2 xy - (x + y) + 1
        wl.clear();
        for (int q = 0; q < nct; q++)
            for (int k = 0; k < p; k++) {
                const size_t j = (size_t)q * p + k;
                STATUS_TRY(ct_alloc(c, &nodes[q][k].lt, ell, 2, s));
                STATUS_TRY(ct_alloc(c, &nodes[q][k].eq, ell, 2, s));
                WlItem w;
                w.kind = WL_LEAF;
                w.level = ell;
                w.comp = (size_t)ell * N;
                w.x = Sd[j].data;
                w.y = Yd[k].data;
                w.z = XY[j].data;
                w.o0 = nodes[q][k].lt.data;
                w.o1 = nodes[q][k].eq.data;
                wl.push_back(w);
            }
        STATUS_TRY(worklist_run(c, wl, 1000, s));
        for (auto *v : {&Y, &XY, &S, &Yd, &Sd})
            for (DCt &t : *v)
                if (t.data) ct_free(&t, s);
    }
    // balanced combine (lt_h + eq_h lt_l, eq_h eq_l); no eq at the root.  Each tree
    // level is one batch: the high nodes' lt switched down to the products' level
    // together, then every product of the level, the lt sums added in the products'
    // finishing store.
    while (nodes[0].size() > 1) {
        const bool root = nodes[0].size() == 2;
        const int npair = (int)(nodes[0].size() / 2);
        std::vector<std::vector<Node>> nx(nct, std::vector<Node>(npair));
        std::vector<const DCt *> hi_lt;
        for (int q = 0; q < nct; q++)
            for (int k = 0; k < npair; k++) {
                const Node &hi = nodes[q][2 * k], &lo = nodes[q][2 * k + 1];
                // hi.lt and hi.eq share a level; lo (possibly carried up) is never lower
                if (hi.lt.level != hi.eq.level || lo.lt.level < hi.eq.level || lo.eq.level < hi.eq.level ||
                    hi.lt.level != nodes[0][0].lt.level) {
                    set_error("internal: unexpected levels in the comparison tree");
                    return COPSE_EINVAL;
                }
                hi_lt.push_back(&hi.lt);
            }
        // the modulus switch on a forked branch, overlapping the products; joined
        // before their finishing store (the frees below are ordered after the join)
        std::vector<DCt> hms;
        STATUS_TRY(fork_begin(c, s, 1, lane));
        STATUS_TRY(op_modswitch_cts(c, hi_lt, hms, fork_stream(c, 0, lane)));
        std::vector<MulJob> mj;
        for (int q = 0; q < nct; q++)
            for (int k = 0; k < npair; k++) {
                Node &hi = nodes[q][2 * k], &lo = nodes[q][2 * k + 1];
                mj.push_back(MulJob{&hi.eq, &lo.lt, &nx[q][k].lt, &hms[(size_t)q * npair + k]});
                if (!root) mj.push_back(MulJob{&hi.eq, &lo.eq, &nx[q][k].eq});
            }
        STATUS_TRY(op_mul_many(c, evk, mj, s, lane));
        for (DCt &h : hms) ct_free(&h, s);
        for (int q = 0; q < nct; q++) {
            for (int k = 0; k < 2 * npair; k++) {
                ct_free(&nodes[q][k].lt, s);
                ct_free(&nodes[q][k].eq, s);
            }
            if (nodes[q].size() % 2) nx[q].push_back(nodes[q].back());
            nodes[q].swap(nx[q]);
        }
    }
    Dc.assign(nct, DCt());
    for (int q = 0; q < nct; q++) {
        Dc[q] = nodes[q][0].lt;
        if (nodes[q][0].eq.data) ct_free(&nodes[q][0].eq, s);
        if (Dc[q].level != (enc ? m->enc->lvl_D : D->lvl_D)) {
            set_error("internal: unexpected level of the decision vector");
            return COPSE_EINVAL;
        }
    }
    return COPSE_OK;
}

// Algorithm 1 for every query ciphertext of `feats` (p feature planes each, one
// ciphertext after another): one result ciphertext per query ciphertext.  With an
// encrypted model the matrix products of all query ciphertexts run together, so
// each encrypted diagonal is read and its mask regenerated once for all of them.
template <class Mark>
static copse_status aggregate(copse_ctx *c, const copse_evk *evk, copse_model *m,
                              std::vector<std::vector<DCt>> &lvs, int nct, std::vector<DCt> &results, cudaStream_t s,
                              Mark &mark);

static copse_status infer_multi(copse_ctx *c, const copse_evk *evk, copse_model *m, const copse_ctbuf *feats,
                                std::vector<DCt> &results, cudaStream_t s, int lane = 0,
                                cudaEvent_t *stage_ev = nullptr) {
    const bool enc = m->f.encrypted;
    if (enc) {
        if (!m->enc || m->enc->ctx_serial != c->serial) {
            set_error("encrypted-mode model has no encryption on this context (copse_encrypt_model)");
            return COPSE_EINVAL;
        }
        if (m->enc->g_r != m->f.g_reshuffle || m->enc->g_l != m->f.g_level) {
            set_error("model was encrypted for another baby-step plan");
            return COPSE_EINVAL;
        }
    } else {
        STATUS_TRY(upload_model(c, m, s));
    }
    const DeviceModel *D = m->dev.get();
    const int p = (int)m->f.precision;
    const size_t n_in = feats->cts.size();
    if (n_in == 0 || n_in % (size_t)p) { set_error("feature buffer does not hold p ciphertexts per query ciphertext"); return COPSE_EINVAL; }
    for (const DCt &x : feats->cts)
        if (x.level != c->L) { set_error("feature ciphertexts must be fresh"); return COPSE_EINVAL; }
    const int nct = (int)(n_in / p);
    // stage boundaries (comparison | reshuffle | levels | aggregation), when timed
    auto mark = [&](int i) -> copse_status {
        if (stage_ev) CUDA_TRY(cudaEventRecord(stage_ev[i], s));
        return COPSE_OK;
    };
    STATUS_TRY(mark(0));
    std::vector<DCt> Dc;
    STATUS_TRY(seccomp(c, evk, m, feats->cts.data(), nct, Dc, s, lane));
    STATUS_TRY(mark(1));
    std::vector<std::vector<DCt>> lvs(nct);
    if (m->f.fused) {
        // fused level products: (S_k R) * Decisions XOR Mask_k, no Branches vector
        STATUS_TRY(mark(2));
        for (int q = 0; q < nct; q++) STATUS_TRY(group_matmul(c, evk, Dc[q], D->Lv, D->mask, lvs[q], s));
        for (DCt &x : Dc) ct_free(&x, s);
        STATUS_TRY(mark(3));
        return aggregate(c, evk, m, lvs, nct, results, s, mark);
    }
    // reshuffle: Branches = R_ext * Decisions
    std::vector<std::vector<DCt>> br(nct);
    if (enc) {
        STATUS_TRY(enc_matmul(c, evk, *m->enc, Dc, 0, br, s));
    } else {
        for (int q = 0; q < nct; q++) STATUS_TRY(group_matmul(c, evk, Dc[q], D->R, {nullptr}, br[q], s));
    }
    for (DCt &x : Dc) ct_free(&x, s);
    STATUS_TRY(mark(2));
    // levels: Lvl_k * Branches XOR Mask_k, rotations of Branches shared by every level
    std::vector<DCt> B(nct);
    for (int q = 0; q < nct; q++) B[q] = br[q][0];
    if (enc) {
        STATUS_TRY(enc_matmul(c, evk, *m->enc, B, 1, lvs, s));
    } else {
        for (int q = 0; q < nct; q++) STATUS_TRY(group_matmul(c, evk, B[q], D->Lv, D->mask, lvs[q], s));
    }
    for (DCt &x : B) ct_free(&x, s);
    STATUS_TRY(mark(3));
    return aggregate(c, evk, m, lvs, nct, results, s, mark);
}

// product across levels (MultAll), then the optional label shuffle; stage mark 4 at the end
template <class Mark>
static copse_status aggregate(copse_ctx *c, const copse_evk *evk, copse_model *m,
                              std::vector<std::vector<DCt>> &lvs, int nct, std::vector<DCt> &results, cudaStream_t s,
                              Mark &mark) {
    // product across levels, balanced; the products of every query ciphertext at one
    // tree level run together
    while (lvs[0].size() > 1) {
        const int npair = (int)(lvs[0].size() / 2);
        std::vector<std::vector<DCt>> nx(nct, std::vector<DCt>(npair));
        std::vector<MulJob> mj;
        for (int q = 0; q < nct; q++)
            for (int k = 0; k < npair; k++) mj.push_back(MulJob{&lvs[q][2 * k], &lvs[q][2 * k + 1], &nx[q][k]});
        STATUS_TRY(op_mul_many(c, evk, mj, s));
        for (int q = 0; q < nct; q++) {
            for (int k = 0; k < 2 * npair; k++) ct_free(&lvs[q][k], s);
            if (lvs[q].size() % 2) nx[q].push_back(lvs[q].back());
            lvs[q].swap(nx[q]);
        }
    }
    results.assign(nct, DCt());
    for (int q = 0; q < nct; q++) results[q] = lvs[q][0];
    // label shuffle with padding (Section 7.2): one more plaintext matrix product
    if (!m->f.shuffle_src.empty()) {
        STATUS_TRY(upload_shuffle(c, m, s));
        for (int q = 0; q < nct; q++) {
            std::vector<DCt> o;
            STATUS_TRY(op_matmul(c, evk, results[q], m->shuf->rots, m->shuf->pt, {nullptr}, o, s));
            ct_free(&results[q], s);
            results[q] = o[0];
        }
    }
    STATUS_TRY(mark(4));
    return COPSE_OK;
}

// one query ciphertext (graph-recorded session items)
static copse_status infer_impl(copse_ctx *c, const copse_evk *evk, copse_model *m, const copse_ctbuf *feats,
                               DCt *result, cudaStream_t s, int lane = 0) {
    if (feats->cts.size() != m->f.precision) { set_error("feature buffer does not hold one ciphertext per bit-plane"); return COPSE_EINVAL; }
    std::vector<DCt> r;
    STATUS_TRY(infer_multi(c, evk, m, feats, r, s, lane));
    *result = r[0];
    return COPSE_OK;
}

extern "C" copse_status copse_infer(copse_ctx *c, const copse_evk *evk, copse_model *m, const copse_ctbuf *feats,
                                    copse_ctbuf **out, void *stream) {
    if (!c || !evk || !m || !feats || !out) { set_error("null argument"); return COPSE_EINVAL; }
    auto buf = std::make_unique<copse_ctbuf>();
    buf->ctx = c;
    buf->stream = as_stream(stream);
    STATUS_TRY(infer_multi(c, evk, m, feats, buf->cts, as_stream(stream)));
    *out = buf.release();
    return COPSE_OK;
}

extern "C" copse_status copse_infer_timed(copse_ctx *c, const copse_evk *evk, copse_model *m,
                                          const copse_ctbuf *feats, copse_ctbuf **out, void *stream,
                                          float stage_ms[4]) {
    if (!c || !evk || !m || !feats || !out || !stage_ms) { set_error("null argument"); return COPSE_EINVAL; }
    if (c->capturing) { set_error("copse_infer_timed cannot be recorded into a graph"); return COPSE_EINVAL; }
    cudaStream_t s = as_stream(stream);
    cudaEvent_t ev[5] = {};
    copse_status st = COPSE_OK;
    for (int i = 0; i < 5 && st == COPSE_OK; i++)
        if (cudaEventCreate(&ev[i]) != cudaSuccess) { set_error("cudaEventCreate failed"); st = COPSE_ECUDA; }
    std::vector<DCt> r;
    if (st == COPSE_OK) st = infer_multi(c, evk, m, feats, r, s, 0, ev);
    if (st == COPSE_OK && cudaEventSynchronize(ev[4]) != cudaSuccess) { set_error("stage event failed"); st = COPSE_ECUDA; }
    for (int i = 0; i < 4 && st == COPSE_OK; i++)
        if (cudaEventElapsedTime(&stage_ms[i], ev[i], ev[i + 1]) != cudaSuccess) { set_error("stage timing failed"); st = COPSE_ECUDA; }
    for (cudaEvent_t e : ev)
        if (e) cudaEventDestroy(e);
    if (st != COPSE_OK) {
        for (DCt &x : r)
            if (x.data) ct_free(&x, s);
        return st;
    }
    auto buf = std::make_unique<copse_ctbuf>();
    buf->ctx = c;
    buf->stream = s;
    buf->cts = r;
    *out = buf.release();
    return COPSE_OK;
}

extern "C" copse_status copse_decrypt_labels(copse_ctx *c, const copse_keys *k, const copse_model *m,
                                             const copse_ctbuf *res, uint8_t *out_bits, size_t nq, int on_device,
                                             void *stream) {
    if (!c || !k || !m || !res || res->cts.empty() || (nq && !out_bits)) { set_error("null argument"); return COPSE_EINVAL; }
    const CompiledForest &f = m->f;
    const size_t per_ct = (size_t)(c->N / f.span());
    if (nq > per_ct * res->cts.size()) { set_error("more queries than slot blocks"); return COPSE_EINVAL; }
    cudaStream_t s = as_stream(stream);
    u64 *slots = nullptr;
    uint8_t *bits = on_device ? out_bits : nullptr;
    STATUS_TRY(dev_alloc(c, (void **)&slots, (size_t)c->N * 8, s));
    const size_t n_out = f.n_out();
    if (!on_device) STATUS_TRY(dev_alloc(c, (void **)&bits, std::max<size_t>(nq * n_out, 1), s));
    // query j is block j mod per_ct of result ciphertext j / per_ct
    for (size_t j0 = 0, q = 0; j0 < nq || (nq == 0 && q == 0); j0 += per_ct, q++) {
        const size_t n = std::min(per_ct, nq - j0);
        STATUS_TRY(decrypt_slots_dev(c, k, res->cts[q], slots, s));
        STATUS_TRY(extract_bits(c, slots, (int)n, seg_layout(f), bits + j0 * n_out, s));
        if (nq == 0) break;
    }
    if (!on_device) {
        CUDA_TRY(cudaMemcpyAsync(out_bits, bits, nq * n_out, cudaMemcpyDeviceToHost, s));
        dev_free(bits, s);
    }
    dev_free(slots, s);
    if (!on_device) CUDA_TRY(cudaStreamSynchronize(s));
    return COPSE_OK;
}

extern "C" copse_status copse_decrypt_slots(copse_ctx *c, const copse_keys *k, const copse_ctbuf *buf, size_t index,
                                            uint64_t *out_slots) {
    if (!c || !k || !buf || !out_slots || index >= buf->cts.size()) { set_error("bad argument"); return COPSE_EINVAL; }
    u64 *slots = nullptr;
    STATUS_TRY(dev_alloc(c, (void **)&slots, (size_t)c->N * 8, 0));
    STATUS_TRY(decrypt_slots_dev(c, k, buf->cts[index], slots, 0));
    CUDA_TRY(cudaMemcpy(out_slots, slots, (size_t)c->N * 8, cudaMemcpyDeviceToHost));
    dev_free(slots, 0);
    CUDA_TRY(cudaStreamSynchronize(0));
    return COPSE_OK;
}

// ---------------------------------------------------------------- buffers
extern "C" size_t copse_ctbuf_count(const copse_ctbuf *b) { return b ? b->cts.size() : 0; }

extern "C" copse_status copse_ctbuf_shape(const copse_ctbuf *b, size_t i, uint32_t *level, uint32_t *ncomp) {
    if (!b || i >= b->cts.size()) { set_error("bad buffer index"); return COPSE_EINVAL; }
    if (level) *level = (uint32_t)b->cts[i].level;
    if (ncomp) *ncomp = (uint32_t)b->cts[i].ncomp;
    return COPSE_OK;
}

extern "C" copse_status copse_ctbuf_export(copse_ctx *c, const copse_ctbuf *b, size_t i, uint64_t *out, size_t words) {
    if (!c || !b || !out || i >= b->cts.size()) { set_error("bad argument"); return COPSE_EINVAL; }
    const DCt &ct = b->cts[i];
    if (words < (size_t)ct.ncomp * ct.level * c->N) { set_error("buffer too small"); return COPSE_EINVAL; }
    return ct_to_coeff_host(c, ct, out, 0);
}

extern "C" copse_status copse_ctbuf_import(copse_ctx *c, const uint64_t *in, size_t n_ct, uint32_t level,
                                           copse_ctbuf **out) {
    if (!c || !in || !out || level < 1 || (int)level > c->L) { set_error("bad argument"); return COPSE_EINVAL; }
    auto buf = std::make_unique<copse_ctbuf>();
    buf->ctx = c;
    for (size_t i = 0; i < n_ct; i++) {
        DCt ct;
        STATUS_TRY(ct_from_coeff_host(c, in + i * 2 * level * (size_t)c->N, (int)level, &ct, 0));
        buf->cts.push_back(ct);
    }
    *out = buf.release();
    return COPSE_OK;
}

extern "C" void copse_ctbuf_destroy(copse_ctbuf *b) {
    // frees are stream-ordered after the work that produced the buffer; work on
    // other streams that still reads it must be ordered before this call
    delete b;
}

// ---------------------------------------------------------------- ring ops
static copse_status one(copse_ctx *c, DCt &r, copse_ctbuf **out, void *stream) {
    auto buf = std::make_unique<copse_ctbuf>();
    buf->ctx = c;
    buf->stream = as_stream(stream);
    buf->cts.push_back(r);
    *out = buf.release();
    return COPSE_OK;
}

extern "C" copse_status copse_ct_mul(copse_ctx *c, const copse_evk *evk, const copse_ctbuf *a, size_t ia,
                                     const copse_ctbuf *b, size_t ib, copse_ctbuf **out, void *stream) {
    if (!c || !evk || !a || !b || !out || ia >= a->cts.size() || ib >= b->cts.size()) { set_error("bad argument"); return COPSE_EINVAL; }
    DCt r;
    STATUS_TRY(op_mul(c, evk, a->cts[ia], b->cts[ib], &r, as_stream(stream)));
    return one(c, r, out, stream);
}

extern "C" copse_status copse_ct_rotate(copse_ctx *c, const copse_evk *evk, const copse_ctbuf *a, size_t ia,
                                        uint32_t k, copse_ctbuf **out, void *stream) {
    if (!c || !evk || !a || !out || ia >= a->cts.size()) { set_error("bad argument"); return COPSE_EINVAL; }
    DCt r;
    STATUS_TRY(op_rotate(c, evk, a->cts[ia], k, &r, as_stream(stream)));
    return one(c, r, out, stream);
}

extern "C" copse_status copse_ct_modswitch(copse_ctx *c, const copse_ctbuf *a, size_t ia, copse_ctbuf **out,
                                           void *stream) {
    if (!c || !a || !out || ia >= a->cts.size()) { set_error("bad argument"); return COPSE_EINVAL; }
    DCt r;
    STATUS_TRY(op_modswitch(c, a->cts[ia], &r, as_stream(stream)));
    return one(c, r, out, stream);
}

extern "C" copse_status copse_ct_mul_plain(copse_ctx *c, const copse_ctbuf *a, size_t ia, const uint64_t *mul_slots,
                                           const uint64_t *add_slots, copse_ctbuf **out, void *stream) {
    if (!c || !a || !mul_slots || !out || ia >= a->cts.size()) { set_error("bad argument"); return COPSE_EINVAL; }
    cudaStream_t s = as_stream(stream);
    const DCt &x = a->cts[ia];
    const int N = c->N;
    std::vector<uint32_t> pat((size_t)2 * N);
    for (int i = 0; i < N; i++) {
        pat[i] = (uint32_t)(mul_slots[i] % c->t);
        pat[(size_t)N + i] = add_slots ? (uint32_t)(add_slots[i] % c->t) : 0;
    }
    u64 *pts = nullptr;
    STATUS_TRY(dev_alloc(c, (void **)&pts, (size_t)2 * x.level * N * 8, s));
    STATUS_TRY(encode_patterns(c, pat, 2, N, N, x.level, 0, pts, s));
    DPt mp{x.level, pts}, ap{x.level, pts + (size_t)x.level * N};
    DCt r;
    copse_status st = op_affine(c, x, mp, add_slots ? &ap : nullptr, &r, s);
    dev_free(pts, s);
    if (st) return st;
    return one(c, r, out, stream);
}

extern "C" copse_status copse_ntt(copse_ctx *c, uint64_t *data, size_t n_polys, uint32_t n_res, int inverse,
                                  void *stream) {
    if (!c || !data || n_res < 1 || (int)n_res > c->L) { set_error("bad argument"); return COPSE_EINVAL; }
    NttBatch b{data, (size_t)n_res * c->N, (int)n_polys, 0, (int)n_res, (int)n_res, -1};
    return inverse ? ntt_inverse(c, b, as_stream(stream)) : ntt_forward(c, b, as_stream(stream));
}

// ---------------------------------------------------------------- sessions (CUDA graphs)
// A session fixes the context, keys and a list of work items (model, number of
// queries) and records one step -- feature encryption, Algorithm 1 and
// decryption of the leaf bits for every item -- once as a CUDA graph.  Items
// run on separate lanes of streams inside the graph, so many queries of many
// forests of uneven size are evaluated by one graph launch.  Every run copies
// the features and a fresh seed into the session's device buffers and
// launches the graph: no host-side kernel launches, allocations or
// synchronisation inside the step.  Intermediates are graph memory nodes
// allocated and freed inside the graph.
struct SessItem {
    copse_model *m = nullptr;
    size_t nq = 0, feat_off = 0, bit_off = 0;
};

struct copse_session {
    copse_ctx *c = nullptr;
    const copse_keys *keys = nullptr;
    const copse_evk *evk = nullptr;
    std::vector<SessItem> items;
    size_t n_feats = 0, n_bits = 0;
    uint32_t *d_feats = nullptr;  // items' features, concatenated
    uint8_t *d_bits = nullptr;    // items' leaf bits, concatenated
    u64 *d_seed = nullptr;        // encryption seed of the next run (item i encrypts with seed + i)
    cudaStream_t cap = nullptr;
    cudaEvent_t ev = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    ~copse_session() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (ev) cudaEventDestroy(ev);
        if (cap) cudaStreamDestroy(cap);
        cudaFree(d_feats);
        cudaFree(d_bits);
        cudaFree(d_seed);
    }
};

// one item's step on stream s and lane `lane`; everything it allocates it also frees
static copse_status item_body(copse_session *S, size_t i, cudaStream_t s, int lane) {
    copse_ctx *c = S->c;
    const SessItem &it = S->items[i];
    const CompiledForest &f = it.m->f;
    copse_ctbuf feats;
    feats.ctx = c;
    feats.stream = s;
    STATUS_TRY(encrypt_planes(c, S->keys, S->d_feats + it.feat_off, (int)it.nq, (int)f.n_features, (int)f.K,
                              (int)f.q, (int)f.pd(), (int)f.block, (int)f.n_seg, (int)f.precision, (u64)i, feats.cts, s,
                              S->d_seed));
    DCt res;
    STATUS_TRY(infer_impl(c, S->evk, it.m, &feats, &res, s, lane));
    u64 *slots = nullptr;
    STATUS_TRY(dev_alloc(c, (void **)&slots, (size_t)c->N * 8, s));
    STATUS_TRY(decrypt_slots_dev(c, S->keys, res, slots, s));
    STATUS_TRY(extract_bits(c, slots, (int)it.nq, seg_layout(f), S->d_bits + it.bit_off, s));
    dev_free(slots, s);
    ct_free(&res, s);
    return COPSE_OK;  // feats frees its ciphertexts on s when it goes out of scope
}

static copse_status session_body(copse_session *S, cudaStream_t cap) {
    copse_ctx *c = S->c;
    const size_t n = S->items.size();
    if (n == 1) return item_body(S, 0, cap, 0);
    const int lanes = (int)std::min<size_t>(n, COPSE_MAX_LANES);
    CUDA_TRY(cudaEventRecord(S->ev, cap));
    for (int l = 0; l < lanes; l++) CUDA_TRY(cudaStreamWaitEvent(lane_stream(c, l), S->ev, 0));
    for (size_t i = 0; i < n; i++) STATUS_TRY(item_body(S, i, lane_stream(c, (int)(i % lanes)), (int)(i % lanes)));
    for (int l = 0; l < lanes; l++) {
        CUDA_TRY(cudaEventRecord(lane_event(c, l), lane_stream(c, l)));
        CUDA_TRY(cudaStreamWaitEvent(cap, lane_event(c, l), 0));
    }
    return COPSE_OK;
}

extern "C" copse_status copse_session_create_batch(copse_ctx *c, const copse_keys *keys, const copse_evk *evk,
                                                   size_t n_items, copse_model *const *models,
                                                   const size_t *n_queries, copse_session **out) {
    if (!c || !keys || !evk || !out || !n_items || !models || !n_queries) { set_error("bad argument"); return COPSE_EINVAL; }
    auto S = std::make_unique<copse_session>();
    S->c = c;
    S->keys = keys;
    S->evk = evk;
    for (size_t i = 0; i < n_items; i++) {
        copse_model *m = models[i];
        if (!m) { set_error("null model"); return COPSE_EINVAL; }
        const CompiledForest &f = m->f;
        if ((int)f.log_n != c->logN) { set_error("model compiled for another ring degree"); return COPSE_EINVAL; }
        if (n_queries[i] > (size_t)(c->N / f.span())) { set_error("more queries than slot blocks"); return COPSE_EINVAL; }
        SessItem it;
        it.m = m;
        it.nq = n_queries[i];
        it.feat_off = S->n_feats;
        it.bit_off = S->n_bits;
        S->n_feats += it.nq * f.n_features;
        S->n_bits += it.nq * f.n_out();
        S->items.push_back(it);
    }
    CUDA_TRY(cudaSetDevice(c->device));
    CUDA_TRY(cudaMalloc(&S->d_feats, std::max<size_t>(S->n_feats, 1) * 4));
    CUDA_TRY(cudaMalloc(&S->d_bits, std::max<size_t>(S->n_bits, 1)));
    CUDA_TRY(cudaMalloc(&S->d_seed, 8));
    CUDA_TRY(cudaMemset(S->d_feats, 0, std::max<size_t>(S->n_feats, 1) * 4));
    CUDA_TRY(cudaMemset(S->d_seed, 0, 8));
    CUDA_TRY(cudaStreamCreateWithFlags(&S->cap, cudaStreamNonBlocking));
    CUDA_TRY(cudaEventCreateWithFlags(&S->ev, cudaEventDisableTiming));
    // everything that synchronises or creates resources happens before capture
    for (const SessItem &it : S->items) {
        if (!it.m->f.encrypted) STATUS_TRY(upload_model(c, it.m, S->cap));
        if (!it.m->f.shuffle_src.empty()) STATUS_TRY(upload_shuffle(c, it.m, S->cap));
    }
    STATUS_TRY(ensure_lanes(c, (int)std::min<size_t>(n_items, COPSE_MAX_LANES)));
    CUDA_TRY(cudaStreamSynchronize(S->cap));
    stats_suspend(true);
    c->capturing = true;
    cudaError_t e = cudaStreamBeginCapture(S->cap, cudaStreamCaptureModeThreadLocal);
    copse_status st = e == cudaSuccess ? session_body(S.get(), S->cap) : COPSE_ECUDA;
    if (e != cudaSuccess) set_error(std::string("cudaStreamBeginCapture: ") + cudaGetErrorString(e));
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(S->cap, &g);
    c->capturing = false;
    stats_suspend(false);
    if (st != COPSE_OK) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return st;
    }
    if (e2 != cudaSuccess || !g) {
        set_error(std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e2));
        return COPSE_ECUDA;
    }
    S->graph = g;
    CUDA_TRY(cudaGraphInstantiate(&S->exec, g, 0));
    *out = S.release();
    return COPSE_OK;
}

extern "C" copse_status copse_session_create(copse_ctx *c, const copse_keys *keys, const copse_evk *evk,
                                             copse_model *m, size_t n_queries, copse_session **out) {
    return copse_session_create_batch(c, keys, evk, 1, &m, &n_queries, out);
}

extern "C" copse_status copse_session_run(copse_session *S, const uint32_t *feats, int feats_on_device,
                                          uint64_t seed, uint8_t *out_bits, int out_on_device, void *stream) {
    if (!S || (S->n_feats && !feats) || (S->n_bits && !out_bits)) { set_error("null argument"); return COPSE_EINVAL; }
    cudaStream_t s = as_stream(stream);
    if (!feats_on_device)
        for (const SessItem &it : S->items) {
            const uint32_t p = it.m->f.precision;
            for (size_t k = it.feat_off; k < it.feat_off + it.nq * it.m->f.n_features; k++)
                if (p < 32 && feats[k] >= (1u << p)) { set_error("feature value needs more bits than the precision"); return COPSE_EINVAL; }
        }
    if (S->n_feats)
        CUDA_TRY(cudaMemcpyAsync(S->d_feats, feats, S->n_feats * 4,
                                 feats_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    // pageable source: the copy is staged before this call returns, so `seed` may go out of scope
    CUDA_TRY(cudaMemcpyAsync(S->d_seed, &seed, 8, cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaGraphLaunch(S->exec, s));
    if (S->n_bits)
        CUDA_TRY(cudaMemcpyAsync(out_bits, S->d_bits, S->n_bits,
                                 out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    if (!out_on_device) CUDA_TRY(cudaStreamSynchronize(s));
    return COPSE_OK;
}

// Asynchronous launch for the server: features and bits may be pinned host or device
// memory (copies by unified addressing), values already validated, nothing synchronised.
copse_status session_launch(copse_session *S, const uint32_t *feats, uint64_t seed, uint8_t *bits, cudaStream_t s,
                            uint64_t *seed_slot) {
    if (S->n_feats) CUDA_TRY(cudaMemcpyAsync(S->d_feats, feats, S->n_feats * 4, cudaMemcpyDefault, s));
    *seed_slot = seed;  // pinned, owned by the caller and not reused before this launch completes
    CUDA_TRY(cudaMemcpyAsync(S->d_seed, seed_slot, 8, cudaMemcpyDefault, s));
    CUDA_TRY(cudaGraphLaunch(S->exec, s));
    if (S->n_bits) CUDA_TRY(cudaMemcpyAsync(bits, S->d_bits, S->n_bits, cudaMemcpyDefault, s));
    return COPSE_OK;
}

size_t session_queries(const copse_session *S) { return S->items.empty() ? 0 : S->items[0].nq; }

extern "C" void copse_session_destroy(copse_session *S) {
    if (!S) return;
    cudaDeviceSynchronize();
    delete S;
}
