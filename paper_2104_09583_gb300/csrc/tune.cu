// Autotuning of the schedule choices that have no single best value across
// workloads: the NTT kernel family (one cluster launch per transform or two
// tiled launches, for plain transforms and for those fused with base
// conversions), the baby-step sizes of the matrix products, and the number
// of key-switching digits.  Every candidate is run on the device and timed
// with CUDA events (median of the timed repetitions after a warm-up); the
// fastest is kept.  Built on the public entry points.
#include <algorithm>
#include <limits>
#include <vector>

#include "internal.cuh"

namespace {

float median(std::vector<float> v) {
    if (v.empty()) return -1.f;
    std::sort(v.begin(), v.end());
    return v[v.size() / 2];
}

// Feature values for timing runs: a fixed pseudo-random sequence below 2^precision.
std::vector<uint32_t> timing_features(const copse_model_info &info, size_t nq) {
    std::vector<uint32_t> f(std::max<size_t>(nq * info.n_features, 1));
    uint64_t x = 0x2545F4914F6CDD1Dull;
    const uint32_t mask = info.precision >= 32 ? 0xffffffffu : ((1u << info.precision) - 1u);
    for (auto &v : f) {
        x ^= x << 13;
        x ^= x >> 7;
        x ^= x << 17;
        v = (uint32_t)(x >> 20) & mask;
    }
    return f;
}

struct Handles {
    copse_keys *k = nullptr;
    copse_evk *e = nullptr;
    copse_ctbuf *f = nullptr;
    ~Handles() {
        copse_ctbuf_destroy(f);
        copse_keys_destroy(k);
        copse_evk_destroy(e);
    }
};

// One inference of the model's current plan on c with keys for that plan: stage
// times (median over reps after one warm-up) into st[4], their sum into *total.
copse_status time_model(copse_ctx *c, copse_model *m, size_t nq, int reps, float st[4], float *total) {
    copse_model_info info;
    STATUS_TRY(copse_model_info_get(m, &info));
    if (nq < 1) nq = 1;
    nq = std::min<size_t>(nq, (size_t)c->N / ((size_t)info.block * info.n_segments));
    Handles h;
    const copse_model *ms[1] = {m};
    STATUS_TRY(copse_keygen(c, 0x5eed, ms, 1, &h.k, &h.e));
    if (copse_model_is_encrypted(m)) STATUS_TRY(copse_encrypt_model(c, h.k, m, 0xe7c));
    const std::vector<uint32_t> feats = timing_features(info, nq);
    STATUS_TRY(copse_encrypt_features(c, h.k, m, feats.data(), nq, 0, 0x7a11, &h.f, nullptr));
    std::vector<float> per[4], tot;
    for (int r = 0; r <= reps; r++) {
        copse_ctbuf *out = nullptr;
        float ms4[4];
        STATUS_TRY(copse_infer_timed(c, h.e, m, h.f, &out, nullptr, ms4));
        copse_ctbuf_destroy(out);
        if (r == 0) continue;  // warm-up (first use uploads the model)
        float s = 0;
        for (int i = 0; i < 4; i++) {
            per[i].push_back(ms4[i]);
            s += ms4[i];
        }
        tot.push_back(s);
    }
    for (int i = 0; i < 4; i++) st[i] = median(per[i]);
    *total = median(tot);
    return COPSE_OK;
}

}  // namespace

extern "C" copse_status copse_tune_ntt(copse_ctx *c, const uint32_t *sizes, size_t n, int reps, float *ms_cluster,
                                       float *ms_tiled, uint32_t *max_cluster) {
    if (!c || !sizes || !ms_cluster || !ms_tiled || !max_cluster || n < 1 || reps < 1) {
        set_error("bad argument");
        return COPSE_EINVAL;
    }
    CUDA_TRY(cudaSetDevice(c->device));
    uint32_t umax = 0;
    for (size_t i = 0; i < n; i++) umax = std::max(umax, sizes[i]);
    if (umax < 1) { set_error("bad argument"); return COPSE_EINVAL; }
    const size_t words = (size_t)umax * c->N;
    u64 *buf = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    copse_status st = COPSE_OK;
    if (cudaMalloc(&buf, words * sizeof(u64)) != cudaSuccess) { set_error("cudaMalloc failed"); return COPSE_ENOMEM; }
    if (cudaMemset(buf, 0, words * sizeof(u64)) != cudaSuccess || cudaEventCreate(&a) != cudaSuccess ||
        cudaEventCreate(&b) != cudaSuccess) {
        set_error("CUDA set-up failed");
        st = COPSE_ECUDA;
    }
    const bool on = c->ntt_clusters;
    const long before = c->ntt_cluster_max;
    // forward + inverse of `sizes[i]` residue polynomials (first prime), each form
    for (size_t i = 0; i < n && st == COPSE_OK; i++) {
        for (int variant = 0; variant < 2 && st == COPSE_OK; variant++) {
            c->ntt_clusters = variant == 0;
            c->ntt_cluster_max = 1L << 30;
            std::vector<float> t;
            for (int r = 0; r <= reps && st == COPSE_OK; r++) {
                cudaEventRecord(a, 0);
                st = copse_ntt(c, buf, sizes[i], 1, 0, nullptr);
                if (st == COPSE_OK) st = copse_ntt(c, buf, sizes[i], 1, 1, nullptr);
                cudaEventRecord(b, 0);
                float x = 0;
                if (st == COPSE_OK &&
                    (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&x, a, b) != cudaSuccess)) {
                    set_error("NTT timing failed");
                    st = COPSE_ECUDA;
                }
                if (r > 0) t.push_back(x);
            }
            (variant == 0 ? ms_cluster : ms_tiled)[i] = median(t);
        }
    }
    c->ntt_clusters = on;
    if (st == COPSE_OK) {
        // the cluster form up to the largest timed size at which it is not slower
        std::vector<size_t> idx(n);
        for (size_t i = 0; i < n; i++) idx[i] = i;
        std::sort(idx.begin(), idx.end(), [&](size_t x, size_t y) { return sizes[x] < sizes[y]; });
        long lim = 0;
        bool tail_tiled = true;
        for (size_t k = n; k-- > 0;) {
            const size_t i = idx[k];
            if (ms_cluster[i] <= ms_tiled[i]) {
                lim = k + 1 == n ? (1L << 30) : (long)sizes[i];
                tail_tiled = false;
                break;
            }
        }
        if (tail_tiled) lim = 0;
        c->ntt_cluster_max = lim;
        *max_cluster = (uint32_t)std::min<long>(lim, 0xffffffffL);
    } else {
        c->ntt_cluster_max = before;
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    cudaFree(buf);
    return st;
}

extern "C" copse_status copse_tune_bsgs(copse_ctx *c, copse_model *m, const uint32_t *g_r, size_t n_r,
                                        const uint32_t *g_l, size_t n_l, size_t n_queries, int reps, float *ms_r,
                                        float *ms_l) {
    if (!c || !m || (n_r && (!g_r || !ms_r)) || (n_l && (!g_l || !ms_l)) || reps < 1) {
        set_error("bad argument");
        return COPSE_EINVAL;
    }
    CUDA_TRY(cudaSetDevice(c->device));
    uint32_t cur_r = 0, cur_l = 0;
    STATUS_TRY(copse_model_get_bsgs(m, &cur_r, &cur_l));
    const float inf = std::numeric_limits<float>::infinity();
    float st[4], tot;
    // reshuffle: time its stage for each candidate with the level plan held
    uint32_t best_r = cur_r;
    float best = inf;
    for (size_t i = 0; i < n_r; i++) {
        ms_r[i] = -1.f;
        if (copse_model_set_bsgs(m, g_r[i], cur_l) != COPSE_OK) continue;  // leaves the block: skipped
        STATUS_TRY(time_model(c, m, n_queries, reps, st, &tot));
        ms_r[i] = st[1];
        if (st[1] < best) {
            best = st[1];
            best_r = g_r[i];
        }
    }
    // levels: with the chosen reshuffle plan
    uint32_t best_l = cur_l;
    best = inf;
    for (size_t i = 0; i < n_l; i++) {
        ms_l[i] = -1.f;
        if (copse_model_set_bsgs(m, best_r, g_l[i]) != COPSE_OK) continue;
        STATUS_TRY(time_model(c, m, n_queries, reps, st, &tot));
        ms_l[i] = st[2];
        if (st[2] < best) {
            best = st[2];
            best_l = g_l[i];
        }
    }
    return copse_model_set_bsgs(m, best_r, best_l);
}

extern "C" copse_status copse_tune_dnum(const copse_params *base, int device, copse_model *m, const uint32_t *dnums,
                                        size_t n, size_t n_queries, int reps, float *ms, uint32_t *best) {
    if (!base || !m || !dnums || !ms || !best || n < 1 || reps < 1) {
        set_error("bad argument");
        return COPSE_EINVAL;
    }
    float bt = std::numeric_limits<float>::infinity();
    *best = base->dnum;
    for (size_t i = 0; i < n; i++) {
        ms[i] = -1.f;
        copse_params p = *base;
        p.dnum = dnums[i];
        copse_ctx *c = nullptr;
        if (copse_ctx_create(&p, device, &c) != COPSE_OK) continue;  // out of range: skipped
        float st[4], tot = -1.f;
        copse_status s = time_model(c, m, n_queries, reps, st, &tot);
        copse_ctx_destroy(c);
        if (s != COPSE_OK) return s;
        ms[i] = tot;
        if (tot < bt) {
            bt = tot;
            *best = dnums[i];
        }
    }
    return COPSE_OK;
}

extern "C" copse_status copse_ctx_set_ntt_cluster_max(copse_ctx *c, uint32_t max_cluster) {
    if (!c) { set_error("null context"); return COPSE_EINVAL; }
    c->ntt_cluster_max = max_cluster >= (1u << 30) ? (1L << 30) : (long)max_cluster;
    return COPSE_OK;
}

extern "C" copse_status copse_ctx_set_ntt_fused_max(copse_ctx *c, uint32_t max_fused) {
    if (!c) { set_error("null context"); return COPSE_EINVAL; }
    c->ntt_fused_max = max_fused >= (1u << 30) ? (1L << 30) : (long)max_fused;
    return COPSE_OK;
}

extern "C" copse_status copse_tune_fused(copse_ctx *c, copse_model *m, const uint32_t *cands, size_t n,
                                         size_t n_queries, int reps, float *ms, uint32_t *best) {
    if (!c || !m || !cands || !ms || !best || n < 1 || reps < 1) {
        set_error("bad argument");
        return COPSE_EINVAL;
    }
    const long before = c->ntt_fused_max;
    *best = (uint32_t)std::min<long>(before, 0xffffffffL);
    if (c->logN < 12 || c->logN > 14) {
        // no fused transform at this ring degree: nothing to choose
        for (size_t i = 0; i < n; i++) ms[i] = -1.f;
        return COPSE_OK;
    }
    CUDA_TRY(cudaSetDevice(c->device));
    float bt = std::numeric_limits<float>::infinity();
    long pick = before;
    for (size_t i = 0; i < n; i++) {
        c->ntt_fused_max = cands[i] >= (1u << 30) ? (1L << 30) : (long)cands[i];
        float st[4], tot = -1.f;
        const copse_status s = time_model(c, m, n_queries, reps, st, &tot);
        if (s != COPSE_OK) {
            c->ntt_fused_max = before;
            return s;
        }
        ms[i] = tot;
        if (tot < bt) {
            bt = tot;
            pick = c->ntt_fused_max;
        }
    }
    c->ntt_fused_max = pick;
    *best = (uint32_t)std::min<long>(pick, 0xffffffffL);
    return COPSE_OK;
}
