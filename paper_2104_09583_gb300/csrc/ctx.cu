// Context: prime chain, NTT twiddle tables, slot index table, base-conversion
// constants, error reporting and the device memory pool.
#include <atomic>
#include <algorithm>
#include <cstring>

#include "internal.cuh"

typedef unsigned __int128 u128;

// ---------------------------------------------------------------- errors
static thread_local std::string g_err = "no error";
void set_error(const std::string &msg) { g_err = msg; }
extern "C" const char *copse_last_error(void) { return g_err.c_str(); }

// ---------------------------------------------------------------- host number theory
static u64 h_mul(u64 a, u64 b, u64 m) { return (u64)((u128)a * b % m); }
static u64 h_pow(u64 a, u64 e, u64 m) {
    u64 r = 1 % m;
    a %= m;
    for (; e; e >>= 1, a = h_mul(a, a, m))
        if (e & 1) r = h_mul(r, a, m);
    return r;
}
static u64 h_inv(u64 a, u64 m) { return h_pow(a % m, m - 2, m); }  // m prime
static u64 h_shoup(u64 w, u64 q) { return (u64)(((u128)w << 64) / q); }
static Shoup mk_shoup(u64 w, u64 q) { return Shoup{w % q, h_shoup(w % q, q)}; }

// Miller-Rabin with the twelve smallest prime bases: exact below 3.3e24.
static bool h_is_prime(u64 n) {
    const u64 bases[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return false;
    for (u64 p : bases) {
        if (n % p == 0) return n == p;
    }
    u64 d = n - 1;
    int r = 0;
    while (!(d & 1)) d >>= 1, r++;
    for (u64 a : bases) {
        u64 x = h_pow(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool witness = true;
        for (int i = 1; i < r && witness; i++) {
            x = h_mul(x, x, n);
            if (x == n - 1) witness = false;
        }
        if (witness) return false;
    }
    return true;
}

// primitive 2N-th root of unity mod q (q = 1 mod 2N)
static u64 root_2n(u64 q, int logN) {
    u64 twoN = 2ull << logN;
    for (u64 x = 2;; x++) {
        u64 r = h_pow(x, (q - 1) / twoN, q);
        if (h_pow(r, twoN / 2, q) == q - 1) return r;
    }
}

static uint32_t h_brev(uint32_t x, int bits) {
    uint32_t r = 0;
    for (int i = 0; i < bits; i++) r |= ((x >> i) & 1u) << (bits - 1 - i);
    return r;
}

// ---------------------------------------------------------------- memory
copse_status dev_alloc(copse_ctx *ctx, void **p, size_t bytes, cudaStream_t s) {
    if (bytes == 0) bytes = 256;
    // inside a stream capture the allocation becomes a graph memory node, whose
    // memory the graph owns between launches
    cudaError_t e = ctx->capturing ? cudaMallocAsync(p, bytes, s) : cudaMallocFromPoolAsync(p, bytes, ctx->pool, s);
    if (e != cudaSuccess) {
        set_error(std::string("device allocation of ") + std::to_string(bytes) + " bytes: " + cudaGetErrorString(e));
        cudaGetLastError();
        return COPSE_ENOMEM;
    }
    return COPSE_OK;
}
void dev_free(void *p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

// ---------------------------------------------------------------- fork / join
// A lane is COPSE_SIDE_STREAMS fork streams plus one lane stream (index
// COPSE_SIDE_STREAMS) with an event each, and one fork event.  Independent
// inferences use different lanes so their forks never share a stream.
static constexpr int LANE_W = COPSE_SIDE_STREAMS + 1;

copse_status ensure_lanes(copse_ctx *c, int lanes) {
    if (lanes > COPSE_MAX_LANES) { set_error("too many lanes"); return COPSE_EINVAL; }
    while ((int)c->fork_ev.size() < lanes) {
        cudaEvent_t fe;
        CUDA_TRY(cudaEventCreateWithFlags(&fe, cudaEventDisableTiming));
        c->fork_ev.push_back(fe);
        for (int i = 0; i < LANE_W; i++) {
            cudaStream_t st;
            cudaEvent_t ev;
            CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
            CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
            c->side.push_back(st);
            c->side_done.push_back(ev);
        }
    }
    return COPSE_OK;
}

copse_status fork_begin(copse_ctx *c, cudaStream_t s, int n, int lane) {
    STATUS_TRY(ensure_lanes(c, lane + 1));
    CUDA_TRY(cudaEventRecord(c->fork_ev[lane], s));
    for (int i = 0; i < n && i < COPSE_SIDE_STREAMS; i++)
        CUDA_TRY(cudaStreamWaitEvent(c->side[lane * LANE_W + i], c->fork_ev[lane], 0));
    return COPSE_OK;
}

cudaStream_t fork_stream(copse_ctx *c, int i, int lane) { return c->side[lane * LANE_W + i % COPSE_SIDE_STREAMS]; }

copse_status fork_join(copse_ctx *c, cudaStream_t s, int n, int lane) {
    for (int i = 0; i < n && i < COPSE_SIDE_STREAMS; i++) {
        const int k = lane * LANE_W + i;
        CUDA_TRY(cudaEventRecord(c->side_done[k], c->side[k]));
        CUDA_TRY(cudaStreamWaitEvent(s, c->side_done[k], 0));
    }
    return COPSE_OK;
}

cudaStream_t lane_stream(copse_ctx *c, int lane) { return c->side[lane * LANE_W + COPSE_SIDE_STREAMS]; }
cudaEvent_t lane_event(copse_ctx *c, int lane) { return c->side_done[lane * LANE_W + COPSE_SIDE_STREAMS]; }

template <class T>
static copse_status upload(copse_ctx *ctx, T **dst, const std::vector<T> &src) {
    void *p = nullptr;
    CUDA_TRY(cudaMalloc(&p, std::max<size_t>(1, src.size()) * sizeof(T)));
    ctx->owned.push_back(p);
    if (!src.empty()) CUDA_TRY(cudaMemcpy(p, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
    *dst = (T *)p;
    return COPSE_OK;
}

// ---------------------------------------------------------------- context
static copse_status build_tables(copse_ctx *c) {
    const int N = c->N, NP = c->NP, L = c->L, A = c->alpha;
    c->hprime.resize(NP);
    std::vector<u64> psi((size_t)NP * N), psi_sh((size_t)NP * N), ipsi((size_t)NP * N), ipsi_sh((size_t)NP * N);
    for (int g = 0; g < NP; g++) {
        u64 q = c->primes[g];
        PrimeDev &P = c->hprime[g];
        memset(&P, 0, sizeof(P));
        P.q = q;
        int bits = 64 - __builtin_clzll(q);
        P.bits = (uint32_t)bits;
        P.mu = (u64)(((u128)1 << (2 * bits)) / q);
        P.ninv = h_inv((u64)N % q, q);
        P.ninv_sh = h_shoup(P.ninv, q);
        P.t_mod = c->t % q;
        P.t_mod_sh = h_shoup(P.t_mod, q);
        P.r64 = (u64)(((u128)1 << 64) % q);
        P.r64_sh = h_shoup(P.r64, q);
        P.one_sh = h_shoup(1, q);
        u64 inv = 1;  // q^-1 mod 2^64 by Newton's iteration (q odd)
        for (int i = 0; i < 6; i++) inv *= 2 - q * inv;
        P.qinv_neg = (u64)0 - inv;
        // The slot structure needs the canonical root zeta = 3^((t-1)/2N) mod t;
        // for the RNS primes any primitive 2N-th root gives the same coefficients.
        u64 root = (g == c->t_index()) ? h_pow(3, (q - 1) / (2ull * N), q) : root_2n(q, c->logN);
        u64 iroot = h_inv(root, q);
        for (int k = 0; k < N; k++) {
            uint32_t e = h_brev((uint32_t)k, c->logN);
            u64 w = h_pow(root, e, q), iw = h_pow(iroot, e, q);
            psi[(size_t)g * N + k] = w;
            psi_sh[(size_t)g * N + k] = h_shoup(w, q);
            ipsi[(size_t)g * N + k] = iw;
            ipsi_sh[(size_t)g * N + k] = h_shoup(iw, q);
        }
    }
    STATUS_TRY(upload(c, &c->d_prime, c->hprime));
    STATUS_TRY(upload(c, &c->d_psi, psi));
    STATUS_TRY(upload(c, &c->d_psi_sh, psi_sh));
    STATUS_TRY(upload(c, &c->d_ipsi, ipsi));
    STATUS_TRY(upload(c, &c->d_ipsi_sh, ipsi_sh));
    // slot s = (row, col) is the evaluation at zeta^e, e = 3^col (row 0) or -3^col
    // (row 1) mod 2N; the bit-reversed NTT holds exponent 2*brev(k)+1 at position k.
    std::vector<uint32_t> slot(N);
    u64 twoN = 2ull * N, p3 = 1;
    for (int col = 0; col < N / 2; col++) {
        u64 e0 = p3, e1 = twoN - p3;
        slot[col] = h_brev((uint32_t)((e0 - 1) / 2), c->logN);
        slot[N / 2 + col] = h_brev((uint32_t)((e1 - 1) / 2), c->logN);
        p3 = p3 * 3 % twoN;
    }
    STATUS_TRY(upload(c, &c->d_slot_index, slot));
    STATUS_TRY(upload(c, &c->d_status, std::vector<int>(1, 0)));

    // base conversion constants
    std::vector<Shoup> modup_inv((size_t)(L + 1) * L), modup_hat((size_t)(L + 1) * L * NP);
    std::vector<u64> modup_qhat((size_t)(L + 1) * L * NP);
    for (int ell = 1; ell <= L; ell++) {
        for (int i = 0; i < ell; i++) {
            int j = i / A, lo = j * A, hi = std::min((j + 1) * A, ell);
            u64 qi = c->primes[i];
            u64 h = 1;
            for (int k = lo; k < hi; k++)
                if (k != i) h = h_mul(h, c->primes[k] % qi, qi);
            modup_inv[(size_t)ell * L + i] = mk_shoup(h_inv(h, qi), qi);
            for (int g = 0; g < NP; g++) {
                u64 qg = c->primes[g];
                u64 hg = 1;
                for (int k = lo; k < hi; k++)
                    if (k != i) hg = h_mul(hg, c->primes[k] % qg, qg);
                modup_hat[((size_t)ell * L + i) * NP + g] = mk_shoup(hg, qg);
                modup_qhat[((size_t)ell * L + i) * NP + g] = h_mul(qi % qg, hg, qg);
            }
        }
    }
    std::vector<Shoup> md_inv(A), md_hat((size_t)A * L), md_Pinv(L);
    std::vector<u64> md_P(L);
    for (int k = 0; k < A; k++) {
        u64 pk = c->primes[L + k];
        u64 ph = 1;
        for (int m = 0; m < A; m++)
            if (m != k) ph = h_mul(ph, c->primes[L + m] % pk, pk);
        md_inv[k] = mk_shoup(h_mul(h_inv(c->t % pk, pk), h_inv(ph, pk), pk), pk);
        for (int i = 0; i < L; i++) {
            u64 qi = c->primes[i], phi = 1;
            for (int m = 0; m < A; m++)
                if (m != k) phi = h_mul(phi, c->primes[L + m] % qi, qi);
            md_hat[(size_t)k * L + i] = mk_shoup(phi, qi);
        }
    }
    for (int i = 0; i < L; i++) {
        u64 qi = c->primes[i], P = 1;
        for (int k = 0; k < A; k++) P = h_mul(P, c->primes[L + k] % qi, qi);
        md_P[i] = P;
        md_Pinv[i] = mk_shoup(h_inv(P, qi), qi);
    }
    std::vector<Shoup> ms_tinv(L + 1), ms_qinv((size_t)(L + 1) * L);
    for (int ell = 2; ell <= L; ell++) {
        u64 ql = c->primes[ell - 1];
        ms_tinv[ell] = mk_shoup(h_inv(c->t % ql, ql), ql);
        for (int i = 0; i < ell - 1; i++) ms_qinv[(size_t)ell * L + i] = mk_shoup(h_inv(ql % c->primes[i], c->primes[i]), c->primes[i]);
    }
    // ModDown over P q_{ell-1} (a relinearisation that also drops a prime): basis
    // b_0 = q_{ell-1}, b_k = p_{k-1}, B = their product
    const int nb = A + 1;
    std::vector<Shoup> mdd_inv((size_t)(L + 1) * nb), mdd_hat((size_t)(L + 1) * nb * L), mdd_Binv((size_t)(L + 1) * L);
    std::vector<u64> mdd_B((size_t)(L + 1) * L);
    for (int ell = 2; ell <= L; ell++) {
        std::vector<u64> bp(nb);
        bp[0] = c->primes[ell - 1];
        for (int k = 1; k < nb; k++) bp[k] = c->primes[L + k - 1];
        for (int k = 0; k < nb; k++) {
            const u64 bk = bp[k];
            u64 bh = 1;
            for (int m = 0; m < nb; m++)
                if (m != k) bh = h_mul(bh, bp[m] % bk, bk);
            mdd_inv[(size_t)ell * nb + k] = mk_shoup(h_mul(h_inv(c->t % bk, bk), h_inv(bh, bk), bk), bk);
            for (int i = 0; i < ell - 1; i++) {
                const u64 qi = c->primes[i];
                u64 bhi = 1;
                for (int m = 0; m < nb; m++)
                    if (m != k) bhi = h_mul(bhi, bp[m] % qi, qi);
                mdd_hat[((size_t)ell * nb + k) * L + i] = mk_shoup(bhi, qi);
            }
        }
        for (int i = 0; i < ell - 1; i++) {
            const u64 qi = c->primes[i];
            u64 B = 1;
            for (int k = 0; k < nb; k++) B = h_mul(B, bp[k] % qi, qi);
            mdd_B[(size_t)ell * L + i] = B;
            mdd_Binv[(size_t)ell * L + i] = mk_shoup(h_inv(B, qi), qi);
        }
    }
    // Montgomery forms of the conversion factors and of the negated corrections
    auto mont = [&](u64 x, int g) { return h_mul(x % c->primes[g], c->hprime[g].r64, c->primes[g]); };
    auto neg = [&](u64 x, int g) { const u64 q = c->primes[g], r = x % q; return r ? q - r : 0; };
    std::vector<u64> modup_hat_m(modup_hat.size()), modup_negq_m(modup_qhat.size());
    for (int ell = 1; ell <= L; ell++)
        for (int i = 0; i < ell; i++)
            for (int g = 0; g < NP; g++) {
                const size_t ti = ((size_t)ell * L + i) * NP + g;
                modup_hat_m[ti] = mont(modup_hat[ti].w, g);
                modup_negq_m[ti] = mont(neg(modup_qhat[ti], g), g);
            }
    std::vector<u64> md_hat_m(md_hat.size()), md_negP_m(L);
    for (int k = 0; k < A; k++)
        for (int i = 0; i < L; i++) md_hat_m[(size_t)k * L + i] = mont(md_hat[(size_t)k * L + i].w, i);
    for (int i = 0; i < L; i++) md_negP_m[i] = mont(neg(md_P[i], i), i);
    std::vector<u64> mdd_hat_m(mdd_hat.size()), mdd_negB_m(mdd_B.size());
    for (size_t x = 0; x < mdd_hat.size(); x++) mdd_hat_m[x] = mont(mdd_hat[x].w, (int)(x % L));
    for (size_t x = 0; x < mdd_B.size(); x++) mdd_negB_m[x] = mont(neg(mdd_B[x], (int)(x % L)), (int)(x % L));
    STATUS_TRY(upload(c, &c->ks.modup_hat_m, modup_hat_m));
    STATUS_TRY(upload(c, &c->ks.modup_negq_m, modup_negq_m));
    STATUS_TRY(upload(c, &c->ks.md_hat_m, md_hat_m));
    STATUS_TRY(upload(c, &c->ks.md_negP_m, md_negP_m));
    STATUS_TRY(upload(c, &c->ks.mdd_hat_m, mdd_hat_m));
    STATUS_TRY(upload(c, &c->ks.mdd_negB_m, mdd_negB_m));
    // first-step factors times N^-1: the scales of the inverse transforms feeding the conversions
    auto scaled = [&](const Shoup &f, int g) { return mk_shoup(h_mul(f.w, c->hprime[g].ninv, c->primes[g]), c->primes[g]); };
    std::vector<Shoup> mu_scale(modup_inv.size()), md_scale(A), ms_scale(L + 1), mdd_scale(mdd_inv.size());
    for (int ell = 1; ell <= L; ell++)
        for (int i = 0; i < ell; i++) mu_scale[(size_t)ell * L + i] = scaled(modup_inv[(size_t)ell * L + i], i);
    for (int k = 0; k < A; k++) md_scale[k] = scaled(md_inv[k], L + k);
    for (int ell = 2; ell <= L; ell++) {
        ms_scale[ell] = scaled(ms_tinv[ell], ell - 1);
        for (int k = 0; k < nb; k++)
            mdd_scale[(size_t)ell * nb + k] = scaled(mdd_inv[(size_t)ell * nb + k], k == 0 ? ell - 1 : L + k - 1);
    }
    STATUS_TRY(upload(c, &c->ks.mu_scale, mu_scale));
    STATUS_TRY(upload(c, &c->ks.md_scale, md_scale));
    STATUS_TRY(upload(c, &c->ks.ms_scale, ms_scale));
    STATUS_TRY(upload(c, &c->ks.mdd_scale, mdd_scale));
    STATUS_TRY(upload(c, &c->ks.mdd_inv, mdd_inv));
    STATUS_TRY(upload(c, &c->ks.mdd_hat, mdd_hat));
    STATUS_TRY(upload(c, &c->ks.mdd_B, mdd_B));
    STATUS_TRY(upload(c, &c->ks.mdd_Binv, mdd_Binv));
    STATUS_TRY(upload(c, &c->ks.modup_inv, modup_inv));
    STATUS_TRY(upload(c, &c->ks.modup_hat, modup_hat));
    STATUS_TRY(upload(c, &c->ks.modup_qhat, modup_qhat));
    STATUS_TRY(upload(c, &c->ks.md_inv, md_inv));
    STATUS_TRY(upload(c, &c->ks.md_hat, md_hat));
    STATUS_TRY(upload(c, &c->ks.md_P, md_P));
    STATUS_TRY(upload(c, &c->ks.md_Pinv, md_Pinv));
    STATUS_TRY(upload(c, &c->ks.ms_tinv, ms_tinv));
    STATUS_TRY(upload(c, &c->ks.ms_qinv, ms_qinv));
    return COPSE_OK;
}

extern "C" copse_status copse_ctx_create(const copse_params *pp, int device, copse_ctx **out) {
    if (!pp || !out) { set_error("null argument"); return COPSE_EINVAL; }
    *out = nullptr;
    if (pp->log_n < 4 || pp->log_n > 15 || pp->prime_bits < 36 || pp->prime_bits > 55 || pp->n_primes < 1 ||
        pp->n_primes > 40 || pp->dnum < 1 || pp->dnum > pp->n_primes) {
        set_error("copse_params out of range");
        return COPSE_EINVAL;
    }
    copse_ctx *c = new copse_ctx();
    static std::atomic<uint64_t> next_serial{1};
    c->serial = next_serial++;
    c->device = device;
    c->logN = (int)pp->log_n;
    c->N = 1 << c->logN;
    c->L = (int)pp->n_primes;
    c->dnum = (int)pp->dnum;
    c->alpha = (c->L + c->dnum - 1) / c->dnum;
    c->ndig = (c->L + c->alpha - 1) / c->alpha;
    c->bits = (int)pp->prime_bits;
    c->NP = c->L + c->alpha + 1;
    const char *nc = getenv("COPSE_NTT_CLUSTERS");
    c->ntt_clusters = !(nc && nc[0] == '0');
    // primes k*2N*t + 1 below 2^bits, k scanned downward: ciphertext primes first
    u64 M = (2ull << c->logN) * c->t;
    u64 k = ((1ull << c->bits) - 2) / M;
    while ((int)c->primes.size() < c->L + c->alpha && k > 0) {
        u64 p = k * M + 1;
        if (h_is_prime(p)) c->primes.push_back(p);
        k--;
    }
    if ((int)c->primes.size() < c->L + c->alpha) {
        set_error("not enough primes of the requested size");
        delete c;
        return COPSE_EINVAL;
    }
    c->primes.push_back(c->t);
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) {
        set_error(std::string("cudaSetDevice: ") + cudaGetErrorString(e));
        delete c;
        return COPSE_ECUDA;
    }
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    e = cudaMemPoolCreate(&c->pool, &props);
    if (e == cudaSuccess) {
        u64 keep = ~0ull;
        e = cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    if (e != cudaSuccess) {
        set_error(std::string("memory pool: ") + cudaGetErrorString(e));
        delete c;
        return COPSE_ECUDA;
    }
    copse_status st = build_tables(c);
    if (st == COPSE_OK) st = ntt_stage_tables(c);
    if (st != COPSE_OK) {
        copse_ctx_destroy(c);
        return st;
    }
    *out = c;
    return COPSE_OK;
}

extern "C" void copse_ctx_destroy(copse_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    for (cudaStream_t st : c->side) cudaStreamDestroy(st);
    for (cudaEvent_t ev : c->side_done) cudaEventDestroy(ev);
    for (cudaEvent_t ev : c->fork_ev) cudaEventDestroy(ev);
    for (void *p : c->owned) cudaFree(p);
    if (c->pool) cudaMemPoolDestroy(c->pool);
    delete c;
}

extern "C" copse_status copse_ctx_device_status(copse_ctx *c, int *status) {
    if (!c || !status) { set_error("null argument"); return COPSE_EINVAL; }
    CUDA_TRY(cudaSetDevice(c->device));
    CUDA_TRY(cudaDeviceSynchronize());
    int v = 0;
    CUDA_TRY(cudaMemcpy(&v, c->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemset(c->d_status, 0, sizeof(int)));
    *status = v;
    if (v) {
        set_error("a kernel's bounded wait ran out (device status " + std::to_string(v) + ")");
        return COPSE_ETIMEOUT;
    }
    return COPSE_OK;
}

extern "C" copse_status copse_ctx_primes(const copse_ctx *c, uint64_t *out, size_t cap, size_t *count) {
    if (!c) { set_error("null context"); return COPSE_EINVAL; }
    size_t n = (size_t)(c->L + c->alpha);
    if (count) *count = n;
    if (out) {
        if (cap < n) { set_error("buffer too small"); return COPSE_EINVAL; }
        for (size_t i = 0; i < n; i++) out[i] = c->primes[i];
    }
    return COPSE_OK;
}
