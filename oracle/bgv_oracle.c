/*
 * CPU oracle for the BGV ring layer underneath COPSE secure forest inference.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the GPU library computes.  Only the test-suite, the smoke
 * check and the benchmark's CPU-baseline leg may load it; the product library
 * never links, includes or calls anything here, and nothing here is shared
 * with the CUDA sources.
 *
 * The COPSE paper (Malik et al., PLDI'21) runs its vectorised primitives on
 * BGV as provided by HElib (Section 5, "COPSE Runtime"; operation list of
 * Section 6: Encrypt, Rotate, Add, Multiply, Constant Add).  It does not
 * specify the ring, the key-switching variant or the modulus-switching policy,
 * so this oracle fixes one canonical reading:
 *
 *   ring      R_Q = Z_Q[X]/(X^N+1), Q a product of primes q = 1 (mod 2N*t)
 *   plaintext t = 65537, N slots (2 rows of N/2), slot values kept in {0,1}
 *   keys      ternary s; pk = (-a*s + t*e, a)
 *   switching hybrid key switching, digits of alpha primes, alpha special
 *             primes P; ModUp by fast base conversion with centred digits;
 *             ModDown by P with a t-multiple correction
 *   modswitch drop the last prime, t-multiple correction (q = 1 mod t keeps m)
 *
 * Everything is kept in coefficient form (residues in [0,q), layout
 * [component][prime][coefficient]); a polynomial product is the negacyclic
 * convolution, computed by the convolution theorem with a textbook
 * radix-2 NTT (pinned against the schoolbook product by the tests).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef uint64_t u64;
typedef int64_t i64;
typedef unsigned __int128 u128;

#define OR_MAXP 64

/* Parameter block shared with the Python wrapper (ctypes Structure). */
typedef struct {
    int32_t logN;
    int32_t N;
    u64 t;
    int32_t L;      /* ciphertext primes q_0..q_{L-1}                    */
    int32_t alpha;  /* special primes p_0..p_{alpha-1} (stored at L..)   */
    int32_t ndig;   /* key-switching digits at the top level = ceil(L/alpha) */
    int32_t pad;
    u64 primes[OR_MAXP]; /* q_0..q_{L-1}, p_0..p_{alpha-1} */
} or_params;

/* ------------------------------------------------------------------ */
/* Modular arithmetic on residues below 2^63 (128-bit products).       */
/* ------------------------------------------------------------------ */
static u64 mulmod(u64 a, u64 b, u64 q) { return (u64)(((u128)a * b) % q); }
static u64 addmod(u64 a, u64 b, u64 q) { u64 s = a + b; return s >= q ? s - q : s; }
static u64 submod(u64 a, u64 b, u64 q) { return a >= b ? a - b : a + (q - b); }
static u64 powmod(u64 a, u64 e, u64 q)
{
    u64 r = 1 % q;
    a %= q;
    while (e) {
        if (e & 1) r = mulmod(r, a, q);
        a = mulmod(a, a, q);
        e >>= 1;
    }
    return r;
}
static u64 invmod(u64 a, u64 q) { return powmod(a, q - 2, q); } /* q prime */
static u64 from_signed(i64 v, u64 q)
{
    i64 r = v % (i64)q;
    return r < 0 ? (u64)(r + (i64)q) : (u64)r;
}
/* centred representative of x in [0,q): (-q/2, q/2] for odd q */
static i64 centred(u64 x, u64 q) { return x > (q - 1) / 2 ? (i64)x - (i64)q : (i64)x; }

u64 or_mulmod(u64 a, u64 b, u64 q) { return mulmod(a, b, q); }
u64 or_powmod(u64 a, u64 e, u64 q) { return powmod(a, e, q); }

/* Threads the oracle's loops over residues and coefficients run on (OpenMP when
 * built with it; every thread computes whole, independent residues or
 * coefficients, so results do not depend on the count). */
int or_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Set that thread count for the calling thread's later calls (n > 0; the benchmark
 * times the oracle on one thread and on all host cores); returns the count in force. */
int or_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* Deterministic Miller-Rabin for 64-bit inputs (first twelve prime bases). */
int or_is_prime(u64 n)
{
    static const u64 bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return 0;
    for (int i = 0; i < 12; i++) {
        if (n == bases[i]) return 1;
        if (n % bases[i] == 0) return 0;
    }
    u64 d = n - 1;
    int s = 0;
    while ((d & 1) == 0) { d >>= 1; s++; }
    for (int i = 0; i < 12; i++) {
        u64 x = powmod(bases[i], d, n);
        if (x == 1 || x == n - 1) continue;
        int comp = 1;
        for (int r = 1; r < s; r++) {
            x = mulmod(x, x, n);
            if (x == n - 1) { comp = 0; break; }
        }
        if (comp) return 0;
    }
    return 1;
}

/* Primes k*2N*t + 1 below 2^bits, scanning k downward; returns how many. */
int or_find_primes(int logN, u64 t, int bits, int count, u64 *out)
{
    u64 M = ((u64)2 << logN) * t;
    u64 top = (bits >= 64) ? ~(u64)0 : (((u64)1 << bits) - 2);
    u64 k = top / M;
    int found = 0;
    while (found < count && k > 0) {
        u64 p = k * M + 1;
        if (or_is_prime(p)) out[found++] = p;
        k--;
    }
    return found;
}

/* Primitive 2N-th root of unity mod q: g^((q-1)/2N) for the least g >= 2
 * whose power has order exactly 2N (psi^N = -1). */
u64 or_root_2n(u64 q, int logN)
{
    u64 twoN = (u64)2 << logN;
    for (u64 g = 2; g < q; g++) {
        u64 psi = powmod(g, (q - 1) / twoN, q);
        if (powmod(psi, twoN >> 1, q) == q - 1) return psi;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Negacyclic NTT, natural order: A[i] = a(psi^(2i+1)).                */
/* ------------------------------------------------------------------ */
static void bit_reverse(u64 *a, int logN)
{
    int N = 1 << logN;
    for (int i = 0, j = 0; i < N; i++) {
        if (i < j) { u64 tmp = a[i]; a[i] = a[j]; a[j] = tmp; }
        int bit = N >> 1;
        while (j & bit) { j ^= bit; bit >>= 1; }
        j |= bit;
    }
}

/* cyclic DFT of length N with root w (textbook iterative Cooley-Tukey) */
static void dft(u64 *a, int logN, u64 q, u64 w)
{
    int N = 1 << logN;
    bit_reverse(a, logN);
    for (int len = 2; len <= N; len <<= 1) {
        u64 wl = powmod(w, (u64)(N / len), q);
        for (int i = 0; i < N; i += len) {
            u64 x = 1;
            for (int j = 0; j < len / 2; j++) {
                u64 u = a[i + j];
                u64 v = mulmod(a[i + j + len / 2], x, q);
                a[i + j] = addmod(u, v, q);
                a[i + j + len / 2] = submod(u, v, q);
                x = mulmod(x, wl, q);
            }
        }
    }
}

void or_ntt_fwd(u64 *a, int logN, u64 q, u64 psi)
{
    int N = 1 << logN;
    u64 x = 1;
    for (int j = 0; j < N; j++) { a[j] = mulmod(a[j], x, q); x = mulmod(x, psi, q); }
    dft(a, logN, q, mulmod(psi, psi, q));
}

void or_ntt_inv(u64 *a, int logN, u64 q, u64 psi)
{
    int N = 1 << logN;
    u64 psi_inv = invmod(psi, q);
    dft(a, logN, q, mulmod(psi_inv, psi_inv, q));
    u64 ninv = invmod((u64)N % q, q);
    u64 x = ninv;
    for (int j = 0; j < N; j++) { a[j] = mulmod(a[j], x, q); x = mulmod(x, psi_inv, q); }
}

/* direct evaluation at psi^(2i+1), O(N^2): the definition the NTT computes */
void or_eval_direct(const u64 *a, int logN, u64 q, u64 psi, u64 *out)
{
    int N = 1 << logN;
    for (int i = 0; i < N; i++) {
        u64 x = powmod(psi, (u64)(2 * i + 1), q), acc = 0, p = 1;
        for (int j = 0; j < N; j++) { acc = addmod(acc, mulmod(a[j], p, q), q); p = mulmod(p, x, q); }
        out[i] = acc;
    }
}

/* schoolbook product in Z_q[X]/(X^N+1) */
void or_negacyclic_schoolbook(const u64 *a, const u64 *b, int logN, u64 q, u64 *out)
{
    int N = 1 << logN;
    for (int k = 0; k < N; k++) out[k] = 0;
    for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++) {
            u64 p = mulmod(a[i], b[j], q);
            int k = i + j;
            if (k < N) out[k] = addmod(out[k], p, q);
            else out[k - N] = submod(out[k - N], p, q);
        }
}

/* product in Z_q[X]/(X^N+1) by the convolution theorem */
void or_negacyclic_mul(const u64 *a, const u64 *b, int logN, u64 q, u64 *out)
{
    int N = 1 << logN;
    u64 psi = or_root_2n(q, logN);
    u64 *fa = malloc(sizeof(u64) * N), *fb = malloc(sizeof(u64) * N);
    memcpy(fa, a, sizeof(u64) * N);
    memcpy(fb, b, sizeof(u64) * N);
    or_ntt_fwd(fa, logN, q, psi);
    or_ntt_fwd(fb, logN, q, psi);
    for (int i = 0; i < N; i++) out[i] = mulmod(fa[i], fb[i], q);
    or_ntt_inv(out, logN, q, psi);
    free(fa);
    free(fb);
}

/* ------------------------------------------------------------------ */
/* Plaintext slots mod t.                                               */
/* Slot s = r*(N/2) + c holds m(zeta^e), zeta = 3^((t-1)/2N) mod t,     */
/* e = 3^c mod 2N for row r = 0 and e = -3^c mod 2N for row r = 1.      */
/* X -> X^(3^k) then moves slot (r, c+k) to (r, c): a left rotation.    */
/* ------------------------------------------------------------------ */
void or_slot_exponents(int logN, u64 *e)
{
    int N = 1 << logN;
    u64 twoN = (u64)2 * N, g = 1;
    for (int c = 0; c < N / 2; c++) {
        e[c] = g;
        e[N / 2 + c] = twoN - g;
        g = (g * 3) % twoN;
    }
}

static u64 slot_root(int logN, u64 t) { return powmod(3, (t - 1) / ((u64)2 << logN), t); }

void or_encode(const u64 *slots, int logN, u64 t, u64 *coeffs)
{
    int N = 1 << logN;
    u64 *e = malloc(sizeof(u64) * N);
    or_slot_exponents(logN, e);
    for (int s = 0; s < N; s++) coeffs[(e[s] - 1) / 2] = slots[s] % t;
    or_ntt_inv(coeffs, logN, t, slot_root(logN, t));
    free(e);
}

void or_decode(const u64 *coeffs, int logN, u64 t, u64 *slots)
{
    int N = 1 << logN;
    u64 *e = malloc(sizeof(u64) * N), *a = malloc(sizeof(u64) * N);
    or_slot_exponents(logN, e);
    for (int j = 0; j < N; j++) a[j] = coeffs[j] % t;
    or_ntt_fwd(a, logN, t, slot_root(logN, t));
    for (int s = 0; s < N; s++) slots[s] = a[(e[s] - 1) / 2];
    free(e);
    free(a);
}

/* ------------------------------------------------------------------ */
/* Counter-based randomness: SplitMix64 (Steele, Lea, Flood, OOPSLA'14) */
/* word(seed, stream, idx) = output number stream*2^40+idx+1 of the    */
/* SplitMix64 sequence started at state `seed`.                         */
/* ------------------------------------------------------------------ */
u64 or_word(u64 seed, u64 stream, u64 idx)
{
    u64 z = seed + 0x9E3779B97F4A7C15ULL * ((stream << 40) + idx + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

void or_sample_ternary(u64 seed, u64 stream, int N, i64 *out)
{
    for (int j = 0; j < N; j++) out[j] = (i64)(or_word(seed, stream, (u64)j) % 3) - 1;
}

/* centred binomial with eta = 21: popcount of 21 bits minus popcount of the next 21 */
void or_sample_cbd(u64 seed, u64 stream, int N, i64 *out)
{
    for (int j = 0; j < N; j++) {
        u64 w = or_word(seed, stream, (u64)j);
        out[j] = (i64)__builtin_popcountll(w & 0x1FFFFFULL) - (i64)__builtin_popcountll((w >> 21) & 0x1FFFFFULL);
    }
}

/* uniform residue mod q for global prime index r: (hi*2^64 + lo) mod q */
static u64 uniform_residue(u64 seed, u64 stream, int N, int r, int j, u64 q)
{
    u64 idx = 2 * ((u64)r * (u64)N + (u64)j);
    u64 hi = or_word(seed, stream, idx), lo = or_word(seed, stream, idx + 1);
    return (u64)((((u128)hi << 64) | lo) % q);
}

/* ------------------------------------------------------------------ */
/* BGV helpers.  A "basis" is a list of global prime indices; level ell */
/* uses q_0..q_{ell-1}; the extended basis appends p_0..p_{alpha-1}.    */
/* ------------------------------------------------------------------ */
static int ext_prime(const or_params *P, int ell, int r) { return r < ell ? r : P->L + (r - ell); }

static void poly_mul_acc(const u64 *a, const u64 *b, int logN, u64 q, u64 *acc)
{
    int N = 1 << logN;
    u64 *tmp = malloc(sizeof(u64) * N);
    or_negacyclic_mul(a, b, logN, q, tmp);
    for (int i = 0; i < N; i++) acc[i] = addmod(acc[i], tmp[i], q);
    free(tmp);
}

/* a(X) -> a(X^g) in Z_q[X]/(X^N+1), g odd */
void or_automorphism(const u64 *a, int logN, u64 q, u64 g, u64 *out)
{
    int N = 1 << logN;
    u64 twoN = (u64)2 * N;
    for (int j = 0; j < N; j++) {
        u64 k = ((u64)j * g) % twoN;
        if (k < (u64)N) out[k] = a[j];
        else out[k - N] = a[j] ? q - a[j] : 0;
    }
}

/* secret key: ternary, stream 1 */
void or_keygen_secret(const or_params *P, u64 seed, i64 *s) { or_sample_ternary(seed, 1, P->N, s); }

/* public key (-a*s + t*e, a) mod q_r for r < L; a from stream 2, e from stream 3 */
void or_keygen_public(const or_params *P, u64 seed, const i64 *s, u64 *pk)
{
    int N = P->N, L = P->L;
    i64 *e = malloc(sizeof(i64) * N);
    u64 *a = malloc(sizeof(u64) * N), *sr = malloc(sizeof(u64) * N), *as = malloc(sizeof(u64) * N);
    or_sample_cbd(seed, 3, N, e);
    for (int r = 0; r < L; r++) {
        u64 q = P->primes[r];
        for (int j = 0; j < N; j++) { a[j] = uniform_residue(seed, 2, N, r, j, q); sr[j] = from_signed(s[j], q); }
        or_negacyclic_mul(a, sr, P->logN, q, as);
        for (int j = 0; j < N; j++) {
            u64 te = mulmod(P->t % q, from_signed(e[j], q), q);
            pk[(size_t)r * N + j] = addmod(submod(0, as[j], q), te, q);
            pk[(size_t)(L + r) * N + j] = a[j];
        }
    }
    free(e); free(a); free(sr); free(as);
}

/* Switching key from s' to s: for digit j (primes [j*alpha, min((j+1)*alpha,L))):
 *   ksk_j = (-a_j*s + t*e_j + g_j*s', a_j) over all L+alpha primes,
 *   g_j = P mod q_r on the digit's primes, 0 elsewhere (P = prod p_k);
 *   a_j from stream sb+2j, e_j from stream sb+2j+1.
 * s_from: residues of s' for every global prime, [L+alpha][N].
 * ksk layout: [ndig][2][L+alpha][N]. */
void or_keygen_switch(const or_params *P, u64 seed, u64 sb, const i64 *s, const u64 *s_from, u64 *ksk)
{
    int N = P->N, L = P->L, nb = P->L + P->alpha;
    i64 *e = malloc(sizeof(i64) * N);
    for (int j = 0; j < P->ndig; j++) {
        or_sample_cbd(seed, sb + 2 * j + 1, N, e);
        int lo = j * P->alpha, hi = (j + 1) * P->alpha < L ? (j + 1) * P->alpha : L;
#pragma omp parallel for schedule(dynamic)
        for (int r = 0; r < nb; r++) {
            u64 *a = malloc(sizeof(u64) * N), *sr = malloc(sizeof(u64) * N), *as = malloc(sizeof(u64) * N);
            u64 q = P->primes[r];
            u64 Pmod = 1;
            for (int k = 0; k < P->alpha; k++) Pmod = mulmod(Pmod, P->primes[L + k] % q, q);
            u64 gj = (r >= lo && r < hi) ? Pmod : 0;
            for (int x = 0; x < N; x++) { a[x] = uniform_residue(seed, sb + 2 * j, N, r, x, q); sr[x] = from_signed(s[x], q); }
            or_negacyclic_mul(a, sr, P->logN, q, as);
            u64 *k0 = ksk + ((size_t)(j * 2 + 0) * nb + r) * N;
            u64 *k1 = ksk + ((size_t)(j * 2 + 1) * nb + r) * N;
            for (int x = 0; x < N; x++) {
                u64 v = submod(0, as[x], q);
                v = addmod(v, mulmod(P->t % q, from_signed(e[x], q), q), q);
                v = addmod(v, mulmod(gj, s_from[(size_t)r * N + x], q), q);
                k0[x] = v;
                k1[x] = a[x];
            }
            free(a); free(sr); free(as);
        }
    }
    free(e);
}

/* Encrypt centred plaintext coefficients m at the top level L:
 * u ternary (stream sb), e0, e1 centred binomial (sb+1, sb+2);
 * c0 = pk0*u + t*e0 + m, c1 = pk1*u + t*e1.  ct layout [2][L][N]. */
void or_encrypt(const or_params *P, const u64 *pk, const i64 *m, u64 seed, u64 sb, u64 *ct)
{
    int N = P->N, L = P->L;
    i64 *u = malloc(sizeof(i64) * N), *e0 = malloc(sizeof(i64) * N), *e1 = malloc(sizeof(i64) * N);
    or_sample_ternary(seed, sb, N, u);
    or_sample_cbd(seed, sb + 1, N, e0);
    or_sample_cbd(seed, sb + 2, N, e1);
#pragma omp parallel for schedule(dynamic)
    for (int r = 0; r < L; r++) {
        u64 q = P->primes[r], tq = P->t % q;
        u64 *urr = malloc(sizeof(u64) * N), *p0 = malloc(sizeof(u64) * N), *p1 = malloc(sizeof(u64) * N);
        for (int j = 0; j < N; j++) urr[j] = from_signed(u[j], q);
        or_negacyclic_mul(pk + (size_t)r * N, urr, P->logN, q, p0);
        or_negacyclic_mul(pk + (size_t)(L + r) * N, urr, P->logN, q, p1);
        for (int j = 0; j < N; j++) {
            ct[(size_t)r * N + j] = addmod(addmod(p0[j], mulmod(tq, from_signed(e0[j], q), q), q), from_signed(m[j], q), q);
            ct[(size_t)(L + r) * N + j] = addmod(p1[j], mulmod(tq, from_signed(e1[j], q), q), q);
        }
        free(urr); free(p0); free(p1);
    }
    free(u); free(e0); free(e1);
}

/* Secret-key encryption at level ell (the model owner holds the secret key
 * when the model is encrypted, Section 8.3 "Maurice = Diane"), with a seeded
 * mask: the evaluations of a at psi_r^(2j+1), j = 0..N-1 in natural order,
 * are uniform residues from stream sb (so a can be regenerated from the seed
 * in evaluation form); e centred binomial from stream sb+1;
 *   c1 = a,  c0 = -a*s + t*e + m.   ct layout [2][ell][N], coefficient form. */
void or_encrypt_sk(const or_params *P, const i64 *s, const i64 *m, u64 seed, u64 sb, int ell, u64 *ct)
{
    int N = P->N;
    i64 *e = malloc(sizeof(i64) * N);
    or_sample_cbd(seed, sb + 1, N, e);
#pragma omp parallel for schedule(dynamic)
    for (int r = 0; r < ell; r++) {
        u64 *a = malloc(sizeof(u64) * N), *sr = malloc(sizeof(u64) * N), *as = malloc(sizeof(u64) * N);
        u64 q = P->primes[r], tq = P->t % q;
        for (int j = 0; j < N; j++) a[j] = uniform_residue(seed, sb, N, r, j, q);
        or_ntt_inv(a, P->logN, q, or_root_2n(q, P->logN));
        for (int j = 0; j < N; j++) sr[j] = from_signed(s[j], q);
        or_negacyclic_mul(a, sr, P->logN, q, as);
        for (int j = 0; j < N; j++) {
            u64 v = addmod(mulmod(tq, from_signed(e[j], q), q), from_signed(m[j], q), q);
            ct[(size_t)r * N + j] = submod(v, as[j], q);
            ct[(size_t)(ell + r) * N + j] = a[j];
        }
        free(a); free(sr); free(as);
    }
    free(e);
}

/* [c0 + c1*s] mod q_r for r < ell (no reduction mod t): used for noise measurement */
void or_decrypt_raw(const or_params *P, const i64 *s, const u64 *ct, int ell, u64 *x)
{
    int N = P->N;
    u64 *sr = malloc(sizeof(u64) * N);
    for (int r = 0; r < ell; r++) {
        u64 q = P->primes[r];
        for (int j = 0; j < N; j++) sr[j] = from_signed(s[j], q);
        memcpy(x + (size_t)r * N, ct + (size_t)r * N, sizeof(u64) * N);
        poly_mul_acc(ct + (size_t)(ell + r) * N, sr, P->logN, q, x + (size_t)r * N);
    }
    free(sr);
}

/* Drop the last prime ql = q_{ell-1} from each of ncomp components:
 *   w = [c * t^-1]_ql (centred),  c'_i = (c_i - t*w) * ql^-1  mod q_i.
 * in: [ncomp][ell][N]; out: [ncomp][ell-1][N]. */
void or_modswitch(const or_params *P, const u64 *ct, int ncomp, int ell, u64 *out)
{
    int N = P->N;
    u64 ql = P->primes[ell - 1], tinv = invmod(P->t % ql, ql);
#pragma omp parallel for collapse(2) schedule(static)
    for (int c = 0; c < ncomp; c++)
        for (int j = 0; j < N; j++) {
            i64 w = centred(mulmod(ct[((size_t)c * ell + ell - 1) * N + j], tinv, ql), ql);
            for (int i = 0; i < ell - 1; i++) {
                u64 q = P->primes[i];
                u64 d = mulmod(P->t % q, from_signed(w, q), q);
                u64 v = submod(ct[((size_t)c * ell + i) * N + j], d, q);
                out[((size_t)c * (ell - 1) + i) * N + j] = mulmod(v, invmod(ql % q, q), q);
            }
        }
}

/* ModUp of digit j of x (x: [ell][N] coefficient residues at level ell) to the
 * extended basis {q_0..q_{ell-1}, p_0..p_{alpha-1}}:
 *   y_i = [x_i * Qhat_i^-1]_{q_i} centred, value mod r = sum_i y_i * (Qhat_i mod r),
 * Qhat_i = prod of the digit's other primes; the digit's own primes are copied. */
static void modup_digit(const or_params *P, const u64 *x, int ell, int j, u64 *y)
{
    int N = P->N, nx = ell + P->alpha;
    int lo = j * P->alpha, hi = (j + 1) * P->alpha < ell ? (j + 1) * P->alpha : ell;
#pragma omp parallel for schedule(static)
    for (int n = 0; n < N; n++) {
        i64 yc[OR_MAXP];
        for (int i = lo; i < hi; i++) {
            u64 qi = P->primes[i], qhat = 1;
            for (int k = lo; k < hi; k++) if (k != i) qhat = mulmod(qhat, P->primes[k] % qi, qi);
            yc[i - lo] = centred(mulmod(x[(size_t)i * N + n], invmod(qhat, qi), qi), qi);
        }
        for (int r = 0; r < nx; r++) {
            int g = ext_prime(P, ell, r);
            u64 qr = P->primes[g];
            if (g >= lo && g < hi) { y[(size_t)r * N + n] = x[(size_t)g * N + n]; continue; }
            u64 acc = 0;
            for (int i = lo; i < hi; i++) {
                u64 qhat = 1;
                for (int k = lo; k < hi; k++) if (k != i) qhat = mulmod(qhat, P->primes[k] % qr, qr);
                acc = addmod(acc, mulmod(from_signed(yc[i - lo], qr), qhat, qr), qr);
            }
            y[(size_t)r * N + n] = acc;
        }
    }
}

/* ModDown of u over the extended basis to level ell:
 *   y_k = [u_k * t^-1 * Phat_k^-1]_{p_k} centred,  W = sum_k y_k * Phat_k  (so W = u/t mod P),
 *   out_i = (u_i - t*W) * P^-1  mod q_i. */
static void moddown(const or_params *P, const u64 *u, int ell, u64 *out)
{
    int N = P->N, A = P->alpha, L = P->L;
#pragma omp parallel for schedule(static)
    for (int n = 0; n < N; n++) {
        i64 yc[OR_MAXP];
        for (int k = 0; k < A; k++) {
            u64 pk = P->primes[L + k], phat = 1;
            for (int m = 0; m < A; m++) if (m != k) phat = mulmod(phat, P->primes[L + m] % pk, pk);
            u64 v = mulmod(u[(size_t)(ell + k) * N + n], invmod(P->t % pk, pk), pk);
            yc[k] = centred(mulmod(v, invmod(phat, pk), pk), pk);
        }
        for (int i = 0; i < ell; i++) {
            u64 q = P->primes[i], W = 0, Pinv = 1;
            for (int k = 0; k < A; k++) {
                u64 phat = 1;
                for (int m = 0; m < A; m++) if (m != k) phat = mulmod(phat, P->primes[L + m] % q, q);
                W = addmod(W, mulmod(from_signed(yc[k], q), phat, q), q);
                Pinv = mulmod(Pinv, P->primes[L + k] % q, q);
            }
            Pinv = invmod(Pinv, q);
            u64 v = submod(u[(size_t)i * N + n], mulmod(P->t % q, W, q), q);
            out[(size_t)i * N + n] = mulmod(v, Pinv, q);
        }
    }
}

/* The key-switching sum before ModDown: over the ceil(ell/alpha) active digits,
 * acc_c = sum_j ModUp(digit j of x) * ksk_j[c] over the extended basis.
 * x: [ell][N] coefficient form; ksk: [ndig][2][L+alpha][N]; acc: [2][ell+alpha][N]. */
static void keyswitch_raw(const or_params *P, const u64 *x, int ell, const u64 *ksk, u64 *acc)
{
    int N = P->N, nx = ell + P->alpha, nb = P->L + P->alpha;
    int nd = (ell + P->alpha - 1) / P->alpha;
    u64 *y = malloc(sizeof(u64) * nx * N);
    memset(acc, 0, sizeof(u64) * 2 * nx * N);
    for (int j = 0; j < nd; j++) {
        modup_digit(P, x, ell, j, y);
#pragma omp parallel for collapse(2) schedule(dynamic)
        for (int c = 0; c < 2; c++)
            for (int r = 0; r < nx; r++) {
                int g = ext_prime(P, ell, r);
                const u64 *k = ksk + ((size_t)(j * 2 + c) * nb + g) * N;
                poly_mul_acc(y + (size_t)r * N, k, P->logN, P->primes[g], acc + ((size_t)c * nx + r) * N);
            }
    }
    free(y);
}

/* Hybrid key switching of x ([ell][N], coefficient form) with ksk
 * ([ndig][2][L+alpha][N]): the raw sum above, then ModDown.  out: [2][ell][N]. */
void or_keyswitch(const or_params *P, const u64 *x, int ell, const u64 *ksk, u64 *out)
{
    int N = P->N, nx = ell + P->alpha;
    u64 *acc = malloc(sizeof(u64) * 2 * nx * N);
    keyswitch_raw(P, x, ell, ksk, acc);
    moddown(P, acc, ell, out);
    moddown(P, acc + (size_t)nx * N, ell, out + (size_t)ell * N);
    free(acc);
}

/* Diagonal matrix-vector products sharing the rotations of one ciphertext
 * (the MatMul of Section 4.1.2: sum over diagonals of d_k * rot(v, k)), with
 * the modulus-down step of key switching applied once to each sum:
 *   for a rotation with Galois element g != 1,
 *     R_g = KSraw(tau_g c1) + (P * tau_g c0, 0)      over q_0..q_{ell-1}, p_0..p_{alpha-1}
 *   acc_a = sum_{g != 1} pt[a][g] * R_g,   out_a = ModDown(acc_a) + pt[a][1] * (c0, c1).
 * R_g is P times the rotated ciphertext (up to key-switching noise), so the
 * result decrypts to the sum of products, with one rounding error per sum.
 * ct: [2][ell][N]; galois[k], gks[k] ([ndig][2][L+alpha][N]) for k < nrot;
 * pts: [nacc][nrot][N] centred plaintext coefficients, present[a*nrot+k] = 0
 * for a zero diagonal; out: [nacc][2][ell][N].  No modulus switch here. */
void or_matmul(const or_params *P, const u64 *ct, int ell, int nrot, const u64 *galois, const u64 *const *gks,
               int nacc, const i64 *pts, const int *present, u64 *out)
{
    int N = P->N, nx = ell + P->alpha;
    u64 Pmod[OR_MAXP];
    for (int i = 0; i < ell; i++) {
        Pmod[i] = 1;
        for (int k = 0; k < P->alpha; k++) Pmod[i] = mulmod(Pmod[i], P->primes[P->L + k] % P->primes[i], P->primes[i]);
    }
    u64 *acc = calloc((size_t)nacc * 2 * nx * N, sizeof(u64));
    u64 *tc = malloc(sizeof(u64) * 2 * ell * N), *R = malloc(sizeof(u64) * 2 * nx * N);
    u64 *pr = malloc(sizeof(u64) * N), *tmp = malloc(sizeof(u64) * N);
    for (int k = 0; k < nrot; k++) {
        u64 g = galois[k];
        if (g == 1) continue;
        int used = 0;
        for (int a = 0; a < nacc; a++) used |= present[a * nrot + k];
        if (!used) continue;
        for (int c = 0; c < 2; c++)
            for (int r = 0; r < ell; r++)
                or_automorphism(ct + ((size_t)c * ell + r) * N, P->logN, P->primes[r], g, tc + ((size_t)c * ell + r) * N);
        keyswitch_raw(P, tc + (size_t)ell * N, ell, gks[k], R);
        for (int r = 0; r < ell; r++) {
            u64 q = P->primes[r];
            for (int j = 0; j < N; j++)
                R[(size_t)r * N + j] = addmod(R[(size_t)r * N + j], mulmod(Pmod[r], tc[(size_t)r * N + j], q), q);
        }
        for (int a = 0; a < nacc; a++) {
            if (!present[a * nrot + k]) continue;
            const i64 *m = pts + ((size_t)a * nrot + k) * N;
#pragma omp parallel for collapse(2) schedule(dynamic)
            for (int c = 0; c < 2; c++)
                for (int r = 0; r < nx; r++) {
                    int gi = ext_prime(P, ell, r);
                    u64 q = P->primes[gi];
                    u64 *prr = malloc(sizeof(u64) * N);
                    for (int j = 0; j < N; j++) prr[j] = from_signed(m[j], q);
                    poly_mul_acc(R + ((size_t)c * nx + r) * N, prr, P->logN, q, acc + (((size_t)a * 2 + c) * nx + r) * N);
                    free(prr);
                }
        }
    }
    for (int a = 0; a < nacc; a++) {
        u64 *o = out + (size_t)a * 2 * ell * N;
        u64 *ac = acc + (size_t)a * 2 * nx * N;
        moddown(P, ac, ell, o);
        moddown(P, ac + (size_t)nx * N, ell, o + (size_t)ell * N);
        for (int k = 0; k < nrot; k++) {
            if (galois[k] != 1 || !present[a * nrot + k]) continue;
            const i64 *m = pts + ((size_t)a * nrot + k) * N;
            for (int r = 0; r < ell; r++) {
                u64 q = P->primes[r];
                for (int j = 0; j < N; j++) pr[j] = from_signed(m[j], q);
                for (int c = 0; c < 2; c++) {
                    or_negacyclic_mul(ct + ((size_t)c * ell + r) * N, pr, P->logN, q, tmp);
                    u64 *d = o + ((size_t)c * ell + r) * N;
                    for (int j = 0; j < N; j++) d[j] = addmod(d[j], tmp[j], q);
                }
            }
        }
    }
    free(acc); free(tc); free(R); free(pr); free(tmp);
}

/* Sum of rotations of several ciphertexts (the giant steps of a baby-step /
 * giant-step matrix product), with the modulus-down step taken once:
 *   acc = sum_{k: g_k != 1} KSraw(tau_{g_k} c_k1) + (P * tau_{g_k} c_k0, 0)   over q and p
 *   out = ModDown(acc) + sum_{k: g_k = 1} c_k.
 * Each rotated term is P times the rotation of c_k up to key-switching noise,
 * so out decrypts to sum_k rot(c_k) with one rounding error for the sum.
 * cts: n ciphertexts [2][ell][N] (pointers); galois[k], gks[k] as in or_matmul;
 * out: [2][ell][N].  No modulus switch here. */
void or_rotsum(const or_params *P, const u64 *const *cts, int ell, int n, const u64 *galois, const u64 *const *gks,
               u64 *out)
{
    int N = P->N, nx = ell + P->alpha;
    u64 Pmod[OR_MAXP];
    for (int i = 0; i < ell; i++) {
        Pmod[i] = 1;
        for (int k = 0; k < P->alpha; k++) Pmod[i] = mulmod(Pmod[i], P->primes[P->L + k] % P->primes[i], P->primes[i]);
    }
    u64 *acc = calloc((size_t)2 * nx * N, sizeof(u64));
    u64 *tc = malloc(sizeof(u64) * 2 * ell * N), *R = malloc(sizeof(u64) * 2 * nx * N);
    for (int k = 0; k < n; k++) {
        u64 g = galois[k];
        if (g == 1) continue;
        const u64 *ct = cts[k];
        for (int c = 0; c < 2; c++)
            for (int r = 0; r < ell; r++)
                or_automorphism(ct + ((size_t)c * ell + r) * N, P->logN, P->primes[r], g, tc + ((size_t)c * ell + r) * N);
        keyswitch_raw(P, tc + (size_t)ell * N, ell, gks[k], R);
        for (int r = 0; r < ell; r++) {
            u64 q = P->primes[r];
            for (int j = 0; j < N; j++)
                R[(size_t)r * N + j] = addmod(R[(size_t)r * N + j], mulmod(Pmod[r], tc[(size_t)r * N + j], q), q);
        }
        for (int c = 0; c < 2; c++)
            for (int r = 0; r < nx; r++) {
                u64 q = P->primes[ext_prime(P, ell, r)];
                u64 *a = acc + ((size_t)c * nx + r) * N;
                const u64 *b = R + ((size_t)c * nx + r) * N;
                for (int j = 0; j < N; j++) a[j] = addmod(a[j], b[j], q);
            }
    }
    moddown(P, acc, ell, out);
    moddown(P, acc + (size_t)nx * N, ell, out + (size_t)ell * N);
    for (int k = 0; k < n; k++) {
        if (galois[k] != 1) continue;
        for (int c = 0; c < 2; c++)
            for (int r = 0; r < ell; r++) {
                u64 q = P->primes[r];
                u64 *d = out + ((size_t)c * ell + r) * N;
                const u64 *b = cts[k] + ((size_t)c * ell + r) * N;
                for (int j = 0; j < N; j++) d[j] = addmod(d[j], b[j], q);
            }
    }
    free(acc); free(tc); free(R);
}

/* (c0,c1) x (d0,d1) -> (c0d0, c0d1 + c1d0, c1d1), out [3][ell][N] */
void or_tensor(const or_params *P, const u64 *a, const u64 *b, int ell, u64 *out)
{
    int N = P->N;
    memset(out, 0, sizeof(u64) * 3 * ell * N);
#pragma omp parallel for schedule(dynamic)
    for (int r = 0; r < ell; r++) {
        u64 q = P->primes[r];
        const u64 *a0 = a + (size_t)r * N, *a1 = a + (size_t)(ell + r) * N;
        const u64 *b0 = b + (size_t)r * N, *b1 = b + (size_t)(ell + r) * N;
        poly_mul_acc(a0, b0, P->logN, q, out + (size_t)r * N);
        poly_mul_acc(a0, b1, P->logN, q, out + (size_t)(ell + r) * N);
        poly_mul_acc(a1, b0, P->logN, q, out + (size_t)(ell + r) * N);
        poly_mul_acc(a1, b1, P->logN, q, out + (size_t)(2 * ell + r) * N);
    }
}

/* relinearise a 3-component ciphertext: (d0, d1) + KS(d2, rlk) */
void or_relin(const or_params *P, const u64 *ct3, int ell, const u64 *rlk, u64 *out)
{
    int N = P->N;
    u64 *ks = malloc(sizeof(u64) * 2 * ell * N);
    or_keyswitch(P, ct3 + (size_t)2 * ell * N, ell, rlk, ks);
    for (int c = 0; c < 2; c++)
        for (int r = 0; r < ell; r++) {
            u64 q = P->primes[r];
            for (int j = 0; j < N; j++) {
                size_t o = ((size_t)c * ell + r) * N + j;
                out[o] = addmod(ct3[o], ks[o], q);
            }
        }
    free(ks);
}

/* ModDown over P and the ciphertext prime q_{ell-1} together: u over
 * {q_0..q_{ell-1}, p_0..p_{alpha-1}} -> out over q_0..q_{ell-2}, dividing by
 * B = q_{ell-1} P with the t-multiple correction (fast base conversion with
 * centred digits over the basis b_0 = q_{ell-1}, b_k = p_{k-1}):
 *   y_k = [u_{b_k} t^-1 (B/b_k)^-1]_{b_k} centred,  W = sum_k y_k (B/b_k),
 *   out_i = (u_i - t W) B^-1 mod q_i   (i < ell - 1). */
static void moddown_drop(const or_params *P, const u64 *u, int ell, u64 *out)
{
    int N = P->N, A = P->alpha, L = P->L, nb = A + 1;
    u64 bp[OR_MAXP];
    int bres[OR_MAXP];
    bp[0] = P->primes[ell - 1];
    bres[0] = ell - 1;
    for (int k = 1; k < nb; k++) { bp[k] = P->primes[L + k - 1]; bres[k] = ell + k - 1; }
#pragma omp parallel for schedule(static)
    for (int n = 0; n < N; n++) {
        i64 yc[OR_MAXP];
        for (int k = 0; k < nb; k++) {
            u64 bk = bp[k], bhat = 1;
            for (int m = 0; m < nb; m++) if (m != k) bhat = mulmod(bhat, bp[m] % bk, bk);
            u64 v = mulmod(u[(size_t)bres[k] * N + n], invmod(P->t % bk, bk), bk);
            yc[k] = centred(mulmod(v, invmod(bhat, bk), bk), bk);
        }
        for (int i = 0; i < ell - 1; i++) {
            u64 q = P->primes[i], W = 0, B = 1;
            for (int k = 0; k < nb; k++) {
                u64 bhat = 1;
                for (int m = 0; m < nb; m++) if (m != k) bhat = mulmod(bhat, bp[m] % q, q);
                W = addmod(W, mulmod(from_signed(yc[k], q), bhat, q), q);
                B = mulmod(B, bp[k] % q, q);
            }
            u64 v = submod(u[(size_t)i * N + n], mulmod(P->t % q, W, q), q);
            out[(size_t)i * N + n] = mulmod(v, invmod(B, q), q);
        }
    }
}

/* Relinearise a 3-component ciphertext and drop one prime in one ModDown:
 * acc = KSraw(d2) + (P d0, P d1) over q_0..q_{ell-1}, p_0..p_{alpha-1} (P times
 * the relinearised ciphertext up to key-switching noise), then
 * out = ModDown over P q_{ell-1} (moddown_drop): the relinearised product at level
 * ell - 1 with one rounding.  out: [2][ell-1][N]. */
void or_relin_drop(const or_params *P, const u64 *ct3, int ell, const u64 *rlk, u64 *out)
{
    int N = P->N, nx = ell + P->alpha;
    u64 *acc = malloc(sizeof(u64) * 2 * nx * N);
    keyswitch_raw(P, ct3 + (size_t)2 * ell * N, ell, rlk, acc);
    for (int c = 0; c < 2; c++)
        for (int r = 0; r < ell; r++) {
            u64 q = P->primes[r], Pm = 1;
            for (int k = 0; k < P->alpha; k++) Pm = mulmod(Pm, P->primes[P->L + k] % q, q);
            u64 *a = acc + ((size_t)c * nx + r) * N;
            const u64 *d = ct3 + ((size_t)c * ell + r) * N;
            for (int j = 0; j < N; j++) a[j] = addmod(a[j], mulmod(Pm, d[j], q), q);
        }
    moddown_drop(P, acc, ell, out);
    moddown_drop(P, acc + (size_t)nx * N, ell, out + (size_t)(ell - 1) * N);
    free(acc);
}

/* rotation by Galois element g: (tau_g c0 + ks0, ks1) with (ks0, ks1) = KS(tau_g c1, gk) */
void or_rotate(const or_params *P, const u64 *ct, int ell, u64 g, const u64 *gk, u64 *out)
{
    int N = P->N;
    u64 *tc = malloc(sizeof(u64) * 2 * ell * N);
    for (int c = 0; c < 2; c++)
        for (int r = 0; r < ell; r++)
            or_automorphism(ct + ((size_t)c * ell + r) * N, P->logN, P->primes[r], g, tc + ((size_t)c * ell + r) * N);
    or_keyswitch(P, tc + (size_t)ell * N, ell, gk, out);
    for (int r = 0; r < ell; r++) {
        u64 q = P->primes[r];
        for (int j = 0; j < N; j++) out[(size_t)r * N + j] = addmod(out[(size_t)r * N + j], tc[(size_t)r * N + j], q);
    }
    free(tc);
}

/* ct (ncomp components) times a plaintext with centred coefficients m */
void or_mul_plain(const or_params *P, const u64 *ct, int ncomp, int ell, const i64 *m, u64 *out)
{
    int N = P->N;
    u64 *mr = malloc(sizeof(u64) * N);
    for (int r = 0; r < ell; r++) {
        u64 q = P->primes[r];
        for (int j = 0; j < N; j++) mr[j] = from_signed(m[j], q);
        for (int c = 0; c < ncomp; c++)
            or_negacyclic_mul(ct + ((size_t)c * ell + r) * N, mr, P->logN, q, out + ((size_t)c * ell + r) * N);
    }
    free(mr);
}

/* c0 += m (centred plaintext coefficients) */
void or_add_plain(const or_params *P, u64 *ct, int ell, const i64 *m)
{
    int N = P->N;
    for (int r = 0; r < ell; r++) {
        u64 q = P->primes[r];
        for (int j = 0; j < N; j++) ct[(size_t)r * N + j] = addmod(ct[(size_t)r * N + j], from_signed(m[j], q), q);
    }
}

/* out = a + sign*b over n residue polynomials whose primes are q_{r mod ell} */
void or_add(const or_params *P, const u64 *a, const u64 *b, int ncomp, int ell, int negate, u64 *out)
{
    int N = P->N;
    for (int c = 0; c < ncomp; c++)
        for (int r = 0; r < ell; r++) {
            u64 q = P->primes[r];
            for (int j = 0; j < N; j++) {
                size_t o = ((size_t)c * ell + r) * N + j;
                out[o] = negate ? submod(a[o], b[o], q) : addmod(a[o], b[o], q);
            }
        }
}

/* Decrypt: modswitch down to level 1, then m = [[c0 + c1*s]_{q_0}]_t, output in [0,t). */
void or_decrypt(const or_params *P, const i64 *s, const u64 *ct, int ell, u64 *m)
{
    int N = P->N;
    u64 *cur = malloc(sizeof(u64) * 2 * ell * N), *nxt = malloc(sizeof(u64) * 2 * ell * N);
    memcpy(cur, ct, sizeof(u64) * 2 * ell * N);
    for (int l = ell; l > 1; l--) {
        or_modswitch(P, cur, 2, l, nxt);
        u64 *tmp = cur; cur = nxt; nxt = tmp;
    }
    u64 *x = malloc(sizeof(u64) * N);
    or_decrypt_raw(P, s, cur, 1, x);
    u64 q0 = P->primes[0];
    for (int j = 0; j < N; j++) m[j] = from_signed(centred(x[j], q0), P->t);
    free(cur); free(nxt); free(x);
}
