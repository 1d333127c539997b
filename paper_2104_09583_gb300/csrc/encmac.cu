// Encrypted-model multiply-accumulate on the fifth-generation tensor cores (tcgen05).
//
// The contraction.  The products of an encrypted matrix with a query ciphertext by the
// baby-step / giant-step diagonal method (Section 4.3, Algorithm 1, with the diagonals
// encrypted: Section 8.3) sum, per accumulator x and slot element e, the ciphertext x
// ciphertext products of diagonal (x, j) with rotation j of the query ciphertext.  For one
// element and one component pair that is a dense matrix product
//   D[x][b] = sum_j d[x][j] R[j][b]          (x: accumulators, j: baby steps, b: queries)
// of residues mod q.  Every element has its own matrices, so the GEMMs are batched over
// the elements, one at a time per CTA.
//
// Exactness.  A residue v < q < 2^55 is written in eight base-256 digits,
// v = sum_{i<8} s_i 256^i: with w = v + C, C = 0x0080808080808080 (128 in bytes 0-6),
// s_i = byte i of w minus 128 for i < 7 (in [-128, 127]) and s_7 = byte 7 of w, which is 0
// or 1 (w < 2^55 + C < 2^57; it is 1 for the top 1/256 of the residues of a prime near
// 2^55).  A digit is exact in fp16 and the product of two digits is at most 2^14 in
// magnitude, so the f32 accumulator of the MMA holds a sum of up to 256 such products
// exactly (|sum| <= 2^22).  The diagonals' digits sit in the M dimension (row 8 x + a for
// digit a of accumulator x) and the rotations' digits in the N dimension (column
// 8 (2 b + c) + a' for digit a' of component c of query b), so the accumulator holds, for
// every digit pair (a, a'), the exact partial sum D_aa' = sum_j s_a(d[x][j]) s_a'(R_c[j][b]),
// and the product sum is sum_aa' D_aa' 256^(a + a'): rebuilt in 128-bit integers and
// reduced mod q once.
//
// One CTA per SM, persistent over work items (element, accumulator tile of 16, run of up
// to 256 baby steps).  Per item the CTA writes the digits of both components of its
// diagonals (c0 read element-major, c1 regenerated from its seed) into shared memory once
// and then, for each pass of 16 query ciphertexts, streams the digits of the rotations
// through a ring of stages (cp.async prefetch of the raw words, digit conversion, one
// elected thread issuing two M 128 x N 256 x K 16 MMAs per stage into the two accumulators
// d0 x [R0 | R1] and d1 x [R0 | R1] of 256 TMEM columns each).  After the pass the eight
// warps read the accumulators back (tcgen05.ld), rebuild the three outputs
// (d0 R0, d0 R1 + d1 R0, d1 R1) exactly, reduce them and add them to acc.
//
// Every wait on an MMA completion is bounded by the global timer: a wait that runs out sets
// COPSE_DEV_MAC_WAIT in the context's device status word, and the CTA stops taking work,
// waits (bounded) for its issued MMAs, releases its tensor memory and exits.
#include <algorithm>
#include <atomic>

#include "internal.cuh"

namespace {

constexpr int TC_THREADS = 256;  // 8 warps
constexpr int TC_MX = 16;        // accumulators per tile: 16 x 8 digit rows = M 128
constexpr int TC_QP = 16;        // query ciphertexts per pass: 16 x 2 components x 8 digits = N 256
constexpr int TC_KR = 256;       // baby steps per run: exact f32 partial sums
constexpr int TC_KS = 16;        // baby steps per MMA (K of kind::f16)
constexpr int TC_NST = 4;        // digit stages of the rotations
constexpr int TC_NRAW = 4;       // raw stages (prefetch distance + 1)
constexpr int TC_TMEM_COLS = 512;
constexpr unsigned long long TC_WAIT_NS = 2000000000ull;  // 2 s per wait

constexpr uint32_t A_SET = TC_MX * 8 * TC_KR * 2;        // digits of one diagonal component: 64 KB
constexpr uint32_t B_STAGE = TC_QP * 2 * 8 * TC_KS * 2;  // digits of one chunk of rotations: 8 KB
constexpr uint32_t RAW_STAGE = TC_QP * TC_KS * 2 * 8;    // raw words of one chunk: 4 KB
constexpr uint32_t OFF_A0 = 0, OFF_A1 = A_SET, OFF_B = 2 * A_SET, OFF_RAW = OFF_B + TC_NST * B_STAGE,
                   OFF_TAB = OFF_RAW + TC_NRAW * RAW_STAGE, OFF_BAR = OFF_TAB + TC_MX * TC_KR * 4,
                   OFF_MISC = OFF_BAR + (TC_NST + 2) * 8, SMEM_TC = OFF_MISC + 16;
static_assert(RAW_STAGE == TC_THREADS * 16, "one 16-byte raw copy per thread and chunk");
static_assert(SMEM_TC <= 227 * 1024, "shared memory");

// kind::f16 instruction descriptor: f32 accumulator (bits 4-5 = 1), f16 A and B (formats 0),
// A and B MN-major (bits 15, 16), N / 8 at bit 17, M / 16 at bit 24
constexpr uint32_t idesc_f16(int M, int N) {
    return (1u << 4) | (1u << 15) | (1u << 16) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
constexpr uint32_t IDESC = idesc_f16(128, TC_QP * 2 * 8);

__device__ __forceinline__ uint32_t sh_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor without swizzle: core matrices of 8 rows x 16 bytes, the
// leading byte offset (bits 16-29) between core matrices adjacent in K, the stride byte
// offset (bits 32-45) between core matrices adjacent in M / N, version 1 at bit 46.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t k_stride, uint32_t mn_stride) {
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)((k_stride & 0x3FFFF) >> 4) << 16) |
           ((uint64_t)((mn_stride & 0x3FFFF) >> 4) << 32) | (1ull << 46);
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(IDESC), "r"(accumulate)
        : "memory");
}
// the barrier completes a phase once every MMA this thread issued before has completed
__device__ __forceinline__ void tc_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(sh_addr(bar))
                 : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void bar_init(uint64_t *bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sh_addr(bar)) : "memory");
}
__device__ __forceinline__ bool bar_test(uint64_t *bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(sh_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
// wait for the completion of the phase with this parity, at most TC_WAIT_NS; false (and the
// CTA's failure flag and the device status set) when the wait ran out or another thread's did
__device__ bool bar_wait(uint64_t *bar, uint32_t parity, volatile int *fail, int *status) {
    unsigned long long t0 = 0;
    for (int it = 0;; it++) {
        if (bar_test(bar, parity)) return true;
        if (*fail) return false;
        if (it == 0) {
            t0 = global_ns();
        } else if (global_ns() - t0 > TC_WAIT_NS) {
            *fail = 1;
            atomicOr(status, COPSE_DEV_MAC_WAIT);
            return false;
        }
    }
}

__device__ __forceinline__ uint32_t hsub2(uint32_t a, uint32_t b) {
    uint32_t d;
    asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
// The eight base-256 digits of v < 2^55 as eight fp16 (digit i in half i): byte i of
// v + 0x0080808080808080 with 0x64 above it is the fp16 of 1024 + byte, less 1152 = 1024 + 128
// for bytes 0-6 and less 1024 for byte 7 (0 or 1).
__device__ __forceinline__ uint4 digits8(u64 v) {
    const u64 w = v + 0x0080808080808080ull;
    const uint32_t lo = (uint32_t)w, hi = (uint32_t)(w >> 32);
    constexpr uint32_t C = 0x64806480u, C7 = 0x64006480u;  // (1152, 1152), (1152 low, 1024 high)
    uint4 r;
    r.x = hsub2(__byte_perm(lo, 0x64u, 0x4140), C);
    r.y = hsub2(__byte_perm(lo, 0x64u, 0x4342), C);
    r.z = hsub2(__byte_perm(hi, 0x64u, 0x4140), C);
    r.w = hsub2(__byte_perm(hi, 0x64u, 0x4342), C7);
    return r;
}
// an integer-valued f32 in [-2^22, 2^22] (its bits) as an int: x + 1.5 2^23 lies in
// [2^23, 2^24], where the f32 spacing is 1, so the sum is exact and its bits are linear in x
__device__ __forceinline__ int f32_int(uint32_t bits) {
    return __float_as_int(__uint_as_float(bits) + 12582912.0f) - 0x4B400000;
}

using u128 = unsigned __int128;
__device__ __forceinline__ u128 shfl_xor_u128(u128 v, int m) {
    const u64 lo = __shfl_xor_sync(0xffffffffu, (u64)v, m), hi = __shfl_xor_sync(0xffffffffu, (u64)(v >> 64), m);
    return ((u128)hi << 64) | lo;
}

struct TcArgs {
    const u64 *mac;       // [n_el][nm][nb] diagonals' c0
    const uint32_t *idx;  // [nm][nb] model ciphertext index (mask stream), ~0u = none
    const u64 *R;         // [n_el][nq][nb][2] rotations
    u64 *acc;             // [nq][nm][3][n_el], added to
    size_t a_ct;          // words per query ciphertext in acc
    int nm, nb, nq, ell, logN, n_mt, n_kr;
    u64 seed;
    const PrimeDev *pr;
    int *status;
};

__global__ void __launch_bounds__(TC_THREADS, 1) k_enc_mac_tc(const TcArgs P) {
    extern __shared__ __align__(1024) uint8_t sm[];
    uint8_t *A0 = sm + OFF_A0, *A1 = sm + OFF_A1, *Bst = sm + OFF_B, *Raw = sm + OFF_RAW;
    uint32_t *tab = (uint32_t *)(sm + OFF_TAB);
    uint64_t *bar = (uint64_t *)(sm + OFF_BAR);  // [0, NST) stages, NST: pass, NST + 1: final drain
    uint32_t *tslot = (uint32_t *)(sm + OFF_MISC);
    volatile int *fail = (volatile int *)(sm + OFF_MISC + 4);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const size_t n_el = (size_t)P.ell << P.logN;
    const uint32_t nmask = (1u << P.logN) - 1;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sh_addr(tslot)),
                     "r"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i < TC_NST + 2; i++) bar_init(&bar[i]);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *fail = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    const int nqp = (P.nq + TC_QP - 1) / TC_QP;
    const size_t n_items = (size_t)P.n_mt * P.n_kr * n_el;
    uint32_t gchunk = 0, npass = 0;  // chunks and passes of this CTA so far (barrier phases)
    int cur_mk = -1;                 // (tile, run) whose index table is in shared memory
    bool issued = false;             // MMAs issued (the final drain waits for them)
    for (size_t it = blockIdx.x; it < n_items; it += gridDim.x) {
        const int mk = (int)(it / n_el);
        const size_t e = it - (size_t)mk * n_el;
        const int mt = mk / P.n_kr, kr = mk - mt * P.n_kr;
        const int x0 = mt * TC_MX, nx = min(TC_MX, P.nm - x0);
        const int j0 = kr * TC_KR, nj = min(TC_KR, P.nb - j0), nk = (nj + TC_KS - 1) / TC_KS, nj16 = nk * TC_KS;
        const uint32_t a_mn = (uint32_t)nj16 * 16;  // bytes between accumulators' core-matrix rows
        const int r = (int)(e >> P.logN);
        const PrimeDev pd = P.pr[r];
        const uint32_t pos = (uint32_t)(e & nmask);
        const int nchunks = nqp * nk;

        // raw rotations of chunk c (pass c / nk, baby steps of MMA c % nk) of this item: thread
        // t copies (R0, R1) of query t / 16 and baby step t % 16
        auto issue = [&](int c) {
            uint8_t *dst = Raw + ((gchunk + (uint32_t)c) % TC_NRAW) * RAW_STAGE + tid * 16;
            if (c < nchunks) {
                const int qp = c / nk, ks = c - qp * nk;
                const int q = qp * TC_QP + (tid >> 4), j = ks * TC_KS + (tid & 15);
                if (q < P.nq && j < nj)
                    cp_async16(dst, P.R + (((e * P.nq + q) * P.nb + j0 + j) << 1));
                else
                    *(uint4 *)dst = make_uint4(0, 0, 0, 0);
            }
            cp_async_commit();
        };
        for (int c = 0; c < TC_NRAW - 1; c++) issue(c);

        if (mk != cur_mk) {
            __syncthreads();  // the previous table's readers are done
            for (int i = tid; i < TC_MX * TC_KR; i += TC_THREADS) {
                const int x = i / TC_KR, j = i - x * TC_KR;
                tab[i] = (x < nx && j < nj) ? P.idx[(size_t)(x0 + x) * P.nb + j0 + j] : ~0u;
            }
            cur_mk = mk;
            __syncthreads();
        }
        // digits of both components of every (accumulator, baby step) of the item: the 16 bytes
        // of accumulator x at baby step j are row j % 8 of core matrix (x, j / 8)
        for (int i = tid; i < TC_MX * nj16; i += TC_THREADS) {
            const int x = i / nj16, j = i - x * nj16;
            const uint32_t id = tab[x * TC_KR + j];
            u64 d0 = 0, d1 = 0;
            if (id != ~0u) {
                d0 = P.mac[(e * P.nm + x0 + x) * P.nb + j0 + j];
                d1 = seeded_mask(P.seed, MODEL_STREAM + 2ull * id, r, pos, P.logN, pd);
            }
            const uint32_t off = (uint32_t)x * a_mn + (uint32_t)(j >> 3) * 128 + (uint32_t)(j & 7) * 16;
            *(uint4 *)(A0 + off) = digits8(d0);
            *(uint4 *)(A1 + off) = digits8(d1);
        }
        fence_async_smem();
        __syncthreads();

        bool ok = true;
        for (int qp = 0; qp < nqp && ok; qp++) {
            for (int ks = 0; ks < nk; ks++) {
                const int c = qp * nk + ks;
                const uint32_t g = gchunk + (uint32_t)c;
                const int st = (int)(g % TC_NST);
                // stage st is free once the MMAs of chunk g - NST have completed
                if (g >= TC_NST) bar_wait(&bar[st], ((g / TC_NST) - 1) & 1, fail, P.status);
                cp_async_wait<TC_NRAW - 2>();
                __syncthreads();
                if (*fail) {
                    ok = false;
                    break;
                }
                {
                    const ulonglong2 v = *(const ulonglong2 *)(Raw + (g % TC_NRAW) * RAW_STAGE + tid * 16);
                    const int q = tid >> 4, j = tid & 15;
                    uint8_t *B = Bst + st * B_STAGE + (j >> 3) * 128 + (j & 7) * 16;
                    *(uint4 *)(B + (2 * q) * 256) = digits8(v.x);
                    *(uint4 *)(B + (2 * q + 1) * 256) = digits8(v.y);
                }
                fence_async_smem();
                __syncthreads();
                issue(c + TC_NRAW - 1);  // into the raw stage read by the previous chunk
                if (tid == 0) {
                    tc_fence_after();
                    const uint64_t bd = smem_desc(sh_addr(Bst + st * B_STAGE), 128, 256);
                    const uint64_t a0 = smem_desc(sh_addr(A0) + (uint32_t)ks * 256, 128, a_mn);
                    const uint64_t a1 = smem_desc(sh_addr(A1) + (uint32_t)ks * 256, 128, a_mn);
                    tc_mma(tmem, a0, bd, ks > 0);
                    tc_mma(tmem + TC_TMEM_COLS / 2, a1, bd, ks > 0);
                    tc_commit(&bar[st]);
                    if (ks == nk - 1) tc_commit(&bar[TC_NST]);
                    issued = true;
                }
            }
            if (!ok) break;
            bar_wait(&bar[TC_NST], npass & 1, fail, P.status);
            npass++;
            __syncthreads();
            if (*fail) {
                ok = false;
                break;
            }
            tc_fence_after();
            // Accumulators back: TMEM lane m = 32 (warp % 4) + lane is digit row a = m % 8 of
            // accumulator x = m / 8; warps 0-3 take queries 0-7 of the pass, warps 4-7 queries 8-15.
            {
                const int m = 32 * (warp & 3) + lane, x = m >> 3, a = m & 7;
                const uint32_t trow = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
                for (int qq = 0; qq < 8; qq++) {
                    const int q = (warp >> 2) * 8 + qq, gq = qp * TC_QP + q;
                    uint32_t v0[16], v1[16];
                    tmem_ld16(trow + (uint32_t)(q * 16), v0);                     // d0 x (R0 | R1)
                    tmem_ld16(trow + (uint32_t)(TC_TMEM_COLS / 2 + q * 16), v1);  // d1 x (R0 | R1)
                    tmem_wait_ld();
                    u128 s0 = 0, s1 = 0, s2 = 0;
#pragma unroll
                    for (int b = 0; b < 8; b++) {
                        s0 += (u128)(__int128)(long long)f32_int(v0[b]) << (8 * b);
                        s1 += (u128)(__int128)(long long)(f32_int(v0[8 + b]) + f32_int(v1[b])) << (8 * b);
                        s2 += (u128)(__int128)(long long)f32_int(v1[8 + b]) << (8 * b);
                    }
                    s0 <<= 8 * a;
                    s1 <<= 8 * a;
                    s2 <<= 8 * a;
#pragma unroll
                    for (int o = 1; o < 8; o <<= 1) {
                        s0 += shfl_xor_u128(s0, o);
                        s1 += shfl_xor_u128(s1, o);
                        s2 += shfl_xor_u128(s2, o);
                    }
                    if (a < 3 && x < nx && gq < P.nq) {
                        const u128 t = a == 0 ? s0 : (a == 1 ? s1 : s2);
                        const u64 v = reduce128(Acc128{(u64)t, (u64)(t >> 64)}, pd);
                        u64 *o = P.acc + (size_t)gq * P.a_ct + ((size_t)(x0 + x) * 3 + a) * n_el + e;
                        *o = add_mod(*o, v, pd.q);
                    }
                }
            }
            tc_fence_before();
            __syncthreads();  // the accumulators are free for the next pass
        }
        gchunk += (uint32_t)nchunks;
        if (!ok) break;
    }
    cp_async_wait<0>();
    // release: every MMA this CTA issued has completed (bounded wait after a failure)
    if (tid == 0 && issued && *fail) {
        tc_commit(&bar[TC_NST + 1]);
        const unsigned long long t0 = global_ns();
        while (!bar_test(&bar[TC_NST + 1], 0) && global_ns() - t0 < TC_WAIT_NS) {
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS) : "memory");
    }
}

// rot [nb][2][n_el] of query ciphertext b -> R [n_el][nq][nb][2]: 32 elements x 32 rows
// (j, c) per block through shared memory, reads coalesced along the elements, writes along
// the rows
__global__ void k_rot_to_elements(const u64 *__restrict__ rot, u64 *__restrict__ R, int nb, int nq, int b,
                                  size_t n_el) {
    __shared__ u64 t[32][33];
    const size_t e0 = (size_t)blockIdx.x * 32;
    const int row0 = blockIdx.y * 32, rows = 2 * nb;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int row = row0 + i;
        const size_t e = e0 + threadIdx.x;
        t[i][threadIdx.x] = (row < rows && e < n_el) ? rot[(size_t)row * n_el + e] : 0;
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const size_t e = e0 + i;
        const int row = row0 + threadIdx.x;
        if (e < n_el && row < rows) R[(e * nq + b) * rows + row] = t[threadIdx.x][i];
    }
}

// c0 [nc][n_el] -> mac [n_el][stride] at pos[i]: 32 ciphertexts x 32 elements per block
__global__ void k_mac_scatter(const u64 *__restrict__ c0, const uint32_t *__restrict__ pos, u64 *__restrict__ mac,
                              int nc, size_t n_el, size_t stride) {
    __shared__ u64 t[32][33];
    const size_t e0 = (size_t)blockIdx.x * 32;
    const int i0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int i = i0 + k;
        const size_t e = e0 + threadIdx.x;
        t[k][threadIdx.x] = (i < nc && e < n_el) ? c0[(size_t)i * n_el + e] : 0;
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const size_t e = e0 + k;
        const int i = i0 + threadIdx.x;
        if (e < n_el && i < nc) mac[e * stride + pos[i]] = t[threadIdx.x][k];
    }
}

__global__ void k_mac_gather(const u64 *__restrict__ mac, size_t stride, uint32_t pos, u64 *__restrict__ c0,
                             size_t n_el) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n_el) c0[e] = mac[e * stride + pos];
}

int tc_grid(int device) {
    static std::atomic<int> cache[64];
    if (device >= 0 && device < 64 && cache[device].load() > 0) return cache[device].load();
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const int g = std::max(1, sms);
    if (device >= 0 && device < 64) cache[device].store(g);
    return g;
}

}  // namespace

copse_status enc_mac_tc_attr(int device) {
    static std::atomic<uint64_t> done{0};
    if (device >= 0 && device < 64 && (done.load(std::memory_order_acquire) & (1ull << device))) return COPSE_OK;
    CUDA_TRY(cudaFuncSetAttribute(k_enc_mac_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_TC));
    if (device >= 0 && device < 64) done.fetch_or(1ull << device, std::memory_order_release);
    return COPSE_OK;
}

copse_status enc_mac_tc(copse_ctx *c, const EncModel::MacMat &M, const u64 *R, int nq, u64 *acc, size_t a_ct,
                        u64 seed, cudaStream_t s) {
    if (nq <= 0 || M.nm <= 0 || M.nb <= 0) return COPSE_OK;
    STATUS_TRY(enc_mac_tc_attr(c->device));
    TcArgs P;
    P.mac = M.c0;
    P.idx = M.idx;
    P.R = R;
    P.acc = acc;
    P.a_ct = a_ct;
    P.nm = M.nm;
    P.nb = M.nb;
    P.nq = nq;
    P.ell = M.ell;
    P.logN = c->logN;
    P.n_mt = (M.nm + TC_MX - 1) / TC_MX;
    P.n_kr = (M.nb + TC_KR - 1) / TC_KR;
    P.seed = seed;
    P.pr = c->d_prime;
    P.status = c->d_status;
    const size_t n_items = (size_t)P.n_mt * P.n_kr * ((size_t)M.ell << c->logN);
    const unsigned grid = (unsigned)std::min<size_t>(n_items, (size_t)tc_grid(c->device));
    k_enc_mac_tc<<<grid, TC_THREADS, SMEM_TC, s>>>(P);
    LAUNCH_CHECK();
    return COPSE_OK;
}

double enc_mac_tc_flops(const EncModel::MacMat &M, int nq, int logN) {
    const double n_el = (double)((size_t)M.ell << logN);
    const int n_mt = (M.nm + TC_MX - 1) / TC_MX, nqp = (nq + TC_QP - 1) / TC_QP;
    int nb16 = 0;
    for (int j0 = 0; j0 < M.nb; j0 += TC_KR) nb16 += (std::min(TC_KR, M.nb - j0) + TC_KS - 1) / TC_KS * TC_KS;
    return n_el * n_mt * nqp * (double)nb16 * 2.0 /* d0, d1 */ * 2.0 * 128 * (TC_QP * 2 * 8);
}

copse_status rot_to_elements(copse_ctx *c, const u64 *rot, int nb, int nq, int b, int ell, u64 *R, cudaStream_t s) {
    const size_t n_el = (size_t)ell << c->logN;
    const dim3 grid((unsigned)((n_el + 31) / 32), (unsigned)((2 * nb + 31) / 32));
    TIMED("rot_layout", 16.0 * (double)n_el * 2.0 * nb, s,
          k_rot_to_elements<<<grid, dim3(32, 8), 0, s>>>(rot, R, nb, nq, b, n_el));
    LAUNCH_CHECK();
    return COPSE_OK;
}

copse_status mac_scatter(copse_ctx *c, const u64 *c0, const uint32_t *pos, int nc, const EncModel::MacMat &M,
                         cudaStream_t s) {
    const size_t n_el = (size_t)M.ell << c->logN;
    const dim3 grid((unsigned)((n_el + 31) / 32), (unsigned)((nc + 31) / 32));
    k_mac_scatter<<<grid, dim3(32, 8), 0, s>>>(c0, pos, M.c0, nc, n_el, (size_t)M.nm * M.nb);
    LAUNCH_CHECK();
    return COPSE_OK;
}

copse_status mac_gather(copse_ctx *c, const EncModel::MacMat &M, uint32_t pos, u64 *c0, cudaStream_t s) {
    const size_t n_el = (size_t)M.ell << c->logN;
    k_mac_gather<<<(unsigned)((n_el + 255) / 256), 256, 0, s>>>(M.c0, (size_t)M.nm * M.nb, pos, c0, n_el);
    LAUNCH_CHECK();
    return COPSE_OK;
}
