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
// Exactness.  A residue v of q < 2^55 is taken centred, v' = v or v - q in (-q/2, q/2), and
// written in seven balanced base-256 digits, v' = sum_{i<7} s_i 256^i with s_i in [-128, 127]:
// s_i = byte i of w = v' + C minus 128, C = 0x0080808080808080 (128 in bytes 0-6); w lies in
// (C - 2^54, C + 2^54), so byte 7 of w is 0 and no carry is lost.  A digit is exact in fp16
// and the product of two digits is at most 2^14 in magnitude, so the f32 accumulator of the
// MMA holds a sum of up to 256 such products exactly (|sum| <= 2^22).  The rotations' digits
// sit in the M dimension (row 8 (2 b + c) + a' for digit a' of component c of query b; a' = 7
// zero) and the diagonals' digits in the N dimension (column 128 c' + 8 x + a for digit a of
// component c' of accumulator x; a = 7 zero), so the accumulator holds, for every digit pair,
// the exact partial sum D_a'a = sum_j s_a'(R_c[j][b]) s_a(d_c'[x][j]), and the product sum
// sum_j R'_c[j][b] d'_c'[x][j] = sum D_a'a 256^(a' + a) (|.| < 2^116, congruent mod q to the
// product sum of the residues) is rebuilt in 128-bit integers and reduced mod q once.
//
// One CTA per SM, persistent over work items (element, tile of 16 accumulators, run of up
// to 256 baby steps), its warps specialised and handing work on through mbarriers:
//   warp 0       allocates the tensor memory; runs the MMA loop, one elected lane issuing
//   warp 1       one thread streams the rotations' raw words, one chunk (8 query
//                ciphertexts x 16 baby steps x 2 components, contiguous) per bulk copy
//                (cp.async.bulk with transaction-count completion) into a ring of stages
//   warps 2-9    producers: per item the digits of both components of every diagonal (c0
//                read element-major, c1 regenerated from its seed) into shared memory; then,
//                in two groups of four (warps 2-5, 6-9) taking alternate chunks, they convert
//                the rotations' raw words into a ring of operand stages
//   warps 10-17  epilogue: per pass (8 query ciphertexts) the accumulators back from tensor
//                memory (tcgen05.ld), the exact outputs rebuilt, reduced and stored in acc;
//                warps 10-13 take accumulators 0-7, warps 14-17 accumulators 8-15; between
//                runs they build half of the next run's diagonal digits with the producers
// Per chunk one M 128 x N 256 x K 16 MMA accumulates [R0 | R1] x [d0 | d1] (all four
// component products) into one of two tensor-memory buffers of 256 columns, so the epilogue
// of one pass overlaps the products of the next.
//
// Every wait is bounded by the global timer: a wait that runs out sets COPSE_DEV_MAC_WAIT in
// the context's device status word and every role of the CTA stops; the copies and MMAs in
// flight are waited for (bounded), the tensor memory released and the CTA exits.
#include <algorithm>
#include <atomic>

#include "internal.cuh"

namespace {

constexpr int TC_MX = 16;         // accumulators per tile: 16 x 8 digit rows, N 128 per component
constexpr int TC_QP = 8;          // query ciphertexts per pass: 8 x 2 components x 8 digit rows = M 128
constexpr int TC_KR = 256;        // baby steps per run: exact f32 partial sums
constexpr int TC_KS = 16;         // baby steps per MMA (K of kind::f16)
constexpr int TC_CJ = 64;         // baby steps per chunk (4 MMAs per operand stage)
constexpr int TC_NB = 4;          // operand stages of the rotations' digits
constexpr int TC_NR = 4;          // raw stages of the rotations
constexpr int TC_PROD_WARPS = 8, TC_EPI_WARPS = 8;
// The producer warps form two groups of four; group g converts the chunks with index g modulo 2
// (a quarter of each per warp).  The barrier waits test a phase parity, which is sound only
// while no waiter runs two phases ahead of a barrier: with the stage counts even, a stage is
// only ever used by one group, whose warps meet every phase of it in order.
constexpr int TC_GROUPS = 2, TC_GROUP_WARPS = TC_PROD_WARPS / TC_GROUPS;
constexpr int TC_THREADS = 32 * (2 + TC_PROD_WARPS + TC_EPI_WARPS);  // 576
constexpr int TC_TMEM_COLS = 512;
constexpr unsigned long long TC_WAIT_NS = 2000000000ull;  // 2 s per wait

constexpr uint32_t A_SET = TC_MX * 8 * TC_KR * 2;        // digits of one diagonal component: 64 KB
constexpr uint32_t B_ROW = TC_CJ / 8 * 128;              // bytes between the rotations' core-matrix rows: 1 KB
constexpr uint32_t B_STAGE = TC_QP * 2 * B_ROW;          // digits of one chunk of rotations: 16 KB
constexpr uint32_t RAW_STAGE = TC_QP * TC_CJ * 2 * 8;    // raw words of one chunk: 8 KB
// barriers: raw full / empty, operand full / empty, diagonals full / empty, accumulators full /
// empty (two buffers), drain
constexpr int BAR_RAW_FULL = 0, BAR_RAW_EMPTY = TC_NR, BAR_B_FULL = 2 * TC_NR, BAR_B_EMPTY = 2 * TC_NR + TC_NB,
              BAR_A_FULL = 2 * TC_NR + 2 * TC_NB, BAR_A_EMPTY = BAR_A_FULL + 1, BAR_T_FULL = BAR_A_FULL + 2,
              BAR_T_EMPTY = BAR_T_FULL + 2, BAR_DRAIN = BAR_T_EMPTY + 2, N_BAR = BAR_DRAIN + 1;
constexpr uint32_t OFF_A0 = 0, OFF_B = 2 * A_SET, OFF_RAW = OFF_B + TC_NB * B_STAGE, OFF_BAR = OFF_RAW + TC_NR * RAW_STAGE,
                   OFF_MISC = OFF_BAR + N_BAR * 8, SMEM_TC = OFF_MISC + 16;
static_assert(TC_QP * TC_CJ == 4 * 32 * TC_GROUP_WARPS, "four (query, baby step) pairs per lane of a group's warps and chunk");
static_assert(TC_NB % TC_GROUPS == 0 && TC_NR % TC_GROUPS == 0, "a stage belongs to one group");
static_assert(TC_KR % TC_CJ == 0, "runs are whole chunks");
static_assert(SMEM_TC <= 227 * 1024, "shared memory");

// kind::f16 instruction descriptor: f32 accumulator (bits 4-5 = 1), f16 A and B (formats 0),
// A and B MN-major (bits 15, 16), N / 8 at bit 17, M / 16 at bit 24
constexpr uint32_t idesc_f16(int M, int N) {
    return (1u << 4) | (1u << 15) | (1u << 16) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
constexpr uint32_t IDESC = idesc_f16(TC_QP * 2 * 8, 2 * TC_MX * 8);  // M 128 (rotation digits), N 256 (both components of the diagonals)

__device__ __forceinline__ uint32_t sh_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor without swizzle: core matrices of 8 rows x 16 bytes, the
// leading byte offset (bits 16-29) between core matrices adjacent in K, the stride byte
// offset (bits 32-45) between core matrices adjacent in M / N, version 1 at bit 46.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t k_stride, uint32_t mn_stride) {
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)((k_stride & 0x3FFFF) >> 4) << 16) |
           ((uint64_t)((mn_stride & 0x3FFFF) >> 4) << 32) | (1ull << 46);
}

// one lane of the (converged) warp: the lowest active one
__device__ __forceinline__ bool elect_one() {
    uint32_t pred;
    asm volatile("{\n.reg .pred p;\nelect.sync _|p, 0xffffffff;\nselp.u32 %0, 1, 0, p;\n}\n" : "=r"(pred));
    return pred != 0;
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
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void bar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sh_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sh_addr(bar)) : "memory");
}
__device__ __forceinline__ void bar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sh_addr(bar)), "r"(bytes) : "memory");
}
// bytes (a multiple of 16, both addresses 16-byte aligned) global -> shared, completing on bar
__device__ __forceinline__ void bulk_copy(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     sh_addr(dst)),
                 "l"(src), "r"(bytes), "r"(sh_addr(bar))
                 : "memory");
}
// bytes (a multiple of 16, 16-byte aligned) of global memory into L2, no completion tracked
__device__ __forceinline__ void l2_prefetch(const void *src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
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
// the same, the thread suspended until the phase completes or about TC_SUSPEND_NS pass (a
// waiting warp then takes no issue slots)
constexpr uint32_t TC_SUSPEND_NS = 20000;
__device__ __forceinline__ bool bar_test_suspend(uint64_t *bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(sh_addr(bar)), "r"(parity), "r"(TC_SUSPEND_NS)
        : "memory");
    return done != 0;
}
// wait for the completion of the phase with this parity, at most TC_WAIT_NS; false (and the
// CTA's failure flag and the device status set) when the wait ran out or another one did
__device__ bool bar_wait(uint64_t *bar, uint32_t parity, volatile int *fail, int *status) {
    unsigned long long t0 = 0;
    for (int it = 0;; it++) {
        if (bar_test_suspend(bar, parity)) return true;
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
// the same for a whole warp: every lane waits (no divergence), the warp agrees on the outcome
__device__ __forceinline__ bool warp_wait(uint64_t *bar, uint32_t parity, volatile int *fail, int *status) {
    const bool ok = bar_wait(bar, parity, fail, status);
    return __all_sync(0xffffffffu, ok) != 0;
}

__device__ __forceinline__ uint32_t hsub2(uint32_t a, uint32_t b) {
    uint32_t d;
    asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
// The seven balanced base-256 digits of the centred residue of v (v < q) and a zero eighth, as
// eight fp16 (digit i in half i): byte i of v' + 0x0080808080808080 with 0x64 above it is the
// fp16 of 1024 + byte, less 1152 = 1024 + 128 for bytes 0-6 and less 1024 for byte 7 (zero).
constexpr u64 DIGIT_BIAS = 0x0080808080808080ull;
// the same from w = v' + DIGIT_BIAS
__device__ __forceinline__ uint4 digits8_biased(u64 w);
__device__ __forceinline__ uint4 digits8(u64 v, u64 q) {
    return digits8_biased((v > (q >> 1) ? v - q : v) + DIGIT_BIAS);  // v' = v - q above q / 2
}
__device__ __forceinline__ uint4 digits8_biased(u64 w) {
    const uint32_t lo = (uint32_t)w, hi = (uint32_t)(w >> 32);
    constexpr uint32_t C = 0x64806480u, C7 = 0x64006480u;  // (1152, 1152), (1152 low, 1024 high)
    uint4 r;
    r.x = hsub2(__byte_perm(lo, 0x64u, 0x4140), C);
    r.y = hsub2(__byte_perm(lo, 0x64u, 0x4342), C);
    r.z = hsub2(__byte_perm(hi, 0x64u, 0x4140), C);
    r.w = hsub2(__byte_perm(hi, 0x64u, 0x4342), C7);
    return r;
}
// An integer-valued f32 x in [-2^22, 2^22] plus 1.5 2^23 lies in [2^23, 2^24], where the f32
// spacing is 1: the sum is exact and its bits are the integer x + 0x4B400000.
constexpr float MAGIC = 12582912.0f;
constexpr uint32_t MAGIC_BITS = 0x4B400000u;
__device__ __forceinline__ uint32_t f32_biased(uint32_t bits) { return __float_as_uint(__uint_as_float(bits) + MAGIC); }

using u128 = unsigned __int128;
__device__ __forceinline__ u128 shfl_xor_u128(u128 v, int m) {
    const u64 lo = __shfl_xor_sync(0xffffffffu, (u64)v, m), hi = __shfl_xor_sync(0xffffffffu, (u64)(v >> 64), m);
    return ((u128)hi << 64) | lo;
}
// sum_{b<7} u_b 256^b for u_b < 2^32 (below 2^81)
__device__ __forceinline__ u128 row_value(const uint32_t (&u)[8]) {
    const u64 L = (u64)u[0] + ((u64)u[1] << 8) + ((u64)u[2] << 16) + ((u64)u[3] << 24);
    const u64 H = (u64)u[4] + ((u64)u[5] << 8) + ((u64)u[6] << 16);
    return (u128)L + ((u128)H << 32);
}
// The biases: an output rebuilt from biased digit sums over a < 8, b < 7,
// sum_{a,b} (D_ab + m MAGIC_BITS) 256^(a+b) with m conversions per (a, b), exceeds the product
// sum by m MAGIC_BITS S8 S7, S_n = sum_{i<n} 256^i (all mod 2^128).
__host__ __device__ constexpr u128 bias_rows() {
    u128 S8 = 0, S7 = 0;
    for (int i = 0; i < 8; i++) S8 += (u128)1 << (8 * i);
    for (int i = 0; i < 7; i++) S7 += (u128)1 << (8 * i);
    return (u128)MAGIC_BITS * S8 * S7;
}

// (t mod 2^128, read as a signed value) mod q
__device__ __forceinline__ u64 reduce_signed128(u128 t, const PrimeDev &pd) {
    if ((u64)(t >> 64) >> 63) {
        const u128 n = (u128)0 - t;
        const u64 r = reduce128(Acc128{(u64)n, (u64)(n >> 64)}, pd);
        return r ? pd.q - r : 0;
    }
    return reduce128(Acc128{(u64)t, (u64)(t >> 64)}, pd);
}

struct TcArgs {
    const u64 *mac;       // [n_el][nm][nb16] diagonals' c0 (rows of nb16 = nb rounded up to 16 words)
    const uint32_t *idx;  // [nm][nb] model ciphertext index (mask stream), ~0u = none
    const u64 *R;         // [n_el][nc][nq][64][2] rotations (nc = baby steps / 64, rounded up)
    u64 *acc;             // [nq][nm][3][n_el], written by the first run, added to by later ones
    size_t a_ct;          // words per query ciphertext in acc
    int nm, nb, nb16, nq, ell, logN, n_mt, n_kr, nc;
    u64 seed;
    const PrimeDev *pr;
    int *status;
};

// A work item is (tile of accumulators, element); its baby steps run in runs of up to 256
// (each run its own accumulation: the f32 sums stay exact), taken in order by the same CTA.
struct Item {
    size_t e;
    int x0, nx;
};
__device__ __forceinline__ Item item_at(const TcArgs &P, size_t it, size_t n_el) {
    Item I;
    const int mt = (int)(it / n_el);
    I.e = it - (size_t)mt * n_el;
    I.x0 = mt * TC_MX;
    I.nx = min(TC_MX, P.nm - I.x0);
    return I;
}
struct Run {
    int j0, nj, nk, ncr;  // first baby step, baby steps, MMAs (16 baby steps), chunks (64)
};
__device__ __forceinline__ Run run_at(const TcArgs &P, int kr) {
    Run R;
    R.j0 = kr * TC_KR;
    R.nj = min(TC_KR, P.nb - R.j0);
    R.nk = (R.nj + TC_KS - 1) / TC_KS;
    R.ncr = (R.nj + TC_CJ - 1) / TC_CJ;
    return R;
}

__global__ void __launch_bounds__(TC_THREADS, 1) k_enc_mac_tc(const TcArgs P) {
    extern __shared__ __align__(1024) uint8_t sm[];
    uint8_t *A0 = sm + OFF_A0, *Bst = sm + OFF_B, *Raw = sm + OFF_RAW;
    uint64_t *bar = (uint64_t *)(sm + OFF_BAR);
    uint32_t *tslot = (uint32_t *)(sm + OFF_MISC);
    volatile int *fail = (volatile int *)(sm + OFF_MISC + 4);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const size_t n_el = (size_t)P.ell << P.logN;
    const uint32_t nmask = (1u << P.logN) - 1;
    const int nqp = (P.nq + TC_QP - 1) / TC_QP;
    const size_t n_items = (size_t)P.n_mt * n_el;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sh_addr(tslot)),
                     "r"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 32) {
        for (int i = 0; i < TC_NR; i++) {
            bar_init(&bar[BAR_RAW_FULL + i], 1);
            bar_init(&bar[BAR_RAW_EMPTY + i], TC_GROUP_WARPS);
        }
        for (int i = 0; i < TC_NB; i++) {
            bar_init(&bar[BAR_B_FULL + i], TC_GROUP_WARPS);
            bar_init(&bar[BAR_B_EMPTY + i], 1);
        }
        bar_init(&bar[BAR_A_FULL], TC_PROD_WARPS + TC_EPI_WARPS);
        bar_init(&bar[BAR_A_EMPTY], 1);
        for (int i = 0; i < 2; i++) {
            bar_init(&bar[BAR_T_FULL + i], 1);
            bar_init(&bar[BAR_T_EMPTY + i], TC_EPI_WARPS);
        }
        bar_init(&bar[BAR_DRAIN], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *fail = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    // The diagonals' digits of run (it, kr), by the producer and epilogue warps together (thread
    // t = tid - 64 of 512): entries 2 (t + 512 k) and the next, k < 4 (entry x nj16 + j for
    // accumulator x, baby step j), c0 read from L2 (where the loader prefetched it), the mask
    // regenerated from its seed; the 16 bytes of accumulator x at baby step j are row j % 8 of
    // core matrix (x, j / 8), the second component's rows following the first's.  Waits until
    // the previous run's products are done with the space (na = runs built so far).
    constexpr int AB_THREADS = 32 * (TC_PROD_WARPS + TC_EPI_WARPS), AB_PAIRS = TC_MX * TC_KR / (2 * AB_THREADS);
    auto build_a = [&](size_t it, int kr, uint32_t na) -> bool {
        const int t = tid - 64;
        const Item I = item_at(P, it, n_el);
        const Run R = run_at(P, kr);
        const int nj16 = R.nk * TC_KS, r = (int)(I.e >> P.logN);
        const uint32_t a_mn = (uint32_t)nj16 * 16, pos = (uint32_t)(I.e & nmask);
        const PrimeDev pd = P.pr[r];
        uint8_t *A1 = A0 + TC_MX * a_mn;
        ulonglong2 cw[AB_PAIRS];
#pragma unroll
        for (int k = 0; k < AB_PAIRS; k++) {
            const int i = 2 * (t + k * AB_THREADS), x = i / nj16, j = i - x * nj16;
            cw[k] = make_ulonglong2(0, 0);
            if (i < TC_MX * nj16 && x < I.nx) cw[k] = *(const ulonglong2 *)(P.mac + (I.e * P.nm + I.x0 + x) * P.nb16 + R.j0 + j);
        }
        if (na > 0 && !warp_wait(&bar[BAR_A_EMPTY], (na - 1) & 1, fail, P.status)) return false;
#pragma unroll
        for (int k = 0; k < AB_PAIRS; k++) {
            const int i = 2 * (t + k * AB_THREADS), x = i / nj16, j = i - x * nj16;
            if (i >= TC_MX * nj16) continue;
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const uint32_t id = (x < I.nx && j + h < R.nj) ? __ldg(P.idx + (size_t)(I.x0 + x) * P.nb + R.j0 + j + h) : ~0u;
                u64 d0 = 0, d1 = 0;
                if (id != ~0u) {
                    d0 = h ? cw[k].y : cw[k].x;
                    d1 = seeded_mask(P.seed, MODEL_STREAM + 2ull * id, r, pos, P.logN, pd);
                }
                const uint32_t off = (uint32_t)x * a_mn + (uint32_t)((j + h) >> 3) * 128 + (uint32_t)((j + h) & 7) * 16;
                *(uint4 *)(A0 + off) = digits8(d0, pd.q);
                *(uint4 *)(A1 + off) = digits8(d1, pd.q);
            }
        }
        fence_async_smem();
        __syncwarp();
        if (lane == 0) bar_arrive(&bar[BAR_A_FULL]);
        return true;
    };

    if (warp == 0) {
        // ---------------------------------------------------------------- MMA issue
        // The whole warp runs the loop (its descriptors and counters are warp-uniform) and waits;
        // one elected lane, always the same one, issues the MMAs and the commits that track them.
        {
            uint32_t nb_c = 0, np_c = 0, na = 0;  // operand stages, passes, runs consumed
            bool ok = true, issued = false;
            for (size_t it = blockIdx.x; it < n_items && ok; it += gridDim.x)
                for (int kr = 0; kr < P.n_kr && ok; kr++, na++) {
                    const Run R = run_at(P, kr);
                    const uint32_t a_mn = (uint32_t)R.nk * TC_KS * 16;  // bytes between accumulators' core-matrix rows
                    // descriptors of the first 16 baby steps; 16 baby steps further is 256 bytes, 16 in
                    // the descriptor's address field
                    const uint64_t dA = smem_desc(sh_addr(A0), 128, a_mn), dB = smem_desc(sh_addr(Bst), 128, B_ROW);
                    if (!(ok = warp_wait(&bar[BAR_A_FULL], na & 1, fail, P.status))) break;
                    for (int p = 0; p < nqp && ok; p++, np_c++) {
                        const uint32_t buf = np_c & 1;
                        if (np_c >= 2 &&
                            !(ok = warp_wait(&bar[BAR_T_EMPTY + buf], ((np_c >> 1) - 1) & 1, fail, P.status)))
                            break;
                        tc_fence_after();
                        const uint32_t d = tmem + buf * 256;
                        for (int kc = 0; kc < R.ncr; kc++, nb_c++) {
                            const int st = (int)(nb_c % TC_NB);
                            if (!(ok = warp_wait(&bar[BAR_B_FULL + st], (nb_c / TC_NB) & 1, fail, P.status))) break;
                            tc_fence_after();
                            // rotations' digits (M: row 8 (2 q + c) + b) x diagonals' digits of both
                            // components (N: column 128 c' + 8 x + a; the second component's core
                            // matrices follow the first's at the same stride), 16 baby steps per MMA
                            const int ns = min(TC_CJ / TC_KS, R.nk - kc * (TC_CJ / TC_KS));
                            const uint64_t b0 = dB + (uint64_t)(st * (B_STAGE >> 4)), a0 = dA + (uint64_t)(kc * (TC_CJ / TC_KS) * 16);
                            if (elect_one()) {
                                for (int s2 = 0; s2 < ns; s2++) tc_mma(d, b0 + (uint64_t)(16 * s2), a0 + (uint64_t)(16 * s2), (kc | s2) != 0);
                                tc_commit(&bar[BAR_B_EMPTY + st]);
                            }
                            __syncwarp();
                            issued = true;
                        }
                        if (ok && elect_one()) tc_commit(&bar[BAR_T_FULL + buf]);
                        __syncwarp();
                    }
                    if (ok && elect_one()) tc_commit(&bar[BAR_A_EMPTY]);
                    __syncwarp();
                }
            if (issued && *fail && elect_one()) {  // the issuing lane waits (bounded) for its MMAs in flight before the memory goes
                tc_commit(&bar[BAR_DRAIN]);
                const unsigned long long t0 = global_ns();
                while (!bar_test(&bar[BAR_DRAIN], 0) && global_ns() - t0 < TC_WAIT_NS) {
                }
            }
        }
    } else if (warp == 1) {
        // ---------------------------------------------------------------- rotation loader
        if (lane == 0) {
            uint32_t nr_c = 0;
            bool ok = true;
            for (size_t it = blockIdx.x; it < n_items && ok; it += gridDim.x) {
                const Item I = item_at(P, it, n_el);
                if (it + gridDim.x < n_items) {
                    // the next item's c0 rows and the chunks of its first pass into L2 while this
                    // one runs (the later chunks stream in through the ring in time; prefetching the
                    // whole rotation block only doubled its DRAM reads, evicted before use)
                    const Item J = item_at(P, it + gridDim.x, n_el);
                    const uint8_t *r0 = (const uint8_t *)(P.R + J.e * (size_t)P.nc * P.nq * TC_CJ * 2);
                    const uint32_t first = (uint32_t)min(TC_QP, P.nq) * TC_CJ * 2 * 8;
                    for (int kc = 0; kc < P.nc && kc < TC_KR / TC_CJ; kc++)
                        l2_prefetch(r0 + (size_t)kc * P.nq * TC_CJ * 2 * 8, first);
                    l2_prefetch(P.mac + (J.e * P.nm + J.x0) * P.nb16, (uint32_t)(J.nx * P.nb16 * 8));
                }
                for (int kr = 0; kr < P.n_kr && ok; kr++) {
                    const Run R = run_at(P, kr);
                    for (int p = 0; p < nqp && ok; p++)
                        for (int kc = 0; kc < R.ncr; kc++, nr_c++) {
                            const int st = (int)(nr_c % TC_NR);
                            if (nr_c >= TC_NR &&
                                !(ok = bar_wait(&bar[BAR_RAW_EMPTY + st], ((nr_c / TC_NR) - 1) & 1, fail, P.status)))
                                break;
                            const int nqq = min(TC_QP, P.nq - p * TC_QP);
                            const uint32_t bytes = (uint32_t)nqq * TC_CJ * 2 * 8;
                            bar_expect_tx(&bar[BAR_RAW_FULL + st], bytes);
                            bulk_copy(Raw + st * RAW_STAGE,
                                      P.R + (((I.e * P.nc + R.j0 / TC_CJ + kc) * P.nq + (size_t)p * TC_QP) * TC_CJ * 2),
                                      bytes, &bar[BAR_RAW_FULL + st]);
                        }
                }
            }
            // no copy may land after the CTA is gone: wait (bounded) for the last stages issued
            if (*fail)
                for (uint32_t k = nr_c > TC_NR ? nr_c - TC_NR : 0; k < nr_c; k++) {
                    const unsigned long long t0 = global_ns();
                    while (!bar_test(&bar[BAR_RAW_FULL + k % TC_NR], (k / TC_NR) & 1) && global_ns() - t0 < TC_WAIT_NS) {
                    }
                }
        }
    } else if (warp < 2 + TC_PROD_WARPS) {
        // ---------------------------------------------------------------- producers
        // The producers build their part of each run's diagonal digits (build_a) first.  Their group
        // (pt / 128) converts every other chunk, the thread pairs gt + 128 u, u < 4, gt = pt % 128
        // (the words come centred and biased, v' + 0x0080808080808080, from the rotations'
        // element-major layout).
        const int pt = tid - 64, grp = pt / (TC_GROUP_WARPS * 32), gt = pt % (TC_GROUP_WARPS * 32);
        uint32_t nb_c = 0, nr_c = 0, na = 0;
        bool ok = true;
        for (size_t it = blockIdx.x; it < n_items && ok; it += gridDim.x) {
            const Item I = item_at(P, it, n_el);
            const int r = (int)(I.e >> P.logN);
            const PrimeDev pd = P.pr[r];
            const uint32_t pos = (uint32_t)(I.e & nmask);
            for (int kr = 0; kr < P.n_kr && ok; kr++, na++) {
                const Run R = run_at(P, kr);
                if (!(ok = build_a(it, kr, na))) break;
                // the rotations' digits, chunk by chunk
                for (int p = 0; p < nqp && ok; p++)
                    for (int kc = 0; kc < R.ncr; kc++, nb_c++, nr_c++) {
                        if ((int)(nb_c % TC_GROUPS) != grp) continue;
                        const int st = (int)(nb_c % TC_NB), rs = (int)(nr_c % TC_NR);
                        if (nb_c >= TC_NB &&
                            !(ok = warp_wait(&bar[BAR_B_EMPTY + st], ((nb_c / TC_NB) - 1) & 1, fail, P.status)))
                            break;
                        if (!(ok = warp_wait(&bar[BAR_RAW_FULL + rs], (nr_c / TC_NR) & 1, fail, P.status))) break;
                        const uint8_t *raw = Raw + rs * RAW_STAGE;
                        uint8_t *Bs = Bst + st * B_STAGE;
#pragma unroll
                        for (int u = 0; u < 4; u++) {
                            const int pr = gt + TC_GROUP_WARPS * 32 * u, q = pr >> 6, j = pr & 63;
                            ulonglong2 v = make_ulonglong2(DIGIT_BIAS, DIGIT_BIAS);  // digits of zero
                            if (p * TC_QP + q < P.nq && kc * TC_CJ + j < R.nj) v = *(const ulonglong2 *)(raw + pr * 16);
                            uint8_t *B = Bs + (j >> 3) * 128 + (j & 7) * 16;
                            *(uint4 *)(B + (2 * q) * B_ROW) = digits8_biased(v.x);
                            *(uint4 *)(B + (2 * q + 1) * B_ROW) = digits8_biased(v.y);
                        }
                        fence_async_smem();
                        __syncwarp();
                        if (lane == 0) {
                            bar_arrive(&bar[BAR_B_FULL + st]);
                            bar_arrive(&bar[BAR_RAW_EMPTY + rs]);
                        }
                    }
            }
        }
    } else {
        // ---------------------------------------------------------------- epilogue
        // TMEM lane m = 32 (warp % 4) + lane is digit b = m % 8 of component c = (m / 8) % 2 of
        // query q = m / 16 of the pass; column 128 c' + 8 x + a holds digit a of component c' of
        // accumulator x.  Warps 10-13 take accumulators 0-7, warps 14-17 accumulators 8-15.
        const int m = 32 * (warp & 3) + lane, b = m & 7, cq = (m >> 3) & 1, qq = m >> 4;
        const int xh = warp >= 2 + TC_PROD_WARPS + 4 ? 8 : 0;
        const uint32_t trow = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
        uint32_t np_c = 0, na = 0;
        bool ok = true;
        // the epilogue warps build their part of each run's diagonal digits too: the first run's
        // before their first pass, each next one after their last pass of the run before
        if ((size_t)blockIdx.x < n_items) ok = build_a(blockIdx.x, 0, na++);
        for (size_t it = blockIdx.x; it < n_items && ok; it += gridDim.x) {
            const Item I = item_at(P, it, n_el);
            const PrimeDev pd = P.pr[(int)(I.e >> P.logN)];
            for (int kr = 0; kr < P.n_kr && ok; kr++) {
                for (int p = 0; p < nqp && ok; p++, np_c++) {
                    const uint32_t buf = np_c & 1;
                    if (!(ok = warp_wait(&bar[BAR_T_FULL + buf], (np_c >> 1) & 1, fail, P.status))) break;
                    tc_fence_after();
                    const uint32_t tb = trow + buf * 256;
                    // Row values sum_{a<7} D 256^a of the 16 items it = 2 (x - xh) + c', summed over the
                    // 8 digit rows b of (q, c) by a reduce-scatter (lane b ends with items 2b and 2b + 1,
                    // both components c' of accumulator xh + b).  Its first round pairs items it and
                    // it + 8, so each half of the loads (items 4h..4h+3 and 8+4h..8+4h+3) is folded at once.
                    const bool b2 = (lane >> 2) & 1, b1 = (lane >> 1) & 1, b0 = lane & 1;
                    u128 v[8];
#pragma unroll
                    for (int h = 0; h < 2; h++) {
                        uint32_t w[8][8];
#pragma unroll
                        for (int i = 0; i < 8; i++) {
                            const int it2 = (i < 4 ? 0 : 8) + 4 * h + (i & 3);
                            tmem_ld8(tb + (uint32_t)(128 * (it2 & 1) + 8 * (xh + (it2 >> 1))), w[i]);
                        }
                        tmem_wait_ld();
#pragma unroll
                        for (int i = 0; i < 4; i++) {
                            uint32_t u[8], z[8];
#pragma unroll
                            for (int k = 0; k < 8; k++) {
                                u[k] = f32_biased(w[i][k]);
                                z[k] = f32_biased(w[4 + i][k]);
                            }
                            const u128 lo = row_value(u), hi = row_value(z);  // items 4h + i and 8 + 4h + i
                            const u128 send = b2 ? lo : hi, keep = b2 ? hi : lo;
                            const u128 got = shfl_xor_u128(send, 4);
                            v[4 * h + i] = b2 ? got + (keep << 32) : keep + (got << 32);
                        }
                    }
#pragma unroll
                    for (int i = 0; i < 4; i++) {
                        const u128 send = b1 ? v[i] : v[4 + i], keep = b1 ? v[4 + i] : v[i];
                        const u128 got = shfl_xor_u128(send, 2);
                        v[i] = b1 ? got + (keep << 16) : keep + (got << 16);
                    }
#pragma unroll
                    for (int i = 0; i < 2; i++) {
                        const u128 send = b0 ? v[i] : v[2 + i], keep = b0 ? v[2 + i] : v[i];
                        const u128 got = shfl_xor_u128(send, 1);
                        v[i] = b0 ? got + (keep << 8) : keep + (got << 8);
                    }
                    u128 t0 = v[0], t1 = v[1];
                    t0 -= bias_rows();
                    t1 -= bias_rows();
                    // c = 0: t0 = d0 R0, t1 = d1 R0;  c = 1: t0 = d0 R1, t1 = d1 R1
                    const u128 other = shfl_xor_u128(t1, 8);  // the partner lane's d1 R0 (for c = 1)
                    const int gq = p * TC_QP + qq, x = xh + b;
                    if (x < I.nx && gq < P.nq) {
                        u64 *o = P.acc + (size_t)gq * P.a_ct + (size_t)(I.x0 + x) * 3 * n_el + I.e;
                        if (cq == 0) {
                            const u64 v0 = reduce_signed128(t0, pd);
                            o[0] = kr == 0 ? v0 : add_mod(o[0], v0, pd.q);
                        } else {
                            const u64 v1 = reduce_signed128(t0 + other, pd), v2 = reduce_signed128(t1, pd);
                            o[n_el] = kr == 0 ? v1 : add_mod(o[n_el], v1, pd.q);
                            o[2 * n_el] = kr == 0 ? v2 : add_mod(o[2 * n_el], v2, pd.q);
                        }
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) bar_arrive(&bar[BAR_T_EMPTY + buf]);
                }
                if (!ok) break;
                if (kr + 1 < P.n_kr)
                    ok = build_a(it, kr + 1, na++);
                else if (it + gridDim.x < n_items)
                    ok = build_a(it + gridDim.x, 0, na++);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS) : "memory");
    }
}

// rot [nb][2][n_el] of query ciphertext b -> R [n_el][nc][nq][64][2] (baby step j in chunk
// j / 64 at j % 64), each residue v stored centred and biased, v' + 0x0080808080808080: 32 elements x 32 rows (j, c) per block through shared memory, reads
// coalesced along the elements, writes along the rows
__global__ void k_rot_to_elements(const u64 *__restrict__ rot, u64 *__restrict__ R, int nb, int nq, int b,
                                  size_t n_el, int logN, const PrimeDev *__restrict__ pr) {
    __shared__ u64 t[32][33];
    const size_t e0 = (size_t)blockIdx.x * 32;
    const int row0 = blockIdx.y * 32, rows = 2 * nb, nc = (nb + TC_CJ - 1) / TC_CJ;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int row = row0 + i;
        const size_t e = e0 + threadIdx.x;
        t[i][threadIdx.x] = (row < rows && e < n_el) ? rot[(size_t)row * n_el + e] : 0;
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const size_t e = e0 + i;
        const int row = row0 + threadIdx.x;
        if (e < n_el && row < rows) {
            const int j = row >> 1;
            const u64 q = pr[e >> logN].q, v = t[threadIdx.x][i];
            R[((e * nc + j / TC_CJ) * nq + b) * (TC_CJ * 2) + (j % TC_CJ) * 2 + (row & 1)] =
                (v > (q >> 1) ? v - q : v) + DIGIT_BIAS;
        }
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
    P.nc = (M.nb + TC_CJ - 1) / TC_CJ;
    P.nb16 = mac_row(M.nb);
    P.seed = seed;
    P.pr = c->d_prime;
    P.status = c->d_status;
    const size_t n_items = (size_t)P.n_mt * ((size_t)M.ell << c->logN);
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
          k_rot_to_elements<<<grid, dim3(32, 8), 0, s>>>(rot, R, nb, nq, b, n_el, c->logN, c->d_prime));
    LAUNCH_CHECK();
    return COPSE_OK;
}

copse_status mac_scatter(copse_ctx *c, const u64 *c0, const uint32_t *pos, int nc, const EncModel::MacMat &M,
                         cudaStream_t s) {
    const size_t n_el = (size_t)M.ell << c->logN;
    const dim3 grid((unsigned)((n_el + 31) / 32), (unsigned)((nc + 31) / 32));
    k_mac_scatter<<<grid, dim3(32, 8), 0, s>>>(c0, pos, M.c0, nc, n_el, (size_t)M.nm * mac_row(M.nb));
    LAUNCH_CHECK();
    return COPSE_OK;
}

copse_status mac_gather(copse_ctx *c, const EncModel::MacMat &M, uint32_t pos, u64 *c0, cudaStream_t s) {
    const size_t n_el = (size_t)M.ell << c->logN;
    k_mac_gather<<<(unsigned)((n_el + 255) / 256), 256, 0, s>>>(M.c0, (size_t)M.nm * mac_row(M.nb), pos, c0, n_el);
    LAUNCH_CHECK();
    return COPSE_OK;
}
