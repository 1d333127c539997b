"""Pins of the oracle's ring layer against facts fixed outside it: primality by
an independent test, the definition of the negacyclic transform, the
schoolbook product checked against integer polynomial multiplication, the
slot-evaluation definition, explicit slot permutations, and the published
SplitMix64 test vector."""
import numpy as np
import pytest

from conftest import read_golden
from oracle import bgv as B

T = 65537


def _fermat_ok(p):
    return all(pow(a, p - 1, p) == 1 for a in (2, 3, 5, 7, 11, 13))


@pytest.mark.parametrize("logN,bits", [(4, 40), (10, 50), (14, 55), (15, 55)])
def test_primes(logN, bits):
    out = np.zeros(12, dtype=np.uint64)
    assert B.lib().or_find_primes(logN, T, bits, 12, out) == 12
    ps = [int(x) for x in out]
    M = 2 * (1 << logN) * T
    assert ps == sorted(ps, reverse=True) and len(set(ps)) == 12
    for p in ps:
        assert p % M == 1 and p < (1 << bits) and p.bit_length() == bits
        assert _fermat_ok(p)
    sympy = pytest.importorskip("sympy")
    assert all(sympy.isprime(p) for p in ps)
    # nothing skipped: every k*M+1 between consecutive picks is composite
    for a, b in zip(ps, ps[1:]):
        for k in range((b - 1) // M + 1, (a - 1) // M):
            assert not sympy.isprime(k * M + 1)


def test_is_prime_small():
    L = B.lib()
    got = [n for n in range(2, 400) if L.or_is_prime(n)]
    sieve = [n for n in range(2, 400) if all(n % d for d in range(2, int(n ** 0.5) + 1))]
    assert got == sieve
    # strong pseudoprimes to small bases must be rejected
    for n in (3215031751, 2152302898747, 3474749660383, 341550071728321, 3825123056546413051):
        assert not L.or_is_prime(n)


@pytest.mark.parametrize("logN", [3, 10, 14])
def test_root_of_unity(logN):
    q = 65537 if logN <= 15 else None
    for q in (T, B.Params(logN=logN, L=1, bits=50, dnum=1).primes[0]):
        psi = B.lib().or_root_2n(q, logN)
        N = 1 << logN
        assert pow(psi, N, q) == q - 1 and pow(psi, 2 * N, q) == 1


def _rand(rng, n, q):
    return rng.integers(0, q, size=n, dtype=np.uint64)


@pytest.mark.parametrize("logN", [1, 2, 5, 6])
def test_ntt_is_evaluation_at_odd_powers(logN):
    """A[i] = a(psi^(2i+1)), computed with Python integers."""
    rng = np.random.default_rng(logN)
    q = B.Params(logN=logN, L=1, bits=50, dnum=1).primes[0]
    psi = B.lib().or_root_2n(q, logN)
    N = 1 << logN
    a = _rand(rng, N, q)
    A = a.copy()
    B.lib().or_ntt_fwd(A, logN, q, psi)
    ai = [int(x) for x in a]
    for i in range(N):
        x = pow(psi, 2 * i + 1, q)
        assert int(A[i]) == sum(c * pow(x, j, q) for j, c in enumerate(ai)) % q
    D = np.zeros(N, dtype=np.uint64)
    B.lib().or_eval_direct(a, logN, q, psi, D)
    assert np.array_equal(A, D)
    B.lib().or_ntt_inv(A, logN, q, psi)
    assert np.array_equal(A, a)


def _negacyclic_py(a, b, q):
    """(a*b) mod (X^N + 1, q) with Python integers: plain product, then X^N = -1."""
    N = len(a)
    full = [0] * (2 * N)
    for i, x in enumerate(a):
        for j, y in enumerate(b):
            full[i + j] += int(x) * int(y)
    return [(full[k] - full[k + N]) % q for k in range(N)]


@pytest.mark.parametrize("logN,bits", [(1, 30), (4, 50), (6, 55)])
def test_schoolbook_and_ntt_product(logN, bits):
    rng = np.random.default_rng(100 + logN)
    q = B.Params(logN=logN, L=1, bits=bits, dnum=1).primes[0]
    N = 1 << logN
    a, b = _rand(rng, N, q), _rand(rng, N, q)
    ref = _negacyclic_py(a, b, q)
    sb = np.zeros(N, dtype=np.uint64)
    B.lib().or_negacyclic_schoolbook(a, b, logN, q, sb)
    nt = np.zeros(N, dtype=np.uint64)
    B.lib().or_negacyclic_mul(a, b, logN, q, nt)
    assert [int(x) for x in sb] == ref
    assert [int(x) for x in nt] == ref


def test_ntt_roundtrip_large():
    rng = np.random.default_rng(5)
    for logN in (10, 14):
        q = B.Params(logN=logN, L=1, bits=55, dnum=1).primes[0]
        psi = B.lib().or_root_2n(q, logN)
        a = _rand(rng, 1 << logN, q)
        A = a.copy()
        B.lib().or_ntt_fwd(A, logN, q, psi)
        B.lib().or_ntt_inv(A, logN, q, psi)
        assert np.array_equal(A, a)


@pytest.mark.parametrize("logN", [3, 5])
def test_slots_are_evaluations(logN):
    """Slot (r,c) = m(zeta^e), zeta = 3^((t-1)/2N), e = 3^c or -3^c mod 2N."""
    N = 1 << logN
    P = B.Params(logN=logN, L=1, bits=40, dnum=1)
    rng = np.random.default_rng(logN)
    v = rng.integers(0, T, size=N)
    m = B.encode(P, v) % T
    zeta = pow(3, (T - 1) // (2 * N), T)
    for s in range(N):
        r, c = divmod(s, N // 2)
        e = pow(3, c, 2 * N) if r == 0 else (2 * N - pow(3, c, 2 * N)) % (2 * N)
        x = pow(zeta, e, T)
        assert sum(int(mj) * pow(x, j, T) for j, mj in enumerate(m)) % T == v[s]


def test_encode_roundtrip_and_product():
    logN = 10
    P = B.Params(logN=logN, L=1, bits=40, dnum=1)
    N = P.N
    rng = np.random.default_rng(3)
    a, b = rng.integers(0, T, size=N), rng.integers(0, T, size=N)
    ma, mb = B.encode(P, a), B.encode(P, b)
    assert np.array_equal(B.decode(P, ma).astype(np.int64), a)
    assert np.all(np.abs(ma) <= (T - 1) // 2)
    prod = np.zeros(N, dtype=np.uint64)
    B.lib().or_negacyclic_mul((ma % T).astype(np.uint64), (mb % T).astype(np.uint64), logN, T, prod)
    assert np.array_equal(B.decode(P, prod).astype(np.int64), (a * b) % T)
    # the all-ones vector is the constant polynomial 1
    one = B.encode(P, np.ones(N, dtype=np.int64))
    assert one[0] == 1 and not one[1:].any()


@pytest.mark.parametrize("logN,k", [(4, 1), (6, 3), (10, 5), (10, 511)])
def test_automorphism_is_rotation(logN, k):
    """X -> X^(3^k) rotates each row left by k; X -> X^(2N-1) swaps the rows."""
    P = B.Params(logN=logN, L=1, bits=40, dnum=1)
    N, h = P.N, P.N // 2
    rng = np.random.default_rng(k)
    v = rng.integers(0, T, size=N)
    m = (B.encode(P, v) % T).astype(np.uint64)
    out = np.zeros(N, dtype=np.uint64)
    B.lib().or_automorphism(m, logN, T, B.galois_rot(logN, k), out)
    got = B.decode(P, out).astype(np.int64)
    want = np.array([v[r * h + (c + k) % h] for r in range(2) for c in range(h)])
    assert np.array_equal(got, want)
    B.lib().or_automorphism(m, logN, T, 2 * N - 1, out)
    got = B.decode(P, out).astype(np.int64)
    assert np.array_equal(got, np.concatenate([v[h:], v[:h]]))


def test_splitmix64_published_vector():
    want = [int(x) for x in read_golden("splitmix64_seed1234567.txt").split()]
    assert [B.lib().or_word(1234567, 0, i) for i in range(5)] == want


def test_samplers_distributions():
    N = 1 << 16
    t_ = np.zeros(N, dtype=np.int64)
    B.lib().or_sample_ternary(11, 5, N, t_)
    assert set(np.unique(t_)) == {-1, 0, 1}
    counts = np.bincount(t_ + 1)
    assert np.all(np.abs(counts - N / 3) < 5 * np.sqrt(N * 2 / 9))
    c = np.zeros(N, dtype=np.int64)
    B.lib().or_sample_cbd(11, 6, N, c)
    assert c.min() >= -21 and c.max() <= 21
    assert abs(c.mean()) < 0.1 and abs(c.var() - 10.5) < 0.4
    # distinct streams and seeds give distinct words
    L = B.lib()
    assert L.or_word(1, 2, 3) != L.or_word(1, 3, 3) != L.or_word(2, 2, 3)


def test_stream_layout_never_wraps():
    """word(seed, stream, idx) = SplitMix64 output stream * 2^40 + idx + 1: every stream
    the layout uses is below 2^24, so distinct (stream, idx) pairs never share an output."""
    from oracle import bgv as B
    used = [B.STREAM_SECRET, B.STREAM_PK_A, B.STREAM_PK_E, B.STREAM_RELIN + 79,
            B.stream_galois(65535) + 79, B.stream_encrypt(0), B.stream_encrypt(0xFFFFF) + 2,
            B.stream_model(0), B.stream_model(0x3FFFFF) + 1]
    assert all(0 < s < (1 << 24) for s in used)
    assert B.stream_galois(65535) + 79 < B.stream_encrypt(0)
    assert B.stream_encrypt(0xFFFFF) + 2 < B.stream_model(0)
    # the two families that collided under a wrapping layout now differ
    assert B.lib().or_word(5, B.stream_encrypt(0) + 1, 0) != B.lib().or_word(5, B.STREAM_SECRET, 0)
