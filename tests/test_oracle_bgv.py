"""Pins of the oracle's BGV layer.  Decryption must give the slotwise result
of each operation (add, constant add, plaintext multiply, ciphertext multiply,
rotation); modulus switching and key switching are checked against their
definitions with exact Python integers over the CRT-reconstructed modulus."""
import numpy as np
import pytest

from oracle import bgv as B

T = 65537


def _setup(logN=6, L=5, bits=50, dnum=2, galois=()):
    P = B.Params(logN=logN, L=L, bits=bits, dnum=dnum)
    bgv = B.Bgv(P)
    keys = bgv.keygen(1234, galois)
    return P, bgv, keys


def _rot(v, k, N):
    h = N // 2
    return np.concatenate([np.roll(v[:h], -k), np.roll(v[h:], -k)])


def _crt(x, qs):
    Q = 1
    for q in qs:
        Q *= q
    out = []
    for j in range(x.shape[1]):
        v = 0
        for r, q in enumerate(qs):
            Qh = Q // q
            v += int(x[r, j]) * Qh * pow(Qh % q, -1, q)
        out.append(v % Q)
    return out, Q


def _centre(v, Q):
    return v - Q if v > Q // 2 else v


@pytest.mark.parametrize("logN,L,dnum", [(4, 3, 1), (6, 5, 2), (10, 6, 3)])
def test_encrypt_decrypt(logN, L, dnum):
    P, bgv, keys = _setup(logN, L, 50, dnum)
    rng = np.random.default_rng(logN)
    v = rng.integers(0, T, size=P.N)
    ct = bgv.encrypt_slots(keys.pk, v, 77, 0)
    assert ct.shape == (2, L, P.N)
    assert np.array_equal(bgv.decrypt_slots(keys.sk, ct).astype(np.int64), v)
    # fresh noise: [c0 + c1 s]_Q = m + t*e with small e
    x, Q = _crt(bgv.decrypt_raw(keys.sk, ct), P.q[:L])
    m = B.encode(P, v)
    for j in range(P.N):
        e = _centre(x[j], Q) - int(m[j])
        assert e % T == 0 and abs(e) < T * (1 << 20)
    # a different encryption index gives a different ciphertext of the same plaintext
    ct2 = bgv.encrypt_slots(keys.pk, v, 77, 1)
    assert not np.array_equal(ct, ct2)


def test_slotwise_arithmetic():
    P, bgv, keys = _setup(6, 5, 50, 2)
    rng = np.random.default_rng(9)
    a, b = rng.integers(0, 2, size=P.N), rng.integers(0, 2, size=P.N)
    ca, cb = bgv.encrypt_slots(keys.pk, a, 5, 0), bgv.encrypt_slots(keys.pk, b, 5, 1)
    dec = lambda c: bgv.decrypt_slots(keys.sk, c).astype(np.int64)
    assert np.array_equal(dec(bgv.add(ca, cb)), (a + b) % T)
    assert np.array_equal(dec(bgv.sub(ca, cb)), (a - b) % T)
    assert np.array_equal(dec(bgv.add_plain(ca, B.encode(P, b))), (a + b) % T)
    w = rng.integers(0, T, size=P.N)
    assert np.array_equal(dec(bgv.mul_plain(ca, B.encode(P, w))), (a * w) % T)
    prod = bgv.mul(ca, cb, keys.rlk)
    assert prod.shape[1] == P.L - 1
    assert np.array_equal(dec(prod), (a * b) % T)
    # XOR as a + b - 2ab (the GF(2) semantics the slots carry)
    x = bgv.sub(bgv.add(ca, cb), bgv.add(prod, prod))
    assert np.array_equal(dec(x), a ^ b)
    # operands at different levels are aligned by modulus switching
    assert np.array_equal(dec(bgv.mul(prod, ca, keys.rlk)), (a * b * a) % T)


@pytest.mark.parametrize("k", [1, 2, 7, 31])
def test_rotation(k):
    logN = 6
    g = B.galois_rot(logN, k)
    P, bgv, keys = _setup(logN, 4, 50, 2, galois=[g])
    rng = np.random.default_rng(k)
    v = rng.integers(0, T, size=P.N)
    ct = bgv.encrypt_slots(keys.pk, v, 3, 0)
    r = bgv.rotate(ct, g, keys.gk[g])
    assert np.array_equal(bgv.decrypt_slots(keys.sk, r).astype(np.int64), _rot(v, k, P.N))
    # rotation at a lower level (fewer active digits)
    low = bgv.modswitch(bgv.modswitch(ct))
    r2 = bgv.rotate(low, g, keys.gk[g])
    assert r2.shape[1] == 2
    assert np.array_equal(bgv.decrypt_slots(keys.sk, r2).astype(np.int64), _rot(v, k, P.N))


@pytest.mark.parametrize("ell", [2, 4, 5])
def test_modswitch_definition(ell):
    """c' * q_last = c - delta with delta = c mod q_last, delta = 0 mod t, |delta| <= t*q_last/2."""
    P, bgv, keys = _setup(4, 5, 50, 2)
    rng = np.random.default_rng(ell)
    ct = np.stack([np.stack([rng.integers(0, q, size=P.N, dtype=np.uint64) for q in P.q[:ell]])
                   for _ in range(2)])
    out = bgv.modswitch(ct)
    ql = P.q[ell - 1]
    for c in range(2):
        x, Q = _crt(ct[c], P.q[:ell])
        y, Q2 = _crt(out[c], P.q[:ell - 1])
        for j in range(P.N):
            delta = _centre((x[j] - ql * y[j]) % Q, Q)
            assert delta % T == 0
            assert (delta - x[j]) % ql == 0
            assert abs(delta) <= T * (ql - 1) // 2


@pytest.mark.parametrize("ell", [1, 3, 5, 6])
def test_keyswitch_definition(ell):
    """KS(x) = (k0, k1) with k0 + k1*s = x*s' + t*e over Q_ell, e small; here s' = s^2."""
    P, bgv, keys = _setup(4, 6, 50, 3)
    rng = np.random.default_rng(ell)
    x = np.stack([rng.integers(0, q, size=P.N, dtype=np.uint64) for q in P.q[:ell]])
    k = bgv.keyswitch(x, keys.rlk)
    qs = P.q[:ell]
    k0, Q = _crt(k[0], qs)
    k1, _ = _crt(k[1], qs)
    xi, _ = _crt(x, qs)
    s = [int(v) for v in keys.sk]
    N = P.N

    def mul(a, b):
        out = [0] * N
        for i in range(N):
            for j in range(N):
                if i + j < N:
                    out[i + j] += a[i] * b[j]
                else:
                    out[i + j - N] -= a[i] * b[j]
        return out

    s2 = mul(s, s)
    lhs = [a + b for a, b in zip(k0, mul(k1, s))]
    rhs = mul(xi, s2)
    for j in range(N):
        e = _centre((lhs[j] - rhs[j]) % Q, Q)
        assert e % T == 0
        assert abs(e) < T * (1 << 24)


def test_noise_budget_consumption():
    """Each multiply-then-modswitch lands back near the fresh noise level."""
    P, bgv, keys = _setup(10, 5, 50, 3)
    rng = np.random.default_rng(1)
    a = rng.integers(0, 2, size=P.N)
    ct = bgv.encrypt_slots(keys.pk, a, 1, 0)
    fresh = bgv.noise_bits(keys.sk, ct)
    cur = ct
    for _ in range(3):
        cur = bgv.mul(cur, cur, keys.rlk)
        assert bgv.noise_bits(keys.sk, cur) < fresh + 8
    assert bgv.budget_bits(keys.sk, cur) > 10
    assert np.array_equal(bgv.decrypt_slots(keys.sk, cur).astype(np.int64), a)


@pytest.mark.parametrize("k", [1, 5])
def test_matmul_with_unit_diagonal_is_rotation(k):
    """ModDown(U + P x) = ModDown(U) + x exactly, so a one-rotation product with the
    constant plaintext 1 must equal the rotation operation bit for bit."""
    logN = 6
    g = B.galois_rot(logN, k)
    P, bgv, keys = _setup(logN, 5, 50, 2, galois=[g])
    rng = np.random.default_rng(k)
    ct = bgv.encrypt_slots(keys.pk, rng.integers(0, T, size=P.N), 3, 0)
    one = B.encode(P, np.ones(P.N, dtype=np.int64))
    (got,) = bgv.matmul(ct, [g], [keys.gk[g]], [[one]])
    assert np.array_equal(got, bgv.rotate(ct, g, keys.gk[g]))
    # the identity term alone is the plaintext product
    (ident,) = bgv.matmul(ct, [1], [None], [[one]])
    assert np.array_equal(ident, ct)


def test_matmul_slot_semantics():
    """Two accumulators over shared rotations decrypt to sum_i d_i * rot(v, i)."""
    logN = 6
    ks = [0, 1, 3, 10]
    gal = [B.galois_rot(logN, k) if k else 1 for k in ks]
    P, bgv, keys = _setup(logN, 5, 50, 2, galois=[g for g in gal if g != 1])
    rng = np.random.default_rng(2)
    v = rng.integers(0, 2, size=P.N)
    ct = bgv.encrypt_slots(keys.pk, v, 3, 0)
    diags = [[rng.integers(0, 3, size=P.N) for _ in ks], [rng.integers(0, 2, size=P.N) if j != 2 else None
                                                           for j in range(len(ks))]]
    pts = [[None if d is None else B.encode(P, d) for d in row] for row in diags]
    outs = bgv.matmul(ct, gal, [keys.gk[g] if g != 1 else None for g in gal], pts)
    for row, out in zip(diags, outs):
        want = np.zeros(P.N, dtype=np.int64)
        for k, d in zip(ks, row):
            if d is not None:
                want = (want + d * _rot(v, k, P.N)) % T
        assert np.array_equal(bgv.decrypt_slots(keys.sk, out).astype(np.int64), want)


def test_relin_drop_without_third_component_is_modswitch():
    """With d2 = 0 the key-switching sum vanishes and the ModDown over P q_{ell-1} of
    P (d0, d1) is exactly the modulus switch of (d0, d1): an identity between two
    independently written routines."""
    P, bgv, keys = _setup(6, 5, 50, 2)
    rng = np.random.default_rng(8)
    ct = bgv.encrypt_slots(keys.pk, rng.integers(0, T, size=P.N), 3, 0)
    ct3 = np.concatenate([ct, np.zeros((1,) + ct.shape[1:], dtype=np.uint64)])
    assert np.array_equal(bgv.relin_drop(ct3, keys.rlk), bgv.modswitch(ct))


@pytest.mark.parametrize("logN,L,dnum", [(6, 5, 2), (10, 6, 3)])
def test_relin_drop_decrypts_like_two_step_path(logN, L, dnum):
    P, bgv, keys = _setup(logN, L, 50, dnum)
    rng = np.random.default_rng(logN + L)
    a, b = rng.integers(0, T, size=P.N), rng.integers(0, T, size=P.N)
    ca, cb = bgv.encrypt_slots(keys.pk, a, 5, 0), bgv.encrypt_slots(keys.pk, b, 5, 1)
    t3 = bgv.tensor(ca, cb)
    one = bgv.relin_drop(t3, keys.rlk)
    two = bgv.modswitch(bgv.relin(t3, keys.rlk))
    assert one.shape == two.shape == (2, L - 1, P.N)
    want = (a * b) % T
    assert np.array_equal(bgv.decrypt_slots(keys.sk, one).astype(np.int64), want)
    assert np.array_equal(bgv.decrypt_slots(keys.sk, two).astype(np.int64), want)
    # one rounding instead of two: no more noise than the two-step path (within a bit)
    assert bgv.noise_bits(keys.sk, one) <= bgv.noise_bits(keys.sk, two) + 1
