"""Pins of the oracle's baby-step / giant-step matrix products (the BSGS form
of the diagonal method of Section 4.1.2).  In the clear, every product equals
numpy's matrix-vector product, block by block; encrypted, it decrypts to the
same; a baby-step size at least the matrix width reproduces the plain
diagonal method ciphertext for ciphertext; the giant-step sum decrypts to
the sum of explicitly permuted slot vectors; whole inferences decrypt to
plaintext classification with fewer rotation keys."""
import numpy as np
import pytest

from oracle import bgv as B
from oracle import copse as Cp
from paper_2104_09583_gb300 import synth

T = 65537


def _rot(v, k, N):
    h = N // 2
    return np.concatenate([np.roll(v[:h], -k), np.roll(v[h:], -k)])


def _model():
    return Cp.compile_forest(synth.random_forest(77, 3, 4, 3, 5, 3, complete=False), 5, 3)


def _periodic(m, x, n, length, N, rng_blocks):
    """per block: x_blk[j mod n] over `length` slots (a different x per block)"""
    out = np.zeros(N, dtype=np.int64)
    for blk, xb in enumerate(rng_blocks):
        out[blk * m.block: blk * m.block + length] = xb[np.arange(length) % n]
    return out


@pytest.mark.parametrize("g", [1, 2, 3, 5, 8, 1000])
def test_bsgs_reshuffle_cleartext_equals_numpy(g):
    m = _model()
    N = 1024
    nb = N // m.block
    rng = np.random.default_rng(g)
    xs = [rng.integers(0, 2, size=m.q) for _ in range(nb)]
    v = _periodic(m, None, m.q, m.pd, N, xs)
    E = Cp.SlotEngine(N)
    Br = Cp.matmul(E, v, [Cp.reshuffle_diagonals(m)], [None], m, N, g)[0]
    for blk, x in enumerate(xs):
        want = (m.R.astype(np.int64) @ x)[np.arange(m.m1) % m.b]
        assert np.array_equal(Br[blk * m.block: blk * m.block + m.m1], want), f"block {blk}"
        assert not Br[blk * m.block + m.m1: (blk + 1) * m.block].any()


@pytest.mark.parametrize("g", [1, 2, 4, 7])
def test_bsgs_levels_cleartext_equals_numpy(g):
    m = _model()
    N = 1024
    nb = N // m.block
    rng = np.random.default_rng(10 + g)
    bs = [rng.integers(0, 2, size=m.b) for _ in range(nb)]
    v = _periodic(m, None, m.b, m.m1, N, bs)
    E = Cp.SlotEngine(N)
    masks = [Cp.tile_blocks(m, m.mask[k - 1], N) for k in range(1, m.d + 1)]
    res = Cp.matmul(E, v, [Cp.level_diagonals(m, k, T) for k in range(1, m.d + 1)], masks, m, N, g)
    for k in range(1, m.d + 1):
        for blk, x in enumerate(bs):
            z = m.lvl[k - 1].astype(np.int64) @ x
            want = z ^ m.mask[k - 1].astype(np.int64)          # Lvl_k * Branches XOR Mask_k
            assert np.array_equal(res[k - 1][blk * m.block: blk * m.block + m.L], want), (k, blk)


def test_bsgs_rotation_counts():
    m = _model()
    rs0, ls0 = Cp.rotation_sets(m)
    for g in (2, 3, 4):
        rs, ls = Cp.rotation_sets(m, (g, g))
        babies = set(i % g for i in Cp.reshuffle_diagonals(m)) - {0}
        giants = set(i - i % g for i in Cp.reshuffle_diagonals(m)) - {0}
        assert set(rs) == babies | giants
        assert len(rs) <= (g - 1) + (m.q - 1) // g
    # a baby step at least the width needs exactly the plain method's rotations
    assert Cp.rotation_sets(m, (m.q, m.b)) == (rs0, ls0)


@pytest.fixture(scope="module")
def enc():
    m = _model()
    P = B.Params(logN=10, L=10, bits=50, dnum=3)
    bgv = B.Bgv(P)
    gal = sorted(set(Cp.galois_elements(m, 10)) | set(Cp.galois_elements(m, 10, (3, 4))))
    keys = bgv.keygen(99, gal)
    return m, P, bgv, keys


def test_rotsum_decrypts_to_permuted_sum(enc):
    m, P, bgv, keys = enc
    rng = np.random.default_rng(5)
    vals = [rng.integers(0, T, size=P.N) for _ in range(3)]
    cts = [bgv.encrypt_slots(keys.pk, v, 7, i) for i, v in enumerate(vals)]
    ks = [3, 0, 6]
    gal = [B.galois_rot(P.logN, k) if k else 1 for k in ks]
    out = bgv.rotsum(cts, gal, [keys.gk[g] if g != 1 else None for g in gal])
    want = sum(_rot(v, k, P.N) for v, k in zip(vals, ks)) % T
    assert np.array_equal(bgv.decrypt_slots(keys.sk, out).astype(np.int64), want)


def test_bsgs_encrypted_matches_numpy_and_plain_limit(enc):
    m, P, bgv, keys = enc
    N = P.N
    nb = N // m.block
    rng = np.random.default_rng(31)
    xs = [rng.integers(0, 2, size=m.q) for _ in range(nb)]
    v = _periodic(m, None, m.q, m.pd, N, xs)
    ct = bgv.encrypt_slots(keys.pk, v, 3, 0)
    E = Cp.BgvEngine(bgv, keys)
    Br3 = Cp.matmul(E, ct, [Cp.reshuffle_diagonals(m)], [None], m, N, 3)[0]
    got = bgv.decrypt_slots(keys.sk, Br3).astype(np.int64)
    for blk, x in enumerate(xs):
        want = (m.R.astype(np.int64) @ x)[np.arange(m.m1) % m.b]
        assert np.array_equal(got[blk * m.block: blk * m.block + m.m1], want)
    # g >= q: one giant step, the plain method's ciphertext exactly
    plain = Cp.matmul(E, ct, [Cp.reshuffle_diagonals(m)], [None], m, N, 0)[0]
    wide = Cp.matmul(E, ct, [Cp.reshuffle_diagonals(m)], [None], m, N, m.q)[0]
    assert np.array_equal(plain, wide)
    assert not np.array_equal(plain, Br3)     # a different (equally valid) rounding


def test_bsgs_inference_decrypts_to_plaintext_classification(enc):
    m, P, bgv, keys = enc
    text = synth.random_forest(77, 3, 4, 3, 5, 3, complete=False)
    nq = P.N // m.block
    qs = synth.random_queries(4242, nq, 3, 5)
    X = Cp.encrypt_queries(bgv, keys, m, qs, 17)
    E = Cp.BgvEngine(bgv, keys)
    out = Cp.infer(E, m, X, P.N, (3, 4))
    slots = bgv.decrypt_slots(keys.sk, out).astype(np.int64)
    ref = Cp.infer(Cp.SlotEngine(P.N), m, list(Cp.feature_planes(m, qs, P.N)), P.N, (3, 4))
    assert np.array_equal(slots, ref)
    _, trees = Cp.parse_forest(text)
    for j, bits in enumerate(Cp.decode_labels(m, slots, nq)):
        assert bits == Cp.classify_plain(trees, qs[j])
    rs, ls = Cp.rotation_sets(m, (3, 4))
    assert E.counts["rot"] <= len(rs) + m.d * len(set(ls))
    assert out.shape[1] == P.L - Cp.levels_needed(m)
