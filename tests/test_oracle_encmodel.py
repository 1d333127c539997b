"""Pins of the oracle's encrypted-model mode (Maurice = Diane, Section 8.3):
secret-key encryption with a seeded mask decrypts to its plaintext and its
mask's evaluations are the seeded uniform residues; SecComp against encrypted
thresholds equals integer '<' exhaustively; whole inferences on encrypted
models (plain and baby-step / giant-step products) decrypt to plaintext
classification, with the encrypted ciphertext count of Table 1d."""
import numpy as np
import pytest

from oracle import bgv as B
from oracle import copse as Cp
from paper_2104_09583_gb300 import synth

T = 65537


def test_secret_key_encryption_decrypts_and_mask_is_seeded():
    P = B.Params(logN=6, L=4, bits=50, dnum=2)
    bgv = B.Bgv(P)
    keys = bgv.keygen(21)
    rng = np.random.default_rng(2)
    v = rng.integers(0, T, size=P.N)
    for ell in (4, 2):
        ct = bgv.encrypt_sk(keys.sk, B.encode(P, v), 99, 7, ell)
        assert ct.shape == (2, ell, P.N)
        assert np.array_equal(bgv.decrypt_slots(keys.sk, ct).astype(np.int64), v)
        # c1 evaluated directly at psi^(2j+1) equals the uniform residue drawn for (prime r, index j)
        for r in range(ell):
            q = P.q[r]
            psi = B.lib().or_root_2n(q, P.logN)
            ev = np.zeros(P.N, dtype=np.uint64)
            B.lib().or_eval_direct(np.ascontiguousarray(ct[1, r]), P.logN, q, psi, ev)
            for j in (0, 1, P.N - 1):
                hi = B.lib().or_word(99, B.stream_model(7), 2 * (r * P.N + j))
                lo = B.lib().or_word(99, B.stream_model(7), 2 * (r * P.N + j) + 1)
                assert int(ev[j]) == ((int(hi) << 64) | int(lo)) % q


@pytest.mark.parametrize("p", [2, 3])
def test_seccomp_encrypted_thresholds_exhaustive(p):
    n = 1 << p
    logN = 7
    N = 1 << logN
    x = np.zeros(N, dtype=np.int64)
    y = np.zeros(N, dtype=np.int64)
    x[: n * n] = np.repeat(np.arange(n), n)
    y[: n * n] = np.tile(np.arange(n), n)
    P = B.Params(logN=logN, L=4, bits=50, dnum=2)
    bgv = B.Bgv(P)
    keys = bgv.keygen(3)
    X = [bgv.encrypt_slots(keys.pk, (x >> i) & 1, 8, i) for i in range(p)]
    Y = [bgv.encrypt_sk(keys.sk, B.encode(P, (y >> i) & 1), 5, i, P.L) for i in range(p)]
    E = Cp.BgvEngine(bgv, keys, encrypted_model=True, enc_model={"thresholds": Y})
    D = Cp.seccomp(E, X, Y, p)
    got = bgv.decrypt_slots(keys.sk, D).astype(np.int64)
    assert np.array_equal(got[: n * n], (x < y).astype(np.int64)[: n * n])


CASES = [
    (synth.random_forest(1001, 1, 3, 2, 4, 2), 4, 2, (0, 0)),
    (synth.random_forest(77, 3, 4, 3, 5, 3, complete=False), 5, 3, (4, 3)),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_encrypted_model_inference(case):
    text, p, nf, g = CASES[case]
    m = Cp.compile_forest(text, p, nf)
    logN = 10
    P = B.Params(logN=logN, L=Cp.levels_needed(m) + 1, bits=50, dnum=3)
    bgv = B.Bgv(P)
    rs, ls = Cp.encrypted_rotation_sets(m, g)
    keys = bgv.keygen(31, sorted(set(B.galois_rot(logN, k) for k in rs + ls)))
    em = Cp.encrypt_model(bgv, keys.sk, m, P.N, 4040, g)
    n_ct = len(em["thresholds"]) + len(em["R"]) + sum(len(x) for x in em["levels"]) + len(em["masks"])
    assert n_ct == m.precision + m.q + m.d * (m.b + 1)          # Table 1d
    nq = P.N // m.block
    qs = synth.random_queries(600 + case, nq, nf, p)
    X = Cp.encrypt_queries(bgv, keys, m, qs, 12)
    E = Cp.BgvEngine(bgv, keys, encrypted_model=True, enc_model=em)
    out = Cp.infer(E, m, X, P.N)
    slots = bgv.decrypt_slots(keys.sk, out).astype(np.int64)
    ref = Cp.infer(Cp.SlotEngine(P.N), m, list(Cp.feature_planes(m, qs, P.N)), P.N)
    assert np.array_equal(slots, ref)
    _, trees = Cp.parse_forest(text)
    for j, bits in enumerate(Cp.decode_labels(m, slots, nq)):
        assert bits == Cp.classify_plain(trees, qs[j]), j
    assert out.shape[1] == P.L - Cp.levels_needed(m)
    assert bgv.budget_bits(keys.sk, out) > 5
