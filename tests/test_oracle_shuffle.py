"""Pins of the oracle's label shuffle with padding (Section 7.2, "Returning
classification bitvectors"): in the clear the shuffled result is numpy's
fancy-indexed permutation of the unshuffled one with zeros at the padding
slots; encrypted it decrypts to the same; the shuffled codebook, read
through the bits, gives each tree's class exactly as the plaintext walk."""
import numpy as np
import pytest

from oracle import bgv as B
from oracle import copse as Cp
from paper_2104_09583_gb300 import synth


def _setup(case):
    text = [synth.random_forest(77, 3, 4, 3, 5, 3, complete=False), synth.random_forest(1001, 1, 3, 2, 4, 2)][case]
    p, nf = [(5, 3), (4, 2)][case]
    m = Cp.compile_forest(text, p, nf)
    return text, p, nf, m


def test_shuffle_plan_is_a_padded_permutation():
    _, _, _, m = _setup(0)
    src, code = synth.shuffle_plan(9, m.labels_per_leaf, 7, 3)
    assert len(src) == m.L + 7 == len(code)
    assert sorted(i for i in src if i >= 0) == list(range(m.L))
    assert sum(1 for i in src if i < 0) == 7
    for j, i in enumerate(src):
        if i >= 0:
            assert code[j] == m.labels_per_leaf[i]


@pytest.mark.parametrize("case", [0, 1])
def test_shuffle_cleartext_is_numpy_permutation(case):
    text, p, nf, m = _setup(case)
    N = 1024
    nq = N // m.block
    qs = synth.random_queries(31 + case, nq, nf, p)
    S = Cp.SlotEngine(N)
    X = list(Cp.feature_planes(m, qs, N))
    plain = Cp.infer(S, m, X, N)
    src, _ = synth.shuffle_plan(5 + case, m.labels_per_leaf, m.block - m.L, 3)
    shuf = Cp.infer(S, m, X, N, shuffle=src)
    for blk in range(nq):
        base = blk * m.block
        want = np.where(src >= 0, plain[base + np.maximum(src, 0)], 0)
        assert np.array_equal(shuf[base: base + len(src)], want), blk
        assert not shuf[base + len(src): base + m.block].any()


def test_shuffle_encrypted_decrypts_and_codebook_classifies():
    text, p, nf, m = _setup(0)
    logN = 10
    src, code = synth.shuffle_plan(17, m.labels_per_leaf, 9, 3)
    P = B.Params(logN=logN, L=Cp.levels_needed(m, shuffle=True) + 1, bits=50, dnum=3)
    bgv = B.Bgv(P)
    keys = bgv.keygen(7, sorted(set(Cp.galois_elements(m, logN)) | set(Cp.shuffle_galois(m, src, logN))))
    nq = P.N // m.block
    qs = synth.random_queries(44, nq, nf, p)
    X = Cp.encrypt_queries(bgv, keys, m, qs, 3)
    out = Cp.infer(Cp.BgvEngine(bgv, keys), m, X, P.N, shuffle=src)
    slots = bgv.decrypt_slots(keys.sk, out).astype(np.int64)
    ref = Cp.infer(Cp.SlotEngine(P.N), m, list(Cp.feature_planes(m, qs, P.N)), P.N, shuffle=src)
    assert np.array_equal(slots, ref)
    _, trees = Cp.parse_forest(text)
    for j, bits in enumerate(Cp.decode_labels(m, slots, nq, len(src))):
        walk = Cp.classify_plain(trees, qs[j])
        chosen = sorted(int(code[k]) for k in range(len(src)) if bits[k])
        assert chosen == sorted(m.labels_per_leaf[i] for i in range(m.L) if walk[i]), j
        assert sum(bits) == len(trees)
    assert out.shape[1] == P.L - Cp.levels_needed(m, shuffle=True)
