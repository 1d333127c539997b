"""Pins of the oracle's row-segment layout: a forest whose query block would not fit
a slot row is split into contiguous groups of trees, each compiled alike (common K,
q, d), with query j owning blocks j*n_seg + s.  The layout is this implementation's
reading; what it must preserve is the paper's result (Section 4.1.2, Classification
Result): every query's leaf bits equal the plaintext tree walk, in the cleartext slot
circuit and after decryption, for plaintext and encrypted models."""
import numpy as np
import pytest

from oracle import bgv as B
from oracle import copse as Cp
from paper_2104_09583_gb300 import synth

LOGN = 10
ROW = 1 << (LOGN - 1)


def _forest():
    # 8 complete trees of depth 5 over 2 features: one block would need 1024 slots
    return synth.random_forest(8181, 8, 5, 2, 6, 3, complete=True)


def test_segments_compile():
    text = _forest()
    whole = Cp.compile_forest(text, 6, 2)
    assert whole.block > ROW
    m = Cp.compile_forest(text, 6, 2, slots_per_row=ROW)
    assert m.n_seg == 2 and m.block <= ROW and m.n_seg * m.block <= 2 * ROW
    assert (m.b_total, m.L_total) == (whole.b, whole.L)
    # the segments are the two halves of the trees, in order
    labels, trees = Cp.parse_forest(text)
    halves = ["\n".join([" ".join(labels)] + text.strip().splitlines()[1 + 4 * h: 5 + 4 * h]) for h in range(2)]
    for sg, ht in zip(m.segs, halves):
        alone = Cp.compile_forest(ht, 6, 2)
        assert (sg.b, sg.L) == (alone.b, alone.L)
        assert sg.K == m.K and sg.q == m.q and sg.d == m.d
        # same reshuffle matrix up to the common K (columns grouped per feature)
        for i in range(alone.b):
            j_alone = alone.slot_branch.index(i)
            f, r = divmod(j_alone, alone.K)
            assert sg.slot_branch[f * m.K + r] == i
    # leaf order: segment 0's leaves, then segment 1's (preorder across the trees)
    assert sum(sg.L for sg in m.segs) == whole.L


def test_segments_slot_circuit_equals_plain():
    text = _forest()
    m = Cp.compile_forest(text, 6, 2, slots_per_row=ROW)
    N = 2 * ROW
    nq = N // (m.block * m.n_seg)
    qs = synth.random_queries(8182, nq, 2, 6)
    slots = Cp.infer(Cp.SlotEngine(N), m, list(Cp.feature_planes(m, qs, N)), N)
    _, trees = Cp.parse_forest(text)
    for j, bits in enumerate(Cp.decode_labels(m, slots, nq)):
        assert bits == Cp.classify_plain(trees, qs[j]), j


@pytest.mark.parametrize("encrypted", [False, True])
def test_segments_bgv_inference(encrypted):
    text = _forest()
    m = Cp.compile_forest(text, 6, 2, slots_per_row=ROW)
    g = (16, 16)
    P = B.Params(logN=LOGN, L=Cp.levels_needed(m) + 1, bits=50, dnum=3)
    bgv = B.Bgv(P)
    rs, ls = Cp.encrypted_rotation_sets(m, g) if encrypted else Cp.rotation_sets(m, g)
    keys = bgv.keygen(91, sorted(set(B.galois_rot(LOGN, k) for k in rs + ls)))
    nq = P.N // (m.block * m.n_seg)
    qs = synth.random_queries(8183, nq, 2, 6)
    X = Cp.encrypt_queries(bgv, keys, m, qs, 19)
    if encrypted:
        em = Cp.encrypt_model(bgv, keys.sk, m, P.N, 5050, g)
        E = Cp.BgvEngine(bgv, keys, encrypted_model=True, enc_model=em)
        out = Cp.infer(E, m, X, P.N)
    else:
        out = Cp.infer(Cp.BgvEngine(bgv, keys), m, X, P.N, g)
    slots = bgv.decrypt_slots(keys.sk, out).astype(np.int64)
    _, trees = Cp.parse_forest(text)
    for j, bits in enumerate(Cp.decode_labels(m, slots, nq)):
        assert bits == Cp.classify_plain(trees, qs[j]), j
