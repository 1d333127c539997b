"""Pins of the oracle's fused level products: Algorithm 1 multiplies Decisions by the
reshuffling matrix R (Section 4.2.2) and Branches by each level matrix (Section 4.2.3);
folding the two into F_k = S_k R (S_k the level matrix with the mask's XOR folded in as
signs) must give, slot for slot, the same cleartext result as the two products, and
after decryption the plaintext tree walk, with one prime fewer."""
import numpy as np
import pytest

from conftest import read_golden
from oracle import bgv as B
from oracle import copse as Cp
from paper_2104_09583_gb300 import synth

T = 65537


def _forests():
    return [(read_golden("fig1_forest.txt"), 4, 2, 0),
            (synth.random_forest(61, 3, 4, 3, 5, 3, complete=False), 5, 3, 0),
            (synth.random_forest(62, 2, 5, 4, 6, 3, complete=True), 6, 4, 0),
            (synth.random_forest(8181, 8, 5, 2, 6, 3, complete=True), 6, 2, 512)]  # row segments at N = 2^10


@pytest.mark.parametrize("case", range(4))
def test_fused_matrix_structure(case):
    text, p, nf, row = _forests()[case]
    m = Cp.compile_forest(text, p, nf, slots_per_row=row)
    for sg in Cp.parts(m):
        for k in range(1, m.d + 1):
            F = Cp.fused_matrix(m, k, sg)
            assert F.shape == (sg.L, m.q)
            for leaf in range(sg.L):
                nz = np.nonzero(F[leaf])[0]
                picked = np.nonzero(sg.lvl[k - 1][leaf])[0]
                assert len(nz) == len(picked) <= 1
                if len(nz):
                    # the one entry sits at the padded slot of the branch the level matrix picks,
                    # with sign -1 exactly when the leaf lies under that branch's true child
                    assert sg.slot_branch[nz[0]] == picked[0]
                    assert F[leaf, nz[0]] == (-1 if sg.mask[k - 1][leaf] else 1)


@pytest.mark.parametrize("case", range(4))
def test_fused_slots_equal_two_products(case):
    text, p, nf, row = _forests()[case]
    m = Cp.compile_forest(text, p, nf, slots_per_row=row)
    N = 1024
    nq = N // (m.block * m.n_seg)
    qs = synth.random_queries(700 + case, nq, nf, p)
    X = list(Cp.feature_planes(m, qs, N))
    E = Cp.SlotEngine(N)
    two = Cp.infer(E, m, X, N)
    fused = Cp.infer(E, m, X, N, fused=True)
    assert np.array_equal(two, fused)
    _, trees = Cp.parse_forest(text)
    for j, bits in enumerate(Cp.decode_labels(m, fused, nq)):
        assert bits == Cp.classify_plain(trees, qs[j])


@pytest.mark.parametrize("g", [0, 4])
def test_fused_bgv_inference(g):
    text, p, nf, _ = _forests()[1]
    m = Cp.compile_forest(text, p, nf)
    logN = 10
    P = B.Params(logN=logN, L=Cp.levels_needed(m, fused=True) + 1, bits=50, dnum=3)
    bgv = B.Bgv(P)
    keys = bgv.keygen(5, Cp.galois_elements(m, logN, (g, 0), fused=True))
    nq = P.N // m.block
    qs = synth.random_queries(81, nq, nf, p)
    X = Cp.encrypt_queries(bgv, keys, m, qs, 3)
    out = Cp.infer(Cp.BgvEngine(bgv, keys), m, X, P.N, (g, 0), fused=True)
    assert out.shape[1] == P.L - Cp.levels_needed(m, fused=True)
    assert Cp.levels_needed(m, fused=True) == Cp.levels_needed(m) - 1
    slots = bgv.decrypt_slots(keys.sk, out).astype(np.int64)
    _, trees = Cp.parse_forest(text)
    for j, bits in enumerate(Cp.decode_labels(m, slots, nq)):
        assert bits == Cp.classify_plain(trees, qs[j]), j
    rs, ls = Cp.rotation_sets(m, (g, 0), fused=True)
    assert rs == [] and all(0 < a < m.q for a in ls)
