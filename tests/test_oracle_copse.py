"""Pins of the oracle's COPSE layer: the worked example of Fig. 1, the
structural properties Section 4.2 states for the padded threshold vector, the
reshuffling matrix and the level matrices, SecComp against integer '<' over
every input pair, and whole inferences against the plaintext tree walk."""
import numpy as np
import pytest

from conftest import read_golden
from oracle import bgv as B
from oracle import copse as Cp
from paper_2104_09583_gb300 import synth

T = 65537


def test_fig1_worked_example():
    text = read_golden("fig1_forest.txt")
    m = Cp.compile_forest(text, 4, 2)
    # Section 3.3 / 4.1.1: K = 3 (y at d0, d2, d4), b = 5, q = K * 2 = 6; 6 labels, max level 3
    assert (m.K, m.b, m.q, m.L, m.d) == (3, 5, 6, 6, 3)
    # levels (Section 4.1.1): d2, d3, d4 at level 1 (Section 3.3, Step 3), d1 at 2, d0 at 3
    assert m.br_level == [3, 2, 1, 1, 1]
    # Section 3.3, Step 0: replicated features [x, x, x, y, y, y]
    assert [(s % m.q) // m.K for s in range(m.q)] == [0, 0, 0, 1, 1, 1]
    # padded thresholds grouped by feature: x-group (d1, d3, S), y-group (d0, d2, d4)
    assert m.slot_branch == [1, 3, -1, 0, 2, 4]
    assert m.thr_slot == [4, 12, 0, 9, 3, 4]
    ones = sorted(zip(*np.nonzero(m.R)))
    assert ones == [(0, 3), (1, 0), (2, 4), (3, 1), (4, 5)]
    assert not m.R[:, 2].any()
    # Section 3.3, Step 3: at level 1, L0, L2, L4 are on the false sides (mask 1)
    assert m.mask[0].tolist() == [1, 0, 1, 0, 1, 0]
    # level 2: d1 above L0..L3; d4 stands in for L4, L5 (Section 4.2.3)
    assert m.mask[1].tolist() == [1, 1, 0, 0, 1, 0]
    assert m.lvl[1][4].tolist() == [0, 0, 0, 0, 1] and m.lvl[1][5].tolist() == [0, 0, 0, 0, 1]
    assert m.mask[2].tolist() == [1, 1, 1, 1, 0, 0]
    # Section 2.1: (x, y) = (0, 5) is assigned L4
    _, trees = Cp.parse_forest(text)
    assert Cp.classify_plain(trees, [0, 5]) == [0, 0, 0, 0, 1, 0]


def _forests():
    out = [read_golden("fig1_forest.txt")]
    for s in range(6):
        out.append(synth.random_forest(50 + s, 1 + s % 3, 2 + s % 4, 1 + s % 5, 6, 3, complete=(s % 2 == 0)))
    # a forest whose second tree is a single leaf
    out.append("a b\nb 0 5 l 0 b 0 9 l 1 l 0\nl 1\n")
    return out


@pytest.mark.parametrize("text", _forests())
def test_structure_invariants(text):
    m = Cp.compile_forest(text, 6)
    _, trees = Cp.parse_forest(text)
    # Section 4.2.2: one 1 per row of R, at most one per column, empty columns are sentinels
    assert np.all(m.R.sum(1) == 1)
    assert np.all(m.R.sum(0) <= 1)
    assert [bool(m.R[:, j].any()) for j in range(m.q)] == [i >= 0 for i in m.slot_branch]
    assert all(m.thr_slot[j] == 0 for j in range(m.q) if m.slot_branch[j] < 0)
    # Section 4.1.1: b = sum of multiplicities, q = K * n_features
    assert m.b == sum(m.br_feature.count(f) for f in range(m.n_features)) and m.q == m.K * m.n_features
    # leaf widths
    width = [0] * m.b

    def walk(n, anc):
        if n.leaf:
            for i in anc:
                width[i] += 1
            return
        i = walk.idx
        walk.idx += 1
        walk(n.left, anc + [i])
        walk(n.right, anc + [i])
    walk.idx = 0
    for t in trees:
        walk(t, [])
    seen = set()
    for k in range(1, m.d + 1):
        M = m.lvl[k - 1]
        rows = M.sum(1)
        # one 1 per row (Section 4.2.3), except a leaf that is a whole tree
        assert np.all((rows == 1) | ((rows == 0) & (m.mask[k - 1] == 1)))
        for j in range(m.b):
            col = int(M[:, j].sum())
            assert col <= width[j]
            if m.br_level[j] == k:
                assert col == width[j]
                seen.add(j)
    # every branch is represented in at least one level
    assert seen == set(range(m.b))


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
def test_seccomp_exhaustive_cleartext(p):
    n = 1 << p
    x = np.repeat(np.arange(n), n)
    y = np.tile(np.arange(n), n)
    N = 2 * len(x)
    X = [np.concatenate([(x >> i) & 1, np.zeros(N - len(x), dtype=np.int64)]) for i in range(p)]
    Y = [np.concatenate([(y >> i) & 1, np.zeros(N - len(x), dtype=np.int64)]) for i in range(p)]
    E = Cp.SlotEngine(N)
    D = Cp.seccomp(E, X, Y, p)
    assert np.array_equal(D[: len(x)], (x < y).astype(np.int64))


@pytest.mark.parametrize("p,logN", [(3, 7), (6, 12)])
def test_seccomp_exhaustive_encrypted(p, logN):
    """Every (x, y) in [0, 2^p)^2 in one ciphertext's slots, thresholds in plaintext."""
    n = 1 << p
    N = 1 << logN
    assert n * n <= N
    x = np.zeros(N, dtype=np.int64)
    y = np.zeros(N, dtype=np.int64)
    x[: n * n] = np.repeat(np.arange(n), n)
    y[: n * n] = np.tile(np.arange(n), n)
    L = 1 + (p - 1).bit_length() + 1
    P = B.Params(logN=logN, L=L, bits=50, dnum=2)
    bgv = B.Bgv(P)
    keys = bgv.keygen(3)
    X = [bgv.encrypt_slots(keys.pk, (x >> i) & 1, 8, i) for i in range(p)]
    Y = [(y >> i) & 1 for i in range(p)]
    E = Cp.BgvEngine(bgv, keys)
    D = Cp.seccomp(E, X, Y, p)
    got = bgv.decrypt_slots(keys.sk, D).astype(np.int64)
    assert np.array_equal(got[: n * n], (x < y).astype(np.int64)[: n * n])
    assert D.shape[1] == P.L - 1 - (p - 1).bit_length()


def _run_inference(text, precision, nf, logN, bits, queries, seed=11):
    m = Cp.compile_forest(text, precision, nf)
    L = Cp.levels_needed(m) + 1
    P = B.Params(logN=logN, L=L, bits=bits, dnum=3)
    bgv = B.Bgv(P)
    keys = bgv.keygen(seed, Cp.galois_elements(m, logN))
    X = Cp.encrypt_queries(bgv, keys, m, queries, seed + 1)
    E = Cp.BgvEngine(bgv, keys)
    out = Cp.infer(E, m, X, P.N)
    return m, P, bgv, keys, out, E


@pytest.mark.parametrize("case", range(4))
def test_inference_matches_plaintext_walk(case):
    specs = [
        (read_golden("fig1_forest.txt"), 4, 2, 7),
        (synth.random_forest(1001, 1, 3, 2, 4, 2), 4, 2, 10),
        (synth.random_forest(77, 3, 4, 3, 5, 3, complete=False), 5, 3, 10),
        ("a b\nb 0 5 l 0 b 0 9 l 1 l 0\nl 1\n", 4, 1, 7),
    ]
    text, p, nf, logN = specs[case]
    m = Cp.compile_forest(text, p, nf)
    nq = (1 << logN) // m.block
    qs = synth.random_queries(500 + case, nq, nf, p)
    m, P, bgv, keys, out, E = _run_inference(text, p, nf, logN, 50, qs)
    slots = bgv.decrypt_slots(keys.sk, out).astype(np.int64)
    # every slot equals the cleartext circuit
    S = Cp.SlotEngine(P.N)
    ref = Cp.infer(S, m, list(Cp.feature_planes(m, qs, P.N)), P.N)
    assert np.array_equal(slots, ref)
    # labels equal the plaintext classification, one 1 per tree
    _, trees = Cp.parse_forest(text)
    for j, bits in enumerate(Cp.decode_labels(m, slots, nq)):
        assert bits == Cp.classify_plain(trees, qs[j])
        assert sum(bits) == len(trees)
    # levels consumed as the policy predicts; rotations: one key switch per distinct amount
    assert out.shape[1] == P.L - Cp.levels_needed(m)
    rs, ls = Cp.rotation_sets(m)
    assert E.counts["rot"] == len(rs) + len(ls)
    # Table 2: the diagonal method needs at most q + d*b products
    assert E.counts["mul_plain"] - 2 * m.precision <= m.q + m.d * m.b
    assert bgv.budget_bits(keys.sk, out) > 10
