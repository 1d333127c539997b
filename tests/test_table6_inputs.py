"""The Table 6 microbenchmark forests (Section 8.4): the generator gives the
stated shape (max depth, precision, trees, branches, 2 features, 3 labels),
and the oracle's cleartext circuit classifies them like the plaintext trees."""
import numpy as np
import pytest

from oracle import copse as Cp
from paper_2104_09583_gb300 import synth


def _tree_depth_and_branches(tokens):
    pos = 0

    def walk():
        nonlocal pos
        kind = tokens[pos]
        if kind == "l":
            pos += 2
            return 0, 0
        pos += 3
        dl, bl = walk()
        dr, br = walk()
        return 1 + max(dl, dr), 1 + bl + br

    out = walk()
    assert pos == len(tokens)
    return out


@pytest.mark.parametrize("name", sorted(synth.TABLE6))
def test_table6_shape(name):
    depth, precision, per_tree = synth.TABLE6[name]
    text = synth.table6_forest(name)
    lines = text.strip().split("\n")
    assert len(lines[0].split()) == 3
    assert len(lines) - 1 == len(per_tree)
    depths = []
    for line, nb in zip(lines[1:], per_tree):
        toks = line.split()
        d, b = _tree_depth_and_branches(toks)
        assert b == nb
        depths.append(d)
        feats = [int(toks[i + 1]) for i in range(len(toks)) if toks[i] == "b"]
        thr = [int(toks[i + 2]) for i in range(len(toks)) if toks[i] == "b"]
        assert all(0 <= f < 2 for f in feats)
        assert all(0 <= v < (1 << precision) for v in thr)
    assert max(depths) == depth
    om = Cp.compile_forest(text, precision, 2)
    assert om.b == sum(per_tree) and om.d == depth


def test_table6_totals_match_the_printed_branch_counts():
    # Table 6: depth4/5/6, width78, prec8, prec16 have 15 branches; width55 10; width677 20 over 3 trees.
    total = {n: sum(v[2]) for n, v in synth.TABLE6.items()}
    assert total == {"depth4": 15, "depth5": 15, "depth6": 15, "width55": 10, "width78": 15,
                     "width677": 20, "prec8": 15, "prec16": 15}
    assert len(synth.TABLE6["width677"][2]) == 3


@pytest.mark.parametrize("name", ["depth6", "width677", "prec16"])
def test_table6_cleartext_circuit_classifies(name):
    depth, precision, _ = synth.TABLE6[name]
    text = synth.table6_forest(name)
    om = Cp.compile_forest(text, precision, 2)
    N = 1024
    nq = N // 2 // om.block
    qs = synth.random_queries(17, nq, 2, precision)
    _, trees = Cp.parse_forest(text)
    out = Cp.infer(Cp.SlotEngine(N), om, list(Cp.feature_planes(om, qs, N)), N)
    bits = Cp.decode_labels(om, out, nq)
    for j in range(nq):
        assert list(bits[j]) == Cp.classify_plain(trees, qs[j]), f"query {j}"
