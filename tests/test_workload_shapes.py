"""The synthetic workloads have the shapes their recipe states (the paper's datasets
are not here, so seeded forests of the configured shapes stand in): tree counts,
depths, branch and leaf counts, features, precision and classes of every forest,
and, compiled by the oracle, the layout the benchmark's headline relies on (the
encrypted 8160-branch model in two row segments of one slot row each at N = 2^15)."""
import pytest

from oracle import copse as Cp
from paper_2104_09583_gb300 import synth


def _shape(text):
    labels, trees = Cp.parse_forest(text)

    def walk(n, dep):
        if n.leaf:
            return 0, 1, dep, set()
        a = walk(n.left, dep + 1)
        b = walk(n.right, dep + 1)
        return a[0] + b[0] + 1, a[1] + b[1], max(a[2], b[2]), a[3] | b[3] | {n.feature}
    per = [walk(t, 0) for t in trees]
    return {"classes": len(labels), "trees": len(trees), "branches": sum(p[0] for p in per),
            "leaves": sum(p[1] for p in per), "depth": max(p[2] for p in per),
            "features": set().union(*(p[3] for p in per))}


@pytest.mark.parametrize("name", sorted(synth.WORKLOADS))
def test_forests_follow_their_recipe(name):
    W = synth.WORKLOADS[name]
    for (seed, n_trees, depth, nf, p, nc, complete, branches), text in zip(W.forests, W.forest_texts()):
        s = _shape(text)
        assert s["classes"] == nc and s["trees"] == n_trees
        assert s["depth"] <= depth and s["features"] <= set(range(nf))
        assert s["leaves"] == s["branches"] + n_trees            # binary trees: L = b + #trees
        if complete:
            assert s["depth"] == depth and s["branches"] == n_trees * (2 ** depth - 1)
        if branches:
            assert branches[0] <= s["branches"] <= branches[1]
        _, trees = Cp.parse_forest(text)
        assert all(0 <= t < 2 ** p for t in Cp._thresholds(trees))
    for (_, _, _, nf, p, _, _, _), qs, n in zip(W.forests, W.query_arrays(), W.queries):
        assert len(qs) == n and all(len(x) == nf and all(0 <= v < 2 ** p for v in x) for x in qs)


def test_headline_encrypted_model_layout():
    W = synth.WORKLOADS["encmodel32-n32768"]
    m = Cp.compile_forest(W.forest_texts()[0], W.precision(), W.n_features(), slots_per_row=1 << (W.log_n - 1))
    assert (m.b_total, m.L_total, m.d) == (8160, 8192, 8)
    assert m.n_seg == 2 and m.block * m.n_seg == 1 << W.log_n    # one query spans both slot rows
    assert m.q == m.K * 32 and m.q == 4736
    # Table 1d: p + q + d(b+1) ciphertexts of the encrypted model, b one slot block's branches
    assert m.precision + m.q + m.d * (m.b + 1) == 37400
