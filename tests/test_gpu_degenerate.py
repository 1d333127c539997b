"""GPU parity on the degenerate forests the method allows, ciphertext for ciphertext
against the oracle (N = 2^10, tolerance zero), with labels against the plaintext
walk and every slot against the cleartext circuit:
  - one bit of precision and one branch: SecComp is a single plane with no combine
    product, the reshuffle a 1 x q matrix, MultAll a single level vector;
  - a tree that is a single leaf beside a branching tree: an empty row in every level
    matrix, mask 1 (Section 4.2.3 with the reading for leaves without ancestors);
  - odd plane and level counts (p = 3, a complete depth-3 tree): the balanced
    reductions of SecComp and MultAll carry an odd element at each round;
  - thresholds at the ends of the range, 0 (x < 0 never holds) and 2^p - 1, queried
    with features equal to the thresholds (the strict comparison of Section 4.1.1)."""
import itertools

import numpy as np
import pytest

from oracle import bgv as B
from oracle import copse as Cp
from paper_2104_09583_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
K = pytest.importorskip("paper_2104_09583_gb300.copse")

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

LOG_N, BITS, DNUM = 10, 50, 3

CASES = {
    "one-plane-one-branch": ("a b\nb 0 1 l 0 l 1\n", 1, 1),
    "single-leaf-tree": ("a b\nb 0 5 l 0 b 0 9 l 1 l 0\nl 1\n", 4, 1),
    "odd-planes-and-levels": (synth.random_forest(4040, 1, 3, 2, 3, 3, complete=True), 3, 2),
    "range-end-thresholds": ("a b\nb 0 0 l 0 b 1 15 l 1 l 0\n", 4, 2),
}


def _queries(name, m, p, nf, n):
    if name == "range-end-thresholds":
        ends = [0, 1, (1 << p) - 2, (1 << p) - 1]
        return [list(x) for x in itertools.product(ends, repeat=nf)][:n]
    return synth.random_queries(17 + len(name), n, nf, p)


@pytest.mark.parametrize("name", list(CASES))
def test_degenerate_forest_matches_oracle(name):
    text, p, nf = CASES[name]
    om = Cp.compile_forest(text, p, nf)
    L = Cp.levels_needed(om) + 1
    P = B.Params(logN=LOG_N, L=L, bits=BITS, dnum=DNUM)
    N = P.N
    qs = _queries(name, om, p, nf, min(16, N // om.block))
    ctx = K.copse_ctx_create(LOG_N, BITS, L, DNUM)
    try:
        assert K.copse_ctx_primes(ctx) == P.primes
        model = K.copse_compile_forest(text, p, nf, LOG_N)
        keys, evk = K.copse_keygen(ctx, 7, [model])
        feats = K.copse_encrypt_features(ctx, keys, model, qs, 99)
        res = K.copse_infer(ctx, evk, model, feats)
        got = K.copse_ctbuf_export(ctx, res, 0, N)
        bits = K.copse_decrypt_labels(ctx, keys, model, res, len(qs))
        slots = K.copse_decrypt_slots(ctx, keys, res, 0, N)
        for h in (res, feats):
            K.copse_ctbuf_destroy(h)
        K.copse_keys_destroy(keys)
        K.copse_evk_destroy(evk)
        K.copse_model_destroy(model)
    finally:
        K.copse_ctx_destroy(ctx)
    bgv = B.Bgv(P)
    okeys = bgv.keygen(7, Cp.galois_elements(om, LOG_N))
    X = Cp.encrypt_queries(bgv, okeys, om, qs, 99)
    want = Cp.infer(Cp.BgvEngine(bgv, okeys), om, X, N)
    got, want = np.asarray(got), np.asarray(want)
    assert got.shape == want.shape, (got.shape, want.shape)
    bad = np.argwhere(got != want)
    assert len(bad) == 0, f"first mismatch at (component, residue, coefficient) {tuple(bad[0])}, {len(bad)} in all"
    _, trees = Cp.parse_forest(text)
    for j, x in enumerate(qs):
        assert bits[j].tolist() == Cp.classify_plain(trees, x), f"query {j}"
    ref = Cp.infer(Cp.SlotEngine(N), om, list(Cp.feature_planes(om, qs, N)), N)
    assert np.array_equal(np.asarray(slots).astype(np.int64), ref)
