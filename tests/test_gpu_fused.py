"""Fused level products on the GPU (the reshuffle folded into every level matrix,
F_k = S_k R, applied to Decisions): whole inferences equal the oracle's coefficient
for coefficient at N = 2^10 (plain and baby-step / giant-step products, one block and
row segments), and at N = 2^14 the forest100 labels equal plaintext classification
with one prime fewer and fewer rotation keys than the two-product circuit."""
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

from test_gpu_parity import assert_same  # noqa: E402

CASES = [(synth.random_forest(61, 3, 4, 3, 5, 3, complete=False), 5, 3, 0),
         (synth.random_forest(61, 3, 4, 3, 5, 3, complete=False), 5, 3, 4),
         (synth.random_forest(8181, 8, 5, 2, 6, 3, complete=True), 6, 2, 16)]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_fused_inference_matches_oracle(case):
    text, p, nf, g = CASES[case]
    logN, bits = 10, 50
    om = Cp.compile_forest(text, p, nf, slots_per_row=1 << (logN - 1))
    L = Cp.levels_needed(om, fused=True) + 1
    P = B.Params(logN=logN, L=L, bits=bits, dnum=3)
    nq = max(1, P.N // (om.block * om.n_seg))
    qs = synth.random_queries(900 + case, nq, nf, p)
    ctx = K.copse_ctx_create(logN, bits, L, 3)
    made = []
    try:
        model = K.copse_compile_forest(text, p, nf, logN)
        K.copse_model_set_fused(model, True)
        assert K.copse_model_is_fused(model)
        K.copse_model_set_bsgs(model, g, 0)
        info = K.copse_model_info_get(model)
        assert info["levels_used"] == Cp.levels_needed(om, fused=True) and info["n_rot_reshuffle"] == 0
        keys, evk = K.copse_keygen(ctx, 23, [model])
        feats = K.copse_encrypt_features(ctx, keys, model, qs, 29)
        res = K.copse_infer(ctx, evk, model, feats)
        made = [res, feats]
        got = K.copse_ctbuf_export(ctx, res, 0, P.N)
        labels = K.copse_decrypt_labels(ctx, keys, model, res, nq)
    finally:
        for h in made:
            K.copse_ctbuf_destroy(h)
        if made:
            K.copse_keys_destroy(keys)
            K.copse_evk_destroy(evk)
            K.copse_model_destroy(model)
        K.copse_ctx_destroy(ctx)
    bgv = B.Bgv(P)
    okeys = bgv.keygen(23, Cp.galois_elements(om, logN, (g, 0), fused=True))
    X = Cp.encrypt_queries(bgv, okeys, om, qs[: P.N // (om.block * om.n_seg)], 29)
    want = Cp.infer(Cp.BgvEngine(bgv, okeys), om, X, P.N, (g, 0), fused=True)
    assert_same(got, want, f"fused inference {case}")
    _, trees = Cp.parse_forest(text)
    for j in range(nq):
        assert labels[j].tolist() == Cp.classify_plain(trees, qs[j]), f"query {j}"


def test_fused_forest100_labels_and_savings():
    W = synth.WORKLOADS["forest100-n16384"]
    text = W.forest_texts()[0]
    ctx = K.copse_ctx_create(W.log_n, W.bits, W.primes, W.dnum)
    try:
        two = K.copse_compile_forest(text, W.precision(), W.n_features(), W.log_n)
        fz = K.copse_compile_forest(text, W.precision(), W.n_features(), W.log_n)
        K.copse_model_set_fused(fz, True)
        i2, i1 = K.copse_model_info_get(two), K.copse_model_info_get(fz)
        assert i1["levels_used"] == i2["levels_used"] - 1 and i1["n_rot_reshuffle"] == 0
        # with baby-step plans the fused products need fewer rotation keys: one q-wide plan
        # instead of a q-wide reshuffle plan plus a b-wide level plan
        K.copse_model_set_bsgs(two, 16, 8)
        K.copse_model_set_bsgs(fz, 16, 0)
        i2, i1 = K.copse_model_info_get(two), K.copse_model_info_get(fz)
        assert i1["n_rot_level"] < i2["n_rot_reshuffle"] + i2["n_rot_level"]
        keys, evk = K.copse_keygen(ctx, 5, [fz])
        nq = (1 << W.log_n) // i1["block"]
        qs = synth.random_queries(4242, nq, W.n_features(), W.precision())
        feats = K.copse_encrypt_features(ctx, keys, fz, qs, 8)
        res = K.copse_infer(ctx, evk, fz, feats)
        labels = K.copse_decrypt_labels(ctx, keys, fz, res, nq)
        K.copse_ctbuf_destroy(res)
        K.copse_ctbuf_destroy(feats)
        assert np.array_equal(labels, K.copse_classify_plain(fz, qs))
        sess = K.copse_session_create(ctx, keys, evk, fz, nq)
        out = np.zeros(nq * i1["n_leaves"], np.uint8)
        K.copse_session_run(sess, qs.reshape(-1), 12, out)
        assert np.array_equal(out.reshape(nq, -1), K.copse_classify_plain(fz, qs))
        K.copse_session_destroy(sess)
        K.copse_keys_destroy(keys)
        K.copse_evk_destroy(evk)
        K.copse_model_destroy(two)
        K.copse_model_destroy(fz)
    finally:
        K.copse_ctx_destroy(ctx)
