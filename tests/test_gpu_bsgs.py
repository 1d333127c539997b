"""Baby-step / giant-step matrix products on the GPU: whole inferences with
BSGS plans against the oracle's, coefficient for coefficient, at N = 2^10;
at N = 2^14 the labels of a ~100-branch forest equal plaintext
classification under several plans, in single inferences and in recorded
sessions."""
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

FOREST = (synth.random_forest(77, 3, 4, 3, 5, 3, complete=False), 5, 3)


@pytest.mark.parametrize("g", [(3, 4), (1, 2), (8, 1)])
def test_bsgs_inference_matches_oracle(g):
    text, p, nf = FOREST
    logN, bits, L = 10, 50, 10
    ctx = K.copse_ctx_create(logN, bits, L, 3)
    made = []
    try:
        P = B.Params(logN=logN, L=L, bits=bits, dnum=3)
        model = K.copse_compile_forest(text, p, nf, logN)
        K.copse_model_set_bsgs(model, *g)
        keys, evk = K.copse_keygen(ctx, 12, [model])
        om = Cp.compile_forest(text, p, nf)
        nq = P.N // om.block
        qs = synth.random_queries(300 + g[0], nq, nf, p)
        feats = K.copse_encrypt_features(ctx, keys, model, qs, 41)
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
    okeys = bgv.keygen(12, Cp.galois_elements(om, logN, g))
    X = Cp.encrypt_queries(bgv, okeys, om, qs, 41)
    want = Cp.infer(Cp.BgvEngine(bgv, okeys), om, X, P.N, g)
    assert_same(got, want, f"BSGS {g} inference")
    _, trees = Cp.parse_forest(text)
    for j in range(nq):
        assert labels[j].tolist() == Cp.classify_plain(trees, qs[j]), f"query {j}"


def test_bsgs_n16384_labels_single_and_session():
    W = synth.WORKLOADS["forest100-n16384"]
    text = W.forest_texts()[0]
    ctx = K.copse_ctx_create(W.log_n, W.bits, W.primes, W.dnum)
    try:
        for g in [(16, 8), (32, 16)]:
            model = K.copse_compile_forest(text, W.precision(), W.n_features(), W.log_n)
            K.copse_model_set_bsgs(model, *g)
            keys, evk = K.copse_keygen(ctx, 3, [model])
            info = K.copse_model_info_get(model)
            nq = (1 << W.log_n) // info["block"]
            qs = synth.random_queries(900 + g[0], nq, W.n_features(), W.precision())
            want = K.copse_classify_plain(model, qs)
            feats = K.copse_encrypt_features(ctx, keys, model, qs, 5)
            res = K.copse_infer(ctx, evk, model, feats)
            labels = K.copse_decrypt_labels(ctx, keys, model, res, nq)
            K.copse_ctbuf_destroy(res)
            K.copse_ctbuf_destroy(feats)
            assert np.array_equal(labels, want), g
            sess = K.copse_session_create(ctx, keys, evk, model, nq)
            out = np.zeros(nq * info["n_leaves"], np.uint8)
            for it in range(2):
                K.copse_session_run(sess, qs.reshape(-1), 60 + it, out)
                assert np.array_equal(out.reshape(nq, -1), want), (g, it)
            K.copse_session_destroy(sess)
            K.copse_keys_destroy(keys)
            K.copse_evk_destroy(evk)
            K.copse_model_destroy(model)
    finally:
        K.copse_ctx_destroy(ctx)
