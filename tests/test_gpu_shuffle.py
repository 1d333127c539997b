"""Label shuffle with padding on the GPU: the shuffled inference against the
oracle's, coefficient for coefficient, at N = 2^10 (plaintext and encrypted
model); at N = 2^14 the bits read through the shuffled codebook give every
tree's class exactly as the plaintext walk, in a recorded session."""
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

TEXT = synth.random_forest(77, 3, 4, 3, 5, 3, complete=False)


@pytest.mark.parametrize("encrypted", [False, True])
def test_shuffled_inference_matches_oracle(encrypted):
    p, nf, logN, bits = 5, 3, 10, 50
    om = Cp.compile_forest(TEXT, p, nf)
    src, code = synth.shuffle_plan(21, om.labels_per_leaf, om.block - om.L, 3)
    L = Cp.levels_needed(om, shuffle=True) + 1
    P = B.Params(logN=logN, L=L, bits=bits, dnum=3)
    ctx = K.copse_ctx_create(logN, bits, L, 3)
    try:
        model = K.copse_compile_forest(TEXT, p, nf, logN)
        K.copse_model_set_encrypted(model, encrypted)
        K.copse_model_set_shuffle(model, src, code)
        keys, evk = K.copse_keygen(ctx, 8, [model])
        if encrypted:
            K.copse_encrypt_model(ctx, keys, model, 555)
        nq = P.N // om.block
        qs = synth.random_queries(61, nq, nf, p)
        feats = K.copse_encrypt_features(ctx, keys, model, qs, 13)
        res = K.copse_infer(ctx, evk, model, feats)
        got = K.copse_ctbuf_export(ctx, res, 0, P.N)
        labels = K.copse_decrypt_labels(ctx, keys, model, res, nq)
        assert labels.shape == (nq, len(src))
        K.copse_ctbuf_destroy(res)
        K.copse_ctbuf_destroy(feats)
        K.copse_keys_destroy(keys)
        K.copse_evk_destroy(evk)
        K.copse_model_destroy(model)
    finally:
        K.copse_ctx_destroy(ctx)
    bgv = B.Bgv(P)
    if encrypted:
        rs, ls = Cp.encrypted_rotation_sets(om)
        gal = set(B.galois_rot(logN, k) for k in rs + ls)
    else:
        gal = set(Cp.galois_elements(om, logN))
    okeys = bgv.keygen(8, sorted(gal | set(Cp.shuffle_galois(om, src, logN))))
    X = Cp.encrypt_queries(bgv, okeys, om, qs, 13)
    E = (Cp.BgvEngine(bgv, okeys, encrypted_model=True, enc_model=Cp.encrypt_model(bgv, okeys.sk, om, P.N, 555))
         if encrypted else Cp.BgvEngine(bgv, okeys))
    assert_same(got, Cp.infer(E, om, X, P.N, shuffle=src), "shuffled inference")
    _, trees = Cp.parse_forest(TEXT)
    for j in range(nq):
        walk = Cp.classify_plain(trees, qs[j])
        assert labels[j][src < 0].sum() == 0
        assert labels[j][src >= 0].tolist() == [walk[i] for i in src if i >= 0], j


def test_shuffled_session_n16384_classes():
    W = synth.WORKLOADS["forest100-n16384"]
    text = W.forest_texts()[0]
    om = Cp.compile_forest(text, W.precision(), W.n_features())
    src, code = synth.shuffle_plan(99, om.labels_per_leaf, 128 - om.L, 4)
    ctx = K.copse_ctx_create(W.log_n, W.bits, W.primes + 1, W.dnum)
    try:
        model = K.copse_compile_forest(text, W.precision(), W.n_features(), W.log_n)
        K.copse_model_set_shuffle(model, src, code)
        keys, evk = K.copse_keygen(ctx, 5, [model])
        info = K.copse_model_info_get(model)
        nq = (1 << W.log_n) // info["block"]
        qs = synth.random_queries(2468, nq, W.n_features(), W.precision())
        sess = K.copse_session_create(ctx, keys, evk, model, nq)
        out = np.zeros(nq * info["n_out"], np.uint8)
        K.copse_session_run(sess, qs.reshape(-1), 3, out)
        out = out.reshape(nq, info["n_out"])
        K.copse_session_destroy(sess)
        codebook = K.copse_model_codebook(model)
        _, trees = Cp.parse_forest(text)
        for j in range(nq):
            walk = Cp.classify_plain(trees, qs[j])
            chosen = sorted(int(codebook[k]) for k in range(info["n_out"]) if out[j, k])
            assert chosen == sorted(om.labels_per_leaf[i] for i in range(om.L) if walk[i]), j
        K.copse_keys_destroy(keys)
        K.copse_evk_destroy(evk)
        K.copse_model_destroy(model)
    finally:
        K.copse_ctx_destroy(ctx)
