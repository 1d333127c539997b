"""Encrypted models on the GPU (Maurice = Diane): the model ciphertexts and
whole inferences against the oracle, coefficient for coefficient, at
N = 2^10 with the plain and the baby-step / giant-step products; at
N = 2^14 the labels of a ~100-branch forest equal plaintext classification,
in single inferences and in a recorded session."""
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

CASES = [
    (synth.random_forest(1001, 1, 3, 2, 4, 2), 4, 2, (0, 0)),
    (synth.random_forest(77, 3, 4, 3, 5, 3, complete=False), 5, 3, (4, 3)),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_encrypted_model_matches_oracle(case):
    text, p, nf, g = CASES[case]
    logN, bits = 10, 50
    om = Cp.compile_forest(text, p, nf)
    L = Cp.levels_needed(om) + 1
    P = B.Params(logN=logN, L=L, bits=bits, dnum=3)
    ctx = K.copse_ctx_create(logN, bits, L, 3)
    made = []
    try:
        model = K.copse_compile_forest(text, p, nf, logN)
        K.copse_model_set_encrypted(model, True)
        K.copse_model_set_bsgs(model, *g)
        keys, evk = K.copse_keygen(ctx, 31, [model])
        K.copse_encrypt_model(ctx, keys, model, 4040)
        bgv = B.Bgv(P)
        rs, ls = Cp.encrypted_rotation_sets(om, g)
        okeys = bgv.keygen(31, sorted(set(B.galois_rot(logN, k) for k in rs + ls)))
        em = Cp.encrypt_model(bgv, okeys.sk, om, P.N, 4040, g)
        # a sample of the model's ciphertexts, one of every kind
        d, b, q = om.d, om.b, om.q
        checks = [(Cp.model_ct_index(om, "thr", i=0), em["thresholds"][0]),
                  (Cp.model_ct_index(om, "thr", i=p - 1), em["thresholds"][p - 1]),
                  (Cp.model_ct_index(om, "R", i=0), em["R"][0]),
                  (Cp.model_ct_index(om, "R", i=q - 1), em["R"][q - 1]),
                  (Cp.model_ct_index(om, "lvl", 1, 0), em["levels"][0][0]),
                  (Cp.model_ct_index(om, "lvl", d, b - 1), em["levels"][d - 1][b - 1]),
                  (Cp.model_ct_index(om, "mask", d), em["masks"][d - 1])]
        for idx, want in checks:
            got = K.copse_encmodel_export(ctx, model, idx, want.shape[1], P.N)
            assert_same(got, want, f"model ciphertext {idx}")
        nq = P.N // om.block
        qs = synth.random_queries(700 + case, nq, nf, p)
        feats = K.copse_encrypt_features(ctx, keys, model, qs, 12)
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
    X = Cp.encrypt_queries(bgv, okeys, om, qs, 12)
    want = Cp.infer(Cp.BgvEngine(bgv, okeys, encrypted_model=True, enc_model=em), om, X, P.N)
    assert_same(got, want, "encrypted-model inference")
    _, trees = Cp.parse_forest(text)
    for j in range(nq):
        assert labels[j].tolist() == Cp.classify_plain(trees, qs[j]), f"query {j}"


def test_encrypted_model_n16384_labels_and_session():
    W = synth.WORKLOADS["forest100-n16384"]
    text = W.forest_texts()[0]
    ctx = K.copse_ctx_create(W.log_n, W.bits, W.primes, W.dnum)
    try:
        model = K.copse_compile_forest(text, W.precision(), W.n_features(), W.log_n)
        K.copse_model_set_encrypted(model, True)
        K.copse_model_set_bsgs(model, 16, 16)
        keys, evk = K.copse_keygen(ctx, 3, [model])
        K.copse_encrypt_model(ctx, keys, model, 77)
        info = K.copse_model_info_get(model)
        nq = (1 << W.log_n) // info["block"]
        qs = synth.random_queries(4321, nq, W.n_features(), W.precision())
        want = K.copse_classify_plain(model, qs)
        feats = K.copse_encrypt_features(ctx, keys, model, qs, 5)
        res = K.copse_infer(ctx, evk, model, feats)
        labels = K.copse_decrypt_labels(ctx, keys, model, res, nq)
        K.copse_ctbuf_destroy(res)
        K.copse_ctbuf_destroy(feats)
        assert np.array_equal(labels, want)
        sess = K.copse_session_create(ctx, keys, evk, model, nq)
        out = np.zeros(nq * info["n_leaves"], np.uint8)
        K.copse_session_run(sess, qs.reshape(-1), 99, out)
        assert np.array_equal(out.reshape(nq, -1), want)
        K.copse_session_destroy(sess)
        # a plan change drops the encryption: inference refuses until re-encrypted
        K.copse_model_set_bsgs(model, 8, 16)
        feats = K.copse_encrypt_features(ctx, keys, model, qs, 6)
        with pytest.raises(K.CopseError) as e:
            K.copse_infer(ctx, evk, model, feats)
        assert e.value.name == "EINVAL"
        K.copse_ctbuf_destroy(feats)
        K.copse_keys_destroy(keys)
        K.copse_evk_destroy(evk)
        K.copse_model_destroy(model)
    finally:
        K.copse_ctx_destroy(ctx)


@pytest.mark.parametrize("encrypted", [True, False])
def test_several_query_ciphertexts_match_oracle(encrypted):
    """More queries than one ciphertext holds: query ciphertext c is encrypted with
    indices c p + i and inferred with the others (sharing every encrypted diagonal
    read); each result equals the oracle's for that ciphertext."""
    text, p, nf, g = CASES[0]
    logN, bits = 10, 50
    om = Cp.compile_forest(text, p, nf)
    L = Cp.levels_needed(om) + 1
    P = B.Params(logN=logN, L=L, bits=bits, dnum=3)
    per_ct = P.N // om.block
    nq = 5 * per_ct + 3                       # six ciphertexts, the last one partly filled
    qs = synth.random_queries(808, nq, nf, p)
    ctx = K.copse_ctx_create(logN, bits, L, 3)
    try:
        model = K.copse_compile_forest(text, p, nf, logN)
        K.copse_model_set_encrypted(model, encrypted)
        K.copse_model_set_bsgs(model, *g)
        keys, evk = K.copse_keygen(ctx, 31, [model])
        if encrypted:
            K.copse_encrypt_model(ctx, keys, model, 4040)
        feats = K.copse_encrypt_features(ctx, keys, model, qs, 12)
        assert K.copse_ctbuf_count(feats) == 6 * p
        res = K.copse_infer(ctx, evk, model, feats)
        assert K.copse_ctbuf_count(res) == 6
        got = [K.copse_ctbuf_export(ctx, res, cq, P.N) for cq in range(6)]
        labels = K.copse_decrypt_labels(ctx, keys, model, res, nq)
        K.copse_ctbuf_destroy(res)
        K.copse_ctbuf_destroy(feats)
        K.copse_keys_destroy(keys)
        K.copse_evk_destroy(evk)
        K.copse_model_destroy(model)
    finally:
        K.copse_ctx_destroy(ctx)
    _, trees = Cp.parse_forest(text)
    for j in range(nq):
        assert labels[j].tolist() == Cp.classify_plain(trees, qs[j]), f"query {j}"
    bgv = B.Bgv(P)
    if encrypted:
        rs, ls = Cp.encrypted_rotation_sets(om, g)
        okeys = bgv.keygen(31, sorted(set(B.galois_rot(logN, k) for k in rs + ls)))
        E = Cp.BgvEngine(bgv, okeys, encrypted_model=True, enc_model=Cp.encrypt_model(bgv, okeys.sk, om, P.N, 4040, g))
    else:
        okeys = bgv.keygen(31, Cp.galois_elements(om, logN))
        E = Cp.BgvEngine(bgv, okeys)
    for cq in (0, 5):                          # the first and the partly filled last ciphertext
        X = Cp.encrypt_queries(bgv, okeys, om, qs[cq * per_ct:(cq + 1) * per_ct], 12, cq * p)
        assert_same(got[cq], Cp.infer(E, om, X, P.N), f"query ciphertext {cq}")
