"""Row segments on the GPU: a forest whose query block would not fit a slot row is
compiled into contiguous groups of trees, one slot block each per query.  At
N = 2^10 whole inferences (plaintext model, plain and baby-step / giant-step
products; encrypted model) equal the oracle's coefficient for coefficient; at
N = 2^15 the complete 32-tree depth-8 forest (8160 branches, 16-bit, encrypted
model) gives every query's leaf bits equal to plaintext classification."""
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

LOGN, BITS = 10, 50


def _forest():
    return synth.random_forest(8181, 8, 5, 2, 6, 3, complete=True)


@pytest.mark.parametrize("mode", ["plain", "bsgs", "encrypted"])
def test_segmented_inference_matches_oracle(mode):
    text, p, nf = _forest(), 6, 2
    om = Cp.compile_forest(text, p, nf, slots_per_row=1 << (LOGN - 1))
    assert om.n_seg == 2
    g = (0, 0) if mode == "plain" else (16, 16)
    enc = mode == "encrypted"
    L = Cp.levels_needed(om) + 1
    P = B.Params(logN=LOGN, L=L, bits=BITS, dnum=3)
    nq = 3  # one query per ciphertext: three query ciphertexts
    qs = synth.random_queries(8190, nq, nf, p)
    ctx = K.copse_ctx_create(LOGN, BITS, L, 3)
    made = []
    try:
        model = K.copse_compile_forest(text, p, nf, LOGN)
        info = K.copse_model_info_get(model)
        assert (info["n_segments"], info["block"], info["b"], info["n_leaves"]) == (2, om.block, om.b_total, om.L_total)
        if enc:
            K.copse_model_set_encrypted(model, True)
        K.copse_model_set_bsgs(model, *g)
        keys, evk = K.copse_keygen(ctx, 44, [model])
        if enc:
            K.copse_encrypt_model(ctx, keys, model, 6060)
        feats = K.copse_encrypt_features(ctx, keys, model, qs, 17)
        res = K.copse_infer(ctx, evk, model, feats)
        made = [res, feats]
        assert K.copse_ctbuf_count(res) == nq
        got = [K.copse_ctbuf_export(ctx, res, c, P.N) for c in range(nq)]
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
    rs, ls = Cp.encrypted_rotation_sets(om, g) if enc else Cp.rotation_sets(om, g)
    okeys = bgv.keygen(44, sorted(set(B.galois_rot(LOGN, k) for k in rs + ls)))
    if enc:
        em = Cp.encrypt_model(bgv, okeys.sk, om, P.N, 6060, g)
        E = Cp.BgvEngine(bgv, okeys, encrypted_model=True, enc_model=em)
    else:
        E = Cp.BgvEngine(bgv, okeys)
    _, trees = Cp.parse_forest(text)
    for c in range(nq):
        X = Cp.encrypt_queries(bgv, okeys, om, qs[c:c + 1], 17, index0=c * p)
        want = Cp.infer(E, om, X, P.N) if enc else Cp.infer(E, om, X, P.N, g)
        assert_same(got[c], want, f"segmented {mode} inference, query ciphertext {c}")
        assert labels[c].tolist() == Cp.classify_plain(trees, qs[c]), f"query {c}"


def test_complete_depth8_forest_n32768_labels():
    """The encrypted-model workload's shape with complete trees: 32 x depth 8 = 8160 branches,
    8192 leaves, 32 features, 16-bit, N = 2^15 with 16 primes; two row segments."""
    W = synth.WORKLOADS["encmodel32-n32768"]
    text = W.forest_texts()[0]
    ctx = K.copse_ctx_create(W.log_n, W.bits, W.primes, W.dnum)
    try:
        model = K.copse_compile_forest(text, W.precision(), W.n_features(), W.log_n)
        info = K.copse_model_info_get(model)
        assert (info["b"], info["n_leaves"], info["n_segments"]) == (8160, 8192, 2)
        K.copse_model_set_encrypted(model, True)
        K.copse_model_set_bsgs(model, 128, 256)
        keys, evk = K.copse_keygen(ctx, 9, [model])
        K.copse_encrypt_model(ctx, keys, model, 77)
        qs = synth.random_queries(8191, 5, W.n_features(), W.precision())
        feats = K.copse_encrypt_features(ctx, keys, model, qs, 3)
        res = K.copse_infer(ctx, evk, model, feats)
        labels = K.copse_decrypt_labels(ctx, keys, model, res, len(qs))
        K.copse_ctbuf_destroy(res)
        K.copse_ctbuf_destroy(feats)
        assert np.array_equal(labels, K.copse_classify_plain(model, qs))
        assert all(labels[j].sum() == 32 for j in range(len(qs)))  # one leaf per tree
        K.copse_keys_destroy(keys)
        K.copse_evk_destroy(evk)
        K.copse_model_destroy(model)
    finally:
        K.copse_ctx_destroy(ctx)
