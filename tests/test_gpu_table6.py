"""The Table 6 microbenchmark forests (Section 8.4) through copse_infer_timed:
the per-stage timed inference returns the same ciphertext as copse_infer,
coefficient for coefficient, and the oracle's at N = 2^10; at N = 2^14 every
label vector equals plaintext classification and every stage time is
positive."""
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

# 3 + ceil(log2 16) + ceil(log2 6) = 10 primes dropped at most, one more to decrypt
PRIMES = 11


def _export(ctx, buf, N):
    return K.copse_ctbuf_export(ctx, buf, 0, N)


@pytest.mark.parametrize("name", ["prec16", "width677"])
def test_timed_inference_matches_oracle_n1024(name):
    depth, p, _ = synth.TABLE6[name]
    text = synth.table6_forest(name)
    logN, bits = 10, 50
    ctx = K.copse_ctx_create(logN, bits, PRIMES, 3)
    try:
        P = B.Params(logN=logN, L=PRIMES, bits=bits, dnum=3)
        assert K.copse_ctx_primes(ctx) == P.primes
        model = K.copse_compile_forest(text, p, 2, logN)
        keys, evk = K.copse_keygen(ctx, 5, [model])
        om = Cp.compile_forest(text, p, 2)
        nq = P.N // om.block
        qs = synth.random_queries(61, nq, 2, p)
        feats = K.copse_encrypt_features(ctx, keys, model, qs, 21)
        res_t, ms = K.copse_infer_timed(ctx, evk, model, feats)
        res = K.copse_infer(ctx, evk, model, feats)
        got_t, got = _export(ctx, res_t, P.N), _export(ctx, res, P.N)
        labels = K.copse_decrypt_labels(ctx, keys, model, res_t, nq)
        for h in (res_t, res, feats):
            K.copse_ctbuf_destroy(h)
        K.copse_keys_destroy(keys)
        K.copse_evk_destroy(evk)
        K.copse_model_destroy(model)
    finally:
        K.copse_ctx_destroy(ctx)
    assert np.array_equal(got_t, got), "timed and untimed inference differ"
    assert set(ms) == {"comparison", "reshuffle", "levels", "aggregation"}
    assert all(v > 0 for v in ms.values()), ms
    bgv = B.Bgv(P)
    okeys = bgv.keygen(5, Cp.galois_elements(om, logN))
    X = Cp.encrypt_queries(bgv, okeys, om, qs, 21)
    want = Cp.infer(Cp.BgvEngine(bgv, okeys), om, X, P.N)
    assert np.array_equal(np.asarray(got_t), np.asarray(want)), "GPU ciphertext differs from the oracle's"
    _, trees = Cp.parse_forest(text)
    for j in range(nq):
        assert labels[j].tolist() == Cp.classify_plain(trees, qs[j]), f"query {j}"


def test_table6_sweep_n16384_labels_and_stages():
    logN, bits = 14, 55
    ctx = K.copse_ctx_create(logN, bits, PRIMES, 3)
    try:
        for name in sorted(synth.TABLE6):
            depth, p, _ = synth.TABLE6[name]
            text = synth.table6_forest(name)
            model = K.copse_compile_forest(text, p, 2, logN)
            keys, evk = K.copse_keygen(ctx, 9, [model])
            info = K.copse_model_info_get(model)
            nq = (1 << logN) // info["block"]
            qs = synth.random_queries(100 + sorted(synth.TABLE6).index(name), nq, 2, p)
            feats = K.copse_encrypt_features(ctx, keys, model, qs, 33)
            res, ms = K.copse_infer_timed(ctx, evk, model, feats)
            labels = K.copse_decrypt_labels(ctx, keys, model, res, nq)
            K.copse_ctbuf_destroy(res)
            K.copse_ctbuf_destroy(feats)
            K.copse_keys_destroy(keys)
            K.copse_evk_destroy(evk)
            K.copse_model_destroy(model)
            assert all(v > 0 for v in ms.values()), (name, ms)
            _, trees = Cp.parse_forest(text)
            for j in range(nq):
                assert labels[j].tolist() == Cp.classify_plain(trees, qs[j]), (name, j)
    finally:
        K.copse_ctx_destroy(ctx)
