"""Autotuning calls: every timed candidate reports a positive time, the choice
is one of the candidates, and inference under the chosen schedule still
decrypts to plaintext classification."""
import numpy as np
import pytest

from paper_2104_09583_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
K = pytest.importorskip("paper_2104_09583_gb300.copse")

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def test_tuned_schedule_is_correct():
    W = synth.WORKLOADS["forest100-n16384"]
    text = W.forest_texts()[0]
    model = K.copse_compile_forest(text, W.precision(), W.n_features(), W.log_n)
    best_d, dn = K.copse_tune_dnum(W.log_n, W.bits, W.primes, model, [2, 3], 1, 2)
    assert best_d in (2, 3) and all(v > 0 for v in dn.values())
    ctx = K.copse_ctx_create(W.log_n, W.bits, W.primes, best_d)
    try:
        lim, t = K.copse_tune_ntt(ctx, (4, 64, 256), 3)
        assert all(a > 0 and b > 0 for a, b in t.values())
        assert lim in (0, 4, 64, 1 << 30)
        rs, ls = K.copse_tune_bsgs(ctx, model, [0, 16, 1 << 20], [0, 8], 1, 2)
        assert all(v > 0 for v in list(rs.values()) + list(ls.values()))
        g = K.copse_model_get_bsgs(model)
        assert g[0] in (0, 16, 1 << 20) and g[1] in (0, 8)
        fb, fm = K.copse_tune_fused(ctx, model, (8, 1 << 30), 1, 2)
        assert fb in (8, 1 << 30) and all(v > 0 for v in fm.values())
        keys, evk = K.copse_keygen(ctx, 4, [model])
        info = K.copse_model_info_get(model)
        nq = (1 << W.log_n) // info["block"]
        qs = synth.random_queries(77, nq, W.n_features(), W.precision())
        feats = K.copse_encrypt_features(ctx, keys, model, qs, 8)
        res = K.copse_infer(ctx, evk, model, feats)
        labels = K.copse_decrypt_labels(ctx, keys, model, res, nq)
        assert np.array_equal(labels, K.copse_classify_plain(model, qs))
        for h in (res, feats):
            K.copse_ctbuf_destroy(h)
        K.copse_keys_destroy(keys)
        K.copse_evk_destroy(evk)
    finally:
        K.copse_model_destroy(model)
        K.copse_ctx_destroy(ctx)
