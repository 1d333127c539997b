"""Graph-replayed sessions: every run of a recorded session must decrypt to the
plaintext classification of that run's queries, and agree bit for bit with the
operation-by-operation path on the same inputs."""
import numpy as np
import pytest

from oracle import copse as Cp
from paper_2104_09583_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
K = pytest.importorskip("paper_2104_09583_gb300.copse")

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _workload(name):
    W = synth.WORKLOADS[name]
    text = W.forest_texts()[0]
    ctx = K.copse_ctx_create(W.log_n, W.bits, W.primes, W.dnum)
    model = K.copse_compile_forest(text, W.precision(), W.n_features(), W.log_n)
    keys, evk = K.copse_keygen(ctx, 5, [model])
    return W, text, ctx, model, keys, evk


def _close(ctx, model, keys, evk):
    K.copse_keys_destroy(keys)
    K.copse_evk_destroy(evk)
    K.copse_model_destroy(model)
    K.copse_ctx_destroy(ctx)


@pytest.mark.parametrize("name,nq", [("toy-n1024", 1), ("toy-n1024", 32), ("forest100-n16384", 1),
                                     ("forest100-n16384", 32)])
def test_session_runs_match_plaintext_and_op_path(name, nq):
    W, text, ctx, model, keys, evk = _workload(name)
    info = K.copse_model_info_get(model)
    _, trees = Cp.parse_forest(text)
    sess = K.copse_session_create(ctx, keys, evk, model, nq)
    try:
        for run in range(3):
            qs = synth.random_queries(100 * run + nq, nq, info["n_features"], W.precision())
            out = np.zeros((nq, info["n_leaves"]), dtype=np.uint8)
            K.copse_session_run(sess, qs, 1000 + run, out)
            for j in range(nq):
                assert out[j].tolist() == Cp.classify_plain(trees, qs[j]), f"run {run} query {j}"
            if run == 0:
                ct = K.copse_encrypt_features(ctx, keys, model, qs, 1000)
                res = K.copse_infer(ctx, evk, model, ct)
                bits = K.copse_decrypt_labels(ctx, keys, model, res, nq)
                K.copse_ctbuf_destroy(res)
                K.copse_ctbuf_destroy(ct)
                assert np.array_equal(bits, out)
        # device-resident input and output
        qs = synth.random_queries(7, nq, info["n_features"], W.precision())
        d_in = torch.from_numpy(qs.astype(np.int32)).cuda()
        d_out = torch.zeros(nq * info["n_leaves"], dtype=torch.uint8, device="cuda")
        K.copse_session_run(sess, None, 42, stream=torch.cuda.current_stream().cuda_stream,
                            feats_ptr=d_in.data_ptr(), out_ptr=d_out.data_ptr())
        torch.cuda.synchronize()
        got = d_out.cpu().numpy().reshape(nq, info["n_leaves"])
        for j in range(nq):
            assert got[j].tolist() == Cp.classify_plain(trees, qs[j])
    finally:
        K.copse_session_destroy(sess)
        _close(ctx, model, keys, evk)


def test_session_rejects_too_many_queries():
    W, text, ctx, model, keys, evk = _workload("toy-n1024")
    try:
        block = K.copse_model_info_get(model)["block"]
        with pytest.raises(K.CopseError) as e:
            K.copse_session_create(ctx, keys, evk, model, (1 << W.log_n) // block + 1)
        assert e.value.name == "EINVAL"
    finally:
        _close(ctx, model, keys, evk)


def test_batch_session_three_forests_in_one_launch():
    """Items of three forests with different query blocks (32, 3 x 32 and 4 queries) in one graph."""
    W = synth.WORKLOADS["batch3-n16384"]
    ctx = K.copse_ctx_create(W.log_n, W.bits, W.primes, W.dnum)
    texts = W.forest_texts()
    models = [K.copse_compile_forest(t, W.precision(k), W.n_features(k), W.log_n) for k, t in enumerate(texts)]
    keys, evk = K.copse_keygen(ctx, 9, models)
    infos = [K.copse_model_info_get(m) for m in models]
    per_ct = [(1 << W.log_n) // i["block"] for i in infos]
    items = [(0, per_ct[0]), (1, per_ct[1]), (1, per_ct[1]), (1, 5), (2, per_ct[2])]
    sess = K.copse_session_create_batch(ctx, keys, evk, [models[k] for k, _ in items], [n for _, n in items])
    trees = [Cp.parse_forest(t)[1] for t in texts]
    try:
        for run in range(2):
            qs = [synth.random_queries(31 * run + i, n, infos[k]["n_features"], W.precision(k))
                  for i, (k, n) in enumerate(items)]
            feats = np.concatenate([q.reshape(-1) for q in qs])
            out = np.zeros(sum(n * infos[k]["n_leaves"] for k, n in items), dtype=np.uint8)
            K.copse_session_run(sess, feats, 77 + run, out)
            off = 0
            for (k, n), q in zip(items, qs):
                L = infos[k]["n_leaves"]
                got = out[off: off + n * L].reshape(n, L)
                off += n * L
                for j in range(n):
                    assert got[j].tolist() == Cp.classify_plain(trees[k], q[j]), f"run {run} forest {k} query {j}"
    finally:
        K.copse_session_destroy(sess)
        K.copse_keys_destroy(keys)
        K.copse_evk_destroy(evk)
        for m in models:
            K.copse_model_destroy(m)
        K.copse_ctx_destroy(ctx)
