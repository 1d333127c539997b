"""Serving: requests against several resident models, batched continuously
into graph launches.  A request's leaf bits must be the same alone and inside
a mixed burst (and equal plaintext classification); a full queue refuses with
EADMIT; bad ids and tickets are errors."""
import numpy as np
import pytest

from oracle import copse as Cp
from paper_2104_09583_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
K = pytest.importorskip("paper_2104_09583_gb300.copse")

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


@pytest.fixture(scope="module")
def served():
    Wb, Wf = synth.WORKLOADS["batch3-n16384"], synth.WORKLOADS["forest100-n16384"]
    ctx = K.copse_ctx_create(Wf.log_n, Wf.bits, Wf.primes, Wf.dnum)
    specs = [(Wf.forest_texts()[0], Wf.precision(), Wf.n_features()),
             (Wb.forest_texts()[0], Wb.precision(0), Wb.n_features(0)),
             (Wb.forest_texts()[1], Wb.precision(1), Wb.n_features(1))]
    models = [K.copse_compile_forest(t, p, nf, Wf.log_n) for t, p, nf in specs]
    keys, evk = K.copse_keygen(ctx, 21, models)
    infos = [K.copse_model_info_get(m) for m in models]
    trees = [Cp.parse_forest(t)[1] for t, _, _ in specs]
    yield ctx, models, keys, evk, infos, trees, [p for _, p, _ in specs]
    K.copse_keys_destroy(keys)
    K.copse_evk_destroy(evk)
    for m in models:
        K.copse_model_destroy(m)
    K.copse_ctx_destroy(ctx)


def test_result_same_alone_and_in_a_mix(served):
    ctx, models, keys, evk, infos, trees, precs = served
    srv = K.copse_server_create(ctx, keys, evk, models)
    try:
        probe = synth.random_queries(5, 1, infos[0]["n_features"], precs[0])[0]
        t = K.copse_server_submit(srv, 0, probe)
        alone, lat = K.copse_server_poll(srv, t, infos[0]["n_leaves"])
        assert alone.tolist() == Cp.classify_plain(trees[0], probe) and lat > 0
        rng = np.random.default_rng(3)
        sent = []
        for i in range(150):
            k = int(rng.integers(3))
            q = probe if (k == 0 and i % 17 == 0) else synth.random_queries(1000 + i, 1, infos[k]["n_features"],
                                                                          precs[k])[0]
            sent.append((k, q, K.copse_server_submit(srv, k, q)))
        repeats = 0
        for k, q, t in sent:
            bits, _ = K.copse_server_poll(srv, t, infos[k]["n_leaves"])
            assert bits.tolist() == Cp.classify_plain(trees[k], q)
            if k == 0 and np.array_equal(q, probe):
                assert np.array_equal(bits, alone)
                repeats += 1
        assert repeats > 0
        assert K.copse_server_pending(srv) == (0, 0)
    finally:
        K.copse_server_destroy(srv)


def test_admission_and_errors(served):
    ctx, models, keys, evk, infos, trees, precs = served
    srv = K.copse_server_create(ctx, keys, evk, models[:1], max_pending=3)
    try:
        admitted, refused = [], 0
        for i in range(400):
            q = synth.random_queries(i, 1, infos[0]["n_features"], precs[0])[0]
            try:
                admitted.append((q, K.copse_server_submit(srv, 0, q)))
            except K.CopseError as e:
                assert e.name == "EADMIT"
                refused += 1
        assert refused > 0
        for q, t in admitted:
            bits, _ = K.copse_server_poll(srv, t, infos[0]["n_leaves"])
            assert bits.tolist() == Cp.classify_plain(trees[0], q)
        with pytest.raises(K.CopseError) as e:
            K.copse_server_submit(srv, 7, admitted[0][0])
        assert e.value.name == "EINVAL"
        with pytest.raises(K.CopseError) as e:
            K.copse_server_poll(srv, 10 ** 9, infos[0]["n_leaves"], 0)
        assert e.value.name == "EINVAL"
    finally:
        K.copse_server_destroy(srv)


def test_admission_by_device_memory(served):
    """Creation measures every launch's device reservation; a submit is refused with EADMIT
    while free device memory is below the admission floor and admitted again once the floor
    is back within what the device holds."""
    ctx, models, keys, evk, infos, trees, precs = served
    srv = K.copse_server_create(ctx, keys, evk, models)
    try:
        reserved, launch_max, floor, launches = K.copse_server_memory(srv)
        assert 0 < launch_max <= reserved and floor == launch_max
        assert len(models) <= launches <= 2 * len(models)
        free, total = torch.cuda.mem_get_info()
        q = synth.random_queries(77, 1, infos[0]["n_features"], precs[0])[0]
        K.copse_server_set_memory_floor(srv, total + 1)  # more than the device has: nothing fits
        with pytest.raises(K.CopseError) as e:
            K.copse_server_submit(srv, 0, q)
        assert e.value.name == "EADMIT"
        assert K.copse_server_pending(srv) == (0, 0)
        K.copse_server_set_memory_floor(srv, launch_max)
        t = K.copse_server_submit(srv, 0, q)
        bits, _ = K.copse_server_poll(srv, t, infos[0]["n_leaves"])
        assert bits.tolist() == Cp.classify_plain(trees[0], q)
    finally:
        K.copse_server_destroy(srv)
