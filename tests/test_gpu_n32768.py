"""Ring degree N = 2^15 (the largest with 2N | t - 1 at t = 65537): the NTT,
keys and a whole inference against the oracle, coefficient for coefficient.
At this degree the transforms take the two-pass tiled kernels by default, and
the 16-CTA cluster kernels (with their fused forms) as an option."""
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

from test_gpu_parity import Setup, assert_same  # noqa: E402


@pytest.fixture(scope="module")
def big():
    W = synth.WORKLOADS["toy-n1024"]
    s = Setup(W.forest_texts()[0], W.precision(), W.n_features(), 15, 55, W.primes, W.dnum)
    yield s
    s.close()


def test_ntt_and_product_n32768(big):
    P = big.P
    rng = np.random.default_rng(15)
    a = np.stack([rng.integers(0, q, size=P.N, dtype=np.uint64) for q in P.q])
    b = np.stack([rng.integers(0, q, size=P.N, dtype=np.uint64) for q in P.q])
    da = torch.from_numpy(a.view(np.int64)).cuda()
    db = torch.from_numpy(b.view(np.int64)).cuda()
    dc = torch.empty_like(da)
    K.copse_poly_mul(big.ctx, da.data_ptr(), db.data_ptr(), dc.data_ptr(), P.L)
    torch.cuda.synchronize()
    want = np.zeros_like(a)
    for r, q in enumerate(P.q):
        B.lib().or_negacyclic_mul(np.ascontiguousarray(a[r]), np.ascontiguousarray(b[r]), P.logN, q, want[r])
    assert_same(dc.cpu().numpy().view(np.uint64), want, "negacyclic product at N = 2^15")
    x = da.clone()
    K.copse_ntt(big.ctx, x.data_ptr(), 1, P.L, inverse=False)
    K.copse_ntt(big.ctx, x.data_ptr(), 1, P.L, inverse=True)
    torch.cuda.synchronize()
    assert_same(x.cpu().numpy().view(np.uint64), a, "INTT(NTT(a)) at N = 2^15")


def test_keys_n32768(big):
    P = big.P
    assert_same(K.copse_keys_export_secret(big.keys, P.N), big.okeys.sk, "secret key")
    words = P.ndig * 2 * (P.L + P.alpha) * P.N
    assert_same(K.copse_evk_export(big.evk, 0, words).reshape(big.okeys.rlk.shape), big.okeys.rlk, "relin key")
    g, gk = next(iter(big.okeys.gk.items()))
    assert_same(K.copse_evk_export(big.evk, g, words).reshape(gk.shape), gk, f"rotation key g={g}")


def test_inference_n32768(big):
    qs = synth.random_queries(1515, 3, big.nf, big.p)
    feats = K.copse_encrypt_features(big.ctx, big.keys, big.model, qs, 77)
    res = K.copse_infer(big.ctx, big.evk, big.model, feats)
    try:
        got = K.copse_ctbuf_export(big.ctx, res, 0, big.N)
        bits = K.copse_decrypt_labels(big.ctx, big.keys, big.model, res, len(qs))
    finally:
        K.copse_ctbuf_destroy(res)
        K.copse_ctbuf_destroy(feats)
    X = Cp.encrypt_queries(big.bgv, big.okeys, big.om, qs, 77)
    want = Cp.infer(Cp.BgvEngine(big.bgv, big.okeys), big.om, X, big.N)
    assert_same(got, want, "inference at N = 2^15")
    _, trees = Cp.parse_forest(big.text)
    for j in range(len(qs)):
        assert bits[j].tolist() == Cp.classify_plain(trees, qs[j]), f"query {j}"


def test_inference_n32768_cluster16(monkeypatch):
    """The one-launch 16-CTA cluster transforms and their fused forms (an option at N = 2^15,
    COPSE_NTT_CLUSTER16=1, read when a context is made): the same inference as the oracle's."""
    monkeypatch.setenv("COPSE_NTT_CLUSTER16", "1")
    W = synth.WORKLOADS["toy-n1024"]
    s = Setup(W.forest_texts()[0], W.precision(), W.n_features(), 15, 55, W.primes, W.dnum)
    try:
        qs = synth.random_queries(1516, 2, s.nf, s.p)
        feats = K.copse_encrypt_features(s.ctx, s.keys, s.model, qs, 78)
        res = K.copse_infer(s.ctx, s.evk, s.model, feats)
        try:
            got = K.copse_ctbuf_export(s.ctx, res, 0, s.N)
        finally:
            K.copse_ctbuf_destroy(res)
            K.copse_ctbuf_destroy(feats)
        X = Cp.encrypt_queries(s.bgv, s.okeys, s.om, qs, 78)
        want = Cp.infer(Cp.BgvEngine(s.bgv, s.okeys), s.om, X, s.N)
        assert_same(got, want, "inference at N = 2^15 with 16-CTA cluster transforms")
    finally:
        s.close()
