"""GPU parity: every result of the CUDA path, through the C ABI, against the
CPU oracle on the same seeded inputs.  All arithmetic is exact modular
integer arithmetic, so ciphertexts must agree coefficient for coefficient
(tolerance zero), and decrypted labels must equal plaintext classification."""
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


def _first_diff(a, b):
    d = np.argwhere(np.asarray(a) != np.asarray(b))
    return None if len(d) == 0 else (tuple(d[0]), int(np.asarray(a)[tuple(d[0])]), int(np.asarray(b)[tuple(d[0])]), len(d))


def assert_same(a, b, what):
    a, b = np.asarray(a), np.asarray(b)
    assert a.shape == b.shape, f"{what}: shape {a.shape} vs {b.shape}"
    diff = _first_diff(a, b)
    assert diff is None, f"{what}: first mismatch at {diff[0]} (gpu {diff[1]}, oracle {diff[2]}), {diff[3]} in all"


class Setup:
    """One workload on both sides: context + oracle parameters with identical primes,
    the compiled model, keys from the same seed."""

    def __init__(self, text, p, nf, logN, bits, L, dnum=3, key_seed=7):
        self.text, self.p, self.nf = text, p, nf
        self.ctx = K.copse_ctx_create(logN, bits, L, dnum)
        self.P = B.Params(logN=logN, L=L, bits=bits, dnum=dnum)
        assert K.copse_ctx_primes(self.ctx) == self.P.primes
        self.N = self.P.N
        self.model = K.copse_compile_forest(text, p, nf, logN)
        self.om = Cp.compile_forest(text, p, nf)
        self.bgv = B.Bgv(self.P)
        self.keys, self.evk = K.copse_keygen(self.ctx, key_seed, [self.model])
        self.okeys = self.bgv.keygen(key_seed, Cp.galois_elements(self.om, logN))

    def close(self):
        K.copse_keys_destroy(self.keys)
        K.copse_evk_destroy(self.evk)
        K.copse_model_destroy(self.model)
        K.copse_ctx_destroy(self.ctx)


TOY = ("toy-n1024",)


@pytest.fixture(scope="module")
def toy():
    W = synth.WORKLOADS["toy-n1024"]
    s = Setup(W.forest_texts()[0], W.precision(), W.n_features(), W.log_n, W.bits, W.primes, W.dnum)
    yield s
    s.close()


def test_ntt_roundtrip_and_negacyclic_product(toy):
    P = toy.P
    rng = np.random.default_rng(1)
    a = np.stack([rng.integers(0, q, size=P.N, dtype=np.uint64) for q in P.q])
    b = np.stack([rng.integers(0, q, size=P.N, dtype=np.uint64) for q in P.q])
    da = torch.from_numpy(a.view(np.int64)).cuda()
    db = torch.from_numpy(b.view(np.int64)).cuda()
    dc = torch.empty_like(da)
    K.copse_poly_mul(toy.ctx, da.data_ptr(), db.data_ptr(), dc.data_ptr(), P.L)
    torch.cuda.synchronize()
    got = dc.cpu().numpy().view(np.uint64)
    want = np.zeros_like(a)
    for r, q in enumerate(P.q):
        B.lib().or_negacyclic_mul(np.ascontiguousarray(a[r]), np.ascontiguousarray(b[r]), P.logN, q, want[r])
    assert_same(got, want, "negacyclic product")
    x = da.clone()
    K.copse_ntt(toy.ctx, x.data_ptr(), 1, P.L, inverse=False)
    K.copse_ntt(toy.ctx, x.data_ptr(), 1, P.L, inverse=True)
    torch.cuda.synchronize()
    assert_same(x.cpu().numpy().view(np.uint64), a, "INTT(NTT(a))")
    # several polys in one batch, ragged residue count
    y = torch.from_numpy(np.concatenate([a[:3], b[:3]]).view(np.int64)).cuda()
    K.copse_ntt(toy.ctx, y.data_ptr(), 2, 3)
    K.copse_ntt(toy.ctx, y.data_ptr(), 2, 3, inverse=True)
    torch.cuda.synchronize()
    assert_same(y.cpu().numpy().view(np.uint64), np.concatenate([a[:3], b[:3]]), "batched roundtrip")


def test_keys_match_oracle(toy):
    P = toy.P
    s = K.copse_keys_export_secret(toy.keys, P.N)
    assert_same(s, toy.okeys.sk, "secret key")
    words = P.ndig * 2 * (P.L + P.alpha) * P.N
    rlk = K.copse_evk_export(toy.evk, 0, words).reshape(toy.okeys.rlk.shape)
    assert_same(rlk, toy.okeys.rlk, "relinearisation key")
    for g, gk in toy.okeys.gk.items():
        got = K.copse_evk_export(toy.evk, g, words).reshape(gk.shape)
        assert_same(got, gk, f"rotation key g={g}")


@pytest.mark.parametrize("nq", [0, 1, 5, 32])
def test_encrypt_matches_oracle(toy, nq):
    qs = synth.random_queries(40 + nq, nq, toy.nf, toy.p)
    buf = K.copse_encrypt_features(toy.ctx, toy.keys, toy.model, qs, 99)
    try:
        assert K.copse_ctbuf_count(buf) == toy.p
        want = Cp.encrypt_queries(toy.bgv, toy.okeys, toy.om, qs, 99)
        for i in range(toy.p):
            assert_same(K.copse_ctbuf_export(toy.ctx, buf, i, toy.N), want[i], f"plane {i}")
    finally:
        K.copse_ctbuf_destroy(buf)


def _oracle_cts(toy, n, seed):
    rng = np.random.default_rng(seed)
    vals = [rng.integers(0, 2, size=toy.N) for _ in range(n)]
    cts = [toy.bgv.encrypt_slots(toy.okeys.pk, v, seed, i) for i, v in enumerate(vals)]
    return vals, cts


def test_ring_ops_match_oracle(toy):
    vals, cts = _oracle_cts(toy, 2, 5)
    buf = K.copse_ctbuf_import(toy.ctx, np.stack(cts))
    made = []
    try:
        got = K.copse_ctbuf_export(toy.ctx, buf, 0, toy.N)
        assert_same(got, cts[0], "import/export")
        r = K.copse_ct_mul(toy.ctx, toy.evk, buf, 0, buf, 1)
        made.append(r)
        assert_same(K.copse_ctbuf_export(toy.ctx, r, 0, toy.N), toy.bgv.mul(cts[0], cts[1], toy.okeys.rlk), "mul")
        r = K.copse_ct_modswitch(toy.ctx, buf, 0)
        made.append(r)
        assert_same(K.copse_ctbuf_export(toy.ctx, r, 0, toy.N), toy.bgv.modswitch(cts[0]), "modswitch")
        rng = np.random.default_rng(3)
        mv = rng.integers(0, B.T_DEFAULT, size=toy.N)
        av = rng.integers(0, B.T_DEFAULT, size=toy.N)
        r = K.copse_ct_mul_plain(toy.ctx, buf, 1, mv, av)
        made.append(r)
        want = toy.bgv.modswitch(toy.bgv.add_plain(toy.bgv.mul_plain(cts[1], B.encode(toy.P, mv)), B.encode(toy.P, av)))
        assert_same(K.copse_ctbuf_export(toy.ctx, r, 0, toy.N), want, "mul_plain + add_plain")
        rs, ls = Cp.rotation_sets(toy.om)
        for k in sorted(set(rs + ls))[:4]:
            g = B.galois_rot(toy.P.logN, k)
            r = K.copse_ct_rotate(toy.ctx, toy.evk, buf, 0, k)
            made.append(r)
            assert_same(K.copse_ctbuf_export(toy.ctx, r, 0, toy.N), toy.bgv.rotate(cts[0], g, toy.okeys.gk[g]),
                        f"rotate {k}")
        # a rotation at a lower level (fewer active digits), and a product of mixed levels
        low = K.copse_ct_modswitch(toy.ctx, buf, 0)
        made.append(low)
        lo = toy.bgv.modswitch(cts[0])
        k = rs[0]
        g = B.galois_rot(toy.P.logN, k)
        r = K.copse_ct_rotate(toy.ctx, toy.evk, low, 0, k)
        made.append(r)
        assert_same(K.copse_ctbuf_export(toy.ctx, r, 0, toy.N), toy.bgv.rotate(lo, g, toy.okeys.gk[g]), "rotate low")
        r = K.copse_ct_mul(toy.ctx, toy.evk, low, 0, buf, 1)
        made.append(r)
        assert_same(K.copse_ctbuf_export(toy.ctx, r, 0, toy.N), toy.bgv.mul(lo, cts[1], toy.okeys.rlk), "mixed-level mul")
        # decryption of every slot
        slots = K.copse_decrypt_slots(toy.ctx, toy.keys, buf, 1, toy.N)
        assert_same(slots.astype(np.int64), vals[1], "decrypt slots")
    finally:
        for h in made:
            K.copse_ctbuf_destroy(h)
        K.copse_ctbuf_destroy(buf)


def test_missing_rotation_key_is_an_error(toy):
    _, cts = _oracle_cts(toy, 1, 8)
    buf = K.copse_ctbuf_import(toy.ctx, np.stack(cts))
    try:
        rs, ls = Cp.rotation_sets(toy.om)
        missing = next(k for k in range(1, toy.N // 2) if k not in rs and k not in ls)
        with pytest.raises(K.CopseError) as e:
            K.copse_ct_rotate(toy.ctx, toy.evk, buf, 0, missing)
        assert e.value.name == "ENOKEY"
    finally:
        K.copse_ctbuf_destroy(buf)


def _run_both(s, qs, seed=99):
    feats = K.copse_encrypt_features(s.ctx, s.keys, s.model, qs, seed)
    res = K.copse_infer(s.ctx, s.evk, s.model, feats)
    try:
        got = K.copse_ctbuf_export(s.ctx, res, 0, s.N)
        bits = K.copse_decrypt_labels(s.ctx, s.keys, s.model, res, len(qs))
        slots = K.copse_decrypt_slots(s.ctx, s.keys, res, 0, s.N)
    finally:
        K.copse_ctbuf_destroy(res)
        K.copse_ctbuf_destroy(feats)
    return got, bits, slots


@pytest.mark.parametrize("nq", [0, 1, 7, 32])
def test_inference_matches_oracle_toy(toy, nq):
    qs = synth.random_queries(1000 + nq, nq, toy.nf, toy.p)
    got, bits, slots = _run_both(toy, qs)
    X = Cp.encrypt_queries(toy.bgv, toy.okeys, toy.om, qs, 99)
    want = Cp.infer(Cp.BgvEngine(toy.bgv, toy.okeys), toy.om, X, toy.N)
    assert_same(got, want, "inference result")
    _, trees = Cp.parse_forest(toy.text)
    for j in range(nq):
        assert bits[j].tolist() == Cp.classify_plain(trees, qs[j]), f"query {j}"
    ref = Cp.infer(Cp.SlotEngine(toy.N), toy.om, list(Cp.feature_planes(toy.om, qs, toy.N)), toy.N)
    assert_same(slots.astype(np.int64), ref, "all slots vs cleartext circuit")


def test_chain_too_short_is_an_error(toy):
    ctx = K.copse_ctx_create(10, 50, 5, 3)
    try:
        model = K.copse_compile_forest(toy.text, toy.p, toy.nf, 10)
        keys, evk = K.copse_keygen(ctx, 1, [model])
        feats = K.copse_encrypt_features(ctx, keys, model, synth.random_queries(1, 1, toy.nf, toy.p), 1)
        with pytest.raises(K.CopseError) as e:
            K.copse_infer(ctx, evk, model, feats)
        assert e.value.name == "ELEVEL"
        K.copse_ctbuf_destroy(feats)
        K.copse_keys_destroy(keys)
        K.copse_evk_destroy(evk)
        K.copse_model_destroy(model)
    finally:
        K.copse_ctx_destroy(ctx)


def test_inference_full_size_matches_oracle():
    """The N = 2^14, 10-prime workload (4 trees, ~100 branches, 8 features, 8-bit), one query,
    ciphertext for ciphertext against the oracle, under three transform schedules: the
    cluster transforms (fused with the base conversions) for every batch, the tiled
    two-pass transforms with separate conversion kernels for every batch, and a mixed
    crossover at 64 residue polynomials."""
    W = synth.WORKLOADS["forest100-n16384"]
    s = Setup(W.forest_texts()[0], W.precision(), W.n_features(), W.log_n, W.bits, W.primes, W.dnum)
    try:
        qs = W.query_arrays()[0]
        got = {}
        for name, cluster_max, fused_max in (("cluster", 1 << 30, 1 << 30), ("tiled", 0, 0), ("mixed", 64, 64)):
            K.copse_ctx_set_ntt_cluster_max(s.ctx, cluster_max)
            K.copse_ctx_set_ntt_fused_max(s.ctx, fused_max)
            got[name], bits, _ = _run_both(s, qs)
            _, trees = Cp.parse_forest(s.text)
            assert bits[0].tolist() == Cp.classify_plain(trees, qs[0]), name
        X = Cp.encrypt_queries(s.bgv, s.okeys, s.om, qs, 99)
        want = Cp.infer(Cp.BgvEngine(s.bgv, s.okeys), s.om, X, s.N)
        for name, g in got.items():
            assert_same(g, want, f"inference result ({name} transforms)")
    finally:
        s.close()


def test_batched_three_forests_properties():
    """256 queries over three forests at N = 2^14: every slot equals the cleartext circuit and
    every label vector equals plaintext classification (properties that hold at any size)."""
    W = synth.WORKLOADS["batch3-n16384"]
    ctx = K.copse_ctx_create(W.log_n, W.bits, W.primes, W.dnum)
    texts, queries = W.forest_texts(), W.query_arrays()
    models = [K.copse_compile_forest(t, W.precision(k), W.n_features(k), W.log_n) for k, t in enumerate(texts)]
    keys, evk = K.copse_keygen(ctx, 11, models)
    try:
        for k, (text, qs, m) in enumerate(zip(texts, queries, models)):
            om = Cp.compile_forest(text, W.precision(k), W.n_features(k))
            per_ct = (1 << W.log_n) // om.block
            _, trees = Cp.parse_forest(text)
            # the first and the last (ragged) ciphertext of each forest's queries
            for c0 in sorted({0, ((len(qs) - 1) // per_ct) * per_ct}):
                chunk = qs[c0: c0 + per_ct]
                feats = K.copse_encrypt_features(ctx, keys, m, chunk, 5 + c0)
                res = K.copse_infer(ctx, evk, m, feats)
                bits = K.copse_decrypt_labels(ctx, keys, m, res, len(chunk))
                slots = K.copse_decrypt_slots(ctx, keys, res, 0, 1 << W.log_n)
                K.copse_ctbuf_destroy(res)
                K.copse_ctbuf_destroy(feats)
                ref = Cp.infer(Cp.SlotEngine(1 << W.log_n), om, list(Cp.feature_planes(om, chunk, 1 << W.log_n)),
                               1 << W.log_n)
                assert_same(slots.astype(np.int64), ref, f"forest {k} chunk {c0}")
                for j in range(len(chunk)):
                    assert bits[j].tolist() == Cp.classify_plain(trees, chunk[j])
    finally:
        K.copse_keys_destroy(keys)
        K.copse_evk_destroy(evk)
        for m in models:
            K.copse_model_destroy(m)
        K.copse_ctx_destroy(ctx)
