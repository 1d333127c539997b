"""The tensor-core multiply-accumulate of the encrypted model (csrc/encmac.cu) against the
oracle, coefficient for coefficient, on shapes that reach its every path: accumulator tiles
beyond the first (more than 16 accumulators per matrix), runs beyond the first (more than 256
baby steps, so more than one exact f32 accumulation), passes beyond the first (more than 8
query ciphertexts per launch), and 55-bit primes (residues in the top 1/256 of [0, q), where
the digits of the uncentred residue would need an eighth place).  Whole inferences go through
the public API; the oracle evaluates Algorithm 1 over BGV with the same keys, model encryption
and query encryption (Section 8.3: the model's diagonals encrypted)."""
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

# (forest generator arguments, log N, plan (reshuffle, level baby steps), query ciphertexts)
CASES = {
    # 164 reshuffle diagonals in 8 baby steps: 21 accumulators (two tiles); 12 query
    # ciphertexts: two passes
    "tiles-passes": ((92, 8, 5, 4, 6, 3), 10, (8, 8), 12),
    # more than 256 reshuffle diagonals in one plan of 300 baby steps: two runs
    "runs": ((95, 16, 5, 4, 6, 3), 11, (300, 16), 2),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_encrypted_multiply_accumulate_matches_oracle(name):
    (fargs, logN, g, n_ct) = CASES[name]
    text = synth.random_forest(*fargs, complete=True)
    p, nf, bits = fargs[4], fargs[3], 55
    N = 1 << logN
    om = Cp.compile_forest(text, p, nf, slots_per_row=N // 2)
    if name == "runs":
        assert g[0] > 256 and om.q > 256, f"reshuffle of {om.q} diagonals does not make two runs"
    else:
        assert -(-om.q // g[0]) > 16, "reshuffle plan does not make two accumulator tiles"
    L = Cp.levels_needed(om) + 1
    P = B.Params(logN=logN, L=L, bits=bits, dnum=3)
    per_ct = N // (om.block * om.n_seg)
    qs = synth.random_queries(9000 + logN, n_ct * per_ct, nf, p)
    ctx = K.copse_ctx_create(logN, bits, L, 3)
    made = []
    try:
        model = K.copse_compile_forest(text, p, nf, logN)
        K.copse_model_set_encrypted(model, True)
        K.copse_model_set_bsgs(model, *g)
        keys, evk = K.copse_keygen(ctx, 57, [model])
        K.copse_encrypt_model(ctx, keys, model, 2468)
        feats = K.copse_encrypt_features(ctx, keys, model, qs, 35)
        res = K.copse_infer(ctx, evk, model, feats)
        made = [res, feats]
        assert K.copse_ctx_device_status(ctx) == 0
        assert K.copse_ctbuf_count(res) == n_ct
        got = [K.copse_ctbuf_export(ctx, res, c, N) for c in range(n_ct)]
        labels = K.copse_decrypt_labels(ctx, keys, model, res, len(qs))
    finally:
        for h in made:
            K.copse_ctbuf_destroy(h)
        if made:
            K.copse_keys_destroy(keys)
            K.copse_evk_destroy(evk)
            K.copse_model_destroy(model)
        K.copse_ctx_destroy(ctx)
    bgv = B.Bgv(P)
    rs, ls = Cp.encrypted_rotation_sets(om, g)
    okeys = bgv.keygen(57, sorted(set(B.galois_rot(logN, k) for k in rs + ls)))
    em = Cp.encrypt_model(bgv, okeys.sk, om, N, 2468, g)
    E = Cp.BgvEngine(bgv, okeys, encrypted_model=True, enc_model=em)
    _, trees = Cp.parse_forest(text)
    for c in range(n_ct):
        part = qs[c * per_ct:(c + 1) * per_ct]
        X = Cp.encrypt_queries(bgv, okeys, om, part, 35, index0=c * p)
        want = Cp.infer(E, om, X, N)
        assert_same(got[c], want, f"{name}: query ciphertext {c}")
    for j in range(len(qs)):
        assert labels[j].tolist() == Cp.classify_plain(trees, qs[j]), f"query {j}"
