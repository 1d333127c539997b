"""Ciphertext parity at the larger configurations' sizes: the GPU's secure-inference
result ciphertexts, residue polynomial by residue polynomial, against SHA-256 digests
of the oracle's (tests/golden/digests_*.json, written by tests/golden/make_digests.py
from oracle/ alone).  The cases: the batching workload's 16-tree depth-6 forest
(N = 2^14, baby-step plan), an encrypted model at the encrypted-model workload's
parameters (N = 2^15, 16 primes, 16-bit, q >= 256 encrypted diagonals, five query
ciphertexts) and the serving workload's 64-tree depth-6 forest (N = 2^15).  Inputs
are regenerated from the seeds and parameters stored with the digests."""
import glob
import hashlib
import json
import os

import numpy as np
import pytest

from paper_2104_09583_gb300 import synth  # noqa: F401  (the generators the cases came from)

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
K = pytest.importorskip("paper_2104_09583_gb300.copse")

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

HERE = os.path.dirname(os.path.abspath(__file__))
FILES = sorted(glob.glob(os.path.join(HERE, "golden", "digests_*.json")))


def _digest(residue):
    return hashlib.sha256(np.asarray(residue, dtype=np.uint64).astype("<u8").tobytes()).hexdigest()[:16]


@pytest.mark.parametrize("path", FILES, ids=[os.path.basename(f)[8:-5] for f in FILES])
def test_inference_digests_match_oracle(path):
    case = json.load(open(path))
    logN, p, nf = case["log_n"], case["precision"], case["n_features"]
    N = 1 << logN
    qs = np.asarray(case["queries"], dtype=np.uint32)
    ctx = K.copse_ctx_create(logN, case["bits"], case["primes"], case["dnum"])
    made = []
    try:
        model = K.copse_compile_forest(case["text"], p, nf, logN)
        if case["encrypted"]:
            K.copse_model_set_encrypted(model, True)
        K.copse_model_set_bsgs(model, *case["bsgs"])
        keys, evk = K.copse_keygen(ctx, case["key_seed"], [model])
        if case["encrypted"]:
            K.copse_encrypt_model(ctx, keys, model, case["model_seed"])
        feats = K.copse_encrypt_features(ctx, keys, model, qs, case["enc_seed"])
        res = K.copse_infer(ctx, evk, model, feats)
        made = [res, feats]
        n_ct = K.copse_ctbuf_count(res)
        assert n_ct == len(case["digests"]), f"{n_ct} result ciphertexts, oracle {len(case['digests'])}"
        bad = []
        for c, want in enumerate(case["digests"]):
            ct = K.copse_ctbuf_export(ctx, res, c, N)
            assert ct.shape[1] == want["level"], f"ciphertext {c}: level {ct.shape[1]}, oracle {want['level']}"
            for comp, row in enumerate(want["residues"]):
                for r, d in enumerate(row):
                    if _digest(ct[comp, r]) != d:
                        bad.append(f"ciphertext {c} component {comp} residue {r}")
        assert not bad, f"{case['name']}: {len(bad)} residue polynomials differ from the oracle, first: {bad[:4]}"
        labels = K.copse_decrypt_labels(ctx, keys, model, res, len(qs))
        assert np.array_equal(labels, K.copse_classify_plain(model, qs))
    finally:
        for h in made:
            K.copse_ctbuf_destroy(h)
        if made:
            K.copse_keys_destroy(keys)
            K.copse_evk_destroy(evk)
            K.copse_model_destroy(model)
        K.copse_ctx_destroy(ctx)
