#!/usr/bin/env python3
"""Writes tests/golden/digests_<case>.json: SHA-256 digests (first 16 hex digits) of
every residue polynomial of the oracle's secure-inference result ciphertexts for
workloads at the sizes of the larger configurations, where a GPU test cannot wait
for the oracle:

  batch3c-n16384    the 16-tree depth-6 forest of the batching workload (32 features,
                    8-bit), N = 2^14, 10 primes, plaintext model, baby-step plan (64, 16),
                    one query ciphertext (4 queries)
  encmodel-n32768   an encrypted model at the encrypted-model workload's parameters
                    (N = 2^15, 16 primes, 16-bit): 4 complete depth-6 trees over 8
                    features (252 branches, q >= 256 diagonals), plan (80, 64), five query
                    ciphertexts of 32 queries
  serving64-n32768  the 64-tree depth-6 forest of the serving workload (16 features,
                    8-bit), N = 2^15, 10 primes, 2 key-switching digits, plan (64, 64), one
                    query ciphertext (2 queries)

Only the oracle computes anything here (Algorithm 1 over BGV, ``oracle.copse.infer``);
the inputs come from the seeded generators in ``paper_2104_09583_gb300.synth``.  The
GPU test (tests/test_gpu_digests.py) reads the case parameters from the same file.
Digest of a residue: sha256 of its N coefficients in [0, q_i) as little-endian
uint64, in coefficient form, layout [component][prime].

Usage: python tests/golden/make_digests.py [case ...]   (default: every case)
"""
import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import bgv as B  # noqa: E402
from oracle import copse as Cp  # noqa: E402
from paper_2104_09583_gb300 import synth  # noqa: E402


def _batch3c():
    W = synth.WORKLOADS["batch3-n16384"]
    return {"name": "batch3c-n16384", "text": W.forest_texts()[2], "precision": W.precision(2),
            "n_features": W.n_features(2), "log_n": 14, "bits": 55, "primes": 10, "dnum": 3,
            "encrypted": False, "bsgs": [64, 16], "key_seed": 17, "model_seed": 0, "enc_seed": 70,
            "queries": W.query_arrays()[2][:4].tolist()}


def _encmodel():
    text = synth.random_forest(4101, 4, 6, 8, 16, 10, complete=True)
    qs = synth.random_queries(4102, 5 * 32, 8, 16)
    return {"name": "encmodel-n32768", "text": text, "precision": 16, "n_features": 8, "log_n": 15, "bits": 55,
            "primes": 16, "dnum": 3, "encrypted": True, "bsgs": [80, 64], "key_seed": 29, "model_seed": 2024,
            "enc_seed": 31, "queries": qs.tolist()}


def _serving64():
    text = synth.random_forest(5004, 64, 6, 16, 8, 4, complete=True)
    qs = synth.random_queries(5005, 2, 16, 8)
    return {"name": "serving64-n32768", "text": text, "precision": 8, "n_features": 16, "log_n": 15, "bits": 55,
            "primes": 10, "dnum": 2, "encrypted": False, "bsgs": [64, 64], "key_seed": 13, "model_seed": 0,
            "enc_seed": 41, "queries": qs.tolist()}


CASES = {"batch3c-n16384": _batch3c, "encmodel-n32768": _encmodel, "serving64-n32768": _serving64}


def residue_digests(ct):
    """[component][prime] -> first 16 hex digits of sha256 of the little-endian residues."""
    ct = np.asarray(ct, dtype=np.uint64)
    return [[hashlib.sha256(ct[c, r].astype("<u8").tobytes()).hexdigest()[:16] for r in range(ct.shape[1])]
            for c in range(ct.shape[0])]


def run(case):
    t0 = time.time()
    logN, p, nf = case["log_n"], case["precision"], case["n_features"]
    N = 1 << logN
    P = B.Params(logN=logN, L=case["primes"], bits=case["bits"], dnum=case["dnum"])
    m = Cp.compile_forest(case["text"], p, nf, slots_per_row=N // 2)
    g = tuple(case["bsgs"])
    bgv = B.Bgv(P)
    rs, ls = Cp.encrypted_rotation_sets(m, g) if case["encrypted"] else Cp.rotation_sets(m, g)
    keys = bgv.keygen(case["key_seed"], sorted(set(B.galois_rot(logN, k) for k in rs + ls)))
    if case["encrypted"]:
        em = Cp.encrypt_model(bgv, keys.sk, m, N, case["model_seed"], g)
        E = Cp.BgvEngine(bgv, keys, encrypted_model=True, enc_model=em)
    else:
        E = Cp.BgvEngine(bgv, keys)
    qs = np.asarray(case["queries"], dtype=np.int64)
    per_ct = N // (m.block * m.n_seg)
    out, labels = [], []
    _, trees = Cp.parse_forest(case["text"])
    for c in range(-(-len(qs) // per_ct)):
        part = qs[c * per_ct:(c + 1) * per_ct]
        X = Cp.encrypt_queries(bgv, keys, m, part, case["enc_seed"], index0=c * p)
        res = Cp.infer(E, m, X, N) if case["encrypted"] else Cp.infer(E, m, X, N, g)
        slots = bgv.decrypt_slots(keys.sk, res).astype(np.int64)
        for j, bits in enumerate(Cp.decode_labels(m, slots, len(part))):
            if bits != Cp.classify_plain(trees, part[j]):
                raise AssertionError(f"{case['name']}: oracle labels differ from plaintext for query {c * per_ct + j}")
            labels.append(bits)
        out.append({"level": int(res.shape[1]), "residues": residue_digests(res)})
        print(f"  {case['name']}: query ciphertext {c} done ({time.time() - t0:.0f} s)", flush=True)
    doc = {"source": "oracle.copse.infer (Algorithm 1, Section 4.3) over oracle.bgv; written by "
                      "tests/golden/make_digests.py, which calls only oracle/"}
    doc.update(case)
    doc["digests"] = out
    doc["oracle_threads"] = B.oracle_threads()
    doc["oracle_seconds"] = round(time.time() - t0, 1)
    path = os.path.join(HERE, f"digests_{case['name']}.json")
    with open(path, "w") as f:
        json.dump(doc, f, indent=1)
        f.write("\n")
    print(f"wrote {path} ({doc['oracle_seconds']} s)")


if __name__ == "__main__":
    names = sys.argv[1:] or list(CASES)
    for n in names:
        run(CASES[n]())
