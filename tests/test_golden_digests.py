"""The stored oracle digests (tests/golden/digests_*.json) are the generator's: every
case's parameters equal tests/golden/make_digests.py's, the inputs come from the seeded
generators, and re-running the oracle on the smallest case reproduces its digests."""
import importlib.util
import json
import os

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = os.path.join(HERE, "golden")


def _generator():
    spec = importlib.util.spec_from_file_location("make_digests", os.path.join(GOLD, "make_digests.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("name", ["batch3c-n16384", "encmodel-n32768", "serving64-n32768"])
def test_digest_files_match_generator(name):
    gen = _generator()
    doc = json.load(open(os.path.join(GOLD, f"digests_{name}.json")))
    case = gen.CASES[name]()
    for k, v in case.items():
        assert doc[k] == v, f"{name}: {k} differs from the generator"
    assert doc["source"].startswith("oracle.copse.infer")
    n_res = [len(d["residues"][0]) for d in doc["digests"]]
    assert all(n == doc["digests"][0]["level"] for n in n_res)


def test_oracle_reproduces_batch3c_digests(tmp_path, monkeypatch):
    gen = _generator()
    monkeypatch.setattr(gen, "HERE", str(tmp_path))
    gen.run(gen.CASES["batch3c-n16384"]())
    got = json.load(open(tmp_path / "digests_batch3c-n16384.json"))
    want = json.load(open(os.path.join(GOLD, "digests_batch3c-n16384.json")))
    assert got["digests"] == want["digests"]
