"""The host forest compiler (C ABI, no GPU needed) on damaged forest texts: seeded
random edits (tokens inserted, deleted, replaced, lines cut short) of valid forests
in the input representation of Section 5.  For every text the library and the
oracle must agree on whether it is a forest; the library must refuse a bad one
with a parse or argument error (never crash or accept it); and where both accept,
the compiled layout (K, q, branches, leaves, depth, block, row segments) and the
plaintext classification must be the oracle's."""
import random

import numpy as np
import pytest

from oracle import copse as Cp
from paper_2104_09583_gb300 import synth

K = pytest.importorskip("paper_2104_09583_gb300.copse", reason="CUDA library not built")

LOG_N = 12                       # slot rows of 2048: the larger forests compile in row segments
TOKENS = ["b", "l", "0", "1", "2", "5", "63", "64", "-1", "x", "\n", "", "99999999999", "b 0", "l 0 l 0", "3.5"]


def _damaged(rng, text):
    words = text.replace("\n", " \n ").split(" ")
    for _ in range(rng.randint(1, 3)):
        if not words:
            words = ["l"]
        i = rng.randrange(len(words))
        op = rng.randrange(6)
        if op >= 4 and words[i].isdigit():             # another feature, threshold or class index
            words[i] = str(rng.randrange(70))
        elif op == 0:
            words.insert(i, rng.choice(TOKENS))
        elif op == 1 and len(words) > 1:
            del words[i]
        elif op == 2:
            words[i] = rng.choice(TOKENS)
        else:
            words = words[:i]
    return " ".join(words).replace(" \n ", "\n")


def _cases(n=3000, seed=2024):
    rng = random.Random(seed)
    base = [synth.random_forest(300 + s, 1 + s % 4, 2 + s % 5, 1 + s % 6, 6, 3, complete=(s % 3 == 0))
            for s in range(6)]
    base.append("a b\nb 0 5 l 0 b 0 9 l 1 l 0\nl 1\n")
    out = []
    for _ in range(n):
        p, nf = rng.choice([(4, 0), (6, 0), (6, 3), (6, 5)])
        out.append((_damaged(rng, rng.choice(base)), p, nf))
    return out


def test_damaged_forests_agree_with_oracle():
    accepted = rejected = 0
    for text, p, nf in _cases():
        try:
            om = Cp.compile_forest(text, p, nf, 1 << (LOG_N - 1))
        except (ValueError, IndexError):
            om = None
        try:
            h = K.copse_compile_forest(text, p, nf, LOG_N)
        except K.CopseError as e:
            assert om is None, f"the library refused a forest the oracle compiles ({e}):\n{text}"
            assert e.name in ("EPARSE", "EINVAL", "EFIT"), e.name
            rejected += 1
            continue
        try:
            assert om is not None, f"the library compiled a text the oracle refuses:\n{text}"
            info = K.copse_model_info_get(h)
            got = (info["K"], info["q"], info["b"], info["n_leaves"], info["depth"], info["block"],
                   info["n_segments"], info["block_branches"], info["block_leaves"], info["n_features"])
            want = (om.K, om.q, om.b_total, om.L_total, om.d, om.block, om.n_seg, om.b, om.L, om.n_features)
            assert got == want, text
            qs = synth.random_queries(accepted, 4, om.n_features, p)
            bits = K.copse_classify_plain(h, qs)
            _, trees = Cp.parse_forest(text)
            assert [b.tolist() for b in bits] == [Cp.classify_plain(trees, x) for x in qs], text
            accepted += 1
        finally:
            K.copse_model_destroy(h)
    # the edits leave both kinds of text in the sample
    assert accepted >= 100 and rejected >= 500, (accepted, rejected)
