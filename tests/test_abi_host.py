"""Host-side checks of the C-ABI library (no GPU needed): it loads, exports
every function include/copse.h declares, and its forest compiler and
plaintext classifier agree with the oracle's exactly."""
import numpy as np
import pytest

from conftest import read_golden
from oracle import copse as Cp
from paper_2104_09583_gb300 import synth

K = pytest.importorskip("paper_2104_09583_gb300.copse", reason="CUDA library not built")


def test_exports_every_declared_symbol():
    names = K.declared_functions()
    assert len(names) >= 25
    lib = K.library()
    assert [n for n in names if not hasattr(lib, n)] == []


def _forests():
    out = [(read_golden("fig1_forest.txt"), 4, 2, 10)]
    for s in range(8):
        out.append((synth.random_forest(300 + s, 1 + s % 4, 2 + s % 5, 1 + s % 6, 6, 3, complete=(s % 3 == 0)),
                    6, 0, 12))
    out.append(("a b\nb 0 5 l 0 b 0 9 l 1 l 0\nl 1\n", 4, 1, 8))
    for name in ("toy-n1024", "forest100-n16384", "batch3-n16384"):
        W = synth.WORKLOADS[name]
        for k, text in enumerate(W.forest_texts()):
            out.append((text, W.precision(k), W.n_features(k), W.log_n))
    return out


@pytest.mark.parametrize("case", range(len(_forests())))
def test_compile_matches_oracle(case):
    text, p, nf, logN = _forests()[case]
    om = Cp.compile_forest(text, p, nf)
    h = K.copse_compile_forest(text, p, nf, logN)
    try:
        info = K.copse_model_info_get(h)
        assert (info["K"], info["q"], info["b"], info["n_leaves"], info["depth"], info["block"]) == \
            (om.K, om.q, om.b, om.L, om.d, om.block)
        assert info["n_features"] == om.n_features and info["levels_used"] == Cp.levels_needed(om)
        ex = K.copse_model_export(h)
        assert ex["thr_slot"].tolist() == om.thr_slot
        assert ex["slot_branch"].tolist() == om.slot_branch
        assert np.array_equal(ex["R"], om.R)
        assert np.array_equal(ex["lvl"], np.stack(om.lvl))
        assert np.array_equal(ex["mask"], np.stack(om.mask))
        assert ex["br_level"].tolist() == om.br_level
        rs, ls = K.copse_model_rotations(h)
        ors, ols = Cp.rotation_sets(om)
        assert rs == ors and ls == ols
        # baby-step / giant-step plans: the same key sets as the oracle's
        for g in [(1, 1), (2, 3), (5, 4), (om.q, om.b)]:
            K.copse_model_set_bsgs(h, *g)
            assert K.copse_model_get_bsgs(h) == g
            assert K.copse_model_rotations(h) == Cp.rotation_sets(om, g), g
        K.copse_model_set_bsgs(h, 0, 0)
        qs = synth.random_queries(case, 20, om.n_features, p)
        got = K.copse_classify_plain(h, qs)
        _, trees = Cp.parse_forest(text)
        for j in range(len(qs)):
            assert got[j].tolist() == Cp.classify_plain(trees, qs[j])
    finally:
        K.copse_model_destroy(h)


@pytest.mark.parametrize("text,p,code", [
    ("a b\n", 4, "EPARSE"),                           # no tree
    ("a b\nb 0 3 l 0\n", 4, "EPARSE"),                # branch missing a subtree
    ("a b\nl 0 l 1\n", 4, "EPARSE"),                  # trailing tokens
    ("a b\nx 0\n", 4, "EPARSE"),                      # unknown token
    ("a b\nb 0 16 l 0 l 1\n", 4, "EINVAL"),           # threshold needs 5 bits
    ("a b\nb 0 3 l 0 l 2\n", 4, "EINVAL"),            # class index out of range
    ("a b\nl 0\n", 4, "EINVAL"),                      # no branches at all
])
def test_compile_errors(text, p, code):
    with pytest.raises(K.CopseError) as e:
        K.copse_compile_forest(text, p, 0, 10)
    assert e.value.name == code


def test_block_must_fit_a_row():
    text = synth.random_forest(5, 4, 5, 8, 8, 4, complete=True)
    with pytest.raises(K.CopseError) as e:
        K.copse_compile_forest(text, 8, 8, 8)   # N = 256: a row has 128 slots
    assert e.value.name == "EFIT"


def test_tuning_calls_marshal_and_reject_null_handles():
    """The autotuning entry points check their handles before any device work."""
    for call in (lambda: K.copse_tune_ntt(None),
                 lambda: K.copse_tune_bsgs(None, None, [0, 8], [0, 4]),
                 lambda: K.copse_tune_dnum(10, 50, 4, None, [1, 2]),
                 lambda: K.copse_tune_fused(None, None),
                 lambda: K.copse_ctx_set_ntt_fused_max(None, 64)):
        with pytest.raises(K.CopseError) as e:
            call()
        assert e.value.name == "EINVAL"


def test_encrypted_mode_key_sets_match_oracle():
    """Encrypted-model mode runs the products over every diagonal: its rotation sets
    (plain and baby-step / giant-step) equal the oracle's."""
    text = synth.random_forest(77, 3, 4, 3, 5, 3, complete=False)
    om = Cp.compile_forest(text, 5, 3)
    h = K.copse_compile_forest(text, 5, 3, 10)
    try:
        K.copse_model_set_encrypted(h, True)
        for g in [(0, 0), (4, 3), (8, 8)]:
            K.copse_model_set_bsgs(h, *g)
            assert K.copse_model_rotations(h) == Cp.encrypted_rotation_sets(om, g), g
        K.copse_model_set_encrypted(h, False)
        K.copse_model_set_bsgs(h, 0, 0)
        assert K.copse_model_rotations(h) == Cp.rotation_sets(om)
    finally:
        K.copse_model_destroy(h)


def test_shuffle_plan_validation_and_codebook():
    """copse_model_set_shuffle accepts a padded permutation whose codebook carries each
    leaf's class, rejects anything else, and adds one prime and the shift rotations."""
    text = synth.random_forest(77, 3, 4, 3, 5, 3, complete=False)
    om = Cp.compile_forest(text, 5, 3)
    h = K.copse_compile_forest(text, 5, 3, 10)
    try:
        base = K.copse_model_info_get(h)
        assert base["n_out"] == om.L
        assert K.copse_model_codebook(h).tolist() == om.labels_per_leaf
        src, code = synth.shuffle_plan(3, om.labels_per_leaf, 11, 3)
        K.copse_model_set_shuffle(h, src, code)
        info = K.copse_model_info_get(h)
        assert info["n_out"] == om.L + 11 and info["levels_used"] == base["levels_used"] + 1
        assert K.copse_model_codebook(h).tolist() == code.tolist()
        want = sorted(set(Cp.shuffle_diagonals(om, src, 1024)) - {0})
        rs, ls = K.copse_model_rotations(h)           # the reshuffle and level sets are unchanged
        assert (rs, ls) == Cp.rotation_sets(om) and want
        bad = src.copy()
        bad[bad == 0] = 1                              # leaf 1 twice, leaf 0 missing
        for s_, c_ in [(bad, code), (src, (code + 1) % 3), (src[: om.L - 1], code[: om.L - 1])]:
            with pytest.raises(K.CopseError) as e:
                K.copse_model_set_shuffle(h, s_, c_)
            assert e.value.name == "EINVAL"
        K.copse_model_set_shuffle(h)
        assert K.copse_model_info_get(h)["n_out"] == om.L
    finally:
        K.copse_model_destroy(h)


def test_no_device_fails_loudly():
    """Without a usable CUDA device the library refuses to make a context (ECUDA): there is
    no host fallback for any step of the path."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    with pytest.raises(K.CopseError) as e:
        K.copse_ctx_create(10, 50, 8)
    assert e.value.name == "ECUDA"


_NULL_CALLS = r'''
import ctypes as C, sys
sys.path.insert(0, sys.argv[1])
import paper_2104_09583_gb300.copse as K
lib = K.library()
SCALARS = (C.c_int, C.c_uint32, C.c_int32, C.c_uint64, C.c_int64, C.c_size_t, C.c_double, C.c_float)
for name in K.declared_functions():
    f = getattr(lib, name)
    types = list(f.argtypes or [])
    f.argtypes = [t if t in SCALARS else C.c_void_p for t in types]
    r = f(*[0 if t in SCALARS else None for t in types])
    print(name, r if isinstance(r, int) or r is None else "value", flush=True)
'''


def test_every_entry_point_refuses_null_arguments():
    """Every function include/copse.h declares, called with null handles and pointers and zero
    sizes, returns (an error status where it returns one) without touching memory: the
    process survives all of them.  Destroy functions take NULL as a no-op."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _NULL_CALLS, root], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    got = dict(ln.rsplit(" ", 1) for ln in r.stdout.splitlines())
    assert sorted(got) == sorted(K.declared_functions())
    # not statuses: a count, flags, the error text, the switch for the kernel timers
    not_status = {"copse_ctbuf_count", "copse_model_is_encrypted", "copse_model_is_fused", "copse_last_error",
                  "copse_stats_enable"}
    for name, ret in got.items():
        if name in not_status or name.endswith("_destroy"):
            continue
        assert int(ret) < 0, f"{name} returned {ret} for null arguments"


def test_fused_mode_key_sets_and_levels_match_oracle():
    """Fused level products (F_k = S_k R on Decisions): the host's rotation sets under plain and
    baby-step / giant-step plans and its prime count equal the oracle's."""
    for s in range(6):
        text = synth.random_forest(300 + s, 1 + s % 4, 2 + s % 5, 1 + s % 6, 6, 3, complete=(s % 3 == 0))
        om = Cp.compile_forest(text, 6, 0)
        h = K.copse_compile_forest(text, 6, 0, 12)
        try:
            K.copse_model_set_fused(h, 1)
            assert K.copse_model_is_fused(h)
            assert K.copse_model_info_get(h)["levels_used"] == Cp.levels_needed(om, fused=True)
            for g in [(0, 0), (2, 3), (5, 4), (om.q, om.b)]:
                K.copse_model_set_bsgs(h, *g)
                assert tuple(K.copse_model_rotations(h)) == tuple(Cp.rotation_sets(om, g, fused=True)), (s, g)
        finally:
            K.copse_model_destroy(h)
