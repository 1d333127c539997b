"""The committed ncu summaries under profiles/: every per-family file carries the
machine-readable lines bench.py reads (source file, its hash, the unit and the per-unit
counters), names a source file that exists, and every ncu command in any summary leaves
the GPU clocks alone."""
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md")))
FAMILIES = [p for p in PROFILES if not os.path.basename(p).startswith("launches_")]


def _kv(path):
    kv = {}
    for ln in open(path).read().splitlines():
        if ln.startswith("- ") and ":" in ln:
            k, v = ln[2:].split(":", 1)
            kv[k.strip()] = v.strip()
    return kv


def test_there_are_summaries():
    assert any(os.path.basename(p).startswith("launches_") for p in PROFILES)
    assert FAMILIES


@pytest.mark.parametrize("path", FAMILIES, ids=os.path.basename)
def test_family_summary_is_machine_readable(path):
    kv = _kv(path)
    assert os.path.exists(os.path.join(ROOT, "paper_2104_09583_gb300", "csrc", kv["source"]))
    assert re.fullmatch(r"[0-9a-f]{16}", kv["source_sha256_16"])
    assert kv["unit"]
    for k in ("unit_algorithmic_bytes", "dram_bytes_per_unit", "warp_instructions_per_unit"):
        assert float(kv[k]) > 0, k


@pytest.mark.parametrize("path", PROFILES, ids=os.path.basename)
def test_ncu_commands_keep_clocks(path):
    text = open(path).read().replace("\\\n", " ")
    cmds = [ln for ln in text.splitlines() if re.search(r"\bncu\b", ln) and "--" in ln]
    assert cmds, "no ncu command recorded"
    for c in cmds:
        assert "--clock-control none" in c, c
