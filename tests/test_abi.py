"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/escape.h (no GPU needed: no compute calls here)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "escape.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(escape_[a-z0-9_]+)\s*\(", src)))


def test_library_builds_and_exports_every_declared_symbol():
    from paper_1610_09411_gb300 import build
    lib = build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (escape_[a-z0-9_]+)", out))
    declared = _declared()
    assert len(declared) >= 9
    missing = [f for f in declared if f not in exported]
    assert not missing, missing


def test_binding_loads_and_has_every_entry_point():
    from paper_1610_09411_gb300 import escape as esc
    for name in _declared():
        assert hasattr(esc.LIB, name)
        assert hasattr(esc, name), f"binding lacks {name}"
    assert esc.escape_status_str(0) == "ok"
    assert "invalid" in esc.escape_status_str(1)
    assert esc.escape_last_cuda_error() == (0, "")      # no CUDA call has failed on this thread


def test_sources_target_sm103a_only():
    from paper_1610_09411_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_no_oracle_on_product_path():
    pkg = os.path.join(ROOT, "paper_1610_09411_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "escape_oracle" not in text, f
