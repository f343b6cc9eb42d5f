"""The C ABI library loads and exports every entry point that include/bdem.h declares (no GPU needed)."""
import os
import re
import subprocess

import pytest

import paper_2308_10459_gb300 as pkg
from paper_2308_10459_gb300 import build as bmod

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    text = open(os.path.join(ROOT, "include", "bdem.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bdem_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared()
    for required in ("bdem_create", "bdem_add_bonds", "bdem_step", "bdem_read_state", "bdem_destroy",
                     "bdem_last_error", "bdem_pcg_static"):
        assert required in names


def test_library_builds_loads_and_exports_every_declared_symbol():
    lib = bmod.build()
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (bdem_[a-z_]+)\b", out))
    missing = [n for n in declared() if n not in exported]
    assert not missing, missing
    L = pkg.load()
    for n in declared():
        assert hasattr(L, n)
    assert set(pkg.exported_symbols()) == set(declared())


def test_binding_fails_loudly_without_the_library(tmp_path):
    import importlib
    with pytest.raises(RuntimeError):
        pkg._lib = None
        try:
            pkg.load(str(tmp_path / "missing.so"))
        finally:
            pkg._lib = None
    pkg.load()
