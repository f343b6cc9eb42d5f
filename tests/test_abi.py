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


def test_binding_structs_match_the_header_layout(tmp_path):
    """Every struct of include/bdem.h has the same size and field offsets in the ctypes binding (compiled and printed
    with the host C compiler)."""
    import ctypes
    structs = {name: getattr(pkg, name) for name in ("bdem_material", "bdem_allocator", "bdem_config", "bdem_step_stats",
                                                   "bdem_profile")}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "bdem.h"', 'int main(void) {']
    for name, cls in structs.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'  printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines += ['  return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for name, cls in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert got[(name, f)] == getattr(cls, f).offset, (name, f)


def test_oracle_binding_structs_match_its_header(tmp_path):
    """The same layout check for the oracle's C structs and their ctypes mirrors (test infrastructure)."""
    import ctypes
    import oracle
    structs = {"orc_config": oracle.OrcConfig, "orc_problem": oracle.OrcProblem, "orc_scene_stats": oracle.OrcStats}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "bdem_oracle.h"', 'int main(void) {']
    for name, cls in structs.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'  printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines += ['  return 0;', '}']
    src = tmp_path / "olayout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "olayout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "oracle"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for name, cls in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert got[(name, f)] == getattr(cls, f).offset, (name, f)
