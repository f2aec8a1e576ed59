"""The C-ABI library loads and exports every entry point that include/amfmm.h
declares (no compute call: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "amfmm.h")


def declared_symbols():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fmm_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("fmm_build_tree", "fmm_upward", "fmm_interact", "fmm_downward", "fmm_forces",
                 "fmm_create", "fmm_destroy", "fmm_get_stats", "fmm_last_error"):
        assert name in syms


def test_library_exports_every_declared_symbol():
    from paper_1706_06989_gb300 import build
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_1706_06989_gb300 import fmm
    monkeypatch.setattr(fmm, "LIB_PATH", str(tmp_path / "absent.so"))
    monkeypatch.setattr(fmm, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        fmm.load()


def test_binding_structs_match_header():
    """ctypes mirrors of fmm_opts / fmm_stats have the header's field order."""
    from paper_1706_06989_gb300 import fmm
    src = open(HEADER).read()
    opts = re.search(r"typedef struct \{(.*?)\} fmm_opts;", src, re.S).group(1)
    names = re.findall(r"\b(\w+)\s*;", re.sub(r"/\*.*?\*/", "", opts, flags=re.S))
    assert names == [f[0] for f in fmm._Opts._fields_]


def test_generated_expansion_header_matches_its_generator():
    """csrc/expansion_gen.cuh is the output of gen_expansion.py (no hand edits)."""
    from paper_1706_06989_gb300 import gen_expansion
    with open(gen_expansion.OUT) as f:
        assert f.read() == gen_expansion.render()
