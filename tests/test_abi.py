"""The C ABI library loads on a machine without a GPU and exports every entry
point that include/fgraft.h declares (no compute calls are made here)."""
import ctypes
import os
import re

from paper_2609_30493_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "fgraft.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fgraft_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared()
    for n in ("fgraft_build_scaffold", "fgraft_harvest_block", "fgraft_prune",
              "fgraft_search", "fgraft_dense_block_dist", "fgraft_prune_lists",
              "fgraft_index_destroy", "fgraft_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(build.build())
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing
    lib.fgraft_last_error.restype = ctypes.c_char_p
    assert lib.fgraft_last_error() is not None


def test_binding_names_match_header():
    from paper_2609_30493_gb300 import fgraft
    assert sorted(fgraft.EXPORTS) == declared()
