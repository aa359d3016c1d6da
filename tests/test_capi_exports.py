"""The C-ABI library builds for sm_103a and exports every symbol of include/*.h (no GPU needed)."""
import ctypes
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(hdr).read()
        for m in re.finditer(r"^SCTM_API\s+[\w\s\*]*?\b(\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


def test_library_builds_and_exports_declared_symbols():
    from paper_2502_10298_gb300 import build
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    names = declared_symbols()
    assert len(names) >= 10
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_load():
    import paper_2502_10298_gb300 as S
    S.load_library()
