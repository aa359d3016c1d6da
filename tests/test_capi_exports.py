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


def _header_source():
    src = "\n".join(open(h).read() for h in glob.glob(os.path.join(ROOT, "include", "*.h")))
    return re.sub(r"/\*.*?\*/", "", src, flags=re.S)   # drop comments


def test_binding_argument_counts_match_header():
    """Every declared entry point has a ctypes signature with as many arguments
    as its prototype, so the binding cannot drift from the header."""
    import paper_2502_10298_gb300 as S
    lib = S.load_library()
    protos = {}
    for m in re.finditer(r"^SCTM_API\s+[\w\s\*]*?\b(\w+)\s*\(([^)]*)\)\s*;", _header_source(), flags=re.M):
        params = [p.strip() for p in m.group(2).split(",") if p.strip() and p.strip() != "void"]
        protos[m.group(1)] = len(params)
    assert protos.keys() == declared_symbols()
    for name, n in protos.items():
        f = getattr(lib, name)
        assert f.argtypes is not None, name
        assert len(f.argtypes) == n, (name, len(f.argtypes), n)


def test_config_struct_matches_header():
    """The ctypes Config lists the fields of sctm_config in the header's order."""
    import paper_2502_10298_gb300 as S
    body = re.search(r"typedef\s+struct\s*\{(.*?)\}\s*sctm_config\s*;", _header_source(), flags=re.S).group(1)
    fields = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        names = decl.split(None, 1)[1]   # drop the type
        fields += [n.strip().lstrip("*") for n in names.split(",")]
    assert [f for f, _ in S.Config._fields_] == fields


def test_missing_library_fails_loudly():
    """Without the built library the binding raises: there is no CPU fallback."""
    import subprocess
    import sys
    code = ("import paper_2502_10298_gb300.api as a\n"
            "try:\n"
            "    a.load_library('/nonexistent/libsplitctmrg.so')\n"
            "except RuntimeError as e:\n"
            "    print('raised:', e)\n"
            "else:\n"
            "    print('no error')\n")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    assert out.stdout.startswith("raised:") and "not found" in out.stdout, out.stdout
