"""The C-ABI library loads without a GPU and exports every declared symbol."""
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"^\s*(?:const\s+)?[\w]+\s*\**\s*(mf_\w+)\s*\(", src, flags=re.M))
    return names


def test_library_exports_every_declared_symbol():
    import ctypes
    import paper_2506_05793_gb300 as mf
    mf.build()
    lib = ctypes.CDLL(mf.build.__globals__["LIB"])
    decl = declared_symbols()
    assert len(decl) >= 20
    missing = [n for n in decl if not hasattr(lib, n)]
    assert not missing, missing
    # the binding wraps exactly the declared entry points
    assert set(mf.exported_symbols()) <= decl


def test_exports_are_c_linkage():
    import paper_2506_05793_gb300 as mf
    mf.build()
    out = subprocess.run(["nm", "-D", "--defined-only", mf.build.__globals__["LIB"]],
                         stdout=subprocess.PIPE, text=True).stdout
    syms = {l.split()[-1] for l in out.splitlines() if l.strip()}
    for n in declared_symbols():
        assert n in syms, n
