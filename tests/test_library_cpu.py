"""CPU-side checks of the CUDA library: it builds, loads without a GPU and exports every entry
point declared in include/dfhf.h (no compute calls here)."""
import ctypes
import os
import re

from paper_1707_03771_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^\s*(?:int|void|long long|const char\*)\s+(\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    declared = _declared()
    assert declared, "no declarations found"
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(binding.EXPORTED) == declared


def test_strerror_without_gpu():
    lib = binding.load()
    assert lib.df_strerror(0) == b"ok"
    assert lib.df_strerror(-1) == b"invalid argument"
