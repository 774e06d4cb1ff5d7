"""The C-ABI library builds, loads and exports every entry point that
include/aether_gb.h declares (no compute calls: runs without a GPU)."""
import ctypes
import os
import re

from paper_2608_14048_gb300 import aether as A
from paper_2608_14048_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "aether_gb.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(aeth_[a-z_]+)\s*\(", txt)))


def test_header_declarations_match_binding():
    assert declared_symbols() == sorted(A.EXPORTS)


def test_library_loads_and_exports_every_symbol():
    path = B.build()
    lib = ctypes.CDLL(path)
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_has_no_cpu_fallback():
    # the binding module must not import the oracle or any CPU solver
    src = open(os.path.join(ROOT, "paper_2608_14048_gb300", "aether.py")).read()
    assert "oracle" not in src.replace("no CPU fallback", "")
    assert "import oracle" not in src
