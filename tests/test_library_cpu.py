"""CPU checks of the C ABI library: it builds for sm_103a, loads without a GPU,
exports every entry point include/sghsc.h declares, and the product path and
the oracle do not import each other."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "sghsc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^[A-Za-z_][\w \*]*?\b((?:sg|hsc|mean)_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("sg_setup", "sg_apply", "hsc_precond_apply", "sg_solve", "sg_qoi_grad", "sg_destroy"):
        assert required in names


def test_library_builds_and_exports_header_symbols():
    import importlib.util
    spec = importlib.util.spec_from_file_location("sghsc_build", os.path.join(ROOT, "paper_1205_1864_gb300", "build.py"))
    B = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(B)
    lib_path = B.build()
    lib = ctypes.CDLL(lib_path)           # loads on a machine without a GPU: no CUDA call at load
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def _imports(path):
    out = []
    for dirpath, _, files in os.walk(path):
        for f in files:
            if f.endswith(".py"):
                txt = open(os.path.join(dirpath, f)).read()
                out += re.findall(r"^\s*(?:from|import)\s+([\w\.]+)", txt, flags=re.M)
    return out


def test_product_and_oracle_do_not_import_each_other():
    prod = _imports(os.path.join(ROOT, "paper_1205_1864_gb300"))
    orc = _imports(os.path.join(ROOT, "oracle"))
    assert not any(m.startswith("oracle") for m in prod)
    assert not any(m.startswith("sg_inputs") for m in prod)
    assert not any(m.startswith("paper_1205_1864_gb300") for m in orc)
    csrc = os.path.join(ROOT, "paper_1205_1864_gb300", "csrc")
    for f in os.listdir(csrc):
        assert "oracle" not in open(os.path.join(csrc, f)).read().lower() or f.endswith(".md")
