"""The C-ABI library builds, loads and exports every function include/qsim.h declares.

No compute call is made (CPU-only check)."""
import ctypes
import os
import re

import pytest

from conftest import ROOT


def _declared():
    src = open(os.path.join(ROOT, "include", "qsim.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z][a-z0-9_]*)\s*\(", src,
                       flags=re.M)
    return sorted({n for n in names if n.startswith(("sv_", "dm_", "qs_"))})


@pytest.fixture(scope="module")
def lib_path():
    from paper_2008_13490_gb300 import _build
    return _build.build()


def test_header_declares_the_abi():
    names = _declared()
    for want in ("sv_create", "sv_apply_circuit", "sv_probs", "dm_apply_channels", "sv_grad"):
        assert want in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_abi(lib_path):
    import paper_2008_13490_gb300 as qs
    qs.load()
    assert set(_declared()) <= set(qs.exported_symbols())
    assert qs.version().startswith("qsim-gb300")


def test_gate_struct_layout():
    import paper_2008_13490_gb300 as qs
    assert qs.GATE_DTYPE.itemsize == 296
    src = open(os.path.join(ROOT, "include", "qsim.h")).read()
    for name, val in qs.KIND.items():
        assert re.search(rf"QS_{name}\s*=\s*{val}\b", src), name
