"""The C-ABI library builds for sm_103a and exports every entry point that
include/imrp.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "imrp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(imrp_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2111_13072_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("imrp_create", "imrp_load_particles", "imrp_step", "imrp_spectrum"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_2111_13072_gb300 import imrp
    assert sorted(imrp.EXPORTS) == _declared()


def test_binding_loads_and_fills_defaults(lib):
    from paper_2111_13072_gb300 import imrp
    p = imrp.default_params()  # host-only call
    assert p.l_max == 8 and p.N == 20000 and p.R_E_m == 4e-3 and p.precision == 0


def test_oracle_is_not_imported_by_the_product():
    pkg = os.path.join(ROOT, "paper_2111_13072_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f), errors="ignore").read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "imrp_oracle" not in text, f
