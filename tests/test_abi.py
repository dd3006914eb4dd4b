"""The C ABI library builds for sm_103a, loads without a GPU and exports every
entry point that include/sie.h declares (no compute call is made here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "sie.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sie_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_binding_symbols():
    import paper_2003_11679_gb300 as sie
    assert sorted(sie.SYMBOLS) == _declared()


def test_library_exports_every_declared_symbol():
    from paper_2003_11679_gb300 import build
    so = build.build()
    L = ctypes.CDLL(so)
    for name in _declared():
        assert hasattr(L, name), name


def test_params_default_matches_paper():
    import paper_2003_11679_gb300 as sie
    from paper_2003_11679_gb300 import build
    build.build()
    p = sie.params()
    assert p.stencil_order == 2 and p.near_radius == 5 and p.skin_cutoff == 5.0
    assert p.tol_outer == 1e-4 and p.tol_inner == 1e-6 and p.maxit == 800


def test_no_device_is_an_error_not_a_crash():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2003_11679_gb300 as sie
    from paper_2003_11679_gb300 import build
    build.build()
    with pytest.raises(sie.SieError):
        sie.Context(0)
