"""The C-ABI library builds for sm_103a, loads, and exports every symbol the
headers declare; the Python binding wraps each of them by the same name.
No GPU is needed (no compute calls)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(tm_\w+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_1311_4521_gb300 import build
    return build.build()


def test_headers_declare_the_boundary():
    names = declared_functions()
    for required in ("tm_hopping_eo", "tm_Qtm", "tm_gauge_create", "tm_ctx_create", "tm_spinor_pack"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_wraps_every_declared_symbol(libpath):
    from paper_1311_4521_gb300 import tmhop
    missing = [n for n in declared_functions() if not callable(getattr(tmhop, n, None))]
    assert not missing, missing


def test_host_side_queries_without_gpu(libpath):
    from paper_1311_4521_gb300 import tmhop
    assert tmhop.tm_spinor_bytes(10, tmhop.TM_F64) == 1920
    assert tmhop.tm_spinor_bytes(10, tmhop.TM_F32) == 960
    assert tmhop.tm_spinor_bytes(10, tmhop.TM_F16) == 520
    assert tmhop.tm_spinor_bytes(10, 7) == 0
    assert tmhop.lib.tm_status_string(tmhop.TM_ERR_ARG).decode() == "invalid argument"
    # a null context is rejected before anything touches a device
    assert tmhop.lib.tm_Qtm(None, None, None, None, 0.1, 0.0, 1, None) == tmhop.TM_ERR_ARG
