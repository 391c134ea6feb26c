"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/spirec.h declares (no compute call: no GPU needed)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(spirec_[a-z0-9_]+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_0908_3252_gb300 import build, spirec
    build.build()
    return spirec.load()


def test_header_declares_entry_points():
    names = _declared()
    for n in ["spirec_plan_create", "spirec_set_trajectory", "spirec_set_data", "spirec_set_reg",
              "spirec_solve", "spirec_plan_destroy", "spirec_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in sorted(_declared()):
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"


def test_binding_covers_every_declared_symbol(lib):
    from paper_0908_3252_gb300 import spirec
    assert set(spirec.SIGNATURES) == _declared()


def test_version_and_error_without_gpu(lib):
    from paper_0908_3252_gb300 import spirec
    assert "sm_103a" in spirec.spirec_version()
    assert isinstance(spirec.spirec_last_error(), str)


def test_null_plan_is_rejected_without_gpu(lib):
    from paper_0908_3252_gb300 import spirec
    assert lib.spirec_plan_destroy(None) == spirec.SPIREC_OK
    assert lib.spirec_plan_info(None, None, None, None, None, None) == spirec.SPIREC_EINVAL
    assert lib.spirec_plan_create(None, 8, 8, 0, 0, None, None, None) == spirec.SPIREC_EINVAL
