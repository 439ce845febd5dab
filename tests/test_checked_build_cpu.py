"""The checked build (shared-memory redzones, csrc/checked.cuh) compiles, links
and exports the whole C ABI, and the status codes of the header and the binding
agree.  No GPU needed: nothing here launches a kernel."""
import ctypes
import os
import re

import pytest

from paper_1505_04979_gb300 import binding as B
from paper_1505_04979_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "polarbp.h")


def declared_functions():
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    return sorted(set(re.findall(r"\b(polarbp_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def checked_lib():
    return ctypes.CDLL(build.build(checked=True))


def test_checked_build_exports_every_declared_symbol(checked_lib):
    for name in declared_functions():
        assert hasattr(checked_lib, name), name


def test_checked_build_says_so(checked_lib):
    checked_lib.polarbp_version.restype = ctypes.c_char_p
    assert checked_lib.polarbp_version().decode().endswith("sm_103a) checked")
    assert not B.polarbp_version().endswith("checked")


def test_checked_build_rejects_a_null_handle(checked_lib):
    assert checked_lib.polarbp_get_status(None, None) == B.POLARBP_ERR_ARG


def test_status_codes_agree_with_the_header():
    text = open(HEADER).read()
    enum = text[text.index("typedef enum polarbp_status"):text.index("} polarbp_status;")]
    codes = dict((k, int(v)) for k, v in re.findall(r"\b(POLARBP_\w+)\s*=\s*(\d+)", enum))
    assert codes["POLARBP_ERR_CHECK"] == 7
    for k, v in codes.items():
        assert getattr(B, k) == v, k
