"""The C ABI library builds, loads, and exports every entry point include/assn.h declares.

No compute call is made here (these run without a GPU).
"""
import ctypes
import os
import re

import pytest

from tests.helpers import ROOT, ensure_built

HEADER = os.path.join(ROOT, "include", "assn.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(assn_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    ensure_built()
    return ctypes.CDLL(os.path.join(ROOT, "paper_1911_08801_gb300", "libassn.so"))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("assn_create", "assn_set_cross_sections", "assn_set_product_quadrature",
                     "assn_set_artificial_scattering", "assn_step", "assn_scalar_flux", "assn_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(lib):
    from paper_1911_08801_gb300 import _lib
    assert set(declared_functions()) <= set(_lib.SIGNATURES), set(declared_functions()) - set(_lib.SIGNATURES)


def test_status_strings_and_version(lib):
    from paper_1911_08801_gb300 import _lib
    assert _lib.assn_abi_version() == 1
    assert _lib.status_string(0) == "ASSN_OK"
    assert _lib.status_string(-4) == "ASSN_ERR_UNSTABLE"
    assert _lib.status_string(-99) == "ASSN_ERR_UNKNOWN"


def test_invalid_arguments_rejected_before_any_device_work(lib):
    from paper_1911_08801_gb300 import _lib
    with pytest.raises(_lib.AssnError) as e:
        _lib.assn_create(0, 4, 0.0, 1.0, 0.0, 1.0, 1)
    assert e.value.status == _lib.ASSN_ERR_ARG
    with pytest.raises(_lib.AssnError) as e:
        _lib.assn_create(4, 4, 0.0, 1.0, 0.0, 1.0, 17)
    assert e.value.status == _lib.ASSN_ERR_ARG
    assert _lib.assn_destroy(None) is None
