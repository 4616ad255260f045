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


def test_header_is_plain_c_and_links(tmp_path):
    """include/assn.h compiles as pedantic C99, and a C program links against libassn.so and calls the
    device-free entry points (no GPU needed)."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    inc = os.path.join(root, "include")
    libdir = os.path.join(root, "paper_1911_08801_gb300")
    src = tmp_path / "abi.c"
    src.write_text('#include "assn.h"\n#include <stdio.h>\n#include <string.h>\n'
                   'int main(void) {\n'
                   '  if (assn_abi_version() != ASSN_ABI_VERSION) return 1;\n'
                   '  if (strcmp(assn_status_string(ASSN_ERR_TIMEOUT), "ASSN_ERR_TIMEOUT")) return 2;\n'
                   '  size_t b = 0;\n'
                   '  if (assn_footprint_bytes(448, 448, 512, ASSN_BF16, &b) != ASSN_OK || b < 822083584u) return 3;\n'
                   '  if (assn_create(NULL, 1, 1, 0, 1, 0, 1, ASSN_BF16, NULL) != ASSN_ERR_ARG) return 4;\n'
                   '  size_t t = 0, x = 0;  /* TF32 words hold as many bytes as the BF16 hi + lo parts */\n'
                   '  if (assn_footprint_bytes(448, 448, 512, ASSN_TF32, &t) != ASSN_OK ||\n'
                   '      assn_footprint_bytes(448, 448, 512, ASSN_BF16X3, &x) != ASSN_OK || t != x || t < b) return 5;\n'
                   '  if (assn_footprint_bytes(448, 448, 512, ASSN_BF16X2, &t) != ASSN_OK || t != x) return 6;\n'
                   '  if (assn_footprint_bytes(448, 448, 512, ASSN_BF16X2 + 1, &t) != ASSN_ERR_ARG) return 7;\n'
                   '  puts("ok");\n  return 0;\n}\n')
    exe = tmp_path / "abi"
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", f"-I{inc}", str(src), f"-L{libdir}",
                        "-lassn", f"-Wl,-rpath,{libdir}", "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.strip() == "ok", (r.returncode, r.stdout, r.stderr)


def test_binding_constants_match_header(lib):
    """Every enumerator of include/assn.h that the ctypes binding names has the header's value (the
    precisions, statuses, schemes, kernel kinds and normalisations are passed as plain ints)."""
    from paper_1911_08801_gb300 import _lib

    text = open(HEADER).read()
    header = {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(ASSN_[A-Z0-9_]+)\s*=\s*(-?\d+)", text)}
    named = {k: v for k, v in vars(_lib).items() if k.startswith("ASSN_") and isinstance(v, int) and k in header}
    for k in ("ASSN_FP64", "ASSN_FP32", "ASSN_BF16", "ASSN_BF16X3", "ASSN_TF32", "ASSN_BF16X2", "ASSN_ERR_UNSUPPORTED",
              "ASSN_ERR_CANCELLED", "ASSN_SCHEME_HEUN_MINMOD", "ASSN_KERNEL_EXP", "ASSN_NORM_ROW"):
        assert k in named, k
    assert {k: header[k] for k in named} == named
    assert set(_lib.PRECISIONS.values()) == {header[k] for k in ("ASSN_FP64", "ASSN_FP32", "ASSN_BF16", "ASSN_BF16X3",
                                                                  "ASSN_TF32", "ASSN_BF16X2")}
