"""The surrogate's C ABI without a GPU: libcno.so builds for sm_103a, loads,
exports every symbol include/cno.h declares (and the binding binds them all),
and rejects bad network shapes before touching a device."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_2511_09422_gb300 import _build, cno

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cno.h")


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return cno.load()


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cno_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 15
    out = subprocess.run(["nm", "-D", "--defined-only", _build.CNO_LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (cno_[a-z0-9_]+)\b", out))
    for n in names:
        assert n in exported, n
        assert hasattr(lib, n)
    assert set(cno.EXPORTS) == set(names)


@pytest.mark.parametrize("cin,widths,cout,nf", [
    (64, (64, 128, 256, 128), 64, 7),   # the level-3 width must equal the level-2 width
    (64, (32, 64, 128, 128), 64, 7),    # widths must be multiples of 64
    (64, (64, 128, 512, 512), 64, 7),   # at most 256
    (48, (64, 128, 256, 256), 64, 7),   # cin a multiple of 64
    (64, (64, 128, 256, 256), 64, 9),   # nf at most 8
    (64, (64, 128, 256, 256), 64, 0),
])
def test_bad_network_shapes_rejected_without_a_device(lib, cin, widths, cout, nf):
    h = C.c_void_p()
    arr = (C.c_int * 4)(*widths)
    assert lib.cno_create(cin, arr, cout, nf, C.byref(h)) == 1  # CNO_ERR_INVALID_ARG
    assert h.value is None
    assert lib.cno_error_string()


def test_null_arguments(lib):
    assert lib.cno_create(64, None, 64, 7, None) == 1
    assert lib.cno_destroy(None) == 0
    out = (C.c_double * 8)()
    assert lib.cno_field_checks(None, None, None, None, 4, 4, out, None) == 1
    assert lib.cno_pack_fields(None, 7, 4, 4, None, None, None, 64, None) == 1
