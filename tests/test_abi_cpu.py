"""The C-ABI library builds, loads and exports every declared symbol (no GPU
needed); argument checks that fail before any device work."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2511_03298_gb300 import ksc
    return ksc.lib()


def declared_symbols():
    syms = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            syms |= set(re.findall(r"\b(ksc_[a-z0-9_]+)\s*\(", txt))
    return sorted(syms)


def test_every_declared_symbol_is_exported(lib):
    syms = declared_symbols()
    assert len(syms) >= 10
    missing = [s for s in syms if not hasattr(lib, s)]
    assert not missing, missing


def test_version_and_error_strings(lib):
    from paper_2511_03298_gb300 import ksc
    assert "sm_103a" in ksc.version()
    assert isinstance(lib.ksc_last_error(), bytes)


def test_argument_errors_before_device_work(lib):
    from paper_2511_03298_gb300 import ksc
    h = C.c_void_p()
    # nbits != 4 is unsupported
    rc = lib.ksc_build_index(C.c_void_p(16), 100, 8, 4, 4, 8, 0, None, None, C.byref(h))
    assert rc == -4 and b"nbits" in lib.ksc_last_error()
    # null pointers
    assert lib.ksc_build_index(None, 100, 8, 4, 4, 4, 0, None, None, C.byref(h)) == -1
    assert lib.ksc_search(None, None, 1, 10, 8, 100, None, None, None, None) == -1
    assert b"null index" in lib.ksc_last_error()
    assert lib.ksc_index_import(None, None, C.byref(h)) == -1
    # M must divide d
    rc = lib.ksc_build_index(C.c_void_p(16), 100, 10, 4, 3, 4, 0, None, None, C.byref(h))
    assert rc == -1 and b"M" in lib.ksc_last_error()
    with pytest.raises(ksc.KscError):
        ksc._check(-1)
