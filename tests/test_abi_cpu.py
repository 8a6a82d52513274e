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


def test_struct_layouts_match_the_binding(tmp_path):
    """Every option / array struct of include/kscann.h has the size and field
    offsets of its ctypes mirror in the binding (a field added on one side
    only fails here: a missing name does not compile, a missing trailing
    field changes the size)."""
    import shutil
    import subprocess
    from paper_2511_03298_gb300 import ksc
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"ksc_build_opts": ksc.BuildOpts, "ksc_index_arrays": ksc.IndexArrays,
               "ksc_adaptive_params": ksc.AdaptiveParams, "ksc_train_opts": ksc.TrainOpts,
               "ksc_search_opts": ksc.SearchOpts}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "kscann.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append('  printf("%s %%zu\\n", sizeof(%s));' % (name, name))
        for fname, _ in cls._fields_:
            lines.append('  printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (name, fname, name, fname))
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                 check=True).stdout.splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == C.sizeof(cls), name
        for fname, _ in cls._fields_:
            assert int(got["%s.%s" % (name, fname)]) == getattr(cls, fname).offset, (name, fname)
