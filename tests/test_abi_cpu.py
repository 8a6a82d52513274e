"""The C-ABI library builds, loads and exports every declared symbol (no GPU
needed); argument checks that fail before any device work."""
import ctypes as C
import os
import re

import numpy as np

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


def _index_file(path, n=64, d=8, nlist=4, M=4, flags=0, codes=None, assign=None, magic=b"KSCIDX01", cut=0):
    """A file in the layout ksc_index_save writes: a 64-byte little-endian
    header (magic, n, d, nlist, M, metric, spherical, flags, full dimensions,
    size of ksc_adaptive_params, 4 reserved) and the interchange arrays."""
    import struct
    from paper_2511_03298_gb300 import ksc
    rng = np.random.default_rng(1)
    hdr = struct.pack("<8sq8i4i", magic, n, d, nlist, M, 0, 0, flags, 0, C.sizeof(ksc.AdaptiveParams), 0, 0, 0, 0)
    assert len(hdr) == 64
    codes = rng.integers(0, 16, (n, M)).astype(np.uint8) if codes is None else codes
    assign = (np.arange(n) % nlist).astype(np.int32) if assign is None else assign
    body = b"".join(a.tobytes() for a in (
        rng.normal(size=(n, d)).astype(np.float32), rng.normal(size=(nlist, d)).astype(np.float32),
        rng.normal(size=(nlist, d)).astype(np.float32), rng.normal(size=(M, 16, d // M)).astype(np.float32),
        codes, assign))
    data = hdr + body
    open(path, "wb").write(data[:len(data) - cut])
    return path


def test_index_load_rejects_bad_files_before_device_work(lib, tmp_path):
    """ksc_index_load checks the whole file on the host: every case below
    returns KSC_EINVAL without touching the device."""
    h = C.c_void_p()
    load = lambda p: lib.ksc_index_load(os.fsencode(str(p)), None, C.byref(h))
    assert load(tmp_path / "missing.ksc") == -1 and b"cannot open" in lib.ksc_last_error()
    assert load(_index_file(tmp_path / "magic.ksc", magic=b"NOTANIDX")) == -1
    assert b"not an index file" in lib.ksc_last_error()
    assert load(_index_file(tmp_path / "short.ksc", cut=4)) == -1 and b"bytes" in lib.ksc_last_error()
    bad_codes = np.zeros((64, 4), np.uint8)
    bad_codes[7, 2] = 16
    assert load(_index_file(tmp_path / "codes.ksc", codes=bad_codes)) == -1 and b"code" in lib.ksc_last_error()
    bad_assign = (np.arange(64) % 4).astype(np.int32)
    bad_assign[9] = 4
    assert load(_index_file(tmp_path / "lists.ksc", assign=bad_assign)) == -1 and b"list" in lib.ksc_last_error()
    assert load(_index_file(tmp_path / "flags.ksc", flags=64)) == -1 and b"sections" in lib.ksc_last_error()
    assert lib.ksc_index_load(None, None, C.byref(h)) == -1
    assert lib.ksc_index_save(None, b"x") == -1
    assert h.value is None


def test_index_import_rejects_foreign_neighbours_before_device_work(lib):
    """ksc_index_import checks on the host that a graph's neighbours and a
    list's entry lie in that list (the device search follows them as
    positions inside the list), and that codes and assignments are in range:
    KSC_EINVAL before any device work."""
    from paper_2511_03298_gb300 import ksc
    rng = np.random.default_rng(2)
    n, d, nlist, M = 64, 8, 4, 4
    X = rng.normal(size=(n, d)).astype(np.float32)
    cr = rng.normal(size=(nlist, d)).astype(np.float32)
    cb = rng.normal(size=(M, 16, d // M)).astype(np.float32)
    assign = (np.arange(n) % nlist).astype(np.int32)
    # neighbours: the other members of the row's own list, -1 padded
    graph = -np.ones((n, 32), np.int32)
    for u in range(n):
        mem = [v for v in range(n) if assign[v] == assign[u] and v != u]
        graph[u, :len(mem)] = mem
    entry = np.arange(nlist, dtype=np.int32)  # row p is in list p

    def attempt(codes, assign, graph, entry):
        a = ksc.IndexArrays(n=n, d=d, nlist=nlist, M=M, metric=0, spherical=0)
        keep = [X, cr, cr, cb, codes, assign, graph, entry]
        for name, arr in zip(("X", "c_rank", "c_mean", "codebook", "codes", "assign", "graph", "entry"), keep):
            setattr(a, name, None if arr is None else arr.ctypes.data)
        h = C.c_void_p()
        rc = lib.ksc_index_import(C.byref(a), None, C.byref(h))
        assert h.value is None
        return rc, lib.ksc_last_error()

    codes = rng.integers(0, 16, (n, M)).astype(np.uint8)
    g = graph.copy()
    g[5, 3] = 6  # row 6 is in list 2, row 5 in list 1
    rc, msg = attempt(codes, assign, g, entry)
    assert rc == -1 and b"another list" in msg
    e = entry.copy()
    e[2] = 7  # row 7 is in list 3
    rc, msg = attempt(codes, assign, graph, e)
    assert rc == -1 and b"not in the list" in msg
    g = graph.copy()
    g[0, 0] = n
    rc, msg = attempt(codes, assign, g, entry)
    assert rc == -1 and b"out of range" in msg
    c = codes.copy()
    c[3, 1] = 16
    rc, msg = attempt(c, assign, graph, entry)
    assert rc == -1 and b"code" in msg
    a2 = assign.copy()
    a2[10] = nlist
    rc, msg = attempt(codes, a2, None, None)
    assert rc == -1 and b"assignment" in msg
