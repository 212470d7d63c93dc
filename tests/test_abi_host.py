"""The C ABI without a GPU: the library loads, exports every symbol include/rsd.h
declares, and rejects bad inputs on the host before any device work."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import synth
from oracle import fem, partition

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1210_6266_gb300 import build
    build.build()
    from paper_1210_6266_gb300 import _lib
    return _lib


def _declared():
    with open(os.path.join(ROOT, "include", "rsd.h")) as fh:
        src = fh.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rsd_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    so = lib.load()
    names = _declared()
    assert "rsd_setup" in names and "rsd_apply" in names and "rsd_solve" in names
    for name in names:
        assert hasattr(so, name), name
    assert sorted(lib.EXPORTS) == sorted(names)


def test_strerror_and_grid_sizes(lib):
    so = lib.load()
    for code in range(-7, 1):
        assert so.rsd_strerror(code)
    nd, nz = C.c_int64(), C.c_int64()
    assert so.rsd_grid_sizes(129, C.byref(nd), C.byref(nz)) == 0
    assert nd.value == 2_048_383 and nz.value == (3 * 127 - 2) ** 3
    assert so.rsd_grid_sizes(2, C.byref(nd), C.byref(nz)) == lib.RSD_ERR_ARG


def test_grid_nnz_matches_oracle(lib):
    so = lib.load()
    for n in (5, 9, 13):
        nd, nz = C.c_int64(), C.c_int64()
        so.rsd_grid_sizes(n, C.byref(nd), C.byref(nz))
        A = fem.assemble(n, np.ones((n - 1) ** 3))
        assert (nd.value, nz.value) == (A.shape[0], A.nnz)


def _host_setup(lib, A, owner, parent):
    so = lib.load()
    rowptr = np.ascontiguousarray(A.indptr.astype(np.int64))
    col = np.ascontiguousarray(A.indices.astype(np.int32))
    val = np.ascontiguousarray(A.data.astype(np.float64))
    own = np.ascontiguousarray(owner.astype(np.int32))
    par = np.ascontiguousarray(parent.astype(np.int32))
    csr = lib.rsd_csr(A.shape[0], A.nnz, rowptr.ctypes.data, col.ctypes.data, val.ctypes.data, lib.RSD_MEM_HOST)
    tree = lib.rsd_tree(len(par), par.ctypes.data)
    opt = lib.rsd_options(0, lib.RSD_PREC_FP64, lib.RSD_PREC_FP64, lib.RSD_PREC_FP64, 10, None, 0)
    out = C.c_void_p()
    return so.rsd_setup(C.byref(csr), own.ctypes.data, C.byref(tree), C.byref(opt), C.byref(out))


def test_partition_violation_rejected_on_host(lib):
    n = 9
    A = fem.assemble(n, np.ones((n - 1) ** 3)).tolil()
    owner = partition.octree_owner(n, 1, fem.interior_coords(n))
    parent = partition.octree_parent(1)
    i, j = int(np.nonzero(owner == 1)[0][0]), int(np.nonzero(owner == 8)[0][-1])
    A[i, j] = A[j, i] = -0.01
    assert _host_setup(lib, A.tocsr(), owner, parent) == lib.RSD_ERR_PARTITION


def test_bad_tree_and_owner_rejected_on_host(lib):
    n = 7
    A = fem.assemble(n, np.ones((n - 1) ** 3))
    owner = partition.octree_owner(n, 1, fem.interior_coords(n))
    parent = partition.octree_parent(1)
    bad_parent = parent.copy()
    bad_parent[3] = 5                       # parent id not smaller than the child id
    assert _host_setup(lib, A, owner, bad_parent) == lib.RSD_ERR_ARG
    root_parent = parent.copy()
    root_parent[0] = 0
    assert _host_setup(lib, A, owner, root_parent) == lib.RSD_ERR_ARG
    bad_owner = owner.copy()
    bad_owner[0] = 99
    assert _host_setup(lib, A, bad_owner, parent) == lib.RSD_ERR_ARG


def test_null_arguments(lib):
    so = lib.load()
    out = C.c_void_p()
    assert so.rsd_setup(None, None, None, None, C.byref(out)) == lib.RSD_ERR_ARG
    assert so.rsd_apply(None, None, None) == lib.RSD_ERR_ARG
    assert so.rsd_solve(None, None, None, 1e-8, None) == lib.RSD_ERR_ARG
    assert so.rsd_check(None) == lib.RSD_ERR_ARG
    so.rsd_destroy(None)


def test_tune_cache_reader_accepts_autotune_format_and_rejects_malformed(tmp_path):
    """rsd_tune_load parses the table rsd_autotune writes (host only, no GPU)."""
    from paper_1210_6266_gb300 import _lib
    import ctypes as C
    lib = _lib.load()
    good = tmp_path / "tune.json"
    good.write_text('{"device": "x", "sms": 152, "entries": [\n'
                    '  {"op": 0, "tiles": 1, "k": 512, "bn": 256, "split": 4, "us": 10.00, "us_rule": 12.00},\n'
                    '  {"op": 1, "tiles": 64, "k": 8192, "bn": 256, "split": 1, "us": 99.50, "us_rule": 99.50}\n'
                    ']}\n')
    n = C.c_int32()
    assert lib.rsd_tune_load(str(good).encode(), C.byref(n)) == 0 and n.value == 2
    for text in ('{"entries": [\n  {"op": 0, "tiles": 1, "k": 512, "bn": 64, "split": 1, "us": 1.0, "us_rule": 1.0}\n]}\n',
                 '{"entries": [\n]}\n',
                 '{"entries": [\n  {"op": 0, "tiles": 1}\n]}\n'):
        bad = tmp_path / "bad.json"
        bad.write_text(text)
        assert lib.rsd_tune_load(str(bad).encode(), C.byref(n)) == _lib.RSD_ERR_ARG
    assert lib.rsd_tune_load(str(tmp_path / "missing.json").encode(), C.byref(n)) == _lib.RSD_ERR_ARG


def test_binding_structs_match_the_header_layout(tmp_path):
    """Every structure the Python binding passes through the C ABI has the header's size
    and field offsets (compiled against include/rsd.h with the host compiler), and the
    profile's class list has the header's class count."""
    import shutil
    import subprocess
    from paper_1210_6266_gb300 import _lib
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    structs = [_lib.rsd_csr, _lib.rsd_tree, _lib.rsd_options, _lib.rsd_stats, _lib.rsd_info_t,
               _lib.rsd_profile_t, _lib.rsd_trace_rec]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "rsd.h"', "int main(void) {",
             '  printf("classes %d\\n", RSD_PROFILE_CLASSES);']
    for s in structs:
        n = s.__name__
        lines.append(f'  printf("{n} sizeof %zu\\n", sizeof({n}));')
        for f in s._fields_:
            lines.append(f'  printf("{n} {f[0]} %zu\\n", offsetof({n}, {f[0]}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], check=True, capture_output=True,
                                                        text=True).stdout.split("\n") if l)
    assert int(out["classes"]) == len(_lib.PROFILE_CLASSES)
    for s in structs:
        n = s.__name__
        assert int(out[f"{n} sizeof"]) == C.sizeof(s), n
        for f in s._fields_:
            assert int(out[f"{n} {f[0]}"]) == getattr(s, f[0]).offset, (n, f[0])
