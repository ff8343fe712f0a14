"""The C-ABI library builds, loads and exports every entry point that
include/pdgrass.h declares (no compute calls: runs without a GPU)."""
from __future__ import annotations

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pdgrass.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[\w\*]+\s+\**(\w+)\s*\(", text, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while")))


@pytest.fixture(scope="module")
def lib():
    from paper_2508_20403_gb300 import build

    try:
        path = build.build()
    except Exception as e:  # nvcc missing on this machine
        pytest.skip(f"cannot build the CUDA library here: {e}")
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("sparsify_init", "recover_offtree", "sparsifier_free", "sparsify_batch_init",
                     "recover_offtree_batch", "pdg_status_string", "pdg_default_options"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_names_match_header():
    from paper_2508_20403_gb300 import binding

    assert set(binding.EXPORTS) <= set(declared_functions())


def test_host_only_calls(lib):
    lib.pdg_status_string.restype = ctypes.c_char_p
    assert lib.pdg_status_string(0) == b"ok"
    assert b"tree" in lib.pdg_status_string(-3)
    from paper_2508_20403_gb300 import binding

    o = binding.default_options()
    assert o.warp_tier_max == 32 and o.k_override == -1 and o.candidate_factor >= 1.0
    # NULL handle arguments are rejected without touching a device
    lib.sparsifier_free(None)
    assert lib.recover_offtree(None, ctypes.c_double(0.1), 2, None, 0, None, None, 0) == binding.PDG_E_INVALID_ARG


def test_library_is_required_not_replaced(tmp_path):
    """The binding raises when the compiled library is missing: no fallback."""
    from paper_2508_20403_gb300 import binding

    with pytest.raises(ImportError):
        binding.load(str(tmp_path / "missing.so"))


def test_options_layout_matches_header(tmp_path):
    """The ctypes mirror of pdg_options has the C struct's size and field offsets (compiled from the header)."""
    import shutil
    import subprocess

    from paper_2508_20403_gb300 import binding

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    fields = [f for f, _ in binding.Options._fields_]
    src = tmp_path / "layout.c"
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pdgrass.h"', "int main(void) {",
             '  printf("size %zu\\n", sizeof(pdg_options));']
    lines += [f'  printf("{f} %zu\\n", offsetof(pdg_options, {f}));' for f in fields]
    lines += ["  return 0;", "}"]
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.check_call([cc, "-I", inc, str(src), "-o", str(exe)])
    out = dict(l.split() for l in subprocess.check_output([str(exe)], text=True).splitlines())
    assert int(out["size"]) == ctypes.sizeof(binding.Options)
    for f in fields:
        assert int(out[f]) == getattr(binding.Options, f).offset, f


def test_new_entry_points_reject_bad_arguments_without_a_device(lib):
    """pdg_spanning_tree and pdg_pcg_quality check their arguments before any CUDA call."""
    from paper_2508_20403_gb300 import binding

    L = binding.load()
    rp = (ctypes.c_int64 * 3)(0, 1, 2)
    col = (ctypes.c_int32 * 2)(1, 0)
    w = (ctypes.c_double * 2)(1.0, 1.0)
    par = (ctypes.c_int32 * 2)(-1, 0)
    out = (ctypes.c_int32 * 2)()
    E = binding.PDG_E_INVALID_ARG
    assert L.pdg_spanning_tree(0, rp, col, w, 0, 0, out, 0, None) == E  # n < 1
    assert L.pdg_spanning_tree(2, rp, col, w, 0, 7, out, 0, None) == E  # unknown tree kind
    assert L.pdg_spanning_tree(2, None, col, w, 0, 0, out, 0, None) == E
    assert L.pdg_spanning_tree(2, rp, col, w, 5, 0, out, 0, None) == E  # memory kind
    b = (ctypes.c_double * 2)(1.0, -1.0)
    ids = (ctypes.c_int32 * 1)(0)
    it = ctypes.c_int32()
    rel = ctypes.c_double()
    args = lambda **kw: dict(dict(n=2, rp=rp, col=col, w=w, par=par, ids=ids, k=1, b=b, tol=1e-3, mi=10, kind=0), **kw)
    call = lambda a: L.pdg_pcg_quality(a["n"], a["rp"], a["col"], a["w"], a["par"], a["ids"], a["k"], a["b"],
                                       a["tol"], a["mi"], a["kind"], ctypes.byref(it), ctypes.byref(rel), None)
    assert call(args(tol=0.0)) == E
    assert call(args(mi=0)) == E
    assert call(args(k=8193)) == E  # dense capacitance bound
    assert call(args(k=-1)) == E
    assert call(args(n=1)) == E
    assert call(args(b=None)) == E
