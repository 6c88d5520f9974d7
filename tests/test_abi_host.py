"""Host-side checks of the C ABI (no GPU work): the library builds, loads and
exports every entry point that include/mwu.h declares."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mwu.h")


def header_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(mwu_[a-z_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_2307_03307_gb300 import _build
    path = _build.build()
    return path


def test_header_declares_the_boundary():
    names = header_functions()
    for required in ["mwu_create", "mwu_iterate", "mwu_solve", "mwu_destroy", "mwu_set_target",
                     "mwu_potential", "mwu_create_batch"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (mwu_[a-z_]+)\b", out))
    missing = [f for f in header_functions() if f not in exported]
    assert not missing, missing
    h = ctypes.CDLL(lib)
    for f in header_functions():
        assert hasattr(h, f)


def test_binding_covers_the_header(lib):
    from paper_2307_03307_gb300 import mwu
    assert sorted(mwu.exported_symbols()) == header_functions()


def test_default_options_host_only(lib):
    from paper_2307_03307_gb300 import mwu
    o = mwu.mwu_default_options()
    assert o.eps == pytest.approx(0.1) and o.max_iter == 5000 and o.K == 8
    assert o.eta_factor == pytest.approx(10.0) and o.double_single == 1
    o2 = mwu.mwu_default_options(eps=0.05, K=4)
    assert o2.eps == pytest.approx(0.05) and o2.K == 4
    # the reproducible defaults: every row kept, automatic tiles, gathers (no atomic sums)
    assert (o.drop_covered, o.spmv_tiles, o.h_scatter, o.dv_scatter) == (0, 0, 0, 0)


def test_struct_sizes_match_header(lib):
    """Compile a tiny C program against mwu.h and compare struct sizes with the ctypes mirrors."""
    from paper_2307_03307_gb300 import mwu
    import tempfile
    src = r'''
#include <stdio.h>
#include "mwu.h"
int main(void){printf("%zu %zu %zu %zu %zu\n", sizeof(mwu_matrix), sizeof(mwu_options),
 sizeof(mwu_iter_stats), sizeof(mwu_result), sizeof(mwu_scalars));return 0;}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "s.c")
        exe = os.path.join(d, "s")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        sizes = [int(v) for v in subprocess.run([exe], capture_output=True, text=True).stdout.split()]
    mine = [ctypes.sizeof(t) for t in (mwu.mwu_matrix, mwu.mwu_options, mwu.mwu_iter_stats,
                                       mwu.mwu_result, mwu.mwu_scalars)]
    assert sizes == mine


def test_missing_library_fails_loudly(tmp_path):
    from paper_2307_03307_gb300 import mwu
    saved = mwu._lib
    try:
        mwu._lib = None
        with pytest.raises(ImportError):
            mwu.load(str(tmp_path / "nope.so"))
    finally:
        mwu._lib = saved
