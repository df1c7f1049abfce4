"""The C-ABI library builds, loads and exports every symbol include/lilac.h
declares; host-only argument checks return the documented status codes
(no call here touches a GPU)."""
import ctypes
import os
import re

import pytest

from paper_2001_07938_gb300 import build as lbuild
from paper_2001_07938_gb300 import lilac as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "lilac.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lilac_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    lbuild.build()
    return L.load()


def test_header_declares_the_binding_exports():
    assert _declared_functions() == sorted(L.EXPORTS)


def test_every_declared_symbol_is_exported(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_status_strings_and_version(lib):
    assert L.lilac_status_string(L.LILAC_OK) == "ok"
    assert "breakdown" in L.lilac_status_string(L.LILAC_ERR_BREAKDOWN).lower()
    assert L.lilac_status_string(999) == "unknown status"
    assert L.lilac_version() == 10000


def test_cg_opts_defaults(lib):
    o = L.lilac_cg_opts_default()
    assert o.max_iter == 1000 and o.rtol == 1e-10 and o.precision == 0
    assert o.inner_rtol == 1e-5 and o.use_graph == 1 and o.check_every == 32


def test_null_and_invalid_arguments_are_rejected_on_the_host(lib):
    assert lib.lilac_csr_destroy(None) == L.LILAC_OK
    info = L.lilac_csr_info_t()
    assert lib.lilac_csr_info(None, ctypes.byref(info)) == L.LILAC_ERR_INVALID_ARG
    assert lib.lilac_spmv(None, None, None, L.LILAC_MEM_DEVICE, None) == L.LILAC_ERR_INVALID_ARG
    assert lib.lilac_cg(None, None, None, 1, None, None, None) == L.LILAC_ERR_INVALID_ARG
    assert lib.lilac_pagerank(None, None, 1, 1, 0.85, None, 1, None) == L.LILAC_ERR_INVALID_ARG
    assert lib.lilac_csr_set_variant(None, 1, 0) == L.LILAC_ERR_INVALID_ARG
    h = ctypes.c_void_p()
    # negative rows / nnz >= 2^31 / bad dtype are refused before any CUDA call
    assert lib.lilac_csr_create(-1, -1, 0, None, None, None, 0, 0, 0, None,
                                ctypes.byref(h)) == L.LILAC_ERR_INVALID_ARG
    assert lib.lilac_csr_create(1, -1, 2 ** 31, None, None, None, 0, 0, 0, None,
                                ctypes.byref(h)) == L.LILAC_ERR_INVALID_ARG
    assert lib.lilac_csr_create(1, -1, 0, None, None, None, 7, 0, 0, None,
                                ctypes.byref(h)) == L.LILAC_ERR_INVALID_ARG
    assert not h.value
    assert "invalid" in L.lilac_last_error()


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    monkeypatch.setattr(L, "_LIB", None)
    monkeypatch.setattr(L, "library_path", lambda: str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="no CPU path"):
        L.load()


def test_struct_layouts_match_the_header(tmp_path):
    """Every struct the binding mirrors has the size and field offsets the C
    compiler gives the header's declaration (the binding is plain ctypes, so a
    field added on one side only would shift every later field)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    structs = [L.lilac_csr_info_t, L.lilac_cg_opts, L.lilac_cg_info, L.lilac_server_opts,
               L.lilac_request, L.lilac_completion, L.lilac_server_stats_t, L.lilac_host_stats_t]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "lilac.h"', "int main(void) {"]
    for st in structs:
        n = st.__name__
        lines.append(f'printf("{n} sizeof %zu\\n", sizeof({n}));')
        for f, _ in st._fields_:
            # a trailing underscore stands for a C field named like a Python keyword
            lines.append(f'printf("{n} {f} %zu\\n", offsetof({n}, {f.rstrip("_")}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    c_layout = {}
    for line in out.splitlines():
        n, f, v = line.split()
        c_layout[(n, f)] = int(v)
    for st in structs:
        n = st.__name__
        assert c_layout[(n, "sizeof")] == ctypes.sizeof(st), n
        for f, _ in st._fields_:
            assert c_layout[(n, f)] == getattr(st, f).offset, f"{n}.{f}"
