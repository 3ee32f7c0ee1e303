"""The C-ABI library builds, loads without a GPU and exports every declared symbol."""
import ctypes
import os
import re

import pytest

from paper_1503_04500_gb300 import build_ext, rsai

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build_ext.build()
    return rsai.load()


def _declared_functions():
    with open(os.path.join(ROOT, "include", "rsai.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rsai_[A-Za-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert len(names) >= 16
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(rsai.EXPORTS) == names


def test_abi_version_and_status_strings(lib):
    assert lib.rsai_abi_version() == 2
    for code in range(0, 14):
        s = rsai.status_string(code)
        assert s and s != "unknown status"
    assert rsai.status_string(999) == "unknown status"


def test_params_default_and_check(lib):
    p = rsai.default_params()
    assert (p.c, p.l_max, p.eps, p.drop_mode, p.tol, p.precision, p.tie_band) == (3, 10, 0.3, 2, 1e-3, 0, 1e-12)
    assert lib.rsai_params_check(ctypes.byref(p)) == 0
    bad = [dict(c=0), dict(c=33), dict(l_max=-1), dict(eps=0.0), dict(eps=float("nan")), dict(drop_mode=3),
           dict(tol=-1.0), dict(precision=2), dict(tie_band=-1e-3), dict(tie_band=1.0), dict(flags=1), dict(flags=8)]
    for b in bad:
        q = rsai.default_params()
        for k, v in b.items():
            setattr(q, k, v)
        assert lib.rsai_params_check(ctypes.byref(q)) == 1, b
    assert lib.rsai_params_check(None) == 1
    ok = rsai.default_params(init="A")
    assert ok.flags == rsai.FLAG_INIT_PATTERN_A and lib.rsai_params_check(ctypes.byref(ok)) == 0
    ok = rsai.default_params(init="A", select="spai")
    assert ok.flags == rsai.FLAG_INIT_PATTERN_A | rsai.FLAG_SELECT_SPAI and lib.rsai_params_check(ctypes.byref(ok)) == 0


def test_null_arguments_rejected_without_device(lib):
    """Argument checks come before any device work."""
    out = ctypes.c_void_p(0)
    p = rsai.default_params()
    assert lib.rsai_build(None, None, ctypes.byref(p), None, ctypes.byref(out)) == 1
    assert out.value is None
    csr = rsai.CSR(4, 4, None, None, None)
    csc = rsai.CSC(4, 4, None, None, None)
    assert lib.rsai_build(ctypes.byref(csr), ctypes.byref(csc), ctypes.byref(p), None, ctypes.byref(out)) == 1
    assert lib.rsai_apply(None, None, None, None) == 1
    assert lib.rsai_get_stats(None, None, None) == 1
    v = ctypes.c_double(0.0)
    assert lib.rsai_peak_fma(0, None, None) == 1
    lib.rsai_handle_free(None)
    del v


@pytest.mark.skipif(os.environ.get("CUDA_VISIBLE_DEVICES", None) not in (None, ""), reason="device may exist")
def test_no_device_status(lib):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is visible")
    v = ctypes.c_double(0.0)
    assert lib.rsai_peak_fma(0, None, ctypes.byref(v)) == 12


def test_set_allocator_arguments(lib):
    """Both callbacks or neither; installing and removing needs no device."""
    seen = []
    alloc = rsai.ALLOC_FN(lambda nbytes, stream, ctx: seen.append(nbytes) or None)
    free = rsai.FREE_FN(lambda ptr, nbytes, stream, ctx: None)
    assert lib.rsai_set_allocator(alloc, rsai.FREE_FN(), None) == 1
    assert lib.rsai_set_allocator(rsai.ALLOC_FN(), free, None) == 1
    assert lib.rsai_set_allocator(alloc, free, None) == 0
    assert lib.rsai_set_allocator(rsai.ALLOC_FN(), rsai.FREE_FN(), None) == 0
    assert seen == []  # nothing allocated by installing


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of rsai_csr, rsai_csc, rsai_params, rsai_stats and
    rsai_tuning have the header's sizes and field offsets (gcc compiles the C
    header and prints them)."""
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"rsai_csr": rsai.CSR, "rsai_csc": rsai.CSC, "rsai_params": rsai.Params, "rsai_stats": rsai.Stats,
               "rsai_tuning": rsai.Tuning}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "rsai.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'    printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'    printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            name, field, value = line.split()
            got[(name, field)] = int(value)
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)


def test_product_path_never_reaches_the_oracle():
    """Only tests, the smoke check and the benchmark's CPU legs may use the
    oracle: no module of the package imports it, and the CUDA sources share no
    file with it."""
    pkg = os.path.join(ROOT, "paper_1503_04500_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import oracle|from oracle)", text, re.M), f
                assert "rsai_oracle" not in text, f
