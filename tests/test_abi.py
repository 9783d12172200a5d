"""The C ABI library builds for sm_103a, loads, and exports every symbol
include/dd.h declares (no GPU needed: no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"^[A-Za-z_][\w \*]*?\b(dd_\w+)\s*\(", src, flags=re.M))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2209_13168_gb300 import _build
    path = _build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for n in ("dd_create", "dd_destroy", "dd_contrast", "dd_bound", "dd_solve", "dd_strerror"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for n in sorted(declared_symbols()):
        assert hasattr(lib, n), n


def test_binding_covers_every_declared_symbol():
    import paper_2209_13168_gb300 as dd
    assert declared_symbols() <= set(dd.SIGNATURES)


def test_strerror_without_gpu(lib):
    import paper_2209_13168_gb300 as dd
    dd.load()
    assert dd.dd_strerror(0) == "ok"
    assert "queue" in dd.dd_strerror(dd.DD_ERR_QUEUE_OVERFLOW)


def test_struct_layouts_match_header(tmp_path):
    # Compile a probe against include/dd.h and compare sizes and offsets with
    # the ctypes mirrors the binding passes across the boundary.
    import subprocess
    import paper_2209_13168_gb300 as dd
    probe = tmp_path / "probe.c"
    fields = {"dd_events": [f for f, _ in dd.dd_events._fields_], "dd_result": [f for f, _ in dd.dd_result._fields_],
              "dd_config": [f for f, _ in dd.dd_config._fields_], "dd_node_rec": [f for f, _ in dd.dd_node_rec._fields_],
              "dd_stats": [f for f, _ in dd.dd_stats._fields_],
              "dd_window_params": [f for f, _ in dd.dd_window_params._fields_],
              "dd_i128": ["lo", "hi"]}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "dd.h"', "int main(void) {"]
    for s, fs in fields.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (s, s))
        for f in fs:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (s, f, s, f))
    lines.append("return 0; }")
    probe.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(probe), "-o", str(exe)])
    got = dict(l.split() for l in subprocess.check_output([str(exe)], text=True).splitlines())
    for s, fs in fields.items():
        cls = getattr(dd, s)
        assert int(got[s]) == ctypes.sizeof(cls), s
        for f in fs:
            assert int(got["%s.%s" % (s, f)]) == getattr(cls, f).offset, (s, f)


def test_create_rejects_bad_geometry(lib):
    import paper_2209_13168_gb300 as dd
    dd.load()
    for args in ((0, 10, 0.0, 0.0), (10, 5000, 5.0, 5.0), (10, 10, 11.0, 5.0), (10, 10, float("nan"), 5.0)):
        with pytest.raises(dd.DDError) as e:
            dd.dd_create(*args)
        assert e.value.status == dd.DD_ERR_ARG


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2209_13168_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in src.lower().replace("oracle_", ""), f
