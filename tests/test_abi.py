"""The C library builds for sm_103a, loads, and exports every entry point include/rt.h declares
(no GPU needed: nothing is called)."""
import ctypes
import os
import re

from paper_2302_12727_gb300 import EXPORTED, build_ext, load_library

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:rt_status|const char\*|void)\s+(rt_\w+)\s*\(", src, flags=re.M)
    return names


def test_library_exports_every_declared_symbol():
    build_ext.build()
    lib = load_library()
    names = declared_functions()
    assert len(names) >= 13
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(EXPORTED)


def test_library_is_sm103a_only():
    flags = " ".join(build_ext.NVCC_FLAGS)
    assert "arch=compute_103a,code=sm_103a" in flags


def test_config_struct_layout_matches_header(tmp_path):
    """ctypes mirrors of rt_config / rt_diag have the C compiler's size and field offsets."""
    import subprocess
    from paper_2302_12727_gb300 import rt_config, rt_diag, rt_tuning
    src = tmp_path / "layout.c"
    fields_c = [f for f, _ in rt_config._fields_]
    fields_d = [f for f, _ in rt_diag._fields_]
    body = ['#include <stdio.h>', '#include <stddef.h>', '#include "rt.h"', "int main(void) {",
            'printf("%zu %zu %zu\\n", sizeof(rt_config), sizeof(rt_diag), sizeof(rt_tuning));']
    for f in fields_c:
        body.append(f'printf("%zu\\n", offsetof(rt_config, {f}));')
    for f in fields_d:
        body.append(f'printf("%zu\\n", offsetof(rt_diag, {f}));')
    body.append("return 0; }")
    src.write_text("\n".join(body))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = subprocess.check_output([str(exe)]).decode().split()
    vals = [int(v) for v in out]
    assert vals[0] == ctypes.sizeof(rt_config) and vals[1] == ctypes.sizeof(rt_diag)
    assert vals[2] == ctypes.sizeof(rt_tuning)
    offs = vals[3:]
    want = [getattr(rt_config, f).offset for f in fields_c] + [getattr(rt_diag, f).offset for f in fields_d]
    assert offs == want
