"""CPU checks of the boundary: libpf.so builds, loads, exports every entry
point include/pf.h declares, and the Python structs match the C layout
(compiled with gcc from the header).  No compute call is made."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pf.h")


@pytest.fixture(scope="module")
def lib_path():
    from paper_1904_10585_gb300 import build
    return build.build()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pf_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("pf_create", "pf_destroy", "pf_filter", "pf_rayleigh_ritz", "pf_prox_step",
                     "pf_solve"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (pf_[a-z_]+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    lib = ctypes.CDLL(lib_path)
    for n in declared_functions():
        assert hasattr(lib, n)


def test_binding_exports_match_header(lib_path):
    import paper_1904_10585_gb300 as pkg
    assert set(pkg.EXPORTED) == set(declared_functions())
    for n in pkg.EXPORTED:
        assert callable(getattr(pkg, n))


def test_struct_layouts_match_c(lib_path):
    import paper_1904_10585_gb300._binding as B
    structs = {"pf_options": B.pf_options, "pf_operator": B.pf_operator,
               "pf_problem": B.pf_problem, "pf_iter_info": B.pf_iter_info,
               "pf_result": B.pf_result}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pf.h"', 'int main(void){']
    for name, cls in structs.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    lines.append("return 0;}")
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "l.c")
        exe = os.path.join(d, "l")
        open(src, "w").write("\n".join(lines))
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    got = dict(line.rsplit(" ", 1) for line in out.strip().splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert int(got[f"{name}.{f}"]) == getattr(cls, f).offset, f"{name}.{f}"


def test_status_strings_need_no_gpu(lib_path):
    import paper_1904_10585_gb300 as pkg
    assert pkg.pf_status_string(pkg.PF_OK) == "ok"
    assert pkg.pf_status_string(pkg.PF_ERR_INVALID_ARG) == "invalid argument"
    # argument validation happens before any CUDA call
    assert pkg.raw_call("pf_create", None, 10, None, None) == pkg.PF_ERR_INVALID_ARG
    assert pkg.raw_call("pf_destroy", None) == pkg.PF_ERR_INVALID_ARG


def test_enum_values_match_header():
    """Every PF_* enumerator of the header has the same value in the binding."""
    import paper_1904_10585_gb300._binding as B
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    found = 0
    for body in re.findall(r"typedef enum\s*\{(.*?)\}", text, flags=re.S):
        value = -1
        for item in body.split(","):
            item = item.strip()
            if not item:
                continue
            m = re.match(r"(PF_\w+)\s*(?:=\s*(-?\d+))?", item)
            value = int(m.group(2)) if m.group(2) is not None else value + 1
            assert getattr(B, m.group(1)) == value, m.group(1)
            found += 1
    assert found >= 19
