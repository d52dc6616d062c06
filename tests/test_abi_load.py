"""The C-ABI library builds, loads without a GPU and exports every declared entry point."""
import ctypes
import os
import re

import pytest

from paper_1702_02207_gb300 import _build, cho

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(inc, f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?\w+\s*\*?\s*(cho_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    path = _build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("cho_create_system", "cho_integrate_batch", "cho_submit", "cho_poll", "cho_energy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in sorted(declared_functions()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    assert set(cho.EXPORTED) == declared_functions()
    for n in cho.EXPORTED:
        assert callable(getattr(cho, n))


def test_struct_layouts_match_the_c_compiler(tmp_path):
    """sizeof and offsetof of every public struct, from gcc, equal the ctypes mirrors."""
    structs = {
        "cho_config": cho.cho_config, "cho_system_desc": cho.cho_system_desc,
        "cho_batch_desc": cho.cho_batch_desc, "cho_request": cho.cho_request, "cho_result": cho.cho_result,
        "cho_tune_result": cho.cho_tune_result,
    }
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "cho.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{name}.{fname} %zu\\n", offsetof({name}, {fname}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    import subprocess

    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = dict(l.split() for l in out if l.strip())
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for fname, _ in cls._fields_:
            assert int(got[f"{name}.{fname}"]) == getattr(cls, fname).offset, f"{name}.{fname}"


def test_calls_without_gpu_fail_cleanly(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    cho.load()
    with pytest.raises(cho.ChoError) as ei:
        cho.cho_init(0)
    assert ei.value.status in (cho.CHO_ECUDA, cho.CHO_EINVAL)
    assert cho.cho_last_error() != ""
