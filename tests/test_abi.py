"""CPU checks of the boundary: the library builds for sm_103a, loads, and exports
every entry point include/pic.h declares; the ctypes structs match the C layout.
No compute calls (no GPU here)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "pic.h")) as f:
        src = f.read()
    return sorted(set(re.findall(r"PIC_API\s+[\w\s\*]*?\b(pic_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1308_2590_gb300 import build
    return build.build()


def test_every_declared_symbol_is_exported(libpath):
    names = _declared()
    assert "pic_init" in names and "pic_step" in names and "pic_last_error" in names
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r" T (pic_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    lib = ctypes.CDLL(libpath)
    for n in names:
        assert hasattr(lib, n)


def test_binding_names_match_header(libpath):
    from paper_1308_2590_gb300 import pic
    assert sorted(pic.EXPORTED) == sorted(n for n in _declared())


def test_struct_layout_matches_c(tmp_path):
    from paper_1308_2590_gb300 import pic
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "pic.h"\n'
                   'int main(){printf("%zu %zu %zu %zu %zu\\n", sizeof(pic_config), sizeof(pic_diag),'
                   ' offsetof(pic_config, cuda_stream), offsetof(pic_config, capacity), offsetof(pic_diag, flags));'
                   'return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert vals == [ctypes.sizeof(pic.PicConfig), ctypes.sizeof(pic.PicDiag), pic.PicConfig.cuda_stream.offset,
                    pic.PicConfig.capacity.offset, pic.PicDiag.flags.offset]


def test_no_cpu_fallback_in_product_path():
    """The product package never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_1308_2590_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h")):
                with open(os.path.join(dirpath, fn)) as f:
                    txt = f.read()
                assert not re.search(r"^\s*(import|from)\s+oracle", txt, re.M), fn


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    from paper_1308_2590_gb300 import pic
    monkeypatch.setattr(pic, "_lib", None)
    with pytest.raises(pic.PicError):
        pic.lib(str(tmp_path / "nope.so"))
