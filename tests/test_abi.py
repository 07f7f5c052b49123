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
                   'int main(){printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(pic_config), sizeof(pic_diag),'
                   ' offsetof(pic_config, cuda_stream), offsetof(pic_config, capacity), offsetof(pic_diag, flags),'
                   ' offsetof(pic_config, shape));'
                   'return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert vals == [ctypes.sizeof(pic.PicConfig), ctypes.sizeof(pic.PicDiag), pic.PicConfig.cuda_stream.offset,
                    pic.PicConfig.capacity.offset, pic.PicDiag.flags.offset, pic.PicConfig.shape.offset]


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


def test_server_struct_layout_matches_c(tmp_path):
    from paper_1308_2590_gb300 import pic
    src = tmp_path / "sz2.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "pic.h"\n'
                   'int main(){printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(pic_server_config), sizeof(pic_species_data),'
                   ' sizeof(pic_request_status), offsetof(pic_request_status, t_submit),'
                   ' offsetof(pic_request_status, device_bytes), offsetof(pic_diag, cn_refinements));'
                   'return 0;}\n')
    exe = tmp_path / "sz2"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert vals == [ctypes.sizeof(pic.PicServerConfig), ctypes.sizeof(pic.PicSpeciesData),
                    ctypes.sizeof(pic.PicRequestStatus), pic.PicRequestStatus.t_submit.offset,
                    pic.PicRequestStatus.device_bytes.offset, pic.PicDiag.cn_refinements.offset]


def test_estimate_bytes_needs_no_gpu_and_scales(libpath):
    """Admission estimate: computed on the host, grows with particles, precision,
    the deterministic deposit and the CN scratch; invalid configurations fail."""
    from paper_1308_2590_gb300 import pic, workloads as W
    cfg = W.config(2)
    n = cfg.n_particles // 2
    b0 = pic.estimate_bytes(cfg, [0, 0])
    b1 = pic.estimate_bytes(cfg, [n, n])
    b2 = pic.estimate_bytes(cfg, [2 * n, 2 * n])
    assert 0 < b0 < b1 < b2
    # particle part: three buffer sets of (4 + 6*8) bytes per slot, >= 1.5 slots per particle, plus sort scratch
    assert (b2 - b1) > 2 * n * (3 * 52 * 1.5)
    f32 = cfg.scaled(precision=W.PREC_FP32)
    assert pic.estimate_bytes(f32, [n, n]) < b1
    det = cfg.scaled(deposit=W.DEPOSIT_DETERMINISTIC)
    nnode, ncell = (cfg.nx + 1) * cfg.ny, cfg.nx * cfg.ny
    # the exact deposit adds its fixed-point sums; the L2-reduction form holds the push's cell sums
    assert pic.estimate_bytes(det, [n, n]) - b1 == 13 * nnode * 8 - 13 * 4 * ncell * 8
    cn = W.config(1)
    lit = cn.scaled(field_mode=W.FIELD_LITERAL)
    assert pic.estimate_bytes(cn, [1000, 1000]) > pic.estimate_bytes(lit, [1000, 1000])
    with pytest.raises(pic.PicError):
        pic.estimate_bytes(cfg.scaled(nx=1), [0, 0])


def test_ionization_struct_layout_matches_c(tmp_path):
    from paper_1308_2590_gb300 import pic
    src = tmp_path / "sz3.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "pic.h"\n'
                   'int main(){printf("%zu %zu %zu %zu\\n", sizeof(pic_ionization), offsetof(pic_ionization, ip_ev),'
                   ' offsetof(pic_ionization, time_unit_au), offsetof(pic_ionization, seed));'
                   'return 0;}\n')
    exe = tmp_path / "sz3"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert vals == [ctypes.sizeof(pic.PicIonization), pic.PicIonization.ip_ev.offset,
                    pic.PicIonization.time_unit_au.offset, pic.PicIonization.seed.offset]


def test_collisions_struct_layout_matches_c(tmp_path):
    from paper_1308_2590_gb300 import pic
    src = tmp_path / "sz4.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "pic.h"\n'
                   'int main(){printf("%zu %zu %zu %zu %d\\n", sizeof(pic_collisions), offsetof(pic_collisions, b),'
                   ' offsetof(pic_collisions, ln_lambda), offsetof(pic_collisions, seed), PIC_MAX_COLLISION_PAIRS);'
                   'return 0;}\n')
    exe = tmp_path / "sz4"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert vals == [ctypes.sizeof(pic.PicCollisions), pic.PicCollisions.b.offset,
                    pic.PicCollisions.ln_lambda.offset, pic.PicCollisions.seed.offset, pic.MAX_COLLISION_PAIRS]
