"""The C ABI library loads and exports every symbol include/mw.h declares
(no compute calls: these run without a GPU)."""
import ctypes
import os
import re

from paper_0809_2811_gb300 import build, mw

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    hdr = open(os.path.join(ROOT, "include", "mw.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return set(re.findall(r"\b(mw_[a-z_0-9]+)\s*\(", hdr))


def test_library_builds_and_exports_every_declared_symbol():
    build.build()
    lib = ctypes.CDLL(mw.LIB_PATH)
    names = declared()
    assert names, "no declarations found"
    for n in names:
        assert hasattr(lib, n), n
    assert names == set(mw.EXPORTS)


def test_params_default_is_the_papers():
    p = mw.mw_params_default()
    assert (p.lambda_, p.epsilon, p.sigma, p.a, p.gamma) == (23.15, 6.189, 2.3925, 1.8, 1.2)
    assert (p.A, p.B, p.p, p.q) == (7.049556277, 0.6022245584, 4, 0)
    assert p.cos_theta0 == -1.0 / 3.0


def test_struct_sizes_match_header_layout():
    # sizes the C compiler gives these structs on LP64
    assert ctypes.sizeof(mw.mw_params) == 72
    assert ctypes.sizeof(mw.mw_integrator) == 56
    assert ctypes.sizeof(mw.mw_thermo) == 168
    assert ctypes.sizeof(mw.mw_info) == 96


def test_struct_layout_matches_the_c_compiler(tmp_path):
    """Every field offset of the ctypes mirrors equals the C compiler's for include/mw.h."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        import pytest
        pytest.skip("no C compiler")
    structs = [mw.mw_params, mw.mw_integrator, mw.mw_thermo, mw.mw_info]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "mw.h"', "int main(void) {"]
    expect = []
    for st in structs:
        name = st.__name__
        lines.append(f'  printf("%zu\\n", sizeof({name}));')
        expect.append(ctypes.sizeof(st))
        for f, _ in st._fields_:
            cf = "lambda" if f == "lambda_" else f
            lines.append(f'  printf("%zu\\n", offsetof({name}, {cf}));')
            expect.append(getattr(st, f).offset)
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert got == expect


def test_oracle_and_library_share_no_code():
    """Neither side includes, imports or links the other."""
    src_dir = os.path.join(ROOT, "paper_0809_2811_gb300")
    for dirpath, _, files in os.walk(src_dir):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".inc", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.findall(r"(?:import|include|from)\s+\"?([a-z_]+)", text), f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".c", ".py", ".h")):
            text = open(os.path.join(ROOT, "oracle", f)).read()
            refs = re.findall(r"^\s*(?:import|from|#\s*include)\s+[\"<]?([\w./]+)", text, flags=re.M)
            assert not [r for r in refs if "paper_0809_2811_gb300" in r or "mw_" in r or r == "mw.h"], (f, refs)


def test_degenerate_systems_are_refused_before_any_device_work():
    """Boxes of fewer than two atoms, an empty batch, non-positive or
    non-finite edges, mass and skin are refused with MW_EINVAL by the argument
    checks, which run before any device allocation (so this runs without a
    GPU)."""
    import pytest
    build.build()
    cases = [
        lambda: mw.mw_system_create(0, [20.0, 20.0, 20.0]),
        lambda: mw.mw_system_create(1, [20.0, 20.0, 20.0]),
        lambda: mw.mw_batch_create([8, 1, 8], [20.0] * 9),
        lambda: mw.mw_batch_create([], []),
        lambda: mw.mw_system_create(8, [20.0, 0.0, 20.0]),
        lambda: mw.mw_system_create(8, [20.0, float("nan"), 20.0]),
        lambda: mw.mw_system_create(8, [20.0, 20.0, 20.0], mass=0.0),
        lambda: mw.mw_system_create(8, [20.0, 20.0, 20.0], skin=-1.0),
    ]
    for make in cases:
        with pytest.raises(mw.MWError) as ei:
            make()
        assert ei.value.status == mw.MW_EINVAL
