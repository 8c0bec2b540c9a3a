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
    assert ctypes.sizeof(mw.mw_integrator) == 40
    assert ctypes.sizeof(mw.mw_thermo) == 136
    assert ctypes.sizeof(mw.mw_info) == 64


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
