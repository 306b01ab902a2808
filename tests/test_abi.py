"""The C ABI library loads and exports every entry point declared in
include/nrt.h (no GPU needed; no compute calls)."""
import ctypes
import os
import re

from paper_2507_04021_gb300 import build, nrt

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    txt = open(os.path.join(ROOT, "include", "nrt.h")).read()
    return sorted(set(re.findall(r"\b(nrt_\w+)\s*\(", txt)))


def test_header_declares_boundary():
    names = declared()
    for n in ("nrt_create", "nrt_scene_upload", "nrt_trace", "nrt_paths_read", "nrt_field_read",
              "nrt_backward", "nrt_set_materials", "nrt_result_free", "nrt_scene_free"):
        assert n in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(build.build())
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_and_defaults():
    L = nrt.lib()
    assert L.nrt_status_string(0) == b"ok"
    assert L.nrt_status_string(4) == b"device buffer overflow"
    p = nrt.default_trace_params()
    assert p.kappa == 10 and abs(p.t_a_deg - 1.0) < 1e-7 and abs(p.t_d - 0.01) < 1e-9
    assert p.max_depth == 5
    assert p.spec_waves == 0  # the specular refinement's persistent pass
