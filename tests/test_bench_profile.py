"""bench.py reports a committed ncu figure only while the sources it was taken
from are unchanged: the validation phase's follow the whole of sim.cu and
nrt_device.cuh, the trace and visibility kernels' follow the part of sim.cu
before its validation code (which holds them) and nrt_device.cuh."""
import hashlib
import os
import shutil

import bench

MARK = bench._VALIDATION_MARK.encode()


def _copy_tree(tmp_path):
    root = tmp_path / "repo"
    (root / "profiles").mkdir(parents=True)
    csrc = root / "paper_2507_04021_gb300" / "csrc"
    csrc.mkdir(parents=True)
    src = os.path.join(bench.ROOT, "paper_2507_04021_gb300", "csrc")
    for f in ("sim.cu", "nrt_device.cuh"):
        shutil.copy(os.path.join(src, f), csrc / f)
    sim = (csrc / "sim.cu").read_bytes()
    dev = (csrc / "nrt_device.cuh").read_bytes()
    whole = hashlib.sha256(sim + dev).hexdigest()
    trav = hashlib.sha256(sim[: sim.index(MARK)] + dev).hexdigest()
    (root / "profiles" / "office_sim_top_kernels.md").write_text(
        "traffic_bytes_per_launch validation 100\n"
        "traffic_bytes_per_launch trace_kernel 200\n"
        "traffic_bytes_per_launch vis_kernel 300\n"
        "l2_bytes_per_unit trace_kernel 4.5\n"
        f"source_sha256 {whole}\nsource_sha256_traversal {trav}\n")
    return root, csrc / "sim.cu"


def test_figures_follow_their_own_sources(tmp_path, monkeypatch):
    root, sim = _copy_tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench._traffic("validation") == 100
    assert bench._traffic("trace_kernel") == 200 and bench._traffic("vis_kernel") == 300
    assert bench._l2_bytes("trace_kernel") == 4.5
    # a change in the validation code leaves the traversal kernels' figures
    text = sim.read_bytes()
    sim.write_bytes(text + b"\n// changed validation code\n")
    assert bench._traffic("validation") is None
    assert bench._traffic("trace_kernel") == 200 and bench._l2_bytes("trace_kernel") == 4.5
    # a change before the validation code invalidates them too
    sim.write_bytes(b"// changed traversal code\n" + text)
    assert bench._traffic("trace_kernel") is None and bench._traffic("vis_kernel") is None
    assert bench._traffic("validation") is None


def test_missing_marker_reports_nothing(tmp_path, monkeypatch):
    root, sim = _copy_tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    sim.write_bytes(sim.read_bytes().replace(MARK, b"// renamed"))
    assert bench._traffic("trace_kernel") is None
