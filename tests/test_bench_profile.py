"""bench.py reports the dominant kernel's DRAM traffic from the committed
ncu summary only while the summary's source hash matches the FP32 sweep's
code (a change to the code must void it, a comment edit must not) and only
on the workload the summary was captured on."""
import os
import shutil

import bench

FILES = ("wcns_device.cuh", "wcns_cvt.cuh", "wcns_sweep.cuh", "sweep_fp32.cu")


def _copy_tree(tmp_path):
    src = os.path.join(bench.ROOT, "paper_1810_07806_gb300", "csrc")
    dst = tmp_path / "paper_1810_07806_gb300" / "csrc"
    dst.mkdir(parents=True)
    for f in FILES:
        shutil.copy(os.path.join(src, f), dst / f)
    return dst


def test_comment_edit_keeps_and_code_edit_voids_the_profile(tmp_path, monkeypatch):
    """A summary written for the current code is used; a comment edit keeps
    it, a code edit voids it."""
    csrc = _copy_tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_source_hash()
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "sweep_fp32_tgv.md").write_text(
        "kernel_source_sha256: %s\ntraffic_bytes_per_full_launch: 1.5e9\n"
        "traffic_workload: taylor_green_3d_256^3_periodic\n" % h0)
    assert bench.profile_traffic("taylor_green_3d_256^3_periodic") == 1.5e9
    # another workload (another grid, another dimension) has no captured traffic
    assert bench.profile_traffic("four_quadrant_riemann_2d_1024^2_lax_liu_3") is None
    f = csrc / "wcns_sweep.cuh"
    src = f.read_text()
    f.write_text(src + "\n// a comment\n\n")
    assert bench.kernel_source_hash() == h0
    assert bench.profile_traffic("taylor_green_3d_256^3_periodic") == 1.5e9
    f.write_text(src.replace("static constexpr int THREADS = 256;", "static constexpr int THREADS = 128;", 1))
    assert bench.kernel_source_hash() != h0
    assert bench.profile_traffic("taylor_green_3d_256^3_periodic") is None
