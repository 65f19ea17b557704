"""Host-side logic of bench.py (CPU only): the profile-traffic lookup that
feeds the roofline's `traffic` field, the launch count, and the oracle's
CPU-baseline sampler on a small workload."""

import os

import bench
import synth
from paper_2410_04974_gb300.render import make_plan, make_settings


def test_profiled_traffic_needs_a_matching_source_digest(tmp_path, monkeypatch):
    kernel = "blend_fused_kernel"
    prof = tmp_path / "profiles"
    prof.mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_digest", lambda k: "abc123")
    (prof / f"{kernel}_wl.md").write_text("traffic_bytes_per_launch: 12345\nsource_digest: abc123\n")
    assert bench.profiled_traffic(kernel, "wl") == 12345
    (prof / f"{kernel}_wl.md").write_text("traffic_bytes_per_launch: 12345\nsource_digest: stale\n")
    assert bench.profiled_traffic(kernel, "wl") is None
    assert bench.profiled_traffic(kernel, "missing") is None


def test_every_committed_profile_names_a_known_kernel():
    names = os.listdir(os.path.join(os.path.dirname(os.path.abspath(bench.__file__)), "profiles"))
    kernels = set(bench.KERNEL_SOURCES)
    for n in names:
        if n.startswith("launch_list_"):
            continue
        assert any(n.startswith(k + "_") for k in kernels), n


def test_launches_per_frame_counts_the_step_kernels():
    cams = synth.ring_cameras(8, 800, 800)
    plan = make_plan(300_000, 3, cams, make_settings())
    # upload, projection, compaction, 4 depth passes, emission scan + expand,
    # 2 tile passes, ranges, fused blend, SH backward, geometry backward
    assert plan.depth_passes == 4 and plan.tile_passes == 2
    assert bench.launches_per_frame(plan, 8) == 1 + 1 + 1 + 4 + 2 + 2 + 1 + 1 + 1 + 1


def test_oracle_baseline_times_whole_views_with_all_and_one_thread():
    w = synth.make_workload(0)
    r = bench.oracle_baseline(w)
    assert r["kind"] == "oracle" and r["unit"] == bench.UNIT and r["value"] > 0 and r["cores"] >= 1
    assert r["sample"].startswith("2 whole views") and r["cpu_model"]
    st = r["single_thread"]
    assert st["cores"] == 1 and st["value"] > 0


def test_reference_arm_line_matches_the_workload_config(capsys):
    """The reference arm prints one line per the contract, with the same
    config as the GPU arm's and one whole view per step."""
    import argparse
    import json

    args = argparse.Namespace(config=0, n=0, steps=1, warmup=0)
    bench.run_reference(args, 1, 0)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == bench.UNIT and line["steps"] == 1
    w = synth.make_workload(0)
    assert line["config"] == bench.workload_config(w, (16, 16), 1)
    assert abs(line["ms_per_step"] - 1000.0 / line["value"]) < 0.02 * line["ms_per_step"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0
