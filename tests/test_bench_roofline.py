"""Host logic of bench.py's roofline entries (no GPU): the algorithmic bytes
and flops per launch that the fractions divide by, and the traffic record's
tie to the kernels' sources."""
import json
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PK = {"hbm": 6773.2, "sm_max_mhz": 2070}
INFO = {"core_dims": [10, 10, 10, 0], "iters": 26, "cg_total": 202}


def test_refine_pass_bytes_are_one_read_of_t_and_the_factors():
    import bench
    r = bench.algorithmic("refine_pass", (200, 200, 200), 10, INFO, 0.05, PK, 2070)
    # T once (32 MB) plus W read and the gradient written (2 x 10 x 600 floats)
    assert r["algorithmic_per_launch"] == 4.0 * 200 ** 3 + 4.0 * 2 * 10 * 600
    assert r["bound"] == "hbm" and r["peak"] == PK["hbm"]
    assert abs(r["achieved"] - r["algorithmic_per_launch"] / 0.05e-3 / 1e9) < 1e-6


def test_tensor_core_gram_reads_the_tensor_once():
    import bench
    r = bench.algorithmic("gram_bf16_tc", (200, 200, 200), 10, INFO, 0.03, PK, 2070)
    assert r["algorithmic_per_launch"] == 4.0 * 200 ** 3
    assert r["flops"] == 2.0 * 200 * 200 ** 3


def test_first_mode_projection_reads_t_and_writes_the_partial_core():
    import bench
    r = bench.algorithmic("project_T", (200, 200, 200), 10, INFO, 0.04, PK, 2070)
    # T once, then the 10 x 200 x 200 result of the first truncation step
    assert r["algorithmic_per_launch"] == 4.0 * 200 ** 3 + 4.0 * 10 * 200 * 200
    assert r["bound"] == "hbm"


def test_later_projections_follow_the_sequential_truncation():
    import bench
    r = bench.algorithmic("project", (200, 200, 200), 10, INFO, 0.01, PK, 2070)
    # mode 2: 10x200x200 -> 10x10x200; mode 3: 10x10x200 -> 10x10x10
    m2 = 4.0 * (10 * 200 * 200 + 10 * 10 * 200)
    m3 = 4.0 * (10 * 10 * 200 + 10 * 10 * 10)
    assert abs(r["algorithmic_per_launch"] - (m2 + m3) / 2) < 1e-6


@pytest.mark.parametrize("bf16,expected", [
    # modes 2 and 3 on the truncated 10x200x200 and 10x10x200 tensors
    (True, (2 * 200 * (10 * 200 * 200) + 2 * 200 * (10 * 10 * 200)) / 2),
    # with mode 1 on the CUDA cores as well: the full tensor's first Gram too
    (False, (2 * 200 * 200 ** 3 + 2 * 200 * (10 * 200 * 200) + 2 * 200 * (10 * 10 * 200)) / 3),
])
def test_fp32_gram_flops_follow_the_sequential_truncation(bf16, expected):
    import bench
    r = bench.algorithmic("gram_fp32", (200, 200, 200), 10, INFO, 0.03, PK, 2070, gram_bf16=bf16)
    assert abs(r["algorithmic_per_launch"] - expected) < 1e-6 * expected
    assert r["frac"] < 1.0


def test_traffic_record_is_reported_only_for_unchanged_sources(tmp_path, monkeypatch):
    import bench
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
        rec = json.load(fh)
    for stage, v in rec.items():
        assert stage in bench.STAGE_SOURCES and v["dram_bytes_per_launch"] > 0
        assert "--clock-control none" in v["capture"]
    # a record whose hash is not the sources' is ignored (reported as null)
    stale = {k: dict(v, sources_sha256="0" * 64) for k, v in rec.items()}
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(stale))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "sources_sha256", lambda stage: "1" * 64)
    for stage in stale:
        assert bench.measured_traffic(stage) is None


def test_default_workload_is_the_largest_single_gpu_configuration():
    import bench
    ap_default = [ln for ln in open(os.path.join(ROOT, "bench.py")) if '"--workload"' in ln][0]
    assert 'default="order4"' in ap_default
    w = bench.WORKLOADS["order4"]
    assert "100x100x100x100_r15" in w["name"] and w["opts"]["init"] == "random"


def test_fp32_peak_is_derived_from_the_sm_count():
    import bench
    a = bench.algorithmic("dgn_core", (200, 200, 200), 10, INFO, 0.7, PK, 2000, sms=152)
    b = bench.algorithmic("dgn_core", (200, 200, 200), 10, INFO, 0.7, PK, 2000, sms=76)
    assert abs(a["peak"] - 152 * 128 * 2 * 2000e6 / 1e12) < 1e-9
    assert abs(b["peak"] - a["peak"] / 2) < 1e-9 and "derived" in a["peak_kind"]
