"""bench.py's accounting, on the CPU: the algorithmic bytes of a stage, the
compulsory values of each kernel, and the gate that keeps a DRAM capture out
of the roofline once the kernel sources it was taken on have changed."""

import pytest

import bench


def test_stage_bytes_are_the_method_s_own():
    # stage 1 reads q (5 values) and S (1) and writes the stage output (5);
    # stages 2-3 also read q^n (5); 8-byte values, the three stages averaged
    per_stage = [8 * (5 + 1 + 5), 8 * (5 + 1 + 5 + 5), 8 * (5 + 1 + 5 + 5)]
    assert bench.STAGE_BYTES_PER_NODE == pytest.approx(sum(per_stage) / 3)
    assert round(bench.STAGE_BYTES_PER_NODE, 1) == 114.7


def test_kernel_values_cover_the_stage():
    v = bench.KERNEL_VALUES_PER_NODE
    # every split pass moves at least the stage's own values: the z pass reads
    # q (and q^n in stages 2-3) and S and writes the output
    assert v["k_line_z"] >= 5 + 1 + 5 + 5 * 2 / 3
    # the fused FP32 pass moves exactly the stage's own values
    assert v["k_f_column"] == pytest.approx(5 + 1 + 5 * 2 / 3 + 5)
    # the mixed y pass hands one plane of face rows (5 values) per segment of
    # N = 4 planes to the z pass, which reads them back
    assert v["k_df_tline_y"] - v["k_line_y"] == pytest.approx(5 / 4)
    assert v["k_df_tline_z"] - v["k_line_z"] == pytest.approx(5 / 4)
    for names in bench.KERNEL_NAMES.values():
        for k in names:
            assert k == "-" or k in v


def _write(path, text):
    with open(path, "w") as f:
        f.write(text)


def test_traffic_is_used_only_for_the_sources_it_was_taken_on(tmp_path, monkeypatch):
    src = tmp_path / "kernel.cuh"
    _write(src, "// one kernel\n")
    monkeypatch.setattr(bench, "KERNEL_SRCS", [str(src)])
    sha = bench.kernel_source_sha()
    assert len(sha) == 16
    traffic = tmp_path / "ncu_traffic.txt"
    _write(traffic, "# a comment line\nsource_sha %s\nk_a 100\nk_b 250.5\n" % sha)
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(traffic))
    assert bench.traffic_per_launch("k_a") == 100.0
    assert bench.traffic_per_launch("k_missing") is None
    assert bench.stage_traffic(["k_a", "k_b"]) == 350.5
    assert bench.stage_traffic(["k_a", "k_missing"]) is None
    _write(src, "// one kernel, changed\n")          # the capture no longer applies
    assert bench.kernel_source_sha() != sha
    assert bench.traffic_per_launch("k_a") is None
    assert bench.stage_traffic(["k_a", "k_b"]) is None
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tmp_path / "absent.txt"))
    assert bench.traffic_per_launch("k_a") is None
