"""Host logic of bench.py (no GPU): the step-kernel launch count it reports as
`gpu_launches`, and the guards on `roofline.traffic`, which is read from an ncu summary in
`profiles/` only while the kernel source, its block size, (for a batch) its tiling and
the way it steps all match the capture."""
import os
import re

import bench


def test_step_launches_counts_graph_runs_and_groups():
    g = bench.GRAPH_STEPS
    assert g == 64
    # one launch per step and launch group
    assert bench.step_launches(100, 2, False) == 200
    assert bench.step_launches(1, 1, False) == 1
    # persistent: one launch per run of up to 64 steps (a run of 100 steps is 64 + 36)
    assert bench.step_launches(100, 1, True) == 2
    assert bench.step_launches(64, 1, True) == 1
    assert bench.step_launches(130, 1, True) == 3
    assert bench.step_launches(0, 1, True) == 0


def test_kernel_source_hash_is_a_stable_digest_per_precision():
    a, b = bench.kernel_source_hash(), bench.kernel_source_hash()
    assert a == b and re.fullmatch(r"[0-9a-f]{16}", a)
    assert bench.kernel_source_hash("fp64") != a  # the FP64 unit differs


def _profile(tmp_path, **vals):
    path = os.path.join(tmp_path, "summary.md")
    with open(path, "w") as fh:
        fh.write("# a summary\n\nsome text: not a value line\n\n")
        for k, v in vals.items():
            fh.write("%s: `%s`\n\n" % (k, v))
    return path


def test_traffic_is_read_only_for_the_captured_configuration(tmp_path):
    h = bench.kernel_source_hash()
    path = _profile(tmp_path, kernel_hash=h, block_size=128, tile="128,2,28",
                    stepping="per-step", dram_bytes_per_node=68.994)
    n = 12272919
    got = bench.load_traffic(n, 128, path, "128,2,28", "per-step")
    assert abs(got - 68.994 * n) < 1e-3 * n
    # without a tile or stepping to check, the value is read as well
    assert bench.load_traffic(n, 128, path) == got
    # anything that differs from the capture gives no traffic figure
    assert bench.load_traffic(n, 128, path, "128,2,32", "per-step") is None
    assert bench.load_traffic(n, 128, path, "128,2,28", "persistent") is None
    assert bench.load_traffic(n, 96, path, "128,2,28", "per-step") is None
    stale = _profile(tmp_path, kernel_hash="0" * 16, block_size=128,
                     tile="128,2,28", stepping="per-step", dram_bytes_per_node=68.994)
    assert bench.load_traffic(n, 128, stale, "128,2,28", "per-step") is None
    assert bench.load_traffic(n, 128, os.path.join(tmp_path, "missing.md")) is None


def test_a_summary_without_a_stepping_line_matches_no_stepping(tmp_path):
    path = _profile(tmp_path, kernel_hash=bench.kernel_source_hash(), block_size=128,
                    dram_bytes_per_node=74.48)
    assert abs(bench.load_traffic(10, 128, path) - 744.8) < 1e-9
    assert bench.load_traffic(10, 128, path, stepping="persistent") is None
