"""Host logic of the benchmark, without a GPU: the algorithmic bytes per
zone-burn, the hash that ties an ncu summary to the kernel sources it was
taken at, and the reading of the summaries' machine-readable blocks."""
import os

import bench


def test_zone_bytes_count_inputs_outputs_counters_and_status():
    # Y0 and Y (16 N), T9 in and out, rho, E (4 doubles), nine int32
    # counters and the int32 status
    assert bench.zone_bytes(13) == 16 * 13 + 8 * 4 + 9 * 4 + 4
    assert bench.zone_bytes(48) == 840


def test_code_hash_ignores_comments_only():
    a = "int f(int x) {  // doubles x\n  /* the\n     rule */\n  return 2 * x;\n}\n"
    b = "// a header line\nint f(int x) {\n\n  return 2 * x;   // same code\n}\n"
    c = "int f(int x) {\n  return 3 * x;\n}\n"
    assert bench._code_only(a) == bench._code_only(b)
    assert bench._code_only(a) != bench._code_only(c)


def test_profiled_traffic_reads_the_matching_block(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    h = bench.kernel_source_hash()
    (prof / "k_demo_work.md").write_text(
        "# demo\n\n| dram | 1 |\n\n"
        "machine-readable (read by bench.py):\n"
        f"dram_bytes_per_launch: 111\nzones: 64\nlaunch: 256,2\nsource_hash: {h}\n\n"
        "machine-readable (read by bench.py):\n"
        f"dram_bytes_per_launch: 222\nzones: 64\nlaunch: 256,3\nsource_hash: {h}\n\n"
        "machine-readable (read by bench.py):\n"
        "dram_bytes_per_launch: 333\nzones: 64\nlaunch: 256,1\nsource_hash: 0000\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: h)
    assert bench.profiled_traffic("k_demo", 64, "256,2", workload="work") == 111
    assert bench.profiled_traffic("k_demo", 64, "256,3", workload="work") == 222
    assert bench.profiled_traffic("k_demo", 64, None, workload="work") == 111
    # another zone count, another launch shape, or another source hash: none
    assert bench.profiled_traffic("k_demo", 65, "256,2", workload="work") is None
    assert bench.profiled_traffic("k_demo", 64, "128,2", workload="work") is None
    assert bench.profiled_traffic("k_demo", 64, "256,1", workload="work") is None
    assert bench.profiled_traffic("k_other", 64, None, workload="work") is None


def test_warp_kernel_launch_shape():
    assert bench.coop_shape({"kernel": "coop", "threads_per_block": 128,
                             "blocks_per_sm": 3}) == "coop,128,3,0"
    assert bench.coop_shape({"kernel": "coop", "warps_per_zone": 2}) == "coop,0,0,2"
    assert bench.coop_shape({"specialize": 2}) is None
    assert bench.launch_shape({"threads_per_block": 256, "blocks_per_sm": 1}, 2) == "256,2"


def test_committed_summaries_parse():
    # every committed summary with a machine-readable block carries all four
    # keys, so the bench can match it
    d = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "profiles")
    found = 0
    for f in sorted(os.listdir(d)):
        text = open(os.path.join(d, f)).read()
        for block in text.split("machine-readable (read by bench.py):")[1:]:
            lines = block.strip().split("\n\n")[0].splitlines()
            keys = {line.split(":", 1)[0] for line in lines}
            assert keys == {"dram_bytes_per_launch", "zones", "source_hash"} | (
                {"launch"} if "launch" in keys else set()), (f, keys)
            found += 1
    assert found >= 6
