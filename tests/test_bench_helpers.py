"""Host-side logic of bench.py (no GPU): the FP32 peak arithmetic, the parsing of the
nvidia-smi clock samples, and the lookup of the committed DRAM-traffic record by plan."""
import json
import os

import bench


def test_fp32_peak_is_two_flop_per_lane_per_clock():
    assert bench.fp32_peak_tflops(152, 2070.0) == 2 * 128 * 152 * 2070e6 / 1e12


def test_clock_summary_parses_samples_and_reasons():
    cs = bench.ClockSampler(0)
    cs.lines = [
        "2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "2055, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "garbage line",
        "2070, 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    s = cs.summary()
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"],
                 "samples": 3}
    cs.lines = []
    assert cs.summary() is None


def test_traffic_record_lookup_by_plan():
    for key, name in bench.TRAFFIC_FILES.items():
        path = os.path.join(bench.ROOT, "profiles", name)
        if not os.path.exists(path):
            continue
        with open(path) as f:
            rec = json.load(f)
        assert rec["records"], "no traffic records"
        for r in rec["records"]:
            got = bench.profiled_traffic(key, r["variant"], r["split"])
            want = r["dram_bytes_read_per_launch"] + r["dram_bytes_write_per_launch"]
            # the record counts while the force-kernel sources are the ones it was taken on
            assert got in (want, None)
    assert bench.profiled_traffic("sphere1m", "no-such-variant", 0) is None
    assert bench.profiled_traffic("no-such-workload", "f32x2.fold64.t64r1k128", 0) is None


def test_workload_key_lookup():
    assert bench.bunch_key(bench.WORKLOAD) == "sphere1m"
    assert bench.bunch_key(bench.SIDE_WORKLOAD) == "gaussian65536"


def test_both_arms_print_the_same_config():
    cfg = bench.bench_config(bench.WORKLOAD, 1)
    assert cfg["N"] == 1 << 20 and cfg["workload"] == bench.WORKLOAD.name
    assert cfg == bench.bench_config(bench.WORKLOAD, 1)
    assert bench.bench_config(bench.WORKLOAD, 2)["parallelism"] == "replicas x2"


def test_default_run_is_short():
    args = bench.parse([])
    assert args.steps >= 1 and args.warmup >= 3
