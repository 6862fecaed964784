"""The bench's own arithmetic, on the CPU: the per-unit algorithmic bytes of the
sampler (8 B of in-CSR offsets per member and per set, 8 B per examined in-edge, 4 B
emitted per member, 8 B of set offsets per set), the weighting of the IC and LT oracle
rates into one step's rate, and the defaults of the command line."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_sampler_bytes_per_unit():
    p = {"pass1_members": 10, "pass1_sets": 3, "pass1_examined": 100}
    # 8 (10 + 3) + 8 * 100 + 4 * 10 + 8 * 3
    assert bench.sampler_bytes(p, 1) == 104 + 800 + 40 + 24
    p = {"pass2_members": 0, "pass2_sets": 0, "pass2_examined": 0}
    assert bench.sampler_bytes(p, 2) == 0


def test_mix_rate_is_a_harmonic_weighting():
    rates = {"IC": (100.0, None), "LT": (400.0, None)}
    # 7 IC sets at 100/s and 2 LT sets at 400/s take 0.07 + 0.005 s
    assert abs(bench.mix_rate(rates, 7, 2) - 9 / 0.075) < 1e-9
    assert bench.mix_rate(rates, 5, 0) == 100.0


def test_default_command_line_is_one_gpu_within_minutes():
    a = bench.parse_args([])
    assert a.gpus == 1 and a.impl == "ours" and a.mode == "timplus"
    assert a.workload == "c3"  # the largest configuration is the headline
    assert a.warmup >= 3 and 1 <= a.steps <= 10
    # the nested R-MAT line
    assert a.scale == 20 and a.k == 50 and a.eps == 0.1 and a.ell == 1.0


def test_roofline_takes_the_pass_with_most_kernel_time():
    p = {f"pass{i}_{k}": 0 for i in (1, 2, 3) for k in ("ms", "launches", "members", "sets",
                                                          "examined")}
    p.update({"pass1_ms": 5.0, "pass1_launches": 2, "pass2_ms": 7.0, "pass2_launches": 2,
              "pass3_ms": 40.0, "pass3_launches": 3, "pass3_batches": 4, "pass3_ms_kernel": 20.0,
              "pass3_members": 100, "pass3_sets": 10, "pass3_examined": 1000})
    r = bench.sampler_roofline(p, "c2")
    assert r["kernel"].startswith("bulk_levels_kernel") and r["launches"] == 4
    # the heavy pass's persistent launches alone: 20 ms over 4 launches
    assert r["ms_per_launch"] == 5.0
    alg = bench.sampler_bytes(p, 3)
    assert abs(r["achieved"] - alg / 0.020 / 1e9) < 1e-9 and r["bytes_per_launch"] == alg / 4


def test_dram_bytes_per_member_are_from_a_capture_or_null():
    for wl in ("c3", "c2"):
        for i in (1, 2, 3):
            v = bench.DRAM_BYTES_PER_MEMBER[wl].get(i)
            assert v is None or 1.0 < v < 10_000.0
