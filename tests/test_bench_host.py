"""Host-side logic of bench.py (no GPU): the roofline arithmetic of the dominant kernel
class, the clock-sample summary that decides whether a run is rejected, and the JSON
fields the bench contract requires."""
import bench


def _prof(ms, launches, byts, flops):
    return {"ms": ms, "launches": launches, "bytes": byts, "flops": flops}


def test_roofline_alu_bound_fp64_class():
    prof = {"jacobi": _prof(162.5, 60, 3.98e10, 2.25e10)}
    r = bench.roofline("jacobi", prof, [], {"name": "block_permuted_200000x100000"})
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert abs(r["achieved"] - 2.25e10 / 0.1625 / 1e12) < 1e-9
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
    assert r["traffic"] == bench.MEASURED_TRAFFIC.get(("block_permuted_200000x100000", "jacobi"))


def test_roofline_tensor_class_counts_slice_products():
    """The Gram and product classes run as 36 BF16 slice products per FP64 product: the
    roofline is against the BF16 tensor peak, with the FP64-equivalent rate beside it."""
    prof = {"gram": _prof(77.1, 70, 1.16e10, 7.04e11)}
    r = bench.roofline("gram", prof, [], {"name": "block_permuted_200000x100000"})
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert abs(r["fp64_equivalent_tflops"] - 7.04e11 / 0.0771 / 1e12) < 1e-9
    assert abs(r["achieved"] - 36 * r["fp64_equivalent_tflops"]) < 1e-9
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12


def test_roofline_hbm_bound_when_intensity_is_low():
    prof = {"spmm": _prof(10.0, 4, 4e10, 1e9)}          # 0.025 flop per byte
    r = bench.roofline("spmm", prof, [], {"name": "x"})
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert abs(r["achieved"] - 4e10 / 0.010 / 1e9) < 1e-6


def test_clock_summary_flags_throttle_reasons():
    c = bench.ClockSampler(0)
    c.lines = ["2070, 2070, 900.0, Not Active, Not Active, Not Active, Not Active",
               "1800, 2070, 1400.0, Not Active, Not Active, Not Active, Active",
               "1900, 2070, 1400.0, Active, Not Active, Not Active, Not Active",
               "garbage"]
    s = c.summary()
    assert s["samples"] == 3 and s["sm_max_mhz"] == 2070.0 and s["sm_mhz"] == 1900.0
    assert s["reasons"] == ["hw_slowdown", "sw_power_cap"]
    assert bench.ClockSampler(0).summary()["sm_mhz"] is None


def test_job_throughput_is_whole_job():
    assert bench.job_throughput(10, 4, 2.0) == 20.0


def test_reference_arm_json_line():
    """`bench.py --impl reference` (the CPU oracle arm) on the small 2000 x 1000 workload
    prints one JSON line with the contract's keys, the requested warm-up and step counts,
    and every solve valid."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--workload",
                        "random_sparse_2000x1000", "--steps", "2", "--warmup", "3"],
                       capture_output=True, text=True, timeout=600, cwd=root)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "e2e", "cpu_baseline"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 3
    assert d["config"]["workload"] == "random_sparse_2000x1000" and d["all_steps_valid"] is True
    assert d["value"] > 0 and d["e2e"]["value"] == d["value"] and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["cores"] >= 1
