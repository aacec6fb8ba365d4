"""The benchmark's reporting logic on the CPU: the roofline object (binding roof, achieved,
fraction, traffic) from per-class launch tallies, and the clock sampler's parsing of the
nvidia-smi CSV. No GPU: the inputs are written out by hand."""

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def prof(**classes):
    base = {"launches": 0, "timed": 0, "ms": 0.0, "flops": 0.0, "bytes": 0.0}
    out = {k: dict(base) for k in ("dst", "coarse", "sweep", "matvec", "multidot", "update", "axpy", "reduce",
                                   "pack")}
    for k, v in classes.items():
        out[k].update(v)
    return out


def test_fp64_alu_bound_kernel_reports_against_the_fp64_peak():
    import bench
    # 10 launches, 100 ms in all, 50 GFLOP and 10 GB: the FP64 roof (50e9 / 1.2586e12 = 40 ms) is
    # above the HBM roof (10e9 / 6800e9 = 1.5 ms)
    p = prof(dst={"launches": 10, "timed": 10, "ms": 100.0, "flops": 50e9, "bytes": 10e9},
             update={"launches": 5, "timed": 5, "ms": 20.0, "flops": 1e9, "bytes": 40e9})
    r = bench.roofline(p, {"hbm_gbs": 6800.0}, "measured")
    assert r["kernel"] == "dst_tile_kernel" and r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(50e9 / 0.1 / 1e12)
    assert r["peak"] == pytest.approx(bench.FP64_PEAK_TFLOPS)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["per_launch_ms"] == pytest.approx(10.0)
    assert r["traffic"] == pytest.approx(1e9 * bench.TRAFFIC_RATIO["dst_tile_kernel"])
    assert r["share_of_step"] == pytest.approx(100.0 / 120.0)


def test_probed_peaks_replace_the_derived_ones():
    """With this run's probe in the peaks, the FP64 kernels report against the measured FMA rate
    and the TF32 transforms against the measured TF32 GEMM."""
    import bench
    p = prof(dst={"launches": 10, "timed": 10, "ms": 100.0, "flops": 50e9, "bytes": 10e9})
    peaks = {"hbm_gbs": 6800.0, "bf16_tflops": 1800.0, "fp64_fma_tflops": 1.04, "tf32_tflops": 900.0}
    r = bench.roofline(p, peaks, "measured")
    assert r["peak"] == pytest.approx(1.04) and "probe" in r["peak_source"]
    assert r["frac"] == pytest.approx(0.5 / 1.04)
    p2 = prof(dst={"launches": 2, "timed": 2, "ms": 2.0, "flops": 2e12, "bytes": 1e9})
    r2 = bench.roofline(p2, peaks, "measured", precision="tf32")
    assert r2["peak"] == pytest.approx(900.0) and r2["bound"] == "tensor"
    p3 = prof(pack={"launches": 2, "timed": 2, "ms": 2.0, "flops": 0.0, "bytes": 12e9})
    r3 = bench.roofline(p3, peaks, "measured", precision="bf16")
    assert r3["kernel"] == "pack_kernel" and r3["bound"] == "hbm"


def test_memory_bound_kernel_reports_against_the_measured_copy_bandwidth():
    import bench
    p = prof(update={"launches": 4, "timed": 4, "ms": 10.0, "flops": 1e9, "bytes": 60e9})
    r = bench.roofline(p, {"hbm_gbs": 6000.0}, "measured")
    assert r["kernel"] == "mgsb_step_kernel" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(60e9 / 0.01 / 1e9)
    assert r["peak"] == 6000.0 and r["frac"] == pytest.approx(1.0)
    ratio = bench.TRAFFIC_RATIO.get("mgsb_step_kernel")
    assert r["traffic"] == (pytest.approx(15e9 * ratio) if ratio else None)
    r0 = bench.roofline(p, {"hbm_gbs": 6000.0}, "measured", orth=0)
    assert r0["kernel"] == "mgs_step_kernel"
    assert r0["traffic"] == pytest.approx(15e9 * bench.TRAFFIC_RATIO["mgs_step_kernel"])


def test_tensor_core_transform_reports_against_its_own_dtype_peak():
    import bench
    p = prof(dst={"launches": 2, "timed": 2, "ms": 2.0, "flops": 2e12, "bytes": 1e9})
    peaks = {"hbm_gbs": 6800.0, "bf16_tflops": 1800.0}
    r_bf16 = bench.roofline(p, peaks, "measured", precision="bf16")
    r_tf32 = bench.roofline(p, peaks, "measured", precision="tf32")
    assert r_bf16["bound"] == r_tf32["bound"] == "tensor"
    assert r_bf16["peak"] == pytest.approx(1800.0)
    assert r_tf32["peak"] == pytest.approx(1800.0 * 1.1 / 2.25)
    assert r_bf16["achieved"] == pytest.approx(1000.0)
    assert r_bf16["traffic"] is None   # no ncu ratio for the GEMM kernel
    r_oz = bench.roofline(p, peaks, "measured", dst_method="tensor")   # FP64 digit-plane products
    assert r_oz["kernel"] == "oz_gemm_kernel" and r_oz["bound"] == "tensor"
    assert r_oz["peak"] == pytest.approx(1800.0)
    ratio = bench.TRAFFIC_RATIO.get("oz_gemm_kernel")
    assert r_oz["traffic"] == (pytest.approx(0.5e9 * ratio) if ratio else None)


def test_clock_sampler_parses_and_flags_throttle_reasons(tmp_path):
    import bench
    csv = tmp_path / "clocks.csv"
    csv.write_text(
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n"
        "0, 1980, 2070, 1400.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active\n"
        "0, 2070, 2070, 950.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n"
        "garbage line\n")
    s = bench.ClockSampler(0)

    class Done:
        def terminate(self):
            pass

        def wait(self):
            pass

    s.proc, s.path = Done(), str(csv)
    out = s.stop()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0 and out["samples"] == 3
    assert out["reasons"] == ["sw_power_cap"]
    assert not csv.exists()


def test_reference_arm_prints_one_complete_line(monkeypatch, capsys):
    """The reference arm's JSON line (the oracle's time per iteration stubbed out: the real
    sample takes tens of seconds) carries the keys the GPU arm's line has, the same config and
    metric, and a cpu_baseline describing itself."""
    import argparse
    import json
    import bench
    monkeypatch.setattr(bench, "oracle_iteration_sample", lambda w, kdim: (0.5, "stub sample"))
    args = argparse.Namespace(gpus=1, steps=2, warmup=1, omega=1e-4, ref_iterations=25, orth=None)
    assert bench.run_reference(args) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["value"] == 1.0 / (0.5 * 25) and line["unit"] == "solves/s"
    assert line["config"] == bench.describe(bench.workload_for(1e-4), 2)
    assert line["config"]["orthogonalisation"] == bench.ORTH_TEXT[2]
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0
    args.orth = "mgs"
    assert bench.run_reference(args) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["config"]["orthogonalisation"] == bench.ORTH_TEXT[0]
