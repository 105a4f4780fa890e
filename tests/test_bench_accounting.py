"""The benchmark's accounting, on the host: the algorithmic flops and bytes
behind the roofline fractions, the whole-job rate, and the stored ncu
traffic being dropped once a kernel's sources change."""
import importlib.util
import json
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


class _Dec:
    in_dim = 32


def test_flops_per_query(bench):
    interp, layer1, out = bench.flops_per_query(32, 5, "bf16")
    assert interp == 2 * 8 * 32 * 5          # 8 corners x 32 channels of FMAs per level
    assert layer1 == 2 * 128 * 32 == 8192    # the 128 x 32 contraction of Eq. 2
    assert out == 256
    assert bench.flops_per_query(35, 1, "f32")[1] == 2 * 128 * 35


def test_traversal_bytes(bench):
    # 2 rays; Decide visits 2 + 3 pairs at depths 0..1; 4 final entries (voxel
    # ids only: the frame's lists carry no t ranges) at depth 2
    sizes = [2, 3, 4]
    assert bench.traversal_bytes(None, sizes) == 36 * 2 + 16 * (2 + 3) + 12 * 4


def test_job_rate(bench):
    assert bench.job_rate(1000, 4, 0.5) == 8000


def test_trace_roofline_units(bench):
    W = {"dec": _Dec(), "lod": 5}
    res = {"queries_per_frame": 4_000_000, "ms_trace": 2.0}
    peaks = {"bf16_tflops": 2000.0}
    r = bench.trace_roofline(W, res, "bf16", peaks)
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(4e6 * 8192 / 2e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / 2000.0)
    assert r["gather_bytes_per_query"] == 8 * 32 * 4 * 5
    # the summed corner table gathers one level
    r1 = bench.trace_roofline(W, res, "bf16", peaks, levels=1)
    assert r1["gather_bytes_per_query"] == 8 * 32 * 4
    assert r1["achieved"] == pytest.approx(r["achieved"])
    f = bench.trace_roofline(W, res, "f32", {"sm_max_mhz": 2000.0})
    assert f["bound"] == "alu"
    assert f["peak"] == pytest.approx(152 * 128 * 2 * 2000e6 / 1e12)


def test_stale_traffic_is_dropped(bench, tmp_path, monkeypatch):
    path = tmp_path / "traffic.json"
    good = bench.source_hash("k_trace_bf16")
    path.write_text(json.dumps({"k_trace_bf16": {"dram_bytes_per_launch": 123, "source_hash": good},
                                "k_trace_bf16@summed": {"dram_bytes_per_launch": 45, "source_hash": good},
                                "k_traverse": {"dram_bytes_per_launch": 7, "source_hash": "0" * 16}}))
    monkeypatch.setattr(bench, "PROFILE_TRAFFIC", str(path))
    assert bench.profiled_traffic("k_trace_bf16") == 123
    assert bench.profiled_traffic("k_trace_bf16", "@summed") == 45
    assert bench.profiled_traffic("k_traverse") is None          # sources changed since the capture
    assert bench.profiled_traffic("k_trace_f32") is None          # never captured


def test_rooflines_use_measured_ceilings(bench):
    # with probe-measured ceilings the FP32 tracer divides by the measured FFMA
    # rate and the gathers are reported against the measured L1 / L2 reads
    W = {"dec": _Dec(), "lod": 5}
    res = {"queries_per_frame": 1_000_000, "ms_trace": 1.0}
    ceil = {"sms": 148, "ffma_tflops": 70.0, "l1_read_GBps": 40000.0, "l2_read_GBps": 20000.0}
    f = bench.trace_roofline(W, res, "f32", {"sm_max_mhz": 2000.0}, ceilings=ceil)
    assert f["peak"] == 70.0 and "measured" in f["peak_source"]
    gbps = 1e6 * 8 * 32 * 4 * 5 / 1e-3 / 1e9
    assert f["gather_GBps"] == pytest.approx(gbps)
    assert f["gather_frac_of_l1"] == pytest.approx(gbps / 40000.0)
    assert f["gather_frac_of_l2"] == pytest.approx(gbps / 20000.0)
    # without a measured FFMA rate: the nominal count from the device's SMs
    g = bench.trace_roofline(W, res, "f32", {"sm_max_mhz": 2000.0}, ceilings={"sms": 148})
    assert g["peak"] == pytest.approx(148 * 128 * 2 * 2000e6 / 1e12)
    b = bench.trace_roofline(W, res, "bf16", {"bf16_tflops": 2000.0}, ceilings=ceil)
    assert b["gather_frac_of_l2"] == pytest.approx(gbps / 20000.0)


def test_source_hash_ignores_comments_only(bench, tmp_path, monkeypatch):
    """Stored DRAM traffic is kept across comment edits and dropped when the
    code changes."""
    src = tmp_path / "k.cu"
    src.write_text("// kernel\n__global__ void k(int* p) { p[0] = 1; }\n")
    monkeypatch.setattr(bench, "CSRC", str(tmp_path))
    monkeypatch.setitem(bench.KERNEL_SRC, "k_probe_hash", ["k.cu"])
    h0 = bench.source_hash("k_probe_hash")
    src.write_text("/* the same kernel,\n   documented */\n__global__ void k(int* p) { p[0] = 1; }  // store\n")
    assert bench.source_hash("k_probe_hash") == h0
    src.write_text("__global__ void k(int* p) { p[0] = 2; }\n")
    assert bench.source_hash("k_probe_hash") != h0
