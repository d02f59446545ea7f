"""Host helpers of bench.py that need no GPU: the figures it takes from a
committed ncu summary only while the kernel source is the one captured, and
only for the kernel and workload captured."""

import hashlib
import os
import re
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _summary(scratch, src_text, sha=None):
    src = scratch / "kernel.cuh"
    src.write_text(src_text)
    sha = sha or hashlib.sha256(src_text.encode()).hexdigest()[:16]
    prof = scratch / "summary.md"
    prof.write_text("# summary\n\n"
                    f"- kernel_source_sha256_16: `{sha}`\n"
                    "- dram_bytes_per_launch_full_size: 1234\n"
                    "- l2_peak_gbs_ncu: 36146\n")
    return str(prof), str(src)


def test_profiled_value_needs_the_captured_source(scratch):
    prof, src = _summary(scratch, "kernel v1")
    assert bench.profiled_value("dram_bytes_per_launch_full_size", prof, src) == 1234.0
    assert bench.profiled_value("l2_peak_gbs_ncu", prof, src) == 36146.0
    assert bench.profiled_value("no_such_key", prof, src) is None
    with open(src, "a") as f:
        f.write(" changed")          # the kernel changed since the capture
    assert bench.profiled_value("dram_bytes_per_launch_full_size", prof, src) is None
    assert bench.profiled_value("dram_bytes_per_launch_full_size", str(scratch / "missing.md"), src) is None


def test_committed_summary_is_used_only_for_the_kernel_it_captured():
    # the bench line cites the committed summary's DRAM and L2 bytes only while
    # the kernel source in the tree is the one that summary captured
    text = open(bench.PROFILE).read()
    vals = dict(re.findall(r"^- (\w+): `?([\w.]+)`?$", text, re.M))
    cur = hashlib.sha256(open(bench.KERNEL_SRC, "rb").read()).hexdigest()[:16]
    if vals["kernel_source_sha256_16"] == cur:
        assert bench.profiled_traffic() == pytest.approx(float(vals["dram_bytes_per_launch_full_size"]))
        assert bench.profiled_value("l2_bytes_per_launch_full_size") == pytest.approx(
            float(vals["l2_bytes_per_launch_full_size"]))
    else:
        assert bench.profiled_traffic() is None
        assert bench.profiled_value("l2_bytes_per_launch_full_size") is None


def test_profiled_case_is_the_default_workload_in_float32_only():
    A = types.SimpleNamespace
    assert bench.is_profiled_case(A(workload=bench.WORKLOAD, u_dtype="f32"), 10)
    assert not bench.is_profiled_case(A(workload=bench.WORKLOAD, u_dtype="bf16"), 10)
    assert not bench.is_profiled_case(A(workload=bench.WORKLOAD, u_dtype="f32"), 12)
    assert not bench.is_profiled_case(A(workload="rgb1920x1080_k15", u_dtype="f32"), 15)
    # the capture advanced a stream by 16 frames per launch
    assert bench.is_profiled_case(A(workload=bench.WORKLOAD, u_dtype="f32", frames_per_call=16), 10)
    assert not bench.is_profiled_case(A(workload=bench.WORKLOAD, u_dtype="f32", frames_per_call=1), 10)


def test_l2_roofline_arithmetic():
    r = bench.l2_roofline(2746.0, True)
    assert r["bound"] == "l2" and r["unit"] == "GB/s"
    assert r["frac"] == pytest.approx(2746.0 / r["peak"])
    # slices x sectors/cycle x bytes/sector x L2 clock, from the capture
    assert r["peak"] == pytest.approx(188 * 3 * 32 * 2.011017, rel=1e-4)
    assert "measured_copy_gbs" not in r
    m = bench.l2_roofline(2746.0, True, 20000.0)
    assert m["measured_copy_gbs"] == 20000.0 and m["frac_of_measured_copy"] == pytest.approx(2746.0 / 20000.0)
    assert bench.l2_roofline(2746.0, False) is None


def test_algorithmic_bytes_of_the_default_workload():
    # (n_cg + 2) reads of U, one write, a frame and a label byte per pass, the mask
    m, P, k, n_cg = 921600, 307200, 10, 5
    assert bench.algorithmic_bytes(m, P, k, n_cg, 1, 4) == 303820800


def test_bytes_of_the_passes_form():
    # 2 n_cg + 3 reads of U and one write; frame and weight byte in 2 n_cg + 2
    # passes; labels and mask written
    m, P, k, n_cg = 921600, 307200, 32, 5
    U = m * k * 4
    assert bench.passes_bytes(m, P, k, n_cg, 1, 4) == 14 * U + 12 * (m + P) + 2 * P == 1666867200
