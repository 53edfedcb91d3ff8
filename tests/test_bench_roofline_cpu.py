"""The roofline arithmetic of bench.py on a synthetic kernel profile (no GPU):
the dominant AP pass is the one with the largest device time; achieved = its
algorithmic bytes per launch / its time per launch; frac = achieved / peak;
traffic = the measured DRAM bytes per right-hand side (from a committed
profile table, only while the kernel's source is the one captured) x
right-hand sides per launch; the SIMT passes are reported against the FP32 (or
FP64) ALU peak."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1811_03557_gb300.workloads import WORKLOADS  # noqa: E402


def rec(ms_total, launches):
    return {"ms_total": ms_total, "launches": launches, "ms_per_launch": ms_total / launches}


def test_tensor_core_roofline_picks_the_dominant_pass(monkeypatch):
    monkeypatch.setattr(bench, "measured_peaks", lambda: ({"hbm_gbs": 7000.0}, "measured"))
    monkeypatch.setattr(bench, "profile_traffic", lambda k, root=None: 16.4e6 if k == "k_tc_pencil" else None)
    w = WORKLOADS["pks_sphere_N128_K8"]
    prof = {"tc_plane_fwd": rec(6.8, 20), "tc_pencil": rec(7.2, 20), "tc_plane_inv": rec(7.0, 20),
            "lsq_cholesky": rec(9.9, 10)}  # not an AP pass: never the roofline kernel
    r = bench.roofline(w, 2, prof, None)
    assert r["kernel"] == "tc_pencil" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    n3 = float(w.N) ** 3
    bytes_per = ((w.ncol + 2) * 8 * n3 + 2 * 8 * n3) / 2  # the two batches' average launch
    assert r["bytes_per_launch"] == pytest.approx(bytes_per)
    ach = bytes_per / (0.36e-3) / 1e9
    assert r["achieved"] == pytest.approx(ach)
    assert r["peak"] == 7000.0 and r["frac"] == pytest.approx(ach / 7000.0)
    rhs_per_launch = ((w.ncol + 2) + 2) / 2
    assert r["traffic"] == pytest.approx(16.4e6 * rhs_per_launch)


def test_profile_traffic_table_and_staleness(tmp_path):
    src = "paper_1811_03557_gb300/csrc/dst_tc.cu"
    (tmp_path / "paper_1811_03557_gb300" / "csrc").mkdir(parents=True)
    (tmp_path / src).write_text("kernel source v1\n")
    (tmp_path / "profiles").mkdir()
    sha = bench.source_sha(src, str(tmp_path))
    (tmp_path / "profiles" / "k.md").write_text(
        "# capture\n\n| kernel | DRAM bytes per right-hand side | source | source sha256 |\n"
        "|---|---|---|---|\n"
        f"| k_tc_plane\\<1> | 6954321 | {src} | {sha} |\n| k_tc_pencil | 16407091 | {src} | {sha} |\n\ntext\n")
    assert bench.profile_traffic("k_tc_pencil", str(tmp_path)) == 16407091.0
    assert bench.profile_traffic("k_tc_plane<1>", str(tmp_path)) == 6954321.0
    assert bench.profile_traffic("k_fft_pencil", str(tmp_path)) is None
    (tmp_path / src).write_text("kernel source v2\n")          # the kernel changed: stale
    assert bench.profile_traffic("k_tc_pencil", str(tmp_path)) is None


def test_simt_roofline_is_alu_bound(monkeypatch):
    monkeypatch.setattr(bench, "measured_peaks", lambda: ({"hbm_gbs": 7000.0, "sm_max_mhz": 2000.0}, "measured"))
    w = WORKLOADS["pks_sphere_N128_K8"]
    prof = {"pass_i": rec(4.0, 10), "pass_j": rec(1.0, 10)}
    r = bench.roofline(w, 0, prof, None)
    assert r["kernel"] == "pass_i" and r["bound"] == "alu" and r["traffic"] is None
    points = ((w.ncol + 2) + 2) / 2 * w.N ** 3
    flops = points * 2 * (2.0 * (w.N // 2) + 1.0)  # two folded transforms in the i pass
    assert r["achieved"] == pytest.approx(flops / 0.4e-3 / 1e12)
    assert r["peak"] == pytest.approx(152 * 128 * 2 * 2000.0 * 1e6 / 1e12)


def test_no_ap_pass_no_roofline():
    assert bench.roofline(WORKLOADS["pks_sphere_N128_K8"], 2, {"lsq_cholesky": rec(1.0, 1)}, None) is None
