"""CPU checks of bench.py's host-side arithmetic: the counted operations and
the issue roofline of the sampling kernel, and the profile-hash gate of
`roofline.traffic`.  No GPU.
"""
import os
import shutil

import pytest

import bench


def test_counted_operations_of_the_headline_integrals():
    """The counts the roofline is built on, at d = 8 with FP32 sampling and FP64
    sums: 180.25 (Gaussian) and 184.25 (oscillatory) operations, of which 48 are
    32x32->64 multiplies (2 Philox calls x 20, plus one per dimension).  The
    Gaussian's (x - 1/2)^2 is one FMA per dimension (its centre is in the
    sampling table), the oscillatory sum one FMA."""
    g = bench.ops_per_sample("gauss_sym", 8, "fp32_acc64")
    o = bench.ops_per_sample("genz_osc", 8, "fp32_acc64")
    assert g["total"] == 180.25 and o["total"] == 184.25
    assert g["mulwide"] == o["mulwide"] == 48
    assert g["fp64"] == 0.25
    # one more Philox call per 4 dimensions, 9 + per-dimension integrand ops per dimension
    g9 = bench.ops_per_sample("gauss_sym", 9, "fp32_acc64")
    assert g9["mulwide"] == 60 + 9
    assert g9["total"] - g["total"] == 40 + (9 + 1)


def test_issue_roofline_at_152_sms_and_2070_mhz():
    """(180.25 - 48) + 4 x 48 = 324.25 issue cycles per sample: 152 x 2.07e9 x 128 / 324.25
    = 124.20 G samples/s; the FP64 and MUFU bounds are far above it."""
    b = bench.roofline_samples_per_s(bench.ops_per_sample("gauss_sym", 8, "fp32_acc64"), 152, 2.07e9)
    assert b["issue"] == pytest.approx(152 * 2.07e9 * 128 / 324.25, rel=1e-12)
    assert b["issue"] == pytest.approx(124.20e9, rel=1e-4)
    assert min(b, key=b.get) == "issue"
    assert b["fp64"] > 10 * b["issue"] and b["mufu"] > 10 * b["issue"]


def test_fp64_path_is_bound_by_its_fp64_pipe():
    """The FP64 path at d = 8, symmetric Gaussian: per dimension the map FMA,
    the Jacobian multiply, the histogram add and the integrand's FMA (4), per
    sample v, v^2 and the two sums (4) and the exponential (one multiply and
    the library's table-driven 2^x at 9.9 DFMA-equivalents, measured): 46.9
    FP64 operations; at the nominal 1.25 TFLOP/s (0.625e12 FMA/s)
    0.625e12 / 46.9 = 13.33 G samples/s, the tightest bound."""
    o = bench.ops_per_sample("gauss_sym", 8, "fp64")
    assert o["fp64"] == pytest.approx(4 * 8 + 4 + 1 + bench.FP64_CALL_DFMA["exp2"]) and o["fp64"] == pytest.approx(46.9)
    b = bench.roofline_samples_per_s(o, 152, 2.07e9)
    assert min(b, key=b.get) == "fp64"
    assert b["fp64"] == pytest.approx(152 * 2.07e9 * (1.25e12 / 2 / (152 * 2.07e9)) / 46.9, rel=1e-12)
    assert b["fp64"] == pytest.approx(13.33e9, rel=1e-3)


def _copy_tree(tmp_path):
    root = tmp_path / "repo"
    (root / "profiles").mkdir(parents=True)
    src = root / "paper_2010_09341_gb300" / "csrc"
    src.mkdir(parents=True)
    shutil.copy(os.path.join(bench.ROOT, "profiles", "sample_kernel_d8_gauss.md"), root / "profiles")
    for f in ("vegas_device.cuh", "vegas_sample.cuh"):
        shutil.copy(os.path.join(bench.ROOT, "paper_2010_09341_gb300", "csrc", f), src / f)
    return root, src


def test_traffic_is_reported_only_for_the_profiled_sources(tmp_path, monkeypatch):
    """roofline.traffic comes from the committed ncu summary only while the
    kernel sources hash to the profiled ones; any edit of them turns it to null."""
    root, src = _copy_tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    first = bench._traffic_from_profile()
    if first is None:
        pytest.skip("the committed sources differ from the profiled ones")
    assert first > 0
    with open(src / "vegas_sample.cuh", "a") as f:
        f.write("\n// edited\n")
    assert bench._traffic_from_profile() is None
    os.remove(root / "profiles" / "sample_kernel_d8_gauss.md")
    assert bench._traffic_from_profile() is None


def test_counted_operations_of_the_density_grid_and_stratified_lines():
    """The LO toy on the density grid: Philox (40) + 3 dimensions x 9 + the
    per-sample terms of the FP32 Kahan mode (2 + 2 + 5 + 8 + 3) + its finish
    (LO kinematics 20, three grid coordinates 27, three weight sets 39, two
    bicubic lookups 78, product 2); 23 wide multiplies.  The stratified hybrid
    with P = 2 at d = 8 adds 8 x 1.5 + 3 + 9 / 2 = 19.5 to the plain count."""
    o = bench.ops_per_sample("lo_pdf", 3, "fp32_kahan")
    assert bench.LO_PDF_FINISH == 166
    assert o["total"] == 40 + 27 + 20 + 166 and o["mulwide"] == 23 and o["mufu"] == 4
    s = bench.strat_ops_per_sample("gauss_sym", 8, "fp32_acc64", 2)
    assert s["total"] == pytest.approx(bench.ops_per_sample("gauss_sym", 8, "fp32_acc64")["total"] + 19.5)
    assert s["mulwide"] == 48
