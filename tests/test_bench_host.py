"""Host-side arithmetic of bench.py's roofline objects, checked without a GPU:
the algorithmic bytes and FLOPs of one SIP apply (2 n_b + 1 words and
16 n^3 + 128 n^2 FLOP per element, n = k + 1) for the bench's workloads, the
intensities quoted against the ridge points, the kernel labels of the
schedule codes, and the DRAM traffic read from the committed ncu summaries
of those kernels."""
import pytest

import bench


def test_algorithmic_apply_counts():
    # FP64 apply of the 128^2, k = 3 headline workload: 520 B and 3072 FLOP per element
    ab, af = bench.algorithmic_apply(3, 128 * 128, 8)
    assert (ab, af) == (16384 * 520, 16384 * 3072) == (8519680, 50331648)
    # FP32 apply at 512^2: k = 3 (260 B, 3072 FLOP) and k = 4 (404 B, 5200 FLOP)
    assert bench.algorithmic_apply(3, 512 * 512, 4) == (262144 * 260, 262144 * 3072)
    ab4, af4 = bench.algorithmic_apply(4, 512 * 512, 4)
    assert (ab4, af4) == (105906176, 1363148800)
    # the intensities the roofline discussion quotes (FLOP/B)
    assert round(af / ab, 1) == 5.9
    assert round(3072 / 260, 1) == 11.8 and round(af4 / ab4, 1) == 12.9


def test_roofline_fraction_and_rate():
    ab, af = bench.algorithmic_apply(3, 128 * 128, 8)
    r = bench.roofline(ab, af, 0.05, "k", None, {"fp64": 1.0})
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(af / 0.05e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / 1.0)
    assert r["hbm_GB_per_s"] == pytest.approx(ab / 0.05e-3 / 1e9)
    # whole-job solves per second: every rank solves `steps` instances
    assert bench.whole_job_rate(10, 2, 2000.0) == pytest.approx(10.0)


def test_kernel_labels_and_captured_traffic():
    assert bench.kernel_name(5, 3, 8) == "k_apply_stage<4,double,double,4,1,0>"
    assert bench.kernel_name(6, 4, 4) == "k_apply_warp<5,1>"
    assert bench.kernel_name(6, 3, 4) == "k_apply_warp<4,1>"
    # DRAM bytes per launch from the committed summaries (read + write)
    assert bench.captured_traffic("k_apply_stage<4,double,double,4,1,0>") == pytest.approx(4464128)
    assert bench.captured_traffic("k_apply_warp<5,1>") == pytest.approx(53549312 + 9768960)
    assert bench.captured_traffic("k_apply_warp<4,1>") == pytest.approx(34649344 + 308480)
    # a kernel without a current summary reports no traffic
    assert bench.captured_traffic("k_apply_elem2<4,double,1>") is None
