"""Host helpers of the bench: the waveguide layout per wall, the per-class roofline ratings, and
the option set of the measured variants."""
import sys

import pytest


@pytest.fixture(scope="module")
def bench():
    sys.argv = ["bench.py"]
    import bench as b
    return b


def test_waveguide_counts(bench):
    assert bench.waveguide_counts(32) == (0, 11, 11, 10)
    for n in range(3, 100):
        c = bench.waveguide_counts(n)
        assert c[0] == 0 and sum(c) == n and max(c[1:]) - min(c[1:]) <= 1


def test_rate_classes(bench):
    prof = {"spmm": {"ms": 2.0, "launches": 4, "bytes": 8e9, "flops": 1e9},
            "gradient": {"ms": 10.0, "launches": 1, "bytes": 1e9, "flops": 8e9},
            "nn_conv": {"ms": 1.0, "launches": 3, "bytes": 1e6, "flops": 2e10},
            "factor": {"ms": 0.0, "launches": 0, "bytes": 0.0, "flops": 0.0}}
    r = bench.rate_classes(prof, 6000.0, {"fp32_tflops": 60.0, "fp64_tflops": 1.0})
    assert set(r) == {"spmm", "gradient", "nn_conv"}                 # classes that never ran are left out
    assert r["spmm"]["bound"] == "hbm" and r["spmm"]["achieved"] == pytest.approx(4000.0)
    assert r["spmm"]["frac"] == pytest.approx(4000.0 / 6000.0)
    assert r["gradient"]["bound"] == "fp64" and r["gradient"]["achieved"] == pytest.approx(0.8)
    assert r["gradient"]["frac"] == pytest.approx(0.8)
    assert r["nn_conv"]["bound"] == "fp32" and r["nn_conv"]["frac"] == pytest.approx(20.0 / 60.0)


def test_variant_options_parse(bench):
    a = bench._args(["--prec", "sparse_bf16", "--parts", "4x4x1", "--overlap", "2", "--antennas", "waveguides"])
    assert a.prec == "sparse_bf16" and a.overlap == 2 and a.antennas == "waveguides"
    assert bench._dims(a.parts) == (4, 4, 1)
    d = bench._args([])
    assert d.prec == "bf16" and d.antennas == "dipoles" and d.gpus == 1 and d.steps >= 1 and d.warmup >= 3


def test_oras_traffic_ratio_follows_its_partition(bench):
    """The roofline's DRAM traffic comes from the committed ncu summary only for the partition
    and kernel sources it was taken on; the default line's partition is that partition."""
    d = bench._args([])
    r = bench.oras_traffic_ratio(d.parts)
    assert r is not None and 1.0 <= r < 1.2
    assert bench.oras_traffic_ratio("16x16x7" if d.parts != "16x16x7" else "22x22x10") is None
    assert d.plain_factor == "fp64" and d.z_storage == "bf16" and d.inner_tol == 1e-2
