"""Host helpers of the bench: the waveguide layout per wall, the FP32 ALU peak it reports the
sparse sweeps against, and the option set of the measured variants."""
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


def test_fp32_peak_from_unit_counts(bench):
    # 152 SMs x 128 FP32 lanes x 2 flop (FMA) x 2.07 GHz
    assert bench.FP32_PEAK_TFLOPS == pytest.approx(80.54784, rel=1e-12)


def test_variant_options_parse(bench):
    a = bench._args(["--prec", "sparse_bf16", "--parts", "4x4x1", "--overlap", "2", "--antennas", "waveguides"])
    assert a.prec == "sparse_bf16" and a.overlap == 2 and a.antennas == "waveguides"
    assert bench._dims(a.parts) == (4, 4, 1)
    d = bench._args([])
    assert d.prec == "bf16" and d.antennas == "dipoles" and d.gpus == 1 and d.steps >= 1 and d.warmup >= 3
