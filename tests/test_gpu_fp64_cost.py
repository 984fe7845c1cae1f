"""The GB300 fact behind the flip-loop design and the roof of the benchmark:
an FP64 FMA warp instruction occupies a sub-partition for tens of cycles
whatever the number of active lanes, while an FP32 FMA issues about once per
cycle, and the device's aggregate FP64 FMA rate (lq_device_fp64_rate) is
about 1.2 TFLOP/s.  So FP64 work is counted in warp instructions, and the
serial per-site chain is latency bound."""
import pytest

pytestmark = pytest.mark.gpu


def test_fp64_instruction_cost_and_rate():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2601_08552_gb300 as lq

    tflops, v = lq.device_fp64_rate(100.0)
    print(tflops, v)
    assert v["dfma_32lanes"] > 16 * v["ffma_32lanes"]
    assert abs(v["dfma_1lane"] - v["dfma_32lanes"]) < 0.25 * v["dfma_32lanes"]
    # 152 SMs x 4 sub-partitions x 0.5 FMA/cycle x 2 flops at 1.0-2.1 GHz
    assert 0.5 < tflops < 1.4


def test_flip_quotient_against_ieee():
    """The flip loop divides with a reciprocal seed and one third-order
    Newton-Raphson step; against CUDA's IEEE quotient it stays within 4 ulp
    over operands spanning the ratio factors 1 + Delta G_tt the loop meets
    (and far beyond), and is exact for d = 0 and r = 1."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import numpy as np
    from paper_2601_08552_gb300.lecqmc import flip_quotient

    rng = np.random.default_rng(2026)
    n = 1 << 18
    d = rng.uniform(-4, 4, n) * np.exp(rng.uniform(-30, 30, n))
    r = rng.choice([-1, 1], n) * np.exp(rng.uniform(-40, 40, n))
    r[:1000] = 1.0 + rng.uniform(-1, 1, 1000) * 1e-12  # near 1
    d[1000:2000] = 0.0
    q, qi = flip_quotient(d, r)
    assert np.all(q[1000:2000] == 0.0)
    assert np.array_equal(q[:1000][r[:1000] == 1.0], d[:1000][r[:1000] == 1.0])
    ulp = np.abs(q - qi) / np.spacing(np.abs(qi))
    print("largest difference in ulp:", ulp.max())
    assert ulp.max() <= 4
