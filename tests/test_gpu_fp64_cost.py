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
    """The flip loops divide (and take reciprocals, d = 1) with a reciprocal
    seed and one third-order Newton-Raphson step; against CUDA's IEEE
    quotient it stays within 4 ulp
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
    d[2000:3000] = 1.0  # the paired flip loop's reciprocal 1 / r is this quotient at d = 1
    q, qi = flip_quotient(d, r)
    assert np.all(q[1000:2000] == 0.0)
    assert np.array_equal(q[:1000][r[:1000] == 1.0], d[:1000][r[:1000] == 1.0])
    ulp = np.abs(q - qi) / np.spacing(np.abs(qi))
    print("largest difference in ulp:", ulp.max())
    assert ulp.max() <= 4


def test_gram_probe_variants_agree():
    """The four Gram forms of lq_probe_gram give the FP64 Gram of the same
    panels: the FP64 CUDA-core and DMMA forms to FP64 round-off, the FP32-panel
    forms to the FP32 level (the inputs themselves are FP32 there)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_08552_gb300.lecqmc import probe_gram

    for m in (16, 64):
        us0, e0 = probe_gram(512, m, 0, 8)
        us1, e1 = probe_gram(512, m, 1, 8)
        us2, e2 = probe_gram(512, m, 2, 8)
        us3, e3 = probe_gram(512, m, 3, 8)
        print(m, (us0, e0), (us1, e1), (us2, e2), (us3, e3))
        assert e0 == 0.0 and e1 < 1e-13 and e2 == 0.0 and e3 < 1e-5
        assert min(us0, us1, us2, us3) > 0
