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
