"""The GB300 fact behind the flip-loop design: an FP64 FMA warp instruction
occupies a sub-partition for tens of cycles whatever the number of active
lanes, while an FP32 FMA issues about once per cycle.  So FP64 work is
counted in warp instructions, and the serial per-site chain is latency bound."""
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def test_fp64_instruction_cost(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = str(tmp_path / "probe")
    subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe,
                           os.path.join(HERE, "fp64_cost_probe.cu")])
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    v = {l.split()[0]: float(l.split()[1]) for l in out.strip().splitlines()}
    print(v)
    assert v["dfma_32lanes"] > 16 * v["ffma_32lanes"]
    assert abs(v["dfma_1lane"] - v["dfma_32lanes"]) < 0.25 * v["dfma_32lanes"]
