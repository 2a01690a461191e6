"""The measurement behind keeping the butterfly apply on mma.sync: a small
tcgen05 program (tests/gpu_probes/tcgen05_probe.cu, not part of the
library) checks that one tcgen05.mma kind::f16 on K-major, unswizzled bf16
operands reproduces an integer product exactly (M = 128 and M = 64, whose
row m sits in TMEM lane (m % 16) + 32 (m / 16)), and measures how many
cycles one thread takes per MMA issued back to back into one accumulator
for the small N this path has (16-64)."""
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def test_tcgen05_exact_product_and_issue_rate(tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = str(tmp_path / "tcgen05_probe")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17",
                    os.path.join(HERE, "gpu_probes", "tcgen05_probe.cu"), "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    lines = [ln.split() for ln in r.stdout.splitlines()]
    exact = [ln for ln in lines if ln[0] == "exact"]
    rate = {(int(ln[1]), int(ln[2])): float(ln[3]) for ln in lines if ln[0] == "rate"}
    assert len(exact) == 2 and all(int(ln[3]) == 0 for ln in exact)
    print("tcgen05 cycles per MMA from one thread:", rate)
    assert len(rate) == 4 and all(c > 0 for c in rate.values())
