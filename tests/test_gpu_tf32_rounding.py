"""The head/tail split of the FP32-accurate three-pass TF32 products rounds by
integer operations (half a TF32 ulp added, the 13 low bits cleared).  This
checks, on the GPU, that the library's rounding gives the bits of
cvt.rna.tf32.f32 (round to nearest, ties away from zero) for every finite
float32 pattern below the overflow threshold."""
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_tf32_split_rounding_equals_cvt_rna(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = str(tmp_path / "tf32_round_check")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                    f"-I{os.path.join(ROOT, 'include')}",
                    f"-I{os.path.join(ROOT, 'paper_2404_10087_gb300', 'csrc')}",
                    os.path.join(HERE, "tf32_round_check.cu"), "-o", exe], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stdout + out.stderr
    words = out.stdout.split()
    assert int(words[1]) > 4_000_000_000 and int(words[3]) == 0, out.stdout
