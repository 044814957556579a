"""The integer-only float <-> double conversions of the mixed forms (df.cuh:
f2d_exact, d2f_rn) against the GPU's conversion instructions: every float,
every double exponent at its rounding boundaries and 2^32 sampled doubles
(tests/conversion_check.cu, built here with nvcc for sm_103a)."""
import json
import os
import shutil
import subprocess
import tempfile

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2605_14103_gb300", "csrc")


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else shutil.which("nvcc")


def test_conversions_match_the_conversion_instructions():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not found")
    with tempfile.TemporaryDirectory() as tmp:
        exe = os.path.join(tmp, "conversion_check")
        subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                        "-I" + CSRC, "-o", exe, os.path.join(HERE, "conversion_check.cu")],
                       check=True, capture_output=True, text=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True, timeout=300)
    r = json.loads(out.stdout.strip().splitlines()[-1])
    assert r["status"] == "no error"
    assert r["widen_mismatches"] == 0
    assert r["narrow_mismatches"] == 0
