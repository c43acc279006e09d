"""Host checks of the corrector's integer-pipe exact arithmetic (no GPU).

The corrector replaces the FP64 divisions by 6, 24 and 120 and the products with
3, 6 and 12 by integer code that must give the bits of the IEEE operation
(Granlund-Montgomery division by an invariant integer, round to nearest). The
same header compiled for the host is checked here against the host's IEEE
double arithmetic on random and edge significands over every exponent."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_integer_division_and_product_match_ieee():
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not found")
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "exact_int_check")
        subprocess.run([nvcc, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "include"),
                        "-I", os.path.join(ROOT, "paper_0711_0643_gb300", "csrc"),
                        "-o", exe, os.path.join(ROOT, "tests", "exact_int_check.cu")], check=True)
        out = subprocess.run([exe, "8000000"], capture_output=True, text=True)
        assert out.returncode == 0, out.stdout + out.stderr
        assert "mismatches 0" in out.stdout
