"""The attribute packing and chi on packed words, compiled for the host from the library's
own sources and checked against the plain definition of chi (Eq. 4-5) over random layouts,
codes, capped query codes and wildcards (tests/native/chi_layout_check.cu)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2203_13601_gb300", "csrc")


def test_chi_on_packed_words_equals_the_definition(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc is not available")
    exe = str(tmp_path / "chi_layout_check")
    subprocess.check_call([nvcc, "-O2", "-std=c++17", "-gencode",
                           "arch=compute_103a,code=sm_103a",
                           "-I", os.path.join(ROOT, "include"), "-I", CSRC,
                           os.path.join(ROOT, "tests", "native", "chi_layout_check.cu"),
                           os.path.join(CSRC, "k_util.cu"), "-o", exe])
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.startswith("ok "), out.stdout
    assert int(out.stdout.split()[1]) > 50_000
