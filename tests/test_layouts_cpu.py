"""The shared-memory layouts of the decoders, checked at compile time in both
builds (tests/layout_check.cu holds the static assertions); no GPU needed."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1505_04979_gb300", "csrc")


@pytest.mark.parametrize("checked", [False, True])
def test_layouts_compile(tmp_path, checked):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    cmd = [nvcc, "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-I", os.path.join(ROOT, "include"),
           "-I", CSRC, "-c", os.path.join(ROOT, "tests", "layout_check.cu"), "-o", str(tmp_path / "layout.o")]
    if checked:
        cmd.insert(1, "-DPOLARBP_CHECKED")
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
