"""The SBP_BOUNDS_CHECK build (the gathers check the table indices they follow): the translation
units that hold those checks compile with the flag for sm_103a (nvcc cross-compiles without a
GPU), and the build script puts that build in its own directory."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1805_06607_gb300", "csrc")


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="no nvcc")
@pytest.mark.parametrize("src", ["sbp3c_kernels.cu", "sbp3_kernels.cu"])
def test_checked_units_compile(tmp_path, src):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    cmd = [nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-I", os.path.join(ROOT, "include"),
           "-I", CSRC, "-DSBP_BOUNDS_CHECK", "-c", os.path.join(CSRC, src), "-o", str(tmp_path / (src + ".o"))]
    out = subprocess.run(cmd, capture_output=True, text=True)
    assert out.returncode == 0, out.stderr[-3000:]


def test_checked_build_has_its_own_directory():
    import importlib.util
    spec = importlib.util.spec_from_file_location("sbp_build", os.path.join(ROOT, "paper_1805_06607_gb300", "build.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    plain, checked = b._paths(False), b._paths(True)
    assert plain[1] == b.LIB and checked[0] != plain[0] and checked[1].endswith("libsbpmrab.so")
