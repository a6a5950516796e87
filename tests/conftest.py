import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "timeout(seconds): per-test time limit (pytest-timeout)")


def golden(name):
    """Rows of a whitespace-separated fixture under tests/golden (comments start with #)."""
    rows = []
    with open(os.path.join(ROOT, "tests", "golden", name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append(line.split())
    return rows


def build_library():
    """Build the CUDA library in-tree (by path: importing the package needs the built file)."""
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "sbp_build", os.path.join(ROOT, "paper_1805_06607_gb300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.build()
