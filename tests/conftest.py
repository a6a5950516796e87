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


def planted_oracle(tmp_path, filename, old, new):
    """A copy of the oracle package with one planted change in one of its source files (a
    mutation that a pin must detect); returns the directory to put first on sys.path."""
    import shutil
    dst = os.path.join(str(tmp_path), "planted", "oracle")
    shutil.copytree(os.path.join(ROOT, "oracle"), dst, ignore=shutil.ignore_patterns("_build", "__pycache__"))
    path = os.path.join(dst, filename)
    with open(path) as fh:
        src = fh.read()
    assert src.count(old) == 1, "planted change does not apply"
    with open(path, "w") as fh:
        fh.write(src.replace(old, new))
    return os.path.dirname(dst)


def run_with_oracle(root, code, timeout=900):
    """Run a Python snippet in a fresh process whose `oracle` package is the one under root
    (tests and workloads importable); returns its last stdout line."""
    import subprocess
    pre = ("import sys; sys.path[:0] = [%r, %r, %r]\n"
           "import oracle; assert oracle.__file__.startswith(%r)\n"
           % (root, ROOT, os.path.join(ROOT, "tests"), root))
    out = subprocess.run([sys.executable, "-c", pre + code], capture_output=True, text=True, timeout=timeout)
    assert out.returncode == 0, out.stderr[-4000:]
    return out.stdout.strip().splitlines()[-1]
