"""The C ABI from a plain C program (tests/c_client/sbp_c_client.c, built with gcc against
include/sbp_mrab.h and the library): five MRAB macro steps of a two-mesh Euler system, bit for
bit the same states and donor tables as the same run through the Python binding (which hands
the library coordinate arrays where the C client gives only lo and h)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import workloads as W
from conftest import ROOT, build_library

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _workload():
    gam, u0 = 1.4, 0.5
    bg = W.cartesian_mesh("background", (48, 48), (-5.0, -5.0), (10.0 / 48, 10.0 / 48), ("periodic",) * 4,
                          periodic=(True, True))
    fine = W.cartesian_mesh("fine", (33, 33), (-1.0, -1.0), (2.0 / 32, 2.0 / 32), ("interface",) * 4)
    qs = []
    for mm in (bg, fine):
        x, y = mm["x"], mm["y"]
        rho = 1.0 + 0.01 * (x * x - y * y) / 25.0
        qs.append(np.stack([rho, rho * u0, 0.0 * rho, (1.0 / gam) / (gam - 1.0) + 0.5 * rho * u0 * u0]))
    params = dict(physics="euler", gamma=gam, mu=0.0, pr=0.72, order=3, hist_len=3, step_ratio=2, fast_mesh=1,
                  cfl=0.5, qinf=np.array([1.0, u0, 0.0, 1.0 / (gam * (gam - 1.0)) + 0.5 * u0 * u0]), twall=1.0,
                  omega_corner=1.0)
    return {"meshes": [bg, fine], "q0": qs, "params": params}


def test_c_client_matches_python_binding(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    lib = build_library()
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    exe = str(tmp_path / "client")
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", os.path.join(ROOT, "tests", "c_client", "sbp_c_client.c"),
                           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(cuda, "include"),
                           lib, "-L", os.path.join(cuda, "lib64"), "-lcudart",
                           "-Wl,-rpath," + os.path.dirname(lib), "-Wl,-rpath," + os.path.join(cuda, "lib64"),
                           "-o", exe])
    out = str(tmp_path / "states.bin")
    res = subprocess.run([exe, out], capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stderr
    import paper_1805_06607_gb300 as sbp
    wl = _workload()
    g = sbp.System(wl)
    g.bind(wl["q0"])
    g.mrab_init()
    g.mrab_step(5)
    g.check()
    blob = open(out, "rb").read()
    nstate = sum(2 * g.info[k].state_bytes for k in range(2))
    raw = np.frombuffer(blob[:nstate], dtype=np.float64)
    o = 0
    planes = []
    for k in range(2):
        inf = g.info[k]
        n = 4 * inf.nj * inf.pitch
        planes.append(raw[o:o + n].reshape(4, inf.nj, inf.pitch)[:, :, :inf.ni])
        o += n
    for k in range(2):
        inf = g.info[k]
        n = 4 * inf.nj * inf.pitch
        c = raw[o:o + n].reshape(4, inf.nj, inf.pitch)[:, :, :inf.ni]
        o += n
        assert np.array_equal(planes[k], wl["q0"][k]), ("initial state", k, np.abs(planes[k] - wl["q0"][k]).max())
        py = g.to_host(k, g.current_state(k))
        assert np.array_equal(c, py), (k, np.abs(c - py).max(), np.argwhere(c != py)[:5].tolist())
    assert o == raw.size
    # the donor tables the C client read back through sbp_get_tables
    off = nstate
    for k in range(2):
        nr = g.info[k].n_receivers
        base = np.frombuffer(blob, dtype=np.int32, count=2 * nr, offset=off)
        off += 8 * nr
        w = np.frombuffer(blob, dtype=np.float64, count=8 * nr, offset=off)
        off += 64 * nr
        t = g.tables(k)
        assert np.array_equal(base.reshape(nr, 2), t["base"]) and np.array_equal(w.reshape(nr, 8), t["w"])
    assert off == len(blob)
    H, t = g.mrab_time()
    assert res.stdout.split()[1] == repr(H) or float(res.stdout.split()[1]) == H
    g.close()
