"""The autotuner's rules (csrc/sbp_tune.h) on the host, with given times: which shapes a mesh's
use times and which one it keeps. A fast mesh's fused step (the critical path of the macro step)
takes shapes that give every SM a CTA and, for Navier-Stokes, flux tiles of at least 8 rows, and
of those within 3 % of the fastest the one with the most CTAs; every other use keeps the fastest.
The cylinder's O-grid (512 x 128 points, 152 SMs) is the case the rules were measured on: its
16-row flux tiles (128 CTAs) time within 2 % of the 8-row ones alone and lose in the macro step."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1805_06607_gb300", "csrc")


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("no g++")
    exe = str(tmp_path_factory.mktemp("tune") / "tune_driver")
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-I", CSRC, os.path.join(ROOT, "tests", "host_tune", "tune_driver.cpp"),
                           "-o", exe])

    def run(ni, nj, viscous, critical, n_sm=152, times=None):
        args = [exe, str(ni), str(nj), str(int(viscous)), str(int(critical)), str(n_sm)]
        args += ["%d,%d,%d=%g" % (s, r, u, ms) for (s, r, u), ms in (times or {}).items()]
        out = subprocess.run(args, capture_output=True, text=True, check=True).stdout.split("\n")
        el = [tuple(int(v) for v in t.split(",")) for t in out[0].split()[1:]]
        pick = tuple(int(v) for v in out[1].split()[1].split(",")) if times else None
        return el, pick
    return run


def test_ogrid_navier_stokes_fast_step(driver):
    el, _ = driver(512, 128, True, True)
    assert el == [(0, 8, 0), (0, 8, 4)]
    # alone within 3 %: the 4-row derivative tiles (256 + 512 CTAs) over 8-row ones (256 + 256)
    _, pick = driver(512, 128, True, True, times={(0, 8, 0): 55.4, (0, 8, 4): 56.0})
    assert pick == (0, 8, 4)
    _, pick = driver(512, 128, True, True, times={(0, 8, 0): 55.4, (0, 8, 4): 57.5})
    assert pick == (0, 8, 0)


def test_ogrid_euler_fast_step_keeps_four_row_tiles(driver):
    el, _ = driver(512, 128, False, True)
    assert el == [(0, 4, 0), (0, 8, 0), (0, 8, 4)]
    _, pick = driver(512, 128, False, True, times={(0, 4, 0): 10.2, (0, 8, 0): 10.0, (0, 8, 4): 10.1})
    assert pick == (0, 4, 0)


def test_other_uses_keep_the_fastest(driver):
    el_bg, _ = driver(1024, 512, True, False)
    assert (0, 16, 4) in el_bg and (0, 32, 16) in el_bg and (58, 64, 0) in el_bg and (116, 64, 0) in el_bg
    _, pick = driver(1024, 512, True, False, times={(0, 16, 4): 10.0, (0, 8, 4): 10.1, (0, 4, 0): 10.05})
    assert pick == (0, 16, 4)
    # the fast mesh's right-hand side alone (not critical) has every usable shape
    el, _ = driver(512, 128, True, False)
    assert (0, 16, 8) in el and (0, 4, 0) in el and len(el) > 10


def test_small_fast_meshes(driver):
    # a 96 x 24 O-grid: the most CTAs any shape gives (9) sets the floor
    el, _ = driver(96, 24, True, True)
    assert el == [(0, 8, 0), (0, 8, 4)]
    # 6 rows: no 8-row tile fits, so the floor on flux rows is dropped; the 4-row pair and the
    # marching kernel's 8-row chunks give 3 and 2 CTAs, and the floor of CTAs keeps the pair
    el, _ = driver(96, 6, True, True)
    assert el == [(0, 4, 0)]


def test_equal_times_keep_the_first(driver):
    _, pick = driver(1024, 512, True, False, times={(0, 8, 0): 10.0, (0, 16, 4): 10.0})
    assert pick == (0, 8, 0)
