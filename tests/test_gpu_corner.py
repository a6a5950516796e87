"""The corner-penalty study (Sec. 4.2, eq. (penalty_interp)) on the GPU path.

- The linearised coupled operator assembled from the library's forward-mode derivative
  (``stability.coupled_jacobian``: one sbp_rhs_eval_jvp per unknown and mesh) equals the oracle's
  exact derivative element by element, on a coarse copy of the box-in-box case (16^2 + 21^2 on the
  same boxes) for both interface penalties and a corner weight of 1/2, and on sampled columns
  (the inner box's corners and random unknowns) of the paper's 31^2 + 41^2 case.
- The library's mirror map (y -> -y) is the reflection of the two meshes' index grids, and the
  spectrum through the mirror blocks equals the oracle operator's dense spectrum.
"""
import numpy as np
import pytest

import workloads as W
from conftest import build_library
from oracle import OracleSystem
from oracle.adjoint import coupled_rhs_jvp

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sbp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build_library()
    import paper_1805_06607_gb300 as mod
    return mod


def _oracle_column(o, q, host_index, c):
    """Column c of the oracle's Jacobian over the unknowns ``host_index`` ((mesh, var, i, j))."""
    k, v, i, j = host_index[c]
    ni = o.meshes[k]["n"][0]
    d = [np.zeros_like(q[0]), np.zeros_like(q[1])]
    d[k][v, j, i] = 1.0
    out = []
    for kk in range(2):
        r = coupled_rhs_jvp(o, kk, q[kk], q[1 - kk], d[kk], d[1 - kk])[1]
        out.append(r)
    return np.array([out[kk][vv, jj, ii] for (kk, vv, ii, jj) in host_index])


def _jac(sbp, wl, sig):
    from paper_1805_06607_gb300.stability import coupled_jacobian
    g = sbp.System(wl, sigma_interface=sig)
    g.bind(wl["q0"])
    Jm, host = coupled_jacobian(g)
    torch.cuda.synchronize()
    g.check()
    return g, Jm.cpu().numpy(), host


@pytest.mark.parametrize("sig", [0.5, 1.0])
def test_coupled_jacobian_matches_oracle(sbp, sig):
    wl = W.corner_box_in_box(0.5, n_bg=16, n_fine=21)
    g, J, host = _jac(sbp, wl, sig)
    g.close()
    o = OracleSystem(wl, sig_int=sig)
    act = [o.iblank[k] != 0 for k in range(2)]
    idx = [(k, v, int(p % wl["meshes"][k]["n"][0]), int(p // wl["meshes"][k]["n"][0]))
           for k in range(2) for v in range(4) for p in np.flatnonzero(act[k].ravel())]
    assert host == idx
    want = np.stack([_oracle_column(o, wl["q0"], idx, c) for c in range(len(idx))], axis=1)
    assert np.abs(J - want).max() <= 1e-12 * np.abs(want).max()


def test_coupled_jacobian_full_case_sampled_columns(sbp):
    wl = W.corner_box_in_box(0.5)
    g, J, host = _jac(sbp, wl, 0.5)
    g.close()
    o = OracleSystem(wl)
    n_f = wl["meshes"][1]["n"]
    corner_cols = [c for c, (k, v, i, j) in enumerate(host)
                   if k == 1 and i in (0, n_f[0] - 1) and j in (0, n_f[1] - 1)]
    rng = np.random.default_rng(5)
    cols = sorted(set(corner_cols) | set(rng.choice(len(host), 48, replace=False).tolist()))
    scale = np.abs(J).max()
    for c in cols:
        want = _oracle_column(o, wl["q0"], host, c)
        assert np.abs(J[:, c] - want).max() <= 1e-12 * scale, c


def test_mirror_map_and_spectrum(sbp):
    from paper_1805_06607_gb300.stability import mirror_permutation, operator_spectrum
    wl = W.corner_box_in_box(0.5, n_bg=16, n_fine=21)
    g, J, host = _jac(sbp, wl, 0.5)
    mirror = mirror_permutation(g, host, axis=1)
    g.close()
    assert mirror is not None
    perm, sign = mirror
    pos = {h: a for a, h in enumerate(host)}
    for a, (k, v, i, j) in enumerate(host):
        nj = wl["meshes"][k]["n"][1]
        jr = (nj - j) % nj if k == 0 else nj - 1 - j
        assert perm[a] == pos[(k, v, i, jr)]
        assert sign[a] == (-1.0 if v == 2 else 1.0)
    lam = operator_spectrum(J, mirror)
    o = OracleSystem(wl)
    want = np.linalg.eigvals(np.stack([_oracle_column(o, wl["q0"], host, c) for c in range(len(host))], axis=1))
    assert lam.size == want.size
    # the growing corner mode of the half weight with sigma^I = 1/2: real, isolated, well conditioned
    a, b = lam[np.argmax(lam.real)], want[np.argmax(want.real)]
    assert abs(a.imag) < 1e-9 and abs(b.imag) < 1e-9 and a.real > 0.5
    assert abs(a - b) <= 1e-9 * abs(b)
    assert abs(np.abs(lam).max() - np.abs(want).max()) <= 1e-9 * np.abs(want).max()
