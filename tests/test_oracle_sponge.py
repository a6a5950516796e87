"""The oracle's sponge layer at far-field faces (Sec. 5.1: sponge boundaries six cells deep).

On a uniform state the SBP flux divergence vanishes exactly (free-stream preservation), so at
points that carry no SAT term the right-hand side is the sponge term alone: it must vanish
beyond the layer's depth, relax every variable toward the far-field state inside it (the sign),
and weaken monotonically away from the face. The strength profile inside the layer is a reading
(the form is cited, not printed)."""
import numpy as np

import workloads as W
from oracle import OracleSystem


def test_sponge_on_uniform_offset_state():
    D = 6
    wl = W.cylinder_small(seed=2, sponge_cells=D, sponge_strength=2.0)
    o = OracleSystem(wl)
    qinf = np.asarray(wl["params"]["qinf"], dtype=np.float64)
    delta = np.array([1e-3, -2e-3, 1.5e-3, 3e-3])
    k = 0  # the Cartesian background, far field on all four faces
    ni, nj = wl["meshes"][k]["n"]
    q = np.broadcast_to((qinf + delta)[:, None, None], (4, nj, ni)).copy()
    qo = np.broadcast_to((qinf + delta)[:, None, None],
                         (4, wl["meshes"][1]["n"][1], wl["meshes"][1]["n"][0])).copy()
    r = o.coupled_rhs(k, q, qo)
    sat = np.zeros((nj, ni), bool)
    pts = o.terms[k]["pt"]
    sat.flat[pts] = True
    act = (o.iblank[k] != 0) & ~sat
    jm = nj // 2
    prof = []
    for d in range(1, D + 3):  # d = 0 is the face itself, which carries the far-field SAT
        i = d
        assert act[jm, i]
        ratio = -r[:, jm, i] / delta
        # the same relaxation rate for every variable
        assert np.allclose(ratio, ratio[0], rtol=1e-9, atol=1e-12)
        prof.append(ratio[0])
    prof = np.array(prof)  # d = 1 .. D + 2
    assert np.all(prof[:D - 1] > 0) and np.all(np.diff(prof[:D - 1]) < 0)
    assert np.all(np.abs(prof[D - 1:]) < 1e-12)
    # away from every far-field face the state is steady
    inner = act.copy()
    inner[:D, :] = inner[-D:, :] = False
    inner[:, :D] = inner[:, -D:] = False
    assert np.abs(r[:, inner]).max() < 1e-12
    # without a sponge the same points are steady
    o0 = OracleSystem(W.cylinder_small(seed=2))
    r0 = o0.coupled_rhs(k, q, qo)
    assert np.abs(r0[:, act]).max() < 1e-12
