"""Pins for the oracle's cluster evaluation of the strong form (Section 6): with no admissible
pair it is Lemma 4.1's direct evaluation (pinned in test_oracle_adaptive), and its error against
that falls geometrically with the Chebyshev order."""
import numpy as np
import pytest

from oracle import OracleMesh
from oracle.adaptive import strong_form
from oracle.cluster import strong_form_cluster
from paper_1708_03912_gb300 import synth


def _u(mesh, s):
    vod, _ = mesh.dofs(s)
    X = mesh.V[vod]
    return np.cos(1.3 * X[:, 0]) * (1.0 - 0.4 * X[:, 1] ** 2) + 0.2 * X[:, 0] * X[:, 1]


@pytest.mark.parametrize("case", ["disc", "lshape"])
def test_no_admissible_pair_is_the_direct_form(case):
    # (the L-shape's 96-cell mesh has corner cells without a DOF vertex)
    V, T = synth.disc(4, 2.0) if case == "disc" else synth.lshape(0.25, 0)
    m = OracleMesh(V, T)
    s = 0.5
    u = _u(m, s)
    S, size = strong_form(m, s, u, with_abs=True)
    Sc = strong_form_cluster(m, s, u, m=3, eta=0.0, leaf=4)
    assert np.max(np.abs(Sc - S) / size) < 1e-13


@pytest.mark.parametrize("s", [0.25])
def test_error_falls_with_the_order(s):
    V, T = synth.disc(5, 2.0)
    mesh = OracleMesh(V, T)
    u = _u(mesh, s)
    S = strong_form(mesh, s, u)
    errs = []
    for m in (2, 3, 4):
        Sc = strong_form_cluster(mesh, s, u, m=m, eta=1.0, leaf=8)
        errs.append(float(np.max(np.abs(Sc - S)) / np.max(np.abs(S))))
    print(s, errs)
    assert all(b < a for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 1e-4 and errs[-1] < errs[0] / 20, errs
