"""Host part of the symmetry reduction (Section 7): the sector handle's orbits and reduced
unknowns equal the oracle's, and its far-field tiles are the ones touching a representative's
support (about 2/K of the whole mesh's)."""
import numpy as np
import pytest

from oracle import symmetry as sym
from paper_1708_03912_gb300 import fraclap as fl
from paper_1708_03912_gb300 import synth


def _lib():
    try:
        return fl.lib()
    except OSError as e:
        pytest.skip(f"library not built: {e}")


@pytest.mark.parametrize("K,M", [(8, 6), (8, 12), (4, 8), (6, 10)])
def test_orbits_match_oracle(K, M):
    _lib()
    V, T = synth.sector(K, M)
    h = fl.fl_create_sector(V, T, K)
    n = fl.fl_num_dofs(h, 0.5)
    vod = fl.fl_dof_vertices(h, 0.5)
    mesh, P, reps = sym.orbits(V, T, K, 0.5)
    assert n == len(reps) and np.array_equal(vod, reps)
    st = fl.fl_get_stats(h, 0.5)
    assert st["n_cells"] == mesh.nc and st["n_vertices"] == mesh.nv and st["n_dofs"] == n
    # the whole mesh has nblk (nblk + 1) / 2 tiles; the reduced plan keeps fewer
    W, C, _, _ = sym.replicate(V, T, K)
    hw = fl.fl_create(W, C)
    tw = fl.fl_get_stats(hw, 0.5)["n_tiles"]
    print(K, M, "tiles", st["n_tiles"], "of", tw)
    assert st["n_tiles"] < tw
    fl.fl_destroy(hw)
    fl.fl_destroy(h)


def test_sector_errors():
    _lib()
    V, T = synth.sector(8, 4)
    with pytest.raises(fl.FlError):
        fl.fl_create_sector(V, T, 1)
    bad = np.array(T).copy()
    bad[0, 0] = len(V) + 3
    with pytest.raises(fl.FlError):
        fl.fl_create_sector(V, bad, 8)
    # a sector of the wrong angle does not close up into orbits
    with pytest.raises(fl.FlError):
        fl.fl_create_sector(V, T, 7)
    h = fl.fl_create_sector(V, T, 8)
    with pytest.raises(fl.FlError) as e:
        fl.fl_cluster_plan(h, 0.5)
    assert e.value.args[0] == 7 or "sector" in str(e.value)
    fl.fl_destroy(h)
