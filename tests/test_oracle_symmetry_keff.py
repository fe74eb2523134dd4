"""Pins for the oracle's effective-kernel form of the symmetry reduction (Section 7): each orbit of
element pairs under the rotation evaluated once gives P^T A P / K of the whole mesh, up to the part of
the quadrature that is not rotation invariant (the boundary facets' singular rules depend on vertex
labels, which the copies number differently; that part converges with k_bnd)."""
import numpy as np
import pytest

from oracle.assemble import QuadOrders
from oracle.symmetry import fold_system, reduced_system_keff
from paper_1708_03912_gb300 import synth


@pytest.mark.parametrize("K", [5, 6, 8])
def test_keff_is_the_folded_whole_matrix(K):
    # for even K every sector cell's opposite image (k, copy K/2 of k) forms an orbit of K/2 pairs
    # (weight 1/2): a wrong weight there would break the agreement
    V, T = synth.sector(K, 4)
    for orders, tol in ((QuadOrders(), 1e-7), (QuadOrders(k_bnd=16), 1e-11)):
        Ak, bk, rk = reduced_system_keff(V, T, K, 0.5, orders=orders)
        Af, bf, rf = fold_system(V, T, K, 0.5, orders=orders)
        assert np.array_equal(rk, rf)
        d = np.sqrt(np.outer(np.diag(Af), np.diag(Af)))
        err = float(np.max(np.abs(Ak - Af) / d))
        assert err < tol, (K, orders, err)
        assert float(np.max(np.abs(Ak - Ak.T) / d)) < 1e-14  # symmetric up to the order of the sums
        assert np.allclose(bk, bf, rtol=0, atol=1e-15)
